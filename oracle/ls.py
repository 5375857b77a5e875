"""Lippmann-Schwinger scattering with the volume potential (Section 5.3),
oracle side, float64.  TEST INFRASTRUCTURE ONLY.

The scattered field u of Delta u + k^2 (1 + q) u = -k^2 q u_inc satisfies
u = k^2 V[q (u + u_inc)] with V the volume potential of the Green's function of
-(Delta + k^2), i.e. the second-kind equation

    A u := u - k^2 V[q u] = k^2 V[q u_inc] =: b.

The paper's dual (density) form of Section 5.3 puts the unknown in the
source: with s = k^2 q (u + u_inc) the scattered field is u = V[s] and

    B s := s - k^2 q V[s] = k^2 q u_inc,

(``op_density``, ``rhs_density``).  V is ``oracle.apply.apply_fft2n`` with the
Helmholtz multiplier.  ``dense_solve`` builds A (or B) column by column and
solves it directly (small N only); ``gmres`` is textbook restarted GMRES and
``bicgstab`` textbook Bi-CGStab, the paper's iteration.
"""
from __future__ import annotations

import numpy as np

from . import apply as A
from . import kernel as K


class LSProblem:
    """The field-form operator on an N^d grid (d = q.ndim); L defaults to the
    paper's 1.8 (3D) or 1.5 (2D)."""

    def __init__(self, N: int, k: float, q: np.ndarray, L: float | None = None):
        self.N, self.k, self.q = N, k, np.asarray(q, dtype=np.float64)
        self.d = self.q.ndim
        L = (1.8 if self.d == 3 else 1.5) if L is None else L
        T = K.T_octant_by_sums(self.d, N, "helmholtz", k, L)
        self.G = K.ghat_full_from_octant(K.ghat_octant_by_sums(T, N))

    def V(self, f):
        return A.apply_fft2n(self.G, f)

    def op(self, u):
        return u - self.k ** 2 * self.V(self.q * u)

    def rhs(self, u_inc):
        return self.k ** 2 * self.V(self.q * u_inc)

    def op_density(self, s):
        return s - self.k ** 2 * self.q * self.V(s)

    def rhs_density(self, u_inc):
        return self.k ** 2 * self.q * u_inc

    def residual(self, u, b) -> float:
        return float(np.linalg.norm((b - self.op(u)).ravel()) / np.linalg.norm(b.ravel()))


def dense_solve(prob: LSProblem, b: np.ndarray, form: str = "field") -> np.ndarray:
    """Builds the N^d x N^d matrix of A (form "field") or B ("density") from
    unit vectors and solves it against b."""
    op = prob.op if form == "field" else prob.op_density
    n = prob.N ** prob.d
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        M[:, j] = op(e.reshape((prob.N,) * prob.d)).ravel()
        e[j] = 0.0
    return np.linalg.solve(M, b.ravel()).reshape(b.shape)


def gmres(matvec, b: np.ndarray, tol: float = 1e-10, restart: int = 40, maxit: int = 2000):
    """Restarted GMRES (Saad & Schultz) with modified Gram-Schmidt and Givens
    rotations; returns (x, iterations, relative residual history)."""
    x = np.zeros_like(b)
    bn = np.linalg.norm(b.ravel())
    hist = []
    it = 0
    while it < maxit:
        r = b - matvec(x)
        beta = np.linalg.norm(r.ravel())
        hist.append(beta / bn)
        if beta / bn < tol:
            break
        V = [r / beta]
        H = np.zeros((restart + 1, restart), dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        cs, sn = [], []
        j_end = 0
        for j in range(restart):
            w = matvec(V[j])
            for i in range(j + 1):
                H[i, j] = np.vdot(V[i].ravel(), w.ravel())
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w.ravel())
            V.append(w / H[j + 1, j] if H[j + 1, j] != 0 else w)
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(abs(H[j, j]), abs(H[j + 1, j]))
            c = abs(H[j, j]) / den if den else 1.0
            s = (H[j, j] / abs(H[j, j])) * np.conj(H[j + 1, j]) / den if abs(H[j, j]) else 1.0
            cs.append(c)
            sn.append(s)
            H[j, j] = c * H[j, j] + s * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(s) * g[j]
            g[j] = c * g[j]
            it += 1
            j_end = j + 1
            hist.append(abs(g[j + 1]) / bn)
            if abs(g[j + 1]) / bn < tol or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_end, :j_end]), g[:j_end])
        for i in range(j_end):
            x = x + y[i] * V[i]
        if hist[-1] < tol:
            break
    return x, it, hist


def arnoldi(matvec, b: np.ndarray, m: int):
    """m steps of the Arnoldi process (Saad & Schultz 1986) from b, modified
    Gram-Schmidt applied twice (Kahan-Parlett "twice is enough"; one pass loses
    orthogonality once h_{j+1,j} becomes small): returns V (m+1 orthonormal
    vectors, v_0 = b/||b||) and the (m+1) x m upper Hessenberg H with
    A V[:m] = V H and h_{j+1,j} > 0."""
    V = [b / np.linalg.norm(b.ravel())]
    H = np.zeros((m + 1, m), dtype=np.complex128)
    for j in range(m):
        w = matvec(V[j])
        for _ in range(2):
            for i in range(j + 1):
                h = np.vdot(V[i].ravel(), w.ravel())
                H[i, j] += h
                w = w - h * V[i]
        H[j + 1, j] = np.linalg.norm(w.ravel())
        V.append(w / H[j + 1, j])
    return np.stack(V), H


def bicgstab(matvec, b: np.ndarray, tol: float = 1e-12, maxit: int = 5000):
    """Unpreconditioned Bi-CGStab (van der Vorst 1992; Saad, Iterative Methods
    for Sparse Linear Systems, Alg. 7.7) from x = 0 with the shadow residual
    r^ = b; two products with A per iteration.  Stops when the recurrence
    residual ||r|| / ||b|| < tol, tested after the half step (||s||) and after
    the full step.  Returns (x, iterations begun, matvecs, relative residual
    history)."""
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    bn = np.linalg.norm(b.ravel())
    rho_prev = alpha = omega = 1.0 + 0j
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    hist = [1.0]
    matvecs = 0
    for it in range(1, maxit + 1):
        rho = np.vdot(rh.ravel(), r.ravel())
        if rho == 0:
            break
        beta = (rho / rho_prev) * (alpha / omega)
        p = r + beta * (p - omega * v)
        v = matvec(p)
        matvecs += 1
        alpha = rho / np.vdot(rh.ravel(), v.ravel())
        s = r - alpha * v
        if np.linalg.norm(s.ravel()) / bn < tol:
            x = x + alpha * p
            hist.append(np.linalg.norm(s.ravel()) / bn)
            return x, it, matvecs, hist
        t = matvec(s)
        matvecs += 1
        omega = np.vdot(t.ravel(), s.ravel()) / np.vdot(t.ravel(), t.ravel())
        x = x + alpha * p + omega * s
        r = s - omega * t
        hist.append(np.linalg.norm(r.ravel()) / bn)
        if hist[-1] < tol or omega == 0:
            return x, it, matvecs, hist
        rho_prev = rho
    return x, it, matvecs, hist
