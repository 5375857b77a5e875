"""Variable-coefficient Poisson equation of Section 5.2 (linearised
Poisson-Boltzmann with lambda = 0), oracle side, float64.  TEST
INFRASTRUCTURE ONLY.

With phi = V[sigma] (V the Laplace volume potential, g = 1/(4 pi r) in 3D,
-log(r)/(2 pi) in 2D, so -Delta phi = sigma), div(eps grad phi) = rho becomes
the second-kind equation of Section 5.2 (eq. pbeq)

    M sigma := -eps sigma + grad(eps) . grad V[sigma] = rho.

The printed equation writes the kernel as 1/|x - y|; with the representation
phi = int sigma/(4 pi |x - y|) that precedes it, the factor 1/(4 pi) belongs
there.  grad V uses the exact derivative kernels T_j (Section 3).
"""
from __future__ import annotations

import numpy as np

from . import apply as A
from . import kernel as K


class PBProblem:
    def __init__(self, N: int, eps: np.ndarray, grad_eps: np.ndarray, L: float | None = None):
        self.N = N
        self.eps = np.asarray(eps, dtype=np.float64)
        self.d = self.eps.ndim
        self.ge = np.asarray(grad_eps, dtype=np.float64)
        L = (1.8 if self.d == 3 else 1.5) if L is None else L
        T = K.T_octant_by_sums(self.d, N, "laplace", 0.0, L)
        self.G = K.ghat_full_from_octant(K.ghat_octant_by_sums(T, N))
        self.Gj = []
        for j in range(self.d):
            Tj = K.T_octant_by_sums(self.d, N, "laplace", 0.0, L, deriv_axis=j)
            self.Gj.append(K.ghat_full_from_octant(K.ghat_octant_by_sums(Tj, N, odd_axis=j), odd_axis=j))

    def V(self, s):
        return A.apply_fft2n(self.G, s)

    def grad_V(self, s):
        return [A.apply_fft2n(g, s) for g in self.Gj]

    def op(self, s):
        out = -self.eps * s
        for j, g in enumerate(self.grad_V(s)):
            out = out + self.ge[j] * g
        return out


def dense_solve(prob: PBProblem, rho: np.ndarray) -> np.ndarray:
    """Builds the N^d x N^d matrix of M from unit vectors and solves M sigma = rho."""
    n = prob.N ** prob.d
    Mx = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for j in range(n):
        e[j] = 1.0
        Mx[:, j] = prob.op(e.reshape((prob.N,) * prob.d)).ravel()
        e[j] = 0.0
    return np.linalg.solve(Mx, np.asarray(rho, dtype=np.complex128).ravel()).reshape(rho.shape)
