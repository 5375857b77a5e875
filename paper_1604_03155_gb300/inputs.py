"""Seeded synthetic inputs shared by the CUDA path's tests, the bench and the oracle.

This module holds no arithmetic of the volume-potential method: it only draws
random numbers and samples the test densities on the grid.  Both sides of every
parity check read the arrays produced here, so the CUDA library and the CPU
oracle always see bit-identical inputs.

Random numbers come from one counter-based generator, splitmix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): the i-th
draw of stream ``seed`` is ``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.  Uniform
doubles take the top 53 bits; normal draws use the Box-Muller transform.

Grid convention (paper Section 4): N even, h = 1/N, storage index p in [0, N)
maps to grid index i = p - N/2 + 1 and coordinate x = i * h, so the origin is a
grid node and the box is [-1/2 + h, 1/2] per axis.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Base seed of the workload recipes; workload c uses BASE_SEED + c.
BASE_SEED = 1604031550


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+count-1`` of the splitmix64 stream ``seed`` (uint64)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def normal(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normal doubles by Box-Muller on pairs of uniforms."""
    npair = (count + 1) // 2
    u = uniform(seed, 2 * npair, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npair)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def grid_coords(N: int) -> np.ndarray:
    """Coordinates x_p = (p - N/2 + 1)/N of one grid axis (paper Section 4)."""
    if N <= 0 or N % 2:
        raise ValueError("N must be a positive even integer")
    p = np.arange(N, dtype=np.float64)
    return (p - N // 2 + 1) / N


@dataclass
class GaussianSources:
    """f(x) = sum_q a_q exp(-|x - c_q|^2 / sigma_q^2)."""

    centres: np.ndarray  # (Q, d)
    sigmas: np.ndarray  # (Q,)
    amps: np.ndarray  # (Q,) complex

    @property
    def d(self) -> int:
        return self.centres.shape[1]


def random_gaussians(seed: int, count: int, d: int, centre_half_width: float = 0.3,
                     sigma_range=(0.03, 0.08), complex_amps: bool = True) -> GaussianSources:
    """Gaussian sources with centres U[-w, w]^d, widths U[sigma_range] and
    amplitudes whose real and imaginary parts are independent N(0, 1)."""
    u = uniform(seed, count * (d + 1))
    centres = (2.0 * u[: count * d].reshape(count, d) - 1.0) * centre_half_width
    lo, hi = sigma_range
    sigmas = lo + (hi - lo) * u[count * d:]
    z = normal(seed ^ 0x5DEECE66D, 2 * count)
    amps = z[:count] + (1j * z[count:] if complex_amps else 0.0)
    return GaussianSources(centres, sigmas, amps.astype(np.complex128))


def sample_gaussians(src: GaussianSources, N: int) -> np.ndarray:
    """Samples the sources on the N^d grid, C order, last axis fastest (complex128)."""
    x = grid_coords(N)
    d = src.d
    f = np.zeros((N,) * d, dtype=np.complex128)
    for c, s, a in zip(src.centres, src.sigmas, src.amps):
        # separable: exp(-sum_j (x_j - c_j)^2 / s^2) = prod_j exp(-(x_j - c_j)^2 / s^2)
        term = np.array(a, dtype=np.complex128)
        for j in range(d):
            e = np.exp(-((x - c[j]) ** 2) / (s * s))
            shape = [1] * d
            shape[j] = N
            term = term * e.reshape(shape)
        f += term
    return f


def random_complex_field(seed: int, shape) -> np.ndarray:
    """Unstructured complex N(0,1) field, for linearity and edge-case checks."""
    n = int(np.prod(shape))
    z = normal(seed, 2 * n)
    return (z[:n] + 1j * z[n:]).reshape(shape)


# ---------------------------------------------------------------------------
# Workload recipes (the five configurations of the benchmark suite)
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    d: int
    N: int
    kernel: str  # "laplace" | "helmholtz"
    k: float
    L: float  # <= 0 selects the paper's default (1.8 in 3D, 1.5 in 2D)
    seed: int
    n_gauss: int
    precision: str  # "fp64" | "fp32"
    grad: bool = False
    extra: dict = field(default_factory=dict)

    def density(self, N: int | None = None) -> np.ndarray:
        """The workload's density, optionally sampled on another grid size."""
        N = self.N if N is None else N
        if self.name == "laplace3d_single_gaussian":
            src = GaussianSources(np.zeros((1, 3)), np.array([0.08]), np.array([1.0 + 0j]))
        else:
            src = random_gaussians(self.seed, self.n_gauss, self.d)
        return sample_gaussians(src, N)


def workload(name: str) -> Workload:
    """The benchmark workloads by name."""
    if name == "laplace3d_single_gaussian":  # 3D Laplace, N=32, one Gaussian sigma=0.08, FP64
        return Workload(name, 3, 32, "laplace", 0.0, 1.8, BASE_SEED + 1, 1, "fp64")
    if name == "helmholtz2d_k40_n1024_grad":  # 2D Helmholtz k=40, N=1024, 8 Gaussians, FP32 + grad
        return Workload(name, 2, 1024, "helmholtz", 40.0, 1.5, BASE_SEED + 2, 8, "fp32", grad=True)
    if name == "helmholtz3d_k60_n256":  # 3D Helmholtz k=60, N=256, 16 Gaussians, FP32
        return Workload(name, 3, 256, "helmholtz", 60.0, 1.8, BASE_SEED + 3, 16, "fp32")
    if name == "biharmonic3d_n256":  # 3D biharmonic, N=256, 16 Gaussians, FP32
        return Workload(name, 3, 256, "biharmonic", 0.0, 1.8, BASE_SEED + 6, 16, "fp32")
    raise KeyError(name)


def batch_recipe(seed: int = BASE_SEED + 4, count: int = 64):
    """64 densities: N uniform in {48, 64, 96, 128}, half Laplace and half
    Helmholtz with k ~ U[5, 40], four Gaussians each (3D, FP32)."""
    u = uniform(seed, 2 * count)
    sizes = np.array([48, 64, 96, 128])
    out = []
    for i in range(count):
        N = int(sizes[min(3, int(u[i] * 4))])
        helm = i >= count // 2
        k = 5.0 + 35.0 * u[count + i] if helm else 0.0
        w = Workload(f"batch{i}", 3, N, "helmholtz" if helm else "laplace", k, 1.8,
                     seed * 1000 + i, 4, "fp32")
        out.append(w)
    return out


def sample_gaussians_grid(src: GaussianSources, Ns) -> np.ndarray:
    """The sources on a grid with Ns[j] points along axis j (complex128)."""
    d = src.d
    xs = [grid_coords(N) for N in Ns]
    f = np.zeros(tuple(Ns), dtype=np.complex128)
    for c, s, a in zip(src.centres, src.sigmas, src.amps):
        g = np.ones((1,) * d)
        for j in range(d):
            shape = [1] * d
            shape[j] = Ns[j]
            g = g * np.exp(-((xs[j] - c[j]) ** 2) / (s * s)).reshape(shape)
        f += a * g
    return f


def batch_recipe_grids(seed: int = BASE_SEED + 8, count: int = 64):
    """The batch with per-axis sizes: 64 densities, each axis's N drawn
    uniformly from {48, 64, 96, 128}; half Laplace and half Helmholtz with
    k ~ U[5, 40]; four Gaussians each (3D, FP32).  Returns (Ns, kernel, k,
    density) tuples."""
    u = uniform(seed, 4 * count)
    sizes = np.array([48, 64, 96, 128])
    out = []
    for i in range(count):
        Ns = tuple(int(sizes[min(3, int(u[3 * i + j] * 4))]) for j in range(3))
        helm = i >= count // 2
        k = 5.0 + 35.0 * u[3 * count + i] if helm else 0.0
        src = random_gaussians(seed * 1000 + i, 4, 3)
        out.append((Ns, "helmholtz" if helm else "laplace", k, sample_gaussians_grid(src, Ns)))
    return out


def to_device_dtype(f: np.ndarray, precision: str) -> np.ndarray:
    """The array both sides consume: complex64 for the FP32 path, complex128 for FP64."""
    return f.astype(np.complex64 if precision == "fp32" else np.complex128)


def gaussian_amplitude(sigma_cfg: float, d: int) -> float:
    """exp(-r^2/sigma^2) = Q * rho(r) with rho the unit-mass Gaussian of standard
    deviation sigma/sqrt(2); returns Q = (pi sigma^2)^(d/2)."""
    return (math.pi * sigma_cfg * sigma_cfg) ** (d / 2)


# ---------------------------------------------------------------------------
# Lippmann-Schwinger inputs (contrast and incident field)
# ---------------------------------------------------------------------------

def cube_bump(N: int) -> np.ndarray:
    """The smoothed cube exp(-1/2 sum_j (x_j/0.25)^8) of the paper's 3D
    scattering example (Section 5.3), sampled on the N^3 grid."""
    x = grid_coords(N)
    e = (x / 0.25) ** 8
    return np.exp(-0.5 * (e[:, None, None] + e[None, :, None] + e[None, None, :]))


def ls_contrast(seed: int, N: int) -> np.ndarray:
    """q = 0.5 * smoothed cube + 6 Gaussian perturbations (centres U[-0.3,0.3]^3,
    widths U[0.03,0.08], amplitudes U[-0.25,0.25]); real, float64."""
    u = uniform(seed, 6 * 5)
    q = 0.5 * cube_bump(N)
    x = grid_coords(N)
    for g in range(6):
        c = (2 * u[g * 5:g * 5 + 3] - 1) * 0.3
        s = 0.03 + 0.05 * u[g * 5 + 3]
        a = (2 * u[g * 5 + 4] - 1) * 0.25
        q = q + a * (np.exp(-((x - c[0]) ** 2) / s ** 2)[:, None, None]
                     * np.exp(-((x - c[1]) ** 2) / s ** 2)[None, :, None]
                     * np.exp(-((x - c[2]) ** 2) / s ** 2)[None, None, :])
    return q


def plane_wave(N: int, k: float, d: int = 3) -> np.ndarray:
    """u_inc = exp(i k x_0): a plane wave travelling along the first axis."""
    x = grid_coords(N)
    shape = (N,) + (1,) * (d - 1)
    return np.broadcast_to(np.exp(1j * k * x).reshape(shape), (N,) * d).astype(np.complex128).copy()


def filtered_disk(N: int) -> np.ndarray:
    """The smoothly filtered dielectric disk of Section 5.3,
    q = exp(-1/2 (|x|/0.25)^8), on the N^2 grid (float64)."""
    x = grid_coords(N)
    r = np.sqrt(x[:, None] ** 2 + x[None, :] ** 2)
    return np.exp(-0.5 * (r / 0.25) ** 8)


def luneburg_lens(N: int) -> np.ndarray:
    """The 2D Luneburg lens of Section 5.3, q = 1 - (|x|/0.45)^2 inside the
    lens (|x| <= 0.45) and 0 outside, on the N^2 grid (float64)."""
    x = grid_coords(N)
    r = np.sqrt(x[:, None] ** 2 + x[None, :] ** 2)
    return np.where(r <= 0.45, 1.0 - (r / 0.45) ** 2, 0.0)


LS_TRAIN_SEED = BASE_SEED + 5000     # contrasts LS_TRAIN_SEED + i, i < 2000
LS_HELDOUT_SEED = BASE_SEED + 9000   # held-out contrasts LS_HELDOUT_SEED + i, i < 50


# ---------------------------------------------------------------------------
# Learned preconditioner: network shape and seeded initial weights
# ---------------------------------------------------------------------------

def unet_layer_shapes(C: int = 16, cin: int = 3, cout: int = 2):
    """(C_out, C_in) of the ten 3x3x3 convolutions of the 3-level U-Net, in order:
    E1a, E1b, E2a, E2b, B1, B2, D2a, D2b, D1a, D1b."""
    return [(C, cin), (C, C), (C, C), (C, C), (C, C), (C, C), (C, 2 * C), (C, C), (C, 2 * C), (cout, C)]


def unet_init_weights(seed: int, C: int = 16, cin: int = 3, cout: int = 2):
    """He-style normal weights [C_out][C_in][27] (float32), zero biases; the last
    layer is scaled by 1/100 so that the residual-learning preconditioner starts
    near the identity."""
    out = []
    for i, (co, ci) in enumerate(unet_layer_shapes(C, cin, cout)):
        z = normal(seed + i, co * ci * 27)
        scale = np.sqrt(2.0 / (ci * 27)) * (0.01 if i == 9 else 1.0)
        out.append(((z * scale).reshape(co, ci, 27).astype(np.float32), np.zeros(co, dtype=np.float32)))
    return out


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Rounds float32 values to bfloat16 (round to nearest even), returned as float32."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


# ---------------------------------------------------------------------------
# Variable-coefficient Poisson (Section 5.2): a synthetic molecule standing in
# for the paper's 1235-atom protein (whose coordinates are not available)
# ---------------------------------------------------------------------------

PB_ATOMS = 1235
PB_RADIUS = 0.022  # van der Waals radius R_i of every atom
PB_MU2 = 2.0  # mu^2
PB_EPS_IN, PB_EPS_OUT = 2.0, 4.0
PB_BALL = 0.2  # atom centres uniform in the ball |x| < 0.2
PB_CUTOFF = 6.0  # alpha_i is taken as 0 beyond r = 6 mu R (exp(-36) = 2.3e-16)


def pb_molecule(seed: int = BASE_SEED + 7000, M: int = PB_ATOMS):
    """M atom centres uniform in a ball of radius 0.2 (splitmix64 rejection
    sampling) and charges uniform in [-1, 1]: (centres (M, 3), charges (M,))."""
    out = []
    off = 0
    while len(out) < M:
        u = uniform(seed, 3 * 4096, off) * 2 - 1
        off += 3 * 4096
        c = u.reshape(-1, 3) * PB_BALL
        out.extend(c[np.sum(c * c, axis=1) < PB_BALL ** 2])
    centres = np.array(out[:M])
    charges = uniform(seed + 1, M) * 2 - 1
    return centres, charges


def pb_fields(mol, N: int, device="cpu", dtype=None, eps_in: float = PB_EPS_IN, eps_out: float = PB_EPS_OUT):
    """The smooth dielectric of Section 5.2 on the N^3 grid: alpha_i =
    exp(-r_i^2/(mu^2 R^2)) (cut off at r = 6 mu R), q = 1 - prod_i (1 - alpha_i),
    eps = q eps_in + (1 - q) eps_out; its exact gradient, and the charge density
    rho = sum_i c_i alpha_i.  Returns torch tensors (eps (N,N,N), grad_eps
    (3,N,N,N), rho (N,N,N)) on `device` (float64 by default).  The product and
    its gradient are accumulated atom by atom over each atom's box:
    P <- P (1 - alpha), G <- G (1 - alpha) - P grad(alpha)."""
    import torch
    dt = torch.float64 if dtype is None else dtype
    x = torch.tensor(grid_coords(N), dtype=dt, device=device)
    h = 1.0 / N
    w2 = PB_MU2 * PB_RADIUS ** 2
    rc = PB_CUTOFF * np.sqrt(w2)
    P = torch.ones((N, N, N), dtype=dt, device=device)
    G = torch.zeros((3, N, N, N), dtype=dt, device=device)
    rho = torch.zeros((N, N, N), dtype=dt, device=device)
    centres, charges = mol
    lo_idx = lambda c: max(0, int(np.ceil((c - rc) / h + N // 2 - 1)))
    hi_idx = lambda c: min(N, int(np.floor((c + rc) / h + N // 2 - 1)) + 1)
    for (cx, cy, cz), ch in zip(centres, charges):
        sl = [slice(lo_idx(c), hi_idx(c)) for c in (cx, cy, cz)]
        if any(s.stop <= s.start for s in sl):
            continue
        dx = (x[sl[0]] - cx).view(-1, 1, 1)
        dy = (x[sl[1]] - cy).view(1, -1, 1)
        dz = (x[sl[2]] - cz).view(1, 1, -1)
        r2 = dx * dx + dy * dy + dz * dz
        a = torch.where(r2 <= rc * rc, torch.exp(-r2 / w2), torch.zeros_like(r2))
        Pb = P[sl[0], sl[1], sl[2]]
        for j, dj in enumerate((dx, dy, dz)):
            ga = -2.0 * dj / w2 * a  # d alpha / d x_j
            G[j, sl[0], sl[1], sl[2]] = G[j, sl[0], sl[1], sl[2]] * (1 - a) - Pb * ga
        P[sl[0], sl[1], sl[2]] = Pb * (1 - a)
        rho[sl[0], sl[1], sl[2]] += float(ch) * a
    q = 1 - P
    eps = q * eps_in + (1 - q) * eps_out
    grad_eps = (eps_in - eps_out) * (-G)  # grad q = -grad P
    return eps, grad_eps, rho
