"""Biharmonic kernels on the GPU (Tables 1-2, row Delta^2): the FP64
precompute, the apply (FP32 and FP64, complex and real data) and gradients
against the FP64 oracle, and spectral accuracy against the Gaussian-source
closed forms of Section 5.1 at full size."""
import math

import numpy as np
import pytest
import torch

from oracle import apply as A
from oracle import closed_forms as CF
from oracle_cases import check, condition, grad_octants, octants, potential
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300.vp import Plan

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = {"fp32": 1e-5, "fp64": 1e-12}
NPC = {"fp32": np.complex64, "fp64": np.complex128}


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("d,L,N", [(3, 1.8, 4), (3, 1.8, 16), (3, 2.6, 12), (2, 1.5, 8), (2, 1.5, 64),
                                   (2, 2.9, 48)])
def test_biharmonic_kernel_and_multiplier_octants(d, L, N):
    plan = Plan(d, N, "biharmonic", 0.0, L)
    T, G = octants(d, N, "biharmonic", 0.0, L)
    assert _relmax(plan.get_array("T"), T) < 1e-13
    assert _relmax(plan.get_array("ghat"), G) < 1e-13
    assert np.abs(plan.get_array("ghat").imag).max() == 0.0
    plan.close()


@pytest.mark.parametrize("d,N", [(3, 12), (2, 32)])
def test_biharmonic_derivative_octants(d, N):
    L = 1.8 if d == 3 else 1.5
    plan = Plan(d, N, "biharmonic", 0.0, L)
    for j in range(d):
        Tj, Gj = grad_octants(d, N, "biharmonic", 0.0, L, j)
        assert _relmax(plan.get_array("Tj", j), Tj) < 1e-13
        assert _relmax(plan.get_array("ghatj", j), Gj) < 1e-13
    plan.close()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("d,N", [(3, 6), (3, 12), (3, 24), (2, 8), (2, 48), (2, 96)])
def test_biharmonic_apply_and_gradient(prec, d, N):
    L = 1.8 if d == 3 else 1.5
    plan = Plan(d, N, "biharmonic", 0.0, 0.0, precision=prec)
    f = I.sample_gaussians(I.random_gaussians(5000 + N, 6, d), N).astype(NPC[prec])
    ft = torch.from_numpy(f).to(DEV)
    phi, g = plan.apply_grad(ft)
    phi, g = phi.cpu().numpy(), g.cpu().numpy()
    ref, gref = potential(d, N, "biharmonic", 0.0, L, f, "exact")
    name = f"biharmonic {d}d N={N} {prec}"
    assert check(name + " phi", A.rel_l2(phi, ref), TOL[prec], condition(d, N, "biharmonic", 0.0, L, f))
    assert check(name + " grad", A.rel_l2(g, gref), TOL[prec],
                 max(condition(d, N, "biharmonic", 0.0, L, f, j) for j in range(d)))
    phi_only = plan.apply(ft).cpu().numpy()
    assert np.array_equal(phi_only, phi) or A.rel_l2(phi_only, phi) < TOL[prec]
    plan.close()


@pytest.mark.parametrize("prec,rdt", [("fp32", np.float32), ("fp64", np.float64)])
def test_biharmonic_real_path(prec, rdt):
    d, N = 3, 16
    plan = Plan(d, N, "biharmonic", 0.0, 0.0, precision=prec)
    f = I.sample_gaussians(I.random_gaussians(5100, 4, d), N).real.astype(rdt)
    phi = plan.apply(torch.from_numpy(f).to(DEV)).cpu().numpy()
    ref, _ = potential(d, N, "biharmonic", 0.0, 1.8, f)
    assert phi.dtype == rdt and A.rel_l2(phi, ref.real) < TOL[prec]
    plan.close()


def _gaussian(d, N, sig):
    x = I.grid_coords(N)
    X = np.meshgrid(*([x] * d), indexing="ij")
    r = np.sqrt(sum(a * a for a in X))
    return r, (2 * math.pi * sig * sig) ** (-d / 2) * np.exp(-r * r / (2 * sig * sig))


@pytest.mark.parametrize("d,N,tol", [(3, 128, 1e-11), (2, 1024, 1e-11)])
def test_biharmonic_gaussian_closed_form_full_size(d, N, tol):
    """The Gaussian of Section 5.1 (sigma = 0.05, unit mass), FP64: the apply
    reaches the corrected closed forms to spectral accuracy."""
    sig = 0.05
    r, rho = _gaussian(d, N, sig)
    plan = Plan(d, N, "biharmonic", 0.0, 0.0, precision="fp64")
    phi = plan.apply(torch.from_numpy(rho).to(DEV)).cpu().numpy()
    ex = CF.biharmonic3(r, sig) if d == 3 else CF.biharmonic2(r, sig)
    assert A.rel_l2(phi, ex) < tol
    plan.close()
