"""GPU FP64 precompute (spectrum sampling, kernel transform, crop and 2N
multiplier; derivative kernels) against the CPU oracle."""
import numpy as np
import pytest

from oracle_cases import grad_octants, octants
from paper_1604_03155_gb300.vp import Plan

pytestmark = pytest.mark.gpu

CASES = [(3, "laplace", 0.0, 1.8, 4), (3, "laplace", 0.0, 1.8, 16), (3, "helmholtz", 60.0, 1.8, 16),
         (3, "helmholtz", 3.0, 2.5, 12), (2, "laplace", 0.0, 1.5, 32), (2, "helmholtz", 40.0, 1.5, 64),
         (2, "helmholtz", 0.3, 1.5, 8), (3, "helmholtz", 0.1, 1.8, 8), (2, "laplace", 0.0, 2.9, 48)]


def _relmax(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("d,kernel,k,L,N", CASES)
def test_kernel_and_multiplier_octants(d, kernel, k, L, N):
    plan = Plan(d, N, kernel, k, L)
    T, G = octants(d, N, kernel, k, L)
    assert _relmax(plan.get_array("T"), T) < 1e-13
    assert _relmax(plan.get_array("ghat"), G) < 1e-13
    plan.close()


@pytest.mark.parametrize("d,kernel,k,L,N", [CASES[1], CASES[2], CASES[4], CASES[5]])
def test_derivative_octants(d, kernel, k, L, N):
    plan = Plan(d, N, kernel, k, L)
    for j in range(d):
        Tj, Gj = grad_octants(d, N, kernel, k, L, j)
        assert _relmax(plan.get_array("Tj", j), Tj) < 1e-13
        assert _relmax(plan.get_array("ghatj", j), Gj) < 1e-13
    plan.close()


def test_default_L_and_info():
    plan = Plan(3, 8, "laplace", 0.0, 0.0)
    info = plan.info()
    assert info["L"] == 1.8 and info["d"] == 3 and info["N"] == 8 and info["device_bytes"] > 0
    plan.close()
    plan = Plan(2, 8, "helmholtz", 5.0, -1.0)
    assert plan.info()["L"] == 1.5
    plan.close()
