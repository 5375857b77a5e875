"""Pins of the Gaussian-source closed forms (Section 5.1) against direct radial
quadrature of the convolution, with the corrections to the printed formulas
(no GPU)."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import closed_forms as CF

RADII = [0.0, 0.01, 0.05, 0.2, 0.45, 0.8]


@pytest.mark.parametrize("r", RADII[1:])
def test_laplace3_vs_quadrature(r):
    assert CF.laplace3(np.array([r]), 0.05)[0] == pytest.approx(
        CF.radial_convolution(3, "laplace", 0.0, 0.05, r).real, rel=1e-12)


@pytest.mark.parametrize("r", RADII[1:])
@pytest.mark.parametrize("k", [2.0, 40.0])
def test_helmholtz3_vs_quadrature(r, k):
    got = CF.helmholtz3(np.array([r]), 0.05, k)[0]
    ref = CF.radial_convolution(3, "helmholtz", k, 0.05, r)
    assert abs(got - ref) < 1e-11 * abs(ref)


def test_helmholtz3_printed_sign_is_negated():
    """As printed, eq. (test_helm_3D) is exactly minus the potential."""
    r, s, k = 0.2, 0.05, 2.0
    arg = (1j * s * s * k - r) / (math.sqrt(2) * s)
    printed = math.exp(-0.5 * s * s * k * k) / (4 * math.pi * r) * (
        np.real(np.exp(-1j * k * r) * special.erf(arg)) - 1j * math.sin(k * r))
    ref = CF.radial_convolution(3, "helmholtz", k, s, r)
    assert abs(printed + ref) < 1e-11 * abs(ref)


def test_helmholtz3_limit_at_origin():
    a = CF.helmholtz3(np.array([0.0, 1e-7]), 0.05, 2.0)
    assert abs(a[0] - a[1]) < 1e-7 * abs(a[0])
    assert CF.laplace3(np.array([0.0]), 0.05)[0] == pytest.approx(CF.laplace3(np.array([1e-8]), 0.05)[0], rel=1e-9)


@pytest.mark.parametrize("r", RADII)
def test_laplace2_vs_quadrature(r):
    got = CF.laplace2(np.array([r]), 0.05)[0]
    ref = CF.radial_convolution(2, "laplace", 0.0, 0.05, max(r, 1e-300)).real
    assert got == pytest.approx(ref, rel=1e-11, abs=1e-13)


def test_laplace2_with_E1_not_Ei():
    """With Ei in place of E_1 the printed formula is off by O(1) (and complex
    for the principal branch); E_1 matches the convolution."""
    r, s = 0.2, 0.05
    x = r * r / (2 * s * s)
    printed = -(special.expi(x) + math.log(r * r)) / (4 * math.pi)
    ref = CF.radial_convolution(2, "laplace", 0.0, s, r).real
    assert abs(printed - ref) > 1.0
    assert CF.laplace2(np.array([r]), s)[0] == pytest.approx(ref, rel=1e-11)


def test_helmholtz2_far_field_and_near_field():
    """Far from the source (r >> sigma) the potential is (i/4) H_0(kr) times the
    Gaussian's transform at k (Graf addition theorem reduces to it exactly for
    r outside the support, up to the exponentially small tail)."""
    s, k = 0.05, 2.0
    r = 0.9
    got = CF.helmholtz2(np.array([r]), s, k)[0]
    ref = 0.25j * special.hankel1(0, k * r) * math.exp(-0.5 * s * s * k * k)
    assert abs(got - ref) < 1e-12 * abs(ref)
    # continuity at the origin
    a = CF.helmholtz2(np.array([0.0, 1e-6]), s, k)
    assert abs(a[0] - a[1]) < 1e-6 * abs(a[0])


@pytest.mark.parametrize("r", RADII)
def test_biharmonic3_vs_quadrature(r):
    got = CF.biharmonic3(np.array([r]), 0.05)[0]
    if r == 0.0:  # the limit: E|Y| = 2 sigma sqrt(2/pi) for Y ~ N(0, sigma^2 I_3), over 8 pi
        assert got == pytest.approx(2 * 0.05 * math.sqrt(2 / math.pi) / (8 * math.pi), rel=1e-15)
        return
    assert got == pytest.approx(CF.radial_convolution(3, "biharmonic", 0.0, 0.05, r).real, rel=1e-12)


def test_biharmonic3_printed_form_misses_the_exponential():
    """As printed (no e^{-r^2/(2 sigma^2)} on sigma sqrt(2/pi)) the far field is
    off by sigma sqrt(2/pi)/(8 pi); with the factor it matches quadrature."""
    sig, r = 0.05, 0.45
    printed = (sig * math.sqrt(2 / math.pi) + special.erf(r / (sig * math.sqrt(2))) * (sig * sig / r + r)) / (8 * math.pi)
    ref = CF.radial_convolution(3, "biharmonic", 0.0, sig, r).real
    assert abs(printed - ref) == pytest.approx(sig * math.sqrt(2 / math.pi) / (8 * math.pi), rel=1e-6)
    assert CF.biharmonic3(np.array([r]), sig)[0] == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("r", [0.0, 0.03, 0.1, 0.3])
def test_biharmonic2_vs_quadrature(r):
    got = CF.biharmonic2(np.array([r]), 0.05)[0]
    ref = CF.radial_convolution(2, "biharmonic", 0.0, 0.05, r).real if r > 0 else None
    if r == 0.0:
        # the limit: -sigma^2/(8 pi) (0 - 1) + c_1, against quadrature just off the origin
        ref = CF.radial_convolution(2, "biharmonic", 0.0, 0.05, 1e-7).real
        assert got == pytest.approx(ref, rel=1e-9)
        return
    assert got == pytest.approx(ref, rel=1e-11)


def test_biharmonic2_printed_linear_term_is_a_constant():
    """With c_1 r (as printed) the formula misses quadrature by c_1 (r - 1)."""
    sig = 0.05
    c1 = sig * sig / (8 * math.pi) * (CF.EULER_GAMMA + math.log(1 / (2 * sig * sig)))
    r = 0.2
    ref = CF.radial_convolution(2, "biharmonic", 0.0, sig, r).real
    assert CF.biharmonic2(np.array([r]), sig)[0] == pytest.approx(ref, rel=1e-11)
    assert abs((CF.biharmonic2(np.array([r]), sig)[0] - c1 + c1 * r) - ref) > 1e-3 * abs(ref)
