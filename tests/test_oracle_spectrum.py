"""Pins of the truncated spectra G^L(s) (Tables 1-2) against the defining radial
integrals of Section 2, limits, the printed table forms and high-precision
arithmetic near the removable singularity s = k (no GPU)."""
import json
import math
import os

import numpy as np
import pytest

from oracle import spectrum as S

CASES = [(3, "laplace", 0.0, 1.8), (3, "helmholtz", 60.0, 1.8), (3, "helmholtz", 2.0, 1.8),
         (2, "laplace", 0.0, 1.5), (2, "helmholtz", 40.0, 1.5), (2, "helmholtz", 2.0, 1.5),
         (3, "biharmonic", 0.0, 1.8), (2, "biharmonic", 0.0, 1.5)]


@pytest.mark.parametrize("d,kernel,k,L", CASES)
@pytest.mark.parametrize("s", [0.0, math.pi / 2, 3.0, 7.3, 39.985, 40.0, 60.0, 61.2, 120.0])
def test_closed_form_vs_radial_quadrature(d, kernel, k, L, s):
    g = S.G_truncated(d, kernel, k, L, np.array([s]))[0]
    q = S.G_quadrature(d, kernel, k, L, s)
    scale = max(abs(q), 1e-3 * abs(S.G_truncated(d, kernel, k, L, np.array([0.0]))[0]))
    assert abs(g - q) <= 1e-11 * scale


def test_default_L_from_paper():
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")) as fh:
        gold = json.load(fh)
    assert S.default_L(3) == gold["L_default_3d"]["value"] > math.sqrt(3)
    assert S.default_L(2) == gold["L_default_2d"]["value"] > math.sqrt(2)


def test_limits_at_zero():
    L = 1.8
    assert S.G_laplace3(np.array([0.0]), L)[0] == pytest.approx(L * L / 2, rel=1e-15)
    assert S.G_laplace3(np.array([1e-6]), L)[0].real == pytest.approx(L * L / 2, rel=1e-11)
    L2 = 1.5
    g0 = L2 * L2 * (1 - 2 * math.log(L2)) / 4
    assert S.G_laplace2(np.array([0.0]), L2)[0].real == pytest.approx(g0, rel=1e-15)
    assert abs(g0 - 0.106352) < 1e-6
    # continuity across the series/direct switch at Ls = 0.5
    a = S.G_laplace2(np.array([0.5 / L2 - 1e-14, 0.5 / L2 + 1e-14]), L2)
    assert abs(a[0] - a[1]) < 1e-12
    k = 3.0
    g3 = S.G_helmholtz3(np.array([0.0, 1e-5]), k, L)
    assert abs(g3[0] - (np.exp(1j * k * L) * (1 - 1j * k * L) - 1) / k ** 2) < 1e-15
    assert abs(g3[1] - g3[0]) < 1e-8
    g2 = S.G_helmholtz2(np.array([0.0, 1e-6]), k, L2)
    assert abs(g2[0] - g2[1]) < 1e-9


@pytest.mark.parametrize("d,L", [(3, 1.8), (2, 1.5), (3, 2.4), (2, 2.9)])
def test_biharmonic_limits_series_switch_and_small_s(d, L):
    """s = 0: the integral of g_b over the ball, L^4/8 (3D) and
    -L^4 (4 log L - 5)/64 (2D); the series and the closed form agree where they
    switch (x = Ls = 2), and at small s the series matches quadrature where the
    closed form has lost its digits to cancellation."""
    G = S.G_biharm3 if d == 3 else S.G_biharm2
    g0 = L ** 4 / 8 if d == 3 else -L ** 4 * (4 * math.log(L) - 5) / 64
    assert G(np.array([0.0]), L)[0].real == pytest.approx(g0, rel=1e-15)
    assert g0 == pytest.approx(S.G_quadrature(d, "biharmonic", 0.0, L, 0.0).real, rel=1e-12)
    x0 = S.BIHARM_SERIES_X / L  # s where x = Ls crosses the switch
    a = G(np.array([np.nextafter(x0, 0.0), np.nextafter(x0, 10.0)]), L)
    assert abs(a[0] - a[1]) < 2e-14 * abs(g0)
    for s in (1e-3, 0.05, 0.7):
        q = S.G_quadrature(d, "biharmonic", 0.0, L, s)
        assert abs(G(np.array([s]), L)[0] - q) < 1e-12 * abs(q)
    # the spectrum is real (g_b is real) and decays like s^-3 (3D) / s^-2.5 (2D) envelopes
    s = np.linspace(0.0, 300.0, 601)
    assert np.all(G(s, L).imag == 0)


def test_helmholtz3_tends_to_laplace_as_k_to_zero():
    s = np.linspace(0.0, 50.0, 101)
    assert np.abs(S.G_helmholtz3(s, 1e-10, 1.8) - S.G_laplace3(s, 1.8)).max() < 1e-9
    # first order in k: Im G_k(0) = k L^3/3
    assert S.G_helmholtz3(np.array([0.0]), 1e-4, 1.8)[0].imag == pytest.approx(1e-4 * 1.8 ** 3 / 3, rel=1e-6)


def test_stable_forms_equal_printed_tables_away_from_pole():
    s = np.linspace(0.5, 200.0, 997)
    for k in (2.0, 40.0, 60.0):
        far = np.abs(s - k) > 2.0
        a = S.G_helmholtz3(s[far], k, 1.8)
        b = S.G_helmholtz3_table(s[far], k, 1.8)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
        a = S.G_helmholtz2(s[far], k, 1.5)
        b = S.G_helmholtz2_table(s[far], k, 1.5)
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


@pytest.mark.parametrize("d", [2, 3])
def test_near_pole_against_high_precision_table(d):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 60
    k = 40.0
    L = 1.8 if d == 3 else 1.5
    for ds in (-0.6, -1e-3, -1e-7, 0.0, 1e-9, 1e-4, 0.3, 0.99):
        s = k + ds
        if d == 3:
            got = S.G_helmholtz3(np.array([s]), k, L)[0]
        else:
            got = S.G_helmholtz2(np.array([s]), k, L)[0]
        if ds == 0.0:
            sm = mpmath.mpf(s) + mpmath.mpf("1e-25")  # the removable value, approached from above
        else:
            sm = mpmath.mpf(s)
        km, Lm = mpmath.mpf(k), mpmath.mpf(L)
        if d == 3:
            num = -1 + mpmath.exp(1j * Lm * km) * (mpmath.cos(Lm * sm) - 1j * (km / sm) * mpmath.sin(Lm * sm))
            ref = num / ((km - sm) * (km + sm))
        else:
            H0 = mpmath.hankel1(0, Lm * km)
            H1 = mpmath.hankel1(1, Lm * km)
            num = (1 + 0.5j * mpmath.pi * Lm * sm * mpmath.besselj(1, Lm * sm) * H0
                   - 0.5j * mpmath.pi * Lm * km * mpmath.besselj(0, Lm * sm) * H1)
            ref = num / (sm * sm - km * km)
        ref = complex(ref)
        assert abs(got - ref) <= 1e-13 * abs(ref), (d, ds, got, ref)


def test_removable_values_at_s_equal_k():
    k, L = 40.0, 1.5
    from scipy import special
    g = S.G_helmholtz2(np.array([k]), k, L)[0]
    ref = 0.25j * math.pi * L * L * (special.j0(k * L) * special.hankel1(0, k * L)
                                    + special.j1(k * L) * special.hankel1(1, k * L))
    assert abs(g - ref) < 1e-14 * abs(ref)
    L3 = 1.8
    g3 = S.G_helmholtz3(np.array([k]), k, L3)[0]
    ref3 = 1j * L3 / (2 * k) - (np.exp(2j * k * L3) - 1) / (4 * k * k)
    assert abs(g3 - ref3) < 1e-14 * abs(ref3)


def test_laplace_spectra_real_and_radial_symmetry_of_inputs():
    s = np.linspace(0, 300, 301)
    assert np.all(S.G_laplace3(s, 1.8).imag == 0)
    assert np.all(S.G_laplace2(s, 1.5).imag == 0)
