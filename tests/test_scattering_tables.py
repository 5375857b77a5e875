"""Host logic of the scattering experiments (no GPU): every grid of the tables
is a built FFT length nested in its reference grid, and the nested sampling
picks the coarse grid's points out of the fine grid."""
import numpy as np
import torch

from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import scattering as S
from paper_1604_03155_gb300 import vp


def test_table_grids_are_built_lengths_nested_in_their_reference():
    lib = vp.lib(build_if_missing=True)
    for spec in (S.TABLES, S.QUICK):
        for name, (d, contrast, rows) in spec.items():
            for size, n_ref, grids in rows:
                assert lib.vp_fft_length_supported(2 * n_ref) == 1, (name, n_ref)
                for N in grids:
                    assert n_ref % N == 0 and N < n_ref, (name, N)
                    assert lib.vp_fft_length_supported(2 * N) == 1, (name, N)
                    # at least ~3 points per wavelength
                    assert N >= 3 * size, (name, size, N)


def test_nested_sampling_picks_the_coarse_points():
    for d, (N, n_ref) in [(2, (24, 768)), (2, (256, 2048)), (3, (32, 384)), (3, (128, 384))]:
        xf, xc = I.grid_coords(n_ref), I.grid_coords(N)
        idx = torch.arange(n_ref, dtype=torch.float64)
        sub = S.nested(idx.reshape((n_ref,) + (1,) * (d - 1)).expand((n_ref,) * d).contiguous(), N)
        assert sub.shape == (N,) * d
        picked = sub.reshape(N, -1)[:, 0].long().numpy()
        assert np.array_equal(xf[picked], xc)
    # errors: zero for identical fields, scale-invariant
    u = torch.randn(8, 8, dtype=torch.complex128)
    assert S.errors(u, u) == (0.0, 0.0)
    e2, einf = S.errors(2 * u, u)
    assert abs(e2 - 1.0) < 1e-15 and abs(einf - 1.0) < 1e-15
