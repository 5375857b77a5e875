"""Pins of the Nystrom matrix view of T (Section 4, the remark after the
discrete convolution; Fig. 2), oracle side, no GPU."""
import numpy as np
import pytest

from oracle import apply as A
from oracle import kernel as K
from paper_1604_03155_gb300 import inputs as I


@pytest.mark.parametrize("d,N,kernel,k,L,odd", [(3, 4, "laplace", 0.0, 1.8, None), (3, 4, "helmholtz", 7.0, 1.8, 2),
                                                (2, 6, "helmholtz", 11.0, 1.5, None), (2, 6, "biharmonic", 0.0, 1.5, 0)])
def test_matrix_times_density_is_the_convolution(d, N, kernel, k, L, odd):
    """The full N^d x N^d matrix applied to f equals the discrete convolution
    (brute force) and hence the potential; even kernels give a symmetric
    matrix, odd (derivative) kernels an antisymmetric one."""
    T = K.T_octant_by_sums(d, N, kernel, k, L, deriv_axis=odd)
    idx = np.arange(N ** d)
    M = K.nystrom_block(T, idx, idx, odd_axis=odd)
    f = I.random_complex_field(21, (N,) * d)
    ref = A.apply_direct(K.T_full_from_octant(T, odd), f)
    assert np.abs(M @ f.ravel() - ref.ravel()).max() < 1e-14 * np.abs(ref).max()
    assert np.array_equal(M, M.T) if odd is None else np.array_equal(M, -M.T)
    # a sub-block is the same entries
    rows, cols = idx[3::5], idx[1::3]
    assert np.array_equal(K.nystrom_block(T, rows, cols, odd_axis=odd), M[np.ix_(rows, cols)])


def test_kernel_line_is_a_mollified_green_function():
    """Fig. 2: along y = z = 0 the 3D Laplace T is finite at the origin and
    tends to the naive trapezoidal weight h^3/(4 pi |x|) away from it."""
    N = 32
    h = 1.0 / N
    T = K.T_octant_by_sums(3, N, "laplace", 0.0, 1.8)
    line = T[:, 0, 0].real
    assert np.isfinite(line[0]) and line[0] > line[1] > line[2] > 0
    naive = h ** 3 / (4 * np.pi * np.arange(1, N + 1) * h)
    ratio = line[1:] / naive
    assert abs(ratio[0] - 1) < 0.1 and np.all(np.abs(ratio[7:N - 2] - 1) < 0.02)
