"""Nystrom entries on the GPU (Section 4, the remark after the discrete
convolution): kernel entries at offsets and dense matrix blocks against the
plan's own FP64 octant (bit for bit) and the oracle, and the block times a
density against the apply."""
import numpy as np
import pytest
import torch

from oracle import kernel as K
from oracle_cases import grad_octants, octants
from paper_1604_03155_gb300 import inputs as I
from paper_1604_03155_gb300 import vp
from paper_1604_03155_gb300.vp import Plan, VPError

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
CASES = [(3, 16, "laplace", 0.0, 1.8), (3, 12, "helmholtz", 9.0, 1.8), (2, 64, "helmholtz", 40.0, 1.5),
         (2, 48, "biharmonic", 0.0, 1.5)]


def _offsets(rng, d, N, count):
    off = rng.integers(-N, N + 1, size=(count, d)).astype(np.int32)
    off[0] = 0
    off[1] = N
    off[2] = -N
    off[3, 0] = N - 1
    return off


@pytest.mark.parametrize("d,N,kernel,k,L", CASES)
def test_entries_equal_the_octant_and_the_oracle(d, N, kernel, k, L):
    plan = Plan(d, N, kernel, k, L, precision="fp64")
    rng = np.random.default_rng(N)
    off = _offsets(rng, d, N, 5000)
    got = plan.kernel_entries(torch.from_numpy(off).to(DEV)).cpu().numpy()
    own = plan.get_array("T")
    exact = own[tuple(np.abs(off).T)]
    assert np.array_equal(got, exact)  # a gather: bit for bit
    T, _ = octants(d, N, kernel, k, L)
    Tf = K.T_full_from_octant(T)
    ref = Tf[tuple((off + N).T)]
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
    # derivative kernel along the last axis: odd
    j = d - 1
    gj = plan.kernel_entries(torch.from_numpy(off).to(DEV), "Tj", j).cpu().numpy()
    Tj, _ = grad_octants(d, N, kernel, k, L, j)
    refj = K.T_full_from_octant(Tj, j)[tuple((off + N).T)]
    assert np.abs(gj - refj).max() <= 1e-13 * np.abs(refj).max()
    # FP32 output is the rounded FP64 value
    g32 = plan.kernel_entries(torch.from_numpy(off).to(DEV), dtype=torch.complex64).cpu().numpy()
    assert np.array_equal(g32, exact.astype(np.complex64))
    plan.close()


@pytest.mark.parametrize("d,N,kernel,k,L", CASES)
def test_block_against_oracle_and_apply(d, N, kernel, k, L):
    plan = Plan(d, N, kernel, k, L, precision="fp64")
    U = N ** d
    rng = np.random.default_rng(7 + N)
    rows = np.unique(rng.integers(0, U, 37))
    rows[0], rows[-1] = 0, U - 1
    cols = np.arange(U, dtype=np.int64)
    blk = plan.matrix_block(torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV)).cpu().numpy()
    T, _ = octants(d, N, kernel, k, L)
    sub = cols[::max(1, U // 300)]
    ref = K.nystrom_block(T, rows, sub)
    assert np.abs(blk[:, ::max(1, U // 300)] - ref).max() <= 1e-13 * np.abs(ref).max()
    # rows of the matrix times f = the apply at those rows
    f = I.sample_gaussians(I.random_gaussians(600 + N, 5, d), N)
    ft = torch.from_numpy(f).to(DEV)
    phi = plan.apply(ft).cpu().numpy().ravel()
    assert np.abs(blk @ f.ravel() - phi[rows]).max() <= 1e-12 * np.abs(phi).max()
    # derivative block rows times f = the exact gradient at those rows
    plan.set_grad_mode("exact")
    _, g = plan.apply_grad(ft)
    g0 = g.cpu().numpy()[0].ravel()
    bj = plan.matrix_block(torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV), "Tj", 0).cpu().numpy()
    assert np.abs(bj @ f.ravel() - g0[rows]).max() <= 1e-12 * np.abs(g0).max()
    plan.close()


def test_full_size_block_and_kernel_line():
    """3D N = 256 (the benchmark grid): a 4096 x 4096 block, entries spot-checked
    against the octant; the kernel line of Fig. 2 is even and peaked at 0."""
    N = 256
    plan = Plan(3, N, "helmholtz", 60.0, 1.8, precision="fp32")
    U = N ** 3
    g = torch.Generator(device="cpu").manual_seed(5)
    rows = torch.randint(0, U, (4096,), generator=g).to(DEV)
    cols = torch.randint(0, U, (4096,), generator=g).to(DEV)
    blk = plan.matrix_block(rows, cols).cpu().numpy()
    own = plan.get_array("T")
    r, c = rows.cpu().numpy(), cols.cpu().numpy()
    for i, j in [(0, 0), (4095, 4095), (17, 3001), (2048, 5)]:
        p = np.array(np.unravel_index(r[i], (N,) * 3))
        q = np.array(np.unravel_index(c[j], (N,) * 3))
        assert blk[i, j] == own[tuple(np.abs(p - q))]
    line = plan.kernel_line(0).cpu().numpy()
    assert line.shape == (2 * N - 1,) and np.array_equal(line, line[::-1])
    assert np.abs(line).argmax() == N - 1
    plan.close()


def test_entries_edge_cases():
    plan = Plan(2, 16, "laplace", 0.0, 0.0, precision="fp64")
    off = torch.tensor([[0, 0], [17, 0], [3, -2]], dtype=torch.int32, device=DEV)
    with pytest.raises(VPError):
        plan.kernel_entries(off)
    # the in-range entries are still written, the bad one is zero
    out = torch.full((3,), 7.0, dtype=torch.complex128, device=DEV)
    code = vp.lib().vp_kernel_entries(plan.handle, vp.VP_ARRAY_T, 0, off.data_ptr(), 3, out.data_ptr(), vp.VP_C128)
    assert code == vp.VP_ERR_INVALID_ARG and out[1] == 0 and out[0] != 0
    # empty request, host pointers, bad which/axis, bad block index
    assert vp.lib().vp_kernel_entries(plan.handle, vp.VP_ARRAY_T, 0, None, 0, None, vp.VP_C128) == vp.VP_OK
    host = np.zeros((2, 2), dtype=np.int32)
    hout = np.zeros(2, dtype=np.complex128)
    assert vp.lib().vp_kernel_entries(plan.handle, vp.VP_ARRAY_T, 0, host.ctypes.data, 2, hout.ctypes.data,
                                      vp.VP_C128) == vp.VP_ERR_INVALID_ARG
    with pytest.raises(VPError):
        plan.kernel_entries(off[:1], "Tj", 5)
    with pytest.raises(VPError):
        plan.matrix_block(torch.tensor([0, 256], dtype=torch.int64, device=DEV),
                          torch.tensor([1], dtype=torch.int64, device=DEV))
    plan.close()
