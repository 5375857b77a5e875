// fourstep.cu -- instantiation and launch of the four-step FP32 pencil passes
// (fourstep.cuh) for the lengths n = 2N they serve: 64, 128, 256, 512, 1024;
// the fused pass of 2N = 512 runs on the TMA kernel.
#include "fourstep.cuh"
#include "vp_internal.cuh"

namespace vp {
namespace {

// Launch configuration per pass (measured on 2N = 512, GB300):
//   rows (contiguous): 128 threads' worth of pencils (W = 128 / Q), input
//     staged 3 tiles ahead for the forward and 2 for the inverse;
//   strided forward: W = 8, 4-deep staging, the exchange in the tile's own
//     staging slot (two rounds of P/2 columns when P = 2Q);
//   strided inverse: W = 8 (16 for Q = 8), 2-deep staging, separate buffer;
//   fused: the TMA kernel for 2N = 512, else W = 16 (8 for Q = 32).
// Measured and dropped: W = 4 (too few pencils per row segment), W = 16 for
// the strided single transforms, an aliased exchange for the inverse and the
// fused passes, more CTAs per SM at a 128-register cap for the fused pass.
constexpr int clampi(int x, int lo, int hi) { return x < lo ? lo : (x > hi ? hi : x); }
constexpr int pick_W(int n, bool contig, int mode) {
  const int Q = n / fs::fs_P(n);
  if (contig) return clampi(128 / Q, 2, 16);
  return clampi((mode == MODE_FUSED1 ? 256 : 128) / Q, 8, 16);
}
constexpr int pick_NSTG(bool contig, int mode) {
  return mode == MODE_FWD ? (contig ? 3 : 4) : 2;
}
constexpr bool pick_ALIAS(int n, bool contig, int mode) {
  return !contig && mode == MODE_FWD && fs::fs_P(n) == 2 * (n / fs::fs_P(n));
}
// CTAs per SM the registers must allow: as many as shared memory admits, at
// most enough for 128 registers per thread.
constexpr int pick_MINB(size_t smem, int threads) {
  const int by_smem = (int)(233472 / (smem + 1024));
  const int by_regs = 65536 / (threads * 128);
  const int m = by_smem < by_regs ? by_smem : by_regs;
  return m < 1 ? 1 : m;
}

template <int n, bool CONTIG, int MODE>
cudaError_t launch_cfg(const PassArgs<float>& a, cudaStream_t s) {
  constexpr int W = pick_W(n, CONTIG, MODE);
  constexpr bool ALIAS = pick_ALIAS(n, CONTIG, MODE);
  constexpr int NSTG = pick_NSTG(CONTIG, MODE);
  using K = fs::Cfg<n, CONTIG, MODE, W, NSTG, ALIAS>;
  static_assert(K::smem <= 227 * 1024, "shared memory");
  return fs::launch<n, CONTIG, MODE, W, NSTG, pick_MINB(K::smem, K::threads), ALIAS>(a, s);
}

template <int n>
cudaError_t launch_len(PassKind kind, const PassArgs<float>& a, cudaStream_t s) {
  switch (kind) {
    case FWD_CONTIG: return launch_cfg<n, true, MODE_FWD>(a, s);
    case FWD_STRIDED: return launch_cfg<n, false, MODE_FWD>(a, s);
    case INV_CONTIG: return launch_cfg<n, true, MODE_INV>(a, s);
    case INV_STRIDED: return launch_cfg<n, false, MODE_INV>(a, s);
    case FUSED_STRIDED:
      if (n == 512 && fs::tma_fused_usable(n, a)) return fs::launch_tma_fused<16, 1>(a, s);
      return launch_cfg<n, false, MODE_FUSED1>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

bool launch_fourstep(PassKind kind, int n, const PassArgs<float>& a, cudaStream_t s, cudaError_t* err) {
  const bool contig = (kind == FWD_CONTIG || kind == INV_CONTIG);
  const int mode = kind == FUSED_STRIDED ? (a.nfields == 1 ? MODE_FUSED1 : MODE_FUSEDN)
                   : (kind == FWD_CONTIG || kind == FWD_STRIDED) ? MODE_FWD
                                                                  : MODE_INV;
  if (!fs::usable(n, mode, contig, a)) return false;
  switch (n) {
    case 64: *err = launch_len<64>(kind, a, s); return true;
    case 128: *err = launch_len<128>(kind, a, s); return true;
    case 256: *err = launch_len<256>(kind, a, s); return true;
    case 512: *err = launch_len<512>(kind, a, s); return true;
    case 1024: *err = launch_len<1024>(kind, a, s); return true;
  }
  return false;
}

}  // namespace vp
