// fourstep.cu -- instantiation and launch of the four-step FP32 pencil passes
// (fourstep.cuh) for the lengths n = 2N they serve: 64, 128, 256, 512, 1024;
// the fused pass of 2N = 512 runs on the TMA kernel.
#include <stdio.h>

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
constexpr int kShapes = 4;  // candidate tile shapes per (2N, pass kind)
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

// Candidate tile shapes of a pass for the autotuner (vp_plan_autotune): the
// table's choice first, then its neighbours in pencils per CTA (W / 2, 2 W),
// staging depth, and the exchange aliased with the staging slot or not
// (where P = 2Q).  Shapes above the shared memory a CTA may use are skipped.
struct Shape {
  int W, NSTG;
  bool ALIAS;
};
template <int n, bool CONTIG, int MODE>
constexpr Shape shape_of(int i) {
  constexpr int P = fs::fs_P(n), Q = n / P;
  constexpr int W0 = pick_W(n, CONTIG, MODE), NS0 = pick_NSTG(CONTIG, MODE);
  constexpr bool A0 = pick_ALIAS(n, CONTIG, MODE), two = (P == 2 * Q);
  if (CONTIG) {
    const Shape c[kShapes] = {{W0, NS0, false}, {W0 > 2 ? W0 / 2 : 4, NS0, false},
                              {W0 * Q < 512 ? 2 * W0 : W0 / 2, NS0, false}, {W0, NS0 == 3 ? 2 : 3, false}};
    return c[i];
  }
  constexpr int Walt = W0 == 16 ? 8 : 16;
  if (MODE == MODE_FWD) {
    const Shape c[kShapes] = {{W0, NS0, A0}, {W0, 3, A0}, {Walt, NS0, A0}, {W0, two ? NS0 : 2, two ? !A0 : A0}};
    return c[i];
  }
  if (MODE == MODE_INV) {
    const Shape c[kShapes] = {{W0, NS0, false}, {Walt, NS0, false}, {W0, 3, false}, {W0, 4, false}};
    return c[i];
  }
  const Shape c[kShapes] = {{W0, 2, false}, {Walt, 2, false}, {W0, 3, false}, {W0, 2, two}};  // fused
  return c[i];
}

template <int n, bool CONTIG, int MODE, int I>
constexpr bool shape_fits() {
  constexpr Shape sh = shape_of<n, CONTIG, MODE>(I);
  using K = fs::Cfg<n, CONTIG, MODE, sh.W, sh.NSTG, sh.ALIAS>;
  return K::smem <= 227 * 1024 && K::threads <= 1024;
}

template <int n, bool CONTIG, int MODE, int I>
cudaError_t launch_shape(const PassArgs<float>& a, cudaStream_t s) {
  constexpr Shape sh = shape_of<n, CONTIG, MODE>(I);
  using K = fs::Cfg<n, CONTIG, MODE, sh.W, sh.NSTG, sh.ALIAS>;
  if constexpr (shape_fits<n, CONTIG, MODE, I>())
    return fs::launch<n, CONTIG, MODE, sh.W, sh.NSTG, pick_MINB(K::smem, K::threads), sh.ALIAS>(a, s);
  else
    return cudaErrorNotSupported;
}
template <int n, bool CONTIG, int MODE>
cudaError_t launch_cfg(const PassArgs<float>& a, cudaStream_t s) {
  switch (a.cfg) {
    case 1: return launch_shape<n, CONTIG, MODE, 1>(a, s);
    case 2: return launch_shape<n, CONTIG, MODE, 2>(a, s);
    case 3: return launch_shape<n, CONTIG, MODE, 3>(a, s);
    default: return launch_shape<n, CONTIG, MODE, 0>(a, s);
  }
}

template <int n>
cudaError_t launch_len(PassKind kind, const PassArgs<float>& a, cudaStream_t s) {
  switch (kind) {
    case FWD_CONTIG: return launch_cfg<n, true, MODE_FWD>(a, s);
    case FWD_STRIDED: return launch_cfg<n, false, MODE_FWD>(a, s);
    case INV_CONTIG: return launch_cfg<n, true, MODE_INV>(a, s);
    case INV_STRIDED: return launch_cfg<n, false, MODE_INV>(a, s);
    case FUSED_STRIDED:
      // candidate 0 of 2N = 512 is the TMA kernel where it applies
      if (n == 512 && a.cfg == 0 && fs::tma_fused_usable(n, a)) return fs::launch_tma_fused<16, 1>(a, s);
      return launch_cfg<n, false, MODE_FUSED1>(a, s);
  }
  return cudaErrorInvalidValue;
}

template <int n, bool CONTIG, int MODE>
void fill_shapes(bool* fits, Shape* sh) {
  fits[0] = shape_fits<n, CONTIG, MODE, 0>();
  fits[1] = shape_fits<n, CONTIG, MODE, 1>();
  fits[2] = shape_fits<n, CONTIG, MODE, 2>();
  fits[3] = shape_fits<n, CONTIG, MODE, 3>();
  for (int i = 0; i < kShapes; ++i) sh[i] = shape_of<n, CONTIG, MODE>(i);
}
template <int n>
void shapes_len(PassKind kind, bool* fits, Shape* sh) {
  switch (kind) {
    case FWD_CONTIG: fill_shapes<n, true, MODE_FWD>(fits, sh); break;
    case FWD_STRIDED: fill_shapes<n, false, MODE_FWD>(fits, sh); break;
    case INV_CONTIG: fill_shapes<n, true, MODE_INV>(fits, sh); break;
    case INV_STRIDED: fill_shapes<n, false, MODE_INV>(fits, sh); break;
    case FUSED_STRIDED: fill_shapes<n, false, MODE_FUSED1>(fits, sh); break;
  }
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

bool fourstep_serves(PassKind kind, int n, const PassArgs<float>& a) {
  const bool contig = (kind == FWD_CONTIG || kind == INV_CONTIG);
  const int mode = kind == FUSED_STRIDED ? (a.nfields == 1 ? MODE_FUSED1 : MODE_FUSEDN)
                   : (kind == FWD_CONTIG || kind == FWD_STRIDED) ? MODE_FWD
                                                                  : MODE_INV;
  return fs::usable(n, mode, contig, a);
}

int fourstep_shapes(PassKind kind, int n, char (*names)[32], bool* fits) {
  Shape sh[kShapes];
  switch (n) {
    case 64: shapes_len<64>(kind, fits, sh); break;
    case 128: shapes_len<128>(kind, fits, sh); break;
    case 256: shapes_len<256>(kind, fits, sh); break;
    case 512: shapes_len<512>(kind, fits, sh); break;
    case 1024: shapes_len<1024>(kind, fits, sh); break;
    default: return 0;
  }
  for (int i = 0; i < kShapes; ++i) {
    if (n == 512 && kind == FUSED_STRIDED && i == 0)
      snprintf(names[i], 32, "tma W16 S2");
    else
      snprintf(names[i], 32, "W%d S%d%s", sh[i].W, sh[i].NSTG, sh[i].ALIAS ? " alias" : "");
  }
  return kShapes;
}

}  // namespace vp
