// apply_dispatch.cuh -- instantiation and launch of the pencil passes for the
// built FFT lengths.  Included by one translation unit per precision.
#pragma once

#include "vp_internal.cuh"

namespace vp {

template <typename Real, int n, bool CONTIG, int MODE, typename Cfg = PassCfg<Real, n, CONTIG, MODE>>
cudaError_t launch_one(const PassArgs<Real>& a0, cudaStream_t s) {
  // per device: shared-memory opt-in and the persistent grid (SMs x resident CTAs)
  static int grid_cap[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!grid_cap[dev]) {
    auto kern = pencil_pass<Real, n, CONTIG, MODE, Cfg>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::smem);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, Cfg::threads, Cfg::smem);
    if (e != cudaSuccess) return e;
    grid_cap[dev] = sms * (per_sm > 0 ? per_sm : 1);
  }
  PassArgs<Real> a = a0;
  long long tiles;
  if (CONTIG) {
    a.nblk_i = 1;
    tiles = (a.O + Cfg::W - 1) / Cfg::W;
  } else {
    a.nblk_i = (a.I + Cfg::W - 1) / Cfg::W;
    tiles = (long long)a.O * a.nblk_i;
  }
  if (tiles <= 0) return cudaSuccess;
  const long long grid = tiles < grid_cap[dev] ? tiles : grid_cap[dev];
  pencil_pass<Real, n, CONTIG, MODE, Cfg><<<(unsigned)grid, Cfg::threads, Cfg::smem, s>>>(a);
  return cudaGetLastError();
}

template <typename Real, int n>
cudaError_t launch_n(PassKind kind, const PassArgs<Real>& a, cudaStream_t s) {
  switch (kind) {
    case FWD_CONTIG: return launch_one<Real, n, true, MODE_FWD>(a, s);
    case FWD_STRIDED: return launch_one<Real, n, false, MODE_FWD>(a, s);
    case INV_CONTIG: return launch_one<Real, n, true, MODE_INV>(a, s);
    case INV_STRIDED: return launch_one<Real, n, false, MODE_INV>(a, s);
    case FUSED_STRIDED:
      return a.nfields == 1 ? launch_one<Real, n, false, MODE_FUSED1>(a, s)
                            : launch_one<Real, n, false, MODE_FUSEDN>(a, s);
  }
  return cudaErrorInvalidValue;
}

template <typename Real, int n>
bool shape_n(PassKind kind, PassShape* out) {
  const bool contig = (kind == FWD_CONTIG || kind == INV_CONTIG);
  out->W = contig ? PassCfg<Real, n, true, MODE_FWD>::W : PassCfg<Real, n, false, MODE_FWD>::W;
  out->threads = contig ? PassCfg<Real, n, true, MODE_FWD>::threads : PassCfg<Real, n, false, MODE_FWD>::threads;
  out->smem = contig ? PassCfg<Real, n, true, MODE_FWD>::smem : PassCfg<Real, n, false, MODE_FWD>::smem;
  return true;
}

}  // namespace vp

// The built FFT lengths 2N (N = n/2 even): powers of two and 3 x powers of two.
#define VP_FOR_EACH_LENGTH(X) \
  X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768) X(1024) X(1536) X(2048) X(4096)
