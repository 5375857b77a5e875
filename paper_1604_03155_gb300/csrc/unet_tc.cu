// unet_tc.cu -- the U-Net's 3x3x3 convolutions as implicit GEMMs on the
// tensor cores (tcgen05.mma kind::f16, BF16 operands, FP32 accumulation).
//
// For an output row segment of 128 voxels (x0 .. x0 + 127 of row (z, y)):
//
//   y[co](x) = b[co] + sum_{tap (kz, ky, kx)} sum_ci w[co][ci][tap] in[ci](z + kz - 1, y + ky - 1, x + kx - 1)
//
// is D (128 x N) = sum over the 27 taps and the 16-channel chunks of
// A_tap (128 voxels x 16 channels) * B_tap (16 channels x N output channels):
// M = 128 voxels (one tensor-memory lane each), N = 16 output channels
// (padded), K = 16 input channels per instruction.  A CTA has 256 threads:
// thread t stages the channel group t / 128 of voxel t mod 128, and in the
// epilogue warp w reads lanes 32 (w mod 4) .. + 31 and output channels
// 8 (w / 4) .. + 7.  The
// weights are BF16 values already (the network rounds its master weights to
// BF16), so B is exact; every FP32 activation is split into two BF16 parts,
// a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi), and both parts
// are multiplied by B into the same FP32 accumulator: the products are exact
// and the split leaves a relative residual below 2^-16, so the convolution
// keeps the FP32 network's arithmetic up to that rounding level.
//
// Shared-memory operands (the tensor core's canonical K-major layout without
// swizzle, 8 x 16-byte core matrices):
//   an input row (z', y') of the segment is staged as planes [part][group]
//   of 130 slots (voxels x0 - 1 .. x0 + 128, the two ends being the zero
//   padding or the neighbouring segment) x 8 channels (16 bytes per slot);
//   in a plane, voxel m of the segment sits at slot m + 1, so the operand of
//   tap kx starts kx slots (16 kx bytes) into the plane and its 8-row groups
//   are 128 bytes apart: the x shift of a tap is a descriptor offset, with no
//   copy.  Channel groups 2c and 2c + 1 (one K = 16 chunk) are one plane apart.
//   B per (tap, chunk): N x 16 BF16, row groups 256 bytes apart.
// A CTA takes work items of YB consecutive output rows of one (z, segment)
// and keeps the input rows of its last y values in a ring of 4 y slots x 3 z
// values, so each new output row stages three input rows (all their loads in
// flight at once); the MMAs of row y run while the CTA stores row y - 1's
// results and stages the input rows of row y + 2, and two accumulators in
// tensor memory alternate.  One launch covers up to 16 input and 16 output
// channels (two CTAs per SM); wider layers run as blocks of 16 output
// channels, and a 32-channel input (the skip concatenation) as two passes
// whose second adds its sums to the first's and then applies the activation.
// The MMA-completion waits are bounded by a clock budget; a timeout sets the
// caller's error word and the CTA stops.
#include <cuda_bf16.h>
#include <stdint.h>

#include "vp_internal.cuh"

namespace vp {
namespace unet_tc {
namespace {

constexpr int kThreads = 256;            // a voxel of the segment (tensor-memory lane) x a channel group
constexpr int kSeg = 128;                // voxels per row segment: the MMA's M
constexpr int kPlane = (kSeg + 2) * 16;  // bytes of one plane: 130 slots x 8 BF16 channels
constexpr int kYB = 8;                   // output rows per work item
constexpr int kYS = 4;                   // y slots of the input ring
constexpr int kG = 2;                    // 8-channel groups of an input block (16 channels, one K = 16 chunk)
constexpr int kN = 16;                   // output channels of a block (accumulator columns)
constexpr uint32_t kTmemCols = 64;       // two accumulators
constexpr size_t kBBytes = (size_t)27 * kN * 32;        // B of every tap: N x 16 BF16
constexpr size_t kRowBytes = (size_t)2 * kG * kPlane;   // one staged input row, both parts
constexpr size_t kOffA = kBBytes;
constexpr size_t kABytes = (size_t)kYS * 3 * kRowBytes;
constexpr size_t kOffBar = kOffA + kABytes;             // mbarrier, tensor-memory slot, stop flag
constexpr size_t kSmem = kOffBar + 16;
static_assert(kBBytes % 16 == 0 && kRowBytes % 16 == 0, "16-byte aligned operands");
static_assert(2 * (kSmem + 1024) <= 233472, "two CTAs per SM");

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: canonical layout without swizzle
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor: D FP32, A and B BF16 (both K-major), M = 128, N = n
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d_tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}
__device__ __forceinline__ bool wait(uint32_t mbar, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}
// generic-proxy shared stores and earlier tensor-memory loads ordered before
// the MMAs issued after this CTA barrier
__device__ __forceinline__ void sync_for_mma() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 8 consecutive FP32 columns of this warp's 32 lanes
__device__ __forceinline__ void tload8(uint32_t addr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(addr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
// two BF16 parts of a pair of values, one 32-bit word each (first value low)
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

// One launch: input block x (c <= 16 channels) against the weights of output
// channels co0 .. co0 + nco - 1 (nco <= 16) and input channels ci0 .. ci0 + c - 1
// of w[co][w_ci][27]; y[co0 + co] = (accumulate ? y : bias) + conv, then the
// activation when act.
struct BlockArgs {
  const float* x;
  int c;
  const float* w;
  int w_ci, ci0, co0, nco;
  const float* bias;
  float* y;
  int S, accumulate, act;
  float slope;
  int* err;
  long long wait_cycles;
  int withhold;
};

}  // namespace

__global__ void __launch_bounds__(kThreads) k_conv3d_tc(const BlockArgs a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int vx = tid & (kSeg - 1), grp = tid >> 7;  // staged voxel and channel group
  const int S = a.S;
  const long long S3 = (long long)S * S * S;
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + kOffBar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kOffBar + 8);
  int* s_stop = reinterpret_cast<int*>(smem + kOffBar + 12);

  // B: w[co0 + n][ci0 + k][tap] as BF16 (exact: the weights are BF16 values), zero padded
  for (int i = tid; i < 27 * kN * 16; i += kThreads) {
    const int k = i & 15, n = (i >> 4) % kN, t = i / (16 * kN);
    const float v = (n < a.nco && k < a.c) ? a.w[((long long)(a.co0 + n) * a.w_ci + a.ci0 + k) * 27 + t] : 0.f;
    const size_t off = (size_t)t * kN * 32 + (size_t)((n >> 3) * 2 + (k >> 3)) * 128 + (n & 7) * 16 + (k & 7) * 2;
    *reinterpret_cast<__nv_bfloat16*>(smem + off) = __float2bfloat16_rn(v);
  }
  // the input ring starts zero: slots no staging writes (the padding) stay zero
  for (size_t i = (size_t)tid * 16; i < kABytes; i += (size_t)kThreads * 16)
    *reinterpret_cast<uint4*>(smem + kOffA + i) = make_uint4(0u, 0u, 0u, 0u);
  float bz[8];  // bias of this thread's epilogue channels
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int co = 8 * (warp >> 2) + j;
    bz[j] = (a.bias && co < a.nco) ? a.bias[a.co0 + co] : 0.f;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(s_mbar)));
    *s_stop = 0;
  }
  sync_for_mma();
  const uint32_t tmem = *s_tmem;
  const uint32_t lane_base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + 8 * (warp >> 2);
  const uint32_t mbar = su32(s_mbar);
  const uint64_t b_desc0 = sdesc(su32(smem), 128, 256), a_desc0 = sdesc(su32(smem + kOffA), kPlane, 128);
  const uint32_t idesc = idesc_bf16(kN);
  uint32_t phase = 0;
  bool ok = true;

  const int nseg = (S + kSeg - 1) / kSeg, nyb = (S + kYB - 1) / kYB;
  const long long items = (long long)S * nyb * nseg;
  for (long long item = blockIdx.x; item < items; item += gridDim.x) {
    const int seg = (int)(item % nseg);
    const long long rest = item / nseg;
    const int yb = (int)(rest % nyb), z = (int)(rest / nyb);
    const int x0 = seg * kSeg, y0 = yb * kYB, y1 = y0 + kYB < S ? y0 + kYB : S;

    // input row yy of the three z values into ring slot yy mod 4: thread
    // (vx, grp) writes channel group grp of slot vx + 1 (voxel x0 + vx); the
    // threads of voxels 0 and 1 also the two end slots when the segment has a
    // neighbour there.  All loads of a slot are issued before any is converted.
    auto stage = [&](int yy) {
      unsigned char* row0 = smem + kOffA + (size_t)((yy + kYS) % kYS) * 3 * kRowBytes;
      const int nslots = (nseg > 1 && vx < 2) ? 2 : 1;
#pragma unroll 1
      for (int e = 0; e < nslots; ++e) {
        const int slot = e == 0 ? vx + 1 : (vx == 0 ? 0 : kSeg + 1);
        const int x = e == 0 ? x0 + vx : (vx == 0 ? x0 - 1 : x0 + kSeg);
        float v[3][8];
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
          const int zz = z + dz - 1;
          const bool in = zz >= 0 && zz < S && yy >= 0 && yy < S && x >= 0 && x < S;
          const float* src = a.x + (long long)(8 * grp) * S3 + ((long long)zz * S + yy) * S + x;
#pragma unroll
          for (int j = 0; j < 8; ++j) v[dz][j] = (in && 8 * grp + j < a.c) ? __ldg(src + j * S3) : 0.f;
        }
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
          unsigned char* row = row0 + (size_t)dz * kRowBytes;
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) split2(v[dz][2 * j], v[dz][2 * j + 1], hi[j], lo[j]);
          *reinterpret_cast<uint4*>(row + (size_t)grp * kPlane + slot * 16) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
          *reinterpret_cast<uint4*>(row + (size_t)(kG + grp) * kPlane + slot * 16) =
              make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
      }
    };
    // the 27 taps x 2 parts of output row y into accumulator buf; a
    // descriptor's address field (bits 0-13, address / 16) takes the operand
    // offsets as plain additions (shared addresses stay below 256 KB)
    auto issue = [&](int y, int buf) {
#pragma unroll
      for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
          const int ys = (y + ky - 1 + kYS) % kYS;
          const uint64_t rd = a_desc0 + (uint64_t)(((ys * 3 + kz) * kRowBytes) >> 4);
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            const int t = (kz * 3 + ky) * 3 + kx;
            const uint64_t bd = b_desc0 + (uint64_t)((t * kN * 32) >> 4);
#pragma unroll
            for (int p = 0; p < 2; ++p)
              mma(tmem + 32 * buf, rd + (uint64_t)((p * kG * kPlane + kx * 16) >> 4), bd, idesc,
                  (t > 0 || p > 0) ? 1u : 0u);
          }
        }
      commit(mbar);
    };
    // output channels 8 (warp / 4) .. + 7 of lane (voxel) 32 (warp mod 4) + lane;
    // an accumulating pass reads the partial sums of row y one iteration early
    const int ex = x0 + (warp & 3) * 32 + (tid & 31), ec0 = 8 * (warp >> 2);
    float pre[8];
    auto prefetch = [&](int y) {
      if (!a.accumulate || ex >= S) return;
      const float* dst = a.y + (long long)(a.co0 + ec0) * S3 + ((long long)z * S + y) * S + ex;
#pragma unroll
      for (int j = 0; j < 8; ++j) pre[j] = ec0 + j < a.nco ? dst[j * S3] : 0.f;
    };
    auto epilogue = [&](int y, int buf) {
      float v[8];
      tload8(lane_base + 32 * buf, v);
      if (ex < S) {
        float* dst = a.y + (long long)(a.co0 + ec0) * S3 + ((long long)z * S + y) * S + ex;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (ec0 + j < a.nco) {
            float r = v[j] + (a.accumulate ? pre[j] : bz[j]);
            if (a.act) r = r > 0.f ? r : a.slope * r;
            dst[j * S3] = r;
          }
        }
      }
    };

    stage(y0 - 1);
    stage(y0);
    stage(y0 + 1);
    for (int y = y0; y < y1; ++y) {
      sync_for_mma();  // rows up to y + 1 staged; the previous epilogue's loads done
      if (*s_stop) break;
      if (tid == 0 && !a.withhold) issue(y, (y - y0) & 1);
      if (y > y0) epilogue(y - 1, (y - 1 - y0) & 1);
      prefetch(y);
      // the slot of row y + 2 held row y - 2, whose last reader, row y - 1's MMAs, is done
      if (y + 2 <= y1) stage(y + 2);
      ok = wait(mbar, phase, a.wait_cycles) && ok;
      phase ^= 1;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (!ok) *s_stop = 1;
    }
    __syncthreads();
    if (*s_stop) break;
    epilogue(y1 - 1, (y1 - 1 - y0) & 1);
  }
  if (tid == 0 && *s_stop && a.err) atomicOr(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

namespace {
cudaError_t launch(const BlockArgs& a, cudaStream_t s) {
  static int grid_cap[64] = {0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev >= 64) return cudaErrorInvalidDevice;
  if (!grid_cap[dev]) {
    e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
    if (e != cudaSuccess) return e;
    // the occupancy below counts the carveout: ask for all of it for shared memory
    e = cudaFuncSetAttribute(k_conv3d_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_conv3d_tc, kThreads, kSmem);
    if (e != cudaSuccess) return e;
    // the residency registers and shared memory allow, when the query reports
    // less (CTAs never wait on one another, so a larger grid only queues)
    cudaFuncAttributes fa;
    int smem_sm = 0;
    if (cudaFuncGetAttributes(&fa, k_conv3d_tc) == cudaSuccess &&
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) == cudaSuccess) {
      const int regs = ((fa.numRegs > 0 ? fa.numRegs : 1) + 7) / 8 * 8;
      const int by_regs = 65536 / (kThreads * regs);
      const int by_smem = smem_sm / (int)(kSmem + 1024);
      const int est = by_regs < by_smem ? by_regs : by_smem;
      if (est > per_sm) per_sm = est;
    }
    if (per_sm > 8) per_sm = 8;  // tensor memory: 64 columns of 512 per CTA
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    grid_cap[dev] = sms * per_sm;
  }
  const long long items = (long long)a.S * ((a.S + kYB - 1) / kYB) * ((a.S + kSeg - 1) / kSeg);
  if (items <= 0) return cudaSuccess;
  const int grid = items < grid_cap[dev] ? (int)items : grid_cap[dev];
  k_conv3d_tc<<<grid, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}
}  // namespace

// Blocks of 16 output channels; the input (x1, then x2 when c2 > 0) in
// blocks of up to 16 channels, the second accumulating onto the first.
cudaError_t conv3d(const ConvArgs& a, cudaStream_t s) {
  const int Ci = a.c1 + a.c2;
  if (a.c1 < 1 || a.c1 > 16 || a.c2 < 0 || a.c2 > 16 || (a.c2 > 0 && !a.x2) || a.co < 1 || a.S < 1)
    return cudaErrorInvalidValue;
  for (int co0 = 0; co0 < a.co; co0 += kN) {
    BlockArgs b;
    b.w = a.w;
    b.w_ci = Ci;
    b.co0 = co0;
    b.nco = a.co - co0 < kN ? a.co - co0 : kN;
    b.y = a.y;
    b.S = a.S;
    b.slope = a.slope;
    b.err = a.err;
    b.wait_cycles = a.wait_cycles;
    b.withhold = a.withhold;
    b.x = a.x1;
    b.c = a.c1;
    b.ci0 = 0;
    b.bias = a.bias;
    b.accumulate = 0;
    b.act = a.c2 > 0 ? 0 : a.act;
    cudaError_t e = launch(b, s);
    if (e != cudaSuccess) return e;
    if (a.c2 > 0) {
      b.x = a.x2;
      b.c = a.c2;
      b.ci0 = a.c1;
      b.bias = nullptr;
      b.accumulate = 1;
      b.act = a.act;
      e = launch(b, s);
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Weight gradients on the tensor cores:
//   dW[co][ci][(kz, ky, kx)] = sum_v dy[co](v) x[ci](v + (kz - 1, ky - 1, kx - 1)),
//   db[co] = sum_v dy[co](v)
// per output row segment (K = its 128 voxels) as D[(input row r, ci)][co] +=
// A * B with A the nine input rows r = 3 kz + ky staged as the convolution
// stages them, read MN-major (a voxel's 16 bytes of 8 channels are one K row
// of a core matrix; channel groups, and then rows, one plane apart, so
// M = (r, ci)), the tap kx a 16-byte K offset; B the segment's dy (K-major,
// N = 16 output channels).  Rows 0-7 take one M = 128 chain and row 8 a second
// one whose window starts at row 1 (its rows 1-7 are not used), three of each
// for kx, six accumulators of 16 columns in tensor memory.  Both operands are
// split into BF16 hi and lo parts and the products hi hi, lo hi, hi lo are
// accumulated (relative residual about 2^-16).  Each CTA sums over its rows
// and writes one partial per CTA in the layout k_wreduce reduces in FP64:
// part[blk][(ci * 27 + tap) * co_n + co], the bias at part[blk][Ci * 27 * co_n + co].
// ---------------------------------------------------------------------------
namespace {
constexpr int kWgThreads = 256;  // a voxel x a channel group in the staging
constexpr size_t kWgB = (size_t)16 * 128 * 2;          // one part of B: 16 co x 128 voxels, BF16
constexpr size_t kWgX = (size_t)9 * kG * kPlane;       // one part of the nine staged input rows
constexpr size_t kWgOffX = 2 * kWgB;
constexpr size_t kWgOffBar = kWgOffX + 2 * kWgX;
constexpr size_t kWgSmem = kWgOffBar + 16;
constexpr uint32_t kWgTmemCols = 128;                   // 6 accumulators of 16 columns
static_assert(2 * (kWgSmem + 1024) <= 233472, "two CTAs per SM");

struct WgBlock {
  const float* x;  // input block: c channels, [c][S^3]
  int c, ci0;      // its channels and their first index in the layer's input
  const float* dy;
  int co;          // output channels of the layer (<= 16)
  float* part;
  int Ci;          // the layer's input channels (partial layout)
  int S, bias;     // bias: write the bias partials (first block only)
  int* err;
  long long wait_cycles;
  int withhold;
};
}  // namespace

__global__ void __launch_bounds__(kWgThreads) k_wgrad_tc(const WgBlock a) {
  extern __shared__ __align__(1024) unsigned char smem[];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int vx = tid & (kSeg - 1), grp = tid >> 7;  // staged voxel and channel group
  const int S = a.S;
  const long long S3 = (long long)S * S * S;
  unsigned char* sB = smem;             // [part][co group][voxel group][8 co][8 voxels]
  unsigned char* sX = smem + kWgOffX;   // [part][row r][channel group][130 slots][8 ch]
  uint64_t* s_mbar = reinterpret_cast<uint64_t*>(smem + kWgOffBar);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + kWgOffBar + 8);
  int* s_stop = reinterpret_cast<int*>(smem + kWgOffBar + 12);
  for (size_t i = (size_t)tid * 16; i < 2 * kWgX; i += (size_t)kWgThreads * 16)
    *reinterpret_cast<uint4*>(sX + i) = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(s_tmem)),
                 "r"(kWgTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(s_mbar)));
    *s_stop = 0;
  }
  sync_for_mma();
  const uint32_t tmem = *s_tmem;
  const uint32_t mbar = su32(s_mbar);
  // A MN-major (bit 15), B K-major; descriptors: A (K stride 128 B, M stride a
  // plane), B (K stride 128 B, N stride 2048 B)
  const uint32_t idesc = idesc_bf16(16) | (1u << 15);
  const uint64_t ad0 = sdesc(su32(sX), 128, kPlane), bd0 = sdesc(su32(sB), 128, 2048);
  uint32_t phase = 0;
  bool ok = true, any = false;
  float bsum = 0.f;  // bias: this thread's output channel (tid / 8) mod 16
  const int bco = (tid >> 3) & 15, bj = tid & 7, bh = tid >> 7;

  const int nseg = (S + kSeg - 1) / kSeg;
  const long long rows = (long long)S * S * nseg;
  for (long long row = blockIdx.x; row < rows; row += gridDim.x) {
    const int seg = (int)(row % nseg);
    const long long r2 = row / nseg;
    const int y = (int)(r2 % S), z = (int)(r2 / S), x0 = seg * kSeg;
    // the nine input rows (z + kz - 1, y + ky - 1), r = 3 kz + ky: thread
    // (vx, grp) writes channel group grp of slot vx + 1, all 72 loads in flight;
    // the threads of voxels 0 and 1 also the end slots of an inner segment
    const int nslots = (nseg > 1 && vx < 2) ? 2 : 1;
#pragma unroll 1
    for (int e = 0; e < nslots; ++e) {
      const int slot = e == 0 ? vx + 1 : (vx == 0 ? 0 : kSeg + 1);
      const int x = e == 0 ? x0 + vx : (vx == 0 ? x0 - 1 : x0 + kSeg);
      float v[9][8];
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        const int zz = z + r / 3 - 1, yy = y + r % 3 - 1;
        const bool in = zz >= 0 && zz < S && yy >= 0 && yy < S && x >= 0 && x < S;
        const float* src = a.x + (long long)(8 * grp) * S3 + ((long long)zz * S + yy) * S + x;
#pragma unroll
        for (int j = 0; j < 8; ++j) v[r][j] = (in && 8 * grp + j < a.c) ? __ldg(src + j * S3) : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 9; ++r) {
        uint32_t hi[4], lo[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) split2(v[r][2 * j], v[r][2 * j + 1], hi[j], lo[j]);
        const size_t off = ((size_t)r * kG + grp) * kPlane + slot * 16;
        *reinterpret_cast<uint4*>(sX + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
        *reinterpret_cast<uint4*>(sX + kWgX + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
      }
    }
    // dy of the segment: thread (co = (tid / 8) mod 16, voxel group tid mod 8 + 8 (tid / 128))
    {
      const int vg = bj + 8 * bh, xs = x0 + 8 * vg;
      float v[8];
      const float* src = a.dy + (long long)bco * S3 + ((long long)z * S + y) * S + xs;
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = (bco < a.co && xs + j < S) ? __ldg(src + j) : 0.f;
#pragma unroll
      for (int j = 0; j < 8; ++j) bsum += v[j];
      uint32_t hi[4], lo[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) split2(v[2 * j], v[2 * j + 1], hi[j], lo[j]);
      const size_t off = ((size_t)(bco >> 3) * 16 + vg) * 128 + (bco & 7) * 16;
      *reinterpret_cast<uint4*>(sB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
      *reinterpret_cast<uint4*>(sB + kWgB + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
    }
    sync_for_mma();
    if (*s_stop) break;
    if (tid == 0 && !a.withhold) {
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll 1
          for (int ks = 0; ks < 8; ++ks)
#pragma unroll
            for (int pr = 0; pr < 3; ++pr) {
              const int pa = pr == 1 ? 1 : 0, pb = pr == 2 ? 1 : 0;  // hi hi, lo hi, hi lo
              const uint64_t ad = ad0 + (uint64_t)((pa * kWgX + (size_t)h * kG * kPlane + ks * 256 + kx * 16) >> 4);
              const uint64_t bd = bd0 + (uint64_t)((pb * kWgB + ks * 256) >> 4);
              mma(tmem + (uint32_t)((kx * 2 + h) * 16), ad, bd, idesc, (any || ks > 0 || pr > 0) ? 1u : 0u);
            }
      commit(mbar);
    }
    ok = wait(mbar, phase, a.wait_cycles) && ok;
    phase ^= 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    any = true;
    if (!ok) *s_stop = 1;
    __syncthreads();  // the operands are free for the next row
  }
  // partials of this CTA: D lane L of accumulator (kx, h) is row r = h + L / 16
  // (chain h = 1 keeps only r = 8) and channel L mod 16; warp w reads lanes
  // 32 (w mod 4) .. + 31 and output channels 8 (w / 4) .. + 7
  float* out = a.part + (long long)blockIdx.x * ((long long)a.Ci * 27 * a.co + a.co);
  const int L = 32 * (warp & 3) + (tid & 31), c0 = 8 * (warp >> 2);
#pragma unroll
  for (int kx = 0; kx < 3; ++kx)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      float v[8];
      if (any) {
        tload8(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((kx * 2 + h) * 16 + c0), v);
      } else {
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = 0.f;
      }
      const int r = h + L / 16, ci = L & 15;
      if ((h == 0 || r == 8) && ci < a.c) {
        const int t = 3 * r + kx;
#pragma unroll
        for (int j = 0; j < 8; ++j)
          if (c0 + j < a.co) out[((long long)(a.ci0 + ci) * 27 + t) * a.co + c0 + j] = v[j];
      }
    }
  if (a.bias) {
    // the two halves of the CTA hold the voxel groups 0-7 and 8-15 of each channel
    bsum += __shfl_xor_sync(0xffffffffu, bsum, 1);
    bsum += __shfl_xor_sync(0xffffffffu, bsum, 2);
    bsum += __shfl_xor_sync(0xffffffffu, bsum, 4);
    float* s_b = reinterpret_cast<float*>(sB);  // the operands are no longer read
    __syncthreads();
    if (bj == 0 && bh == 1) s_b[bco] = bsum;
    __syncthreads();
    if (bj == 0 && bh == 0 && bco < a.co) out[(long long)a.Ci * 27 * a.co + bco] = bsum + s_b[bco];
  }
  if (tid == 0 && *s_stop && a.err) atomicOr(a.err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWgTmemCols));
}

// Per-CTA partials of the layer's weight and bias gradients for nblk CTAs:
// part[blk][(ci * 27 + tap) * co + co'] and part[blk][Ci * 27 * co + co'].
cudaError_t wgrad3d(const WgradArgs& a, cudaStream_t s) {
  const int Ci = a.c1 + a.c2;
  if (a.c1 < 1 || a.c1 > 16 || a.c2 < 0 || a.c2 > 16 || (a.c2 > 0 && !a.x2) || a.co < 1 || a.co > 16 || a.S < 1 ||
      a.nblk < 1)
    return cudaErrorInvalidValue;
  static bool attr[64] = {false};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  if (!attr[dev]) {
    e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    attr[dev] = true;
  }
  WgBlock b;
  b.dy = a.dy;
  b.co = a.co;
  b.part = a.part;
  b.Ci = Ci;
  b.S = a.S;
  b.err = a.err;
  b.wait_cycles = a.wait_cycles;
  b.withhold = a.withhold;
  b.x = a.x1;
  b.c = a.c1;
  b.ci0 = 0;
  b.bias = 1;
  k_wgrad_tc<<<a.nblk, kWgThreads, kWgSmem, s>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess || a.c2 == 0) return e;
  b.x = a.x2;
  b.c = a.c2;
  b.ci0 = a.c1;
  b.bias = 0;
  k_wgrad_tc<<<a.nblk, kWgThreads, kWgSmem, s>>>(b);
  return cudaGetLastError();
}

// CTAs a layer's weight gradient uses: one output row segment or more each.
long long wgrad_rows(int S) { return (long long)S * S * ((S + kSeg - 1) / kSeg); }

}  // namespace unet_tc
}  // namespace vp
