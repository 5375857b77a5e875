// vp_capi.cu -- the C ABI declared in include/vp.h: plan lifecycle, the FP64
// precompute driver (Sections 2 and 4) and the pass sequence of the apply
// (Section 4: pad, FFT, multiply, inverse FFT, crop; Section 3 gradients).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "../../include/vp.h"
#include "vp_internal.cuh"

using namespace vp;

namespace {

thread_local std::string g_thread_error;

struct TimedLaunch {
  int pass;
  cudaEvent_t start, stop;
};

const char* kPassNames[5] = {"fwd_rows", "fwd_axis1", "fused_axis0", "inv_axis1", "inv_rows"};
enum { P_FWD_ROWS = 0, P_FWD_AX1 = 1, P_FUSED = 2, P_INV_AX1 = 3, P_INV_ROWS = 4, NPASS = 5 };

}  // namespace

struct vp_plan_s {
  int d = 0, N = 0, kernel = 0;
  // points per axis (all N for a cubic grid; axis 0 slowest); aniso: not all equal
  int Nv[3] = {0, 0, 0};
  int aniso = 0;
  double k = 0.0, L = 0.0;
  int n2 = 0;  // FFT length 2N
  int device = 0;
  cudaStream_t stream = nullptr;
  vp_precision prec = VP_FP32;
  vp_grad_mode gmode = VP_GRAD_EXACT;

  long long oct = 0;  // (N+1)^d
  // FP64 precompute results (octants, complex128)
  double2* T64 = nullptr;
  double2* G64u = nullptr;  // unscaled multiplier
  double2* G64 = nullptr;   // scaled by 1/(2N)^d
  float2* G32 = nullptr;
  double2* Tj64[3] = {nullptr, nullptr, nullptr};
  // FP32 copies of T and T_j for FP32 Nystrom entries (built on first use)
  float2* T32 = nullptr;
  float2* Tj32[3] = {nullptr, nullptr, nullptr};
  double2* Gj64u[3] = {nullptr, nullptr, nullptr};
  double2* Gj64[3] = {nullptr, nullptr, nullptr};
  float2* Gj32[3] = {nullptr, nullptr, nullptr};
  bool grad_built = false;
  double2* tw64 = nullptr;  // twiddles of axis 0 (every axis of a cubic grid)
  float2* tw32 = nullptr;
  double2* twv64[3] = {nullptr, nullptr, nullptr};  // per axis; twv[j] may alias an earlier axis's table
  float2* twv32[3] = {nullptr, nullptr, nullptr};
  // tensor-core fused pass (VP_TC_*): DFT matrices of the current split, error word
  uint16_t* tcB = nullptr;
  int tc_split = -1;
  int* d_err = nullptr;
  int* d_flag = nullptr;  // range flag of the Nystrom entry kernels

  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  size_t device_bytes = 0;

  bool timing = false;
  int host_direct = 1;  // pinned host buffers: access them in place (0: stage through device memory); set at creation
  int pass_cfg[5] = {0, 0, 0, 0, 0};  // tile shape of each FP32 four-step pass (vp_plan_autotune)
  std::vector<TimedLaunch> timed;
  std::vector<cudaEvent_t> event_pool;
  // vp_apply_pipeline (made on first use): two copy streams, kPipeSlots device
  // slots (a density and its output fields each) and per slot the events
  // "input copied", "apply done", "outputs copied"
  cudaStream_t pipe_h2d = nullptr, pipe_d2h = nullptr;
  void* pipe_buf = nullptr;
  size_t pipe_bytes = 0;
  cudaEvent_t pipe_ev[3][3] = {};
  cudaEvent_t pipe_start = nullptr;

  std::string last_error;
};

namespace {

vp_status fail(vp_plan p, vp_status st, const std::string& msg) {
  vp::log_line(1, "plan", msg);
  if (p)
    p->last_error = msg;
  else
    g_thread_error = msg;
  return st;
}

vp_status cuda_fail(vp_plan p, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(p, e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA, m);
}

#define VP_CUDA(p, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(p, e_, #call); \
  } while (0)
// makes the plan's device current until the end of the enclosing scope (the
// caller's device is restored then); a failure returns from the function
#define VP_ON_DEVICE(p, dev)                 \
  vp::DeviceGuard VP_CAT(dg_, __LINE__)(dev); \
  VP_CUDA(p, VP_CAT(dg_, __LINE__).error())

template <typename T> cudaError_t dalloc(vp_plan p, T** ptr, size_t count) {
  cudaError_t e = cudaMalloc((void**)ptr, count * sizeof(T));
  if (e == cudaSuccess) p->device_bytes += count * sizeof(T);
  return e;
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on the
// three-term recurrence of P_n (host, FP64).
void gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double z = cos(pi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int kk = 2; kk <= n; ++kk) {
        const double p2 = ((2.0 * kk - 1.0) * z * p1 - (kk - 1.0) * p0) / kk;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Separable transform chain: applies mats[a] (Q_a x P_a) along each axis a.
cudaError_t run_chain(const double2* src, double2* dst, double2* t0, double2* t1, int d, const int* dims_in,
                      double* const* mats, const int* qs, cudaStream_t s) {
  long long dims[3] = {dims_in[0], dims_in[1], d == 3 ? dims_in[2] : 1};
  const double2* cur = src;
  for (int a = 0; a < d; ++a) {
    long long O = 1, I = 1;
    for (int j = 0; j < a; ++j) O *= dims[j];
    for (int j = a + 1; j < d; ++j) I *= dims[j];
    double2* out = (a == d - 1) ? dst : ((a % 2 == 0) ? t0 : t1);
    cudaError_t e = launch_axis_transform(cur, out, mats[a], O, (int)dims[a], qs[a], I, s);
    if (e != cudaSuccess) return e;
    dims[a] = qs[a];
    cur = out;
  }
  return cudaSuccess;
}

struct Scratch {
  double2* G = nullptr;
  double2* t0 = nullptr;
  double2* t1 = nullptr;
  double2* Traw = nullptr;
  // per-axis transform matrices; an axis with the same N as an earlier one shares them
  double* C4[3] = {nullptr, nullptr, nullptr};
  double* S4[3] = {nullptr, nullptr, nullptr};
  double* C2[3] = {nullptr, nullptr, nullptr};
  double* S2[3] = {nullptr, nullptr, nullptr};
  bool own[3] = {false, false, false};
  void release() {
    cudaFree(G);
    cudaFree(t0);
    cudaFree(t1);
    cudaFree(Traw);
    for (int a = 0; a < 3; ++a)
      if (own[a]) {
        cudaFree(C4[a]);
        cudaFree(S4[a]);
        cudaFree(C2[a]);
        cudaFree(S2[a]);
      }
    *this = Scratch();
  }
};

cudaError_t scratch_alloc(vp_plan p, Scratch& sc) {
  long long gsz = 1, tsz = 1;
  int M1s[3] = {1, 1, 1};
  for (int a = 0; a < p->d; ++a) {
    M1s[a] = 2 * p->Nv[a] + 1;
    gsz *= M1s[a];
    tsz *= (a == 0) ? p->Nv[a] + 1 : M1s[a];  // the chain's largest intermediate (after axis 0)
  }
  cudaError_t e;
  if ((e = cudaMalloc(&sc.G, gsz * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sc.t0, tsz * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sc.t1, tsz * sizeof(double2))) != cudaSuccess) return e;
  if ((e = cudaMalloc(&sc.Traw, p->oct * sizeof(double2))) != cudaSuccess) return e;
  for (int a = 0; a < p->d; ++a) {
    int same = -1;
    for (int b = 0; b < a; ++b)
      if (p->Nv[b] == p->Nv[a]) same = b;
    if (same >= 0) {
      sc.C4[a] = sc.C4[same];
      sc.S4[a] = sc.S4[same];
      sc.C2[a] = sc.C2[same];
      sc.S2[a] = sc.S2[same];
      continue;
    }
    const long long M1 = 2LL * p->Nv[a] + 1, Np1 = p->Nv[a] + 1;
    sc.own[a] = true;
    if ((e = cudaMalloc(&sc.C4[a], Np1 * M1 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sc.S4[a], Np1 * M1 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sc.C2[a], Np1 * Np1 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMalloc(&sc.S2[a], Np1 * Np1 * sizeof(double))) != cudaSuccess) return e;
    if ((e = launch_matrix(sc.C4[a], p->Nv[a], 0, 0)) != cudaSuccess) return e;
    if ((e = launch_matrix(sc.S4[a], p->Nv[a], 1, 0)) != cudaSuccess) return e;
    if ((e = launch_matrix(sc.C2[a], p->Nv[a], 2, 0)) != cudaSuccess) return e;
    if ((e = launch_matrix(sc.S2[a], p->Nv[a], 3, 0)) != cudaSuccess) return e;
  }
  return launch_spectrum(sc.G, p->d, M1s, p->kernel, p->k, p->L, 0);
}

// T (odd_axis < 0) or T_j, then the multiplier, into the plan's arrays.
cudaError_t build_kernel(vp_plan p, Scratch& sc, int odd_axis, double2* Tout, double2* Gu, double2* G64, float2* G32) {
  int dims4[3], qs[3];
  double* m4[3];
  double* m2[3];
  double scale = 1.0;
  for (int a = 0; a < 3; ++a) {
    const int N = a < p->d ? p->Nv[a] : 1;
    dims4[a] = 2 * N + 1;
    qs[a] = N + 1;
    m4[a] = (a == odd_axis) ? sc.S4[a] : sc.C4[a];
    m2[a] = (a == odd_axis) ? sc.S2[a] : sc.C2[a];
    if (a < p->d) scale /= 2.0 * N;
  }
  cudaError_t e = run_chain(sc.G, Tout, sc.t0, sc.t1, p->d, dims4, m4, qs, 0);
  if (e != cudaSuccess) return e;
  e = run_chain(Tout, sc.Traw, sc.t0, sc.t1, p->d, qs, m2, qs, 0);
  if (e != cudaSuccess) return e;
  return launch_finalize(sc.Traw, Gu, G64, G32, p->oct, scale, odd_axis >= 0 ? 1 : 0, 0);
}

vp_status build_grad(vp_plan p) {
  if (p->grad_built) return VP_OK;
  VP_CUDA(p, cudaStreamSynchronize(p->stream));
  for (int j = 0; j < p->d; ++j) {
    VP_CUDA(p, dalloc(p, &p->Tj64[j], p->oct));
    VP_CUDA(p, dalloc(p, &p->Gj64u[j], p->oct));
    VP_CUDA(p, dalloc(p, &p->Gj64[j], p->oct));
    VP_CUDA(p, dalloc(p, &p->Gj32[j], p->oct));
  }
  Scratch sc;
  cudaError_t e = scratch_alloc(p, sc);
  for (int j = 0; j < p->d && e == cudaSuccess; ++j) e = build_kernel(p, sc, j, p->Tj64[j], p->Gj64u[j], p->Gj64[j], p->Gj32[j]);
  if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  sc.release();
  if (e != cudaSuccess) return cuda_fail(p, e, "gradient precompute");
  p->grad_built = true;
  return VP_OK;
}

size_t elem_bytes(vp_dtype t) {
  switch (t) {
    case VP_R32: return 4;
    case VP_C64: return 8;
    case VP_R64: return 8;
    case VP_C128: return 16;
  }
  return 0;
}

// The device mapping of page-locked (pinned) host memory, else NULL.
void* mapped_host_ptr(const void* ptr) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, ptr) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return attr.type == cudaMemoryTypeHost ? attr.devicePointer : nullptr;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes attr;
  cudaError_t e = cudaPointerGetAttributes(&attr, ptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

cudaEvent_t pool_event(vp_plan p) {
  if (!p->event_pool.empty()) {
    cudaEvent_t e = p->event_pool.back();
    p->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Whether a pass's input rows can be staged with 16-byte copies.
template <typename Real>
void set_async(PassArgs<Real>& a, bool contig, int nin) {
  const long long es = a.in_real ? (long long)sizeof(Real) : 2LL * (long long)sizeof(Real);
  bool ok = (reinterpret_cast<uintptr_t>(a.in) % 16 == 0) && ((a.in_pitch_o * es) % 16 == 0) &&
            ((nin * es) % 16 == 0);
  if (!contig) ok = ok && ((a.in_pitch_pos * es) % 16 == 0);
  a.async_ok = ok ? 1 : 0;
}

bool is_tc(vp_precision pr) { return pr == VP_TC_BF16X2 || pr == VP_TC_FP16X2 || pr == VP_TC_BF16X3; }

template <typename Real>
cudaError_t launch_pass(vp_plan p, int pass, PassKind kind, const PassArgs<Real>& a, int len) {
  vp::NvtxRange range(kPassNames[pass]);
  TimedLaunch tl{pass, nullptr, nullptr};
  if (p->timing && p->timed.size() < 100000) {
    tl.start = pool_event(p);
    tl.stop = pool_event(p);
    cudaEventRecord(tl.start, p->stream);
  }
  cudaError_t e;
  if (sizeof(Real) == 4 && pass == P_FUSED && p->tc_split >= 0 && is_tc(p->prec)) {
    const PassArgs<float>& f = reinterpret_cast<const PassArgs<float>&>(a);
    TcFusedArgs t;
    t.in = reinterpret_cast<const float2*>(f.in);
    t.out = reinterpret_cast<float2*>(f.out);
    t.pitch_pos = f.in_pitch_pos;
    t.npencils = (long long)f.O * f.I;
    t.mult = reinterpret_cast<const float2*>(f.fields[0].mult);
    t.tw = p->tw32;
    t.bmat = p->tcB;
    t.err = p->d_err;
    e = launch_tc_fused(len, p->tc_split, t, p->stream);
  } else if (sizeof(Real) == 4)
    e = launch_pass_f32(kind, len, reinterpret_cast<const PassArgs<float>&>(a), p->stream);
  else
    e = launch_pass_f64(kind, len, reinterpret_cast<const PassArgs<double>&>(a), p->stream);
  if (tl.start) {
    cudaEventRecord(tl.stop, p->stream);
    p->timed.push_back(tl);
  }
  return e;
}

// Workspace (complex Real elements, U = N^d): 3D: F x 2U (rows) + F x 4U
// (two-axis spectra); 2D: F x 2U.
// grid points of the plan
size_t grid_points(vp_plan p) {
  size_t U = 1;
  for (int a = 0; a < p->d; ++a) U *= (size_t)p->Nv[a];
  return U;
}

// scratch of one apply with F output fields: 3D rows F x [N0][N1][2N2] and
// two-axis spectra F x [N0][2N1][2N2]; 2D F x [N0][2N1]
size_t workspace_bytes(vp_plan p, int F, size_t csize) {
  const size_t U = grid_points(p);
  if (p->d == 3) return (size_t)F * (U * 2 + U * 4) * csize;
  return (size_t)F * 2 * U * csize;
}

vp_status ensure_workspace(vp_plan p, size_t bytes) {
  if (p->ws_bytes >= bytes) return VP_OK;
  if (p->ws) {
    VP_CUDA(p, cudaStreamSynchronize(p->stream));
    cudaFree(p->ws);
    p->device_bytes -= p->ws_bytes;
    p->ws = nullptr;
    p->ws_bytes = 0;
  }
  VP_CUDA(p, cudaMalloc(&p->ws, bytes));
  p->ws_bytes = bytes;
  p->device_bytes += bytes;
  return VP_OK;
}

// The apply on device pointers: F fields (phi and/or gradient components).
template <typename Real>
vp_status run_apply_ws(vp_plan p, void* ws, const void* f, void* const* outs, const FieldDesc* fields, int F,
                       bool real_io);

template <typename Real>
vp_status run_apply(vp_plan p, const void* f, void* const* outs, const FieldDesc* fields, int F, bool real_io) {
  using C = typename CxT<Real>::T;
  vp_status st = ensure_workspace(p, workspace_bytes(p, F, sizeof(C)));
  if (st != VP_OK) return st;
  return run_apply_ws<Real>(p, p->ws, f, outs, fields, F, real_io);
}

// The pass sequence of one apply on a given workspace of
// workspace_bytes(d, N, F, ...) bytes: (pass id, kind, arguments) per launch.
template <typename Real>
struct PassLaunch {
  int pass;
  PassKind kind;
  int len;  // transform length of the pass's axis
  PassArgs<Real> a;
};

template <typename Real>
int build_pass_list(vp_plan p, void* ws, const void* f, void* const* outs, const FieldDesc* fields, int F,
                    bool real_io, PassLaunch<Real>* list) {
  using C = typename CxT<Real>::T;
  const int d = p->d;
  // grid N0 x N1 (x N2), axis 0 slowest; transform lengths n_j = 2 N_j
  const int N0 = p->Nv[0], N1 = p->Nv[1], N2 = d == 3 ? p->Nv[2] : 1;
  const int n0 = 2 * N0, n1 = 2 * N1, n2 = 2 * N2;
  const long long U = (long long)grid_points(p);
  C* wsA = reinterpret_cast<C*>(ws);    // rows: F x 2U
  C* wsB = wsA + (long long)F * 2 * U;  // 3D spectra: F x 4U
  auto tw_of = [&](int axis) -> const C* {
    return sizeof(Real) == 4 ? reinterpret_cast<const C*>(p->twv32[axis]) : reinterpret_cast<const C*>(p->twv64[axis]);
  };
  int np = 0;
  PassArgs<Real> a;
  memset(&a, 0, sizeof(a));
  a.err = p->d_err;
  a.d = d;
  a.Nh = N0;
  for (int j = 0; j < 3; ++j) {
    a.Nhs[j] = j < d ? p->Nv[j] : 1;
    a.nn[j] = 2 * a.Nhs[j];
  }
  auto push = [&](int pass, PassKind kind, bool contig, int nin, int axis) {
    a.tw = tw_of(axis);
    a.cfg = p->pass_cfg[pass];
    set_async(a, contig, nin);
    list[np].pass = pass;
    list[np].kind = kind;
    list[np].len = 2 * p->Nv[axis];
    list[np].a = a;
    ++np;
  };
  const int last = d - 1;       // the contiguous axis
  const int Nl = p->Nv[last];   // its points and transform length
  const int nl = 2 * Nl;
  // first pass: rows along the last axis, N_l -> 2N_l
  a.in = f;
  a.out = wsA;
  a.O = (int)(U / Nl);
  a.I = 1;
  a.in_pitch_o = Nl;
  a.in_pitch_pos = 1;
  a.out_pitch_o = nl;
  a.out_pitch_pos = 1;
  a.in_real = real_io;
  push(P_FWD_ROWS, FWD_CONTIG, true, Nl, last);
  a.in_real = 0;
  if (d == 3) {
    // axis 1, N1 -> 2N1, slabs i0: [N0][N1][n2] -> [N0][n1][n2]
    a.in = wsA;
    a.out = wsB;
    a.O = N0;
    a.I = n2;
    a.in_pitch_o = (long long)N1 * n2;
    a.in_pitch_pos = n2;
    a.out_pitch_o = (long long)n1 * n2;
    a.out_pitch_pos = n2;
    push(P_FWD_AX1, FWD_STRIDED, false, N1, 1);
    // axis 0 fused, N0 -> N0 per field (field 0 in place): [N0][n1][n2]
    a.in = wsB;
    a.out = wsB;
    a.O = 1;
    a.I = n1 * n2;
    a.in_pitch_o = 0;
    a.in_pitch_pos = (long long)n1 * n2;
    a.out_pitch_o = 0;
    a.out_pitch_pos = (long long)n1 * n2;
    a.out_field_stride = (long long)N0 * n1 * n2;
    a.nfields = F;
    for (int i = 0; i < F; ++i) a.fields[i] = fields[i];
    push(P_FUSED, FUSED_STRIDED, false, N0, 0);
    a.nfields = 0;
    // axis 1 inverse, 2N1 -> N1, all fields as slabs: [F N0][n1][n2] -> [F N0][N1][n2]
    a.in = wsB;
    a.out = wsA;
    a.O = F * N0;
    a.I = n2;
    a.in_pitch_o = (long long)n1 * n2;
    a.in_pitch_pos = n2;
    a.out_pitch_o = (long long)N1 * n2;
    a.out_pitch_pos = n2;
    push(P_INV_AX1, INV_STRIDED, false, n1, 1);
  } else {
    // axis 0 fused (field 0 in place): [N0][n1]
    a.in = wsA;
    a.out = wsA;
    a.O = 1;
    a.I = n1;
    a.in_pitch_o = 0;
    a.in_pitch_pos = n1;
    a.out_pitch_o = 0;
    a.out_pitch_pos = n1;
    a.out_field_stride = (long long)N0 * n1;
    a.nfields = F;
    for (int i = 0; i < F; ++i) a.fields[i] = fields[i];
    push(P_FUSED, FUSED_STRIDED, false, N0, 0);
    a.nfields = 0;
  }
  (void)n0;
  // rows inverse, 2N_l -> N_l, all fields in one launch
  a.in = wsA;
  a.out = outs[0];
  a.O = (int)(F * (U / Nl));
  a.I = 1;
  a.in_pitch_o = nl;
  a.in_pitch_pos = 1;
  a.out_pitch_o = Nl;
  a.out_pitch_pos = 1;
  a.out_real = real_io;
  a.nout = F;
  a.rows_per_field = (long long)(U / Nl);
  for (int i = 0; i < F; ++i) a.outs[i] = outs[i];
  push(P_INV_ROWS, INV_CONTIG, true, nl, last);
  return np;
}

template <typename Real>
vp_status run_apply_ws(vp_plan p, void* ws, const void* f, void* const* outs, const FieldDesc* fields, int F,
                       bool real_io) {
  PassLaunch<Real> list[6];
  const int np = build_pass_list<Real>(p, ws, f, outs, fields, F, real_io, list);
  static const char* what[NPASS] = {"pass fwd_rows", "pass fwd_axis1", "pass fused_axis0", "pass inv_axis1",
                                    "pass inv_rows"};
  for (int i = 0; i < np; ++i) {
    cudaError_t e = launch_pass<Real>(p, list[i].pass, list[i].kind, list[i].a, list[i].len);
    if (e != cudaSuccess) return cuda_fail(p, e, what[list[i].pass]);
  }
  return VP_OK;
}

vp_status check_dtype(vp_plan p, vp_dtype dtype, bool* real_io) {
  const bool fp64 = p->prec == VP_FP64;
  if (dtype == VP_R32 || dtype == VP_R64) {
    if (p->kernel == VP_HELMHOLTZ)
      return fail(p, VP_ERR_INVALID_ARG, "real data types need a real multiplier (the Laplace or biharmonic kernel)");
    *real_io = true;
  } else if (dtype == VP_C64 || dtype == VP_C128) {
    *real_io = false;
  } else {
    return fail(p, VP_ERR_INVALID_ARG, "unknown dtype");
  }
  const bool dt64 = (dtype == VP_R64 || dtype == VP_C128);
  if (dt64 != fp64) return fail(p, VP_ERR_INVALID_ARG, "dtype does not match the plan's precision");
  return VP_OK;
}

// The output fields of one apply: phi (when with_phi) and then the d gradient
// components, each with its multiplier (or its 2N-mode derivative axis).
int make_fields(vp_plan p, bool with_phi, bool want_grad, FieldDesc* fields) {
  const bool fp64 = p->prec == VP_FP64;
  int F = 0;
  if (with_phi) fields[F++] = FieldDesc{fp64 ? (const void*)p->G64 : (const void*)p->G32, -1, -1};
  if (want_grad) {
    for (int j = 0; j < p->d; ++j) {
      if (p->gmode == VP_GRAD_EXACT)
        fields[F++] = FieldDesc{fp64 ? (const void*)p->Gj64[j] : (const void*)p->Gj32[j], j, -1};
      else
        fields[F++] = FieldDesc{fp64 ? (const void*)p->G64 : (const void*)p->G32, -1, j};
    }
  }
  return F;
}

vp_status apply_common(vp_plan p, const void* f, void* phi, void* grad, vp_dtype dtype, bool want_grad) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (!f) return fail(p, VP_ERR_INVALID_ARG, "f is NULL");
  if (!want_grad && !phi) return fail(p, VP_ERR_INVALID_ARG, "phi is NULL");
  if (want_grad && !grad) return fail(p, VP_ERR_INVALID_ARG, "grad is NULL");
  if (phi && phi == f) return fail(p, VP_ERR_INVALID_ARG, "phi may not alias f");
  bool real_io = false;
  vp_status st = check_dtype(p, dtype, &real_io);
  if (st != VP_OK) return st;
  if (want_grad && is_tc(p->prec))
    return fail(p, VP_ERR_UNSUPPORTED, "the tensor-core precisions serve vp_apply only; use VP_FP32 for gradients");
  VP_ON_DEVICE(p, p->device);
  if (want_grad && p->gmode == VP_GRAD_EXACT) {
    st = build_grad(p);
    if (st != VP_OK) return st;
  }
  const bool fp64 = p->prec == VP_FP64;
  const size_t eb = elem_bytes(dtype);
  const size_t U = grid_points(p);

  FieldDesc fields[4];
  const int F = make_fields(p, phi != nullptr, want_grad, fields);

  const bool host_io = !is_device_ptr(f);
  void* outs[4];
  if (host_io && p->host_direct) {
    // page-locked host buffers: the first pass reads f and the last pass writes
    // the outputs through their device mappings, across the CPU-GPU link,
    // with no staging copies (the result is in host memory after the sync)
    const void* fm = mapped_host_ptr(f);
    void* pm = phi ? mapped_host_ptr(phi) : nullptr;
    void* gm = want_grad ? mapped_host_ptr(grad) : nullptr;
    if (fm && (!phi || pm) && (!want_grad || gm)) {
      int i = 0;
      if (phi) outs[i++] = pm;
      if (want_grad)
        for (int j = 0; j < p->d; ++j) outs[i++] = reinterpret_cast<char*>(gm) + (size_t)j * U * eb;
      st = fp64 ? run_apply<double>(p, fm, outs, fields, F, real_io) : run_apply<float>(p, fm, outs, fields, F, real_io);
      if (st != VP_OK) return st;
      VP_CUDA(p, cudaStreamSynchronize(p->stream));
      return VP_OK;
    }
  }
  // other host pointers are staged through device memory
  const void* fd = f;
  char* out_base = nullptr;
  if (host_io) {
    const size_t need = (1 + (size_t)F) * U * eb;
    if (p->stage_bytes < need) {
      if (p->stage) {
        cudaStreamSynchronize(p->stream);
        cudaFree(p->stage);
        p->device_bytes -= p->stage_bytes;
        p->stage = nullptr;
        p->stage_bytes = 0;
      }
      VP_CUDA(p, cudaMalloc(&p->stage, need));
      p->stage_bytes = need;
      p->device_bytes += need;
    }
    char* sbase = reinterpret_cast<char*>(p->stage);
    VP_CUDA(p, cudaMemcpyAsync(sbase, f, U * eb, cudaMemcpyHostToDevice, p->stream));
    fd = sbase;
    out_base = sbase + U * eb;
    for (int i = 0; i < F; ++i) outs[i] = out_base + (size_t)i * U * eb;
  } else {
    int i = 0;
    if (phi) outs[i++] = phi;
    if (want_grad)
      for (int j = 0; j < p->d; ++j) outs[i++] = reinterpret_cast<char*>(grad) + (size_t)j * U * eb;
  }
  st = fp64 ? run_apply<double>(p, fd, outs, fields, F, real_io) : run_apply<float>(p, fd, outs, fields, F, real_io);
  if (st != VP_OK) return st;
  if (host_io) {
    int i = 0;
    if (phi) {
      VP_CUDA(p, cudaMemcpyAsync(phi, outs[i], U * eb, cudaMemcpyDeviceToHost, p->stream));
      ++i;
    }
    if (want_grad)
      VP_CUDA(p, cudaMemcpyAsync(grad, outs[i], (size_t)p->d * U * eb, cudaMemcpyDeviceToHost, p->stream));
    VP_CUDA(p, cudaStreamSynchronize(p->stream));
  }
  return VP_OK;
}

constexpr int kPipeSlots = 3;

// Copy streams, events and `bytes` of device slots for vp_apply_pipeline.
vp_status pipeline_resources(vp_plan p, size_t bytes) {
  if (!p->pipe_h2d) VP_CUDA(p, cudaStreamCreateWithFlags(&p->pipe_h2d, cudaStreamNonBlocking));
  if (!p->pipe_d2h) VP_CUDA(p, cudaStreamCreateWithFlags(&p->pipe_d2h, cudaStreamNonBlocking));
  if (!p->pipe_start) VP_CUDA(p, cudaEventCreateWithFlags(&p->pipe_start, cudaEventDisableTiming));
  for (int s = 0; s < kPipeSlots; ++s)
    for (int e = 0; e < 3; ++e)
      if (!p->pipe_ev[s][e]) VP_CUDA(p, cudaEventCreateWithFlags(&p->pipe_ev[s][e], cudaEventDisableTiming));
  if (p->pipe_bytes < bytes) {
    if (p->pipe_buf) {
      cudaFree(p->pipe_buf);
      p->device_bytes -= p->pipe_bytes;
      p->pipe_buf = nullptr;
      p->pipe_bytes = 0;
    }
    VP_CUDA(p, cudaMalloc(&p->pipe_buf, bytes));
    p->pipe_bytes = bytes;
    p->device_bytes += bytes;
  }
  return VP_OK;
}

// Issues the pipeline: density i is copied in on the h2d stream, applied on
// the plan's stream and its fields copied out on the d2h stream, in slot
// i mod R; the copy into a slot waits for the apply that last read it, the
// apply for the copy-out that last emptied it.  So the copies of densities
// i + 1 and i - 1 overlap the apply of density i.
vp_status pipeline_issue(vp_plan p, int count, const void* const* f, void* const* phi, void* const* grad,
                         size_t fb, const FieldDesc* fields, int F, bool real_io) {
  const int R = count < kPipeSlots ? count : kPipeSlots;
  const size_t slot = (1 + (size_t)F) * fb;
  char* base = reinterpret_cast<char*>(p->pipe_buf);
  VP_CUDA(p, cudaEventRecord(p->pipe_start, p->stream));
  VP_CUDA(p, cudaStreamWaitEvent(p->pipe_h2d, p->pipe_start, 0));
  for (int i = 0; i < count; ++i) {
    const int s = i % R;
    char* in = base + (size_t)s * slot;
    char* out = in + fb;
    cudaEvent_t* ev = p->pipe_ev[s];
    if (i >= R) VP_CUDA(p, cudaStreamWaitEvent(p->pipe_h2d, ev[1], 0));
    VP_CUDA(p, cudaMemcpyAsync(in, f[i], fb, cudaMemcpyDefault, p->pipe_h2d));
    VP_CUDA(p, cudaEventRecord(ev[0], p->pipe_h2d));
    VP_CUDA(p, cudaStreamWaitEvent(p->stream, ev[0], 0));
    if (i >= R) VP_CUDA(p, cudaStreamWaitEvent(p->stream, ev[2], 0));
    void* outs[4];
    for (int j = 0; j < F; ++j) outs[j] = out + (size_t)j * fb;
    vp_status st = p->prec == VP_FP64 ? run_apply_ws<double>(p, p->ws, in, outs, fields, F, real_io)
                                      : run_apply_ws<float>(p, p->ws, in, outs, fields, F, real_io);
    if (st != VP_OK) return st;
    VP_CUDA(p, cudaEventRecord(ev[1], p->stream));
    VP_CUDA(p, cudaStreamWaitEvent(p->pipe_d2h, ev[1], 0));
    int j = 0;
    if (phi) VP_CUDA(p, cudaMemcpyAsync(phi[i], out + fb * j++, fb, cudaMemcpyDefault, p->pipe_d2h));
    if (grad) VP_CUDA(p, cudaMemcpyAsync(grad[i], out + fb * j, (size_t)p->d * fb, cudaMemcpyDefault, p->pipe_d2h));
    VP_CUDA(p, cudaEventRecord(ev[2], p->pipe_d2h));
  }
  return VP_OK;
}

vp_status apply_pipeline(vp_plan p, int count, const void* const* f, void* const* phi, void* const* grad,
                         vp_dtype dtype) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (count < 0) return fail(p, VP_ERR_INVALID_ARG, "count is negative");
  if (count > 0 && !f) return fail(p, VP_ERR_INVALID_ARG, "f is NULL");
  if (!phi && !grad) return fail(p, VP_ERR_INVALID_ARG, "phi and grad are both NULL");
  for (int i = 0; i < count; ++i) {
    if (!f[i] || (phi && !phi[i]) || (grad && !grad[i]))
      return fail(p, VP_ERR_INVALID_ARG, "a NULL entry in f, phi or grad");
    if (phi && phi[i] == f[i]) return fail(p, VP_ERR_INVALID_ARG, "phi may not alias f");
  }
  bool real_io = false;
  vp_status st = check_dtype(p, dtype, &real_io);
  if (st != VP_OK) return st;
  if (grad && is_tc(p->prec))
    return fail(p, VP_ERR_UNSUPPORTED, "the tensor-core precisions serve vp_apply only; use VP_FP32 for gradients");
  if (count == 0) return VP_OK;
  VP_ON_DEVICE(p, p->device);
  if (grad && p->gmode == VP_GRAD_EXACT) {
    st = build_grad(p);
    if (st != VP_OK) return st;
  }
  FieldDesc fields[4];
  const int F = make_fields(p, phi != nullptr, grad != nullptr, fields);
  const size_t fb = grid_points(p) * elem_bytes(dtype);
  const size_t csize = p->prec == VP_FP64 ? sizeof(double2) : sizeof(float2);
  const int R = count < kPipeSlots ? count : kPipeSlots;
  if ((st = ensure_workspace(p, workspace_bytes(p, F, csize))) != VP_OK) return st;
  if ((st = pipeline_resources(p, (size_t)R * (1 + F) * fb)) != VP_OK) return st;
  st = pipeline_issue(p, count, f, phi, grad, fb, fields, F, real_io);
  // every copy into the caller's buffers has ended when the call returns,
  // whether or not issuing failed part-way
  const cudaError_t e1 = cudaStreamSynchronize(p->pipe_d2h);
  const cudaError_t e2 = cudaStreamSynchronize(p->stream);
  const cudaError_t e3 = cudaStreamSynchronize(p->pipe_h2d);
  if (st != VP_OK) return st;
  VP_CUDA(p, e1);
  VP_CUDA(p, e2);
  VP_CUDA(p, e3);
  return VP_OK;
}

}  // namespace


// ---------------------------------------------------------------------------
// internal hooks for other translation units
// ---------------------------------------------------------------------------
namespace vp {

int log_level() {
  static const int level = [] {
    const char* s = getenv("VP_LOG");
    return (s && *s >= '0' && *s <= '9') ? atoi(s) : 0;
  }();
  return level;
}

void log_line(int level, const char* what, const std::string& msg) {
  if (log_level() >= level) fprintf(stderr, "vp: %s: %s\n", what, msg.c_str());
}

int plan_device(vp_plan p) { return p ? p->device : -1; }

cudaStream_t plan_stream(vp_plan p) { return p ? p->stream : nullptr; }

int plan_is_fp32(vp_plan p) { return p && p->prec == VP_FP32; }

int plan_is_fp64(vp_plan p) { return p && p->prec == VP_FP64; }

vp_status entries_fail(vp_plan p, vp_status st, const char* msg) { return fail(p, st, msg); }

int plan_kernel(vp_plan p) { return p ? p->kernel : -1; }

int plan_is_aniso(vp_plan p) { return p ? p->aniso : 0; }

long long plan_points(vp_plan p) { return p ? (long long)grid_points(p) : 0; }

void plan_dims(vp_plan p, int* N) {
  for (int a = 0; a < 3; ++a) N[a] = a < p->d ? p->Nv[a] : 1;
}

vp_status plan_prepare_grad(vp_plan p) {
  VP_ON_DEVICE(p, p->device);
  return build_grad(p);
}

size_t plan_grad_workspace_bytes(vp_plan p) {
  const size_t csize = p->prec == VP_FP64 ? sizeof(double2) : sizeof(float2);
  return workspace_bytes(p, p->d, csize);
}

vp_status apply_grad_with_workspace(vp_plan p, const void* f, void* grad, vp_dtype dtype, void* ws, size_t ws_bytes) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (!f || !grad) return fail(p, VP_ERR_INVALID_ARG, "f and grad must be non-NULL");
  bool real_io = false;
  vp_status st = check_dtype(p, dtype, &real_io);
  if (st != VP_OK) return st;
  if (!p->grad_built) return fail(p, VP_ERR_INVALID_ARG, "the derivative multipliers are not built");
  if (ws_bytes < plan_grad_workspace_bytes(p)) return fail(p, VP_ERR_UNSUPPORTED, "gradient workspace too small");
  const bool fp64 = p->prec == VP_FP64;
  const size_t U = grid_points(p);
  FieldDesc fields[3];
  void* outs[3];
  for (int j = 0; j < p->d; ++j) {
    fields[j] = FieldDesc{fp64 ? (const void*)p->Gj64[j] : (const void*)p->Gj32[j], j, -1};
    outs[j] = reinterpret_cast<char*>(grad) + (size_t)j * U * elem_bytes(dtype);
  }
  const bool timing = p->timing;
  p->timing = false;
  st = fp64 ? run_apply_ws<double>(p, ws, f, outs, fields, p->d, real_io)
            : run_apply_ws<float>(p, ws, f, outs, fields, p->d, real_io);
  p->timing = timing;
  return st;
}

vp_status plan_kernel_octant(vp_plan p, int which, int axis, const double2** oct) {
  VP_ON_DEVICE(p, p->device);
  if (which == VP_ARRAY_T) {
    *oct = p->T64;
    return VP_OK;
  }
  if (which != VP_ARRAY_TJ) return fail(p, VP_ERR_INVALID_ARG, "which must be VP_ARRAY_T or VP_ARRAY_TJ");
  if (axis < 0 || axis >= p->d) return fail(p, VP_ERR_INVALID_ARG, "axis out of range");
  vp_status st = build_grad(p);
  if (st != VP_OK) return st;
  *oct = p->Tj64[axis];
  return VP_OK;
}

vp_status plan_kernel_octant32(vp_plan p, int which, int axis, const float2** oct) {
  const double2* o64 = nullptr;
  vp_status st = plan_kernel_octant(p, which, axis, &o64);
  if (st != VP_OK) return st;
  float2** slot = which == VP_ARRAY_T ? &p->T32 : &p->Tj32[axis];
  if (!*slot) {
    VP_CUDA(p, dalloc(p, slot, p->oct));
    VP_CUDA(p, launch_narrow(o64, *slot, p->oct, p->stream));
  }
  *oct = *slot;
  return VP_OK;
}

int* plan_flag_word(vp_plan p) {
  if (!p->d_flag && cudaMalloc(&p->d_flag, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    p->d_flag = nullptr;
  }
  return p->d_flag;
}

int plan_pass_args_f32(vp_plan p, float2* ws, PassArgs<float>* args, int* kinds, int* lens) {
  FieldDesc field{(const void*)p->G32, -1, -1};
  void* outs[1] = {nullptr};
  PassLaunch<float> list[6];
  const int np = build_pass_list<float>(p, ws, nullptr, outs, &field, 1, false, list);
  for (int i = 0; i < np; ++i) {
    args[i] = list[i].a;
    kinds[i] = (int)list[i].kind;
    lens[i] = list[i].len;
  }
  return np;
}

size_t plan_apply_workspace_bytes(vp_plan p) {
  const size_t csize = p->prec == VP_FP64 ? sizeof(double2) : sizeof(float2);
  return workspace_bytes(p, 1, csize);
}

vp_status apply_with_workspace(vp_plan p, const void* f, void* phi, vp_dtype dtype, void* ws, size_t ws_bytes) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (!f || !phi) return fail(p, VP_ERR_INVALID_ARG, "f and phi must be non-NULL");
  if (phi == f) return fail(p, VP_ERR_INVALID_ARG, "phi may not alias f");
  bool real_io = false;
  vp_status st = check_dtype(p, dtype, &real_io);
  if (st != VP_OK) return st;
  if (!is_device_ptr(f) || !is_device_ptr(phi))
    return fail(p, VP_ERR_INVALID_ARG, "this entry point takes device pointers only");
  const size_t need = plan_apply_workspace_bytes(p);
  if (ws_bytes < need) {
    char msg[200];
    snprintf(msg, sizeof(msg), "grid needs %zu bytes of scratch, the static array holds %zu", need, ws_bytes);
    return fail(p, VP_ERR_UNSUPPORTED, msg);
  }
  const bool fp64 = p->prec == VP_FP64;
  FieldDesc field{fp64 ? (const void*)p->G64 : (const void*)p->G32, -1, -1};
  void* outs[1] = {phi};
  const bool timing = p->timing;  // no event objects are created on this path
  p->timing = false;
  st = fp64 ? run_apply_ws<double>(p, ws, f, outs, &field, 1, real_io)
            : run_apply_ws<float>(p, ws, f, outs, &field, 1, real_io);
  p->timing = timing;
  return st;
}

}  // namespace vp

extern "C" {

int vp_fft_length_supported(int n2) { return fft_length_built(n2) ? 1 : 0; }

namespace {

// Host copies of a saved plan's FP64 precompute results (vp_plan_save): T and
// the unscaled multiplier, and with `grad` the derivative kernels T_j and their
// multipliers; every other array of a plan follows from these.
struct PlanPayload {
  std::vector<double2> T, Gu;
  std::vector<double2> Tj[3], Gju[3];
  bool grad = false;
};

// The multiplier arrays the apply reads, from an uploaded unscaled multiplier
// (the same scaling and rounding as the precompute's last step).
cudaError_t upload_kernel(vp_plan p, const std::vector<double2>& T, const std::vector<double2>& Gu, double2* Tout,
                          double2* Gu_dev, double2* G64, float2* G32, double scale) {
  const size_t bytes = (size_t)p->oct * sizeof(double2);
  cudaError_t e = cudaMemcpy(Tout, T.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(Gu_dev, Gu.data(), bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_finalize(Gu_dev, nullptr, G64, G32, p->oct, scale, 0, 0);
  return e;
}

vp_status plan_create_common(vp_plan* out, int d, const int* Ns, vp_kernel kernel, double k, double L,
                             const PlanPayload* saved = nullptr) {
  if (!out) return fail(nullptr, VP_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (d != 2 && d != 3) return fail(nullptr, VP_ERR_INVALID_ARG, "d must be 2 or 3");
  for (int a = 0; a < d; ++a)
    if (Ns[a] < 4 || Ns[a] % 2) return fail(nullptr, VP_ERR_INVALID_ARG, "N must be even and >= 4");
  if (kernel != VP_LAPLACE && kernel != VP_HELMHOLTZ && kernel != VP_BIHARMONIC)
    return fail(nullptr, VP_ERR_INVALID_ARG, "unknown kernel");
  if (!isfinite(k) || (kernel != VP_HELMHOLTZ && k != 0.0) || (kernel == VP_HELMHOLTZ && !(k > 0.0)))
    return fail(nullptr, VP_ERR_INVALID_ARG, "k must be 0 for Laplace and biharmonic, > 0 for Helmholtz");
  if (!isfinite(L)) return fail(nullptr, VP_ERR_INVALID_ARG, "L must be finite");
  if (L <= 0.0) L = (d == 3) ? 1.8 : 1.5;
  if (!(L > sqrt((double)d)) || L > 3.0) return fail(nullptr, VP_ERR_INVALID_ARG, "L must satisfy sqrt(d) < L <= 3");
  long long oct = 1;
  for (int a = 0; a < d; ++a) {
    if (!fft_length_built(2 * Ns[a])) return fail(nullptr, VP_ERR_UNSUPPORTED, "2N is not a built FFT length");
    oct *= Ns[a] + 1;
  }

  vp_plan p = new vp_plan_s();
  p->d = d;
  p->N = Ns[0];
  for (int a = 0; a < d; ++a) {
    p->Nv[a] = Ns[a];
    if (Ns[a] != Ns[0]) p->aniso = 1;
  }
  p->kernel = kernel;
  p->k = k;
  p->L = L;
  p->n2 = 2 * Ns[0];
  p->oct = oct;
  cudaError_t e = cudaGetDevice(&p->device);
  // in-place access to pinned host buffers by default only where the device
  // reads host memory coherently through the host's page tables (a CPU-GPU
  // link such as NVLink-C2C); over PCIe the buffers are staged
  if (e == cudaSuccess) {
    int coherent = 0;
    if (cudaDeviceGetAttribute(&coherent, cudaDevAttrPageableMemoryAccessUsesHostPageTables, p->device) != cudaSuccess)
      coherent = 0;
    p->host_direct = coherent ? 1 : 0;
  }
  if (e == cudaSuccess) {
    double x[GL_NODES], w[GL_NODES];
    gauss_legendre(GL_NODES, x, w);
    e = set_gauss_legendre(x, w);
  }
  if (e == cudaSuccess) e = dalloc(p, &p->T64, oct);
  if (e == cudaSuccess) e = dalloc(p, &p->G64u, oct);
  if (e == cudaSuccess) e = dalloc(p, &p->G64, oct);
  if (e == cudaSuccess) e = dalloc(p, &p->G32, oct);
  // twiddles per distinct axis length (axis 0's are the plan's tw64/tw32)
  for (int a = 0; a < d && e == cudaSuccess; ++a) {
    int same = -1;
    for (int b = 0; b < a; ++b)
      if (Ns[b] == Ns[a]) same = b;
    if (same >= 0) {
      p->twv64[a] = p->twv64[same];
      p->twv32[a] = p->twv32[same];
      continue;
    }
    e = dalloc(p, &p->twv64[a], 2 * Ns[a]);
    if (e == cudaSuccess) e = dalloc(p, &p->twv32[a], 2 * Ns[a]);
    if (e == cudaSuccess) e = launch_twiddles(p->twv64[a], p->twv32[a], 2 * Ns[a], 0);
  }
  p->tw64 = p->twv64[0];
  p->tw32 = p->twv32[0];
  // device error word of the bounded waits in the pass kernels (TMA and
  // tensor-core pipelines), read and cleared by vp_plan_status
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (!saved) {
    Scratch sc;
    if (e == cudaSuccess) e = scratch_alloc(p, sc);
    if (e == cudaSuccess) e = build_kernel(p, sc, -1, p->T64, p->G64u, p->G64, p->G32);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    sc.release();
  } else {
    // a saved plan: its FP64 arrays replace the precompute
    double scale = 1.0;
    for (int a = 0; a < d; ++a) scale /= 2.0 * Ns[a];
    if (e == cudaSuccess) e = upload_kernel(p, saved->T, saved->Gu, p->T64, p->G64u, p->G64, p->G32, scale);
    if (saved->grad) {
      for (int j = 0; j < d && e == cudaSuccess; ++j) {
        e = dalloc(p, &p->Tj64[j], oct);
        if (e == cudaSuccess) e = dalloc(p, &p->Gj64u[j], oct);
        if (e == cudaSuccess) e = dalloc(p, &p->Gj64[j], oct);
        if (e == cudaSuccess) e = dalloc(p, &p->Gj32[j], oct);
        if (e == cudaSuccess)
          e = upload_kernel(p, saved->Tj[j], saved->Gju[j], p->Tj64[j], p->Gj64u[j], p->Gj64[j], p->Gj32[j], scale);
      }
      p->grad_built = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
  }
  if (e != cudaSuccess) {
    std::string msg = std::string("precompute: ") + cudaGetErrorString(e);
    vp_status st = (e == cudaErrorMemoryAllocation) ? VP_ERR_OOM : VP_ERR_CUDA;
    vp_destroy(p);
    return fail(nullptr, st, msg);
  }
  *out = p;
  return VP_OK;
}

}  // namespace

vp_status vp_plan_create(vp_plan* out, int d, int N, vp_kernel kernel, double k, double L) {
  const int Ns[3] = {N, N, N};
  return plan_create_common(out, d, Ns, kernel, k, L);
}

vp_status vp_plan_create_aniso(vp_plan* out, int d, const int* N, vp_kernel kernel, double k, double L) {
  if (!N) {
    if (out) *out = nullptr;
    return fail(nullptr, VP_ERR_INVALID_ARG, "N is NULL");
  }
  return plan_create_common(out, d, N, kernel, k, L);
}

vp_status vp_plan_dims(vp_plan p, int* N) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (!N) return fail(p, VP_ERR_INVALID_ARG, "N is NULL");
  for (int a = 0; a < p->d; ++a) N[a] = p->Nv[a];
  return VP_OK;
}

namespace {

// Saved-plan file: a 96-byte header, then the FP64 octants (complex128, axis 0
// slowest) T, G (unscaled) and, when the gradient kernels were built, T_j and
// G_j for j < d.  Host byte order.
constexpr char kPlanMagic[8] = {'V', 'P', 'P', 'L', 'A', 'N', '0', '1'};
struct PlanFileHeader {
  char magic[8];
  uint32_t version, header_bytes;
  int32_t d, N[3], kernel, grad;
  double k, L;
  int64_t oct;
  uint64_t payload_bytes, checksum;
  uint8_t reserved[16];
};
static_assert(sizeof(PlanFileHeader) == 96, "plan file header is 96 bytes");

// 64-bit FNV-1a over the payload's 8-byte words (offset basis and prime of
// FNV-1a 64), continued from h
uint64_t payload_hash(const std::vector<double2>& v, uint64_t h) {
  const uint64_t* w = reinterpret_cast<const uint64_t*>(v.data());
  for (size_t i = 0, n = v.size() * 2; i < n; ++i) {
    h ^= w[i];
    h *= 1099511628211ULL;
  }
  return h;
}
constexpr uint64_t kHashBasis = 14695981039346656037ULL;

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

}  // namespace

vp_status vp_plan_save(vp_plan p, const char* path) {
  if (!p || !path) return fail(p, VP_ERR_INVALID_ARG, "plan or path is NULL");
  VP_ON_DEVICE(p, p->device);
  VP_CUDA(p, cudaStreamSynchronize(p->stream));
  std::vector<const double2*> arrays = {p->T64, p->G64u};
  if (p->grad_built)
    for (int j = 0; j < p->d; ++j) {
      arrays.push_back(p->Tj64[j]);
      arrays.push_back(p->Gj64u[j]);
    }
  PlanFileHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kPlanMagic, 8);
  h.version = 1;
  h.header_bytes = sizeof(h);
  h.d = p->d;
  for (int a = 0; a < 3; ++a) h.N[a] = a < p->d ? p->Nv[a] : 0;
  h.kernel = p->kernel;
  h.grad = p->grad_built ? 1 : 0;
  h.k = p->k;
  h.L = p->L;
  h.oct = p->oct;
  h.payload_bytes = (uint64_t)arrays.size() * (uint64_t)p->oct * sizeof(double2);
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) return fail(p, VP_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
  if (fwrite(&h, sizeof(h), 1, out.f) != 1) return fail(p, VP_ERR_INVALID_ARG, "write failed");
  std::vector<double2> buf;
  try {
    buf.resize((size_t)p->oct);
  } catch (const std::bad_alloc&) {
    return fail(p, VP_ERR_OOM, "saving the plan: host memory for one octant");
  }
  uint64_t hash = kHashBasis;
  for (const double2* a : arrays) {
    VP_CUDA(p, cudaMemcpy(buf.data(), a, buf.size() * sizeof(double2), cudaMemcpyDeviceToHost));
    hash = payload_hash(buf, hash);
    if (fwrite(buf.data(), sizeof(double2), buf.size(), out.f) != buf.size())
      return fail(p, VP_ERR_INVALID_ARG, "write failed");
  }
  h.checksum = hash;
  if (fseek(out.f, 0, SEEK_SET) != 0 || fwrite(&h, sizeof(h), 1, out.f) != 1)
    return fail(p, VP_ERR_INVALID_ARG, "write failed");
  if (fclose(out.f) != 0) {
    out.f = nullptr;
    return fail(p, VP_ERR_INVALID_ARG, "write failed");
  }
  out.f = nullptr;
  return VP_OK;
}

vp_status vp_plan_load(vp_plan* out, const char* path) {
  if (!out || !path) return fail(nullptr, VP_ERR_INVALID_ARG, "out or path is NULL");
  *out = nullptr;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return fail(nullptr, VP_ERR_INVALID_ARG, std::string("cannot open: ") + path);
  PlanFileHeader h;
  if (fread(&h, sizeof(h), 1, in.f) != 1 || memcmp(h.magic, kPlanMagic, 8) != 0 || h.version != 1 ||
      h.header_bytes != sizeof(h))
    return fail(nullptr, VP_ERR_INVALID_ARG, "not a saved plan (magic, version or header size)");
  if ((h.d != 2 && h.d != 3) || (h.grad != 0 && h.grad != 1))
    return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: bad dimension or flags");
  int Ns[3] = {0, 0, 0};
  long long oct = 1;
  for (int a = 0; a < h.d; ++a) {
    if (h.N[a] < 4 || h.N[a] > (1 << 16)) return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: bad grid size");
    Ns[a] = h.N[a];
    oct *= h.N[a] + 1;
  }
  const uint64_t narrays = 2 + (h.grad ? 2 * h.d : 0);
  if (h.oct != oct || h.payload_bytes != narrays * (uint64_t)oct * sizeof(double2))
    return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: sizes do not match the grid");
  // the file must hold exactly the header and the payload it announces; checked
  // before anything of the payload's size is allocated
  if (fseek(in.f, 0, SEEK_END) != 0) return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: cannot seek");
  const long long fsize = (long long)ftell(in.f);
  if (fsize < (long long)sizeof(h) + (long long)h.payload_bytes)
    return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: the file is truncated");
  if (fsize > (long long)sizeof(h) + (long long)h.payload_bytes)
    return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: trailing bytes");
  if (fseek(in.f, (long)sizeof(h), SEEK_SET) != 0) return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: cannot seek");
  PlanPayload pl;
  pl.grad = h.grad != 0;
  std::vector<std::vector<double2>*> arrays = {&pl.T, &pl.Gu};
  if (pl.grad)
    for (int j = 0; j < h.d; ++j) {
      arrays.push_back(&pl.Tj[j]);
      arrays.push_back(&pl.Gju[j]);
    }
  uint64_t hash = kHashBasis;
  for (std::vector<double2>* a : arrays) {
    try {
      a->resize((size_t)oct);
    } catch (const std::bad_alloc&) {
      return fail(nullptr, VP_ERR_OOM, "saved plan: host memory for the payload");
    }
    if (fread(a->data(), sizeof(double2), a->size(), in.f) != a->size())
      return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: the file is truncated");
    hash = payload_hash(*a, hash);
  }
  if (fgetc(in.f) != EOF) return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: trailing bytes");
  if (hash != h.checksum) return fail(nullptr, VP_ERR_INVALID_ARG, "saved plan: checksum mismatch");
  return plan_create_common(out, h.d, Ns, (vp_kernel)h.kernel, h.k, h.L, &pl);
}

vp_status vp_plan_kernel(vp_plan p, vp_kernel* kernel) {
  if (!p || !kernel) return fail(p, VP_ERR_INVALID_ARG, "plan or kernel is NULL");
  *kernel = (vp_kernel)p->kernel;
  return VP_OK;
}

vp_status vp_plan_set_host_access(vp_plan p, int direct) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  p->host_direct = direct ? 1 : 0;
  return VP_OK;
}

// Pass `pass` of the plan's FP32 apply: its candidate tile shapes (count 0 when
// the pass does not run on the four-step engine), the current choice and its name.
vp_status vp_plan_pass_config(vp_plan p, int pass, int* cfg, int* count, char* name, size_t cap) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (pass < 0 || pass >= NPASS) return fail(p, VP_ERR_INVALID_ARG, "pass index out of range");
  int nc = 0;
  char names[4][32];
  bool fits[4];
  const PassLaunch<float>* L = nullptr;
  PassLaunch<float> list[6];
  FieldDesc field{(const void*)p->G32, -1, -1};
  void* base = reinterpret_cast<void*>((uintptr_t)1 << 20);  // kinds and lengths only: nothing is read
  void* outs[1] = {base};
  const int np = build_pass_list<float>(p, base, base, outs, &field, 1, false, list);
  for (int i = 0; i < np; ++i)
    if (list[i].pass == pass) L = &list[i];
  if (L) nc = fourstep_shapes(L->kind, L->len, names, fits);
  if (cfg) *cfg = p->pass_cfg[pass];
  if (count) *count = nc;
  if (name && cap) snprintf(name, cap, "%s", !L ? "absent" : nc ? names[p->pass_cfg[pass]] : "stockham");
  return VP_OK;
}

vp_status vp_plan_set_pass_config(vp_plan p, int pass, int cfg) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  int nc = 0;
  vp_status st = vp_plan_pass_config(p, pass, nullptr, &nc, nullptr, 0);
  if (st != VP_OK) return st;
  if (cfg < 0 || cfg >= (nc > 0 ? nc : 1)) return fail(p, VP_ERR_INVALID_ARG, "no such tile shape for this pass");
  if (nc > 0) {
    PassLaunch<float> list[6];
    FieldDesc field{(const void*)p->G32, -1, -1};
    void* base = reinterpret_cast<void*>((uintptr_t)1 << 20);
    void* outs[1] = {base};
    const int np = build_pass_list<float>(p, base, base, outs, &field, 1, false, list);
    char names[4][32];
    bool fits[4];
    for (int i = 0; i < np; ++i)
      if (list[i].pass == pass && fourstep_shapes(list[i].kind, list[i].len, names, fits) && !fits[cfg])
        return fail(p, VP_ERR_UNSUPPORTED, "this tile shape exceeds a CTA's shared memory");
  }
  p->pass_cfg[pass] = cfg;
  return VP_OK;
}

// Tries every candidate tile shape of each four-step pass of the FP32 apply,
// pass by pass, timing whole applies on the plan's own workspace and stream
// (2 warm-ups, 10 timed applies, CUDA events), so that each pass is measured
// with the cache state the passes before it leave; a candidate replaces the
// current choice when the apply gets more than 1% faster.  The choices are
// cached on disk per device, driver and grid; flags & 1 ignores the cache.
vp_status vp_plan_autotune(vp_plan p, int flags) {
  vp::NvtxRange range("vp_plan_autotune");
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (p->prec != VP_FP32) return fail(p, VP_ERR_UNSUPPORTED, "the autotuner tunes the FP32 passes: set VP_FP32 first");
  VP_ON_DEVICE(p, p->device);
  cudaDeviceProp prop;
  VP_CUDA(p, cudaGetDeviceProperties(&prop, p->device));
  int drv = 0;
  VP_CUDA(p, cudaDriverGetVersion(&drv));
  std::string key = std::string(prop.name) + "|drv" + std::to_string(drv) + "|passes|" + std::to_string(p->d) + "d";
  for (int a = 0; a < p->d; ++a) key += (a ? "x" : "") + std::to_string(p->Nv[a]);
  if (!(flags & 1)) {
    const int c = autotune_cache_lookup(key);
    if (c > 0) {
      for (int i = 0; i < NPASS; ++i) p->pass_cfg[i] = ((c - 1) >> (3 * i)) & 7;
      for (int i = 0; i < NPASS; ++i)
        if (p->pass_cfg[i] >= 4) p->pass_cfg[i] = 0;
      return VP_OK;
    }
  }
  const size_t U = grid_points(p);
  vp_status st = ensure_workspace(p, workspace_bytes(p, 1, sizeof(float2)));
  if (st != VP_OK) return st;
  float2 *fin = nullptr, *fout = nullptr;
  VP_CUDA(p, cudaMalloc(&fin, U * sizeof(float2)));
  cudaError_t e = cudaMalloc(&fout, U * sizeof(float2));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaMemsetAsync(fin, 0, U * sizeof(float2), p->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  PassLaunch<float> list[6];
  FieldDesc field{(const void*)p->G32, -1, -1};
  void* outs[1] = {fout};
  for (int i = 0; i < NPASS; ++i) p->pass_cfg[i] = 0;
  const int np = e == cudaSuccess ? build_pass_list<float>(p, p->ws, fin, outs, &field, 1, false, list) : 0;
  // one apply's time with the current choices: 2 warm-ups, 10 timed applies
  auto time_apply = [&](float* ms) -> cudaError_t {
    for (int w = 0; w < 2; ++w)
      if (run_apply_ws<float>(p, p->ws, fin, outs, &field, 1, false) != VP_OK) return cudaErrorUnknown;
    cudaError_t le = cudaEventRecord(e0, p->stream);
    for (int r = 0; r < 10 && le == cudaSuccess; ++r)
      if (run_apply_ws<float>(p, p->ws, fin, outs, &field, 1, false) != VP_OK) le = cudaErrorUnknown;
    if (le == cudaSuccess) le = cudaEventRecord(e1, p->stream);
    if (le == cudaSuccess) le = cudaEventSynchronize(e1);
    if (le == cudaSuccess) le = cudaEventElapsedTime(ms, e0, e1);
    return le;
  };
  float cur = 0.f;
  if (e == cudaSuccess && np > 0) e = time_apply(&cur);
  // coordinate descent over the passes: a candidate replaces the current
  // choice when whole applies get more than 1% faster
  for (int i = 0; i < np && e == cudaSuccess; ++i) {
    const PassLaunch<float>& L = list[i];
    char names[4][32];
    bool fits[4];
    const int nc = fourstep_shapes(L.kind, L.len, names, fits);
    if (!nc || !fourstep_serves(L.kind, L.len, L.a)) continue;
    int bc = 0;
    for (int c = 1; c < nc && e == cudaSuccess; ++c) {
      if (!fits[c]) continue;
      p->pass_cfg[L.pass] = c;
      float ms = 0.f;
      e = time_apply(&ms);
      if (e == cudaSuccess && ms < 0.99f * cur) {
        cur = ms;
        bc = c;
      }
    }
    p->pass_cfg[L.pass] = bc;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(p->stream);
  cudaFree(fin);
  if (fout) cudaFree(fout);
  if (e != cudaSuccess) {
    for (int i = 0; i < NPASS; ++i) p->pass_cfg[i] = 0;
    return cuda_fail(p, e, "vp_plan_autotune");
  }
  int code = 0;
  for (int i = 0; i < NPASS; ++i) code |= p->pass_cfg[i] << (3 * i);
  autotune_cache_store(key, code + 1);
  if (vp::log_level() >= 2) {
    std::string m = key + " ->";
    for (int pass = 0; pass < NPASS; ++pass) m += " " + std::string(kPassNames[pass]) + "=" + std::to_string(p->pass_cfg[pass]);
    vp::log_line(2, "autotune", m);
  }
  return VP_OK;
}

vp_status vp_plan_set_stream(vp_plan p, void* stream) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  p->stream = reinterpret_cast<cudaStream_t>(stream);
  return VP_OK;
}

vp_status vp_plan_set_precision(vp_plan p, vp_precision precision) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (precision != VP_FP32 && precision != VP_FP64 && !is_tc(precision))
    return fail(p, VP_ERR_INVALID_ARG, "unknown precision");
  if (is_tc(precision)) {
    if (p->d != 3 || p->aniso || !tc_length_supported(p->n2))
      return fail(p, VP_ERR_UNSUPPORTED, "tensor-core precisions need a cubic 3D plan with N = 128 or 256");
    const int split = precision == VP_TC_BF16X2 ? 0 : (precision == VP_TC_FP16X2 ? 1 : 2);
    if (p->tc_split != split) {
      VP_ON_DEVICE(p, p->device);
      VP_CUDA(p, cudaStreamSynchronize(p->stream));
      const size_t bytes = tc_bmat_bytes(p->n2, split);
      if (p->tcB) {
        cudaFree(p->tcB);
        p->device_bytes -= tc_bmat_bytes(p->n2, p->tc_split);
        p->tcB = nullptr;
        p->tc_split = -1;
      }
      VP_CUDA(p, cudaMalloc(&p->tcB, bytes));
      p->device_bytes += bytes;
      if (!p->d_err) {
        VP_CUDA(p, cudaMalloc(&p->d_err, sizeof(int)));
        VP_CUDA(p, cudaMemset(p->d_err, 0, sizeof(int)));
      }
      VP_CUDA(p, tc_build_bmat(p->n2, split, p->tcB, p->stream));
      VP_CUDA(p, cudaStreamSynchronize(p->stream));
      p->tc_split = split;
    }
  }
  p->prec = precision;
  return VP_OK;
}

vp_status vp_plan_set_grad_mode(vp_plan p, vp_grad_mode mode) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (mode != VP_GRAD_EXACT && mode != VP_GRAD_SPECTRAL2N) return fail(p, VP_ERR_INVALID_ARG, "unknown gradient mode");
  p->gmode = mode;
  return VP_OK;
}

vp_status vp_apply(vp_plan p, const void* f, void* phi, vp_dtype dtype) {
  vp::NvtxRange range("vp_apply");
  return apply_common(p, f, phi, nullptr, dtype, false);
}

vp_status vp_apply_pipeline(vp_plan p, int count, const void* const* f, void* const* phi, void* const* grad,
                            vp_dtype dtype) {
  vp::NvtxRange range("vp_apply_pipeline");
  return apply_pipeline(p, count, f, phi, grad, dtype);
}

vp_status vp_apply_grad(vp_plan p, const void* f, void* phi, void* grad, vp_dtype dtype) {
  vp::NvtxRange range("vp_apply_grad");
  return apply_common(p, f, phi, grad, dtype, true);
}

vp_status vp_plan_get_array(vp_plan p, vp_array which, int axis, double* host_dst, size_t count) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (!host_dst) return fail(p, VP_ERR_INVALID_ARG, "host_dst is NULL");
  if (count < (size_t)(2 * p->oct)) return fail(p, VP_ERR_INVALID_ARG, "host buffer too small");
  const double2* src = nullptr;
  if (which == VP_ARRAY_T) {
    src = p->T64;
  } else if (which == VP_ARRAY_GHAT) {
    src = p->G64u;
  } else if (which == VP_ARRAY_TJ || which == VP_ARRAY_GHATJ) {
    if (axis < 0 || axis >= p->d) return fail(p, VP_ERR_INVALID_ARG, "axis out of range");
    VP_ON_DEVICE(p, p->device);
    vp_status st = build_grad(p);
    if (st != VP_OK) return st;
    src = which == VP_ARRAY_TJ ? p->Tj64[axis] : p->Gj64u[axis];
  } else {
    return fail(p, VP_ERR_INVALID_ARG, "unknown array");
  }
  VP_ON_DEVICE(p, p->device);
  VP_CUDA(p, cudaStreamSynchronize(p->stream));
  VP_CUDA(p, cudaMemcpy(host_dst, src, p->oct * sizeof(double2), cudaMemcpyDeviceToHost));
  return VP_OK;
}

vp_status vp_plan_info(vp_plan p, int* d, int* N, double* k, double* L, size_t* device_bytes) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (d) *d = p->d;
  if (N) *N = p->N;
  if (k) *k = p->k;
  if (L) *L = p->L;
  if (device_bytes) *device_bytes = p->device_bytes;
  return VP_OK;
}

vp_status vp_plan_set_timing(vp_plan p, int enable) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  p->timing = enable != 0;
  return VP_OK;
}

vp_status vp_plan_get_timing(vp_plan p, int cap, int* npass, const char** names, int* launches, double* total_ms) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  if (cap < 0) return fail(p, VP_ERR_INVALID_ARG, "cap < 0");
  VP_ON_DEVICE(p, p->device);
  VP_CUDA(p, cudaStreamSynchronize(p->stream));
  double sums[NPASS] = {0};
  int counts[NPASS] = {0};
  for (const TimedLaunch& t : p->timed) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
      sums[t.pass] += ms;
      counts[t.pass] += 1;
    }
    p->event_pool.push_back(t.start);
    p->event_pool.push_back(t.stop);
  }
  p->timed.clear();
  if (npass) *npass = NPASS;
  for (int i = 0; i < NPASS && i < cap; ++i) {
    if (names) names[i] = kPassNames[i];
    if (launches) launches[i] = counts[i];
    if (total_ms) total_ms[i] = sums[i];
  }
  return VP_OK;
}

vp_status vp_plan_launch_count(vp_plan p, int grad, int* launches) {
  if (!p || !launches) return fail(p, VP_ERR_INVALID_ARG, "NULL argument");
  (void)grad;
  *launches = (p->d == 3) ? 5 : 3;
  return VP_OK;
}

vp_status vp_plan_status(vp_plan p) {
  if (!p) return fail(nullptr, VP_ERR_INVALID_ARG, "plan is NULL");
  VP_ON_DEVICE(p, p->device);
  VP_CUDA(p, cudaStreamSynchronize(p->stream));
  VP_CUDA(p, cudaGetLastError());
  if (p->d_err) {
    int h = 0;
    VP_CUDA(p, cudaMemcpy(&h, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) {
      VP_CUDA(p, cudaMemset(p->d_err, 0, sizeof(int)));
      return fail(p, VP_ERR_TIMEOUT, "a bounded wait in a pass kernel (tensor-core or TMA pipeline) timed out");
    }
  }
  return VP_OK;
}

const char* vp_last_error(vp_plan p) { return p ? p->last_error.c_str() : g_thread_error.c_str(); }

const char* vp_status_string(vp_status s) {
  switch (s) {
    case VP_OK: return "VP_OK";
    case VP_ERR_INVALID_ARG: return "VP_ERR_INVALID_ARG";
    case VP_ERR_UNSUPPORTED: return "VP_ERR_UNSUPPORTED";
    case VP_ERR_OOM: return "VP_ERR_OOM";
    case VP_ERR_CUDA: return "VP_ERR_CUDA";
    case VP_ERR_TIMEOUT: return "VP_ERR_TIMEOUT";
    case VP_ERR_NUMERICAL: return "VP_ERR_NUMERICAL";
  }
  return "unknown status";
}

vp_status vp_destroy(vp_plan p) {
  if (!p) return VP_OK;
  vp::DeviceGuard dg_(p->device);
  if (p->stream) cudaStreamSynchronize(p->stream);
  cudaFree(p->T64);
  cudaFree(p->T32);
  cudaFree(p->G64u);
  cudaFree(p->G64);
  cudaFree(p->G32);
  for (int j = 0; j < 3; ++j) {
    cudaFree(p->Tj64[j]);
    cudaFree(p->Tj32[j]);
    cudaFree(p->Gj64u[j]);
    cudaFree(p->Gj64[j]);
    cudaFree(p->Gj32[j]);
  }
  for (int a = 0; a < 3; ++a) {
    bool dup = false;
    for (int b = 0; b < a; ++b) dup = dup || p->twv64[b] == p->twv64[a];
    if (!dup) {
      cudaFree(p->twv64[a]);
      cudaFree(p->twv32[a]);
    }
  }
  cudaFree(p->tcB);
  cudaFree(p->d_err);
  cudaFree(p->d_flag);
  cudaFree(p->ws);
  cudaFree(p->stage);
  if (p->pipe_h2d) cudaStreamSynchronize(p->pipe_h2d);
  if (p->pipe_d2h) cudaStreamSynchronize(p->pipe_d2h);
  cudaFree(p->pipe_buf);
  if (p->pipe_h2d) cudaStreamDestroy(p->pipe_h2d);
  if (p->pipe_d2h) cudaStreamDestroy(p->pipe_d2h);
  if (p->pipe_start) cudaEventDestroy(p->pipe_start);
  for (int s = 0; s < 3; ++s)
    for (int e = 0; e < 3; ++e)
      if (p->pipe_ev[s][e]) cudaEventDestroy(p->pipe_ev[s][e]);
  for (const TimedLaunch& t : p->timed) {
    cudaEventDestroy(t.start);
    cudaEventDestroy(t.stop);
  }
  for (cudaEvent_t e : p->event_pool) cudaEventDestroy(e);
  delete p;
  return VP_OK;
}

}  // extern "C"
