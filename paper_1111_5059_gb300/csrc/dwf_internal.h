// Internal declarations of the GB300 domain-wall library (not part of the ABI).
//
// Internal layouts (one checkerboard, "half" lattice of Vh = V4/2 sites):
//   spinor  : the Ls slices of a 4D site are split into Lh = ceil(Ls/2) pairs
//             of neighbouring slices (2j, 2j + 1).  Element order [h][k][j][4]
//             with the 4 elements (re s0, re s1, im s0, im s1), s0 = 2j,
//             s1 = 2j + 1, complex component k = spin * 3 + colour (spins 0,1
//             = P+ half).  One 16-byte FP32 chunk therefore holds one complex
//             component of two slices, so a thread owning the pair (h, j)
//             computes both slices with packed FP32x2 instructions, the Ls / 2
//             threads of a site read consecutive chunks, and the slice
//             recurrences of the fifth-dimension operators pass one value
//             between neighbouring threads.  All precisions share the element
//             order (FP64: 32-byte chunks; FP16: 8-byte chunks plus one FP32
//             scale per (h, slice), stored [h][j][2]), so precision casts and
//             level-1 kernels are flat element-wise loops.  For odd Ls the
//             slot s1 = Ls of the last pair is padding and is kept zero.
//   links   : per output parity, [Vh][8][18] reals: directions 0..3 are
//             U_mu(n), 4..7 are U_mu(n - mu)^+, t boundary phase folded in.
//             The FP32 pipelined kernel reads a second, direction-major copy
//             [8][Vh][20] (links_dm), so one direction of consecutive sites
//             is one contiguous run.
//   nbr     : per output parity, int32 [8][Vh] half-site index of the
//             neighbour n + mu (d < 4) or n - mu (d >= 4) on the other parity.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
#include <functional>
#include <map>
#include <string>
#include <vector>

#include "../../include/dwf.h"

namespace dwf {

constexpr int kMaxLs = 64;
constexpr int kBlasThreads = 256;

// ---------------------------------------------------------------- storage traits

template <class S> struct Store;
template <> struct Store<double> {
  typedef double calc_t;
};
template <> struct Store<float> {
  typedef float calc_t;
};
template <> struct Store<__half> {
  typedef float calc_t;
};

// A one-parity spinor field of storage type S (norm: FP16 only, [Vh][Lh][2]).
template <class S> struct FieldRef {
  S* v;
  float* norm;
};
template <class S> struct CFieldRef {
  const S* v;
  const float* norm;
};

__device__ __forceinline__ float to_f(__half x) { return __half2float(x); }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ double to_f(double x) { return x; }

// ---------------------------------------------------------------- per-slice spinor io
// (h, s) access: 24 reals of slice s of site h; used by the kernels that are not
// bandwidth-critical (packing, s-local operators, the FP64 hop).

__host__ __device__ __forceinline__ long elem_index(long h, int k, int j, int Lh) {
  return (((long)h * 12 + k) * Lh + j) * 4;
}

template <class S>
__device__ __forceinline__ void load_spinor(CFieldRef<S> f, long h, int s, int Lh,
                                            typename Store<S>::calc_t* v) {
  typedef typename Store<S>::calc_t C;
  const int half = s & 1;
  const int j = s >> 1;
  const S* base = f.v + elem_index(h, 0, j, Lh) + half;
  C sc = 1;
  if constexpr (sizeof(S) == 2) sc = __ldg(f.norm + ((long)h * Lh + j) * 2 + half);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[2 * k] = (C)to_f(base[(long)k * Lh * 4]) * sc;
    v[2 * k + 1] = (C)to_f(base[(long)k * Lh * 4 + 2]) * sc;
  }
}

// FP16: a slice whose largest component is below the normal FP32 range is
// stored as zero (1/max would overflow and turn exact zeros into NaN).
__device__ __forceinline__ float half_scale(float mx, float* inv) {
  const bool keep = mx >= 1.17549435e-38f;
  *inv = keep ? 1.0f / mx : 0.f;
  return keep ? mx : 0.f;
}

template <class S>
__device__ __forceinline__ void store_spinor(FieldRef<S> f, long h, int s, int Lh,
                                             const typename Store<S>::calc_t* v) {
  const int half = s & 1;
  const int j = s >> 1;
  S* base = f.v + elem_index(h, 0, j, Lh) + half;
  if constexpr (sizeof(S) == 2) {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf(v[k]));
    float inv;
    f.norm[((long)h * Lh + j) * 2 + half] = half_scale(mx, &inv);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      base[(long)k * Lh * 4] = __float2half_rn(v[2 * k] * inv);
      base[(long)k * Lh * 4 + 2] = __float2half_rn(v[2 * k + 1] * inv);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      base[(long)k * Lh * 4] = (S)v[2 * k];
      base[(long)k * Lh * 4 + 2] = (S)v[2 * k + 1];
    }
  }
}

// ---------------------------------------------------------------- per-pair io (FP32 arithmetic)
// re[k] = (re s0, re s1), im[k] = (im s0, im s1) of site h, pair j.

__device__ __forceinline__ void load_pair(CFieldRef<float> f, long h, int j, int Lh, float2* re, float2* im) {
  const float4* p = reinterpret_cast<const float4*>(f.v) + ((long)h * 12) * Lh + j;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float4 a = __ldg(p + (long)k * Lh);
    re[k] = make_float2(a.x, a.y);
    im[k] = make_float2(a.z, a.w);
  }
}
__device__ __forceinline__ void load_pair(CFieldRef<__half> f, long h, int j, int Lh, float2* re, float2* im) {
  const uint2* p = reinterpret_cast<const uint2*>(f.v) + ((long)h * 12) * Lh + j;
  const float2 sc = __ldg(reinterpret_cast<const float2*>(f.norm) + (long)h * Lh + j);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const uint2 a = __ldg(p + (long)k * Lh);
    const float2 r = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
    const float2 i = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
    re[k] = make_float2(r.x * sc.x, r.y * sc.y);
    im[k] = make_float2(i.x * sc.x, i.y * sc.y);
  }
}
__device__ __forceinline__ void store_pair(FieldRef<float> f, long h, int j, int Lh, const float2* re,
                                           const float2* im) {
  float4* p = reinterpret_cast<float4*>(f.v) + ((long)h * 12) * Lh + j;
#pragma unroll
  for (int k = 0; k < 12; ++k) p[(long)k * Lh] = make_float4(re[k].x, re[k].y, im[k].x, im[k].y);
}
__device__ __forceinline__ void store_pair(FieldRef<__half> f, long h, int j, int Lh, const float2* re,
                                           const float2* im) {
  float m0 = 0.f, m1 = 0.f;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    m0 = fmaxf(m0, fmaxf(fabsf(re[k].x), fabsf(im[k].x)));
    m1 = fmaxf(m1, fmaxf(fabsf(re[k].y), fabsf(im[k].y)));
  }
  float i0, i1;
  const float n0 = half_scale(m0, &i0), n1 = half_scale(m1, &i1);
  reinterpret_cast<float2*>(f.norm)[(long)h * Lh + j] = make_float2(n0, n1);
  uint2* p = reinterpret_cast<uint2*>(f.v) + ((long)h * 12) * Lh + j;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const __half2 r = __floats2half2_rn(re[k].x * i0, re[k].y * i1);
    const __half2 i = __floats2half2_rn(im[k].x * i0, im[k].y * i1);
    uint2 a;
    a.x = *reinterpret_cast<const unsigned*>(&r);
    a.y = *reinterpret_cast<const unsigned*>(&i);
    p[(long)k * Lh] = a;
  }
}

// Load one SU(3) link (18 reals) of storage type S.
__device__ __forceinline__ void load_link(const double* p, double* u) {
  const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    double2 a = __ldg(q + k);
    u[2 * k] = a.x;
    u[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void load_link(const float* p, float* u) {
  const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float2 a = __ldg(q + k);
    u[2 * k] = a.x;
    u[2 * k + 1] = a.y;
  }
}
__device__ __forceinline__ void load_link(const __half* p, float* u) {
  const __half2* q = reinterpret_cast<const __half2*>(p);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    float2 a = __half22float2(q[k]);
    u[2 * k] = a.x;
    u[2 * k + 1] = a.y;
  }
}

// ---------------------------------------------------------------- reductions

template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    for (int i = 0; i < nw; ++i) r += sh[i];
  }
  return r;  // valid in thread 0
}

// ---------------------------------------------------------------- handle

// y = (g1 + d1 Q)(g2 + d2 Q)^-1 x per chirality (see hop.cu); kind 0 identity,
// 1 structured O(Ls) recurrence, 2 dense Ls x Ls fallback.
struct SOpDesc {
  int kind, trans, has_inv, dense_kind;
  double g1, d1, ginv, rho, m, c0;
};

struct SOps {  // fifth-dimension operators for one mass
  enum Kind { A, AT, AINV, AINVT, B, BT, BINV, BINVT, E1, E1T, E0, E0T, NKIND };
  double m;
  SOpDesc desc[NKIND];
  double* d64;  // device [NKIND][2][Ls][Ls]
  float* d32;
  const double* k64(Kind k, int Ls) const { return d64 + (size_t)k * 2 * Ls * Ls; }
  const float* k32(Kind k, int Ls) const { return d32 + (size_t)k * 2 * Ls * Ls; }
};

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace dwf

struct dwf_lattice {
  dwf_params p;
  int X, Y, Z, T;
  long V4, Vh;
  int Ls, Lh;  // Lh = ceil(Ls / 2) slice pairs
  cudaStream_t stream;
  int* nbr[2] = {nullptr, nullptr};
  void* links[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  // FP32 links direction-major per output parity, [8][Vh][20] floats (9 complex + 8 bytes of
  // padding: the 80-byte rows of consecutive sites are one contiguous, 16-byte aligned copy)
  float* links_dm[2] = {nullptr, nullptr};
  // > 0: hops on FP64 fields compute in FP32 (hop.cu, hop_lp_kernel); set by
  // Fp32StepScope around approximate steps, and by dwf_set_fp64_arithmetic
  int fp64_in_fp32 = 0;
  int fp64_arith = 0;  // dwf_set_fp64_arithmetic: 1 = every FP64-field hop in FP32
  bool gauge_set = false;
  std::deque<dwf::SOps> sops;  // deque: pointers stay valid on growth
  std::map<std::string, dwf::Buffer> ws;
  double* partials = nullptr;  // device, 2 * kPartials doubles
  double* scal = nullptr;      // device scalars
  double* hscal = nullptr;     // pinned host mirror
  int* dev_err = nullptr;      // device error flag (bounded waits that gave up)
  long wait_limit = 1L << 22;  // polls of a hop kernel's consumer wait (dwf_set_wait_limit)
  std::string err;
  // instrumentation
  long long launches = 0;  // every kernel this handle has launched
  bool timing = false;     // bracket hop launches with events
  struct Pending {
    int prec;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_free;
  double t_ms[3] = {0, 0, 0}, t_bytes[3] = {0, 0, 0};
  long long t_n[3] = {0, 0, 0};
};

namespace dwf {

constexpr int kPartials = 1 << 18;
constexpr long kHopWaitLimit = 1L << 22;  // default polls of a bounded device wait
constexpr int kScalars = 256;  // [0, 64): single solves; [64, 64 + 8 DWF_MAX_RHS): multi-RHS
constexpr int kMaxBatch = 8;          // right-hand sides in one hop launch

// error helpers (lattice.cu)
dwf_status fail(dwf_lattice* L, dwf_status st, const std::string& msg);
dwf_status cuda_check(dwf_lattice* L, cudaError_t e, const char* what);
#define DWF_CUDA(L, call)                                            \
  do {                                                               \
    cudaError_t _e = (call);                                         \
    if (_e != cudaSuccess) return ::dwf::cuda_check((L), _e, #call); \
  } while (0)
// after exactly one kernel launch: count it and check the launch
#define DWF_LAUNCHED(L)              \
  do {                               \
    ::dwf::counted(L);               \
    DWF_CUDA(L, cudaGetLastError()); \
  } while (0)
#define DWF_TRY(call)            \
  do {                           \
    dwf_status _s = (call);      \
    if (_s != DWF_OK) return _s; \
  } while (0)

// instrumentation (lattice.cu)
inline void counted(dwf_lattice* L, int n = 1) { L->launches += n; }
dwf_status timing_begin(dwf_lattice* L, cudaEvent_t* a, cudaEvent_t* b);
void timing_end(dwf_lattice* L, int prec, double bytes, cudaEvent_t a, cudaEvent_t b);
dwf_status timing_drain(dwf_lattice* L);  // stream must be idle

// workspace (lattice.cu)
dwf_status ws_get(dwf_lattice* L, const std::string& name, size_t bytes, void** out);
long field_elems(const dwf_lattice* L);                   // reals per one-parity field, incl. padding
size_t field_bytes(const dwf_lattice* L, dwf_prec prec);  // excluding FP16 scales
const SOps* sops_for(dwf_lattice* L, double m, dwf_status* st);
// The structured descriptors of every fifth-dimension operator for mass m
// (kind 0 identity, 1 structured recurrence, 2 needs the dense fallback).
void fifth_descriptors(const dwf_params& p, int Ls, double m, SOpDesc* desc /* [SOps::NKIND] */);

// one-parity field handle used by the host drivers
struct Field {
  void* v = nullptr;
  float* norm = nullptr;
  dwf_prec prec = DWF_F64;
};
// Allocates (first use: zero-filled, so odd-Ls padding starts at zero).
dwf_status field_alloc(dwf_lattice* L, const std::string& name, dwf_prec prec, Field* f);
// Checks and clears the device error flag (after the stream is idle).
dwf_status check_dev_err(dwf_lattice* L);

// ---------------------------------------------------------------- kernels (launchers)

// hop.cu: out = Eout( xscale * Ex x + scale * Dhop_{parity<-1-parity}(in) )
//   Ex / Eout = NKIND means identity; x may be absent (no site term).
//   If partials != null, writes per-block partial sums of |out|^2 and returns
//   the number of blocks in *nblocks.
struct HopCall {
  int out_parity = 0;
  int dag = 0;
  Field in, out, x;
  bool has_x = false;
  SOps::Kind ex = SOps::NKIND, eout = SOps::NKIND;
  const SOps* ops = nullptr;
  double scale = 1.0, xscale = 1.0;
  double* partials = nullptr;
  int* nblocks = nullptr;
};
dwf_status launch_hop(dwf_lattice* L, const HopCall& c);

// Hops on FP64 fields compute in FP32 while one of these is alive (on)
struct Fp32StepScope {
  dwf_lattice* L;
  bool on;
  Fp32StepScope(dwf_lattice* l, bool o) : L(l), on(o) {
    if (on) ++L->fp64_in_fp32;
  }
  ~Fp32StepScope() {
    if (on) --L->fp64_in_fp32;
  }
  Fp32StepScope(const Fp32StepScope&) = delete;
  Fp32StepScope& operator=(const Fp32StepScope&) = delete;
};

// One hop launch over several right-hand sides that share the links: the
// fields and fifth-dimension operators (one mass each) come from the batch,
// everything else from c (c.in / c.out / c.x / c.ops / c.partials unused).
// partials[r] receives right-hand side r's per-block partial sums of |out|^2
// (kPartials doubles each).  ctas_per_sm = 0: as many as fit.  Needs an
// FP32 / FP16 shape the pipelined kernel takes (hop_batch_max).
struct HopBatch {
  int nrhs = 0;
  Field in[kMaxBatch], out[kMaxBatch], x[kMaxBatch];
  const SOps* ops[kMaxBatch] = {};
  double* partials[kMaxBatch] = {};
};
dwf_status launch_hop_batch(dwf_lattice* L, const HopCall& c, const HopBatch& b, int ctas_per_sm);
// largest batch a single launch takes at this Ls and precision (0: none)
int hop_batch_max(int Ls, dwf_prec prec);

// cg.cu: the even-odd solve of D(m) x = b on FP64 parity fields (xe holds the
// guess).  zero_guess: xe is known to be zero (skips the FP64 residual of the
// guess); full_check = false: report the CG residual |b' - M~ x~| / |b| (equal
// to the full one up to rounding) instead of recomputing |b - D x| in FP64.
struct SolveOpts {
  bool zero_guess = false;
  bool full_check = true;
};
dwf_status solve_eo(dwf_lattice* L, double m, Field be, Field bo, Field xe, Field xo, const dwf_cg_params& prm,
                    dwf_stats* st, double* true_res_full, const SolveOpts& opts = SolveOpts());
// lattice.cu: out_e/out_o = D(m) x or D(m)^+ x on FP64 fields
dwf_status apply_D(dwf_lattice* L, const SOps* ops, bool dag, Field xe, Field xo, Field oe, Field oo);

// tune.cu: launch-shape autotuner for batched hops
struct HopShape {
  long Vh;
  int Ls, prec, nrhs, dag, has_x, ex_kind, eout_kind;
  std::string key() const;
};
struct HopChoice {
  int batch = 1;        // right-hand sides per launch
  int ctas_per_sm = 0;  // 0: as many as fit
  double ms = 0.0;      // measured time of the whole step
};
std::vector<HopChoice> hop_candidates(const HopShape& s, int bmax);
// The cached choice for s, or (first time) the fastest candidate: each is run
// through `run` (which must launch the whole step on L->stream) and timed.
dwf_status tune_hop(dwf_lattice* L, const HopShape& s, int bmax, const std::function<dwf_status(const HopChoice&)>& run,
                    HopChoice* choice, double* tune_seconds);

// s-local: out = a * E x + bcoef * y   (E may be identity), on one parity
dwf_status launch_sop(dwf_lattice* L, Field x, Field out, const SOps* ops, SOps::Kind e, double a,
                      const Field* y, double bcoef);

// pack / unpack boundary complex128 whole-lattice spinors <-> one-parity fields
dwf_status launch_pack(dwf_lattice* L, const void* boundary, int parity, Field out);
dwf_status launch_unpack(dwf_lattice* L, Field in, int parity, void* boundary, bool zero_other);
dwf_status launch_pack_gauge(dwf_lattice* L, const void* U);

// blas.cu (one-parity fields of L).  Reductions write per-block partials;
// finalise with blas_sum / scal_*.
dwf_status blas_norm2(dwf_lattice* L, Field x, double* partials, int* nb);
dwf_status blas_sum(dwf_lattice* L, const double* partials, int nb, double* dst);  // device dst
dwf_status blas_copy(dwf_lattice* L, Field x, Field y);                             // y = x (any precisions)
dwf_status blas_zero(dwf_lattice* L, Field x);
// y = a*x + b*y with host scalars (any precisions)
dwf_status blas_axpby(dwf_lattice* L, double a, Field x, double b, Field y);
// CG steps with device scalars (pointers into L->scal)
// r -= alpha q with partial sums of |r|^2 (q, r same precision)
dwf_status blas_cg_r(dwf_lattice* L, const double* alpha, Field q, Field r, double* partials, int* nb);
// x += alpha p; p = s + beta p  (the solution moves with the old direction in the same pass)
dwf_status blas_cg_xp(dwf_lattice* L, const double* alpha, const double* beta, Field s, Field p, Field x);
// add a lower-precision field into another: y += x
dwf_status blas_accum(dwf_lattice* L, Field x, Field y);
// scalar kernels
dwf_status scal_alpha(dwf_lattice* L, const double* partials, int nb, double* num, double* den, double* alpha);
dwf_status scal_beta(dwf_lattice* L, const double* pr, int nbr, const double* ps, int nbs, double* rr,
                     double* gam, double* beta);

}  // namespace dwf
