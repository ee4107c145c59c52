// Internal declarations of the GB300 domain-wall library (not part of the ABI).
//
// Internal layouts (one checkerboard, "half" lattice of Vh = V4/2 sites):
//   spinor  : chunks of 16 bytes, index ((h * NC + c) * Ls + s), s fastest, so
//             the Ls threads of a 4D site read consecutive 16-byte words.
//             FP64: NC = 12 chunks of one complex; FP32: NC = 6 chunks of two
//             complex; FP16: NC = 3 chunks of four complex plus one float
//             scale per (h, s).  Complex component k = spin * 3 + colour.
//   links   : per output parity, [Vh][8][18] reals: directions 0..3 are
//             U_mu(n), 4..7 are U_mu(n - mu)^+, t boundary phase folded in.
//   nbr     : per output parity, int32 [8][Vh] half-site index of the
//             neighbour n + mu (d < 4) or n - mu (d >= 4) on the other parity.
//   s-ops   : fifth-dimension operators, two real Ls x Ls matrices
//             (P+ block, P- block), row-major, in FP64 and FP32.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <deque>
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
  typedef double2 chunk_t;
  typedef double calc_t;
  static constexpr int NC = 12;
  static constexpr int PER = 1;  // complex per chunk
};
template <> struct Store<float> {
  typedef float4 chunk_t;
  typedef float calc_t;
  static constexpr int NC = 6;
  static constexpr int PER = 2;
};
template <> struct Store<__half> {
  typedef uint4 chunk_t;
  typedef float calc_t;
  static constexpr int NC = 3;
  static constexpr int PER = 4;
};

// A one-parity spinor field of storage type S.
template <class S> struct FieldRef {
  typename Store<S>::chunk_t* v;
  float* norm;  // FP16 only: per (h, s) scale
};
template <class S> struct CFieldRef {
  const typename Store<S>::chunk_t* v;
  const float* norm;
};

// ---------------------------------------------------------------- spinor io

__device__ __forceinline__ void load_chunk(const double2* p, double* out) {
  double2 a = __ldg(p);
  out[0] = a.x;
  out[1] = a.y;
}
__device__ __forceinline__ void load_chunk(const float4* p, float* out) {
  float4 a = __ldg(p);
  out[0] = a.x;
  out[1] = a.y;
  out[2] = a.z;
  out[3] = a.w;
}

// Load the 24 reals of spinor (h, s).
template <class S>
__device__ __forceinline__ void load_spinor(CFieldRef<S> f, long h, int s, int Ls,
                                            typename Store<S>::calc_t* v) {
  constexpr int NC = Store<S>::NC;
  if constexpr (sizeof(S) == 2) {
    const float sc = __ldg(f.norm + h * Ls + s);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uint4 a = __ldg(f.v + (h * NC + c) * Ls + s);
      const __half2* hp = reinterpret_cast<const __half2*>(&a);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float2 t = __half22float2(hp[j]);
        v[8 * c + 2 * j] = t.x * sc;
        v[8 * c + 2 * j + 1] = t.y * sc;
      }
    }
  } else {
    constexpr int R = 2 * Store<S>::PER;
#pragma unroll
    for (int c = 0; c < NC; ++c) load_chunk(f.v + (h * NC + c) * Ls + s, v + R * c);
  }
}

template <class S>
__device__ __forceinline__ void store_spinor(FieldRef<S> f, long h, int s, int Ls,
                                             const typename Store<S>::calc_t* v) {
  constexpr int NC = Store<S>::NC;
  if constexpr (sizeof(S) == 8) {
#pragma unroll
    for (int c = 0; c < NC; ++c) f.v[(h * NC + c) * Ls + s] = make_double2(v[2 * c], v[2 * c + 1]);
  } else if constexpr (sizeof(S) == 4) {
#pragma unroll
    for (int c = 0; c < NC; ++c)
      f.v[(h * NC + c) * Ls + s] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
  } else {
    float mx = 0.f;
#pragma unroll
    for (int k = 0; k < 24; ++k) mx = fmaxf(mx, fabsf(v[k]));
    // A site whose largest component is below the normal FP32 range is
    // stored as zero (1/mx would overflow and turn exact zeros into NaN).
    const bool keep = mx >= 1.17549435e-38f;
    const float inv = keep ? 1.0f / mx : 0.f;
    f.norm[h * Ls + s] = keep ? mx : 0.f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      uint4 a;
      __half2* hp = reinterpret_cast<__half2*>(&a);
#pragma unroll
      for (int j = 0; j < 4; ++j) hp[j] = __floats2half2_rn(v[8 * c + 2 * j] * inv, v[8 * c + 2 * j + 1] * inv);
      f.v[(h * NC + c) * Ls + s] = a;
    }
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
  int Ls;
  cudaStream_t stream;
  int* nbr[2] = {nullptr, nullptr};
  void* links[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};
  bool gauge_set = false;
  std::deque<dwf::SOps> sops;  // deque: pointers stay valid on growth
  std::map<std::string, dwf::Buffer> ws;
  double* partials = nullptr;  // device, kPartials doubles
  double* scal = nullptr;      // device scalars
  double* hscal = nullptr;     // pinned host mirror
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
constexpr int kScalars = 64;

// error helpers (lattice.cu)
dwf_status fail(dwf_lattice* L, dwf_status st, const std::string& msg);
dwf_status cuda_check(dwf_lattice* L, cudaError_t e, const char* what);
#define DWF_CUDA(L, call)                                           \
  do {                                                              \
    cudaError_t _e = (call);                                        \
    if (_e != cudaSuccess) return ::dwf::cuda_check((L), _e, #call); \
  } while (0)
// after exactly one kernel launch: count it and check the launch
#define DWF_LAUNCHED(L)         \
  do {                          \
    ::dwf::counted(L);          \
    DWF_CUDA(L, cudaGetLastError()); \
  } while (0)
#define DWF_TRY(call)                   \
  do {                                  \
    dwf_status _s = (call);             \
    if (_s != DWF_OK) return _s;        \
  } while (0)

// instrumentation (lattice.cu)
inline void counted(dwf_lattice* L, int n = 1) { L->launches += n; }
dwf_status timing_begin(dwf_lattice* L, cudaEvent_t* a, cudaEvent_t* b);
void timing_end(dwf_lattice* L, int prec, double bytes, cudaEvent_t a, cudaEvent_t b);
dwf_status timing_drain(dwf_lattice* L);  // stream must be idle

// workspace (lattice.cu)
dwf_status ws_get(dwf_lattice* L, const std::string& name, size_t bytes, void** out);
size_t field_bytes(const dwf_lattice* L, dwf_prec prec);  // one parity, excluding FP16 norms
const SOps* sops_for(dwf_lattice* L, double m, dwf_status* st);

// one-parity field handle used by the host drivers
struct Field {
  void* v = nullptr;
  float* norm = nullptr;
  dwf_prec prec = DWF_F64;
};
dwf_status field_alloc(dwf_lattice* L, const std::string& name, dwf_prec prec, Field* f);

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

// s-local: out = a * E x + bcoef * y   (E may be identity), on one parity
dwf_status launch_sop(dwf_lattice* L, Field x, Field out, const SOps* ops, SOps::Kind e, double a,
                      const Field* y, double bcoef);

// pack / unpack boundary complex128 whole-lattice spinors <-> one-parity fields
dwf_status launch_pack(dwf_lattice* L, const void* boundary, int parity, Field out);
dwf_status launch_unpack(dwf_lattice* L, Field in, int parity, void* boundary, bool zero_other);
dwf_status launch_pack_gauge(dwf_lattice* L, const void* U);

// blas.cu (all on one-parity fields of L; n = Vh * Ls * 24 reals)
// Reductions write per-block partials; finalise with launch_sum.
dwf_status blas_norm2(dwf_lattice* L, Field x, double* partials, int* nb);
dwf_status blas_sum(dwf_lattice* L, const double* partials, int nb, double* dst);  // device dst
dwf_status blas_copy(dwf_lattice* L, Field x, Field y);                             // y = x (any precisions)
dwf_status blas_zero(dwf_lattice* L, Field x);
// y = a*x + b*y with host scalars
dwf_status blas_axpby(dwf_lattice* L, double a, Field x, double b, Field y);
// CG steps with device scalars (pointers into L->scal)
dwf_status blas_cg_xr(dwf_lattice* L, const double* alpha, Field p, Field q, Field x, Field r,
                      double* partials, int* nb);                   // x += a p; r -= a q; |r|^2
dwf_status blas_cg_p(dwf_lattice* L, const double* beta, Field s, Field p);  // p = s + b p
// add a low-precision field into a FP64 one: y64 += x
dwf_status blas_accum(dwf_lattice* L, Field x, Field y64);
// scalar kernels
dwf_status scal_alpha(dwf_lattice* L, const double* partials, int nb, double* num, double* den, double* alpha);
dwf_status scal_beta(dwf_lattice* L, const double* pr, int nbr, const double* ps, int nbs,
                     double* rr, double* gam, double* beta);

}  // namespace dwf
