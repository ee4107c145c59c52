// Level-1 vector kernels on one-parity spinor fields and the CG scalar
// recurrences.
//
// All precisions share one element order (see dwf_internal.h), so kernels
// whose output is FP64 or FP32 stream the fields chunk by chunk (4 reals: the
// re and im parts of one complex component of a slice pair), whatever the
// input precisions.  An FP16 output needs the largest component of each slice
// for its scale, so those kernels walk whole slice pairs (h, j) instead.
// Reductions are deterministic: per-block partials, then one block sums them
// in a fixed order.  Per-chunk sums of squares are formed in the data's own
// precision (FP64 issue rate is low on GB300) and accumulated in FP64.
#include "dwf_internal.h"

namespace dwf {

namespace {

template <class S> CFieldRef<S> cr(const Field& f) { return CFieldRef<S>{reinterpret_cast<const S*>(f.v), f.norm}; }
template <class S> FieldRef<S> wr(const Field& f) { return FieldRef<S>{reinterpret_cast<S*>(f.v), f.norm}; }

int grid_for(long n) {
  long b = (n + kBlasThreads - 1) / kBlasThreads;
  const long cap = 152L * 16;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

// ---- chunk io: chunk q = (h * 12 + k) * Lh + j holds (re s0, re s1, im s0, im s1)
__device__ __forceinline__ void ld_chunk(CFieldRef<double> f, long q, int, double* v) {
  const double2* p = reinterpret_cast<const double2*>(f.v) + 2 * q;
  const double2 a = __ldg(p), b = __ldg(p + 1);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void ld_chunk(CFieldRef<float> f, long q, int, float* v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(f.v) + q);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void ld_chunk(CFieldRef<__half> f, long q, int Lh, float* v) {
  const long j = q % Lh, h = q / ((long)12 * Lh);
  const float2 sc = __ldg(reinterpret_cast<const float2*>(f.norm) + h * Lh + j);
  const uint2 a = __ldg(reinterpret_cast<const uint2*>(f.v) + q);
  const float2 r = __half22float2(*reinterpret_cast<const __half2*>(&a.x));
  const float2 i = __half22float2(*reinterpret_cast<const __half2*>(&a.y));
  v[0] = r.x * sc.x;
  v[1] = r.y * sc.y;
  v[2] = i.x * sc.x;
  v[3] = i.y * sc.y;
}
__device__ __forceinline__ void st_chunk(FieldRef<double> f, long q, const double* v) {
  double2* p = reinterpret_cast<double2*>(f.v) + 2 * q;
  p[0] = make_double2(v[0], v[1]);
  p[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void st_chunk(FieldRef<float> f, long q, const float* v) {
  reinterpret_cast<float4*>(f.v)[q] = make_float4(v[0], v[1], v[2], v[3]);
}

// ---- norm
template <class S>
__global__ void __launch_bounds__(kBlasThreads) k_norm2(CFieldRef<S> x, long nq, int Lh, double* partials) {
  __shared__ double red[32];
  typedef typename Store<S>::calc_t C;
  double acc = 0.0;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long)gridDim.x * blockDim.x) {
    C v[4];
    ld_chunk(x, q, Lh, v);
    acc += (double)(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
  }
  double t = block_sum<kBlasThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---- y = a x + b y  (y FP64 / FP32)
template <class SX, class SY>
__global__ void __launch_bounds__(kBlasThreads) k_axpby_c(double a, CFieldRef<SX> x, double b, FieldRef<SY> y,
                                                         long nq, int Lh, int read_y) {
  typedef typename Store<SY>::calc_t CY;
  typedef typename Store<SX>::calc_t CX;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (long)gridDim.x * blockDim.x) {
    CX xv[4] = {0, 0, 0, 0};
    CY yv[4] = {0, 0, 0, 0};
    if (a != 0.0) ld_chunk(x, q, Lh, xv);
    if (read_y) ld_chunk(CFieldRef<SY>{y.v, y.norm}, q, Lh, yv);
#pragma unroll
    for (int e = 0; e < 4; ++e) yv[e] = (CY)(a * (double)xv[e] + b * (double)yv[e]);
    st_chunk(y, q, yv);
  }
}

// ---- y = a x + b y  (y FP16: whole slice pairs)
template <class SX>
__global__ void __launch_bounds__(kBlasThreads) k_axpby_p(double a, CFieldRef<SX> x, double b, FieldRef<__half> y,
                                                         long npairs, int Lh, int read_y) {
  typedef typename Store<SX>::calc_t CX;
  for (long pi = (long)blockIdx.x * blockDim.x + threadIdx.x; pi < npairs; pi += (long)gridDim.x * blockDim.x) {
    const long h = pi / Lh;
    const int j = (int)(pi - h * Lh);
    float2 re[12], im[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const long q = (h * 12 + k) * Lh + j;
      CX xv[4] = {0, 0, 0, 0};
      float yv[4] = {0, 0, 0, 0};
      if (a != 0.0) ld_chunk(x, q, Lh, xv);
      if (read_y) ld_chunk(CFieldRef<__half>{y.v, y.norm}, q, Lh, yv);
      float o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = (float)(a * (double)xv[e] + b * (double)yv[e]);
      re[k] = make_float2(o[0], o[1]);
      im[k] = make_float2(o[2], o[3]);
    }
    store_pair(y, h, j, Lh, re, im);
  }
}

// ---- r -= alpha q; partial |r|^2   (the CG residual update; x moves with p below)
template <class S>
__global__ void __launch_bounds__(kBlasThreads) k_cg_r_c(const double* alpha, CFieldRef<S> q, FieldRef<S> r, long nq,
                                                        int Lh, double* partials) {
  __shared__ double red[32];
  typedef typename Store<S>::calc_t C;
  const C a = (C)(*alpha);
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (long)gridDim.x * blockDim.x) {
    C qv[4], rv[4];
    ld_chunk(q, i, Lh, qv);
    ld_chunk(CFieldRef<S>{r.v, r.norm}, i, Lh, rv);
    C ps = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      rv[e] = fma(-a, qv[e], rv[e]);
      ps = fma(rv[e], rv[e], ps);
    }
    st_chunk(r, i, rv);
    acc += (double)ps;
  }
  double t = block_sum<kBlasThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(kBlasThreads) k_cg_r_p(const double* alpha, CFieldRef<__half> q, FieldRef<__half> r,
                                                        long npairs, int Lh, double* partials) {
  __shared__ double red[32];
  const float a = (float)(*alpha);
  double acc = 0.0;
  for (long pi = (long)blockIdx.x * blockDim.x + threadIdx.x; pi < npairs; pi += (long)gridDim.x * blockDim.x) {
    const long h = pi / Lh;
    const int j = (int)(pi - h * Lh);
    float2 re[12], im[12];
    float ps = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const long c = (h * 12 + k) * Lh + j;
      float qv[4], rv[4];
      ld_chunk(q, c, Lh, qv);
      ld_chunk(CFieldRef<__half>{r.v, r.norm}, c, Lh, rv);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        rv[e] = fmaf(-a, qv[e], rv[e]);
        ps = fmaf(rv[e], rv[e], ps);
      }
      re[k] = make_float2(rv[0], rv[1]);
      im[k] = make_float2(rv[2], rv[3]);
    }
    store_pair(r, h, j, Lh, re, im);
    acc += (double)ps;
  }
  double t = block_sum<kBlasThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// ---- x += alpha p; p = s + beta p   (x may be stored at a higher precision)
template <class S, class SX>
__global__ void __launch_bounds__(kBlasThreads) k_cg_xp_c(const double* alpha, const double* beta, CFieldRef<S> sv,
                                                         FieldRef<S> p, FieldRef<SX> x, long nq, int Lh) {
  typedef typename Store<S>::calc_t C;
  typedef typename Store<SX>::calc_t CX;
  const C a = (C)(*alpha), b = (C)(*beta);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += (long)gridDim.x * blockDim.x) {
    C sw[4], pv[4];
    CX xv[4];
    ld_chunk(sv, i, Lh, sw);
    ld_chunk(CFieldRef<S>{p.v, p.norm}, i, Lh, pv);
    ld_chunk(CFieldRef<SX>{x.v, x.norm}, i, Lh, xv);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      xv[e] = fma((CX)a, (CX)pv[e], xv[e]);
      pv[e] = fma(b, pv[e], sw[e]);
    }
    st_chunk(x, i, xv);
    st_chunk(p, i, pv);
  }
}

__global__ void __launch_bounds__(kBlasThreads) k_cg_xp_p(const double* alpha, const double* beta,
                                                         CFieldRef<__half> sv, FieldRef<__half> p, FieldRef<float> x,
                                                         long npairs, int Lh) {
  const float a = (float)(*alpha), b = (float)(*beta);
  for (long pi = (long)blockIdx.x * blockDim.x + threadIdx.x; pi < npairs; pi += (long)gridDim.x * blockDim.x) {
    const long h = pi / Lh;
    const int j = (int)(pi - h * Lh);
    float2 re[12], im[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const long c = (h * 12 + k) * Lh + j;
      float sw[4], pv[4], xv[4];
      ld_chunk(sv, c, Lh, sw);
      ld_chunk(CFieldRef<__half>{p.v, p.norm}, c, Lh, pv);
      ld_chunk(CFieldRef<float>{x.v, x.norm}, c, Lh, xv);
#pragma unroll
      for (int e = 0; e < 4; ++e) xv[e] = fmaf(a, pv[e], xv[e]);
      st_chunk(x, c, xv);
      re[k] = make_float2(fmaf(b, pv[0], sw[0]), fmaf(b, pv[1], sw[1]));
      im[k] = make_float2(fmaf(b, pv[2], sw[2]), fmaf(b, pv[3], sw[3]));
    }
    store_pair(p, h, j, Lh, re, im);
  }
}

__global__ void k_sum(const double* partials, int nb, double* dst) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
  double t = block_sum<1024>(acc, red);
  if (threadIdx.x == 0) *dst = t;
}

__global__ void k_alpha(const double* partials, int nb, double* num, double* den, double* alpha) {
  __shared__ double red[32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += partials[i];
  double t = block_sum<1024>(acc, red);
  if (threadIdx.x == 0) {
    *den = t;
    *alpha = (t > 0.0) ? (*num) / t : 0.0;
  }
}

// rr = sum(pr); ss = sum(ps); beta = ss / gam; gam = ss
__global__ void k_beta(const double* pr, int nbr, const double* ps, int nbs, double* rr, double* gam, double* beta) {
  __shared__ double red[32];
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < nbr; i += blockDim.x) a += pr[i];
  for (int i = threadIdx.x; i < nbs; i += blockDim.x) b += ps[i];
  double ta = block_sum<1024>(a, red);
  double tb = block_sum<1024>(b, red);
  if (threadIdx.x == 0) {
    *rr = ta;
    *beta = (*gam > 0.0) ? tb / (*gam) : 0.0;
    *gam = tb;
  }
}

}  // namespace

static long nchunks(const dwf_lattice* L) { return field_elems(L) / 4; }
static long npairs(const dwf_lattice* L) { return L->Vh * L->Lh; }

dwf_status blas_norm2(dwf_lattice* L, Field x, double* partials, int* nb) {
  const long n = nchunks(L);
  const int g = grid_for(n);
  switch (x.prec) {
    case DWF_F64: k_norm2<double><<<g, kBlasThreads, 0, L->stream>>>(cr<double>(x), n, L->Lh, partials); break;
    case DWF_F32: k_norm2<float><<<g, kBlasThreads, 0, L->stream>>>(cr<float>(x), n, L->Lh, partials); break;
    case DWF_F16: k_norm2<__half><<<g, kBlasThreads, 0, L->stream>>>(cr<__half>(x), n, L->Lh, partials); break;
  }
  *nb = g;
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status blas_sum(dwf_lattice* L, const double* partials, int nb, double* dst) {
  k_sum<<<1, 1024, 0, L->stream>>>(partials, nb, dst);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

template <class SX>
static void axpby_x(dwf_lattice* L, double a, Field x, double b, Field y, int read_y) {
  const long nq = nchunks(L), np = npairs(L);
  switch (y.prec) {
    case DWF_F64:
      k_axpby_c<SX, double><<<grid_for(nq), kBlasThreads, 0, L->stream>>>(a, cr<SX>(x), b, wr<double>(y), nq, L->Lh,
                                                                          read_y);
      break;
    case DWF_F32:
      k_axpby_c<SX, float><<<grid_for(nq), kBlasThreads, 0, L->stream>>>(a, cr<SX>(x), b, wr<float>(y), nq, L->Lh,
                                                                         read_y);
      break;
    case DWF_F16:
      k_axpby_p<SX><<<grid_for(np), kBlasThreads, 0, L->stream>>>(a, cr<SX>(x), b, wr<__half>(y), np, L->Lh, read_y);
      break;
  }
}

static dwf_status axpby_any(dwf_lattice* L, double a, Field x, double b, Field y, int read_y) {
  switch (x.prec) {
    case DWF_F64: axpby_x<double>(L, a, x, b, y, read_y); break;
    case DWF_F32: axpby_x<float>(L, a, x, b, y, read_y); break;
    case DWF_F16: axpby_x<__half>(L, a, x, b, y, read_y); break;
  }
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status blas_axpby(dwf_lattice* L, double a, Field x, double b, Field y) { return axpby_any(L, a, x, b, y, 1); }
dwf_status blas_copy(dwf_lattice* L, Field x, Field y) { return axpby_any(L, 1.0, x, 0.0, y, 0); }
dwf_status blas_zero(dwf_lattice* L, Field x) { return axpby_any(L, 0.0, x, 0.0, x, 0); }
dwf_status blas_accum(dwf_lattice* L, Field x, Field y) { return axpby_any(L, 1.0, x, 1.0, y, 1); }

dwf_status blas_cg_r(dwf_lattice* L, const double* alpha, Field q, Field r, double* partials, int* nb) {
  const long nq = nchunks(L), np = npairs(L);
  if (q.prec != r.prec) return fail(L, DWF_ERR_INVALID_ARG, "cg_r: mixed precisions");
  int g;
  switch (r.prec) {
    case DWF_F64:
      g = grid_for(nq);
      k_cg_r_c<double><<<g, kBlasThreads, 0, L->stream>>>(alpha, cr<double>(q), wr<double>(r), nq, L->Lh, partials);
      break;
    case DWF_F32:
      g = grid_for(nq);
      k_cg_r_c<float><<<g, kBlasThreads, 0, L->stream>>>(alpha, cr<float>(q), wr<float>(r), nq, L->Lh, partials);
      break;
    default:
      g = grid_for(np);
      k_cg_r_p<<<g, kBlasThreads, 0, L->stream>>>(alpha, cr<__half>(q), wr<__half>(r), np, L->Lh, partials);
      break;
  }
  *nb = g;
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status blas_cg_xp(dwf_lattice* L, const double* alpha, const double* beta, Field s, Field p, Field x) {
  const long nq = nchunks(L), np = npairs(L);
  if (s.prec != p.prec) return fail(L, DWF_ERR_INVALID_ARG, "cg_xp: mixed precisions");
  if (p.prec == DWF_F64 && x.prec == DWF_F64) {
    k_cg_xp_c<double, double><<<grid_for(nq), kBlasThreads, 0, L->stream>>>(alpha, beta, cr<double>(s),
                                                                             wr<double>(p), wr<double>(x), nq, L->Lh);
  } else if (p.prec == DWF_F32 && x.prec == DWF_F32) {
    k_cg_xp_c<float, float><<<grid_for(nq), kBlasThreads, 0, L->stream>>>(alpha, beta, cr<float>(s), wr<float>(p),
                                                                           wr<float>(x), nq, L->Lh);
  } else if (p.prec == DWF_F16 && x.prec == DWF_F32) {
    k_cg_xp_p<<<grid_for(np), kBlasThreads, 0, L->stream>>>(alpha, beta, cr<__half>(s), wr<__half>(p), wr<float>(x),
                                                             np, L->Lh);
  } else {
    return fail(L, DWF_ERR_INVALID_ARG, "cg_xp: unsupported precision pair");
  }
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status scal_alpha(dwf_lattice* L, const double* partials, int nb, double* num, double* den, double* alpha) {
  k_alpha<<<1, 1024, 0, L->stream>>>(partials, nb, num, den, alpha);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status scal_beta(dwf_lattice* L, const double* pr, int nbr, const double* ps, int nbs, double* rr, double* gam,
                     double* beta) {
  k_beta<<<1, 1024, 0, L->stream>>>(pr, nbr, ps, nbs, rr, gam, beta);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

}  // namespace dwf
