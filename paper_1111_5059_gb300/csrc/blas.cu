// Level-1 vector kernels on one-parity spinor fields and the CG scalar
// recurrences.  Every kernel walks the (h, s) sites with a grid-stride loop;
// each thread loads and stores whole 24-real spinors through the storage
// traits, so FP64, FP32 and FP16 (scaled) fields share one code path.
// Reductions are deterministic: FP64 per-block partials, then one block sums
// them in a fixed order.
#include "dwf_internal.h"

namespace dwf {

namespace {

template <class S> CFieldRef<S> cr(const Field& f) {
  return CFieldRef<S>{reinterpret_cast<const typename Store<S>::chunk_t*>(f.v), f.norm};
}
template <class S> FieldRef<S> wr(const Field& f) {
  return FieldRef<S>{reinterpret_cast<typename Store<S>::chunk_t*>(f.v), f.norm};
}

int grid_for(long n) {
  long b = (n + kBlasThreads - 1) / kBlasThreads;
  const long cap = 152L * 16;
  return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <class S>
__global__ void __launch_bounds__(kBlasThreads) k_norm2(CFieldRef<S> x, long n, int Ls, double* partials) {
  __shared__ double red[32];
  typedef typename Store<S>::calc_t C;
  double acc = 0.0;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const long h = q / Ls;
    const int s = (int)(q - h * Ls);
    C v[24];
    load_spinor<S>(x, h, s, Ls, v);
    C ps = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) ps = fma(v[k], v[k], ps);
    acc += (double)ps;
  }
  double t = block_sum<kBlasThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

template <class SX, class SY>
__global__ void __launch_bounds__(kBlasThreads) k_axpby(double a, CFieldRef<SX> x, double b, FieldRef<SY> y,
                                                       long n, int Ls, int read_y) {
  typedef typename Store<SX>::calc_t CX;
  typedef typename Store<SY>::calc_t CY;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
    const long h = q / Ls;
    const int s = (int)(q - h * Ls);
    CX xv[24];
    CY yv[24];
    if (a != 0.0) load_spinor<SX>(x, h, s, Ls, xv);
    if (read_y) {
      load_spinor<SY>(CFieldRef<SY>{y.v, y.norm}, h, s, Ls, yv);
    }
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      CY r = 0;
      if (read_y) r = (CY)(b * (double)yv[k]);
      if (a != 0.0) r += (CY)(a * (double)xv[k]);
      yv[k] = r;
    }
    store_spinor<SY>(y, h, s, Ls, yv);
  }
}

// x += alpha p;  r -= alpha q;  partial |r|^2.  The solution accumulator x
// may be stored at a higher precision (SX) than the iterated vectors (S).
template <class S, class SX>
__global__ void __launch_bounds__(kBlasThreads) k_cg_xr(const double* alpha, CFieldRef<S> p, CFieldRef<S> q,
                                                       FieldRef<SX> x, FieldRef<S> r, long n, int Ls,
                                                       double* partials) {
  __shared__ double red[32];
  typedef typename Store<S>::calc_t C;
  typedef typename Store<SX>::calc_t CX;
  const C a = (C)(*alpha);
  double acc = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long h = i / Ls;
    const int s = (int)(i - h * Ls);
    C pv[24], qv[24], rv[24];
    CX xv[24];
    load_spinor<S>(p, h, s, Ls, pv);
    load_spinor<S>(q, h, s, Ls, qv);
    load_spinor<SX>(CFieldRef<SX>{x.v, x.norm}, h, s, Ls, xv);
    load_spinor<S>(CFieldRef<S>{r.v, r.norm}, h, s, Ls, rv);
#pragma unroll
    for (int k = 0; k < 24; ++k) {
      xv[k] = fma((CX)a, (CX)pv[k], xv[k]);
      rv[k] = fma(-a, qv[k], rv[k]);
    }
    store_spinor<SX>(x, h, s, Ls, xv);
    store_spinor<S>(r, h, s, Ls, rv);
    C ps = 0;
#pragma unroll
    for (int k = 0; k < 24; ++k) ps = fma(rv[k], rv[k], ps);
    acc += (double)ps;
  }
  double t = block_sum<kBlasThreads>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// p = s + beta p
template <class S>
__global__ void __launch_bounds__(kBlasThreads) k_cg_p(const double* beta, CFieldRef<S> sv, FieldRef<S> p,
                                                      long n, int Ls) {
  typedef typename Store<S>::calc_t C;
  const C b = (C)(*beta);
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long h = i / Ls;
    const int s = (int)(i - h * Ls);
    C a[24], c[24];
    load_spinor<S>(sv, h, s, Ls, a);
    load_spinor<S>(CFieldRef<S>{p.v, p.norm}, h, s, Ls, c);
#pragma unroll
    for (int k = 0; k < 24; ++k) c[k] = fma(b, c[k], a[k]);
    store_spinor<S>(p, h, s, Ls, c);
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
__global__ void k_beta(const double* pr, int nbr, const double* ps, int nbs, double* rr, double* gam,
                       double* beta) {
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

#define DISPATCH1(prec, FN, ...)                            \
  switch (prec) {                                            \
    case DWF_F64: FN<double>(__VA_ARGS__); break;            \
    case DWF_F32: FN<float>(__VA_ARGS__); break;             \
    case DWF_F16: FN<__half>(__VA_ARGS__); break;            \
  }

template <class S> static void norm2_t(dwf_lattice* L, Field x, double* partials, int g) {
  k_norm2<S><<<g, kBlasThreads, 0, L->stream>>>(cr<S>(x), L->Vh * L->Ls, L->Ls, partials);
}

dwf_status blas_norm2(dwf_lattice* L, Field x, double* partials, int* nb) {
  const int g = grid_for(L->Vh * L->Ls);
  DISPATCH1(x.prec, norm2_t, L, x, partials, g);
  *nb = g;
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status blas_sum(dwf_lattice* L, const double* partials, int nb, double* dst) {
  k_sum<<<1, 1024, 0, L->stream>>>(partials, nb, dst);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

template <class SX, class SY>
static void axpby_t(dwf_lattice* L, double a, Field x, double b, Field y, int read_y) {
  const long n = L->Vh * L->Ls;
  k_axpby<SX, SY><<<grid_for(n), kBlasThreads, 0, L->stream>>>(a, cr<SX>(x), b, wr<SY>(y), n, L->Ls, read_y);
}

template <class SX>
static void axpby_x(dwf_lattice* L, double a, Field x, double b, Field y, int read_y) {
  switch (y.prec) {
    case DWF_F64: axpby_t<SX, double>(L, a, x, b, y, read_y); break;
    case DWF_F32: axpby_t<SX, float>(L, a, x, b, y, read_y); break;
    case DWF_F16: axpby_t<SX, __half>(L, a, x, b, y, read_y); break;
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
dwf_status blas_accum(dwf_lattice* L, Field x, Field y64) { return axpby_any(L, 1.0, x, 1.0, y64, 1); }

template <class S, class SX>
static void cg_xr_t(dwf_lattice* L, const double* alpha, Field p, Field q, Field x, Field r, double* partials, int g) {
  k_cg_xr<S, SX><<<g, kBlasThreads, 0, L->stream>>>(alpha, cr<S>(p), cr<S>(q), wr<SX>(x), wr<S>(r),
                                                     L->Vh * L->Ls, L->Ls, partials);
}

dwf_status blas_cg_xr(dwf_lattice* L, const double* alpha, Field p, Field q, Field x, Field r, double* partials,
                      int* nb) {
  const int g = grid_for(L->Vh * L->Ls);
  if (p.prec == DWF_F64 && x.prec == DWF_F64) {
    cg_xr_t<double, double>(L, alpha, p, q, x, r, partials, g);
  } else if (p.prec == DWF_F32 && x.prec == DWF_F32) {
    cg_xr_t<float, float>(L, alpha, p, q, x, r, partials, g);
  } else if (p.prec == DWF_F16 && x.prec == DWF_F32) {
    cg_xr_t<__half, float>(L, alpha, p, q, x, r, partials, g);
  } else {
    return fail(L, DWF_ERR_INVALID_ARG, "cg_xr: unsupported precision pair");
  }
  *nb = g;
  DWF_LAUNCHED(L);
  return DWF_OK;
}

template <class S> static void cg_p_t(dwf_lattice* L, const double* beta, Field s, Field p) {
  const long n = L->Vh * L->Ls;
  k_cg_p<S><<<grid_for(n), kBlasThreads, 0, L->stream>>>(beta, cr<S>(s), wr<S>(p), n, L->Ls);
}

dwf_status blas_cg_p(dwf_lattice* L, const double* beta, Field s, Field p) {
  DISPATCH1(p.prec, cg_p_t, L, beta, s, p);
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
