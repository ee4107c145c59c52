// 4D Wilson hop at every fifth-dimension slice, with fused s-local epilogues.
//
//   out(n,.) = Eout( xscale * Ex x(n,.) + scale * Dhop(in)(n,.) )
//   Dhop psi(n) = sum_mu (1 - g_mu) U_mu(n) psi(n+mu) + (1 + g_mu) U_mu(n-mu)^+ psi(n-mu)
//
// The 4D Wilson hop inside D_DW (Sec. 4, Eq. dirac_eq) applied on one
// checkerboard; the dagger flips the projectors (Dhop^+ = g5 Dhop g5).
// Ex and Eout are fifth-dimension (s-local) operators, which the even-odd
// Schur operator needs right before or after the hop; they are applied in
// the same CTA, which holds every s of its 4D sites.
//
// Thread mapping: one CTA handles NS 4D half-sites x all Ls slices; thread
// (i, s) computes site i, slice s.  Neighbour spinors are read as 16-byte
// words in the s-fastest layout (consecutive s -> consecutive words); the 8
// links of a site are read by all Ls threads of that site (broadcast), so
// each link is fetched from DRAM once and reused over Ls.
//
// Spin projection in the chiral basis (g_k = [[0,-i sigma_k],[i sigma_k,0]],
// g_t = [[0,1],[1,0]]), with psi = (u; l) in 2-spin halves and sg = +-1:
//   (1 - sg g_k) psi = (h; -sg i sigma_k h),  h = u + sg i sigma_k l
//   (1 - sg g_t) psi = (h; -sg h),            h = u - sg l
// so only the 2-spin half h is multiplied by the link.
#include "dwf_internal.h"

#include "hop_common.cuh"

namespace dwf {

// hop2.cu: the slice-pair kernel with bulk-copy staging for FP32 / FP16 storage
int hop2_sites(int Ls, int prec, int nr);
dwf_status launch_hop2(dwf_lattice* L, const HopCall& c, const HopBatch& b, const SOpK<float>* ex,
                       const SOpK<float>* eout, int G, int ctas_per_sm);

// ---------------------------------------------------------------- hop kernel

template <class S> struct HopArgs {
  typedef typename Store<S>::calc_t C;
  CFieldRef<S> in;
  FieldRef<S> out;
  CFieldRef<S> x;  // x.v == nullptr: no site term
  const S* links;  // [Vh][8][18]
  const int* nbr;  // [8][Vh]
  long Vh;
  int Ls, Lh;
  int NS;  // 4D sites per CTA; threads beyond NS * Ls (warp padding) are idle
  SOpK<C> ex, eout;
  C scale, xscale;
  double* partials;
};

template <int MU, int SG, class S>
__device__ __forceinline__ void do_dir(const HopArgs<S>& a, long h, int s, int d,
                                       typename Store<S>::calc_t* acc) {
  typedef typename Store<S>::calc_t C;
  const long hn = __ldg(a.nbr + (long)d * a.Vh + h);
  C psi[24];
  load_spinor<S>(a.in, hn, s, a.Lh, psi);
  C u[18];
  load_link(a.links + (h * 8 + d) * 18, u);
  hop_dir<MU, SG>(psi, u, acc);
}

// out = Eout( xscale * Ex x + scale * Dhop in )
template <class S, int DAG>
__global__ void __launch_bounds__(256) hop_kernel(const HopArgs<S> a) {
  typedef typename Store<S>::calc_t C;
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  C* tile = reinterpret_cast<C*>(smraw);
  const int Ls = a.Ls;
  const int NS = a.NS;
  const int i = threadIdx.x / Ls;
  const int s = threadIdx.x - i * Ls;
  const long h = (long)blockIdx.x * NS + i;
  const bool act = (i < NS) && (h < a.Vh);
  const long left = a.Vh - (long)blockIdx.x * NS;
  const int nact = left < NS ? (int)left : NS;

  C acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0;
  if (act) {
    constexpr int F = DAG ? -1 : 1;
    do_dir<0, F>(a, h, s, 0, acc);
    do_dir<1, F>(a, h, s, 1, acc);
    do_dir<2, F>(a, h, s, 2, acc);
    do_dir<3, F>(a, h, s, 3, acc);
    do_dir<0, -F>(a, h, s, 4, acc);
    do_dir<1, -F>(a, h, s, 5, acc);
    do_dir<2, -F>(a, h, s, 6, acc);
    do_dir<3, -F>(a, h, s, 7, acc);
  }
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] *= a.scale;
  if (a.x.v != nullptr) {
    C xv[24];
    if (act) load_spinor<S>(a.x, h, s, a.Lh, xv);
    if (a.ex.kind != 0) sop_apply(a.ex, xv, tile, i, s, act, nact, Ls);
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = fma(a.xscale, xv[k], acc[k]);
  }
  if (a.eout.kind != 0) sop_apply(a.eout, acc, tile, i, s, act, nact, Ls);

  double part = 0.0;
  if (act) {
    store_spinor<S>(a.out, h, s, a.Lh, acc);
    if (a.partials) {
      // per-site sum in the kernel's precision (FP64 issue rate is tiny on
      // GB300); the block and grid sums are FP64
      C ps = 0;
#pragma unroll
      for (int k = 0; k < 24; ++k) ps = fma(acc[k], acc[k], ps);
      part = (double)ps;
    }
  }
  if (a.partials) {
    double t = block_sum<256>(part, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- FP64 fields, FP32 arithmetic
//
// The same hop on FP64-stored fields computed in FP32 (FP32 links), for the
// operator applications and solves inside an approximate step whose result
// needs only a few digits (the MADWF passes' Pauli-Villars and Moebius
// solves and their sources).  GB300 converts between FP64 and FP32 at its
// FP64 rate (about 1/70 of the FP32 rate), so the conversions use integer
// operations: a load keeps the top 24 significand bits (truncation: relative
// error below 2^-23; values below 2^-126 become zero) and a store widens the
// FP32 result exactly.

__device__ __forceinline__ float narrow_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hw = (unsigned)(b >> 32), lw = (unsigned)b;
  const unsigned sign = hw & 0x80000000u;
  const int e = (int)((hw >> 20) & 0x7ffu);
  if (e < 897) return __uint_as_float(sign);
  if (e > 1150) return __uint_as_float(sign | 0x7f800000u | ((e == 2047 && ((hw & 0xfffffu) | lw)) ? 0x400000u : 0u));
  return __uint_as_float(sign | ((unsigned)(e - 896) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
}
__device__ __forceinline__ double widen_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned sign = u & 0x80000000u;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned m = u & 0x7fffffu;
  unsigned hw;
  if (e == 0) hw = sign;  // zero; FP32 subnormals are taken as zero
  else if (e == 255) hw = sign | 0x7ff00000u | (m ? 0x80000u : 0u);
  else hw = sign | ((e + 896u) << 20) | (m >> 3);
  const unsigned lw = (e == 0 || e == 255) ? 0u : (m << 29);
  return __longlong_as_double((long long)(((unsigned long long)hw << 32) | lw));
}

struct HopLPArgs {
  const double* in;
  double* out;
  const double* x;     // nullptr: no site term
  const float* links;  // FP32 [Vh][8][18]
  const int* nbr;
  long Vh;
  int Ls, Lh, NS;
  SOpK<float> ex, eout;
  float scale, xscale;
  double* partials;
};

__device__ __forceinline__ void load_narrow(const double* f, long h, int s, int Lh, float* v) {
  const double* base = f + elem_index(h, 0, s >> 1, Lh) + (s & 1);
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[2 * k] = narrow_bits(__ldg(base + (long)k * Lh * 4));
    v[2 * k + 1] = narrow_bits(__ldg(base + (long)k * Lh * 4 + 2));
  }
}

template <int MU, int SG>
__device__ __forceinline__ void dir_lp(const HopLPArgs& a, long h, int s, int d, float* acc) {
  const long hn = __ldg(a.nbr + (long)d * a.Vh + h);
  float psi[24];
  load_narrow(a.in, hn, s, a.Lh, psi);
  float u[18];
  load_link(a.links + (h * 8 + d) * 18, u);
  hop_dir<MU, SG>(psi, u, acc);
}

template <int DAG>
__global__ void __launch_bounds__(256) hop_lp_kernel(const HopLPArgs a) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ double red[32];
  float* tile = reinterpret_cast<float*>(smraw);
  const int Ls = a.Ls;
  const int NS = a.NS;
  const int i = threadIdx.x / Ls;
  const int s = threadIdx.x - i * Ls;
  const long h = (long)blockIdx.x * NS + i;
  const bool act = (i < NS) && (h < a.Vh);
  const long left = a.Vh - (long)blockIdx.x * NS;
  const int nact = left < NS ? (int)left : NS;
  float acc[24];
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] = 0.f;
  if (act) {
    constexpr int F = DAG ? -1 : 1;
    dir_lp<0, F>(a, h, s, 0, acc);
    dir_lp<1, F>(a, h, s, 1, acc);
    dir_lp<2, F>(a, h, s, 2, acc);
    dir_lp<3, F>(a, h, s, 3, acc);
    dir_lp<0, -F>(a, h, s, 4, acc);
    dir_lp<1, -F>(a, h, s, 5, acc);
    dir_lp<2, -F>(a, h, s, 6, acc);
    dir_lp<3, -F>(a, h, s, 7, acc);
  }
#pragma unroll
  for (int k = 0; k < 24; ++k) acc[k] *= a.scale;
  if (a.x != nullptr) {
    float xv[24];
    if (act) load_narrow(a.x, h, s, a.Lh, xv);
    if (a.ex.kind != 0) sop_apply(a.ex, xv, tile, i, s, act, nact, Ls);
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = fmaf(a.xscale, xv[k], acc[k]);
  }
  if (a.eout.kind != 0) sop_apply(a.eout, acc, tile, i, s, act, nact, Ls);
  double part = 0.0;
  if (act) {
    double* base = a.out + elem_index(h, 0, s >> 1, a.Lh) + (s & 1);
    float ps = 0.f;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      base[(long)k * a.Lh * 4] = widen_bits(acc[2 * k]);
      base[(long)k * a.Lh * 4 + 2] = widen_bits(acc[2 * k + 1]);
      ps = fmaf(acc[2 * k], acc[2 * k], fmaf(acc[2 * k + 1], acc[2 * k + 1], ps));
    }
    part = (double)ps;
  }
  if (a.partials) {
    const double t = block_sum<256>(part, red);
    if (threadIdx.x == 0) a.partials[blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------- s-local kernel

template <class S> struct SopArgs {
  typedef typename Store<S>::calc_t C;
  CFieldRef<S> x;
  FieldRef<S> out;
  CFieldRef<S> y;  // optional
  long Vh;
  int Ls, Lh;
  int NS;
  SOpK<C> e;
  C a, b;
};

// out = a * E x + b * y
template <class S>
__global__ void __launch_bounds__(256) sop_kernel(const SopArgs<S> a) {
  typedef typename Store<S>::calc_t C;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* tile = reinterpret_cast<C*>(smraw);
  const int Ls = a.Ls;
  const int NS = a.NS;
  const int i = threadIdx.x / Ls;
  const int s = threadIdx.x - i * Ls;
  const long h = (long)blockIdx.x * NS + i;
  const bool act = (i < NS) && (h < a.Vh);
  const long left = a.Vh - (long)blockIdx.x * NS;
  const int nact = left < NS ? (int)left : NS;
  C v[24];
  if (act) load_spinor<S>(a.x, h, s, a.Lh, v);
  if (a.e.kind != 0) sop_apply(a.e, v, tile, i, s, act, nact, Ls);
  if (!act) return;
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] *= a.a;
  if (a.y.v) {
    C w[24];
    load_spinor<S>(a.y, h, s, a.Lh, w);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = fma(a.b, w[k], v[k]);
  }
  store_spinor<S>(a.out, h, s, a.Lh, v);
}

// ---------------------------------------------------------------- launchers

static int sites_per_cta(int Ls) {
  int ns = 128 / Ls;
  return ns < 1 ? 1 : ns;
}
static int warp_round(int n) { return (n + 31) / 32 * 32; }

template <class S> static CFieldRef<S> cref(const Field& f) {
  return CFieldRef<S>{reinterpret_cast<const S*>(f.v), f.norm};
}
template <class S> static FieldRef<S> ref(const Field& f) {
  return FieldRef<S>{reinterpret_cast<S*>(f.v), f.norm};
}

template <class C>
static SOpK<C> sop_k(const SOps* ops, SOps::Kind k, int Ls) {
  SOpK<C> o{};
  o.kind = 0;
  if (!ops || k == SOps::NKIND) return o;
  const SOpDesc& d = ops->desc[k];
  o.kind = d.kind;
  o.trans = d.trans;
  o.has_inv = d.has_inv;
  o.g1 = (C)d.g1;
  o.d1 = (C)d.d1;
  o.ginv = (C)d.ginv;
  o.rho = (C)d.rho;
  o.m = (C)d.m;
  o.c0 = (C)d.c0;
  if constexpr (sizeof(C) == 8)
    o.dense = ops->k64((SOps::Kind)d.dense_kind, Ls);
  else
    o.dense = ops->k32((SOps::Kind)d.dense_kind, Ls);
  return o;
}

template <class C> static size_t tile_bytes(int NS, int Ls) { return (size_t)NS * 12 * tile_row(Ls) * sizeof(C); }

template <class S>
static dwf_status hop_t(dwf_lattice* L, const HopCall& c) {
  typedef typename Store<S>::calc_t C;
  const int pi = c.in.prec;
  HopArgs<S> a;
  a.in = cref<S>(c.in);
  a.out = ref<S>(c.out);
  a.x = c.has_x ? cref<S>(c.x) : CFieldRef<S>{nullptr, nullptr};
  a.links = reinterpret_cast<const S*>(L->links[pi][c.out_parity]);
  a.nbr = L->nbr[c.out_parity];
  a.Vh = L->Vh;
  a.Ls = L->Ls;
  a.Lh = L->Lh;
  a.ex = sop_k<C>(c.has_x ? c.ops : nullptr, c.ex, L->Ls);
  a.eout = sop_k<C>(c.ops, c.eout, L->Ls);
  a.scale = (C)c.scale;
  a.xscale = (C)c.xscale;
  a.partials = c.partials;
  const int NS = sites_per_cta(L->Ls);
  const int threads = warp_round(NS * L->Ls);
  const long blocks = (L->Vh + NS - 1) / NS;
  a.NS = NS;
  if (c.partials && blocks > kPartials) return fail(L, DWF_ERR_INVALID_ARG, "lattice too large for the partial-sum buffer");
  const size_t smem = (a.ex.kind || a.eout.kind) ? tile_bytes<C>(NS, L->Ls) : 0;
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (L->timing) DWF_TRY(timing_begin(L, &ta, &tb));
  int NS2 = 0;
  if constexpr (sizeof(S) <= 4) NS2 = hop2_sites(L->Ls, pi, 1);
  const bool lp = sizeof(S) == 8 && (L->fp64_in_fp32 > 0 || L->fp64_arith == 1);
  if (lp) {
    HopLPArgs b;
    b.in = reinterpret_cast<const double*>(c.in.v);
    b.out = reinterpret_cast<double*>(c.out.v);
    b.x = c.has_x ? reinterpret_cast<const double*>(c.x.v) : nullptr;
    b.links = reinterpret_cast<const float*>(L->links[DWF_F32][c.out_parity]);
    b.nbr = L->nbr[c.out_parity];
    b.Vh = L->Vh;
    b.Ls = L->Ls;
    b.Lh = L->Lh;
    b.NS = NS;
    b.ex = sop_k<float>(c.has_x ? c.ops : nullptr, c.ex, L->Ls);
    b.eout = sop_k<float>(c.ops, c.eout, L->Ls);
    b.scale = (float)c.scale;
    b.xscale = (float)c.xscale;
    b.partials = c.partials;
    const size_t smem32 = (b.ex.kind || b.eout.kind) ? tile_bytes<float>(NS, L->Ls) : 0;
    if (c.dag) {
      if (smem32 > 48 * 1024)
        DWF_CUDA(L, cudaFuncSetAttribute(hop_lp_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
      hop_lp_kernel<1><<<(unsigned)blocks, threads, smem32, L->stream>>>(b);
    } else {
      if (smem32 > 48 * 1024)
        DWF_CUDA(L, cudaFuncSetAttribute(hop_lp_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
      hop_lp_kernel<0><<<(unsigned)blocks, threads, smem32, L->stream>>>(b);
    }
  } else if (NS2 > 0) {
    if constexpr (sizeof(S) <= 4) {
      HopBatch b;
      b.nrhs = 1;
      b.in[0] = c.in;
      b.out[0] = c.out;
      b.x[0] = c.x;
      b.partials[0] = c.partials;
      DWF_TRY(launch_hop2(L, c, b, &a.ex, &a.eout, NS2, 0));
    }
  } else if (c.dag) {
    if (smem > 48 * 1024)
      DWF_CUDA(L, cudaFuncSetAttribute(hop_kernel<S, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hop_kernel<S, 1><<<(unsigned)blocks, threads, smem, L->stream>>>(a);
  } else {
    if (smem > 48 * 1024)
      DWF_CUDA(L, cudaFuncSetAttribute(hop_kernel<S, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    hop_kernel<S, 0><<<(unsigned)blocks, threads, smem, L->stream>>>(a);
  }
  counted(L);
  if (L->timing) {
    // algorithmic bytes: each spinor read or written once, each 4D site's 8 links once
    const double w = sizeof(S);
    const double spin = 24.0 * w + (sizeof(S) == 2 ? 4.0 : 0.0);
    const double sites = (double)L->Vh * L->Ls;
    const double bytes = sites * spin * (c.has_x ? 3.0 : 2.0) + (double)L->Vh * 8 * 18 * w;
    timing_end(L, pi, bytes, ta, tb);
  }
  if (c.nblocks && NS2 == 0) *c.nblocks = (int)blocks;
  DWF_CUDA(L, cudaGetLastError());
  return DWF_OK;
}

dwf_status launch_hop(dwf_lattice* L, const HopCall& c) {
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "gauge field not set");
  if (c.in.prec != c.out.prec || (c.has_x && c.x.prec != c.in.prec))
    return fail(L, DWF_ERR_INVALID_ARG, "hop: mixed precisions");
  switch (c.in.prec) {
    case DWF_F64: return hop_t<double>(L, c);
    case DWF_F32: return hop_t<float>(L, c);
    case DWF_F16: return hop_t<__half>(L, c);
  }
  return fail(L, DWF_ERR_INVALID_ARG, "hop: bad precision");
}

int hop_batch_max(int Ls, dwf_prec prec) {
  for (int n = kMaxBatch; n >= 1; --n)
    if (hop2_sites(Ls, prec, n) > 0) return n;
  return 0;
}

dwf_status launch_hop_batch(dwf_lattice* L, const HopCall& c, const HopBatch& b, int ctas_per_sm) {
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "gauge field not set");
  const int nr = b.nrhs;
  if (nr < 1 || nr > kMaxBatch) return fail(L, DWF_ERR_INVALID_ARG, "hop batch: bad number of right-hand sides");
  const dwf_prec pi = b.in[0].prec;
  const int G = hop2_sites(L->Ls, pi, nr);
  if (G < 1) return fail(L, DWF_ERR_INVALID_ARG, "hop batch: shape not supported by the pipelined kernel");
  SOpK<float> ex[kMaxBatch], eout[kMaxBatch];
  for (int r = 0; r < nr; ++r) {
    if (b.in[r].prec != pi || b.out[r].prec != pi || (c.has_x && b.x[r].prec != pi) || !b.ops[r])
      return fail(L, DWF_ERR_INVALID_ARG, "hop batch: mixed precisions or missing operators");
    if ((b.partials[r] != nullptr) != (b.partials[0] != nullptr))
      return fail(L, DWF_ERR_INVALID_ARG, "hop batch: partial sums for some right-hand sides only");
    ex[r] = sop_k<float>(c.has_x ? b.ops[r] : nullptr, c.ex, L->Ls);
    eout[r] = sop_k<float>(b.ops[r], c.eout, L->Ls);
    if (ex[r].kind != ex[0].kind || eout[r].kind != eout[0].kind)
      return fail(L, DWF_ERR_INVALID_ARG, "hop batch: operator kinds differ between masses");
  }
  cudaEvent_t ta = nullptr, tb = nullptr;
  if (L->timing) DWF_TRY(timing_begin(L, &ta, &tb));
  DWF_TRY(launch_hop2(L, c, b, ex, eout, G, ctas_per_sm));
  counted(L);
  if (L->timing) {
    const double w = pi == DWF_F32 ? 4.0 : 2.0;
    const double spin = 24.0 * w + (pi == DWF_F16 ? 4.0 : 0.0);
    const double sites = (double)L->Vh * L->Ls * nr;
    const double bytes = sites * spin * (c.has_x ? 3.0 : 2.0) + (double)L->Vh * 8 * 18 * w;
    timing_end(L, pi, bytes, ta, tb);
  }
  DWF_CUDA(L, cudaGetLastError());
  return DWF_OK;
}

template <class S>
static dwf_status sop_t(dwf_lattice* L, Field x, Field out, const SOps* ops, SOps::Kind e, double aa,
                        const Field* y, double bb) {
  typedef typename Store<S>::calc_t C;
  SopArgs<S> a;
  a.x = cref<S>(x);
  a.out = ref<S>(out);
  a.y = y ? cref<S>(*y) : CFieldRef<S>{nullptr, nullptr};
  a.Vh = L->Vh;
  a.Ls = L->Ls;
  a.Lh = L->Lh;
  a.e = sop_k<C>(ops, e, L->Ls);
  a.a = (C)aa;
  a.b = (C)bb;
  const int NS = sites_per_cta(L->Ls);
  const long blocks = (L->Vh + NS - 1) / NS;
  a.NS = NS;
  const size_t smem = a.e.kind ? tile_bytes<C>(NS, L->Ls) : 0;
  if (smem > 48 * 1024)
    DWF_CUDA(L, cudaFuncSetAttribute(sop_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  sop_kernel<S><<<(unsigned)blocks, warp_round(NS * L->Ls), smem, L->stream>>>(a);
  counted(L);
  DWF_CUDA(L, cudaGetLastError());
  return DWF_OK;
}

dwf_status launch_sop(dwf_lattice* L, Field x, Field out, const SOps* ops, SOps::Kind e, double a,
                      const Field* y, double b) {
  if (x.prec != out.prec || (y && y->prec != x.prec)) return fail(L, DWF_ERR_INVALID_ARG, "sop: mixed precisions");
  switch (x.prec) {
    case DWF_F64: return sop_t<double>(L, x, out, ops, e, a, y, b);
    case DWF_F32: return sop_t<float>(L, x, out, ops, e, a, y, b);
    case DWF_F16: return sop_t<__half>(L, x, out, ops, e, a, y, b);
  }
  return fail(L, DWF_ERR_INVALID_ARG, "sop: bad precision");
}

}  // namespace dwf
