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

namespace dwf {

// acc += c * z with c in {+1, -1, +i, -i} given at compile time as (CR, CI).
template <int CR, int CI, class C>
__device__ __forceinline__ void cmadd(C& ar, C& ai, C zr, C zi) {
  static_assert(CR * CR + CI * CI == 1, "unit coefficient");
  if constexpr (CR == 1) {
    ar += zr;
    ai += zi;
  } else if constexpr (CR == -1) {
    ar -= zr;
    ai -= zi;
  } else if constexpr (CI == 1) {
    ar -= zi;
    ai += zr;
  } else {
    ar += zi;
    ai -= zr;
  }
}

// Projection table for (1 - SG g_mu):
//   h0 = psi_0 + c1 psi_J1,  h1 = psi_1 + c2 psi_J2,  g = U h,
//   out_0 += g0, out_1 += g1, out_2 += d2 g_{S2}, out_3 += d3 g_{S3}.
template <int MU, int SG> struct Proj;
template <int SG> struct Proj<0, SG> {  // x: i sigma_1 l = (i l1, i l0)
  static constexpr int J1 = 3, C1R = 0, C1I = SG, J2 = 2, C2R = 0, C2I = SG;
  static constexpr int S2 = 1, D2R = 0, D2I = -SG, S3 = 0, D3R = 0, D3I = -SG;
};
template <int SG> struct Proj<1, SG> {  // y: i sigma_2 l = (l1, -l0)
  static constexpr int J1 = 3, C1R = SG, C1I = 0, J2 = 2, C2R = -SG, C2I = 0;
  static constexpr int S2 = 1, D2R = -SG, D2I = 0, S3 = 0, D3R = SG, D3I = 0;
};
template <int SG> struct Proj<2, SG> {  // z: i sigma_3 l = (i l0, -i l1)
  static constexpr int J1 = 2, C1R = 0, C1I = SG, J2 = 3, C2R = 0, C2I = -SG;
  static constexpr int S2 = 0, D2R = 0, D2I = -SG, S3 = 1, D3R = 0, D3I = SG;
};
template <int SG> struct Proj<3, SG> {  // t
  static constexpr int J1 = 2, C1R = -SG, C1I = 0, J2 = 3, C2R = -SG, C2I = 0;
  static constexpr int S2 = 0, D2R = -SG, D2I = 0, S3 = 1, D3R = -SG, D3I = 0;
};

// acc += (1 - SG g_MU) U psi   (psi, acc: 24 reals, complex k = spin*3 + colour)
template <int MU, int SG, class C>
__device__ __forceinline__ void hop_dir(const C* __restrict__ psi, const C* __restrict__ u,
                                        C* __restrict__ acc) {
  typedef Proj<MU, SG> P;
  C h[12];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h[2 * a] = psi[2 * a];
    h[2 * a + 1] = psi[2 * a + 1];
    cmadd<P::C1R, P::C1I>(h[2 * a], h[2 * a + 1], psi[2 * (P::J1 * 3 + a)], psi[2 * (P::J1 * 3 + a) + 1]);
    h[6 + 2 * a] = psi[2 * (3 + a)];
    h[6 + 2 * a + 1] = psi[2 * (3 + a) + 1];
    cmadd<P::C2R, P::C2I>(h[6 + 2 * a], h[6 + 2 * a + 1], psi[2 * (P::J2 * 3 + a)],
                          psi[2 * (P::J2 * 3 + a) + 1]);
  }
  C g[12];
#pragma unroll
  for (int j = 0; j < 2; ++j) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      C gr = 0, gi = 0;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const C ur = u[2 * (3 * a + b)], ui = u[2 * (3 * a + b) + 1];
        const C hr = h[6 * j + 2 * b], hi = h[6 * j + 2 * b + 1];
        gr = fma(ur, hr, gr);
        gr = fma(-ui, hi, gr);
        gi = fma(ur, hi, gi);
        gi = fma(ui, hr, gi);
      }
      g[6 * j + 2 * a] = gr;
      g[6 * j + 2 * a + 1] = gi;
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    acc[2 * a] += g[2 * a];
    acc[2 * a + 1] += g[2 * a + 1];
    acc[6 + 2 * a] += g[6 + 2 * a];
    acc[6 + 2 * a + 1] += g[6 + 2 * a + 1];
    cmadd<P::D2R, P::D2I>(acc[12 + 2 * a], acc[12 + 2 * a + 1], g[6 * P::S2 + 2 * a], g[6 * P::S2 + 2 * a + 1]);
    cmadd<P::D3R, P::D3I>(acc[18 + 2 * a], acc[18 + 2 * a + 1], g[6 * P::S3 + 2 * a], g[6 * P::S3 + 2 * a + 1]);
  }
}

// ---------------------------------------------------------------- fifth-dimension operators
//
// Every s-local operator of the even-odd Schur form is, per chirality,
//   y = (g1 + d1 Q)(g2 + d2 Q)^-1 x
// with Q the one-step fifth-dimension hop carrying the -m wall: on the P+
// half Q z_s = z_{s-1} (z_{-1} := -m z_{Ls-1}); on the P- half
// Q z_s = z_{s+1} (z_{Ls} := -m z_0); the transpose swaps the two.  With
// rho = -d2/g2 the inverse is a Horner sum for z_0 followed by the forward
// recurrence z_s = x_s / g2 + rho z_{s-1}:
//   z_0 = (x_0 - m rho sum_{j=1}^{Ls-1} rho^{Ls-1-j} x_j) / (g2 (1 + m rho^Ls)),
// i.e. O(Ls) work per (4D site, component) instead of the O(Ls^2) of a
// dense Ls x Ls matrix.  Kinds: 0 identity, 1 structured, 2 dense fallback
// (used when |rho| > 1 would make the recurrence amplify rounding).

template <class C> struct SOpK {
  int kind;
  int trans;
  int has_inv;
  C g1, d1, ginv, rho, m, c0;
  const C* dense;  // kind 2: [2][Ls][Ls] row-major (P+ block, P- block)
};

// Tile layout in shared memory: [site][12 complex][R], complex (re, im) at
// 2s within a row; R = 2 Ls + 2 (or + 4) keeps both access patterns
// (lanes over s, lanes over components) free of most bank conflicts.
__host__ __device__ inline int tile_row(int Ls) { return (Ls & 1) ? 2 * Ls + 4 : 2 * Ls + 2; }

template <class C>
__device__ __forceinline__ void tile_put(C* tile, int R, int i, int s, const C* v) {
  C* base = tile + (i * 12) * R + 2 * s;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    base[k * R] = v[2 * k];
    base[k * R + 1] = v[2 * k + 1];
  }
}
template <class C>
__device__ __forceinline__ void tile_get(const C* tile, int R, int i, int s, C* v) {
  const C* base = tile + (i * 12) * R + 2 * s;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    v[2 * k] = base[k * R];
    v[2 * k + 1] = base[k * R + 1];
  }
}

// In-place structured operator on the rows of the first `nsites` sites.
template <class C>
__device__ void sop_rows(const SOpK<C>& op, C* tile, int nsites, int Ls, int R) {
  for (int w = threadIdx.x; w < nsites * 12; w += blockDim.x) {
    const int k = w % 12;
    const int up = ((k >= 6) ? 1 : 0) ^ op.trans;  // P+ (k < 6) walks down in s unless transposed
    C* row = tile + w * R;
    const int s0 = up ? Ls - 1 : 0;
    const int ds = up ? -1 : 1;
    if (op.has_inv) {
      C wr = 0, wi = 0;
      for (int j = 1; j < Ls; ++j) {
        const C* p = row + 2 * (s0 + ds * j);
        wr = fma(wr, op.rho, p[0]);
        wi = fma(wi, op.rho, p[1]);
      }
      const C mr = op.m * op.rho;
      const C z0r = fma(-mr, wr, row[2 * s0]) * op.c0;
      const C z0i = fma(-mr, wi, row[2 * s0 + 1]) * op.c0;
      C pr = z0r, pi = z0i;
      for (int j = 1; j < Ls; ++j) {
        C* p = row + 2 * (s0 + ds * j);
        const C zr = fma(op.rho, pr, p[0] * op.ginv);
        const C zi = fma(op.rho, pi, p[1] * op.ginv);
        p[0] = fma(op.d1, pr, op.g1 * zr);
        p[1] = fma(op.d1, pi, op.g1 * zi);
        pr = zr;
        pi = zi;
      }
      const C dm = op.d1 * op.m;
      row[2 * s0] = fma(-dm, pr, op.g1 * z0r);
      row[2 * s0 + 1] = fma(-dm, pi, op.g1 * z0i);
    } else {
      // y_j = (g1 x_j + d1 x_{j-1}) / g2 for j >= 1, y_0 = (g1 x_0 - d1 m x_{Ls-1}) / g2
      C* pl = row + 2 * (s0 + ds * (Ls - 1));
      const C lr = pl[0], li = pl[1];
      const C g1 = op.g1 * op.ginv, d1 = op.d1 * op.ginv;
      for (int j = Ls - 1; j >= 1; --j) {
        C* p = row + 2 * (s0 + ds * j);
        const C* q = row + 2 * (s0 + ds * (j - 1));
        p[0] = fma(d1, q[0], g1 * p[0]);
        p[1] = fma(d1, q[1], g1 * p[1]);
      }
      const C dm = d1 * op.m;
      row[2 * s0] = fma(-dm, lr, g1 * row[2 * s0]);
      row[2 * s0 + 1] = fma(-dm, li, g1 * row[2 * s0 + 1]);
    }
  }
}

// v (the 24 reals of thread (i, s)) <- op v, across the CTA through the tile.
// Called by every thread of the CTA; the tile is free again on return.
template <class C>
__device__ __forceinline__ void sop_apply(const SOpK<C>& op, C* v, C* tile, int i, int s, bool act, int nact,
                                          int Ls) {
  const int R = tile_row(Ls);
  if (act) tile_put(tile, R, i, s, v);
  __syncthreads();
  if (op.kind == 1) {
    sop_rows(op, tile, nact, Ls, R);
    __syncthreads();
    if (act) tile_get(tile, R, i, s, v);
  } else if (act) {
    // dense matrices are stored already transposed where the operator is
    const C* Ep = op.dense + s * Ls;
    const C* Em = op.dense + Ls * Ls + s * Ls;
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = 0;
    const C* base = tile + (i * 12) * R;
    for (int t = 0; t < Ls; ++t) {
      const C ep = Ep[t], em = Em[t];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const C e = k < 6 ? ep : em;
        v[2 * k] = fma(e, base[k * R + 2 * t], v[2 * k]);
        v[2 * k + 1] = fma(e, base[k * R + 2 * t + 1], v[2 * k + 1]);
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------- hop kernel

template <class S> struct HopArgs {
  typedef typename Store<S>::calc_t C;
  CFieldRef<S> in;
  FieldRef<S> out;
  CFieldRef<S> x;  // x.v == nullptr: no site term
  const S* links;  // [Vh][8][18]
  const int* nbr;  // [8][Vh]
  long Vh;
  int Ls;
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
  load_spinor<S>(a.in, hn, s, a.Ls, psi);
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
    if (act) load_spinor<S>(a.x, h, s, Ls, xv);
    if (a.ex.kind != 0) sop_apply(a.ex, xv, tile, i, s, act, nact, Ls);
#pragma unroll
    for (int k = 0; k < 24; ++k) acc[k] = fma(a.xscale, xv[k], acc[k]);
  }
  if (a.eout.kind != 0) sop_apply(a.eout, acc, tile, i, s, act, nact, Ls);

  double part = 0.0;
  if (act) {
    store_spinor<S>(a.out, h, s, Ls, acc);
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

// ---------------------------------------------------------------- s-local kernel

template <class S> struct SopArgs {
  typedef typename Store<S>::calc_t C;
  CFieldRef<S> x;
  FieldRef<S> out;
  CFieldRef<S> y;  // optional
  long Vh;
  int Ls;
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
  if (act) load_spinor<S>(a.x, h, s, Ls, v);
  if (a.e.kind != 0) sop_apply(a.e, v, tile, i, s, act, nact, Ls);
  if (!act) return;
#pragma unroll
  for (int k = 0; k < 24; ++k) v[k] *= a.a;
  if (a.y.v) {
    C w[24];
    load_spinor<S>(a.y, h, s, Ls, w);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = fma(a.b, w[k], v[k]);
  }
  store_spinor<S>(a.out, h, s, Ls, v);
}

// ---------------------------------------------------------------- launchers

static int sites_per_cta(int Ls) {
  int ns = 128 / Ls;
  return ns < 1 ? 1 : ns;
}
static int warp_round(int n) { return (n + 31) / 32 * 32; }

template <class S> static CFieldRef<S> cref(const Field& f) {
  return CFieldRef<S>{reinterpret_cast<const typename Store<S>::chunk_t*>(f.v), f.norm};
}
template <class S> static FieldRef<S> ref(const Field& f) {
  return FieldRef<S>{reinterpret_cast<typename Store<S>::chunk_t*>(f.v), f.norm};
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
  if (c.dag) {
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
  if (c.nblocks) *c.nblocks = (int)blocks;
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
