// Wilson hop at every fifth-dimension slice for FP32- and FP16-stored
// spinors (FP32 arithmetic), the bandwidth-critical kernel of the mixed
// precision and MADWF solves:
//
//   out(n,.) = Eout( xscale * Ex x(n,.) + scale * Dhop(in)(n,.) )
//
// (the 4D Wilson hop inside D_DW, Sec. 4 Eq. dirac_eq, on one checkerboard,
// with the fifth-dimension operators of the even-odd Schur form fused).
//
// GB300 design:
//  * A CTA owns NS 4D sites; thread (i, j) owns the slice pair (j, j + Lh) of
//    site i, so both lanes of every packed FP32x2 FMA (__ffma2_rn) use the
//    same link element and the arithmetic instruction count halves.
//  * A neighbour site's whole 5D spinor block is contiguous in the pair
//    layout, so each direction's NS neighbour blocks are fetched by the bulk
//    copy engine (cp.async.bulk, completion counted on an mbarrier) into a
//    two-slot shared-memory ring: direction d + 2 streams in while d is
//    computed, independently of occupancy.
//  * The 8 links of each site are read once per CTA into shared memory,
//    duplicated as (u, u) pairs so they feed the packed FMAs directly, and
//    reused over all Ls slices.
//  * Waits on the mbarriers are bounded: a wait that gives up sets the
//    handle's device error flag (reported as DWF_ERR_TIMEOUT), waits once more
//    for the CTA's own copies and skips the store.
#include "dwf_internal.h"

#include "hop_common.cuh"

namespace dwf {

namespace {

constexpr int kThreads2 = 128;
constexpr long kWaitLimit = 1L << 22;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (long it = 0; it < kWaitLimit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// z = a + c*b for c in {+1, -1, +i, -i} on complex pairs (re, im as float2 over slices)
template <int CR, int CI>
__device__ __forceinline__ void cpair(float2 ar, float2 ai, float2 br, float2 bi, float2& zr, float2& zi) {
  if constexpr (CR == 1) {
    zr = add2(ar, br);
    zi = add2(ai, bi);
  } else if constexpr (CR == -1) {
    zr = sub2(ar, br);
    zi = sub2(ai, bi);
  } else if constexpr (CI == 1) {
    zr = sub2(ar, bi);
    zi = add2(ai, br);
  } else {
    zr = add2(ar, bi);
    zi = sub2(ai, br);
  }
}
// acc += c * g
template <int CR, int CI>
__device__ __forceinline__ void cacc(float2& ar, float2& ai, float2 gr, float2 gi) {
  if constexpr (CR == 1) {
    ar = add2(ar, gr);
    ai = add2(ai, gi);
  } else if constexpr (CR == -1) {
    ar = sub2(ar, gr);
    ai = sub2(ai, gi);
  } else if constexpr (CI == 1) {
    ar = sub2(ar, gi);
    ai = add2(ai, gr);
  } else {
    ar = add2(ar, gi);
    ai = sub2(ai, gr);
  }
}

// acc += (1 - SG g_MU) U psi on a slice pair; psi given by (pr, pi)[12],
// link from shared memory as 9 complex (ur, ur, ui, ui) float4.
template <int MU, int SG>
__device__ __forceinline__ void hop_dir2(const float2* pr, const float2* pi, const float4* __restrict__ U,
                                         float2* ar, float2* ai) {
  typedef Proj<MU, SG> P;
  float2 hr[6], hi[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpair<P::C1R, P::C1I>(pr[a], pi[a], pr[P::J1 * 3 + a], pi[P::J1 * 3 + a], hr[a], hi[a]);
    cpair<P::C2R, P::C2I>(pr[3 + a], pi[3 + a], pr[P::J2 * 3 + a], pi[P::J2 * 3 + a], hr[3 + a], hi[3 + a]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float4 u[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) u[b] = U[3 * a + b];
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      // g = sum_b U_ab h_b :  gr = sum ur hr - sum ui hi,  gi = sum ur hi + ui hr
      float2 A = make_float2(0.f, 0.f), B = A, gi = A;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        const float2 ur = make_float2(u[b].x, u[b].y), ui = make_float2(u[b].z, u[b].w);
        A = fma2(ur, hr[3 * hh + b], A);
        B = fma2(ui, hi[3 * hh + b], B);
        gi = fma2(ur, hi[3 * hh + b], gi);
        gi = fma2(ui, hr[3 * hh + b], gi);
      }
      const float2 gr = sub2(A, B);
      // upper spins 0, 1
      ar[3 * hh + a] = add2(ar[3 * hh + a], gr);
      ai[3 * hh + a] = add2(ai[3 * hh + a], gi);
      // lower spins 2, 3
      if (hh == P::S2) cacc<P::D2R, P::D2I>(ar[6 + a], ai[6 + a], gr, gi);
      if (hh == P::S3) cacc<P::D3R, P::D3I>(ar[9 + a], ai[9 + a], gr, gi);
    }
  }
}

template <class S> struct Hop2Args {
  CFieldRef<S> in;
  FieldRef<S> out;
  CFieldRef<S> x;
  const S* links;  // [Vh][8][18]
  const int* nbr;  // [8][Vh]
  long Vh;
  int Ls, Lh, NS;
  int ring_bytes;  // the ring region (also the s-op tile after the direction loop)
  SOpK<float> ex, eout;
  float scale, xscale;
  double* partials;
  int* err;
};

// bytes of one site's spinor block and of its FP16 scales
template <class S> __host__ __device__ constexpr int chunk_bytes() { return sizeof(S) == 4 ? 16 : 8; }

template <class S> struct Ring;  // per-slot view helpers

// Write the pair (re, im) of slices j, j + Lh of site i into the s-op tile.
__device__ __forceinline__ void tile_put_pair(float* tile, int R, int i, int j, int Lh, int Ls, const float2* re,
                                              const float2* im) {
  float* base = tile + (i * 12) * R;
  const bool two = j + Lh < Ls;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    reinterpret_cast<float2*>(base + k * R)[j] = make_float2(re[k].x, im[k].x);
    if (two) reinterpret_cast<float2*>(base + k * R)[j + Lh] = make_float2(re[k].y, im[k].y);
  }
}
__device__ __forceinline__ void tile_get_pair(const float* tile, int R, int i, int j, int Lh, int Ls, float2* re,
                                              float2* im) {
  const float* base = tile + (i * 12) * R;
  const bool two = j + Lh < Ls;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 a = reinterpret_cast<const float2*>(base + k * R)[j];
    const float2 b = two ? reinterpret_cast<const float2*>(base + k * R)[j + Lh] : make_float2(0.f, 0.f);
    re[k] = make_float2(a.x, b.x);
    im[k] = make_float2(a.y, b.y);
  }
}

// (re, im) <- op (re, im) across the CTA, through the tile (all threads call).
__device__ __forceinline__ void sop_pair(const SOpK<float>& op, float2* re, float2* im, float* tile, int i, int j,
                                         bool act, int nact, int Ls, int Lh) {
  const int R = tile_row(Ls);
  if (act) tile_put_pair(tile, R, i, j, Lh, Ls, re, im);
  __syncthreads();
  if (op.kind == 1) {
    sop_rows(op, tile, nact, Ls, R);
    __syncthreads();
    if (act) tile_get_pair(tile, R, i, j, Lh, Ls, re, im);
  } else if (act) {
    // dense fallback: row s of the (already transposed where needed) matrix
    const float* base = tile + (i * 12) * R;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re[k] = make_float2(0.f, 0.f);
      im[k] = re[k];
    }
    const int s0 = j, s1 = j + Lh < Ls ? j + Lh : j;
    for (int t = 0; t < Ls; ++t) {
      const float e0p = op.dense[s0 * Ls + t], e0m = op.dense[Ls * Ls + s0 * Ls + t];
      const float e1p = op.dense[s1 * Ls + t], e1m = op.dense[Ls * Ls + s1 * Ls + t];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const float2 v = reinterpret_cast<const float2*>(base + k * R)[t];
        const float2 e = k < 6 ? make_float2(e0p, e1p) : make_float2(e0m, e1m);
        re[k] = fma2(e, f2(v.x), re[k]);
        im[k] = fma2(e, f2(v.y), im[k]);
      }
    }
    if (!(j + Lh < Ls))
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        re[k].y = 0.f;
        im[k].y = 0.f;
      }
  }
  __syncthreads();
}

__device__ __forceinline__ void unpack_chunk(const float4& a, float2& r, float2& i) {
  r = make_float2(a.x, a.y);
  i = make_float2(a.z, a.w);
}

// ---------------------------------------------------------------- the pipelined kernel
//
// One CTA = one warp.  The warp walks site groups g = blockIdx.x, blockIdx.x +
// gridDim.x, ...; a group is G = 32 / Lh sites, thread (i, j) owning slice pair
// j of site i.  Each group is a sequence of stages: directions d = 0..7 (the G
// neighbour blocks of that direction; stage 0 also brings the group's links)
// and, if the hop has a site term, the group's own x block.  Stages stream
// through a two-slot ring in issue order, so the stages of the next group are
// in flight while this group finishes; the s-op tile of the epilogue reuses
// the slot of the stage just consumed.

// expanded links: 72 float4 per site, padded so consecutive sites start in different banks
constexpr int kDupStride = 74;

struct Ctx {  // per-CTA shared-memory layout (byte offsets)
  int slot_bytes, raw_off, dup_off, total;
};

__host__ __device__ inline Ctx make_ctx(int Ls, int prec, int G) {
  const int Lh = (Ls + 1) / 2;
  const int cb = prec == DWF_F32 ? 16 : 8;
  int blocks = G * 12 * Lh * cb + (prec == DWF_F16 ? G * Lh * 8 : 0);
  const int tile = G * 12 * tile_row(Ls) * 4;
  int slot = blocks > tile ? blocks : tile;
  slot = (slot + 127) / 128 * 128;
  Ctx c;
  c.slot_bytes = slot;
  c.raw_off = 2 * slot;
  c.dup_off = c.raw_off + (G * 8 * 18 * 4 + 127) / 128 * 128;
  c.total = c.dup_off + G * kDupStride * 16;
  return c;
}

template <class S> struct Hop3Args {
  CFieldRef<S> in;
  FieldRef<S> out;
  CFieldRef<S> x;
  const S* links;  // [Vh][8][18]
  const int* nbr;  // [8][Vh]
  long Vh;
  long ngroups;
  int Ls, Lh, G;
  Ctx ctx;
  SOpK<float> ex, eout;
  float scale, xscale;
  double* partials;
  int* err;
};

template <class S> struct Pipe {
  const Hop3Args<S>* a;
  unsigned char* sm;
  unsigned bar0;
  int nstage;  // stages per group
  int blk, sblk;
};

// Issue stage k (0 .. nstage-1) of group g into ring slot `slot`; nb holds
// the group's neighbour index for direction k (per lane < nact).
template <class S>
__device__ __forceinline__ void issue_stage(const Pipe<S>& P, long g, int k, int slot, int nb_k) {
  const Hop3Args<S>& a = *P.a;
  if (g >= a.ngroups) return;
  const long h0 = g * a.G;
  const long left = a.Vh - h0;
  const int nact = left < a.G ? (int)left : a.G;
  const int lane = threadIdx.x;
  const unsigned bar = P.bar0 + 8u * slot;
  unsigned char* dst = P.sm + slot * a.ctx.slot_bytes;
  const bool fp16 = sizeof(S) == 2;
  fence_async_smem();
  unsigned bytes;
  if (k < 8) {
    bytes = nact * (P.blk + (fp16 ? P.sblk : 0)) + (k == 0 ? nact * 8 * 18 * (int)sizeof(S) : 0);
  } else {
    bytes = nact * (P.blk + (fp16 ? P.sblk : 0));
  }
  if (lane == 0) mbar_expect_tx(bar, bytes);
  __syncwarp();
  if (k < 8) {
    if (lane < nact) {
      bulk_g2s(smem_addr(dst + lane * P.blk), reinterpret_cast<const unsigned char*>(a.in.v) + (long)nb_k * P.blk,
               P.blk, bar);
      if (fp16)
        bulk_g2s(smem_addr(dst + a.G * P.blk + lane * P.sblk),
                 reinterpret_cast<const unsigned char*>(a.in.norm) + (long)nb_k * P.sblk, P.sblk, bar);
    }
    if (k == 0 && lane == 0)
      bulk_g2s(smem_addr(P.sm + a.ctx.raw_off), a.links + h0 * 8 * 18, nact * 8 * 18 * (int)sizeof(S), bar);
  } else if (lane == 0) {
    bulk_g2s(smem_addr(dst), reinterpret_cast<const unsigned char*>(a.x.v) + h0 * P.blk, nact * P.blk, bar);
    if (fp16)
      bulk_g2s(smem_addr(dst + a.G * P.blk), reinterpret_cast<const unsigned char*>(a.x.norm) + h0 * P.sblk,
               nact * P.sblk, bar);
  }
}

// (re, im) of pair j of site i from a slot holding G site blocks
template <class S>
__device__ __forceinline__ void read_pair(const Pipe<S>& P, const unsigned char* slot, int i, int j, float2* re,
                                          float2* im) {
  const int Lh = P.a->Lh;
  if constexpr (sizeof(S) == 4) {
    const float4* c4 = reinterpret_cast<const float4*>(slot + i * P.blk);
#pragma unroll
    for (int k = 0; k < 12; ++k) unpack_chunk(c4[k * Lh + j], re[k], im[k]);
  } else {
    const uint2* c2 = reinterpret_cast<const uint2*>(slot + i * P.blk);
    const float2 sc = reinterpret_cast<const float2*>(slot + P.a->G * P.blk + i * P.sblk)[j];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const uint2 v = c2[k * Lh + j];
      const float2 r = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
      const float2 m = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
      re[k] = make_float2(r.x * sc.x, r.y * sc.y);
      im[k] = make_float2(m.x * sc.x, m.y * sc.y);
    }
  }
}

template <class S, int DAG, int HX>
__global__ void __launch_bounds__(32, 11) hop3_kernel(const Hop3Args<S> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bars[2];
  const int Lh = a.Lh, G = a.G, Ls = a.Ls;
  const int lane = threadIdx.x;
  const int i = lane / Lh;
  const int j = lane - i * Lh;
  Pipe<S> P;
  P.a = &a;
  P.sm = sm;
  P.bar0 = smem_addr(&bars[0]);
  P.nstage = HX ? 9 : 8;
  P.blk = 12 * Lh * chunk_bytes<S>();
  P.sblk = Lh * 8;
  const float4* dup = reinterpret_cast<const float4*>(sm + a.ctx.dup_off);
  if (lane == 0) {
    mbar_init(P.bar0, 1);
    mbar_init(P.bar0 + 8, 1);
    fence_async_smem();
  }
  __syncwarp();
  const long stride = gridDim.x;
  // neighbour indices of the current and the next group (lane = site)
  int nb_cur[8], nb_next[8];
  auto load_nb = [&](long g, int* nb) {
#pragma unroll
    for (int d = 0; d < 8; ++d) nb[d] = 0;
    if (g < a.ngroups && lane < G) {
      const long hh = g * G + lane;
      if (hh < a.Vh) {
#pragma unroll
        for (int d = 0; d < 8; ++d) nb[d] = __ldg(a.nbr + (long)d * a.Vh + hh);
      }
    }
  };
  long g = blockIdx.x;
  load_nb(g, nb_cur);
  issue_stage<S>(P, g, 0, 0, nb_cur[0]);
  issue_stage<S>(P, g, 1, 1, nb_cur[1]);
  unsigned seq = 0;  // index of the stage being consumed
  bool bad = false;
  double part = 0.0;
  for (; g < a.ngroups; g += stride) {
    load_nb(g + stride, nb_next);
    const long h0 = g * G;
    const long left = a.Vh - h0;
    const int nact = left < G ? (int)left : G;
    const bool act = i < nact;
    float2 ar[12], ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      ar[k] = make_float2(0.f, 0.f);
      ai[k] = ar[k];
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      const int slot = seq & 1;
      if (!mbar_wait(P.bar0 + 8u * slot, (seq >> 1) & 1)) bad = true;
      const unsigned char* sl = sm + slot * a.ctx.slot_bytes;
      if (d == 0) {
        // expand this group's links to (ur, ur, ui, ui)
        const S* raw = reinterpret_cast<const S*>(sm + a.ctx.raw_off);
        float4* dw = reinterpret_cast<float4*>(sm + a.ctx.dup_off);
        for (int q = lane; q < nact * 72; q += 32) {
          float ur, ui;
          if constexpr (sizeof(S) == 4) {
            const float2 v = reinterpret_cast<const float2*>(raw)[q];
            ur = v.x;
            ui = v.y;
          } else {
            const float2 v = __half22float2(reinterpret_cast<const __half2*>(raw)[q]);
            ur = v.x;
            ui = v.y;
          }
          dw[(q / 72) * kDupStride + q % 72] = make_float4(ur, ur, ui, ui);
        }
        __syncwarp();
      }
      if (act) {
        float2 pr[12], pi[12];
        read_pair<S>(P, sl, i, j, pr, pi);
        const float4* U = dup + i * kDupStride + d * 9;
        constexpr int F = DAG ? -1 : 1;
        if (d == 0) hop_dir2<0, F>(pr, pi, U, ar, ai);
        if (d == 1) hop_dir2<1, F>(pr, pi, U, ar, ai);
        if (d == 2) hop_dir2<2, F>(pr, pi, U, ar, ai);
        if (d == 3) hop_dir2<3, F>(pr, pi, U, ar, ai);
        if (d == 4) hop_dir2<0, -F>(pr, pi, U, ar, ai);
        if (d == 5) hop_dir2<1, -F>(pr, pi, U, ar, ai);
        if (d == 6) hop_dir2<2, -F>(pr, pi, U, ar, ai);
        if (d == 7) hop_dir2<3, -F>(pr, pi, U, ar, ai);
      }
      __syncwarp();
      // refill this slot with the stage two ahead (unless this was the group's last stage)
      constexpr int NST = HX ? 9 : 8;
      if (!(NST == 8 && d == 7)) {
        const int k2 = d + 2;
        if (k2 < NST)
          issue_stage<S>(P, g, k2, slot, nb_cur[k2 < 8 ? k2 : 0]);
        else
          issue_stage<S>(P, g + stride, k2 - NST, slot, nb_next[k2 - NST < 8 ? k2 - NST : 0]);
      }
      ++seq;
    }
    // epilogue
    const float sc = a.scale;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      ar[k] = make_float2(ar[k].x * sc, ar[k].y * sc);
      ai[k] = make_float2(ai[k].x * sc, ai[k].y * sc);
    }
    const int last_slot = (seq - 1) & 1;
    if (HX) {
      const int slot = seq & 1;
      if (!mbar_wait(P.bar0 + 8u * slot, (seq >> 1) & 1)) bad = true;
      float2 xr[12], xi[12];
      if (act) read_pair<S>(P, sm + slot * a.ctx.slot_bytes, i, j, xr, xi);
      __syncwarp();
      float* tile = reinterpret_cast<float*>(sm + slot * a.ctx.slot_bytes);
      if (a.ex.kind != 0) sop_pair(a.ex, xr, xi, tile, i, j, act, nact, Ls, Lh);
      const float2 xs = f2(a.xscale);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        ar[k] = fma2(xs, xr[k], ar[k]);
        ai[k] = fma2(xs, xi[k], ai[k]);
      }
      if (a.eout.kind != 0) sop_pair(a.eout, ar, ai, tile, i, j, act, nact, Ls, Lh);
      issue_stage<S>(P, g + stride, 1, slot, nb_next[1]);
      ++seq;
    } else {
      float* tile = reinterpret_cast<float*>(sm + last_slot * a.ctx.slot_bytes);
      if (a.eout.kind != 0) sop_pair(a.eout, ar, ai, tile, i, j, act, nact, Ls, Lh);
      issue_stage<S>(P, g + stride, 1, last_slot, nb_next[1]);
    }
    if (j + Lh >= Ls) {  // odd Ls: the padding slot stays zero
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        ar[k].y = 0.f;
        ai[k].y = 0.f;
      }
    }
    if (act && !bad) {
      const long h = h0 + i;
      store_pair(a.out, h, j, Lh, ar, ai);
      if (a.partials) {
        float ps = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ps = fmaf(ar[k].x, ar[k].x, fmaf(ar[k].y, ar[k].y, ps));
          ps = fmaf(ai[k].x, ai[k].x, fmaf(ai[k].y, ai[k].y, ps));
        }
        part += (double)ps;
      }
    }
#pragma unroll
    for (int d = 0; d < 8; ++d) nb_cur[d] = nb_next[d];
  }
  if (bad) {
    if (lane == 0) atomicExch(a.err, 1);
    mbar_wait(P.bar0, (seq >> 1) & 1);  // once more, bounded, for copies still in flight
    mbar_wait(P.bar0 + 8, (seq >> 1) & 1);
  }
  if (a.partials) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if (lane == 0) a.partials[blockIdx.x] = part;
  }
}

}  // namespace

// Sites per group for the pipelined kernel, or 0 if the shape needs the per-slice kernel.
int hop2_sites(int Ls, int prec) {
  const int Lh = (Ls + 1) / 2;
  if (prec != DWF_F32 && prec != DWF_F16) return 0;
  if (Lh > 32) return 0;
  if (prec == DWF_F16 && (Lh % 2)) return 0;  // FP16 scale blocks must be multiples of 16 bytes
  return 32 / Lh;
}

template <class S>
static dwf_status hop3_t(dwf_lattice* L, const HopCall& c, const SOpK<float>& ex, const SOpK<float>& eout, int G) {
  Hop3Args<S> a;
  a.in = CFieldRef<S>{reinterpret_cast<const S*>(c.in.v), c.in.norm};
  a.out = FieldRef<S>{reinterpret_cast<S*>(c.out.v), c.out.norm};
  a.x = c.has_x ? CFieldRef<S>{reinterpret_cast<const S*>(c.x.v), c.x.norm} : CFieldRef<S>{nullptr, nullptr};
  a.links = reinterpret_cast<const S*>(L->links[c.in.prec][c.out_parity]);
  a.nbr = L->nbr[c.out_parity];
  a.Vh = L->Vh;
  a.G = G;
  a.ngroups = (L->Vh + G - 1) / G;
  a.Ls = L->Ls;
  a.Lh = L->Lh;
  a.ctx = make_ctx(L->Ls, c.in.prec, G);
  a.ex = ex;
  a.eout = eout;
  a.scale = (float)c.scale;
  a.xscale = (float)c.xscale;
  a.partials = c.partials;
  a.err = L->dev_err;
  // persistent grid: enough warps to keep every SM's copy engine and issue slots busy
  const long want = 152L * 12;
  const long grid = a.ngroups < want ? a.ngroups : want;
  const size_t smem = (size_t)a.ctx.total;
  auto run = [&](auto kern) -> dwf_status {
    DWF_CUDA(L, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<(unsigned)grid, 32, smem, L->stream>>>(a);
    return DWF_OK;
  };
  if (c.dag)
    DWF_TRY(c.has_x ? run(hop3_kernel<S, 1, 1>) : run(hop3_kernel<S, 1, 0>));
  else
    DWF_TRY(c.has_x ? run(hop3_kernel<S, 0, 1>) : run(hop3_kernel<S, 0, 0>));
  if (c.nblocks) *c.nblocks = (int)grid;
  return DWF_OK;
}

dwf_status launch_hop2(dwf_lattice* L, const HopCall& c, const SOpK<float>& ex, const SOpK<float>& eout, int G) {
  if (c.in.prec == DWF_F32) return hop3_t<float>(L, c, ex, eout, G);
  return hop3_t<__half>(L, c, ex, eout, G);
}

}  // namespace dwf
