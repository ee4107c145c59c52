// Wilson hop at every fifth-dimension slice for FP32- and FP16-stored
// spinors (FP32 arithmetic), the bandwidth-critical kernel of the mixed
// precision and MADWF solves:
//
//   out(n,.) = Eout( xscale * Ex x(n,.) + scale * Dhop(in)(n,.) )
//
// (the 4D Wilson hop inside D_DW, Sec. 4 Eq. dirac_eq, on one checkerboard,
// with the fifth-dimension operators of the even-odd Schur form fused).
//
// Two kernels share the design below.  hopf_kernel (further down) is the
// FP32 single-right-hand-side fast path for even Ls with Lh in {4, 6, 8, 16,
// 32}: Lh fixed at compile time, each direction stage carrying its own links,
// every slot refilled as soon as its data are in registers.  hop3_kernel is
// the general one: FP16 storage, odd Ls, dense fifth-dimension fallbacks and
// launches over several right-hand sides.
//
// GB300 design:
//  * Thread (i, j) owns the slice pair (2j, 2j + 1) of 4D site i, so both
//    lanes of every packed FP32x2 FMA (__ffma2_rn) use the same link element.
//  * A CTA is one warp that walks a stream of site groups (G = 32 / Lh
//    consecutive sites per group).  A group is a sequence of stages: the 8
//    directions (the neighbour blocks of that direction -- a neighbour's 5D
//    spinor block is contiguous in the pair layout, and the neighbours of
//    consecutive sites are usually consecutive, so a stage is one bulk copy;
//    stage 0 also brings the group's links) and, if the hop has a site term,
//    the group's own blocks.  A launch over several right-hand sides (a mass
//    ladder) runs these stages for each of them in turn, so a group's links
//    and neighbour indices are staged once for all of them.  Stages are
//    fetched by the bulk copy engine (cp.async.bulk, completion counted on an
//    mbarrier per slot) into a ring of kSlots shared-memory slots in issue
//    order, across group boundaries; no block barrier exists.  Two slots (one
//    stage in flight per warp) leave room for more resident warps, which
//    measured faster than deeper rings.
//  * Links are read once per group from shared memory and reused over all Ls
//    slices (and right-hand sides).
//  * The fifth-dimension epilogue stays in registers for even Ls: the s
//    recurrence of an inverse is a log-depth scan across the site's lanes by
//    warp shuffles; odd Ls and dense fallbacks go through a shared-memory
//    tile in the slot just consumed.
//  * Waits on the mbarriers are bounded (the consumer's limit is a launch
//    argument, normally kWaitLimit polls): a wait that gives up sets the
//    handle's device error flag (reported as DWF_ERR_TIMEOUT); the warp then
//    stops at once (a warp vote makes the decision uniform), issues no
//    further copy, waits -- with the normal limit -- for every copy it has
//    issued and not consumed, so that no bulk copy is still writing into its
//    shared memory when it exits, and returns.
#include <map>
#include <mutex>

#include "dwf_internal.h"

#include "hop_common.cuh"

namespace dwf {

namespace {

constexpr long kWaitLimit = kHopWaitLimit;
constexpr int kSlots = 2;

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
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity, long limit = kWaitLimit) {
  for (long it = 0; it < limit; ++it)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// z = a + c b on complex pairs, c = sg * (CR + i CI) with the unit (CR, CI)
// fixed at compile time and the sign sg = +-1 at run time (sgp = (sg, sg)).
template <int CR, int CI>
__device__ __forceinline__ void cpair_s(float2 sgp, float2 ar, float2 ai, float2 br, float2 bi, float2& zr,
                                        float2& zi) {
  if constexpr (CI == 0) {
    const float2 c = CR == 1 ? sgp : make_float2(-sgp.x, -sgp.y);
    zr = fma2(c, br, ar);
    zi = fma2(c, bi, ai);
  } else {
    const float2 c = CI == 1 ? sgp : make_float2(-sgp.x, -sgp.y);
    zr = fma2(make_float2(-c.x, -c.y), bi, ar);
    zi = fma2(c, br, ai);
  }
}

// acc += (1 - sg g_MU) U psi on a slice pair; psi given by (pr, pi)[12], link
// U as 9 complex (ur, ui), broadcast to both lanes.  Every coefficient of the
// projector is proportional to sg, so one body serves both signs (forward
// and backward neighbours, and the dagger), which keeps the kernel's code
// small enough for the instruction cache.
template <int MU>
__device__ __forceinline__ void hop_dir2(float sg, const float2* pr, const float2* pi, const float2* U, float2* ar,
                                         float2* ai) {
  typedef Proj<MU, 1> P;
  const float2 sgp = f2(sg);
  float2 hr[6], hi[6];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    cpair_s<P::C1R, P::C1I>(sgp, pr[a], pi[a], pr[P::J1 * 3 + a], pi[P::J1 * 3 + a], hr[a], hi[a]);
    cpair_s<P::C2R, P::C2I>(sgp, pr[3 + a], pi[3 + a], pr[P::J2 * 3 + a], pi[P::J2 * 3 + a], hr[3 + a], hi[3 + a]);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 ur[3], ui[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      ur[b] = f2(U[3 * a + b].x);
      ui[b] = f2(U[3 * a + b].y);
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      // g = sum_b U_ab h_b :  gr = sum ur hr - sum ui hi,  gi = sum ur hi + sum ui hr
      float2 A = make_float2(0.f, 0.f), B = A, C = A, D = A;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        A = fma2(ur[b], hr[3 * hh + b], A);
        B = fma2(ui[b], hi[3 * hh + b], B);
        C = fma2(ur[b], hi[3 * hh + b], C);
        D = fma2(ui[b], hr[3 * hh + b], D);
      }
      const float2 gr = fma2(f2(-1.f), B, A), gi = add2(C, D);
      ar[3 * hh + a] = add2(ar[3 * hh + a], gr);  // upper spins 0, 1
      ai[3 * hh + a] = add2(ai[3 * hh + a], gi);
      // lower spins 2, 3: += d g with d = sg * (DR + i DI)
      if (hh == P::S2) {
        float2 zr, zi;
        cpair_s<P::D2R, P::D2I>(sgp, ar[6 + a], ai[6 + a], gr, gi, zr, zi);
        ar[6 + a] = zr;
        ai[6 + a] = zi;
      }
      if (hh == P::S3) {
        float2 zr, zi;
        cpair_s<P::D3R, P::D3I>(sgp, ar[9 + a], ai[9 + a], gr, gi, zr, zi);
        ar[9 + a] = zr;
        ai[9 + a] = zi;
      }
    }
  }
}

// bytes of one complex-component chunk of a slice pair
template <class S> __host__ __device__ constexpr int chunk_bytes() { return sizeof(S) == 4 ? 16 : 8; }

// Write the pair (re, im) of slices 2j, 2j + 1 of tile block bi into the s-op tile.
__device__ __forceinline__ void tile_put_pair(float* tile, int R, int bi, int j, int Lh, int Ls, const float2* re,
                                              const float2* im) {
  float* base = tile + (bi * 12) * R;
  const bool two = 2 * j + 1 < Ls;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    reinterpret_cast<float2*>(base + k * R)[2 * j] = make_float2(re[k].x, im[k].x);
    if (two) reinterpret_cast<float2*>(base + k * R)[2 * j + 1] = make_float2(re[k].y, im[k].y);
  }
}
__device__ __forceinline__ void tile_get_pair(const float* tile, int R, int bi, int j, int Lh, int Ls, float2* re,
                                              float2* im) {
  const float* base = tile + (bi * 12) * R;
  const bool two = 2 * j + 1 < Ls;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    const float2 a = reinterpret_cast<const float2*>(base + k * R)[2 * j];
    const float2 b = two ? reinterpret_cast<const float2*>(base + k * R)[2 * j + 1] : make_float2(0.f, 0.f);
    re[k] = make_float2(a.x, b.x);
    im[k] = make_float2(a.y, b.y);
  }
}

// y <- op y on the slice pairs a lane holds, for a structured operator and
// even Ls >= 2, without shared memory: the Ls slices of a site live in its Lh
// lanes base .. base + Lh - 1, slice 2j in .x and 2j + 1 in .y of lane
// base + j.  With u = x / g2, the inverse (g2 + d2 Q)^-1 is the first-order
// recurrence z_s = rho z_{s-1} + u_s closed by the wall term -m: each lane
// first folds its own two slices, a log-depth scan across the lanes (factor
// rho^2 per lane) gives the open prefix P at every odd slice, one more
// neighbour value gives it at the even ones, and the wall adds rho^s w with
// w = -rho m P_{Ls-1} / (1 + m rho^Ls).  Rows that walk down in s (P- rows,
// or P+ rows of a transposed operator) use the mirrored suffix form.
// y = g1 z + d1 Q z then needs one neighbouring slice, at most one shuffle
// away.  The (re, im) pair of a slice moves as one float2.
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

__device__ __forceinline__ void sop_shfl(const SOpK<float>& op, float2* re, float2* im, int j, int Lh) {
  const int lane = threadIdx.x, base = lane - j;
  const float rho = op.rho, m = op.m;
  // lane powers of rho: rho^(2j), rho^(Ls-1-2j) (Ls = 2 Lh)
  float p2j = 1.f, pr2j = 1.f;
  if (op.has_inv)
    for (int q = 0; q < Lh; ++q) {
      if (q < j) p2j *= rho * rho;
      if (q > j) pr2j *= rho * rho;
    }
  const float wk = op.has_inv ? -rho * m * (op.c0 / op.ginv) : 0.f;  // -rho m / (1 + m rho^Ls)
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int up = half ^ op.trans;  // 0: z_s from z_{s-1} (prefix); 1: from z_{s+1} (suffix)
    // per component k: a = slice 2j, b = slice 2j + 1, each (re, im)
    float2 A[6], B[6];
    const float2 gi = f2(op.ginv);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kk = 6 * half + k;
      A[k] = mul2(gi, make_float2(re[kk].x, im[kk].x));
      B[k] = mul2(gi, make_float2(re[kk].y, im[kk].y));
    }
    if (op.has_inv) {
      const float2 r1 = f2(rho);
      if (!up) {
        // fold the lane's two slices, scan the odd-slice values across lanes
#pragma unroll
        for (int k = 0; k < 6; ++k) B[k] = fma2(r1, A[k], B[k]);
        float rd = rho * rho;
        for (int d = 1; d < Lh; d <<= 1) {
          const bool ok = j >= d;
          const int src = ok ? lane - d : lane;
          const float2 f = f2(ok ? rd : 0.f);
#pragma unroll
          for (int k = 0; k < 6; ++k) B[k] = fma2(f, shfl2(B[k], src), B[k]);
          rd *= rd;
        }
        // even slices: P_{2j} = u_{2j} + rho P_{2j-1}; then the wall, P_{Ls-1} in .y of the last lane
        const int src = j > 0 ? lane - 1 : lane;
        const float2 f = f2(j > 0 ? rho : 0.f);
        const float2 ps = make_float2(p2j, p2j * rho);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          A[k] = fma2(f, shfl2(B[k], src), A[k]);
          const float2 w = mul2(f2(wk), shfl2(B[k], base + Lh - 1));
          A[k] = fma2(f2(ps.x), w, A[k]);
          B[k] = fma2(f2(ps.y), w, B[k]);
        }
      } else {
        // mirrored: fold from the right, scan the even-slice values across lanes
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = fma2(r1, B[k], A[k]);
        float rd = rho * rho;
        for (int d = 1; d < Lh; d <<= 1) {
          const bool ok = j + d < Lh;
          const int src = ok ? lane + d : lane;
          const float2 f = f2(ok ? rd : 0.f);
#pragma unroll
          for (int k = 0; k < 6; ++k) A[k] = fma2(f, shfl2(A[k], src), A[k]);
          rd *= rd;
        }
        // odd slices: S_{2j+1} = u_{2j+1} + rho S_{2j+2}; then the wall, S_0 in .x of the first lane
        const int src = j < Lh - 1 ? lane + 1 : lane;
        const float2 f = f2(j < Lh - 1 ? rho : 0.f);
        const float2 ps = make_float2(pr2j * rho, pr2j);  // rho^(Ls-1-2j), rho^(Ls-2-2j)
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          B[k] = fma2(f, shfl2(A[k], src), B[k]);
          const float2 w = mul2(f2(wk), shfl2(A[k], base));
          A[k] = fma2(f2(ps.x), w, A[k]);
          B[k] = fma2(f2(ps.y), w, B[k]);
        }
      }
    }
    // y = g1 z + d1 Q z: the neighbouring slice (in this lane or the next /
    // previous one), or -m times the slice at the other wall
    const float2 g1 = f2(op.g1), d1 = f2(op.d1);
    const bool edge = up ? (j == Lh - 1) : (j == 0);
    const int src = up ? (edge ? base : lane + 1) : (edge ? base + Lh - 1 : lane - 1);
    const float2 fe = f2(edge ? -m : 1.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kk = 6 * half + k;
      float2 ya, yb;
      if (!up) {
        const float2 q = mul2(fe, shfl2(B[k], src));  // slice 2j-1 (or -m slice Ls-1)
        ya = fma2(d1, q, mul2(g1, A[k]));
        yb = fma2(d1, A[k], mul2(g1, B[k]));
      } else {
        const float2 q = mul2(fe, shfl2(A[k], src));  // slice 2j+2 (or -m slice 0)
        ya = fma2(d1, B[k], mul2(g1, A[k]));
        yb = fma2(d1, q, mul2(g1, B[k]));
      }
      re[kk] = make_float2(ya.x, yb.x);
      im[kk] = make_float2(ya.y, yb.y);
    }
  }
}

// (re, im) <- op (re, im) for slot block bi, pair j (every lane calls): in
// registers for a structured operator and even Ls, otherwise through the
// shared-memory tile (the slot just consumed).
__device__ __forceinline__ void sop_pair(const SOpK<float>& op, float2* re, float2* im, float* tile, int bi, int j,
                                         bool act, int G, int nact, int Ls, int Lh) {
  if (op.kind == 1 && !(Ls & 1)) {
    sop_shfl(op, re, im, j, Lh);
    return;
  }
  const int R = tile_row(Ls);
  if (act) tile_put_pair(tile, R, bi, j, Lh, Ls, re, im);
  __syncwarp();
  if (op.kind == 1) {
    for (int w = threadIdx.x; w < nact * 12; w += 32) sop_row(op, tile + w * R, w % 12, Ls);
    __syncwarp();
    if (act) tile_get_pair(tile, R, bi, j, Lh, Ls, re, im);
  } else if (act) {
    // dense fallback: row s of the (already transposed where needed) matrix
    const float* base = tile + (bi * 12) * R;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      re[k] = make_float2(0.f, 0.f);
      im[k] = re[k];
    }
    const int s0 = 2 * j, s1 = 2 * j + 1 < Ls ? 2 * j + 1 : 2 * j;
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
    if (!(2 * j + 1 < Ls))
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        re[k].y = 0.f;
        im[k].y = 0.f;
      }
  }
  __syncwarp();
}

// ---------------------------------------------------------------- the pipelined kernel

struct Ctx {        // per-CTA shared-memory layout (byte offsets)
  int slot_bytes;   // one ring slot: G site blocks (+ FP16 scales), or the s-op tile
  int raw_off;      // two link buffers (groups alternate), one padded block per site
  int link_stride;  // bytes between two sites' link blocks
  int nb_off;       // neighbour indices [2 groups][8 directions][G sites]
  int part_off;     // per-right-hand-side partial sums [kMaxBatch][32] (batched launches)
  int total;
};

// need_tile: an epilogue runs through shared memory (odd Ls or a dense operator)
__host__ __device__ inline Ctx make_ctx(int Ls, int prec, int G, bool batched, bool need_tile) {
  const int Lh = (Ls + 1) / 2;
  const int cb = prec == DWF_F32 ? 16 : 8;
  const int blocks = G * 12 * Lh * cb + (prec == DWF_F16 ? G * Lh * 8 : 0);
  const int tile = need_tile ? G * 12 * tile_row(Ls) * 4 : 0;
  int slot = blocks > tile ? blocks : tile;
  slot = (slot + 127) / 128 * 128;
  Ctx c;
  c.slot_bytes = slot;
  c.raw_off = kSlots * slot;
  // 8 links x 18 reals per site, +16 bytes so consecutive sites start in different banks
  c.link_stride = 8 * 18 * (prec == DWF_F32 ? 4 : 2) + 16;
  c.nb_off = c.raw_off + 2 * G * c.link_stride;
  c.part_off = (c.nb_off + 2 * 8 * G * 4 + 7) / 8 * 8;
  c.total = c.part_off + (batched ? kMaxBatch * 32 * 8 : 0);
  return c;
}

// One launch over nr right-hand sides that share the links (nr = 1: a single field).
template <class S> struct Hop3Args {
  CFieldRef<S> in[kMaxBatch];
  FieldRef<S> out[kMaxBatch];
  CFieldRef<S> x[kMaxBatch];
  SOpK<float> ex[kMaxBatch], eout[kMaxBatch];
  double* partials[kMaxBatch];  // per right-hand side, one double per CTA (or null)
  const S* links;               // [Vh][8][18]
  const int* nbr;               // [8][Vh]
  long Vh;
  long ngroups;
  int Ls, Lh, G, nr;
  Ctx ctx;
  float scale, xscale;
  int* err;
  long wait_limit;  // polls of a consumer wait before it gives up
};

template <class S> struct Pipe {
  const Hop3Args<S>* a;
  unsigned char* sm;
  unsigned bar0;
  int blk, sblk;
  int* nbs;  // neighbour table in shared memory
};

// Issue stage t of group g into ring slot `slot` (all lanes call).  Stage
// t = r * NST + d of a group is, for right-hand side r, neighbour direction
// d < 8 (the G neighbour blocks, site i into slot block i; stage 0 also brings
// the group's links) or d = 8, the group's own blocks of the site term.  The
// group's neighbour indices and links sit in buffer lb.
template <class S, int NST>
__device__ __forceinline__ bool issue_stage(const Pipe<S>& P, long g, int t, int slot, int lb) {
  const Hop3Args<S>& a = *P.a;
  if (g >= a.ngroups) return false;  // past the CTA's last group: nothing issued
  const int r = t / NST, d = t - r * NST;
  const long h0 = g * a.G;
  const long left = a.Vh - h0;
  const int nact = left < a.G ? (int)left : a.G;
  const int lane = threadIdx.x;
  const unsigned bar = P.bar0 + 8u * slot;
  unsigned char* dst = P.sm + slot * a.ctx.slot_bytes;
  const bool fp16 = sizeof(S) == 2;
  const int lbytes = 8 * 18 * (int)sizeof(S);
  const int G = a.G;
  // earlier generic-proxy reads of this slot must be ordered before the copies
  fence_async_smem();
  const unsigned bytes = nact * (P.blk + (fp16 ? P.sblk : 0)) + (t == 0 ? nact * lbytes : 0);
  if (lane == 0) mbar_expect_tx(bar, bytes);
  __syncwarp();
  if (d < 8) {
    const CFieldRef<S> src = a.in[r];
    const int nb_k = lane < G ? P.nbs[(lb * 8 + d) * G + lane] : 0;
    // When the group's neighbours in this direction are consecutive sites (a
    // group inside one x-row, whose y/z/t neighbours shift as a block), one
    // copy moves them all; otherwise one copy per site.
    const int nb0 = __shfl_sync(0xffffffffu, nb_k, 0);
    const unsigned run = __ballot_sync(0xffffffffu, lane >= nact || nb_k == nb0 + lane);
    if (run == 0xffffffffu) {
      if (lane == 0) {
        bulk_g2s(smem_addr(dst), reinterpret_cast<const unsigned char*>(src.v) + (long)nb0 * P.blk, nact * P.blk,
                 bar);
        if (fp16)
          bulk_g2s(smem_addr(dst + G * P.blk), reinterpret_cast<const unsigned char*>(src.norm) + (long)nb0 * P.sblk,
                   nact * P.sblk, bar);
      }
    } else if (lane < nact) {
      bulk_g2s(smem_addr(dst + lane * P.blk), reinterpret_cast<const unsigned char*>(src.v) + (long)nb_k * P.blk,
               P.blk, bar);
      if (fp16)
        bulk_g2s(smem_addr(dst + G * P.blk + lane * P.sblk),
                 reinterpret_cast<const unsigned char*>(src.norm) + (long)nb_k * P.sblk, P.sblk, bar);
    }
    if (t == 0 && lane < nact) {
      // the links of consecutive groups of this CTA alternate between two
      // buffers: this copy is issued while the previous group still reads its own
      bulk_g2s(smem_addr(P.sm + a.ctx.raw_off + (lb * G + lane) * a.ctx.link_stride),
               a.links + (h0 + lane) * 8 * 18, lbytes, bar);
    }
  } else if (lane == 0) {
    const CFieldRef<S> src = a.x[r];
    bulk_g2s(smem_addr(dst), reinterpret_cast<const unsigned char*>(src.v) + h0 * P.blk, nact * P.blk, bar);
    if (fp16)
      bulk_g2s(smem_addr(dst + G * P.blk), reinterpret_cast<const unsigned char*>(src.norm) + h0 * P.sblk,
               nact * P.sblk, bar);
  }
  return true;
}

// (re, im) of pair j of slot block bi
template <class S>
__device__ __forceinline__ void read_pair(const Pipe<S>& P, const unsigned char* slot, int bi, int j, float2* re,
                                          float2* im) {
  const int Lh = P.a->Lh;
  if constexpr (sizeof(S) == 4) {
    const float4* c4 = reinterpret_cast<const float4*>(slot + bi * P.blk);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const float4 v = c4[k * Lh + j];
      re[k] = make_float2(v.x, v.y);
      im[k] = make_float2(v.z, v.w);
    }
  } else {
    const uint2* c2 = reinterpret_cast<const uint2*>(slot + bi * P.blk);
    const float2 sc = reinterpret_cast<const float2*>(slot + P.a->G * P.blk + bi * P.sblk)[j];
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

// links of site i, direction d, from link buffer lb, as 9 complex (ur, ui) in FP32
template <class S>
__device__ __forceinline__ void site_links(const Pipe<S>& P, int lb, int i, int d, float2* U) {
  const unsigned char* base = P.sm + P.a->ctx.raw_off + (lb * P.a->G + i) * P.a->ctx.link_stride;
  if constexpr (sizeof(S) == 4) {
    const float2* u = reinterpret_cast<const float2*>(base) + d * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = u[e];
  } else {
    const __half2* u = reinterpret_cast<const __half2*>(base) + d * 9;
#pragma unroll
    for (int e = 0; e < 9; ++e) U[e] = __half22float2(u[e]);
  }
}

// Lane (i, j) = (lane / Lh, lane % Lh) owns slice pair j of site i of a group
// of G consecutive sites.  A batched launch (BATCH = 1) walks the group's
// stages for each right-hand side in turn: the links and neighbour indices
// of a group are staged once for all of them, every other quantity is the
// single-field kernel's.
template <class S, int DAG, int HX, int BATCH>
__global__ void __launch_bounds__(32, 12) hop3_kernel(const Hop3Args<S> a) {
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bars[kSlots];
  __shared__ double red[32];
  constexpr int NST = HX ? 9 : 8;  // stages per right-hand side and group
  const int Lh = a.Lh, G = a.G, Ls = a.Ls;
  const int NSG = BATCH ? a.nr * NST : NST;  // stages per group
  const int lane = threadIdx.x;
  const int i = lane / Lh;
  const int j = lane - i * Lh;
  const int bi = i;  // this lane's block in a slot or the tile
  double* sp = reinterpret_cast<double*>(sm + a.ctx.part_off);  // batched: [kMaxBatch][32]
  Pipe<S> P;
  P.a = &a;
  P.sm = sm;
  P.bar0 = smem_addr(&bars[0]);
  P.blk = 12 * Lh * chunk_bytes<S>();
  P.sblk = Lh * 8;
  P.nbs = reinterpret_cast<int*>(sm + a.ctx.nb_off);
  if (lane == 0) {
    for (int s = 0; s < kSlots; ++s) mbar_init(P.bar0 + 8u * s, 1);
    fence_async_smem();
  }
  if (BATCH)
    for (int q = 0; q < kMaxBatch; ++q) sp[q * 32 + lane] = 0.0;
  __syncwarp();
  const long stride = gridDim.x;
  // neighbour indices of a group for this lane's site, into buffer lb
  // (each lane reads back only what it wrote)
  auto load_nb = [&](long g, int lb) {
    if (lane < G) {
      const long hh = g * G + lane;
      const bool ok = g < a.ngroups && hh < a.Vh;
#pragma unroll
      for (int d = 0; d < 8; ++d) P.nbs[(lb * 8 + d) * G + lane] = ok ? __ldg(a.nbr + (long)d * a.Vh + hh) : 0;
    }
  };
  long g = blockIdx.x;
  load_nb(g, 0);
  unsigned issued = 0;  // stages issued so far (issue order = consumption order)
#pragma unroll
  for (int s = 0; s < kSlots; ++s) issued += issue_stage<S, NST>(P, g, s, s, 0);
  unsigned seq = 0;  // global index of the stage being consumed; slot seq % kSlots
  bool bad = false;
  double part = 0.0;
  int lb = 0;  // this group's link / neighbour buffer; groups of a CTA alternate
  for (; g < a.ngroups; g += stride, lb ^= 1) {
    load_nb(g + stride, lb ^ 1);
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
#pragma unroll 1
    for (int t = 0; t < NSG; ++t) {
      const int r = BATCH ? t / NST : 0;
      const int d = t - r * NST;
      const int slot = seq % kSlots;
      unsigned char* sl = sm + slot * a.ctx.slot_bytes;
      if (__any_sync(0xffffffffu, !mbar_wait(P.bar0 + 8u * slot, (seq / kSlots) & 1, a.wait_limit))) {
        bad = true;
        break;
      }
      float2 xr[12], xi[12];  // the site term (d = 8)
      if (d < 8) {
        if (act) {
          float2 pr[12], pi[12], U[9];
          read_pair<S>(P, sl, bi, j, pr, pi);
          site_links<S>(P, lb, i, d, U);
          // (1 - sg g_mu): sg = +1 forward / -1 backward, flipped by the dagger
          const float sg = ((d < 4) != (DAG != 0)) ? 1.f : -1.f;
          switch (d & 3) {
            case 0: hop_dir2<0>(sg, pr, pi, U, ar, ai); break;
            case 1: hop_dir2<1>(sg, pr, pi, U, ar, ai); break;
            case 2: hop_dir2<2>(sg, pr, pi, U, ar, ai); break;
            default: hop_dir2<3>(sg, pr, pi, U, ar, ai); break;
          }
        }
      } else if (HX) {
        if (act) read_pair<S>(P, sl, bi, j, xr, xi);
      }
      __syncwarp();
      // refill this slot with the stage kSlots ahead; after the last stage of
      // a right-hand side the slot first serves as the epilogue's tile
      const bool last = d == NST - 1;
      const int k2 = t + kSlots;
      if (!last) {
        if (k2 < NSG)
          issued += issue_stage<S, NST>(P, g, k2, slot, lb);
        else
          issued += issue_stage<S, NST>(P, g + stride, k2 - NSG, slot, lb ^ 1);
      }
      ++seq;
      if (last) {
        // epilogue for right-hand side r
        const float2 sc = f2(a.scale);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ar[k] = __fmul2_rn(sc, ar[k]);
          ai[k] = __fmul2_rn(sc, ai[k]);
        }
        float* tile = reinterpret_cast<float*>(sl);
        if (HX) {
          const SOpK<float> ex = a.ex[r];
          if (ex.kind != 0) sop_pair(ex, xr, xi, tile, bi, j, act, G, nact, Ls, Lh);
          const float2 xs = f2(a.xscale);
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            ar[k] = fma2(xs, xr[k], ar[k]);
            ai[k] = fma2(xs, xi[k], ai[k]);
          }
        }
        const SOpK<float> eout = a.eout[r];
        if (eout.kind != 0) sop_pair(eout, ar, ai, tile, bi, j, act, G, nact, Ls, Lh);
        // the delayed refill of the tile's slot
        if (k2 < NSG)
          issued += issue_stage<S, NST>(P, g, k2, slot, lb);
        else
          issued += issue_stage<S, NST>(P, g + stride, k2 - NSG, slot, lb ^ 1);
        if (2 * j + 1 >= Ls) {  // odd Ls: the padding slot stays zero
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            ar[k].y = 0.f;
            ai[k].y = 0.f;
          }
        }
        if (act) {
          store_pair(a.out[r], h0 + i, j, Lh, ar, ai);
          float2 p0 = make_float2(0.f, 0.f), p1 = p0;
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            p0 = fma2(ar[k], ar[k], p0);
            p1 = fma2(ai[k], ai[k], p1);
          }
          const double ps = (double)((p0.x + p0.y) + (p1.x + p1.y));
          if (BATCH)
            sp[r * 32 + lane] += ps;
          else
            part += ps;
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ar[k] = make_float2(0.f, 0.f);
          ai[k] = ar[k];
        }
      }
    }
    if (bad) break;
  }
  if (bad) {
    // stages seq .. issued - 1 are in flight: wait (normal limit) for each
    // before the CTA's shared memory is released
    if (lane == 0) atomicExch(a.err, 1);
    for (unsigned q = seq; q < issued; ++q) mbar_wait(P.bar0 + 8u * (q % kSlots), (q / kSlots) & 1);
    return;
  }
  if (a.partials[0]) {
    // per right-hand side: sum the lanes (i, j) in a fixed order
    if (!BATCH) sp = red;
    if (!BATCH) red[lane] = part;
    __syncwarp();
    const int nr = BATCH ? a.nr : 1;
    if (lane < nr) {
      double t = 0.0;
      for (int q = 0; q < G * Lh; ++q) t += sp[lane * 32 + q];
      a.partials[lane][blockIdx.x] = t;
    }
  }
}

// ---------------------------------------------------------------- the FP32 fast path
//
// Single right-hand side, FP32 storage, even Ls with structured fifth-dimension
// operators, Lh (and so G = 32 / Lh) fixed at compile time.  Differences from
// hop3_kernel, each measured on GB300:
//  * a direction stage carries its G sites' links for that direction (one
//    contiguous copy from the direction-major link array), so no per-group link
//    buffer is kept and the warp's shared memory is two slots plus the
//    neighbour indices;
//  * a slot is refilled as soon as its data are in registers: the neighbour
//    spinor is spin-projected straight out of shared memory into the 6-complex
//    half spinor and the direction's links are loaded, then the copy for the
//    stage two ahead is issued, before the SU(3) products;
//  * the site term, if any, is the group's first stage: its fifth-dimension
//    operator runs on it at once and it seeds the accumulator (scaled by
//    xscale / scale, the hop sum is scaled at the end);
//  * compile-time Lh turns the slot addressing into immediates and unrolls the
//    epilogue's scan; the epilogue's per-lane powers of rho are computed once.

// psi projected by (1 - sg g_MU) straight from the slot block of this lane's
// site (chunk j of each complex component)
template <int MU>
__device__ __forceinline__ void project_smem(float sg, const float4* c4, int j, int Lh, float2* hr, float2* hi) {
  typedef Proj<MU, 1> P;
  const float2 sgp = f2(sg);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float4 v0 = c4[a * Lh + j], v1 = c4[(P::J1 * 3 + a) * Lh + j];
    cpair_s<P::C1R, P::C1I>(sgp, make_float2(v0.x, v0.y), make_float2(v0.z, v0.w), make_float2(v1.x, v1.y),
                            make_float2(v1.z, v1.w), hr[a], hi[a]);
    const float4 v2 = c4[(3 + a) * Lh + j], v3 = c4[(P::J2 * 3 + a) * Lh + j];
    cpair_s<P::C2R, P::C2I>(sgp, make_float2(v2.x, v2.y), make_float2(v2.z, v2.w), make_float2(v3.x, v3.y),
                            make_float2(v3.z, v3.w), hr[3 + a], hi[3 + a]);
  }
}

// acc += (1 - sg g_MU) U psi given the projected half spinor h = (hr, hi)
template <int MU>
__device__ __forceinline__ void su3_accumulate(float sg, const float2* hr, const float2* hi, const float2* U,
                                               float2* ar, float2* ai) {
  typedef Proj<MU, 1> P;
  const float2 sgp = f2(sg);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    float2 ur[3], ui[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      ur[b] = f2(U[3 * a + b].x);
      ui[b] = f2(U[3 * a + b].y);
    }
#pragma unroll
    for (int hh = 0; hh < 2; ++hh) {
      float2 A = make_float2(0.f, 0.f), B = A, C = A, D = A;
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        A = fma2(ur[b], hr[3 * hh + b], A);
        B = fma2(ui[b], hi[3 * hh + b], B);
        C = fma2(ur[b], hi[3 * hh + b], C);
        D = fma2(ui[b], hr[3 * hh + b], D);
      }
      const float2 gr = fma2(f2(-1.f), B, A), gi = add2(C, D);
      ar[3 * hh + a] = add2(ar[3 * hh + a], gr);
      ai[3 * hh + a] = add2(ai[3 * hh + a], gi);
      if (hh == P::S2) {
        float2 zr, zi;
        cpair_s<P::D2R, P::D2I>(sgp, ar[6 + a], ai[6 + a], gr, gi, zr, zi);
        ar[6 + a] = zr;
        ai[6 + a] = zi;
      }
      if (hh == P::S3) {
        float2 zr, zi;
        cpair_s<P::D3R, P::D3I>(sgp, ar[9 + a], ai[9 + a], gr, gi, zr, zi);
        ar[9 + a] = zr;
        ai[9 + a] = zi;
      }
    }
  }
}

// rho^(2j) and rho^(2(LH-1-j)) of this lane's pair j (computed once per launch)
template <int LH>
__device__ __forceinline__ float2 lane_powers(const SOpK<float>& op, int j) {
  float a = 1.f, b = 1.f;
  if (op.has_inv) {
    const float r2 = op.rho * op.rho;
#pragma unroll
    for (int q = 0; q < LH; ++q) {
      if (q < j) a *= r2;
      if (q > j) b *= r2;
    }
  }
  return make_float2(a, b);
}

// sop_shfl with Lh fixed at compile time and the lane powers given
template <int LH>
__device__ __forceinline__ void sop_reg(const SOpK<float>& op, float2 pw, float2* re, float2* im, int j) {
  const int lane = threadIdx.x, base = lane - j;
  const float rho = op.rho, m = op.m;
  const float wk = op.has_inv ? -rho * m * (op.c0 / op.ginv) : 0.f;
#pragma unroll
  for (int half = 0; half < 2; ++half) {
    const int up = half ^ op.trans;
    float2 A[6], B[6];
    const float2 gi = f2(op.ginv);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kk = 6 * half + k;
      A[k] = mul2(gi, make_float2(re[kk].x, im[kk].x));
      B[k] = mul2(gi, make_float2(re[kk].y, im[kk].y));
    }
    if (op.has_inv) {
      const float2 r1 = f2(rho);
      if (!up) {
#pragma unroll
        for (int k = 0; k < 6; ++k) B[k] = fma2(r1, A[k], B[k]);
        float rd = rho * rho;
#pragma unroll
        for (int d = 1; d < LH; d <<= 1) {
          const bool ok = j >= d;
          const int src = ok ? lane - d : lane;
          const float2 f = f2(ok ? rd : 0.f);
#pragma unroll
          for (int k = 0; k < 6; ++k) B[k] = fma2(f, shfl2(B[k], src), B[k]);
          rd *= rd;
        }
        const int src = j > 0 ? lane - 1 : lane;
        const float2 f = f2(j > 0 ? rho : 0.f);
        const float2 wa = f2(wk * pw.x), wb = f2(wk * pw.x * rho);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          A[k] = fma2(f, shfl2(B[k], src), A[k]);
          const float2 w = shfl2(B[k], base + LH - 1);
          A[k] = fma2(wa, w, A[k]);
          B[k] = fma2(wb, w, B[k]);
        }
      } else {
#pragma unroll
        for (int k = 0; k < 6; ++k) A[k] = fma2(r1, B[k], A[k]);
        float rd = rho * rho;
#pragma unroll
        for (int d = 1; d < LH; d <<= 1) {
          const bool ok = j + d < LH;
          const int src = ok ? lane + d : lane;
          const float2 f = f2(ok ? rd : 0.f);
#pragma unroll
          for (int k = 0; k < 6; ++k) A[k] = fma2(f, shfl2(A[k], src), A[k]);
          rd *= rd;
        }
        const int src = j < LH - 1 ? lane + 1 : lane;
        const float2 f = f2(j < LH - 1 ? rho : 0.f);
        const float2 wa = f2(wk * pw.y * rho), wb = f2(wk * pw.y);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
          B[k] = fma2(f, shfl2(A[k], src), B[k]);
          const float2 w = shfl2(A[k], base);
          A[k] = fma2(wa, w, A[k]);
          B[k] = fma2(wb, w, B[k]);
        }
      }
    }
    const float2 g1 = f2(op.g1), d1 = f2(op.d1);
    const bool edge = up ? (j == LH - 1) : (j == 0);
    const int src = up ? (edge ? base : lane + 1) : (edge ? base + LH - 1 : lane - 1);
    const float2 fe = f2(edge ? -m : 1.f);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const int kk = 6 * half + k;
      float2 ya, yb;
      if (!up) {
        const float2 q = mul2(fe, shfl2(B[k], src));
        ya = fma2(d1, q, mul2(g1, A[k]));
        yb = fma2(d1, A[k], mul2(g1, B[k]));
      } else {
        const float2 q = mul2(fe, shfl2(A[k], src));
        ya = fma2(d1, B[k], mul2(g1, A[k]));
        yb = fma2(d1, q, mul2(g1, B[k]));
      }
      re[kk] = make_float2(ya.x, yb.x);
      im[kk] = make_float2(ya.y, yb.y);
    }
  }
}

struct HopFArgs {
  const float* in;
  float* out;
  const float* x;
  SOpK<float> ex, eout;
  const float* links_dm;  // [8][Vh][20]
  const int* nbr;         // [8][Vh]
  double* partials;       // one double per CTA (or null)
  long Vh, ngroups;
  float scale, xfold;     // xfold = xscale / scale
  int* err;
  long wait_limit;
};

template <int LH> struct HopFShape {
  static constexpr int G = 32 / LH;
  static constexpr int BLK = 12 * LH * 16;                       // one site's FP32 spinor block
  static constexpr int LK_OFF = G * BLK;                         // the links of the stage's direction
  // 16-byte granularity (what the bulk copies need): rounding the slot up to
  // 128 bytes made 16 warps' shared memory exceed the SM's at Lh = 8
  static constexpr int SLOT = (LK_OFF + G * 80 + 15) / 16 * 16;
  static constexpr int NB_OFF = 2 * SLOT;                        // neighbour indices [2 groups][8][G]
  static constexpr int SMEM = NB_OFF + 2 * 8 * G * 4;
};

template <int LH, int DAG, int HX, int MINB>
__global__ void __launch_bounds__(32, MINB) hopf_kernel(const HopFArgs a) {
  typedef HopFShape<LH> Sh;
  constexpr int G = Sh::G, BLK = Sh::BLK, SLOT = Sh::SLOT;
  constexpr int NST = HX ? 9 : 8;  // stages per group (HX: the site term first)
  extern __shared__ __align__(128) unsigned char sm[];
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ double red[32];
  const int lane = threadIdx.x;
  const int i = lane / LH;
  const int j = lane - i * LH;
  int* nbs = reinterpret_cast<int*>(sm + Sh::NB_OFF);
  const unsigned bar0 = smem_addr(&bars[0]);
  if (lane == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8u, 1);
    fence_async_smem();
  }
  __syncwarp();
  const float2 pw_ex = HX ? lane_powers<LH>(a.ex, j) : make_float2(1.f, 1.f);
  const float2 pw_eo = lane_powers<LH>(a.eout, j);
  const long stride = gridDim.x;
  // neighbour indices of group g into buffer lb (each lane reads back only what it wrote)
  auto load_nb = [&](long g, int lb) {
    if (lane < G) {
      const long hh = g * G + lane;
      const bool ok = g < a.ngroups && hh < a.Vh;
#pragma unroll
      for (int d = 0; d < 8; ++d) nbs[(lb * 8 + d) * G + lane] = ok ? __ldg(a.nbr + (long)d * a.Vh + hh) : 0;
    }
  };
  // stage t of group g into slot `slot`; returns whether anything was issued
  auto issue = [&](long g, int t, int slot, int lb) -> bool {
    if (g >= a.ngroups) return false;
    const long h0 = g * G;
    const long left = a.Vh - h0;
    const int nact = left < G ? (int)left : G;
    const unsigned bar = bar0 + 8u * slot;
    unsigned char* dst = sm + slot * SLOT;
    const int d = HX ? t - 1 : t;
    fence_async_smem();  // earlier generic reads of this slot before the copies
    const unsigned bytes = nact * BLK + (d >= 0 ? nact * 80 : 0);
    if (lane == 0) mbar_expect_tx(bar, bytes);
    __syncwarp();
    if (d >= 0) {
      const int nb_k = lane < G ? nbs[(lb * 8 + d) * G + lane] : 0;
      const int nb0 = __shfl_sync(0xffffffffu, nb_k, 0);
      const unsigned run = __ballot_sync(0xffffffffu, lane >= nact || nb_k == nb0 + lane);
      if (run == 0xffffffffu) {
        if (lane == 0)
          bulk_g2s(smem_addr(dst), reinterpret_cast<const unsigned char*>(a.in) + (long)nb0 * BLK, nact * BLK, bar);
      } else if (lane < nact) {
        bulk_g2s(smem_addr(dst + lane * BLK), reinterpret_cast<const unsigned char*>(a.in) + (long)nb_k * BLK, BLK,
                 bar);
      }
      if (lane == 0) bulk_g2s(smem_addr(dst + Sh::LK_OFF), a.links_dm + ((long)d * a.Vh + h0) * 20, nact * 80, bar);
    } else if (lane == 0) {
      bulk_g2s(smem_addr(dst), reinterpret_cast<const unsigned char*>(a.x) + h0 * BLK, nact * BLK, bar);
    }
    return true;
  };
  long g = blockIdx.x;
  load_nb(g, 0);
  unsigned issued = 0;  // stages issued so far (issue order = consumption order)
  issued += issue(g, 0, 0, 0);
  issued += issue(g, 1, 1, 0);
  unsigned seq = 0;  // the stage being consumed: slot seq & 1, phase (seq >> 1) & 1
  bool bad = false;
  red[lane] = 0.0;  // this lane's partial sum of |out|^2 (kept out of the registers)
  int lb = 0;
  for (; g < a.ngroups; g += stride, lb ^= 1) {
    load_nb(g + stride, lb ^ 1);
    const long h0 = g * G;
    const long left = a.Vh - h0;
    const int nact = left < G ? (int)left : G;
    const bool act = i < nact;
    float2 ar[12], ai[12];  // seeded by the site term (HX) or zeroed at the first direction
#pragma unroll 1
    for (int t = 0; t < NST; ++t) {
      const int slot = seq & 1;
      const unsigned char* sl = sm + slot * SLOT;
      if (__any_sync(0xffffffffu, !mbar_wait(bar0 + 8u * slot, (seq >> 1) & 1, a.wait_limit))) {
        bad = true;
        break;
      }
      const int k2 = t + 2;
      const int d = HX ? t - 1 : t;
      if (d < 0) {
        // the site term seeds the accumulator: xfold * Ex x
        const float4* c4 = reinterpret_cast<const float4*>(sl + i * BLK) + j;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          const float4 v = act ? c4[k * LH] : make_float4(0.f, 0.f, 0.f, 0.f);
          ar[k] = make_float2(v.x, v.y);
          ai[k] = make_float2(v.z, v.w);
        }
        __syncwarp();
        issued += k2 < NST ? issue(g, k2, slot, lb) : issue(g + stride, k2 - NST, slot, lb ^ 1);
        if (a.ex.kind != 0) sop_reg<LH>(a.ex, pw_ex, ar, ai, j);
        const float2 xf = f2(a.xfold);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          ar[k] = mul2(xf, ar[k]);
          ai[k] = mul2(xf, ai[k]);
        }
      } else {
        // (1 -+ g_mu) sign: +1 forward / -1 backward, flipped by the dagger
        const float sg = ((d < 4) != (DAG != 0)) ? 1.f : -1.f;
        float2 hr[6], hi[6], U[9];
        if (act) {
          const float4* c4 = reinterpret_cast<const float4*>(sl + i * BLK);
          switch (d & 3) {
            case 0: project_smem<0>(sg, c4, j, LH, hr, hi); break;
            case 1: project_smem<1>(sg, c4, j, LH, hr, hi); break;
            case 2: project_smem<2>(sg, c4, j, LH, hr, hi); break;
            default: project_smem<3>(sg, c4, j, LH, hr, hi); break;
          }
          const float2* u = reinterpret_cast<const float2*>(sl + Sh::LK_OFF + i * 80);
#pragma unroll
          for (int e = 0; e < 9; ++e) U[e] = u[e];
        }
        __syncwarp();
        issued += k2 < NST ? issue(g, k2, slot, lb) : issue(g + stride, k2 - NST, slot, lb ^ 1);
        if (!HX && t == 0) {
          // zeroed here rather than before the stage loop: the accumulator is
          // not live across the group's first wait and copy issue (fewer spills)
#pragma unroll
          for (int k = 0; k < 12; ++k) {
            ar[k] = make_float2(0.f, 0.f);
            ai[k] = ar[k];
          }
        }
        if (act) {
          switch (d & 3) {
            case 0: su3_accumulate<0>(sg, hr, hi, U, ar, ai); break;
            case 1: su3_accumulate<1>(sg, hr, hi, U, ar, ai); break;
            case 2: su3_accumulate<2>(sg, hr, hi, U, ar, ai); break;
            default: su3_accumulate<3>(sg, hr, hi, U, ar, ai); break;
          }
        }
      }
      ++seq;
    }
    if (bad) break;
    const float2 sc = f2(a.scale);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      ar[k] = mul2(sc, ar[k]);
      ai[k] = mul2(sc, ai[k]);
    }
    if (a.eout.kind != 0) sop_reg<LH>(a.eout, pw_eo, ar, ai, j);
    if (act) {
      store_pair(FieldRef<float>{a.out, nullptr}, h0 + i, j, LH, ar, ai);
      if (a.partials) {
        float2 p0 = make_float2(0.f, 0.f), p1 = p0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          p0 = fma2(ar[k], ar[k], p0);
          p1 = fma2(ai[k], ai[k], p1);
        }
        red[lane] += (double)((p0.x + p0.y) + (p1.x + p1.y));
      }
    }
  }
  if (bad) {
    // stages seq .. issued - 1 are in flight: wait (normal limit) for each
    // before the CTA's shared memory is released
    if (lane == 0) atomicExch(a.err, 1);
    for (unsigned q = seq; q < issued; ++q) mbar_wait(bar0 + 8u * (q & 1), (q >> 1) & 1);
    return;
  }
  if (a.partials) {
    __syncwarp();
    if (lane == 0) {
      double t = 0.0;
      for (int q = 0; q < 32; ++q) t += red[q];  // fixed order
      a.partials[blockIdx.x] = t;
    }
  }
}

}  // namespace

// Sites per group for the pipelined kernel, or 0 if the shape needs the
// per-slice kernel (a batched launch takes the same groups).
int hop2_sites(int Ls, int prec, int nr) {
  const int Lh = (Ls + 1) / 2;
  if (prec != DWF_F32 && prec != DWF_F16) return 0;
  if (nr < 1 || nr > kMaxBatch || Lh > 32) return 0;
  if (prec == DWF_F16 && (Lh % 2)) return 0;  // FP16 scale blocks must be multiples of 16 bytes
  return 32 / Lh;
}

// Resident CTAs per SM for a kernel and dynamic smem size (cached).
static int resident_per_sm(const void* kern, size_t smem, int* per_sm, int* sms_out) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, std::pair<int, int>> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(kern, smem);
  auto it = cache.find(key);
  if (it != cache.end()) {
    *per_sm = it->second.first;
    *sms_out = it->second.second;
    return 0;
  }
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32, smem) != cudaSuccess || per < 1)
    return 1;
  cache[key] = std::make_pair(per, sms);
  *per_sm = per;
  *sms_out = sms;
  return 0;
}

template <class S>
static dwf_status hop3_t(dwf_lattice* L, const HopCall& c, const HopBatch& b, const SOpK<float>* ex,
                         const SOpK<float>* eout, int G, int ctas_per_sm) {
  const bool dense = (c.has_x && ex[0].kind == 2) || eout[0].kind == 2;
  const bool any = (c.has_x && ex[0].kind != 0) || eout[0].kind != 0;
  const bool need_tile = any && ((L->Ls & 1) || dense);
  Hop3Args<S> a{};
  for (int r = 0; r < b.nrhs; ++r) {
    a.in[r] = CFieldRef<S>{reinterpret_cast<const S*>(b.in[r].v), b.in[r].norm};
    a.out[r] = FieldRef<S>{reinterpret_cast<S*>(b.out[r].v), b.out[r].norm};
    a.x[r] = c.has_x ? CFieldRef<S>{reinterpret_cast<const S*>(b.x[r].v), b.x[r].norm} : CFieldRef<S>{nullptr, nullptr};
    a.ex[r] = ex[r];
    a.eout[r] = eout[r];
    a.partials[r] = b.partials[r];
  }
  const bool batched = b.nrhs > 1;
  a.links = reinterpret_cast<const S*>(L->links[b.in[0].prec][c.out_parity]);
  a.nbr = L->nbr[c.out_parity];
  a.Vh = L->Vh;
  a.G = G;
  a.nr = b.nrhs;
  a.ngroups = (L->Vh + G - 1) / G;
  a.Ls = L->Ls;
  a.Lh = L->Lh;
  a.ctx = make_ctx(L->Ls, b.in[0].prec, G, batched, need_tile);
  a.scale = (float)c.scale;
  a.xscale = (float)c.xscale;
  a.err = L->dev_err;
  a.wait_limit = L->wait_limit;
  const size_t smem = (size_t)a.ctx.total;
  auto run = [&](auto kern) -> dwf_status {
    DWF_CUDA(L, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per = 0, sms = 0;
    if (resident_per_sm(reinterpret_cast<const void*>(kern), smem, &per, &sms))
      return fail(L, DWF_ERR_CUDA, "hop: occupancy query failed");
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    const long resident = (long)per * sms;
    const long grid = a.ngroups < resident ? a.ngroups : resident;  // persistent: one wave
    if (b.partials[0] && grid > kPartials) return fail(L, DWF_ERR_INVALID_ARG, "partial-sum buffer too small");
    kern<<<(unsigned)grid, 32, smem, L->stream>>>(a);
    if (c.nblocks) *c.nblocks = (int)grid;
    return DWF_OK;
  };
  if (batched) {
    if (c.dag) return c.has_x ? run(hop3_kernel<S, 1, 1, 1>) : run(hop3_kernel<S, 1, 0, 1>);
    return c.has_x ? run(hop3_kernel<S, 0, 1, 1>) : run(hop3_kernel<S, 0, 0, 1>);
  }
  if (c.dag) return c.has_x ? run(hop3_kernel<S, 1, 1, 0>) : run(hop3_kernel<S, 1, 0, 0>);
  return c.has_x ? run(hop3_kernel<S, 0, 1, 0>) : run(hop3_kernel<S, 0, 0, 0>);
}

// The FP32 fast path takes one right-hand side, even Ls with Lh in {4, 6, 8, 16,
// 32} and structured fifth-dimension operators.
static bool hopf_takes(const dwf_lattice* L, const HopCall& c, const HopBatch& b, const SOpK<float>& ex,
                       const SOpK<float>& eout) {
  if (b.nrhs != 1 || b.in[0].prec != DWF_F32 || (L->Ls & 1) || !L->links_dm[c.out_parity]) return false;
  if (L->Lh != 4 && L->Lh != 6 && L->Lh != 8 && L->Lh != 16 && L->Lh != 32) return false;
  if (c.has_x && (ex.kind == 2 || c.scale == 0.0)) return false;
  return eout.kind != 2;
}

template <int LH, int MINB0, int MINB1>
static dwf_status hopf_t(dwf_lattice* L, const HopCall& c, const HopBatch& b, const SOpK<float>& ex,
                         const SOpK<float>& eout, int ctas_per_sm) {
  typedef HopFShape<LH> Sh;
  HopFArgs a{};
  a.in = reinterpret_cast<const float*>(b.in[0].v);
  a.out = reinterpret_cast<float*>(b.out[0].v);
  a.x = c.has_x ? reinterpret_cast<const float*>(b.x[0].v) : nullptr;
  if (c.has_x) a.ex = ex;
  a.eout = eout;
  a.links_dm = L->links_dm[c.out_parity];
  a.nbr = L->nbr[c.out_parity];
  a.partials = b.partials[0];
  a.Vh = L->Vh;
  a.ngroups = (L->Vh + Sh::G - 1) / Sh::G;
  a.scale = (float)c.scale;
  a.xfold = c.has_x ? (float)(c.xscale / c.scale) : 0.f;
  a.err = L->dev_err;
  a.wait_limit = L->wait_limit;
  auto run = [&](auto kern) -> dwf_status {
    DWF_CUDA(L, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, Sh::SMEM));
    int per = 0, sms = 0;
    if (resident_per_sm(reinterpret_cast<const void*>(kern), Sh::SMEM, &per, &sms))
      return fail(L, DWF_ERR_CUDA, "hop: occupancy query failed");
    if (ctas_per_sm > 0 && ctas_per_sm < per) per = ctas_per_sm;
    const long resident = (long)per * sms;
    const long grid = a.ngroups < resident ? a.ngroups : resident;  // persistent: one wave
    if (b.partials[0] && grid > kPartials) return fail(L, DWF_ERR_INVALID_ARG, "partial-sum buffer too small");
    kern<<<(unsigned)grid, 32, Sh::SMEM, L->stream>>>(a);
    if (c.nblocks) *c.nblocks = (int)grid;
    return DWF_OK;
  };
  if (c.dag) return c.has_x ? run(hopf_kernel<LH, 1, 1, MINB1>) : run(hopf_kernel<LH, 1, 0, MINB0>);
  return c.has_x ? run(hopf_kernel<LH, 0, 1, MINB1>) : run(hopf_kernel<LH, 0, 0, MINB0>);
}

dwf_status launch_hop2(dwf_lattice* L, const HopCall& c, const HopBatch& b, const SOpK<float>* ex,
                       const SOpK<float>* eout, int G, int ctas_per_sm) {
  if (hopf_takes(L, c, b, ex[0], eout[0])) {
    // resident warps per SM (without / with a site term) as measured best on
    // GB300: 16 (128 registers) or 12 (168 registers); at Lh = 16 the hop
    // with a site term ran 11 % slower when held to 128 registers
    switch (L->Lh) {
      case 4: return hopf_t<4, 12, 12>(L, c, b, ex[0], eout[0], ctas_per_sm);
      case 6: return hopf_t<6, 16, 16>(L, c, b, ex[0], eout[0], ctas_per_sm);
      case 8: return hopf_t<8, 16, 16>(L, c, b, ex[0], eout[0], ctas_per_sm);
      case 16: return hopf_t<16, 16, 12>(L, c, b, ex[0], eout[0], ctas_per_sm);
      default: return hopf_t<32, 12, 12>(L, c, b, ex[0], eout[0], ctas_per_sm);
    }
  }
  if (b.in[0].prec == DWF_F32) return hop3_t<float>(L, c, b, ex, eout, G, ctas_per_sm);
  return hop3_t<__half>(L, c, b, ex, eout, G, ctas_per_sm);
}

}  // namespace dwf
