// Device code shared by the hop kernels (hop.cu, hop2.cu): spin projection
// tables of the Wilson hop and the fifth-dimension (s-local) operators.
#pragma once

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

// In-place structured operator on one tile row (complex component k of a
// site, all Ls slices).
template <class C>
__device__ __forceinline__ void sop_row(const SOpK<C>& op, C* row, int k, int Ls) {
  const int up = ((k >= 6) ? 1 : 0) ^ op.trans;  // P+ (k < 6) walks down in s unless transposed
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

// In-place structured operator on the rows of the first `nsites` sites.
template <class C>
__device__ void sop_rows(const SOpK<C>& op, C* tile, int nsites, int Ls, int R) {
  for (int w = threadIdx.x; w < nsites * 12; w += blockDim.x) sop_row(op, tile + w * R, w % 12, Ls);
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

}  // namespace dwf
