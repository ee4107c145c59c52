// Pseudofermion action, fermion force and the force-gradient link update
// (Sec. 2 and 3).
//
// Quotient action for det(M1^+ M1) / det(M2^+ M2) (Sec. 3, Hasenbusch factor):
//   S = phi^+ M2 (M1^+ M1)^-1 M2^+ phi = |Y|^2,  X = (M1^+ M1)^-1 M2^+ phi,  Y = M1 X,
// with M = M_pc the even-odd Schur operator.  Its Lie derivative
// F^j(n, mu) = e_j S along U_mu(n) -> e^{h T_j} U_mu(n), T_j = i lambda_j / 2, is
//   dS = 2 Re[phi^+ dM2 X] - 2 Re[Y^+ dM1 X],
//   Re[L^+ dM R] = 1/2 Re[L_full^+ dDhop R_full],  L_full = (L, A^-+ M_eo^+ L),
//                                                  R_full = (B A^-1 M_oe R, B R)  (odd, even parts)
// so each term reduces to one "link outer product" of two whole-lattice
// fields.  Per link, with P = 1 - g_mu, P' = 1 + g_mu and the two-spin
// projections of the hop (proj = upper half of P psi):
//   M  = sum_s sum_i proj_P (R(n+mu))_i (x) proj_P (L(n))_i^+
//   M' = sum_s sum_i proj_P'(R(n))_i    (x) proj_P'(L(n+mu))_i^+
//   G  = U M - M' U^+,  F^j = Re tr(T_j G),
// and the complex-matrix gradient (torch convention, 2 dS/d conj U) is M^+ + M'.
#include <chrono>
#include <cmath>

#include "dwf_internal.h"
#include "hop_common.cuh"

namespace dwf {

dwf_status apply_Mpc_internal(dwf_lattice* L, const SOps* ops, bool dag, Field xe, Field oe);
dwf_status cgne_core(dwf_lattice* L, const SOps* ops, Field v, Field x64, const dwf_cg_params& prm, dwf_stats* st,
                     long long* hops);

namespace {

// two-spin projection h = upper half of (1 - SG g_MU) psi (psi: 24 reals)
template <int MU, int SG>
__device__ __forceinline__ void proj2(const double* psi, double* h) {
  typedef Proj<MU, SG> P;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    h[2 * a] = psi[2 * a];
    h[2 * a + 1] = psi[2 * a + 1];
    cmadd<P::C1R, P::C1I>(h[2 * a], h[2 * a + 1], psi[2 * (P::J1 * 3 + a)], psi[2 * (P::J1 * 3 + a) + 1]);
    h[6 + 2 * a] = psi[2 * (3 + a)];
    h[6 + 2 * a + 1] = psi[2 * (3 + a) + 1];
    cmadd<P::C2R, P::C2I>(h[6 + 2 * a], h[6 + 2 * a + 1], psi[2 * (P::J2 * 3 + a)], psi[2 * (P::J2 * 3 + a) + 1]);
  }
}

// out[a][b] (complex, 18 reals) = sum_{i=0,1} k_i[a] conj(h_i[b])
__device__ __forceinline__ void outer2(const double* k, const double* h, double* out) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      double re = 0, im = 0;
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const double kr = k[6 * i + 2 * a], ki = k[6 * i + 2 * a + 1];
        const double hr = h[6 * i + 2 * b], hi = h[6 * i + 2 * b + 1];
        re = fma(kr, hr, fma(ki, hi, re));
        im = fma(ki, hr, fma(-kr, hi, im));
      }
      out[2 * (3 * a + b)] = re;
      out[2 * (3 * a + b) + 1] = im;
    }
}

// proj_{SG}(spinor (h, s) of field f) -> k (12 reals); the full spinor lives only here
template <int MU, int SG>
__device__ __forceinline__ void load_proj(CFieldRef<double> f, long h, int s, int Lh, double* k) {
  double psi[24];
  load_spinor<double>(f, h, s, Lh, psi);
  proj2<MU, SG>(psi, k);
}

// dst[0..17] = M = P R(n+mu) (x) P L(n);  dst[18..35] = M' = P' R(n) (x) P' L(n+mu)
template <int MU>
__device__ __forceinline__ void link_terms(CFieldRef<double> Rn, CFieldRef<double> Ln, CFieldRef<double> Rf,
                                           CFieldRef<double> Lf, long h, long hn, int s, int Lh, double* dst) {
  double k[12], q[12], M[18];
  load_proj<MU, 1>(Rf, hn, s, Lh, k);
  load_proj<MU, 1>(Ln, h, s, Lh, q);
  outer2(k, q, M);
#pragma unroll
  for (int e = 0; e < 18; ++e) dst[e] = M[e];
  load_proj<MU, -1>(Rn, h, s, Lh, k);
  load_proj<MU, -1>(Lf, hn, s, Lh, q);
  outer2(k, q, M);
#pragma unroll
  for (int e = 0; e < 18; ++e) dst[18 + e] = M[e];
}

struct ForceArgs {
  CFieldRef<double> L[2], R[2];  // by parity
  const double* links[2];        // FP64 [Vh][8][18] per parity (t phase folded in)
  const int* nbr[2];
  long Vh;
  int Ls, Lh, NS;
  int X, Y, Z, T, bc_t;
  double sign;
  double* F;  // [4][V4][8] (accumulated) or null
  double* G;  // [4][V4][3][3] complex (accumulated) or null
};

// thread (i, s): site i of the CTA's NS sites of parity p (blockIdx.y), slice s
__global__ void __launch_bounds__(256) force_kernel(const ForceArgs a) {
  extern __shared__ __align__(16) double fsm[];  // [NS][Ls][36] then [NS][36]
  const int p = blockIdx.y;
  const int Ls = a.Ls, NS = a.NS;
  const int i = threadIdx.x / Ls;
  const int s = threadIdx.x - i * Ls;
  const long h = (long)blockIdx.x * NS + i;
  const bool act = (i < NS) && (h < a.Vh);
  double* part = fsm;
  double* sum = fsm + (size_t)NS * Ls * 36;
  // site coordinates (for the output index and the t boundary phase)
  long n = 0;
  int tt = 0;
  if (act) {
    const int Xh = a.X / 2;
    long rest = h / Xh;
    const int xh = (int)(h - rest * Xh);
    const int y = (int)(rest % a.Y);
    rest /= a.Y;
    const int z = (int)(rest % a.Z);
    tt = (int)(rest / a.Z);
    const int x = 2 * xh + ((p + y + z + tt) & 1);
    n = (((long)tt * a.Z + z) * a.Y + y) * a.X + x;
  }
  const long V4 = 2 * a.Vh;
#pragma unroll 1
  for (int mu = 0; mu < 4; ++mu) {
    if (act) {
      const long hn = __ldg(a.nbr[p] + (long)mu * a.Vh + h);
      double* dst = part + ((size_t)i * Ls + s) * 36;
      const CFieldRef<double> Rn = a.R[p], Ln = a.L[p], Rf = a.R[1 - p], Lf = a.L[1 - p];
      switch (mu) {
        case 0: link_terms<0>(Rn, Ln, Rf, Lf, h, hn, s, a.Lh, dst); break;
        case 1: link_terms<1>(Rn, Ln, Rf, Lf, h, hn, s, a.Lh, dst); break;
        case 2: link_terms<2>(Rn, Ln, Rf, Lf, h, hn, s, a.Lh, dst); break;
        default: link_terms<3>(Rn, Ln, Rf, Lf, h, hn, s, a.Lh, dst); break;
      }
    }
    __syncthreads();
    // sum over s
    for (int w = threadIdx.x; w < NS * 36; w += blockDim.x) {
      const int site = w / 36, e = w - site * 36;
      double acc = 0.0;
      for (int t = 0; t < Ls; ++t) acc += part[((size_t)site * Ls + t) * 36 + e];
      sum[w] = acc;
    }
    __syncthreads();
    if (act && s == 0) {
      const double* Ms = sum + i * 36;
      const double* Mps = Ms + 18;
      const double* U = a.links[p] + (h * 8 + mu) * 18;
      const double ph = (mu == 3 && a.bc_t < 0 && tt == a.T - 1) ? -1.0 : 1.0;  // folded into U
      if (a.F) {
        // G = U M - M' U^+
        double Gm[18];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            double re = 0, im = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
              const double ur = U[2 * (3 * r + k)], ui = U[2 * (3 * r + k) + 1];
              const double mr = Ms[2 * (3 * k + c)], mi = Ms[2 * (3 * k + c) + 1];
              re += ur * mr - ui * mi;
              im += ur * mi + ui * mr;
              // (M' U^+)_rc = sum_k M'_rk conj(U_ck)
              const double pr = Mps[2 * (3 * r + k)], pi = Mps[2 * (3 * r + k) + 1];
              const double vr = U[2 * (3 * c + k)], vi = U[2 * (3 * c + k) + 1];
              re -= pr * vr + pi * vi;
              im -= pi * vr - pr * vi;
            }
            Gm[2 * (3 * r + c)] = re;
            Gm[2 * (3 * r + c) + 1] = im;
          }
        // F^j = Re tr(T_j G) = -1/2 Im tr(lambda_j G)
#define GR(r, c) Gm[2 * (3 * (r) + (c))]
#define GI(r, c) Gm[2 * (3 * (r) + (c)) + 1]
        double f[8];
        f[0] = -0.5 * (GI(1, 0) + GI(0, 1));
        f[1] = 0.5 * (GR(1, 0) - GR(0, 1));
        f[2] = -0.5 * (GI(0, 0) - GI(1, 1));
        f[3] = -0.5 * (GI(2, 0) + GI(0, 2));
        f[4] = 0.5 * (GR(2, 0) - GR(0, 2));
        f[5] = -0.5 * (GI(2, 1) + GI(1, 2));
        f[6] = 0.5 * (GR(2, 1) - GR(1, 2));
        f[7] = -0.5 * (GI(0, 0) + GI(1, 1) - 2.0 * GI(2, 2)) * 0.57735026918962576451;
#undef GR
#undef GI
        double* out = a.F + ((long)mu * V4 + n) * 8;
#pragma unroll
        for (int j = 0; j < 8; ++j) out[j] += a.sign * f[j];
      }
      if (a.G) {
        // 2 dS / d conj(U_true) = phase (M^+ + M')
        double* out = a.G + ((long)mu * V4 + n) * 18;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            out[2 * (3 * r + c)] += a.sign * ph * (Ms[2 * (3 * c + r)] + Mps[2 * (3 * r + c)]);
            out[2 * (3 * r + c) + 1] += a.sign * ph * (-Ms[2 * (3 * c + r) + 1] + Mps[2 * (3 * r + c) + 1]);
          }
      }
    }
    __syncthreads();
  }
}

// ---- SU(3) exponential of an anti-hermitian matrix: scaled Taylor series
// (Moler & Van Loan, "Nineteen dubious ways", method 3): exp(X) = (T_q(X/2^k))^(2^k)
__device__ void cmul3(const double* A, const double* B, double* C) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double re = 0, im = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const double ar = A[2 * (3 * r + k)], ai = A[2 * (3 * r + k) + 1];
        const double br = B[2 * (3 * k + c)], bi = B[2 * (3 * k + c) + 1];
        re += ar * br - ai * bi;
        im += ar * bi + ai * br;
      }
      C[2 * (3 * r + c)] = re;
      C[2 * (3 * r + c) + 1] = im;
    }
}

__device__ void su3_exp(const double* X, double* E) {
  double nrm = 0;
#pragma unroll
  for (int e = 0; e < 18; ++e) nrm = fmax(nrm, fabs(X[e]));
  nrm *= 3.0;  // bound on the infinity norm
  int k = 0;
  while (nrm > 0.125 && k < 60) {
    nrm *= 0.5;
    ++k;
  }
  const double sc = ldexp(1.0, -k);
  double Y[18], term[18], tmp[18];
#pragma unroll
  for (int e = 0; e < 18; ++e) {
    Y[e] = X[e] * sc;
    E[e] = 0.0;
    term[e] = 0.0;
  }
  E[0] = E[8] = E[16] = 1.0;
  term[0] = term[8] = term[16] = 1.0;
  for (int q = 1; q <= 12; ++q) {
    cmul3(term, Y, tmp);
    const double inv = 1.0 / q;
#pragma unroll
    for (int e = 0; e < 18; ++e) {
      term[e] = tmp[e] * inv;
      E[e] += term[e];
    }
  }
  for (int q = 0; q < k; ++q) {
    cmul3(E, E, tmp);
#pragma unroll
    for (int e = 0; e < 18; ++e) E[e] = tmp[e];
  }
}

// X = coeff * sum_j comp^j T_j, T_j = i lambda_j / 2 (anti-hermitian, traceless)
__device__ void algebra_matrix(const double* f, double coeff, double* X) {
  const double c = 0.5 * coeff;
  const double s3 = 0.57735026918962576451;
  // i lambda_j entries (re, im):  entries of i*lambda
  // diagonal: i (f3 + f8/sqrt3), i (-f3 + f8/sqrt3), i (-2 f8 / sqrt3)
  X[0] = 0;
  X[1] = c * (f[2] + s3 * f[7]);
  X[8] = 0;
  X[9] = c * (-f[2] + s3 * f[7]);
  X[16] = 0;
  X[17] = c * (-2.0 * s3 * f[7]);
  // (0,1): i (f1 - i f2) = f2 + i f1 ; (1,0): i (f1 + i f2) = -f2 + i f1
  X[2] = c * f[1];
  X[3] = c * f[0];
  X[6] = -c * f[1];
  X[7] = c * f[0];
  // (0,2): i (f4 - i f5) = f5 + i f4 ; (2,0): -f5 + i f4
  X[4] = c * f[4];
  X[5] = c * f[3];
  X[12] = -c * f[4];
  X[13] = c * f[3];
  // (1,2): f7 + i f6 ; (2,1): -f7 + i f6
  X[10] = c * f[6];
  X[11] = c * f[5];
  X[14] = -c * f[6];
  X[15] = c * f[5];
}

__global__ void link_update_kernel(const double* __restrict__ f, double coeff, const double* __restrict__ Uin,
                                   double* __restrict__ Uout, long nlinks) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nlinks) return;
  double X[18], E[18], U[18], R[18];
  algebra_matrix(f + q * 8, coeff, X);
  su3_exp(X, E);
#pragma unroll
  for (int e = 0; e < 18; ++e) U[e] = Uin[q * 18 + e];
  cmul3(E, U, R);
#pragma unroll
  for (int e = 0; e < 18; ++e) Uout[q * 18 + e] = R[e];
}

__global__ void axpy_real_kernel(double a, const double* __restrict__ x, double* __restrict__ y, long n) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) y[q] = fma(a, x[q], y[q]);
}

__global__ void sumsq_kernel(const double* __restrict__ x, long n, double* partials) {
  __shared__ double red[32];
  double acc = 0.0;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
    acc = fma(x[q], x[q], acc);
  double t = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

CFieldRef<double> c64(const Field& f) { return CFieldRef<double>{reinterpret_cast<const double*>(f.v), nullptr}; }

dwf_status launch_force(dwf_lattice* L, Field Le, Field Lo, Field Re, Field Ro, double sign, double* F, double* G) {
  ForceArgs a;
  a.L[0] = c64(Le);
  a.L[1] = c64(Lo);
  a.R[0] = c64(Re);
  a.R[1] = c64(Ro);
  a.links[0] = reinterpret_cast<const double*>(L->links[0][0]);
  a.links[1] = reinterpret_cast<const double*>(L->links[0][1]);
  a.nbr[0] = L->nbr[0];
  a.nbr[1] = L->nbr[1];
  a.Vh = L->Vh;
  a.Ls = L->Ls;
  a.Lh = L->Lh;
  int ns = 128 / L->Ls;
  a.NS = ns < 1 ? 1 : ns;
  a.X = L->X;
  a.Y = L->Y;
  a.Z = L->Z;
  a.T = L->T;
  a.bc_t = L->p.bc_t;
  a.sign = sign;
  a.F = F;
  a.G = G;
  const int threads = (a.NS * L->Ls + 31) / 32 * 32;
  const size_t smem = ((size_t)a.NS * L->Ls * 36 + (size_t)a.NS * 36) * sizeof(double);
  if (smem > 48 * 1024)
    DWF_CUDA(L, cudaFuncSetAttribute(force_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  dim3 grid((unsigned)((L->Vh + a.NS - 1) / a.NS), 2);
  force_kernel<<<grid, threads, smem, L->stream>>>(a);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

void add_stats(dwf_stats* a, const dwf_stats& b) {
  a->iters += b.iters;
  a->reliable_updates += b.reliable_updates;
  a->hop_calls += b.hop_calls;
  a->op_count += b.op_count;
  if (b.true_resid > a->true_resid) a->true_resid = b.true_resid;
}

}  // namespace

}  // namespace dwf

using namespace dwf;

extern "C" {

dwf_status dwf_force(dwf_lattice_t L, int nterms, const dwf_quotient* terms, const void* const* phi,
                     void* const* X_io, void* F, void* G, double* S, const dwf_cg_params* prm, dwf_stats* stats) {
  if (!L || nterms < 1 || !terms || !phi || !prm) return fail(L, DWF_ERR_INVALID_ARG, "dwf_force: bad argument");
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "dwf_force: gauge field not set");
  for (int t = 0; t < nterms; ++t)
    if (!phi[t] || !std::isfinite(terms[t].m1) || !std::isfinite(terms[t].m2))
      return fail(L, DWF_ERR_INVALID_ARG, "dwf_force: bad quotient term");
  auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  dwf_stats st{};
  long long hops = 0;
  const long V4 = L->V4;
  Field pe, v, xt, X, Y, Le, Lo, Re, Ro, tmp;
  DWF_TRY(field_alloc(L, "f.phi", DWF_F64, &pe));
  DWF_TRY(field_alloc(L, "f.v", DWF_F64, &v));
  DWF_TRY(field_alloc(L, "f.xt", DWF_F64, &xt));
  DWF_TRY(field_alloc(L, "f.X", DWF_F64, &X));
  DWF_TRY(field_alloc(L, "f.Y", DWF_F64, &Y));
  DWF_TRY(field_alloc(L, "f.Lo", DWF_F64, &Lo));
  DWF_TRY(field_alloc(L, "f.Re", DWF_F64, &Re));
  DWF_TRY(field_alloc(L, "f.Ro", DWF_F64, &Ro));
  DWF_TRY(field_alloc(L, "f.tmp", DWF_F64, &tmp));
  double *Facc = nullptr, *Gacc = nullptr;
  if (F) {
    void* p;
    DWF_TRY(ws_get(L, "f.F", (size_t)4 * V4 * 8 * sizeof(double), &p));
    Facc = reinterpret_cast<double*>(p);
    DWF_CUDA(L, cudaMemsetAsync(Facc, 0, (size_t)4 * V4 * 8 * sizeof(double), L->stream));
  }
  if (G) {
    void* p;
    DWF_TRY(ws_get(L, "f.G", (size_t)4 * V4 * 18 * sizeof(double), &p));
    Gacc = reinterpret_cast<double*>(p);
    DWF_CUDA(L, cudaMemsetAsync(Gacc, 0, (size_t)4 * V4 * 18 * sizeof(double), L->stream));
  }
  double Stot = 0.0;
  for (int t = 0; t < nterms; ++t) {
    dwf_status s0;
    const SOps* o1 = sops_for(L, terms[t].m1, &s0);
    if (!o1) return s0;
    const SOps* o2 = sops_for(L, terms[t].m2, &s0);
    if (!o2) return s0;
    DWF_TRY(launch_pack(L, phi[t], 0, pe));
    // v = M2^+ phi;  solve (M~^+ M~) x~ = B^-+ v with M_pc = M~ B, then X = B^-1 x~
    DWF_TRY(apply_Mpc_internal(L, o2, true, pe, tmp));
    hops += 2;
    DWF_TRY(launch_sop(L, tmp, v, o1, SOps::BINVT, 1.0, nullptr, 0.0));
    if (X_io && X_io[t]) {
      DWF_TRY(launch_pack(L, X_io[t], 0, X));
      DWF_TRY(launch_sop(L, X, xt, o1, SOps::B, 1.0, nullptr, 0.0));
    } else {
      DWF_TRY(blas_zero(L, xt));
    }
    dwf_stats cs{};
    dwf_status s = cgne_core(L, o1, v, xt, *prm, &cs, &hops);
    if (s != DWF_OK) return s;
    add_stats(&st, cs);
    DWF_TRY(launch_sop(L, xt, X, o1, SOps::BINV, 1.0, nullptr, 0.0));
    // Y = M1 X and S_t = |Y|^2
    DWF_TRY(apply_Mpc_internal(L, o1, false, X, Y));
    hops += 2;
    int nb;
    DWF_TRY(blas_norm2(L, Y, L->partials, &nb));
    DWF_TRY(blas_sum(L, L->partials, nb, L->scal + 50));
    DWF_CUDA(L, cudaMemcpyAsync(L->hscal + 50, L->scal + 50, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    DWF_CUDA(L, cudaStreamSynchronize(L->stream));
    Stot += L->hscal[50];
    if (X_io && X_io[t]) DWF_TRY(launch_unpack(L, X, 0, X_io[t], true));
    if (!F && !G) continue;
    // the two outer-product terms: (phi, X; m2, +1) and (Y, X; m1, -1)
    for (int k = 0; k < 2; ++k) {
      const SOps* o = k == 0 ? o2 : o1;
      Le = k == 0 ? pe : Y;
      // R_e = B X,  R_o = B A^-1 M_oe X = E1 (-1/2 Dhop_oe R_e)
      DWF_TRY(launch_sop(L, X, Re, o, SOps::B, 1.0, nullptr, 0.0));
      HopCall cr;
      cr.out_parity = 1;
      cr.in = Re;
      cr.out = Ro;
      cr.eout = SOps::E1;
      cr.ops = o;
      cr.scale = -0.5;
      DWF_TRY(launch_hop(L, cr));
      // L_o = A^-+ M_eo^+ L_e = E1^T (-1/2 Dhop^+ L_e)
      HopCall cl;
      cl.out_parity = 1;
      cl.dag = 1;
      cl.in = Le;
      cl.out = Lo;
      cl.eout = SOps::E1T;
      cl.ops = o;
      cl.scale = -0.5;
      DWF_TRY(launch_hop(L, cl));
      hops += 2;
      DWF_TRY(launch_force(L, Le, Lo, Re, Ro, k == 0 ? 1.0 : -1.0, Facc, Gacc));
    }
  }
  if (F) DWF_CUDA(L, cudaMemcpyAsync(F, Facc, (size_t)4 * V4 * 8 * sizeof(double), cudaMemcpyDeviceToDevice, L->stream));
  if (G)
    DWF_CUDA(L, cudaMemcpyAsync(G, Gacc, (size_t)4 * V4 * 18 * sizeof(double), cudaMemcpyDeviceToDevice, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  if (S) *S = Stot;
  st.hop_calls = hops;
  st.op_count = (long long)st.iters * L->Ls;
  st.launches = L->launches - l0;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return DWF_OK;
}

dwf_status dwf_heatbath(dwf_lattice_t L, dwf_quotient term, const void* eta, void* phi, const dwf_cg_params* prm,
                        dwf_stats* stats) {
  if (!L || !eta || !phi || !prm) return fail(L, DWF_ERR_INVALID_ARG, "dwf_heatbath: null argument");
  if (eta == phi) return fail(L, DWF_ERR_INVALID_ARG, "dwf_heatbath: eta and phi must not alias");
  if (!std::isfinite(term.m1) || !std::isfinite(term.m2))
    return fail(L, DWF_ERR_INVALID_ARG, "dwf_heatbath: non-finite mass");
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "dwf_heatbath: gauge field not set");
  auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  dwf_status s0;
  const SOps* o1 = sops_for(L, term.m1, &s0);
  if (!o1) return s0;
  const SOps* o2 = sops_for(L, term.m2, &s0);
  if (!o2) return s0;
  Field ee, w, v, xt, X, Y;
  DWF_TRY(field_alloc(L, "hb.eta", DWF_F64, &ee));
  DWF_TRY(field_alloc(L, "hb.w", DWF_F64, &w));
  DWF_TRY(field_alloc(L, "hb.v", DWF_F64, &v));
  DWF_TRY(field_alloc(L, "hb.xt", DWF_F64, &xt));
  DWF_TRY(field_alloc(L, "hb.X", DWF_F64, &X));
  DWF_TRY(field_alloc(L, "hb.Y", DWF_F64, &Y));
  long long hops = 0;
  // phi = M2^-+ M1^+ eta = M2 (M2^+ M2)^-1 M1^+ eta: then M1^-+ M2^+ phi = eta
  // and the quotient's action is |eta|^2
  DWF_TRY(launch_pack(L, eta, 0, ee));
  DWF_TRY(apply_Mpc_internal(L, o1, true, ee, w));
  hops += 2;
  // (M2^+ M2) X = w with M2 = M~ B: (M~^+ M~) x~ = B^-+ w, X = B^-1 x~
  DWF_TRY(launch_sop(L, w, v, o2, SOps::BINVT, 1.0, nullptr, 0.0));
  DWF_TRY(blas_zero(L, xt));
  dwf_stats st{};
  DWF_TRY(cgne_core(L, o2, v, xt, *prm, &st, &hops));
  DWF_TRY(launch_sop(L, xt, X, o2, SOps::BINV, 1.0, nullptr, 0.0));
  DWF_TRY(apply_Mpc_internal(L, o2, false, X, Y));
  hops += 2;
  DWF_TRY(launch_unpack(L, Y, 0, phi, true));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  DWF_TRY(check_dev_err(L));
  st.hop_calls = hops;
  st.op_count = (long long)st.iters * L->Ls;
  st.launches = L->launches - l0;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = st;
  return DWF_OK;
}

dwf_status fgi_link_update(dwf_lattice_t L, const void* Xc, double coeff, const void* U_in, void* U_out) {
  if (!L || !Xc || !U_in || !U_out || !std::isfinite(coeff))
    return fail(L, DWF_ERR_INVALID_ARG, "fgi_link_update: bad argument");
  const long n = 4 * L->V4;
  link_update_kernel<<<(unsigned)((n + 127) / 128), 128, 0, L->stream>>>(
      reinterpret_cast<const double*>(Xc), coeff, reinterpret_cast<const double*>(U_in),
      reinterpret_cast<double*>(U_out), n);
  DWF_LAUNCHED(L);
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}

dwf_status dwf_momentum_update(dwf_lattice_t L, const void* F, double coeff, void* p) {
  if (!L || !F || !p || !std::isfinite(coeff)) return fail(L, DWF_ERR_INVALID_ARG, "dwf_momentum_update: bad argument");
  const long n = 4 * L->V4 * 8;
  axpy_real_kernel<<<(unsigned)((n + 255) / 256), 256, 0, L->stream>>>(
      coeff, reinterpret_cast<const double*>(F), reinterpret_cast<double*>(p), n);
  DWF_LAUNCHED(L);
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}

dwf_status fgi_step(dwf_lattice_t L, int nterms, const dwf_quotient* terms, const void* const* phi, void* U, void* p,
                    double tau, int forecast, const dwf_cg_params* cg, dwf_stats* stats, int* fg_iters) {
  if (!L || nterms < 1 || nterms > 64 || !terms || !phi || !U || !p || !cg || !std::isfinite(tau))
    return fail(L, DWF_ERR_INVALID_ARG, "fgi_step: bad argument");
  auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  const long V4 = L->V4;
  const size_t fbytes = (size_t)4 * V4 * 8 * sizeof(double);
  const size_t ubytes = (size_t)4 * V4 * 18 * sizeof(double);
  const size_t sbytes = (size_t)2 * L->Vh * L->Ls * 24 * sizeof(double);
  void *F, *Up, *xbuf;
  DWF_TRY(ws_get(L, "fgi.F", fbytes, &F));
  DWF_TRY(ws_get(L, "fgi.Up", ubytes, &Up));
  DWF_TRY(ws_get(L, "fgi.X", sbytes * nterms, &xbuf));
  std::vector<void*> X(nterms);
  for (int t = 0; t < nterms; ++t) X[t] = reinterpret_cast<char*>(xbuf) + t * sbytes;
  dwf_stats tot{};
  auto force = [&](const void* Ucur, bool keep, bool guess, int* iters) -> dwf_status {
    DWF_TRY(dwf_set_gauge(L, Ucur));
    if (!guess) DWF_CUDA(L, cudaMemsetAsync(xbuf, 0, sbytes * nterms, L->stream));
    dwf_stats s{};
    DWF_TRY(dwf_force(L, nterms, terms, phi, (keep || guess) ? X.data() : nullptr, F, nullptr, nullptr, cg, &s));
    add_stats(&tot, s);
    if (iters) *iters = s.iters;
    return DWF_OK;
  };
  int it_fg[2] = {0, 0};
  // P(tau/6)
  DWF_TRY(force(U, false, false, nullptr));
  DWF_TRY(dwf_momentum_update(L, F, -tau / 6.0, p));
  // Q(tau/2)
  DWF_TRY(fgi_link_update(L, p, tau / 2.0, U, U));
  // force-gradient step: F(U); U' = exp(-tau^2/24 F) U; p -= 2/3 tau F(U')
  DWF_TRY(force(U, true, false, &it_fg[0]));
  DWF_TRY(fgi_link_update(L, F, -tau * tau / 24.0, U, Up));
  DWF_TRY(force(Up, true, forecast != 0, &it_fg[1]));
  DWF_TRY(dwf_momentum_update(L, F, -2.0 * tau / 3.0, p));
  // Q(tau/2)
  DWF_TRY(fgi_link_update(L, p, tau / 2.0, U, U));
  // P(tau/6)
  DWF_TRY(force(U, false, false, nullptr));
  DWF_TRY(dwf_momentum_update(L, F, -tau / 6.0, p));
  tot.launches = L->launches - l0;
  tot.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = tot;
  if (fg_iters) {
    fg_iters[0] = it_fg[0];
    fg_iters[1] = it_fg[1];
  }
  return DWF_OK;
}

// Omelyan, Mryglod and Folk, Comput. Phys. Commun. 151 (2003) 272: the
// second-order minimum-norm ("2MN") parameter of the integrator that Sec. 2
// compares the force-gradient integrator with.
static constexpr double kOmelyanLambda = 0.1931833275037836;

dwf_status dwf_md_trajectory(dwf_lattice_t L, int nterms, const dwf_quotient* terms, const void* const* phi, void* U,
                             void* p, double tau, int nsteps, dwf_integrator integ, int forecast,
                             const dwf_cg_params* cg, double* H0, double* H1, dwf_stats* stats, int* nforce) {
  if (!L || nterms < 1 || nterms > 64 || !terms || !phi || !U || !p || !cg || !std::isfinite(tau) || nsteps < 1 ||
      (integ != DWF_INTEGRATOR_FGI && integ != DWF_INTEGRATOR_OMELYAN))
    return fail(L, DWF_ERR_INVALID_ARG, "dwf_md_trajectory: bad argument");
  auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  const long V4 = L->V4;
  const size_t fbytes = (size_t)4 * V4 * 8 * sizeof(double);
  const size_t ubytes = (size_t)4 * V4 * 18 * sizeof(double);
  const size_t sbytes = (size_t)2 * L->Vh * L->Ls * 24 * sizeof(double);
  void *F, *Up, *xbuf;
  DWF_TRY(ws_get(L, "fgi.F", fbytes, &F));
  DWF_TRY(ws_get(L, "fgi.Up", ubytes, &Up));
  DWF_TRY(ws_get(L, "fgi.X", sbytes * nterms, &xbuf));
  std::vector<void*> X(nterms);
  for (int t = 0; t < nterms; ++t) X[t] = reinterpret_cast<char*>(xbuf) + t * sbytes;
  dwf_stats tot{};
  int count = 0;
  // F (and the action S) at Ucur; keep: store the solutions; guess: start from them
  auto force = [&](const void* Ucur, bool keep, bool guess, double* S) -> dwf_status {
    DWF_TRY(dwf_set_gauge(L, Ucur));
    if (!guess) DWF_CUDA(L, cudaMemsetAsync(xbuf, 0, sbytes * nterms, L->stream));
    dwf_stats s{};
    DWF_TRY(dwf_force(L, nterms, terms, phi, (keep || guess) ? X.data() : nullptr, F, nullptr, S, cg, &s));
    add_stats(&tot, s);
    ++count;
    return DWF_OK;
  };
  const bool fgi = integ == DWF_INTEGRATOR_FGI;
  const double a = fgi ? 1.0 / 6.0 : kOmelyanLambda;  // weight of the end momentum updates
  double S = 0.0, T = 0.0;
  DWF_TRY(force(U, false, false, &S));
  if (H0) {
    DWF_TRY(dwf_kinetic(L, p, &T));
    *H0 = T + S;
  }
  DWF_TRY(dwf_momentum_update(L, F, -a * tau, p));
  for (int k = 0; k < nsteps; ++k) {
    DWF_TRY(fgi_link_update(L, p, tau / 2.0, U, U));
    if (fgi) {
      // force-gradient step: F(U); U' = exp(-tau^2/24 F) U; p -= 2/3 tau F(U')
      DWF_TRY(force(U, forecast != 0, false, nullptr));
      DWF_TRY(fgi_link_update(L, F, -tau * tau / 24.0, U, Up));
      DWF_TRY(force(Up, false, forecast != 0, nullptr));
      DWF_TRY(dwf_momentum_update(L, F, -2.0 * tau / 3.0, p));
    } else {
      DWF_TRY(force(U, false, false, nullptr));
      DWF_TRY(dwf_momentum_update(L, F, -(1.0 - 2.0 * a) * tau, p));
    }
    DWF_TRY(fgi_link_update(L, p, tau / 2.0, U, U));
    // the closing update of this step and the opening one of the next act at the same U
    DWF_TRY(force(U, false, false, &S));
    DWF_TRY(dwf_momentum_update(L, F, -(k == nsteps - 1 ? a : 2.0 * a) * tau, p));
  }
  if (H1) {
    DWF_TRY(dwf_kinetic(L, p, &T));
    *H1 = T + S;
  }
  tot.launches = L->launches - l0;
  tot.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = tot;
  if (nforce) *nforce = count;
  return DWF_OK;
}

dwf_status dwf_kinetic(dwf_lattice_t L, const void* p, double* T) {
  if (!L || !p || !T) return fail(L, DWF_ERR_INVALID_ARG, "dwf_kinetic: bad argument");
  const long n = 4 * L->V4 * 8;
  const int g = 152 * 8;
  sumsq_kernel<<<g, 256, 0, L->stream>>>(reinterpret_cast<const double*>(p), n, L->partials);
  DWF_LAUNCHED(L);
  DWF_TRY(blas_sum(L, L->partials, g, L->scal + 51));
  DWF_CUDA(L, cudaMemcpyAsync(L->hscal + 51, L->scal + 51, sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  *T = 0.5 * L->hscal[51];
  return DWF_OK;
}

}  // extern "C"

extern "C" dwf_status dwf_action(dwf_lattice_t L, int nterms, const dwf_quotient* terms, const void* const* phi,
                                 const dwf_cg_params* prm, double* S) {
  if (!S) return fail(L, DWF_ERR_INVALID_ARG, "dwf_action: null result pointer");
  return dwf_force(L, nterms, terms, phi, nullptr, nullptr, nullptr, S, prm, nullptr);
}
