// Moebius-accelerated DWF solve (Sec. 4, four-step algorithm; Sec. 5,
// defect correction; Table 1 cost model).
//
// For D_DW(m) x = b on the Shamir lattice of extent Ls, each
// defect-correction pass takes the current residual r = b - D(m) x and
//   1. c  = P^-1 D(1)^-1 r                       (Eq. trans_5d_4d_source; a Pauli-Villars solve)
//   2-3. D'(m) z = D'(1) P c',  c' = (c_1, 0, ..., 0) on the Moebius lattice
//        of extent Ls' (Eq. mob_eq_5d); y'_1 = (P^-1 z)_1 solves Eq. mob_eq_4d
//   4. (., y'_2, ..., y'_L) = P^-1 D(1)^-1 D(m) P (-y'_1, c_2, ..., c_L)  (Eq. recon;
//        the second Pauli-Villars solve), y' = (y'_1, y'_2, ...), x += P y'
// and the accumulated guess then starts the final DWF solve (Sec. 4, the
// approximate solution is used as the initial guess).  Each pass costs two
// Pauli-Villars solves and one Moebius solve.
//
// P shifts the P+ half of the spinor by one slice: (P y)_s = P- y_s + P+ y_{s+1},
// (P^-1 x)_s = P- x_s + P+ x_{s-1} (indices mod Ls); the paper's slice "1" is s = 0.
#include <algorithm>
#include <chrono>
#include <cmath>

#include "dwf_internal.h"

namespace dwf {


namespace {

// out(h,s) = P- in(h,s) + P+ in(h, s + dir mod Ls)   (dir = +1: P, dir = -1: P^-1)
// on FP64 fields; the P+ half is spins 0,1 = reals 0..11 of the spinor.
__global__ void k_pshift(CFieldRef<double> in, FieldRef<double> out, long Vh, int Ls, int Lh, int dir) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Vh * Ls) return;
  const long h = q / Ls;
  const int s = (int)(q - h * Ls);
  int s2 = s + dir;
  s2 = s2 < 0 ? s2 + Ls : (s2 >= Ls ? s2 - Ls : s2);
  double a[24], b[24];
  load_spinor<double>(in, h, s, Lh, a);
  load_spinor<double>(in, h, s2, Lh, b);
#pragma unroll
  for (int k = 0; k < 12; ++k) a[k] = b[k];
  store_spinor<double>(out, h, s, Lh, a);
}

// dst(h, s) = (s == sd) ? scale * src(h, ss) : (zero_rest ? 0 : dst(h, s))
__global__ void k_slice(FieldRef<double> dst, int Ld, int Lhd, int sd, CFieldRef<double> src, int Lhs, int ss,
                        double scale, int zero_rest, long Vh) {
  const long q = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= Vh * Ld) return;
  const long h = q / Ld;
  const int s = (int)(q - h * Ld);
  double v[24];
  if (s == sd) {
    load_spinor<double>(src, h, ss, Lhs, v);
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] *= scale;
  } else if (zero_rest) {
#pragma unroll
    for (int k = 0; k < 24; ++k) v[k] = 0.0;
  } else {
    return;
  }
  store_spinor<double>(dst, h, s, Lhd, v);
}

CFieldRef<double> c64(const Field& f) { return CFieldRef<double>{reinterpret_cast<const double*>(f.v), nullptr}; }
FieldRef<double> w64(const Field& f) { return FieldRef<double>{reinterpret_cast<double*>(f.v), nullptr}; }

dwf_status pshift(dwf_lattice* L, Field in, Field out, int dir) {
  const long n = L->Vh * L->Ls;
  k_pshift<<<(unsigned)((n + 255) / 256), 256, 0, L->stream>>>(c64(in), w64(out), L->Vh, L->Ls, L->Lh, dir);
  DWF_LAUNCHED(L);
  return DWF_OK;
}

dwf_status slice(dwf_lattice* Ld, Field dst, int sd, const dwf_lattice* Lsrc, Field src, int ss, double scale,
                 bool zero_rest) {
  const long n = Ld->Vh * Ld->Ls;
  k_slice<<<(unsigned)((n + 255) / 256), 256, 0, Ld->stream>>>(w64(dst), Ld->Ls, Ld->Lh, sd, c64(src), Lsrc->Lh, ss,
                                                                scale, zero_rest ? 1 : 0, Ld->Vh);
  DWF_LAUNCHED(Ld);
  return DWF_OK;
}

void add_stats(dwf_stats* a, const dwf_stats& b) {
  a->iters += b.iters;
  a->reliable_updates += b.reliable_updates;
  a->hop_calls += b.hop_calls;
  a->op_count += b.op_count;
  a->launches += b.launches;
}

dwf_status norm_pair(dwf_lattice* L, Field e, Field o, double* out) {
  int nb;
  DWF_TRY(blas_norm2(L, e, L->partials, &nb));
  DWF_TRY(blas_sum(L, L->partials, nb, L->scal + 40));
  DWF_TRY(blas_norm2(L, o, L->partials, &nb));
  DWF_TRY(blas_sum(L, L->partials, nb, L->scal + 41));
  DWF_CUDA(L, cudaMemcpyAsync(L->hscal + 40, L->scal + 40, 2 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  *out = std::sqrt(L->hscal[40] + L->hscal[41]);
  return DWF_OK;
}

// one intermediate solve from a zero guess, with its own statistics and
// launch count; its accuracy is the CG residual (no separate FP64 check)
dwf_status timed_solve(dwf_lattice* L, double m, Field be, Field bo, Field xe, Field xo, const dwf_cg_params& prm,
                       dwf_stats* acc) {
  dwf_stats st{};
  const long long l0 = L->launches;
  DWF_TRY(blas_zero(L, xe));
  SolveOpts so;
  so.zero_guess = true;
  so.full_check = false;
  dwf_status s = solve_eo(L, m, be, bo, xe, xo, prm, &st, nullptr, so);
  st.launches = L->launches - l0;
  add_stats(acc, st);
  acc->true_resid = st.true_resid;
  if (s == DWF_ERR_NOT_CONVERGED) return DWF_OK;  // an inexact inner solve is tolerated
  return s;
}

}  // namespace

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status madwf_solve(dwf_lattice_t L, dwf_lattice_t Li, double m, const void* b, void* x,
                                  const madwf_params* prm, madwf_stats* out) {
  if (!L || !Li || !b || !x || !prm) return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: null argument");
  if (b == x) return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: b and x must not alias");
  if (L->X != Li->X || L->Y != Li->Y || L->Z != Li->Z || L->T != Li->T)
    return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: the two lattices must have the same 4D extents");
  if (!L->gauge_set || !Li->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: gauge field not set");
  if (L->p.b != 1.0 || L->p.c != 0.0)
    return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: the outer lattice must be Shamir (b = 1, c = 0)");
  if (prm->n_dc < 0 || prm->n_dc > MADWF_MAX_PASSES || !(prm->tol_final > 0.0) || !(prm->tol_pv > 0.0) ||
      !(prm->tol_mob > 0.0) || prm->max_iter < 1 || !(prm->delta > 0.0 && prm->delta < 1.0) ||
      prm->inner < DWF_F64 || prm->inner > DWF_F16)
    return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: bad parameters");
  if (!std::isfinite(m)) return fail(L, DWF_ERR_INVALID_ARG, "madwf_solve: non-finite mass");
  if (Li->stream != L->stream) DWF_CUDA(L, cudaStreamSynchronize(Li->stream));
  auto t0 = std::chrono::steady_clock::now();
  madwf_stats st{};
  dwf_status s0;
  const SOps* ops_m = sops_for(L, m, &s0);
  if (!ops_m) return s0;
  const SOps* ops1_in = sops_for(Li, 1.0, &s0);
  if (!ops1_in) return fail(L, s0, Li->err);

  Field be, bo, xe, xo, re, ro, ce, co, te, to, ue, uo, ye, yo;
  DWF_TRY(field_alloc(L, "madwf.be", DWF_F64, &be));
  DWF_TRY(field_alloc(L, "madwf.bo", DWF_F64, &bo));
  DWF_TRY(field_alloc(L, "madwf.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "madwf.xo", DWF_F64, &xo));
  DWF_TRY(field_alloc(L, "madwf.re", DWF_F64, &re));
  DWF_TRY(field_alloc(L, "madwf.ro", DWF_F64, &ro));
  DWF_TRY(field_alloc(L, "madwf.ce", DWF_F64, &ce));
  DWF_TRY(field_alloc(L, "madwf.co", DWF_F64, &co));
  DWF_TRY(field_alloc(L, "madwf.te", DWF_F64, &te));
  DWF_TRY(field_alloc(L, "madwf.to", DWF_F64, &to));
  DWF_TRY(field_alloc(L, "madwf.ue", DWF_F64, &ue));
  DWF_TRY(field_alloc(L, "madwf.uo", DWF_F64, &uo));
  DWF_TRY(field_alloc(L, "madwf.ye", DWF_F64, &ye));
  DWF_TRY(field_alloc(L, "madwf.yo", DWF_F64, &yo));
  Field pe, po, qe, qo, ze, zo;  // on the Moebius lattice
  DWF_TRY(field_alloc(Li, "madwf.pe", DWF_F64, &pe));
  DWF_TRY(field_alloc(Li, "madwf.po", DWF_F64, &po));
  DWF_TRY(field_alloc(Li, "madwf.qe", DWF_F64, &qe));
  DWF_TRY(field_alloc(Li, "madwf.qo", DWF_F64, &qo));
  DWF_TRY(field_alloc(Li, "madwf.ze", DWF_F64, &ze));
  DWF_TRY(field_alloc(Li, "madwf.zo", DWF_F64, &zo));

  const long long l0 = L->launches, li0 = Li->launches;
  DWF_TRY(launch_pack(L, b, 0, be));
  DWF_TRY(launch_pack(L, b, 1, bo));
  DWF_TRY(blas_zero(L, xe));
  DWF_TRY(blas_zero(L, xo));
  double bnorm;
  DWF_TRY(norm_pair(L, be, bo, &bnorm));
  if (!std::isfinite(bnorm)) return fail(L, DWF_ERR_NAN, "madwf_solve: non-finite source");

  // The intermediate solves only need their own loose tolerance.  With FP32
  // inner iterations an FP64 reliable update once the residual has dropped
  // by sqrt(tol) (but by no more than 1e-3: over such a reduction the FP32
  // rounding of the recursed residual stays far below the residual) keeps the
  // recursion accurate enough and saves an FP64 residual per solve against a
  // trigger of 1e-2; FP16 storage keeps the caller's delta.
  auto inter_delta = [&](double tol) {
    return prm->inner == DWF_F32 ? std::min(prm->delta, std::max(std::sqrt(tol), 1e-3)) : prm->delta;
  };
  dwf_cg_params pv{prm->tol_pv, prm->max_iter, prm->inner, inter_delta(prm->tol_pv), prm->check_every};
  dwf_cg_params mob{prm->tol_mob, prm->max_iter, prm->inner, inter_delta(prm->tol_mob), prm->check_every};
  dwf_cg_params fin{prm->tol_final, prm->max_iter, prm->inner, prm->delta, prm->check_every};

  // FP32 arithmetic for the passes' FP64-field hops (see below) where its
  // residual floor, ~1e-7 times the operator's condition number, stays well
  // under the tolerances: the Pauli-Villars operator (mass 1) is well
  // conditioned; the Moebius one at the light mass much less so
  const bool pass_fp32 = prm->inner != DWF_F64 && prm->tol_pv >= 1e-5 && prm->tol_mob >= 1e-4;
  dwf_status status = DWF_OK;
  if (bnorm > 0.0) {
    for (int pass = 0; pass < prm->n_dc; ++pass) {
      // r = b - D(m) x  (x = 0 on the first pass: r = b)
      double rn = bnorm;
      if (pass == 0) {
        DWF_TRY(blas_copy(L, be, re));
        DWF_TRY(blas_copy(L, bo, ro));
      } else {
        DWF_TRY(apply_D(L, ops_m, false, xe, xo, re, ro));
        DWF_TRY(blas_axpby(L, 1.0, be, -1.0, re));
        DWF_TRY(blas_axpby(L, 1.0, bo, -1.0, ro));
        DWF_TRY(norm_pair(L, re, ro, &rn));
      }
      if (pass > 0) st.pass_resid[pass - 1] = rn / bnorm;
      if (rn <= prm->tol_final * bnorm) break;
      {
        // The pass's solves and the operator applications that make their
        // sources need only their own loose tolerances, so (pass_fp32) their
        // FP64-field hops compute in FP32: GB300 runs FP64 at ~1/70 of its
        // FP32 rate.  The residuals b - D x between passes stay FP64.
        Fp32StepScope lp_outer(L, pass_fp32), lp_inner(Li, pass_fp32);
        // 1. c = P^-1 D(1)^-1 r
        DWF_TRY(timed_solve(L, 1.0, re, ro, te, to, pv, &st.pv));
        DWF_TRY(pshift(L, te, ce, -1));
        DWF_TRY(pshift(L, to, co, -1));
        // 2-3. c' = (c_1, 0, ...) on the Moebius lattice; D'(m) z = D'(1) P c'
        DWF_TRY(slice(Li, qe, 0, L, ce, 0, 1.0, true));
        DWF_TRY(slice(Li, qo, 0, L, co, 0, 1.0, true));
        DWF_TRY(pshift(Li, qe, pe, +1));
        DWF_TRY(pshift(Li, qo, po, +1));
        DWF_TRY(apply_D(Li, ops1_in, false, pe, po, qe, qo));
        {
          dwf_status s = timed_solve(Li, m, qe, qo, ze, zo, mob, &st.mobius);
          if (s != DWF_OK) return fail(L, s, "madwf_solve (Moebius solve): " + Li->err);
        }
        // y'_1 = (P^-1 z)_1
        DWF_TRY(pshift(Li, ze, pe, -1));
        DWF_TRY(pshift(Li, zo, po, -1));
        // 4. w = (-y'_1, c_2, ..., c_L); u = P^-1 D(1)^-1 D(m) P w
        DWF_TRY(blas_copy(L, ce, ue));
        DWF_TRY(blas_copy(L, co, uo));
        DWF_TRY(slice(L, ue, 0, Li, pe, 0, -1.0, false));
        DWF_TRY(slice(L, uo, 0, Li, po, 0, -1.0, false));
        DWF_TRY(pshift(L, ue, ye, +1));
        DWF_TRY(pshift(L, uo, yo, +1));
        DWF_TRY(apply_D(L, ops_m, false, ye, yo, re, ro));
        DWF_TRY(timed_solve(L, 1.0, re, ro, te, to, pv, &st.pv));
        DWF_TRY(pshift(L, te, ue, -1));
        DWF_TRY(pshift(L, to, uo, -1));
        // y' = (y'_1, u_2, ..., u_L); x += P y'
        DWF_TRY(slice(L, ue, 0, Li, pe, 0, 1.0, false));
        DWF_TRY(slice(L, uo, 0, Li, po, 0, 1.0, false));
        DWF_TRY(pshift(L, ue, ye, +1));
        DWF_TRY(pshift(L, uo, yo, +1));
        DWF_TRY(blas_axpby(L, 1.0, ye, 1.0, xe));
        DWF_TRY(blas_axpby(L, 1.0, yo, 1.0, xo));
      }
      ++st.passes;
    }
    if (st.passes > 0) {
      // the last pass's residual (a statistic: the final solve computes its
      // own).  With pass_fp32, FP32 arithmetic first: its error, ~1e-7 |b|
      // times the operator's condition number, is negligible against a
      // residual of 1e-5 |b| or more; a smaller one is recomputed in FP64.
      double rel = 0.0;
      for (int fp64 = pass_fp32 ? 0 : 1; fp64 < 2; ++fp64) {
        Fp32StepScope lp(L, fp64 == 0);
        DWF_TRY(apply_D(L, ops_m, false, xe, xo, re, ro));
        DWF_TRY(blas_axpby(L, 1.0, be, -1.0, re));
        DWF_TRY(blas_axpby(L, 1.0, bo, -1.0, ro));
        double rn;
        DWF_TRY(norm_pair(L, re, ro, &rn));
        rel = rn / bnorm;
        if (rel >= 1e-5) break;
      }
      st.pass_resid[st.passes - 1] = rel;
    }
    // final DWF solve started from the MADWF guess
    dwf_stats fs{};
    const long long lf = L->launches;
    status = solve_eo(L, m, be, bo, xe, xo, fin, &fs, nullptr);
    fs.launches = L->launches - lf;
    st.final_cg = fs;
    if (status != DWF_OK && status != DWF_ERR_NOT_CONVERGED) return status;
  }
  DWF_TRY(launch_unpack(L, xe, 0, x, false));
  DWF_TRY(launch_unpack(L, xo, 1, x, false));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  st.total = st.pv;
  add_stats(&st.total, st.mobius);
  add_stats(&st.total, st.final_cg);
  st.total.true_resid = bnorm > 0.0 ? st.final_cg.true_resid : 0.0;
  st.total.launches = (L->launches - l0) + (Li->launches - li0);
  st.total.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (out) *out = st;
  return status;
}
