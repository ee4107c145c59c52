// Conjugate gradient on the normal equations of the even-odd operator.
//
// The solve of D(m) x = b (Sec. 4, Eq. dirac_eq) runs on even sites:
//   b'_e = b_e - M_eo A^-1 b_o = b_e + 1/2 Dhop_eo (B A^-1 b_o)
//   M~ x~ = b'_e  with  M~ = M_pc B^-1 = A B^-1 - 1/4 Dhop_eo (B A^-1) Dhop_oe,  x~ = B x_e
//   x_e = B^-1 x~,  x_o = A^-1 b_o + 1/2 A^-1 Dhop_oe x~
// Writing the Schur operator with x~ = B x_e puts every fifth-dimension
// operator after a hop (E1 = B A^-1, E0 = A B^-1), so each application of M~
// or M~^+ is two hop launches with fused epilogues.  For Shamir B = 1.
//
// CG on M~^+ M~ in CGLS form monitors r = b' - M~ x~, whose norm equals the
// full unpreconditioned residual |b - D x| (the odd rows are solved exactly
// by the reconstruction).  Scalars live on the device; the host polls the
// residual every `check_every` iterations.
//
// Mixed precision: the iteration runs on FP32 or FP16-stored vectors (FP32
// arithmetic); the solution accumulates in FP64 and the residual is
// recomputed in FP64 (a reliable update) whenever the iterated residual has
// dropped by `delta` since the last update, and before exit.
#include <chrono>
#include <cmath>

#include "dwf_internal.h"

namespace dwf {

namespace {

enum { S_GAM = 0, S_QQ, S_ALPHA, S_RR, S_BETA, S_TMP0, S_TMP1, S_TMP2 };

struct Op {
  dwf_lattice* L;
  const SOps* ops;
  long long* hops;
};

// out = M~ in (dag = false) or M~^+ in; `u` is an odd temporary of the same precision.
dwf_status apply_Mt(const Op& o, bool dag, Field in, Field out, Field u, double* partials, int* nb) {
  HopCall c1, c2;
  c1.ops = c2.ops = o.ops;
  c1.out_parity = 1;
  c1.dag = dag;
  c1.in = in;
  c1.out = u;
  c1.eout = dag ? SOps::E1T : SOps::E1;
  c2.out_parity = 0;
  c2.dag = dag;
  c2.in = u;
  c2.out = out;
  c2.x = in;
  c2.has_x = true;
  c2.ex = dag ? SOps::E0T : SOps::E0;
  c2.scale = -0.25;
  c2.partials = partials;
  c2.nblocks = nb;
  DWF_TRY(launch_hop(o.L, c1));
  DWF_TRY(launch_hop(o.L, c2));
  *o.hops += 2;
  return DWF_OK;
}

dwf_status fetch_scalars(dwf_lattice* L) {
  DWF_CUDA(L, cudaMemcpyAsync(L->hscal, L->scal, kScalars * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  if (L->timing) DWF_TRY(timing_drain(L));
  return check_dev_err(L);
}

// r64 = b' - M~ x64 (FP64) and |r64|^2 -> hscal[S_TMP0] (synchronises)
dwf_status true_residual(const Op& o, Field bp, Field x64, Field r64, Field u64, double* rr) {
  dwf_lattice* L = o.L;
  DWF_TRY(apply_Mt(o, false, x64, r64, u64, nullptr, nullptr));
  DWF_TRY(blas_axpby(L, 1.0, bp, -1.0, r64));
  int nb;
  DWF_TRY(blas_norm2(L, r64, L->partials, &nb));
  DWF_TRY(blas_sum(L, L->partials, nb, L->scal + S_TMP0));
  DWF_TRY(fetch_scalars(L));
  *rr = L->hscal[S_TMP0];
  return DWF_OK;
}

}  // namespace

// Solve M~ x64 = bp to |b' - M~ x| <= tol * bnorm.  x64 holds the guess.
dwf_status cg_core(dwf_lattice* L, const SOps* ops, Field bp, Field x64, double bnorm,
                   const dwf_cg_params& prm, dwf_stats* st, long long* hops, bool x_zero) {
  const dwf_prec ip = prm.inner;
  Op o{L, ops, hops};
  Field r64, u64;
  DWF_TRY(field_alloc(L, "cg.r64", DWF_F64, &r64));
  DWF_TRY(field_alloc(L, "cg.u64", DWF_F64, &u64));
  Field x, r, s, p, q, u;
  const bool mixed = ip != DWF_F64;
  // The inner solution accumulator stays at least FP32: with 16-bit storage
  // its rounding (relative to |x|, amplified by the condition number) would
  // swamp the residual it is meant to reduce.
  if (mixed) {
    DWF_TRY(field_alloc(L, "cg.x", ip == DWF_F16 ? DWF_F32 : ip, &x));
    DWF_TRY(field_alloc(L, "cg.r", ip, &r));
    DWF_TRY(field_alloc(L, "cg.u", ip, &u));
  } else {
    x = x64;
    r = r64;
    u = u64;
  }
  DWF_TRY(field_alloc(L, "cg.s", ip, &s));
  DWF_TRY(field_alloc(L, "cg.p", ip, &p));
  DWF_TRY(field_alloc(L, "cg.q", ip, &q));
  double* pr = L->partials;
  double* ps = L->partials + kPartials;
  double* sc = L->scal;
  const double tol2 = prm.tol * prm.tol * bnorm * bnorm;
  const double delta2 = prm.delta * prm.delta;
  const int check = prm.check_every < 1 ? 1 : prm.check_every;

  double rr64;
  if (x_zero) {  // r = b' exactly: no operator application needed
    DWF_TRY(blas_copy(L, bp, r64));
    int n0;
    DWF_TRY(blas_norm2(L, r64, L->partials, &n0));
    DWF_TRY(blas_sum(L, L->partials, n0, L->scal + S_TMP0));
    DWF_TRY(fetch_scalars(L));
    rr64 = L->hscal[S_TMP0];
  } else {
    DWF_TRY(true_residual(o, bp, x64, r64, u64, &rr64));
  }
  if (!std::isfinite(rr64)) return fail(L, DWF_ERR_NAN, "cg: non-finite initial residual");
  if (rr64 <= tol2) {
    st->true_resid = std::sqrt(rr64) / bnorm;
    return DWF_OK;
  }
  double maxrr = rr64;
  int nb;
  // start: r = r64 (cast), x = 0, s = M~^+ r, p = s, gam = |s|^2
  if (mixed) {
    DWF_TRY(blas_copy(L, r64, r));
    DWF_TRY(blas_zero(L, x));
  }
  DWF_TRY(apply_Mt(o, true, r, s, u, ps, &nb));
  DWF_TRY(blas_sum(L, ps, nb, sc + S_GAM));
  DWF_TRY(blas_copy(L, s, p));
  int it = 0;
  double rr_host = rr64;
  while (true) {
    // one CGLS iteration
    int nq, nr, ns;
    DWF_TRY(apply_Mt(o, false, p, q, u, pr, &nq));
    DWF_TRY(scal_alpha(L, pr, nq, sc + S_GAM, sc + S_QQ, sc + S_ALPHA));
    DWF_TRY(blas_cg_r(L, sc + S_ALPHA, q, r, pr, &nr));
    DWF_TRY(apply_Mt(o, true, r, s, u, ps, &ns));
    DWF_TRY(scal_beta(L, pr, nr, ps, ns, sc + S_RR, sc + S_GAM, sc + S_BETA));
    DWF_TRY(blas_cg_xp(L, sc + S_ALPHA, sc + S_BETA, s, p, x));
    ++it;
    const bool last = it >= prm.max_iter;
    if (it % check != 0 && !last) continue;
    DWF_TRY(fetch_scalars(L));
    rr_host = L->hscal[S_RR];
    if (!std::isfinite(rr_host) || !std::isfinite(L->hscal[S_GAM])) {
      st->iters += it;
      return fail(L, DWF_ERR_NAN, "cg: non-finite residual norm");
    }
    const bool converged_inner = rr_host <= tol2;
    const bool trigger = mixed && (rr_host < delta2 * maxrr);
    if (converged_inner || trigger || last) {
      // reliable update / final check in FP64
      if (mixed) {
        DWF_TRY(blas_accum(L, x, x64));
        DWF_TRY(blas_zero(L, x));
      }
      DWF_TRY(true_residual(o, bp, x64, r64, u64, &rr64));
      ++st->reliable_updates;
      if (!std::isfinite(rr64)) {
        st->iters += it;
        return fail(L, DWF_ERR_NAN, "cg: non-finite true residual");
      }
      if (rr64 <= tol2) break;
      if (last) {
        st->iters += it;
        st->true_resid = std::sqrt(rr64) / bnorm;
        return fail(L, DWF_ERR_NOT_CONVERGED, "cg: max_iter reached");
      }
      // restart the recursion from the FP64 residual, keeping p
      if (mixed) DWF_TRY(blas_copy(L, r64, r));
      DWF_TRY(apply_Mt(o, true, r, s, u, ps, &ns));
      DWF_TRY(blas_sum(L, ps, ns, sc + S_GAM));
      maxrr = rr64;
    } else if (rr_host > maxrr) {
      maxrr = rr_host;
    }
  }
  st->iters += it;
  st->true_resid = std::sqrt(rr64) / bnorm;
  return DWF_OK;
}

// CG on the normal operator: solve M~^+ M~ x64 = v to |v - M~^+ M~ x| <= tol |v|
// (the force solve X = (M^+ M)^-1 M2^+ phi of Sec. 2-3).  x64 holds the guess.
// Same reliable-update scheme as cg_core.
dwf_status cgne_core(dwf_lattice* L, const SOps* ops, Field v, Field x64, const dwf_cg_params& prm, dwf_stats* st,
                     long long* hops) {
  const dwf_prec ip = prm.inner;
  Op o{L, ops, hops};
  Field r64, w64, u64;
  DWF_TRY(field_alloc(L, "ne.r64", DWF_F64, &r64));
  DWF_TRY(field_alloc(L, "ne.w64", DWF_F64, &w64));
  DWF_TRY(field_alloc(L, "ne.u64", DWF_F64, &u64));
  const bool mixed = ip != DWF_F64;
  Field x, r, p, w, q, u;
  if (mixed) {
    DWF_TRY(field_alloc(L, "ne.x", ip == DWF_F16 ? DWF_F32 : ip, &x));
    DWF_TRY(field_alloc(L, "ne.r", ip, &r));
    DWF_TRY(field_alloc(L, "ne.u", ip, &u));
    DWF_TRY(field_alloc(L, "ne.w", ip, &w));
  } else {
    x = x64;
    r = r64;
    u = u64;
    w = w64;
  }
  DWF_TRY(field_alloc(L, "ne.p", ip, &p));
  DWF_TRY(field_alloc(L, "ne.q", ip, &q));
  double* pr = L->partials;
  double* sc = L->scal;
  int nb;
  DWF_TRY(blas_norm2(L, v, pr, &nb));
  DWF_TRY(blas_sum(L, pr, nb, sc + S_TMP1));
  DWF_TRY(fetch_scalars(L));
  const double vv = L->hscal[S_TMP1];
  if (!std::isfinite(vv)) return fail(L, DWF_ERR_NAN, "cgne: non-finite right-hand side");
  if (vv == 0.0) {
    DWF_TRY(blas_zero(L, x64));
    st->true_resid = 0.0;
    return DWF_OK;
  }
  const double tol2 = prm.tol * prm.tol * vv;
  const double delta2 = prm.delta * prm.delta;
  const int check = prm.check_every < 1 ? 1 : prm.check_every;
  // r64 = v - M~^+ M~ x64
  auto true_res = [&](double* rr) -> dwf_status {
    DWF_TRY(apply_Mt(o, false, x64, w64, u64, nullptr, nullptr));
    DWF_TRY(apply_Mt(o, true, w64, r64, u64, nullptr, nullptr));
    DWF_TRY(blas_axpby(L, 1.0, v, -1.0, r64));
    int n2;
    DWF_TRY(blas_norm2(L, r64, pr, &n2));
    DWF_TRY(blas_sum(L, pr, n2, sc + S_TMP0));
    DWF_TRY(fetch_scalars(L));
    *rr = L->hscal[S_TMP0];
    return DWF_OK;
  };
  double rr64;
  DWF_TRY(true_res(&rr64));
  if (!std::isfinite(rr64)) return fail(L, DWF_ERR_NAN, "cgne: non-finite initial residual");
  if (rr64 <= tol2) {
    st->true_resid = std::sqrt(rr64 / vv);
    return DWF_OK;
  }
  if (mixed) {
    DWF_TRY(blas_copy(L, r64, r));
    DWF_TRY(blas_zero(L, x));
  }
  DWF_TRY(blas_copy(L, r, p));
  DWF_TRY(blas_norm2(L, r, pr, &nb));
  DWF_TRY(blas_sum(L, pr, nb, sc + S_GAM));  // gam = |r|^2
  double maxrr = rr64;
  int it = 0;
  while (true) {
    int nw, nr;
    DWF_TRY(apply_Mt(o, false, p, w, u, pr, &nw));  // |w|^2 = <p, N p>
    DWF_TRY(scal_alpha(L, pr, nw, sc + S_GAM, sc + S_QQ, sc + S_ALPHA));
    DWF_TRY(apply_Mt(o, true, w, q, u, nullptr, nullptr));
    DWF_TRY(blas_cg_r(L, sc + S_ALPHA, q, r, pr, &nr));
    DWF_TRY(scal_beta(L, pr, nr, pr, nr, sc + S_RR, sc + S_GAM, sc + S_BETA));
    DWF_TRY(blas_cg_xp(L, sc + S_ALPHA, sc + S_BETA, r, p, x));
    ++it;
    const bool last = it >= prm.max_iter;
    if (it % check != 0 && !last) continue;
    DWF_TRY(fetch_scalars(L));
    const double rr = L->hscal[S_RR];
    if (!std::isfinite(rr)) {
      st->iters += it;
      return fail(L, DWF_ERR_NAN, "cgne: non-finite residual norm");
    }
    if (rr <= tol2 || (mixed && rr < delta2 * maxrr) || last) {
      if (mixed) {
        DWF_TRY(blas_accum(L, x, x64));
        DWF_TRY(blas_zero(L, x));
      }
      DWF_TRY(true_res(&rr64));
      ++st->reliable_updates;
      if (rr64 <= tol2) break;
      if (last) {
        st->iters += it;
        st->true_resid = std::sqrt(rr64 / vv);
        return fail(L, DWF_ERR_NOT_CONVERGED, "cgne: max_iter reached");
      }
      if (mixed) DWF_TRY(blas_copy(L, r64, r));
      DWF_TRY(blas_norm2(L, r, pr, &nb));
      DWF_TRY(blas_sum(L, pr, nb, sc + S_GAM));
      maxrr = rr64;
    } else if (rr > maxrr) {
      maxrr = rr;
    }
  }
  st->iters += it;
  st->true_resid = std::sqrt(rr64 / vv);
  return DWF_OK;
}

// Full solve on FP64 parity fields: b (be, bo) -> x (xe, xo; xe holds the guess).
dwf_status solve_eo(dwf_lattice* L, double m, Field be, Field bo, Field xe, Field xo, const dwf_cg_params& prm,
                    dwf_stats* st, double* true_res_full, const SolveOpts& opts) {
  dwf_status s0;
  const SOps* ops = sops_for(L, m, &s0);
  if (!ops) return s0;
  long long hops = 0;
  Field bp, xt, t, ye, yo;
  DWF_TRY(field_alloc(L, "solve.bp", DWF_F64, &bp));
  DWF_TRY(field_alloc(L, "solve.xt", DWF_F64, &xt));
  DWF_TRY(field_alloc(L, "solve.t", DWF_F64, &t));
  // |b|
  int nb;
  DWF_TRY(blas_norm2(L, be, L->partials, &nb));
  DWF_TRY(blas_sum(L, L->partials, nb, L->scal + S_TMP1));
  DWF_TRY(blas_norm2(L, bo, L->partials, &nb));
  DWF_TRY(blas_sum(L, L->partials, nb, L->scal + S_TMP2));
  DWF_TRY(fetch_scalars(L));
  const double bnorm = std::sqrt(L->hscal[S_TMP1] + L->hscal[S_TMP2]);
  if (!std::isfinite(bnorm)) return fail(L, DWF_ERR_NAN, "cg: non-finite source");
  if (bnorm == 0.0) {
    DWF_TRY(blas_zero(L, xe));
    DWF_TRY(blas_zero(L, xo));
    st->true_resid = 0.0;
    if (true_res_full) *true_res_full = 0.0;
    return DWF_OK;
  }
  // b' = b_e + 1/2 Dhop_eo (B A^-1 b_o)
  DWF_TRY(launch_sop(L, bo, t, ops, SOps::E1, 1.0, nullptr, 0.0));
  {
    HopCall c;
    c.out_parity = 0;
    c.in = t;
    c.out = bp;
    c.x = be;
    c.has_x = true;
    c.scale = 0.5;
    c.ops = ops;
    DWF_TRY(launch_hop(L, c));
    ++hops;
  }
  // x~ = B x_e
  if (opts.zero_guess)
    DWF_TRY(blas_zero(L, xt));
  else
    DWF_TRY(launch_sop(L, xe, xt, ops, SOps::B, 1.0, nullptr, 0.0));
  dwf_status cs = DWF_OK;
  double res = 0.0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    cs = cg_core(L, ops, bp, xt, bnorm, prm, st, &hops, opts.zero_guess && attempt == 0);
    if (cs != DWF_OK && cs != DWF_ERR_NOT_CONVERGED) return cs;
    // reconstruct: x_e = B^-1 x~;  x_o = A^-1 b_o + 1/2 A^-1 Dhop_oe x~
    DWF_TRY(launch_sop(L, xt, xe, ops, SOps::BINV, 1.0, nullptr, 0.0));
    HopCall c;
    c.out_parity = 1;
    c.in = xt;
    c.out = xo;
    c.x = bo;
    c.has_x = true;
    c.eout = SOps::AINV;
    c.scale = 0.5;
    c.ops = ops;
    DWF_TRY(launch_hop(L, c));
    ++hops;
    if (!opts.full_check) {  // the CG residual |b' - M~ x~| stands for |b - D x|
      res = st->true_resid;
      break;
    }
    // true residual of the full system
    DWF_TRY(field_alloc(L, "solve.ye", DWF_F64, &ye));
    DWF_TRY(field_alloc(L, "solve.yo", DWF_F64, &yo));
    DWF_TRY(apply_D(L, ops, false, xe, xo, ye, yo));
    hops += 2;
    DWF_TRY(blas_axpby(L, 1.0, be, -1.0, ye));
    DWF_TRY(blas_axpby(L, 1.0, bo, -1.0, yo));
    DWF_TRY(blas_norm2(L, ye, L->partials, &nb));
    DWF_TRY(blas_sum(L, L->partials, nb, L->scal + S_TMP1));
    DWF_TRY(blas_norm2(L, yo, L->partials, &nb));
    DWF_TRY(blas_sum(L, L->partials, nb, L->scal + S_TMP2));
    DWF_TRY(fetch_scalars(L));
    res = std::sqrt(L->hscal[S_TMP1] + L->hscal[S_TMP2]) / bnorm;
    if (cs != DWF_OK || res <= prm.tol || st->iters >= prm.max_iter) break;
  }
  st->true_resid = res;
  st->hop_calls += hops;
  st->op_count += (long long)st->iters * L->Ls;
  if (true_res_full) *true_res_full = res;
  if (cs == DWF_OK && res > prm.tol) return fail(L, DWF_ERR_NOT_CONVERGED, "cg: true residual above tolerance");
  return cs;
}

}  // namespace dwf

using namespace dwf;

// M_pc x (or M_pc^+ x) at storage precision `prec` through the solver's own
// hop launches: M_pc = M~ B, so M_pc x = M~ (B x) and M_pc^+ x = B^+ (M~^+ x).
extern "C" dwf_status dwf_apply_Mpc_prec(dwf_lattice_t L, double m, int dag, dwf_prec prec, const void* in,
                                         void* out) {
  if (!L || !in || !out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_prec: null argument");
  if (in == out) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_prec: in and out must not alias");
  if (prec < DWF_F64 || prec > DWF_F16) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_prec: bad precision");
  if (!std::isfinite(m)) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_prec: non-finite mass");
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "dwf_apply_Mpc_prec: gauge field not set");
  dwf_status st;
  const SOps* ops = sops_for(L, m, &st);
  if (!ops) return st;
  Field xe, t, ye, u;
  DWF_TRY(field_alloc(L, "applyp.xe", prec, &xe));
  DWF_TRY(field_alloc(L, "applyp.t", prec, &t));
  DWF_TRY(field_alloc(L, "applyp.ye", prec, &ye));
  DWF_TRY(field_alloc(L, "applyp.u", prec, &u));
  DWF_TRY(launch_pack(L, in, 0, xe));
  long long hops = 0;
  Op o{L, ops, &hops};
  if (!dag) {
    DWF_TRY(launch_sop(L, xe, t, ops, SOps::B, 1.0, nullptr, 0.0));
    DWF_TRY(apply_Mt(o, false, t, ye, u, nullptr, nullptr));
  } else {
    DWF_TRY(apply_Mt(o, true, xe, t, u, nullptr, nullptr));
    DWF_TRY(launch_sop(L, t, ye, ops, SOps::BT, 1.0, nullptr, 0.0));
  }
  DWF_TRY(launch_unpack(L, ye, 0, out, true));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return check_dev_err(L);
}

extern "C" dwf_status dwf_cg(dwf_lattice_t L, double m, const void* b, void* x, const dwf_cg_params* prm,
                             dwf_stats* stats) {
  if (!L || !b || !x || !prm) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg: null argument");
  if (b == x) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg: b and x must not alias");
  if (!(prm->tol > 0.0) || prm->max_iter < 1 || prm->inner < DWF_F64 || prm->inner > DWF_F16 ||
      !(prm->delta > 0.0 && prm->delta < 1.0))
    return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg: bad solver parameters");
  if (!std::isfinite(m)) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg: non-finite mass");
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg: gauge field not set");
  auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  dwf_stats st{};
  Field be, bo, xe, xo;
  DWF_TRY(field_alloc(L, "io.be", DWF_F64, &be));
  DWF_TRY(field_alloc(L, "io.bo", DWF_F64, &bo));
  DWF_TRY(field_alloc(L, "io.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "io.xo", DWF_F64, &xo));
  DWF_TRY(launch_pack(L, b, 0, be));
  DWF_TRY(launch_pack(L, b, 1, bo));
  DWF_TRY(launch_pack(L, x, 0, xe));
  dwf_status s = solve_eo(L, m, be, bo, xe, xo, *prm, &st, nullptr);
  if (s == DWF_OK || s == DWF_ERR_NOT_CONVERGED) {
    DWF_TRY(launch_unpack(L, xe, 0, x, false));
    DWF_TRY(launch_unpack(L, xo, 1, x, false));
    DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  }
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  st.launches = L->launches - l0;
  if (stats) *stats = st;
  return s;
}
