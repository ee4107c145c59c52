// Multi-right-hand-side CG for a Hasenbusch mass ladder.
//
// The mass splitting of Sec. 3 (the product of determinant ratios over
// m + mu_i) gives, on one gauge field, one Dirac equation per mass of the
// ladder.  They are solved together: each right-hand side r runs its own CG
// on the normal equations of M~(m_r) (the even-odd Schur operator with
// x~ = B x_e, as in the single solve), with its own scalars and FP64
// reliable updates, but the iterations are taken in lockstep so that every
// Wilson hop step of an iteration covers all still-unconverged right-hand
// sides in one launch (the 8 links of a 4D site are staged once for all of
// them; the fused fifth-dimension epilogues use each right-hand side's mass).
// A right-hand side that converges leaves the batch, so the work per
// iteration shrinks with the ladder.
//
// One iteration for a fixed batch is recorded as a CUDA graph the first time
// that batch occurs and replayed afterwards (scalars live on the device, so
// the host only polls every check_every iterations).  Launch shapes (right-
// hand sides per launch, CTAs per SM) come from the autotuner in tune.cu.
#include <chrono>
#include <cmath>
#include <cstring>

#include "dwf_internal.h"

namespace dwf {


namespace {

constexpr int kScalBase = 64;  // per-right-hand-side scalars: L->scal + kScalBase + 8 r
enum { M_GAM = 0, M_QQ, M_ALPHA, M_RR, M_BETA, M_TMP0, M_TMP1 };

struct Rhs {
  double m = 0.0;
  const SOps* ops = nullptr;
  Field bp, xt;                // FP64: b'_e and x~ = B x_e (the accumulated solution)
  Field x, r, s, p, q, u;      // iteration vectors at the inner precision (x: FP64 / FP32)
  double* pr = nullptr;        // partial sums (device, kPartials doubles each)
  double* ps = nullptr;
  int nq = 0, nr = 0, ns = 0;  // their block counts
  double bnorm = 0.0, tol2 = 0.0, maxrr = 0.0;
  bool active = false, zero = false;
  dwf_status status = DWF_OK;
  dwf_stats st{};
};

struct Multi {
  dwf_lattice* L = nullptr;
  dwf_cg_params prm{};
  bool mixed = false, autotune = true, graphs = true;
  std::vector<Rhs> R;
  std::map<std::string, HopChoice> choice;  // per call: (batch size, step) -> launch shape
  std::map<unsigned, cudaGraphExec_t> exec;
  std::map<unsigned, long long> exec_launches;
  double tune_seconds = 0.0;
  long long replays = 0;
  int iterations = 0;
  int first_k = 0, first_batch = 0, first_ctas = 0;
  ~Multi() {
    for (auto& kv : exec) cudaGraphExecDestroy(kv.second);
  }
  double* sc(int r, int k) { return L->scal + kScalBase + 8 * r + k; }
  double hs(int r, int k) const { return L->hscal[kScalBase + 8 * r + k]; }
};

// Runs the solve on a private non-blocking stream (graphs cannot be recorded
// on the legacy default stream) joined to the caller's stream on both ends.
struct StreamSwap {
  dwf_lattice* L = nullptr;
  cudaStream_t user = nullptr, own = nullptr;
  cudaEvent_t ev = nullptr;
  dwf_status begin(dwf_lattice* Lp) {
    L = Lp;
    user = L->stream;
    DWF_CUDA(L, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    DWF_CUDA(L, cudaStreamCreateWithFlags(&own, cudaStreamNonBlocking));
    DWF_CUDA(L, cudaEventRecord(ev, user));
    DWF_CUDA(L, cudaStreamWaitEvent(own, ev, 0));
    L->stream = own;
    return DWF_OK;
  }
  ~StreamSwap() {
    if (!L) return;
    if (own) {
      cudaEventRecord(ev, own);
      cudaStreamWaitEvent(user, ev, 0);
      cudaStreamDestroy(own);
    }
    if (ev) cudaEventDestroy(ev);
    L->stream = user;
  }
};

dwf_status fetch(dwf_lattice* L) {
  DWF_CUDA(L, cudaMemcpyAsync(L->hscal, L->scal, (kScalars - 1) * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  if (L->timing) DWF_TRY(timing_drain(L));
  return check_dev_err(L);
}

int sop_kind(const SOps* ops, SOps::Kind k) { return k == SOps::NKIND ? 0 : ops->desc[k].kind; }

// One hop step (c's parity / dagger / kinds / scales) over the right-hand
// sides `set`: out[i] = step(in[i], x[i]) with the operators of set[i].
dwf_status hop_step(Multi& M, const std::vector<int>& set, const HopCall& c, const Field* in, const Field* out,
                    const Field* x, double* const* part, int* nb) {
  dwf_lattice* L = M.L;
  const int k = (int)set.size();
  const dwf_prec prec = in[0].prec;
  const int bmax = hop_batch_max(L->Ls, prec);
  auto launch = [&](const HopChoice& ch) -> dwf_status {
    if (bmax == 0) {  // FP64 or a shape the pipelined kernel does not take: one launch each
      for (int i = 0; i < k; ++i) {
        HopCall h = c;
        h.in = in[i];
        h.out = out[i];
        if (c.has_x) h.x = x[i];
        h.ops = M.R[set[i]].ops;
        h.partials = part ? part[i] : nullptr;
        h.nblocks = nb ? &nb[i] : nullptr;
        DWF_TRY(launch_hop(L, h));
      }
      return DWF_OK;
    }
    for (int a0 = 0; a0 < k; a0 += ch.batch) {
      HopBatch b;
      b.nrhs = k - a0 < ch.batch ? k - a0 : ch.batch;
      for (int q = 0; q < b.nrhs; ++q) {
        b.in[q] = in[a0 + q];
        b.out[q] = out[a0 + q];
        if (c.has_x) b.x[q] = x[a0 + q];
        b.ops[q] = M.R[set[a0 + q]].ops;
        b.partials[q] = part ? part[a0 + q] : nullptr;
      }
      int g = 0;
      HopCall h = c;
      h.nblocks = &g;
      DWF_TRY(launch_hop_batch(L, h, b, ch.ctas_per_sm));
      if (nb)
        for (int q = 0; q < b.nrhs; ++q) nb[a0 + q] = g;
    }
    return DWF_OK;
  };
  HopChoice ch;
  ch.batch = bmax > 0 ? (k < bmax ? k : bmax) : 1;
  if (bmax > 0 && M.autotune) {
    const HopShape s{L->Vh, L->Ls, (int)prec, k, c.dag, c.has_x ? 1 : 0, sop_kind(M.R[set[0]].ops, c.ex),
                     sop_kind(M.R[set[0]].ops, c.eout)};
    const std::string key = std::to_string(k) + "/" + std::to_string(c.dag) + std::to_string(c.has_x);
    auto it = M.choice.find(key);
    if (it != M.choice.end()) {
      ch = it->second;
    } else {
      DWF_TRY(tune_hop(L, s, bmax, launch, &ch, &M.tune_seconds));
      M.choice[key] = ch;
    }
  }
  if (k > M.first_k) {  // report the shape chosen for the largest batch
    M.first_k = k;
    M.first_batch = ch.batch;
    M.first_ctas = ch.ctas_per_sm;
  }
  return launch(ch);
}

// out = M~ in (dag = false) or M~^+ in for every right-hand side of the set;
// part / nb (optional) receive the partial sums of |out|^2.
dwf_status apply_Mt_set(Multi& M, const std::vector<int>& set, bool dag, const Field* in, const Field* out,
                        const Field* u, double* const* part, int* nb) {
  HopCall c1;
  c1.out_parity = 1;
  c1.dag = dag;
  c1.eout = dag ? SOps::E1T : SOps::E1;
  DWF_TRY(hop_step(M, set, c1, in, u, nullptr, nullptr, nullptr));
  HopCall c2;
  c2.out_parity = 0;
  c2.dag = dag;
  c2.has_x = true;
  c2.ex = dag ? SOps::E0T : SOps::E0;
  c2.scale = -0.25;
  return hop_step(M, set, c2, u, out, in, part, nb);
}

template <class F> std::vector<Field> gather(Multi& M, const std::vector<int>& set, F f) {
  std::vector<Field> v;
  for (int r : set) v.push_back(f(M.R[r]));
  return v;
}

// One CG iteration (CGLS form, as in the single solve) for every right-hand side of the set.
dwf_status iterate(Multi& M, const std::vector<int>& set) {
  dwf_lattice* L = M.L;
  const int k = (int)set.size();
  std::vector<double*> pr(k), ps(k);
  std::vector<int> nq(k), ns(k);
  for (int i = 0; i < k; ++i) {
    pr[i] = M.R[set[i]].pr;
    ps[i] = M.R[set[i]].ps;
  }
  const auto P = gather(M, set, [](Rhs& r) { return r.p; });
  const auto Q = gather(M, set, [](Rhs& r) { return r.q; });
  const auto U = gather(M, set, [](Rhs& r) { return r.u; });
  const auto Rr = gather(M, set, [](Rhs& r) { return r.r; });
  const auto S = gather(M, set, [](Rhs& r) { return r.s; });
  DWF_TRY(apply_Mt_set(M, set, false, P.data(), Q.data(), U.data(), pr.data(), nq.data()));
  for (int i = 0; i < k; ++i) {
    const int r = set[i];
    DWF_TRY(scal_alpha(L, pr[i], nq[i], M.sc(r, M_GAM), M.sc(r, M_QQ), M.sc(r, M_ALPHA)));
  }
  for (int i = 0; i < k; ++i) {
    Rhs& R = M.R[set[i]];
    DWF_TRY(blas_cg_r(L, M.sc(set[i], M_ALPHA), R.q, R.r, pr[i], &R.nr));
  }
  DWF_TRY(apply_Mt_set(M, set, true, Rr.data(), S.data(), U.data(), ps.data(), ns.data()));
  for (int i = 0; i < k; ++i) {
    const int r = set[i];
    DWF_TRY(scal_beta(L, pr[i], M.R[r].nr, ps[i], ns[i], M.sc(r, M_RR), M.sc(r, M_GAM), M.sc(r, M_BETA)));
  }
  for (int i = 0; i < k; ++i) {
    Rhs& R = M.R[set[i]];
    DWF_TRY(blas_cg_xp(L, M.sc(set[i], M_ALPHA), M.sc(set[i], M_BETA), R.s, R.p, R.x));
  }
  return DWF_OK;
}

// r64 = b' - M~ x~ in FP64 for right-hand side r; |r64|^2 -> *rr (synchronises)
dwf_status true_residual(Multi& M, int r, Field r64, Field u64, double* rr) {
  dwf_lattice* L = M.L;
  const std::vector<int> one{r};
  Rhs& R = M.R[r];
  DWF_TRY(apply_Mt_set(M, one, false, &R.xt, &r64, &u64, nullptr, nullptr));
  DWF_TRY(blas_axpby(L, 1.0, R.bp, -1.0, r64));
  int nb = 0;
  DWF_TRY(blas_norm2(L, r64, R.pr, &nb));
  DWF_TRY(blas_sum(L, R.pr, nb, M.sc(r, M_TMP0)));
  DWF_TRY(fetch(L));
  *rr = M.hs(r, M_TMP0);
  R.st.hop_calls += 2;
  return DWF_OK;
}

// Restart the recursion of r from the FP64 residual r64: r = r64, s = M~^+ r, gam = |s|^2.
dwf_status restart(Multi& M, int r, Field r64) {
  dwf_lattice* L = M.L;
  Rhs& R = M.R[r];
  const std::vector<int> one{r};
  DWF_TRY(blas_copy(L, r64, R.r));
  int ns = 0;
  DWF_TRY(apply_Mt_set(M, one, true, &R.r, &R.s, &R.u, &R.ps, &ns));
  DWF_TRY(blas_sum(L, R.ps, ns, M.sc(r, M_GAM)));
  R.st.hop_calls += 2;
  return DWF_OK;
}

unsigned mask_of(const std::vector<int>& set) {
  unsigned m = 0;
  for (int r : set) m |= 1u << r;
  return m;
}

// Run n iterations of the set: eagerly, or through its graph (recorded on first use).
dwf_status run_iterations(Multi& M, const std::vector<int>& set, int n) {
  dwf_lattice* L = M.L;
  int done = 0;
  if (M.graphs) {
    const unsigned key = mask_of(set);
    if (!M.exec.count(key)) {
      DWF_TRY(iterate(M, set));  // eager: tunes any new launch shape outside the recording
      ++done;
      const bool timing = L->timing;  // launches inside a graph are not bracketed by events
      L->timing = false;
      const long long l0 = L->launches;
      DWF_CUDA(L, cudaStreamBeginCapture(L->stream, cudaStreamCaptureModeThreadLocal));
      const dwf_status s = iterate(M, set);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(L->stream, &g);
      L->timing = timing;
      const long long nl = L->launches - l0;
      L->launches = l0;
      if (s != DWF_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e != cudaSuccess) return cuda_check(L, e, "cudaStreamEndCapture");
      cudaGraphExec_t x = nullptr;
      const cudaError_t ei = cudaGraphInstantiate(&x, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) return cuda_check(L, ei, "cudaGraphInstantiate");
      M.exec[key] = x;
      M.exec_launches[key] = nl;
    }
    const cudaGraphExec_t x = M.exec[key];
    for (; done < n; ++done) {
      DWF_CUDA(L, cudaGraphLaunch(x, L->stream));
      counted(L, (int)M.exec_launches[key]);
      ++M.replays;
    }
    return DWF_OK;
  }
  for (; done < n; ++done) DWF_TRY(iterate(M, set));
  return DWF_OK;
}

// Allocates every field and prepares b'_r and x~_r; marks zero sources.
dwf_status setup(Multi& M, const double* masses, const void* const* b, void* const* x) {
  dwf_lattice* L = M.L;
  const dwf_prec ip = M.prm.inner;
  double* part = nullptr;
  DWF_TRY(ws_get(L, "multi.partials", 2 * M.R.size() * (size_t)kPartials * sizeof(double),
                 reinterpret_cast<void**>(&part)));
  Field be, bo, xe, t;
  DWF_TRY(field_alloc(L, "io.be", DWF_F64, &be));
  DWF_TRY(field_alloc(L, "io.bo", DWF_F64, &bo));
  DWF_TRY(field_alloc(L, "io.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "solve.t", DWF_F64, &t));
  for (size_t r = 0; r < M.R.size(); ++r) {
    Rhs& R = M.R[r];
    const std::string n = std::to_string(r);
    R.m = masses[r];
    dwf_status s0;
    R.ops = sops_for(L, R.m, &s0);
    if (!R.ops) return s0;
    R.pr = part + 2 * r * (size_t)kPartials;
    R.ps = R.pr + kPartials;
    DWF_TRY(field_alloc(L, "multi.bp." + n, DWF_F64, &R.bp));
    DWF_TRY(field_alloc(L, "multi.xt." + n, DWF_F64, &R.xt));
    if (M.mixed) {
      DWF_TRY(field_alloc(L, "multi.x." + n, ip == DWF_F16 ? DWF_F32 : ip, &R.x));
    } else {
      R.x = R.xt;
    }
    DWF_TRY(field_alloc(L, "multi.r." + n, ip, &R.r));
    DWF_TRY(field_alloc(L, "multi.s." + n, ip, &R.s));
    DWF_TRY(field_alloc(L, "multi.p." + n, ip, &R.p));
    DWF_TRY(field_alloc(L, "multi.q." + n, ip, &R.q));
    DWF_TRY(field_alloc(L, "multi.u." + n, ip, &R.u));
    // |b|, b' = b_e + 1/2 Dhop_eo (B A^-1 b_o), x~ = B x_e
    DWF_TRY(launch_pack(L, b[r], 0, be));
    DWF_TRY(launch_pack(L, b[r], 1, bo));
    DWF_TRY(launch_pack(L, x[r], 0, xe));
    int nb = 0;
    DWF_TRY(blas_norm2(L, be, R.pr, &nb));
    DWF_TRY(blas_sum(L, R.pr, nb, M.sc((int)r, M_TMP0)));
    DWF_TRY(blas_norm2(L, bo, R.pr, &nb));
    DWF_TRY(blas_sum(L, R.pr, nb, M.sc((int)r, M_TMP1)));
    DWF_TRY(fetch(L));
    R.bnorm = std::sqrt(M.hs((int)r, M_TMP0) + M.hs((int)r, M_TMP1));
    if (!std::isfinite(R.bnorm)) return fail(L, DWF_ERR_NAN, "cg_multi: non-finite source");
    R.tol2 = M.prm.tol * M.prm.tol * R.bnorm * R.bnorm;
    if (R.bnorm == 0.0) {
      R.zero = true;
      continue;
    }
    DWF_TRY(launch_sop(L, bo, t, R.ops, SOps::E1, 1.0, nullptr, 0.0));
    HopCall c;
    c.out_parity = 0;
    c.in = t;
    c.out = R.bp;
    c.x = be;
    c.has_x = true;
    c.scale = 0.5;
    c.ops = R.ops;
    DWF_TRY(launch_hop(L, c));
    DWF_TRY(launch_sop(L, xe, R.xt, R.ops, SOps::B, 1.0, nullptr, 0.0));
    R.st.hop_calls += 1;
  }
  return DWF_OK;
}

// The joint iteration until every right-hand side has converged or hit max_iter.
dwf_status solve_all(Multi& M) {
  dwf_lattice* L = M.L;
  Field r64, u64;
  DWF_TRY(field_alloc(L, "cg.r64", DWF_F64, &r64));
  DWF_TRY(field_alloc(L, "cg.u64", DWF_F64, &u64));
  const double delta2 = M.prm.delta * M.prm.delta;
  const int check = M.prm.check_every < 1 ? 1 : M.prm.check_every;
  // start every right-hand side from its FP64 residual
  for (size_t r = 0; r < M.R.size(); ++r) {
    Rhs& R = M.R[r];
    if (R.zero) continue;
    double rr64 = 0.0;
    DWF_TRY(true_residual(M, (int)r, r64, u64, &rr64));
    if (!std::isfinite(rr64)) {
      R.status = fail(L, DWF_ERR_NAN, "cg_multi: non-finite initial residual");
      continue;
    }
    R.st.true_resid = std::sqrt(rr64) / R.bnorm;
    if (rr64 <= R.tol2) continue;
    if (M.mixed) DWF_TRY(blas_zero(L, R.x));
    DWF_TRY(restart(M, (int)r, r64));
    DWF_TRY(blas_copy(L, R.s, R.p));
    R.maxrr = rr64;
    R.active = true;
  }
  while (true) {
    std::vector<int> set;
    for (size_t r = 0; r < M.R.size(); ++r)
      if (M.R[r].active) set.push_back((int)r);
    if (set.empty()) break;
    int n = check;
    for (int r : set) {
      const int left = M.prm.max_iter - M.R[r].st.iters;
      if (left < n) n = left;
    }
    if (n < 1) n = 1;
    DWF_TRY(run_iterations(M, set, n));
    M.iterations += n;
    for (int r : set) {
      M.R[r].st.iters += n;
      M.R[r].st.hop_calls += 4LL * n;
    }
    DWF_TRY(fetch(L));
    for (int r : set) {
      Rhs& R = M.R[r];
      const double rr = M.hs(r, M_RR);
      if (!std::isfinite(rr) || !std::isfinite(M.hs(r, M_GAM))) {
        R.status = fail(L, DWF_ERR_NAN, "cg_multi: non-finite residual norm");
        R.active = false;
        continue;
      }
      const bool last = R.st.iters >= M.prm.max_iter;
      if (rr <= R.tol2 || (M.mixed && rr < delta2 * R.maxrr) || last) {
        if (M.mixed) {
          DWF_TRY(blas_accum(L, R.x, R.xt));
          DWF_TRY(blas_zero(L, R.x));
        }
        double rr64 = 0.0;
        DWF_TRY(true_residual(M, r, r64, u64, &rr64));
        ++R.st.reliable_updates;
        R.st.true_resid = std::sqrt(rr64) / R.bnorm;
        if (!std::isfinite(rr64)) {
          R.status = fail(L, DWF_ERR_NAN, "cg_multi: non-finite true residual");
          R.active = false;
        } else if (rr64 <= R.tol2) {
          R.active = false;
        } else if (last) {
          R.status = DWF_ERR_NOT_CONVERGED;
          R.active = false;
        } else {
          DWF_TRY(restart(M, r, r64));
          R.maxrr = rr64;
        }
      } else if (rr > R.maxrr) {
        R.maxrr = rr;
      }
    }
  }
  return DWF_OK;
}

// x_r = the reconstructed whole-lattice solution; checks the full FP64 residual
// and, should it miss the tolerance, continues with the single-RHS solver.
dwf_status finish(Multi& M, const void* const* b, void* const* x) {
  dwf_lattice* L = M.L;
  Field be, bo, xe, xo, ye, yo;
  DWF_TRY(field_alloc(L, "io.be", DWF_F64, &be));
  DWF_TRY(field_alloc(L, "io.bo", DWF_F64, &bo));
  DWF_TRY(field_alloc(L, "io.xe", DWF_F64, &xe));
  DWF_TRY(field_alloc(L, "io.xo", DWF_F64, &xo));
  DWF_TRY(field_alloc(L, "solve.ye", DWF_F64, &ye));
  DWF_TRY(field_alloc(L, "solve.yo", DWF_F64, &yo));
  for (size_t r = 0; r < M.R.size(); ++r) {
    Rhs& R = M.R[r];
    if (R.zero) {
      DWF_CUDA(L, cudaMemsetAsync(x[r], 0, (size_t)2 * L->Vh * L->Ls * 12 * 2 * sizeof(double), L->stream));
      R.st.true_resid = 0.0;
      continue;
    }
    if (R.status != DWF_OK && R.status != DWF_ERR_NOT_CONVERGED) continue;
    DWF_TRY(launch_pack(L, b[r], 0, be));
    DWF_TRY(launch_pack(L, b[r], 1, bo));
    DWF_TRY(launch_sop(L, R.xt, xe, R.ops, SOps::BINV, 1.0, nullptr, 0.0));
    HopCall c;
    c.out_parity = 1;
    c.in = R.xt;
    c.out = xo;
    c.x = bo;
    c.has_x = true;
    c.eout = SOps::AINV;
    c.scale = 0.5;
    c.ops = R.ops;
    DWF_TRY(launch_hop(L, c));
    DWF_TRY(apply_D(L, R.ops, false, xe, xo, ye, yo));
    R.st.hop_calls += 3;
    DWF_TRY(blas_axpby(L, 1.0, be, -1.0, ye));
    DWF_TRY(blas_axpby(L, 1.0, bo, -1.0, yo));
    int nb = 0;
    DWF_TRY(blas_norm2(L, ye, R.pr, &nb));
    DWF_TRY(blas_sum(L, R.pr, nb, M.sc((int)r, M_TMP0)));
    DWF_TRY(blas_norm2(L, yo, R.pr, &nb));
    DWF_TRY(blas_sum(L, R.pr, nb, M.sc((int)r, M_TMP1)));
    DWF_TRY(fetch(L));
    double res = std::sqrt(M.hs((int)r, M_TMP0) + M.hs((int)r, M_TMP1)) / R.bnorm;
    if (R.status == DWF_OK && res > M.prm.tol) {
      // rounding in the reconstruction left the full residual above the
      // target: continue from this solution with the single-RHS solver
      dwf_cg_params p = M.prm;
      p.max_iter = M.prm.max_iter - R.st.iters > 1 ? M.prm.max_iter - R.st.iters : 1;
      dwf_stats s2{};
      R.status = solve_eo(L, R.m, be, bo, xe, xo, p, &s2, &res);
      R.st.iters += s2.iters;
      R.st.reliable_updates += s2.reliable_updates;
      R.st.hop_calls += s2.hop_calls;
      if (R.status != DWF_OK && R.status != DWF_ERR_NOT_CONVERGED) return R.status;
    }
    R.st.true_resid = res;
    DWF_TRY(launch_unpack(L, xe, 0, x[r], false));
    DWF_TRY(launch_unpack(L, xo, 1, x[r], false));
  }
  DWF_CUDA(L, cudaStreamSynchronize(L->stream));
  return DWF_OK;
}

}  // namespace

}  // namespace dwf

using namespace dwf;

extern "C" dwf_status dwf_cg_multi(dwf_lattice_t L, int nrhs, const double* masses, const void* const* b,
                                   void* const* x, const dwf_cg_params* prm, const dwf_multi_options* opt,
                                   dwf_stats* stats, dwf_multi_info* info) {
  if (!L || !masses || !b || !x || !prm) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: null argument");
  if (nrhs < 1 || nrhs > DWF_MAX_RHS) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: nrhs out of range");
  if (!(prm->tol > 0.0) || prm->max_iter < 1 || prm->inner < DWF_F64 || prm->inner > DWF_F16 ||
      !(prm->delta > 0.0 && prm->delta < 1.0))
    return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: bad solver parameters");
  for (int r = 0; r < nrhs; ++r) {
    if (!b[r] || !x[r]) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: null spinor");
    if (!std::isfinite(masses[r])) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: non-finite mass");
    for (int q = 0; q < nrhs; ++q)
      if (x[r] == b[q] || (q != r && (x[r] == x[q] || masses[r] == masses[q])))
        return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: aliased spinors or repeated mass");
  }
  if (!L->gauge_set) return fail(L, DWF_ERR_INVALID_ARG, "dwf_cg_multi: gauge field not set");
  const auto t0 = std::chrono::steady_clock::now();
  const long long l0 = L->launches;
  Multi M;
  M.L = L;
  M.prm = *prm;
  M.mixed = prm->inner != DWF_F64;
  M.graphs = opt ? opt->use_graph != 0 : true;
  M.autotune = opt ? opt->autotune != 0 : true;
  M.R.resize(nrhs);
  dwf_status s = DWF_OK;
  {
    StreamSwap swap;
    if (M.graphs) DWF_TRY(swap.begin(L));
    s = setup(M, masses, b, x);
    if (s == DWF_OK) s = solve_all(M);
    if (s == DWF_OK) s = finish(M, b, x);
  }
  if (s != DWF_OK) return s;
  const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  dwf_status worst = DWF_OK;
  for (int r = 0; r < nrhs; ++r) {
    Rhs& R = M.R[r];
    R.st.op_count = (long long)R.st.iters * L->Ls;
    R.st.seconds = secs;
    R.st.launches = L->launches - l0;
    if (stats) stats[r] = R.st;
    if (R.status != DWF_OK && worst == DWF_OK) worst = R.status;
  }
  if (info) {
    info->batch = M.first_batch;
    info->ctas_per_sm = M.first_ctas;
    info->tune_seconds = M.tune_seconds;
    info->graphs = (int)M.exec_launches.size();
    info->replays = M.replays;
    info->iterations = M.iterations;
    info->seconds = secs;
    info->launches = L->launches - l0;
  }
  if (worst == DWF_ERR_NOT_CONVERGED) return fail(L, worst, "dwf_cg_multi: max_iter reached for some right-hand side");
  if (worst != DWF_OK) return worst;
  return DWF_OK;
}
