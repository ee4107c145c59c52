/*
 * dwf.h -- C ABI of the GB300 (sm_103a) domain-wall fermion library.
 *
 * Paper: H. Yin and R. D. Mawhinney, "Improving DWF Simulations: the Force
 * Gradient Integrator and the Moebius Accelerated DWF Solver", Lattice 2011.
 *
 * Operator (Sec. 4, Eq. dirac_eq names D_DW(m); its form is the standard one):
 *   D(m) = D_W (b + c Q(m)) + 1 - Q(m)            (Shamir: b = 1, c = 0)
 *   D_W  = (4 - M5) - 1/2 sum_mu [ (1 - g_mu) U_mu(n) d_{n+mu} + (1 + g_mu) U_mu(n-mu)^+ d_{n-mu} ]
 *   Q(m) psi_s = P- psi_{s+1} + P+ psi_{s-1},  psi_{Ls} := -m psi_0,  psi_{-1} := -m psi_{Ls-1}
 * with hermitian Euclidean gamma matrices in the chiral basis,
 * gamma5 = g1 g2 g3 g4 = diag(1,1,-1,-1), P+- = (1 +- gamma5)/2:
 *   g_k = [[0, -i sigma_k], [i sigma_k, 0]] (k = x,y,z),  g_t = [[0, 1], [1, 0]].
 *
 * Boundary layouts (all complex numbers are interleaved re, im; C order):
 *   gauge field : complex128 [4][T][Z][Y][X][3][3]    (mu = x, y, z, t; U[a][b] row-major)
 *   5D spinor   : complex128 [Ls][T][Z][Y][X][4][3]   (spin, colour)
 *   su(3) field : float64    [4][T][Z][Y][X][8]       (components X^j on T_j = i lambda_j / 2)
 * The lattice site parity is (x + y + z + t) mod 2; "even" is parity 0.
 *
 * Ownership: every field pointer is a DEVICE pointer owned by the caller and
 * must stay valid for the duration of the call.  The library owns only the
 * lattice handle, its internal (packed) copies of the gauge field and its
 * workspace, all released by dwf_destroy_lattice.  Work is issued on the
 * stream given at creation; calls return after the stream has finished the
 * call's work unless stated otherwise.
 *
 * Errors: every call returns a dwf_status and never aborts.  The text of the
 * last error on a handle is returned by dwf_last_error(handle);
 * dwf_last_error(NULL) gives the last error of a call that had no valid
 * handle (for example a failed dwf_create_lattice).
 */
#ifndef DWF_H
#define DWF_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DWF_OK = 0,
  DWF_ERR_INVALID_ARG = 1,   /* bad pointer, size, parameter or precision */
  DWF_ERR_CUDA = 2,          /* a CUDA runtime call failed; text has the CUDA error */
  DWF_ERR_OOM = 3,           /* the library could not allocate its workspace */
  DWF_ERR_NOT_CONVERGED = 4, /* solver hit max_iter; stats and x hold the last iterate */
  DWF_ERR_NAN = 5,           /* a NaN or Inf appeared in a solver norm */
  DWF_ERR_TIMEOUT = 6        /* a bounded device wait gave up */
} dwf_status;

typedef enum { DWF_F64 = 0, DWF_F32 = 1, DWF_F16 = 2 } dwf_prec;

typedef struct {
  int dims[4];  /* X, Y, Z, T: each even and >= 2 */
  int Ls;       /* fifth-dimension extent, 1 <= Ls <= 64 */
  double M5;    /* domain-wall height (1.8 in all of the paper's setups) */
  double b, c;  /* Moebius parameters; Shamir DWF is b = 1, c = 0 */
  int bc_t;     /* +1 periodic or -1 antiperiodic in t (x, y, z are periodic) */
} dwf_params;

typedef struct dwf_lattice* dwf_lattice_t;

/* Create a lattice handle.  `stream` is a cudaStream_t (NULL = legacy default
 * stream) on which all of the handle's work is issued.  Sec. 4 (D_DW at Ls,
 * D'_DW at Ls' are two handles on the same gauge field). */
dwf_status dwf_create_lattice(const dwf_params* params, void* stream, dwf_lattice_t* out);
dwf_status dwf_destroy_lattice(dwf_lattice_t h);
const char* dwf_last_error(dwf_lattice_t h);

/* Upload the gauge field (device complex128 boundary layout).  The library
 * keeps packed FP64/FP32/FP16 copies with the t boundary phase folded in. */
dwf_status dwf_set_gauge(dwf_lattice_t h, const void* U);

/* Full 5D operator on whole-lattice spinors (Sec. 4, Eq. dirac_eq):
 * out = D(m) in, D(m)^+ in, D(m)^+ D(m) in.  `in` and `out` must not alias. */
dwf_status dwf_apply_M(dwf_lattice_t h, double m, const void* in, void* out);
dwf_status dwf_apply_Mdag(dwf_lattice_t h, double m, const void* in, void* out);
dwf_status dwf_apply_MdagM(dwf_lattice_t h, double m, const void* in, void* out);

/* Even-odd Schur operator on even sites: M_pc = A - M_eo A^-1 M_oe with
 * A = (4-M5)(b+cQ) + 1 - Q and M_eo = -1/2 D_hop^{eo} (b+cQ); dag != 0 gives
 * M_pc^+.  Whole-lattice boundary layout: odd sites of `in` are ignored, odd
 * sites of `out` are set to zero. */
dwf_status dwf_apply_Mpc(dwf_lattice_t h, double m, int dag, const void* in, void* out);

/* Solver controls and statistics. */
typedef struct {
  double tol;            /* target |b - D(m) x| / |b| (full, unpreconditioned system) */
  int max_iter;          /* iteration cap over all inner iterations */
  dwf_prec inner;        /* DWF_F64: plain FP64 CG; DWF_F32/F16: mixed with FP64 reliable updates */
  double delta;          /* reliable-update trigger: |r| < delta * max|r| since the last update */
  int check_every;       /* iterations between host convergence polls (>= 1) */
} dwf_cg_params;

typedef struct {
  int iters;             /* CG iterations (each applies M_pc and M_pc^+ once) */
  int reliable_updates;  /* FP64 residual recomputations */
  long long hop_calls;   /* 4D Wilson hop applications, each over all Ls slices */
  long long op_count;    /* the paper's "Op. count" (Table 1): CG iterations x Ls, summed over solves */
  double true_resid;     /* |b - D(m) x| / |b| in FP64 at exit */
  double seconds;        /* wall time of the call */
  long long launches;    /* CUDA kernels the call launched */
} dwf_stats;

/* Solve D(m) x = b (Sec. 4, Eq. dirac_eq) by even-odd CG on the normal
 * equations of M_pc.  `x` holds the initial guess on entry (zeros for a cold
 * start) and the solution on exit.  Returns DWF_ERR_NOT_CONVERGED with the
 * best iterate if max_iter is reached, DWF_ERR_NAN on a non-finite norm. */
dwf_status dwf_cg(dwf_lattice_t h, double m, const void* b, void* x,
                  const dwf_cg_params* params, dwf_stats* stats);

/* Multi-right-hand-side solve for a Hasenbusch mass ladder (Sec. 3: the
 * determinant ratios over the masses m + mu_i of the splitting put one Dirac
 * equation per mass on the same gauge field): D(m_r) x_r = b_r for
 * r = 0 .. nrhs-1, each by the even-odd CG of dwf_cg (same tolerance, inner
 * precision and FP64 reliable updates, per right-hand side), iterated in
 * lockstep so that each Wilson hop step of an iteration covers every
 * unconverged right-hand side in as few launches as the kernel takes (the
 * links of a 4D site are read once for all of them; each right-hand side's
 * fifth-dimension operators use its own mass).  Converged right-hand sides
 * leave the batch.  masses[nrhs] must be distinct; b[nrhs] and x[nrhs] are
 * host arrays of device pointers to whole-lattice boundary-layout spinors
 * (x: initial guess in, solution out; no x may alias a b or another x).
 * stats[nrhs] (may be NULL) receives per-right-hand-side statistics (seconds
 * and launches are those of the whole call).  opt may be NULL (graphs and
 * autotuning on).  Work runs on the handle's stream; with graphs on it is
 * recorded and replayed on a private stream joined to it on both ends.
 * Returns DWF_ERR_NOT_CONVERGED if some right-hand side hit max_iter (the
 * others are solved), DWF_ERR_NAN on a non-finite norm. */
#define DWF_MAX_RHS 16
typedef struct {
  int use_graph;  /* 1: record one iteration of a batch as a CUDA graph and replay it */
  int autotune;   /* 1: pick launch shapes by timing candidates (cached per process,
                     and in the file named by DWF_TUNE_CACHE if set); 0: defaults */
} dwf_multi_options;
typedef struct {
  int batch;            /* right-hand sides per hop launch for the largest batch */
  int ctas_per_sm;      /* CTAs per SM for that launch (0: all that fit) */
  double tune_seconds;  /* time this call spent autotuning */
  int graphs;           /* CUDA graphs recorded */
  long long replays;    /* graph launches */
  int iterations;       /* iterations of the joint loop */
  double seconds;       /* wall time of the call */
  long long launches;   /* kernels launched (graph replays count their kernels) */
} dwf_multi_info;
dwf_status dwf_cg_multi(dwf_lattice_t h, int nrhs, const double* masses, const void* const* b,
                        void* const* x, const dwf_cg_params* params, const dwf_multi_options* opt,
                        dwf_stats* stats, dwf_multi_info* info);

/* Moebius-accelerated DWF solve (Sec. 4, the four-step algorithm with
 * Eqs. trans_5d_4d_source, mob_eq_4d, mob_eq_5d and recon; Sec. 5, defect
 * correction; Table 1).  `outer` is the Shamir lattice (b = 1, c = 0) of
 * extent Ls on which D_DW(m) x = b is solved; `inner` is a Moebius lattice
 * with the same 4D extents and gauge field (set on both handles) and extent
 * Ls' (usually Ls' < Ls).  Each of the n_dc defect-correction passes does two
 * Pauli-Villars solves D_DW(1) (tolerance tol_pv) and one Moebius solve
 * D'_DW(m) (tol_mob) on the current residual and adds the reconstructed 5D
 * guess to x; a final DWF solve to tol_final starts from that guess.  All
 * solves use CG on the normal equations at the `inner` precision with FP64
 * reliable updates; residuals and the accumulated solution stay FP64.
 * With inner != DWF_F64, tol_pv >= 1e-5 and tol_mob >= 1e-4 the passes'
 * Pauli-Villars and Moebius solves, and the operator applications that make
 * their sources, compute their FP64-field Wilson hops in FP32 (FP32 links;
 * inputs truncated to FP32): their results need only those tolerances, and
 * GB300 runs FP64 arithmetic at ~1/70 of its FP32 rate.  The residual
 * b - D x between passes, the final solve and x stay FP64.
 * `x` need not be initialised; b and x are whole-lattice boundary-layout
 * device spinors of the outer lattice.  Work runs on the outer handle's
 * stream.  Returns DWF_ERR_NOT_CONVERGED if the final solve hits max_iter
 * (an inexact intermediate solve is tolerated and visible in the stats). */
#define MADWF_MAX_PASSES 16
typedef struct {
  int n_dc;            /* defect-correction passes (3 in the paper's Table 1), 0..16 */
  double tol_pv;       /* relative residual of the Pauli-Villars solves */
  double tol_mob;      /* relative residual of the Moebius solves */
  double tol_final;    /* target |b - D(m) x| / |b| of the final DWF solve */
  dwf_prec inner;      /* precision of the inner CG iterations */
  int max_iter;        /* iteration cap per solve */
  double delta;        /* reliable-update trigger of every solve; with DWF_F32 the Pauli-Villars
                          and Moebius solves use min(delta, max(sqrt(their tolerance), 1e-3)) */
  int check_every;     /* host convergence polls */
} madwf_params;

typedef struct {
  dwf_stats total;     /* sums over all solves; total.true_resid is the result's */
  dwf_stats pv;        /* the 2 n_dc Pauli-Villars solves (op_count in units of Ls) */
  dwf_stats mobius;    /* the n_dc Moebius solves (op_count in units of Ls') */
  dwf_stats final_cg;  /* the final warm-started DWF solve */
  int passes;          /* defect-correction passes done */
  double pass_resid[MADWF_MAX_PASSES]; /* |b - D x| / |b| after each pass (the last one in FP32
                                          arithmetic when the passes use it and it is >= 1e-5) */
} madwf_stats;

dwf_status madwf_solve(dwf_lattice_t outer, dwf_lattice_t inner, double m, const void* b, void* x,
                       const madwf_params* params, madwf_stats* stats);

/* Pseudofermion action and fermion force (Sec. 2 and 3).
 *
 * A quotient term (m1, m2) is the Hasenbusch factor det(M1^+ M1)/det(M2^+ M2)
 * of Sec. 3 (m2 = 1: Pauli-Villars denominator), with M = M_pc the even-odd
 * Schur operator of the lattice; its action is
 *   S = phi^+ M2 (M1^+ M1)^-1 M2^+ phi = |M1 X|^2,   X = (M1^+ M1)^-1 M2^+ phi.
 * dwf_force solves for X with CG on the normal equations (parameters `cg`),
 * and writes, summed over the `nterms` terms:
 *   S  (host double, may be NULL): the total action;
 *   F  (device float64 [4][T][Z][Y][X][8], may be NULL): the force components
 *      F^j(n, mu) = e_j S, the derivative of S along U_mu(n) -> exp(h T_j) U_mu(n),
 *      T_j = i lambda_j / 2 (Sec. 2: F^j = e^j(S));
 *   G  (device complex128 [4][T][Z][Y][X][3][3], may be NULL): the complex-
 *      matrix gradient 2 dS / d conj(U) of S as a function of the boundary-
 *      layout links (the convention of torch.autograd for complex inputs).
 * phi[t] are device whole-lattice spinors (only even sites are used).
 * X_io (may be NULL; entries may be NULL): device whole-lattice spinors that
 * hold the initial guess for term t's solve on entry and its solution X on
 * exit (even sites; odd sites set to zero) -- the "force gradient
 * forecasting" of Sec. 2 passes the first solve's X to the second. */
typedef struct {
  double m1, m2;
} dwf_quotient;

dwf_status dwf_force(dwf_lattice_t h, int nterms, const dwf_quotient* terms, const void* const* phi,
                     void* const* X_io, void* F, void* G, double* S, const dwf_cg_params* cg, dwf_stats* stats);

/* Heat-bath pseudofermion of one quotient term (Sec. 3): given eta (device
 * whole-lattice spinor, even sites used; Gaussian in an HMC trajectory's
 * refresh), phi = M2^-+ M1^+ eta (device whole-lattice spinor, written on
 * even sites, odd sites zero), so that the term's action at this gauge field
 * is S = |M1^-+ M2^+ phi|^2 = |eta_e|^2.  One CG solve with M2 on the normal
 * equations (parameters `cg`; stats may be NULL).  eta and phi must not
 * alias. */
dwf_status dwf_heatbath(dwf_lattice_t h, dwf_quotient term, const void* eta, void* phi, const dwf_cg_params* cg,
                        dwf_stats* stats);

/* The action alone: S (host double, required) = sum over the terms of
 * |M1 (M1^+ M1)^-1 M2^+ phi|^2, as dwf_force computes it with F = G = NULL. */
dwf_status dwf_action(dwf_lattice_t h, int nterms, const dwf_quotient* terms, const void* const* phi,
                      const dwf_cg_params* cg, double* S);

/* The force-gradient link update (Sec. 2, Eq. for U'): for every link,
 * U_out = exp(coeff * sum_j X^j T_j) U_in with X float64 [4][T][Z][Y][X][8]
 * and U complex128 boundary layout (U_out may equal U_in).  coeff =
 * -tau^2/24 with X = F gives U' of the force-gradient step; coeff = dt with
 * X = p is the link (Q) update of the integrator. */
dwf_status fgi_link_update(dwf_lattice_t h, const void* X, double coeff, const void* U_in, void* U_out);

/* p += coeff * F on float64 [4][T][Z][Y][X][8] su(3) components (the
 * momentum (P) update). */
dwf_status dwf_momentum_update(dwf_lattice_t h, const void* F, double coeff, void* p);

/* Kinetic energy 1/2 sum (p^j)^2 (FP64). */
dwf_status dwf_kinetic(dwf_lattice_t h, const void* p, double* T);

/* One force-gradient PQPQP step (Sec. 2, Eq. 1, with the two-step
 * implementation of the force-gradient term):
 *   P(tau/6) Q(tau/2) [F = F(U); U' = exp(-tau^2/24 F^j T_j) U; p -= 2/3 tau F(U')] Q(tau/2) P(tau/6)
 * U (device complex128 boundary layout) and p (device float64 components)
 * are updated in place; the handle's gauge field is left set to the new U.
 * With forecast != 0 the solve of F(U') starts from the solutions of F(U).
 * stats->iters sums the CG iterations of the five force evaluations;
 * fg_iters[0] and fg_iters[1] (may be NULL) receive those of F(U) and F(U')
 * in the force-gradient step. */
dwf_status fgi_step(dwf_lattice_t h, int nterms, const dwf_quotient* terms, const void* const* phi, void* U, void* p,
                    double tau, int forecast, const dwf_cg_params* cg, dwf_stats* stats, int* fg_iters);

/* A molecular-dynamics trajectory of nsteps steps of length tau (Sec. 2):
 * DWF_INTEGRATOR_FGI, the force-gradient step of fgi_step,
 *   P(tau/6) Q(tau/2) [F(U); U' = exp(-tau^2/24 F^j T_j) U; p -= 2/3 tau F(U')] Q(tau/2) P(tau/6),
 * or DWF_INTEGRATOR_OMELYAN, the second-order minimum-norm step the paper
 * compares it with (Omelyan, Mryglod and Folk 2003, lambda = 0.1931833275037836),
 *   P(lambda tau) Q(tau/2) P((1 - 2 lambda) tau) Q(tau/2) P(lambda tau).
 * The closing momentum update of a step and the opening one of the next act
 * at the same U and are applied as one, so a trajectory evaluates the force
 * 3 nsteps + 1 (FGI) or 2 nsteps + 1 (Omelyan) times.  With forecast != 0 the
 * FGI solve at U' starts from the solutions at U (Sec. 2).  U (device
 * complex128 boundary layout) and p (device float64 [4][T][Z][Y][X][8]) are
 * updated in place and the handle's gauge field is left set to the final U.
 * H0 and H1 (may be NULL) receive H = 1/2 sum (p^j)^2 + S at the start and the
 * end in FP64; S comes from the first and the last force evaluation, so they
 * cost no extra solve.  stats (may be NULL) sums the solves; nforce (may be
 * NULL) receives the number of force evaluations. */
typedef enum { DWF_INTEGRATOR_FGI = 0, DWF_INTEGRATOR_OMELYAN = 1 } dwf_integrator;
dwf_status dwf_md_trajectory(dwf_lattice_t h, int nterms, const dwf_quotient* terms, const void* const* phi, void* U,
                             void* p, double tau, int nsteps, dwf_integrator integ, int forecast,
                             const dwf_cg_params* cg, double* H0, double* H1, dwf_stats* stats, int* nforce);

/* dwf_apply_Mpc without any device allocation (the paper has no counterpart;
 * this serves callers that must not allocate while they run: code whose
 * allocator owns all device memory, loops that may not stall on the driver).  Same operator, arguments and boundary
 * layout as dwf_apply_Mpc.  The handle must already exist (creation and
 * dwf_set_gauge allocate; this call does not).
 *
 * Scratch: one file-scope device array of DWF_NOALLOC_SCRATCH_BYTES bytes,
 * present on every GPU that loads the library until the process exits.  The
 * call needs 4 FP64 half-lattice fields (each Vh * 12 * ceil(Ls/2) * 32 bytes,
 * rounded up to 256); larger lattices are rejected with DWF_ERR_INVALID_ARG
 * and a message giving both sizes.  Möbius parameters whose fifth-dimension
 * inverse would need the dense fallback are rejected the same way.
 * The first call on a device looks up the array's device address there
 * (cudaGetSymbolAddress, once per device, with that device current); make
 * that first call before any stream capture.  All calls on a device share
 * the array and it keeps the last call's contents (every word a call reads
 * is written earlier in the same call), so calls that overlap on the GPU --
 * on different streams or handles at the same time -- race.  Kernel timing
 * (dwf_set_kernel_timing) is suspended during the call. */
#define DWF_NOALLOC_SCRATCH_BYTES (32u << 20)
dwf_status dwf_apply_Mpc_noalloc(dwf_lattice_t h, double m, int dag, const void* in, void* out);

/* Arithmetic of the Wilson hops on FP64 fields (no counterpart in the
 * paper): mode 0 (the default) FP64; mode 1 FP32 (FP32 links, inputs
 * truncated to FP32, results widened exactly to FP64), for every FP64-field
 * hop of the handle -- the dwf_apply_* operators, the FP64 steps of every
 * solve.  A test and experimentation switch: madwf_solve uses the same
 * arithmetic for its passes by itself (see there).  Errors:
 * DWF_ERR_INVALID_ARG for a null handle or another mode. */
dwf_status dwf_set_fp64_arithmetic(dwf_lattice_t h, int mode);

/* Page-locked HOST memory for the host side of copies to and from the GPU
 * (the paper has no counterpart): bytes (> 0) of zeroed host memory, mapped
 * on a huge-page boundary, advised for transparent huge pages and
 * registered with the CUDA driver (cudaHostRegister).  Each copy between the
 * GPU and page-locked memory translates the host pages it touches; with the
 * host's base pages a multi-GB buffer is tens of thousands of pages, and the
 * first copy after other GPU work runs several times slower while their
 * translations are fetched again, which huge pages avoid.  Where the host
 * kernel has transparent huge pages off the memory is still page-locked,
 * without that gain.  *ptr receives the buffer (NULL on error); the caller
 * owns it and releases it with dwf_host_free.  Errors (dwf_last_error(NULL)):
 * DWF_ERR_INVALID_ARG for a NULL ptr or zero bytes, DWF_ERR_OOM if the
 * mapping fails, DWF_ERR_CUDA if registration fails (e.g. no GPU).
 * dwf_host_free(NULL) is a no-op; a pointer that dwf_host_alloc did not
 * return gives DWF_ERR_INVALID_ARG. */
dwf_status dwf_host_alloc(size_t bytes, void** ptr);
dwf_status dwf_host_free(void* ptr);

/* Instrumentation (no counterpart in the paper; used to measure the Wilson
 * hop kernels against the HBM roofline).  With timing enabled every hop
 * launch on the handle's stream is bracketed by CUDA events.
 * dwf_set_kernel_timing(h, 1) enables and resets the accumulators, 0 disables.
 * dwf_get_kernel_time synchronises the stream and returns, for the hop
 * kernels of precision `prec` since the last reset, the summed device time
 * in milliseconds, the number of launches and the summed algorithmic bytes
 * (spinors read and written once, links read once per 4D site).
 * dwf_get_launch_count returns the number of kernels the handle has
 * launched since it was created. */
dwf_status dwf_set_kernel_timing(dwf_lattice_t h, int enable);
dwf_status dwf_get_kernel_time(dwf_lattice_t h, dwf_prec prec, double* ms, long long* launches, double* bytes);
dwf_status dwf_get_launch_count(dwf_lattice_t h, long long* launches);

/* The even-odd Schur operator M_pc (or M_pc^+ if dag != 0) of dwf_apply_Mpc
 * (Sec. 4; same operator, mass, boundary layout and result layout: odd sites
 * of `out` set to zero), evaluated with its fields stored at precision
 * `prec` through the launches the solvers use for their inner iterations:
 * M_pc = M~ B with M~ the right-preconditioned operator of dwf_cg (two
 * Wilson hops with fused fifth-dimension epilogues).  DWF_F64 computes in
 * FP64; DWF_F32 and DWF_F16 (FP16 storage with one FP32 scale per site and
 * slice) compute in FP32, so the result carries the rounding of that storage
 * (about 1e-7 and 1e-3 relative).  The input is rounded to `prec` on entry.
 * Returns DWF_ERR_TIMEOUT if a bounded device wait of the hop kernel gave up
 * (see dwf_set_wait_limit); the handle stays usable. */
dwf_status dwf_apply_Mpc_prec(dwf_lattice_t h, double m, int dag, dwf_prec prec, const void* in, void* out);

/* Instrumentation of the bounded device waits (no counterpart in the paper).
 * The FP32/FP16 hop kernel waits for its asynchronous shared-memory copies
 * on mbarriers; each wait gives up after a number of polls (default 2^22),
 * sets the handle's error flag -- reported by the next synchronising call
 * as DWF_ERR_TIMEOUT -- and the kernel then waits, with the default limit,
 * for the copies it has already issued and returns.  This call sets the
 * number of polls of the consumer waits on the handle's later launches
 * (polls < 0 restores the default; 0 makes every consumer wait give up at
 * once, which tests the error path without any stalled copy). */
dwf_status dwf_set_wait_limit(dwf_lattice_t h, long long polls);

#ifdef __cplusplus
}
#endif

#endif /* DWF_H */
