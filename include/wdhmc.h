/*
 * wdhmc.h -- C ABI of the GB300 Wilson-fermion PF/Hasenbusch HMC hot path.
 *
 * The method (Haar, Kamleh, Zanotti, Nakamura, "Improving polynomial-filtered
 * Hybrid Monte Carlo with Hasenbusch", INPC 2016):
 *   Section 2   lattice action S = S_G + S_F; momenta P with
 *               H = sum tr P^2 + S; steps T[eps]: U -> exp(i eps P) U and
 *               S[eps]: P -> P - eps F; Metropolis test; two-flavour fermion
 *               action S_F = phi^dag (M^dag M)^-1 phi and its force; mass
 *               preconditioning (Hasenbusch) and polynomial filtering.
 *   Section 3   Wilson fermions with hopping parameter kappa and even-odd
 *               preconditioning; cost in multiplications by K (N_mat);
 *               leapfrog, nested and generalised multi-scale integrators.
 *   Section 4   PF-MP and three-filter actions.
 *
 * Conventions for every call
 *   - Every pointer to field data is DEVICE memory owned by the caller unless
 *     the comment says "host".  The library never frees caller memory.
 *   - The library allocates device memory in wd_context_create (gauge field
 *     copies, reduction scratch) and, the first time an operation needs more
 *     half-lattice workspace vectors than the context holds, grows the
 *     context's pool (cudaMalloc); the pool is kept until
 *     wd_context_destroy, so repeated calls allocate nothing.
 *   - Work is ordered on the stream given to wd_context_create.  Calls that
 *     return a scalar to a host pointer synchronise that stream.
 *   - Return value: WD_OK or an error code; wd_last_error() gives a message.
 *     Arguments are validated before any launch; no error aborts the process.
 *
 * Lattice: dims[4] = {Lx, Ly, Lz, Lt}, every extent even and >= 2.  Site
 * (x,y,z,t) has parity (x+y+z+t) mod 2 and checkerboard index
 * cb = (x + Lx (y + Ly (z + Lz t))) / 2 in [0, Vh), Vh = V/2.  Fermions are
 * periodic in space and antiperiodic in time; links periodic.  Wilson r = 1,
 * M = 1 - kappa D, D = sum_mu [(1-g_mu) U_mu(x) psi(x+mu)
 * + (1+g_mu) U_mu(x-mu)^dag psi(x-mu)], DeGrand-Rossi gamma basis.
 *
 * Field layouts (all FP64):
 *   lexicographic spinor  complex128 [Lt][Lz][Ly][Lx][4 spin][3 colour]
 *   lexicographic gauge   complex128 [Lt][Lz][Ly][Lx][4 mu][3][3]
 *   lexicographic algebra float64    [Lt][Lz][Ly][Lx][4 mu][8]
 *   half spinor (EO)      double2 [12][Vh]: component j = 3*spin + colour of
 *                         the sites of one parity, structure-of-arrays
 *   algebra field (EO)    double [4 mu][2 parity][8][Vh]: coordinates
 *                         X_a of X = sum_a X_a T_a, T_a = lambda_a / 2
 * Momenta and forces are algebra fields; F_a(x,mu) = dS/dw for
 * U_mu(x) -> exp(i w T_a) U_mu(x).
 */
#ifndef WDHMC_H
#define WDHMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wd_ctx wd_ctx;

enum wd_status_code {
  WD_OK = 0,
  WD_ERR_ARG = 1,      /* invalid argument (null, size, value); nothing launched */
  WD_ERR_CUDA = 2,     /* a CUDA call failed */
  WD_ERR_NOCONV = 3,   /* solver reached maxiter before the tolerance */
  WD_ERR_NAN = 4,      /* non-finite value met in a solver */
  WD_ERR_STATE = 5,    /* call made before the state it needs (e.g. no gauge field) */
  WD_ERR_TIMEOUT = 6   /* a bounded device-side wait expired (see wd_kernel_status) */
};

/* Arithmetic used inside an operator application or for the bulk of a solve.
 * WD_DF (operator calls wd_hop / wd_apply / mdagm_apply only): double-float,
 * two FP32 words per real with error-free FP32 arithmetic, about 48 bits. */
enum wd_prec { WD_F64 = 0, WD_F32 = 1, WD_F16 = 2, WD_BF16 = 3, WD_DF = 4 };

/* Storage of the low-precision links: 18 reals, or 12 with the third row
 * rebuilt as (r0 x r1)^* (SU(3)); the antiperiodic sign is never folded in. */
enum wd_recon { WD_RECON_18 = 0, WD_RECON_12 = 1 };

/* Kernel of the FP32/FP16/BF16 hopping stencil with 12-real links (Section 3.1;
 * a kernel choice, the arithmetic is the same):
 *   WD_STENCIL_THREAD  (default) one thread per output site, each thread
 *                      copying its own links two directions ahead into shared
 *                      memory (cp.async) and its next neighbour spinor into
 *                      registers;
 *   WD_STENCIL_TILE    one persistent block per SM; a producer warp copies the
 *                      links and neighbour-spinor faces of 512-site tiles, one
 *                      direction at a time, into a ring of shared-memory stages
 *                      with bulk asynchronous copies (cp.async.bulk, mbarrier
 *                      completion); 512 consumer threads compute from shared
 *                      memory.  Used where the lattice allows it (Lx/2 a
 *                      multiple of 4 that divides 512 in at most 32 x rows, Vh a
 *                      multiple of 512), elsewhere the thread kernel runs.  At
 *                      32^3 x 64 it takes 0.70 ms per FP32 K_hat against 0.54 ms
 *                      for the thread kernel. */
enum wd_stencil { WD_STENCIL_THREAD = 0, WD_STENCIL_TILE = 1 };

/* Pseudofermion term kinds (Section 2; Section 4.1):
 *   PLAIN       S = phi^dag K^-1 phi,          K = K_hat(kappa)
 *   HASENBUSCH  S = phi^dag M_h K^-1 M_h^dag phi,  M_h = M_hat(kappa_h), kappa_h < kappa
 *               (the Hermitian reading of the printed phi^dag J K^-1 phi)
 *   POLY        S = phi^dag P(K) phi
 *   FILTERED    S = phi^dag [P(K) K]^-1 phi
 *   RATIO       S = phi^dag Q(K) phi, Q = P / P_lo (Section 3.3, the middle term of
 *               the two-filter action); Q is a polynomial when (n_lo + 1) divides
 *               (n + 1) on the same [eps, lam]: its roots are those of P whose index k
 *               is not a multiple of (n + 1) / (n_lo + 1), its scale c / c_lo.
 * Composite actions: 1MP, 2MP, PF-MP, 1PF-2MP from PLAIN / HASENBUSCH / POLY /
 * FILTERED; 2PF = [POLY(P_1), RATIO(P_2 / P_1), FILTERED(P_2)]; 2PF-1MP adds a
 * HASENBUSCH term (Section 4.2). */
enum wd_term_kind { WD_TERM_PLAIN = 0, WD_TERM_HASENBUSCH = 1, WD_TERM_POLY = 2,
                    WD_TERM_FILTERED = 3, WD_TERM_RATIO = 4 };

/* Chebyshev filter P of even degree n approximating 1/x on [eps, lam]
 * (Section 2: "Chebyshev polynomials ... order p").  Reading: the minimax
 * relative-error polynomial, x P(x) = 1 - T_{n+1}((mu-x)/nu) / T_{n+1}(mu/nu),
 * mu = (lam+eps)/2, nu = (lam-eps)/2. */
typedef struct { int n; double eps; double lam; } wd_poly;

typedef struct {
  int kind;          /* enum wd_term_kind */
  double kappa;      /* operator K = K_hat(kappa) */
  double kappa_h;    /* heavy kappa of a HASENBUSCH term */
  wd_poly poly;      /* POLY / FILTERED; the numerator P of RATIO */
  wd_poly poly_lo;   /* RATIO: the denominator P_lo */
} wd_term;

typedef struct {
  double tol;        /* stop on the FP64 true residual |b - A x| / |b| <= tol */
  int maxiter;       /* total iterations allowed */
  int prec;          /* enum wd_prec: arithmetic of the bulk operator */
  double delta;      /* reliable update when |r| drops by this factor (mixed) */
  int check_every;   /* iterations queued between host checks (>= 1) */
} wd_cg_params;

typedef struct {
  int iters;                 /* CG iterations */
  int reliable_updates;      /* FP64 residual recomputations (mixed precision) */
  long long n_mat;           /* K_hat applications, any precision */
  double true_rel_resid;     /* FP64 |b - A x| / |b| at return */
} wd_cg_info;

/* ---- context, fields ------------------------------------------------------ */

/* Create a context for one lattice (Section 3.1: the lattice of the Wilson
 * action; extents even for the even-odd split) on the current device; stream
 * may be NULL (legacy default stream) or a cudaStream_t.  Allocates the link
 * copies and reduction scratch; *out = NULL and WD_ERR_ARG on odd or < 2
 * extents, WD_ERR_CUDA when an allocation fails. */
int wd_context_create(const int dims[4], void* stream, wd_ctx** out);
/* Synchronise the context's stream and free everything it allocated (no
 * counterpart in the paper).  NULL is accepted. */
int wd_context_destroy(wd_ctx* ctx);
/* Message of the last error on the calling thread (static storage; no
 * counterpart in the paper). */
const char* wd_last_error(void);
/* Low-precision link storage (enum wd_recon) of the links U_mu(x) of the Wilson
 * action (Section 3.1); a storage choice, takes effect at the next load. */
int wd_set_recon(wd_ctx* ctx, int recon);
/* Arithmetic of the residual recomputation r = b - A x inside mixed-precision
 * solves of K (Section 2, the iterative solver; the precision is not the
 * paper's, which states none): mode 0 = FP64 (default); mode 1 =
 * double-float, x split into two FP32 words and A applied with error-free
 * FP32 arithmetic (about 48 significant bits, 1e-14 relative; b, x, r, dots
 * stay FP64).  GB300 runs FP64 at 1/60 of its FP32 rate, and a filtered
 * operator's residual costs n+1 K_hat.  Mode 1 allocates a double-float copy
 * of the links (as much as the FP64 copy) on first use. */
int wd_set_residual(wd_ctx* ctx, int mode);
/* Stencil kernel (enum wd_stencil) of the context's later hop launches. */
int wd_set_stencil(wd_ctx* ctx, int stencil);
/* Device error word of the context (no counterpart in the paper): the stencil
 * kernels bound every wait on a shared-memory barrier (about two seconds) and
 * record an expiry here instead of hanging.  Synchronises the context's
 * stream, stores the word in *word (may be NULL), clears it, and returns
 * WD_ERR_TIMEOUT if it was set, else WD_OK.  Solvers report an expiry inside
 * their iterations as WD_ERR_TIMEOUT themselves. */
int wd_kernel_status(wd_ctx* ctx, unsigned* word);
/* Self-test of the bounded device-side wait (no counterpart in the paper):
 * launches one block on the context's stream whose first thread waits on a
 * shared-memory barrier that nothing arrives at, with the bound timeout_ns
 * (1e6 .. 1e10 ns) in place of the stencil's two seconds.  The wait expires,
 * the kernel records it in the device error word and ends, so a following
 * wd_kernel_status returns WD_ERR_TIMEOUT (and clears the word).  Nothing else
 * of the context changes.  WD_ERR_ARG for a bound outside the range. */
int wd_selftest_wait_timeout(wd_ctx* ctx, long long timeout_ns);
/* Launch-shape autotuner of the hop kernels (no counterpart in the paper; on
 * by default): the first launch
 * of each (formats, link storage, dagger, epilogue) outside a queued CG chunk
 * times the candidate block sizes and register caps on the context stream and
 * keeps the fastest for the context's volume.  enable: 1 on, 0 off, -1 leave;
 * *n_tuned (may be NULL) = number of tuned keys. */
int wd_set_autotune(wd_ctx* ctx, int enable, int* n_tuned);
/* The index-th tuned entry (no counterpart in the paper; WD_ERR_ARG when
 * index is out of range): its key (((in*8 + out)*8 + y)*4 + links)*4 +
 * 2 dagger + xpay, with formats as enum wd_prec (y = 7 without epilogue) and
 * links 0 FP64, 1 FP32 18 reals, 2 FP32 12 reals, 3 double-float), the chosen
 * block size and the launch bound (128 or 256) the chosen kernel is compiled for. */
int wd_tune_entry(wd_ctx* ctx, int index, long long* key, int* threads, int* maxt);
/* Volume of the lattice (Section 3.1): out[0] = V, out[1] = Vh = V/2 sites per parity. */
int wd_volume(const wd_ctx* ctx, long long out[2]);

/* Load the gauge field U (Section 2: the links the action and the trajectory
 * act on) from a lexicographic FP64 array (device, V * 72 doubles, read only);
 * builds the FP64 even-odd copy and the FP32 copies used by low-precision
 * operators. */
int wd_gauge_load(wd_ctx* ctx, const double* U_lex);
/* Write the context's current links to a lexicographic FP64 array (device,
 * V * 72 doubles).  WD_ERR_STATE before any load. */
int wd_gauge_store(wd_ctx* ctx, double* U_lex);

/* Lexicographic spinor <-> half spinor of one parity (Section 3.1, even-odd
 * preconditioning splits fields by parity; the other parity is ignored by
 * pack and left untouched by unpack).  WD_ERR_ARG unless parity is 0 or 1. */
int wd_spinor_pack(wd_ctx* ctx, int parity, const double* lex, double* eo);
int wd_spinor_unpack(wd_ctx* ctx, int parity, const double* eo, double* lex);
/* Lexicographic algebra field <-> EO algebra field (Section 2: momenta P and
 * forces F live on the links, one su(3) element each). */
int wd_algebra_pack(wd_ctx* ctx, const double* lex, double* eo);
int wd_algebra_unpack(wd_ctx* ctx, const double* eo, double* lex);

/* ---- operators (Section 3.1: Wilson, even-odd) ------------------------------ */

/* out = D_{out_parity <- 1-out_parity} in (dagger: D^dag), half spinors: the
 * hopping term of the Wilson matrix M = 1 - kappa D (Section 3.1), one parity
 * block of the even-odd split.  prec selects the arithmetic: inputs are
 * converted, outputs returned in FP64.  in and out distinct; WD_ERR_STATE
 * before a gauge load. */
int wd_hop(wd_ctx* ctx, int out_parity, int dagger, int prec, const double* in, double* out);
/* out = M_hat in or M_hat^dag in, M_hat = 1 - kappa^2 D_eo D_oe (even sites):
 * the even-odd preconditioned Wilson matrix of Section 3.1, det M = det M_hat. */
int wd_apply(wd_ctx* ctx, double kappa, int dagger, int prec, const double* in, double* out);
/* out = K_hat in, K_hat = M_hat^dag M_hat (Section 2: K = M^dag M; Section 3.1:
 * one multiplication by K is the unit N_mat of the cost); nrhs consecutive half
 * spinors (stride 24*Vh doubles).  One K_hat per right-hand side counts as N_mat. */
int mdagm_apply(wd_ctx* ctx, double kappa, int prec, int nrhs, const double* in, double* out);

/* ---- solvers (Section 2: "iterative solvers (e.g. conjugate gradient)") ----- */

/* Solve A x = b on even sites, A = K_hat(kappa) (Section 2: K inverted by an
 * iterative solver such as CG), or A = K_hat P(K_hat) when filt != NULL (the
 * [P(K) K]^-1 of the filtered action S_PF, Section 2).  x is the initial guess
 * on entry.  Mixed precision (p->prec != WD_F64) runs the bulk in that
 * precision and recomputes the residual in FP64 (reliable updates).
 * WD_ERR_NOCONV at maxiter, WD_ERR_NAN on a non-finite value. */
int cg_solve(wd_ctx* ctx, double kappa, const wd_poly* filt, const double* b, double* x,
             const wd_cg_params* p, wd_cg_info* info);
/* out = P(K_hat(kappa)) in, the polynomial filter P(K) ~ K^-1 of Section 2,
 * by the Chebyshev three-term recurrence (n K_hat).  prec WD_F64 or WD_F32;
 * in and out must differ. */
int poly_filter_apply(wd_ctx* ctx, double kappa, const wd_poly* poly, int prec,
                      const double* in, double* out);

/* ---- actions and forces (Section 2, eq. of the fermion force) --------------- */

/* S of one term for the half spinor phi (Section 2: S_F, the Hasenbusch and
 * filtered terms of S_MP and S_PF; Section 4.1: S_PF-MP; Section 3.3: the
 * ratio term of S_2PF); *S is HOST memory. */
int pf_action(wd_ctx* ctx, const wd_term* term, const double* phi, const wd_cg_params* p,
              double* S);
/* phi such that S(phi) = chi^dag chi for a Gaussian half spinor chi (Section 2:
 * the pseudofermions are drawn from exp(-S)).  chi and phi must differ. */
int pf_heatbath(wd_ctx* ctx, const wd_term* term, const double* chi, const wd_cg_params* p,
                double* phi);
/* F += coef * dS/dw (algebra field): the fermion force of Section 2,
 * -phi^dag K^-1 (dK/dU) K^-1 phi for the two-flavour term and its analogues for
 * the other kinds.  Stores only X = A^-1 psi and Y = M_hat X per term;
 * polynomial intermediates are recomputed from checkpoints. */
int fermion_force(wd_ctx* ctx, const wd_term* term, const double* phi, const wd_cg_params* p,
                  double coef, double* F);
/* pf_action that also returns the vectors the force needs (differentiation
 * without re-solving): X = A^-1 psi (psi = phi, or M_h^dag phi for
 * HASENBUSCH; A = K_hat, or K_hat P(K_hat) for FILTERED) and, for PLAIN and
 * HASENBUSCH, Y = M_hat X.  X and Y are caller half spinors or NULL (not
 * written for POLY and RATIO / not needed). */
int pf_action_xy(wd_ctx* ctx, const wd_term* term, const double* phi, const wd_cg_params* p,
                 double* S, double* X, double* Y);
/* F += coef * dS/dw from the X (and Y) of pf_action_xy: the adjoint of the
 * action without a solve (Section 2, fermion force; only X and Y are kept per
 * term, polynomial-term vectors are recomputed).  Y may be NULL (formed from
 * X); POLY and RATIO need neither.  prec: WD_F64 or WD_F32 arithmetic. */
int fermion_force_xy(wd_ctx* ctx, const wd_term* term, const double* phi, const double* X,
                     const double* Y, int prec, double coef, double* F);
/* Gauge action S_G of Section 2 (named there only; reading: the Wilson plaquette
 * action S_G = beta sum_{x, mu<nu} (1 - Re tr U_p / 3)); *S host. */
int gauge_action(wd_ctx* ctx, double beta, double* S);
/* F += coef * dS_G/dw, the gauge part of the force F = dS/dU of Section 2
 * (staple sum per link); prec WD_F64 or WD_F32. */
int gauge_force(wd_ctx* ctx, double beta, int prec, double coef, double* F);

/* ---- HMC steps (Section 2, eqs. for T-hat and S-hat) ------------------------ */

/* T[eps] of Section 2: U <- exp(i eps P) U on every link, reunitarised, FP64;
 * refreshes the low-precision link copies. */
int step_T(wd_ctx* ctx, const double* P, double eps);
/* S[eps] of Section 2: P <- P - eps F (algebra fields, FP64). */
int step_S(wd_ctx* ctx, double* P, const double* F, double eps);
/* The kinetic term of H = sum tr P^2 + S (Section 2): sum tr P^2 =
 * (1/2) sum_a P_a^2, FP64; *out host. */
int kinetic_energy(wd_ctx* ctx, const double* P, double* out);
/* Gaussian draws for the momenta and the pseudofermion noise (Section 2: P and
 * chi Gaussian distributed) by Philox4x64-10 (Salmon et al. 2011; key (seed,0),
 * counter (j, stream, 0, 0)):
 * what = 0: half spinor of parity `parity` with N(0,1) real and imaginary parts
 *           (lexicographic element order decides the draw);
 * what = 1: algebra field (momenta), N(0,1) per coordinate. */
int gaussian_draw(wd_ctx* ctx, int what, int parity, uint64_t seed, uint64_t stream, double* out);
/* The Metropolis test of Section 2: accept iff u < exp(-dH), u in [0, 1) (else
 * WD_ERR_ARG); host-only, no device work. */
int metropolis(double dH, double u, int* accept);
/* The same test with u drawn from (seed, counter), the caller's position in
 * its accept/reject stream: u = ((x0 >> 11) + 1/2) 2^-53 with x0 the first word
 * of the Philox4x64-10 block of key (seed, 0) and counter (counter,
 * WD_METROPOLIS_STREAM, 0, 0), the generator of gaussian_draw on a stream of
 * its own.  u (may be NULL) receives the draw.  Host-only, no device work. */
#define WD_METROPOLIS_STREAM 0x8000000000000000ull
int metropolis_philox(double dH, uint64_t seed, uint64_t counter, double* u, int* accept);

/* Cost of an action over n trajectories (Section 3.1, the cost metric):
 * C = <N_mat> / P_acc, N_mat the K_hat multiplications of one trajectory
 * (wd_hmc_result.n_mat) and P_acc the Metropolis acceptance rate.  Inputs are
 * host arrays of length n >= 1: n_mat[i] >= 0, accepted[i] in {0, 1}, dH[i]
 * not NaN.  Also returned: p_acc_est = <min(1, exp(-dH))>, an estimator of
 * P_acc with less variance, and <exp(-dH)> with its standard error, which is
 * 1 at equilibrium for a reversible, area-preserving integrator.  C is +inf
 * when no trajectory was accepted.  Host-only; needs no context and no GPU. */
typedef struct {
  double C, p_acc, p_acc_est, mean_nmat, exp_mdH, exp_mdH_err;
  double C_est;   /* <N_mat> / p_acc_est, +inf when p_acc_est is 0 */
} wd_cost_result;
int wd_cost(const long long* n_mat, const int* accepted, const double* dH, int n, wd_cost_result* out);

/* ---- HMC trajectory ---------------------------------------------------------- */

/* One operation of an integrator (Section 2: T[eps] and S[eps]; Section 3.2:
 * one time scale per group): kind 0 = T[eps]; kind 1 = S[eps] for the terms in
 * group `group` (group -1 = gauge action). */
typedef struct { int kind; int group; double eps; } wd_op;

typedef struct {
  int nterms;
  const wd_term* terms;      /* host array of fermion terms */
  const int* term_group;     /* host array: integrator group of each term */
  double beta;               /* gauge action coupling; <= 0 disables S_G */
  int nops;
  const wd_op* ops;          /* host array: the integrator */
  wd_cg_params cg_md;        /* solves inside the molecular dynamics */
  wd_cg_params cg_acc;       /* solves for the accept/reject actions */
  int force_prec;            /* arithmetic of force kernels (WD_F64 / WD_F32) */
  uint64_t seed;             /* Philox key for momenta and pseudofermions */
  uint64_t traj_index;       /* counter stream: trajectory number */
  int h0_solve;              /* 0: the starting pseudofermion actions are the heat
                                bath's sum_i chi_i^dag chi_i (exact up to the heat
                                bath's solver tolerance); 1: each is re-evaluated by
                                its solve, as the final ones always are */
} wd_hmc_params;

typedef struct {
  double H0, H1, dH;
  double S_gauge0, S_gauge1;
  int accepted;
  long long n_mat;           /* K_hat applications in the trajectory */
  int n_force_evals;
  /* device time (CUDA events on the context stream), ms: heat bath and
   * momenta, the two Hamiltonians, all T steps, the gauge force, and the
   * fermion forces of integrator groups 0..3 */
  double t_heatbath_ms, t_hamiltonian_ms, t_T_ms, t_gauge_force_ms;
  double t_force_group_ms[4];
} wd_hmc_result;

/* One HMC trajectory (Section 2): heat bath, momentum draw, integration,
 * accept/reject with uniform u (host).
 * Draws: momenta P_a ~ N(0,1) per coordinate (density exp(-sum tr P^2)) from
 * Philox stream 64 traj_index; the noise of term i is chi ~ exp(-chi^dag chi)
 * (Section 2: real and imaginary parts N(0, 1/2)), the stream 64 traj_index
 * + 1 + i draw of gaussian_draw scaled by 1/sqrt(2).
 * On rejection the context's gauge field is restored. */
int hmc_trajectory(wd_ctx* ctx, const wd_hmc_params* p, double u, wd_hmc_result* res);

/* hmc_trajectory on host buffers (Section 2: one trajectory, as above): the
 * lexicographic FP64 links U_in (HOST, V * 72 doubles) are copied to the
 * device with one cudaMemcpyAsync and loaded, the trajectory runs, and the
 * context's links afterwards (the new ones if accepted, else U_in's) are
 * stored and copied back to U_out (HOST, may be U_in) with one
 * cudaMemcpyAsync; the call returns after that copy.  Pinned host memory
 * makes the copies asynchronous DMA.  The device staging buffer (V * 72
 * doubles) is allocated on the first call and kept by the context. */
int hmc_trajectory_host(wd_ctx* ctx, const wd_hmc_params* p, double u, const double* U_in, double* U_out,
                        wd_hmc_result* res);

/* The molecular-dynamics integration alone, on caller-held momenta (Section 2,
 * eqs. for T-hat and S-hat: T[eps] U = exp(i eps P) U, S[eps] P = P - eps F;
 * Section 3.2 for the schedule): ops are applied in order to the context's
 * links and to P (device algebra field); an S op of group g adds -eps F of
 * every term with term_group g (g = -1: the gauge action, beta > 0) to P.
 * The pseudofermions phi[i] (host array of nterms device half spinors) are
 * held fixed.  No heat bath, no Hamiltonian, no Metropolis test, no restore
 * of the links.  Solves inside forces use cg_md (FP64 when force_prec is
 * WD_F64).  *n_force_evals (may be NULL) = force evaluations made. */
typedef struct {
  int nterms;
  const wd_term* terms;      /* host array */
  const int* term_group;     /* host array: integrator group of each term */
  const double* const* phi;  /* host array of nterms device half spinors */
  double beta;               /* gauge action coupling; <= 0 disables S_G */
  int nops;
  const wd_op* ops;          /* host array: the integrator */
  wd_cg_params cg_md;
  int force_prec;            /* WD_F64 or WD_F32 force kernels */
} wd_integrate_params;
int integrate(wd_ctx* ctx, double* P, const wd_integrate_params* p, int* n_force_evals);

/* Build integrator schedules on the host (Section 3.2).  kind 0 = leapfrog,
 * 1 = Omelyan 2MN.  nested: levels[i] = steps of group i per enclosing T,
 * outermost first (groups -1 = gauge allowed).  Writes up to cap ops; *nops is
 * the full length (call with cap 0 to size).  Consecutive S steps of one group
 * are merged. */
int wd_schedule_nested(int kind, double tau, int nlevels, const int* groups, const int* steps,
                       wd_op* ops, int cap, int* nops);
/* Generalised scheme: overlay per-group integrators of nsteps[i] steps each in
 * time (Section 3.2), ties ordered by group position (ascending before tau/2,
 * descending after). */
int wd_schedule_generalised(int kind, double tau, int ngroups, const int* groups,
                            const int* nsteps, wd_op* ops, int cap, int* nops);

/* ---- batched solves over many lattices and right-hand sides -------------------
 * Section 2 of the paper: the pseudofermion terms of a trajectory and, here,
 * many independent lattices each need solves with K_hat.  A batch groups
 * contexts (lattices of any even extents, gauge fields loaded, one shared
 * stream) with a hopping parameter and 1..8 right-hand sides each; every
 * (lattice, rhs) pair is one system.  The right-hand sides of a lattice are
 * interleaved in the batch's FP32 fields so one warp reads a site's links
 * once for all of them, and one launch covers every lattice.  Allocates its
 * fields (6 FP32 vectors per lattice and rhs) at creation. */
typedef struct wd_batch wd_batch;
/* Group nlat contexts (host array) with kappas[l] and nrhs[l] in 1..8 (host
 * arrays) into one batch (Section 2: several pseudofermion solves with K).
 * WD_ERR_ARG on mixed streams, a context without links or nrhs out of range. */
int wd_batch_create(wd_ctx* const* ctxs, int nlat, const double* kappas, const int* nrhs, wd_batch** out);
/* Free the batch's fields (not the contexts).  NULL is accepted. */
int wd_batch_destroy(wd_batch* b);
/* out[l] = K_hat in[l] per system (Section 2: K = M^dag M), FP32 with FP32 links of the contexts'
 * storage (12 or 18 reals, from the first context).  in[l], out[l]: nrhs[l]
 * consecutive FP64 half spinors of lattice l (device). */
int wd_batch_mdagm(wd_batch* b, const double* const* in, double* const* out);
/* CG (Section 2: the iterative solver of K) for every system from x = 0,
 * mixed precision: FP32 batched iterations,
 * FP64 reliable updates per system (through its context) to the FP64 true
 * residual p->tol; K_hat x of a reliable update is formed in double-float
 * when the system's context has wd_set_residual(ctx, 1).  p->check_every
 * iterations (default 16) run between host checks: use_graph = 0 as plain
 * launches (eight per iteration), 1 as one captured CUDA graph of those
 * launches, 2 as one persistent cooperative kernel per chunk whose phases are
 * separated by grid barriers (every block resident; each barrier wait bounded
 * to two seconds, an expiry returns WD_ERR_TIMEOUT).  Systems that have
 * converged or wait for a reliable update do no work inside a chunk.  infos: one per system, in
 * lattice order, or NULL.  The first call times the candidate tile shapes of
 * the batched kernels (items per block, right-hand sides per thread of the
 * hop; wd_batch_shape) on K_hat b and keeps the fastest. */
int wd_batch_cg(wd_batch* b, const double* const* bvec, double* const* x, const wd_cg_params* p, int use_graph,
                wd_cg_info* infos);
/* Systems, block size chosen by the tuner, kernels launched so far (no
 * counterpart in the paper). */
int wd_batch_info(wd_batch* b, int* n_systems, int* threads, long long* launches);
/* Tile shape of the batched kernels chosen by the tuner (no counterpart in the
 * paper): (site, rhs) items per block; right-hand sides of one site that one
 * thread of the batched hop applies its link to (1, 2 or 4; the link is loaded
 * and rebuilt once for them); link_staging = 1 when the hop runs on the
 * per-thread pipeline that copies each thread's links two directions ahead
 * into shared memory (128 items, one rhs per thread, 12-real links).  Any
 * pointer may be NULL. */
int wd_batch_shape(wd_batch* b, int* items_per_block, int* rhs_per_thread, int* link_staging);
/* Fix the tile shape instead of tuning it (no counterpart in the paper):
 * items_per_block 64, 128 or 256; rhs_per_thread 1, 2 or 4 dividing every
 * lattice's nrhs; link_staging 0 or 1 (1 needs 128 items, one rhs per thread
 * and 12-real links).  WD_ERR_ARG otherwise; the batch is unchanged then. */
int wd_batch_set_shape(wd_batch* b, int items_per_block, int rhs_per_thread, int link_staging);

/* ---- allocation-free K_hat ----------------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers that
 * cannot allocate device memory: code whose device memory belongs to a host
 * application's own pool manager, latency-critical code that cannot afford the
 * implicit device-wide synchronisation of cudaMalloc, or code that must not fail
 * on allocation under memory pressure.  It needs no context.
 *
 * out = K_hat in = M_hat^dag M_hat in (FP64, even sites), M_hat = 1 - kappa^2 D_eo D_oe.
 *   dims      {Lx, Ly, Lz, Lt}, even, >= 2, with V/2 <= 32768 sites per parity
 *             (e.g. 16^4); larger lattices return WD_ERR_ARG before any launch.
 *   gauge_eo  device, FP64 links in the even-odd layout
 *             complex double [4 mu][2 parity][9 = 3 row + col][Vh] (the layout of
 *             the context's own FP64 copy): U_mu(x) of the site with parity p and
 *             checkerboard index cb at element ((mu*2 + p)*9 + 3*row + col)*Vh + cb.
 *   in, out   device half spinors (double2 [12][Vh]); may be the same buffer.
 *   stream    cudaStream_t or NULL; the call is asynchronous on it.
 * Allocates nothing: the two intermediate half spinors live in one static device
 * array (12.6 MB) held on every device that loads the library until exit.
 * Every call shares that array and overwrites it; calls that overlap on the
 * GPU race on it and must be serialised by the caller.  The first call on a
 * device looks up the array's address with that device current; make that
 * first call before any stream capture.  That address is kept per device for
 * the life of the process and belongs to the device's primary context: after
 * cudaDeviceReset, or under another driver-API context, do not call this. */
int mdagm_apply_noalloc(const int dims[4], const double* gauge_eo, double kappa, const double* in,
                        double* out, void* stream);

/* ---- counters and timing ---------------------------------------------------- */

/* N_mat (Section 3.1: the multiplications by K that the cost counts): K_hat
 * applications since the context was created or reset. */
int wd_nmat(wd_ctx* ctx, long long* count, int reset);
/* Measurement, no counterpart in the paper.  Sample every n-th launch of the
 * hop kernels with CUDA events on the context
 * stream (n = 0 disables; launches queued inside a CG chunk, which may return
 * early after convergence, are not sampled).  wd_profile_read gives, for the
 * hop kernels whose input spinors have format fmt (enum wd_prec, or -1 for
 * all), the sampled launches, their total device time (ms) and the
 * algorithmic bytes of those launches (every input site, link and output site
 * moved once). */
int wd_profile_enable(wd_ctx* ctx, int every_n);
int wd_profile_read(wd_ctx* ctx, int fmt, long long* launches, double* total_ms, double* bytes);
/* Kernels launched by this context since it was created (no counterpart in
 * the paper). */
int wd_launch_count(wd_ctx* ctx, long long* count);
/* Hop launches per input format (FP64, FP32, FP16, BF16, double-float) since
 * the last wd_profile_enable, sampled or not (no counterpart in the paper). */
int wd_hop_counts(wd_ctx* ctx, long long counts[5]);

#ifdef __cplusplus
}
#endif
#endif
