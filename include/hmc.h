/*
 * hmc.h -- C ABI of libhmc, the GB300 (sm_103a) hot path of Hybrid Monte Carlo
 * for the Hubbard model on the honeycomb lattice (Krieg, Luu, Ostmeyer,
 * Papaphilippou, Urbach, arXiv:1804.07195).
 *
 * Conventions shared by every call
 * --------------------------------
 * Lattice.  An n x m honeycomb torus (rhombic unit cells, one A and one B site
 *   each, periodic along both oblique axes) with nt time slices; delta = beta/nt
 *   (Section 2). A(i,j) is bonded to B(i,j), B(i-1,j), B(i,j-1) (indices mod n, m).
 * Layout.  Every space-time array holds N = 2*n*m*nt entries in the canonical
 *   order  idx = ((s*nt + t)*m + j)*n + i,  s = 0 for A, 1 for B.
 *   Complex vectors are interleaved (re, im): complex128 = two doubles (16 B),
 *   complex64 = two floats (8 B). The field phi and momenta pi are real doubles.
 * Memory.  Every array argument is DEVICE memory owned by the caller, contiguous,
 *   in the canonical layout and at least 16-byte aligned. The library never
 *   frees or retains caller pointers beyond the call. The context owns its own
 *   workspace (phase tables, Krylov vectors, reduction partials), allocated at
 *   creation or on first use and freed by hmc_destroy.
 * Streams.  A context is bound to one CUDA stream; all work is enqueued on it.
 *   Calls that return host scalars (solve info, actions, Hamiltonians) synchronise
 *   that stream before returning; pure operator applications do not.
 * Errors.  Every call returns an hmc_status. HMC_ERR_INVALID for null pointers,
 *   non-positive sizes, a precision other than 32 or 64, a negative shift sigma,
 *   a time hop that vanishes (1 - delta*m_s == 0) or a misaligned pointer.
 *   HMC_ERR_CUDA when a CUDA call fails (the message is in hmc_last_error).
 *   HMC_ERR_NOT_CONVERGED when a solver reaches its iteration limit: x then
 *   holds the last iterate and info->true_rel_res its true residual.
 *   HMC_ERR_NAN when a reduction produced NaN/Inf or a non-positive curvature.
 *   No call aborts the process.
 * Thread safety.  A context may be used by one host thread at a time.
 */
#ifndef HMC_H
#define HMC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HMC_ABI_VERSION 1
#define HMC_MAX_MASSES 8

typedef enum {
  HMC_OK = 0,
  HMC_ERR_INVALID = -1,
  HMC_ERR_CUDA = -2,
  HMC_ERR_NOT_CONVERGED = -3,
  HMC_ERR_NAN = -4,
  HMC_ERR_TIMEOUT = -5,
  HMC_ERR_NOMEM = -6
} hmc_status;

/* Lattice and couplings (Section 2): kappa the hopping, U the on-site coupling,
 * beta the inverse temperature; delta = beta / nt. */
typedef struct {
  int n, m, nt;
  double kappa, U, beta;
} hmc_lattice;

/* Report of one linear solve. iters: CG iterations, or Arnoldi steps of FGMRES;
 * iters_outer: FGMRES restarts (0 for CG); iters_inner: single-precision CG
 * iterations summed over all preconditioner solves; true_rel_res: |b - A x| / |b|
 * recomputed in FP64 after the solve; applies64/applies32: applications of
 * M M^dagger in each precision; bytes: algorithmic HBM bytes of all kernels;
 * seconds: wall time of the call. */
typedef struct {
  int iters;
  int iters_outer;
  int iters_inner;
  int status;
  double true_rel_res;
  double seconds;
  long long applies64;
  long long applies32;
  long long bytes;
} hmc_solve_info;

/* Solver selection for calls that solve internally (forces, actions, MD). */
enum {
  HMC_SOLVER_CG64 = 0,         /* plain FP64 CG (Section 3) */
  HMC_SOLVER_FGMRES_MIXED = 1, /* FGMRES with FP32 CG preconditioner (Algorithm A.1) */
  HMC_SOLVER_FGMRES_FP64 = 2,  /* Algorithm A.1 with an FP64 CG preconditioner: all FP64,
                                  true residual recomputed at every restart */
  HMC_SOLVER_FCG_MIXED = 3     /* flexible CG with FP32 CG preconditioner (Section 3) */
};

typedef struct {
  int method;          /* HMC_SOLVER_* */
  double tol;          /* relative residual target */
  int maxit;           /* CG iterations, or FGMRES Arnoldi steps */
  int restart;         /* FGMRES restart length m (Appendix A: 10) */
  double a;            /* FGMRES inner tolerance factor (Appendix A: 5) */
  double inner_floor;  /* smallest tolerance asked of the FP32 inner CG (1e-6) */
  int inner_maxit;     /* FP32 inner CG iteration limit (2000) */
} hmc_solver_opts;

/* Integrators for hmc_md_trajectory (Sections 4 and 5.2). */
enum {
  HMC_INTEG_NESTED_OMELYAN = 0, /* multi-time-scale Omelyan, force first */
  HMC_INTEG_LEAPFROG = 1,       /* all forces on one scale */
  HMC_INTEG_FORCE_GRADIENT = 2  /* Eq. force_cal, all forces on one scale */
};

typedef struct {
  int kind;                 /* HMC_INTEG_* */
  int nmd;                  /* N_MD: innermost steps per trajectory */
  int N[HMC_MAX_MASSES];    /* time-scale ratios N_0..N_{n-1} (Section 5.2):
                               the chi_k force is applied nmd/N_k times */
  double zeta;              /* Omelyan parameter (Section 4.1: 0.193) */
  double tau;               /* trajectory length (Section 7.1: 1) */
} hmc_integrator;

typedef struct hmc_ctx hmc_ctx;

/* ---- library and context -------------------------------------------------- */

/* Version of this header's ABI (HMC_ABI_VERSION). */
int hmc_abi_version(void);
/* Static text for a status code. */
const char* hmc_status_string(hmc_status s);
/* Text of the last error recorded on ctx (empty if none); owned by ctx. */
const char* hmc_last_error(const hmc_ctx* ctx);

/* Create a context for one lattice on the current CUDA device, bound to
 * cuda_stream (a cudaStream_t; NULL = the legacy default stream). Allocates the
 * phase tables and the reduction scratch. */
hmc_status hmc_create(hmc_ctx** out, const hmc_lattice* lat, void* cuda_stream);
/* Free the context and all of its workspace (synchronises its stream). */
hmc_status hmc_destroy(hmc_ctx* ctx);
/* Rebind the context to another stream (the caller orders the two streams). */
hmc_status hmc_set_stream(hmc_ctx* ctx, void* cuda_stream);

/* ---- the auxiliary field --------------------------------------------------- */

/* Every call below that takes `phi` derives the phase table e^{i phi} (and a
 * float copy of phi for the single-precision kernels) from it on entry, one
 * elementwise pass. Passing phi = NULL instead reuses the tables of the field
 * last given to hmc_load_field, which saves that pass when many calls share one
 * field. The loaded tables are a copy: changing phi afterwards does not change
 * them until hmc_load_field is called again. Asynchronous. */
hmc_status hmc_load_field(hmc_ctx* ctx, const double* phi);

/* ---- operator (Eq. ferm_op) ----------------------------------------------- */

/* out = M[phi; m_s] in  (Eq. ferm_op). phi: N doubles. in, out: N complex of
 * precision prec (64: complex128, 32: complex64); in and out must not overlap.
 * The anti-periodic time boundary flips the sign of the wrapping time hop.
 * Asynchronous. */
hmc_status hmc_apply_M(hmc_ctx* ctx, const double* phi, double ms, const void* in, void* out,
                       int prec);
/* out = M[phi; m_s]^dagger in, the conjugate transpose (Eq. ferm_op). */
hmc_status hmc_apply_Mdag(hmc_ctx* ctx, const double* phi, double ms, const void* in, void* out,
                          int prec);
/* out = M M^dagger in + sigma in, the Hermitian positive definite operator of the
 * solves (Eq. hamiltonian; the shifted form of Section 5.1). sigma >= 0. */
hmc_status hmc_apply_MMdag(hmc_ctx* ctx, const double* phi, double ms, double sigma, const void* in,
                           void* out, int prec);

/* ---- solvers (Section 3, Algorithm A.1) ------------------------------------ */

/* Plain FP64 CG for (M M^dagger + sigma) x = b (Section 3). b, x: complex128;
 * x holds the initial guess on entry and the solution on return. Stops when the
 * recursive residual satisfies |r| <= tol |b| or after maxit iterations.
 * info may be NULL. Synchronous. */
hmc_status hmc_solve_cg(hmc_ctx* ctx, const double* phi, double ms, double sigma, const void* b,
                        void* x, double tol, int maxit, hmc_solve_info* info);
/* The single-precision CG of Section 3 on its own: b, x complex64, x = 0 start,
 * vectors and operator in FP32, dot products accumulated in FP64. */
hmc_status hmc_solve_spcg(hmc_ctx* ctx, const double* phi, double ms, double sigma, const void* b,
                          void* x, double tol, int maxit, hmc_solve_info* info);
/* Flexible GMRES (Algorithm A.1): outer Arnoldi, residuals and Gram-Schmidt in
 * FP64; preconditioner = CG in precision inner_prec (32: spCG, 64: FP64 CG) with
 * tolerance max(tol*a*|b|/ERR, inner_floor), skipped once tol*a*|b|/ERR >= 1;
 * restart length `restart`; least squares through h^H h y = |r| h^H e1 by
 * Cholesky. b, x complex128; x is output only (the first spCG solve starts at 0).
 * maxit bounds the Arnoldi steps. Synchronous. */
hmc_status hmc_solve_fgmres(hmc_ctx* ctx, const double* phi, double ms, double sigma, const void* b,
                            void* x, double tol, int restart, double a, int inner_prec, int maxit,
                            hmc_solve_info* info);

/* Flexibly preconditioned CG (Section 3: the FP64 CG with the single-precision
 * CG as its preconditioner, made flexible because a CG stopped at a tolerance
 * is not a fixed linear map). One previous direction is kept:
 *   z_i = spCG(r_i), p_i = z_i - (p_{i-1}^H A z_i / p_{i-1}^H A p_{i-1}) p_{i-1},
 *   alpha = p_i^H r_i / p_i^H A p_i, x += alpha p_i, r -= alpha A p_i,
 * with the spCG tolerance max(tol*a*|b|/|r_i|, 1e-6) and z_i = r_i once that
 * ratio reaches 1. Stops when |r| <= tol |b| (recursive residual; info reports
 * the true one). b, x complex128; x is output only. Synchronous. */
hmc_status hmc_solve_fcg(hmc_ctx* ctx, const double* phi, double ms, double sigma, const void* b,
                         void* x, double tol, double a, int maxit, hmc_solve_info* info);

/* One independent system of a batched solve. Lattices may differ between
 * systems; phi, b, x are device arrays in each system's own canonical layout. */
typedef struct {
  hmc_lattice lat;
  const double* phi;
  double ms;
  double sigma;
  const void* b;  /* complex128 */
  void* x;        /* complex128, output (the solve starts at 0) */
  double tol;
  int maxit;
} hmc_system;

/* Solve nsys independent systems together: every CG iteration of all systems
 * runs as one launch per kernel over a descriptor table, converged systems are
 * masked out, and the iteration loop is replayed as a captured CUDA graph.
 * mixed = 0: FP64 CG; mixed = 1: FP32 CG iterations under FP64 defect correction
 * (x += e after each FP32 solve of A e = r, with r = b - A x recomputed in FP64)
 * until |b - A x| <= tol |b| in FP64. infos: nsys entries or NULL. Synchronous. */
hmc_status hmc_solve_batched(hmc_ctx* ctx, int nsys, const hmc_system* sys, int mixed,
                             hmc_solve_info* infos);

/* ---- action and force (Eqs. hamiltonian, p_dot, eta_xi, f_chi_i, def_xi_i) --- */

/* Flags for hmc_force / hmc_action. */
enum {
  HMC_GAUSSIAN = 1,      /* include (1/2) phi^2 / (delta U) and its derivative */
  HMC_FERMION = 2,       /* include the pseudofermion terms selected by `term` */
  HMC_ACCUMULATE = 4     /* hmc_force: add into dSdphi instead of overwriting */
};

/* Pseudofermions from heat-bath vectors (Section 5.1), for nmass staggered
 * masses mu_0 < ... < mu_{n-1} (nmass = 0: the single term chi = M rho):
 *   chi_n = M_{mu_{n-1}} rho_n,
 *   chi_i = M_{mu_i}^dagger (M_{mu_i} M_{mu_i}^dagger)^{-1} M_{mu_{i-1}} rho_i,  M_{mu_{-1}} = M.
 * rho, chi: arrays of nmass+1 device pointers to complex128 vectors. */
hmc_status hmc_make_chi(hmc_ctx* ctx, const double* phi, int nmass, const double* masses,
                        const void* const* rho, void* const* chi, const hmc_solver_opts* opts,
                        hmc_solve_info* info);

/* dS/dphi of S = (1/2) phi^2/(delta U) + sum_i S_i (Eq. hamiltonian with the
 * Hasenbusch terms of Section 5.1), as N doubles; the MD force of Eq. p_dot is
 * its negative. term = -1 selects all nmass+1 pseudofermion terms, 0..nmass one
 * of them; flags select the Gaussian / fermion parts and accumulation.
 * Per term: eta_i = (M_{i-1} M_{i-1}^dagger)^{-1} src_i (src_n = chi_n, src_i =
 * M_{mu_i} chi_i), xi_i = M_{i-1}^dagger eta_i, and
 * dS_i/dphi_{x,t} = -2 Re(eta_i^*(x,t) dM_{(x,t),tp} (xi_i - chi_i)(tp)), chi_i
 * omitted for the top term (Eqs. f_chi_i, def_xi_i). Synchronous. */
hmc_status hmc_force(hmc_ctx* ctx, const double* phi, int nmass, const double* masses,
                     const void* const* chi, int term, int flags, const hmc_solver_opts* opts,
                     double* dSdphi, hmc_solve_info* info);

/* The action S (same terms and flags as hmc_force) as one host double. Each
 * S_i = src_i^dagger (M_{i-1} M_{i-1}^dagger)^{-1} src_i is evaluated in the
 * stationary form 2 Re(src_i^dagger eta_i) - |M_{i-1}^dagger eta_i|^2, equal to
 * the definition for the exact eta_i and with an error second order in the
 * solve residual (flexible GMRES is not a Galerkin method, so src^dagger eta
 * alone would carry a first-order error). Synchronous. */
hmc_status hmc_action(hmc_ctx* ctx, const double* phi, int nmass, const double* masses,
                      const void* const* chi, int term, int flags, const hmc_solver_opts* opts,
                      double* S_out, hmc_solve_info* info);

/* ---- molecular dynamics (Sections 2, 4, 5.2) ------------------------------- */

/* One MD trajectory: pseudofermions from rho (nmass+1 vectors, complex128),
 * H0 = (1/2)phi^2/(delta U) + sum_i rho_i^dagger rho_i + (1/2)pi^2 (exact at the
 * start), the integrator `integ` with the forces of hmc_force (level k < nmass:
 * the chi_k term; the innermost level: Gaussian + chi_n), then
 * H1 = S(phi', pi') with solves at action_opts' tolerance. phi and pi are
 * updated in place (device, N doubles each). The accept/reject step is the
 * caller's. md_opts: the solver of the MD forces. agg: summed solve report.
 * Synchronous. */
hmc_status hmc_md_trajectory(hmc_ctx* ctx, double* phi, double* pi, int nmass,
                             const double* masses, const void* const* rho,
                             const hmc_integrator* integ, const hmc_solver_opts* md_opts,
                             const hmc_solver_opts* action_opts, double* H0, double* H1,
                             hmc_solve_info* agg);

/* One Markov chain of a batched trajectory: its lattice (chains may differ in
 * size and couplings), its field phi and momenta pi (device, N doubles each,
 * updated in place) and its nmass+1 heat-bath vectors rho (device pointers to
 * complex128 vectors). */
typedef struct {
  hmc_lattice lat;
  double* phi;
  double* pi;
  const void* const* rho;
} hmc_chain;

/* One MD trajectory for each of nchains independent chains, advanced in
 * lockstep (Section 2's HMC outline, the integrators of Sections 4 and 5.2, the
 * Hasenbusch terms of Section 5.1 with the same masses for every chain): the
 * same steps as hmc_md_trajectory for each chain, but every solve the chains
 * need at one point of the schedule -- one per chain and term -- runs as one
 * batched solve (hmc_solve_batched; FP64 CG for HMC_SOLVER_CG64, else FP32 CG
 * under FP64 defect correction to the options' tolerance). H0, H1 and infos
 * (may be NULL) receive nchains entries. The context keeps one internal context
 * per chain (recreated when that chain's lattice changes), freed by
 * hmc_destroy. Synchronous. */
hmc_status hmc_md_trajectory_batched(hmc_ctx* ctx, int nchains, const hmc_chain* chains, int nmass,
                                     const double* masses, const hmc_integrator* integ,
                                     const hmc_solver_opts* md_opts, const hmc_solver_opts* action_opts,
                                     double* H0, double* H1, hmc_solve_info* infos);

/* ---- launch shapes and graphs ----------------------------------------------- */

/* The calls of this section and the next choose or report how the library
 * runs the paper's operations on the GPU; they have no counterpart in the
 * paper and, apart from the wait test hook, change no result beyond the
 * rounding order of floating-point sums. */

/* The CG kernels' launch shapes are chosen by an autotuner on a context's first
 * solve in each precision (timed candidates; see hmc_profile_read for the
 * choice). FP32 CG has four kernel designs: three two-kernel-per-iteration
 * pairs — grid-stride kernels with neighbours read through the caches;
 * shared-memory tiled kernels that stage each time slice of a cell tile with
 * its neighbour halo; marching kernels in which each thread keeps one cell
 * and walks up in time, carrying its time neighbours in registers — and a
 * persistent kernel that runs the whole solve in one cooperative launch with
 * grid barriers (bounded waits; a wait that gives up returns
 * HMC_ERR_TIMEOUT) and keeps x and its own entries of r and p in shared
 * memory. The grid-stride pair also comes with two cells per thread: the
 * neighbouring cells (i, i+1), i even, of a row, whose complex64 values are one
 * 16-byte access in every vector (n even only). The sixth design runs ONE
 * kernel and one grid-wide reduction per iteration: the single-reduction form
 * of CG (Chronopoulos and Gear 1989; the same iterates as CG in exact
 * arithmetic), whose kernel applies M M^dagger + sigma over tiles with
 * M^dagger r kept in shared memory as hmc_apply_MMdag's fused kernel does,
 * and updates x, r, p and the recurrences of w = A r and s = A p as the
 * slices arrive. The seventh runs the whole solve in one cooperative launch
 * in which each block keeps p and M^dagger p of its tile (all n cells of a
 * row, a few rows and time slices) in shared memory and exchanges the tile's
 * edges through memory between grid barriers (bounded waits, as for the
 * persistent kernel). variant: 0 = let the autotuner choose among all of
 * them (default), 1 = grid-stride with one cell per thread, 2 = tiled only,
 * 3 = marching only, 4 = persistent, 5 = grid-stride with two cells per
 * thread, 6 = single-reduction, 7 = resident tiles (2 to 7 fall back to
 * variant 1 where they do not fit the lattice). Setting it re-runs the
 * tuner at the next FP32 solve. */
hmc_status hmc_set_cg_variant(hmc_ctx* ctx, int variant);

/* The FP32 CG of hmc_solve_batched (mixed = 1) runs in one of two designs:
 * 1 = a captured graph whose device-side loop repeats chunks of per-iteration
 * kernels (two launches per iteration over all systems); 2 = one persistent
 * cooperative launch per inner solve, whose blocks walk the systems' blocks
 * and separate the halves of an iteration by grid barriers (bounded waits: a
 * wait that gives up returns HMC_ERR_TIMEOUT). variant 0 (default) runs the
 * first inner solve of the context with 1 and the second with 2 and keeps the
 * one with the shorter time per iteration; 1 or 2 pins one. The variant in
 * use (0 = not chosen yet) is reported by hmc_batched_variant. */
hmc_status hmc_set_batched_variant(hmc_ctx* ctx, int variant);
hmc_status hmc_batched_variant(hmc_ctx* ctx, int* variant);

/* M M^dagger applications (hmc_apply_MMdag) run in one of two designs:
 * 1 = two passes, u = M^dagger in written to and read back from memory, then
 * M u + sigma in; 2 = one fused kernel: each block stages the time slices of a
 * tile of cells plus a one-cell ring in shared memory (cp.async, two slices
 * ahead), forms u there and applies M to it, so u never reaches memory
 * (20 bytes per site in FP32, 48 in FP64, against 40 and 96 for two passes).
 * variant 0 (default) times both on the first application in each precision
 * and keeps the faster; 1 or 2 pins one. Results agree to rounding order. */
hmc_status hmc_set_apply_variant(hmc_ctx* ctx, int variant);
/* The variant used for precision prec (0 = not chosen yet). */
hmc_status hmc_apply_variant(hmc_ctx* ctx, int prec, int* variant);
/* Pin the fused kernel's tile for precision prec: Ti x Tj cells per block
 * (clamped to the lattice), Tt time slices per block, `depth` time slices
 * staged ahead of the one in use (2 or 6 in FP32, 2 in FP64), and pairs = 1 for the FP32 kernel
 * whose threads own two neighbouring cells as one 16-byte complex64 pair
 * (n and Ti even; (Ti/2+2)(Tj+2) <= 256 threads) or 0 for one cell per thread
 * ((Ti+2)(Tj+2) <= 1024 threads in FP32, 512 in FP64). Without it the tile
 * is chosen by timing candidates on the first fused application. A call whose
 * vectors are not 16-byte aligned runs the one-cell kernel. HMC_ERR_INVALID
 * when the tile does not fit (threads, shared memory, parity). */
hmc_status hmc_set_fused_tile(hmc_ctx* ctx, int prec, int Ti, int Tj, int Tt, int depth, int pairs);
/* The fused kernel's tile in use for precision prec (zeros before the first
 * fused application). */
hmc_status hmc_fused_tile(hmc_ctx* ctx, int prec, int* Ti, int* Tj, int* Tt, int* depth, int* pairs);
/* Pin the tile of the single-reduction FP32 CG kernel (variant 6 of
 * hmc_set_cg_variant): Ti x Tj cells per block plus a one-cell ring
 * ((Ti+2)(Tj+2) <= 512 threads, clamped to the lattice), Tt time slices per
 * block, `depth` time slices staged ahead (2 or 6). All three sizes 0 return
 * the choice to the tuner. HMC_ERR_INVALID when the tile does not fit
 * (threads, shared memory, more blocks than the reduction buffers hold). */
hmc_status hmc_set_cg_fused_tile(hmc_ctx* ctx, int Ti, int Tj, int Tt, int depth);
/* The single-reduction kernel's tile and whether FP32 solves use it
 * (in_use = 1: chosen by the tuner or pinned by variant 6). */
hmc_status hmc_cg_fused_tile(hmc_ctx* ctx, int* Ti, int* Tj, int* Tt, int* depth, int* in_use);

/* Test hook for the bounded waits of the persistent FP32 CG kernel (variant 4
 * above): from the next persistent solve on, every grid barrier waits for
 * `extra` more arrivals than the launch has blocks (with extra > 0 no barrier
 * can complete, a wait that nothing ends) and gives up after `limit_cycles`
 * SM clock cycles (0: the default, about one second). A solve whose wait gave
 * up returns HMC_ERR_TIMEOUT and the context stays usable. extra = 0 and
 * limit_cycles = 0 restore normal operation. */
hmc_status hmc_set_wait_test(hmc_ctx* ctx, int extra, long long limit_cycles);

/* How the context runs CG iterations: 2 = each solve is one CUDA-graph launch
 * whose device-side while loop repeats captured chunks of iterations until
 * the solve is done (the host waits once); 1 = captured chunks replayed with
 * host checks in between (used when the loop graph cannot be built);
 * 0 = kernels launched one by one (per-kernel timing on, or no graphs). */
hmc_status hmc_graph_mode(hmc_ctx* ctx, int* mode);
/* Choose it: 2 (default) or 1. Profilers that replay single kernels cannot see
 * kernels inside a graph with a conditional node, so kernel profiles of the
 * CG iterations are taken in mode 1 (the same kernels, replayed in chunks). */
hmc_status hmc_set_graph_mode(hmc_ctx* ctx, int mode);

/* ---- instrumentation ------------------------------------------------------- */

#define HMC_NKERNELS 40  /* at least the number of kernel groups the library reports */

typedef struct {
  char name[48];
  long long launches;   /* launches since the last reset */
  double ms_total;      /* summed CUDA-event time (0 unless timing was on) */
  double bytes_total;   /* algorithmic HBM bytes summed over those launches: each
                           array the kernel must read or write, counted once */
  int threads;          /* launch shape chosen by the autotuner (CG kernels) */
  int waves;            /* grid = waves x resident blocks (0: one item per thread);
                           -tt: the tiled FP32 CG kernels with tt time slices
                           per tile of `threads` cells; -(1000 + tt): the
                           marching kernels, tt slices per block */
  int design;           /* FP32 CG kernels: 0 grid-stride (one cell per thread),
                           1 tiled, 2 marching, 4 grid-stride with two cells
                           per thread */
} hmc_kernel_stat;

/* Every device buffer a context allocates carries guard bands of 256 bytes
 * before and after it, filled with the byte 0xA5. Check them all (synchronises
 * the context's stream); *nbad receives the number of buffers with a changed
 * band, and hmc_last_error names the first. A kernel that writes past either
 * end of a workspace buffer shows up here. */
hmc_status hmc_check_guards(hmc_ctx* ctx, int* nbad);
/* Test hook for hmc_check_guards: writes one byte into the band just after the
 * context's phase table (inside its allocation, no kernel involved). */
hmc_status hmc_guard_test_write(hmc_ctx* ctx);

/* Per-kernel launch counters are always kept. With timing on, every launch of
 * a library kernel is bracketed by CUDA events on the context's stream and
 * the elapsed times are summed at read time (which synchronises). */
hmc_status hmc_profile(hmc_ctx* ctx, int timing_on, int reset);
/* Copy up to max entries of the per-kernel statistics; *count receives the number written. */
hmc_status hmc_profile_read(hmc_ctx* ctx, hmc_kernel_stat* out, int max, int* count);

/* ---- one call that allocates nothing ----------------------------------------- */

/* The paper has no counterpart to this entry point.
 *
 * out = (M[phi; m_s] M[phi; m_s]^dagger + sigma) in for complex128 vectors, the
 * same operator as hmc_apply_MMdag, for callers that cannot allocate device
 * memory: code that runs while its stream is being captured into a CUDA graph
 * (cudaMalloc is not permitted there), frameworks whose memory pool already
 * owns the device (a raw cudaMalloc beside it fails or fragments it), and
 * latency-bound loops that cannot afford an allocation and the device
 * synchronisation it implies. It needs no context and allocates nothing: the
 * M^dagger intermediate lives in a static device array of
 * HMC_NOALLOC_MAX_SITES complex128 entries (16 MiB), which every GPU that
 * loads this library holds until the process exits, and the phases e^{i phi}
 * are computed from phi inline.
 *
 * lat: the lattice (as for hmc_create); phi: N doubles; in, out: N complex128,
 * device memory of the current device, not overlapping; sigma >= 0;
 * cuda_stream: a cudaStream_t (NULL = the legacy default stream).
 * Returns HMC_ERR_NOMEM for a lattice with more than HMC_NOALLOC_MAX_SITES
 * sites (N = 2 n m nt), HMC_ERR_INVALID for bad arguments, HMC_ERR_CUDA when a
 * CUDA call fails. The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress): make that first call before any stream
 * capture. All calls share the one array and it keeps the last call's
 * contents: calls that overlap on the GPU (on different streams or from
 * different host threads) race on it and corrupt each other's results, so
 * serialise them. Asynchronous. */
#define HMC_NOALLOC_MAX_SITES (1 << 20)
hmc_status hmc_apply_MMdag_noalloc(const hmc_lattice* lat, const double* phi, double ms, double sigma,
                                   const void* in, void* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* HMC_H */
