/*
 * wcmg.h -- C-ABI of the GB300 Wilson-clover multigrid library (libwcmg.so).
 *
 * Method: Richtmann, Boyle, Wettig, "Multigrid for Wilson Clover Fermions in
 * Grid" (LATTICE2018, arXiv:1904.08678).  The calls follow the paper's statement
 * of the problem: set the gauge field and clover term (Sec. 1, Sec. 2.1); build
 * near-null vectors by the initial and the iterative-refinement setup (Sec. 2.1);
 * apply D, restrict, prolong and the coarse D (Sec. 2.1 Aggregation /
 * CoarsenedMatrix Mdiag + Mdir); solve D x = b with FGMRES preconditioned by the
 * multigrid cycle (Sec. 2.1).  Everything runs on one CUDA device.
 *
 * Conventions
 *  - Every call returns WCMG_OK (0) or a negative wcmg_status.  No exception
 *    crosses the ABI.  wcmg_last_error() gives a message for the last failure.
 *  - External buffers are complex128 (interleaved re, im doubles) in these
 *    layouts, site index s = x + Lx*(y + Ly*(z + Lz*t)) on the level's lattice:
 *      gauge        [4][V][3][3]           U_mu(x), link x -> x + mu, mu = x,y,z,t
 *      fine field   [nrhs][V][4][3]        spin-major, colour-minor, chiral gamma basis
 *      coarse field [nrhs][Vc][nbasis]     first Nvec components chirality +, then -
 *      coarse links [9][Vc][nbasis][nbasis] block d = 0 self, 1+2mu reads
 *                                           phi(x+mu), 2+2mu reads phi(x-mu)
 *      clover       [V][12][12]            C(x) including (4 + m0)
 *  - `where` says whether a buffer pointer is host (WCMG_HOST) or device
 *    (WCMG_DEVICE) memory.  Host buffers are copied through library-owned device
 *    staging; device buffers are read/written in place.  The caller keeps
 *    ownership of its buffers; they must stay valid until the call returns
 *    (host) or until `stream` has completed the call's work (device).
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are stream
 *    ordered; a call that needs a host decision (a solver's stopping test)
 *    synchronises `stream` itself.
 *  - `prec` selects the arithmetic of a single operator application:
 *    WCMG_F64 or WCMG_F32 (external data stays complex128).
 *  - A context is not thread safe: use one per host thread.  The library owns
 *    all internal buffers, allocated on the device current at wcmg_create.
 */
#ifndef WCMG_H
#define WCMG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WCMG_MAX_LEVELS 4

typedef enum {
  WCMG_OK = 0,
  WCMG_ERR_ARG = -1,            /* invalid argument or size */
  WCMG_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  WCMG_ERR_STATE = -3,          /* call out of order (e.g. solve before setup) */
  WCMG_ERR_NOT_CONVERGED = -4,  /* iteration limit hit; outputs and stats are valid */
  WCMG_ERR_NAN = -5,            /* non-finite norm or rank-deficient aggregate */
  WCMG_ERR_TIMEOUT = -6,        /* a bounded device-side wait gave up */
  WCMG_ERR_OOM = -7             /* device allocation failed */
} wcmg_status;

typedef enum { WCMG_F64 = 0, WCMG_F32 = 1, WCMG_BF16 = 2, WCMG_F16 = 3 } wcmg_prec;
typedef enum { WCMG_HOST = 0, WCMG_DEVICE = 1 } wcmg_where;

typedef struct wcmg_params {
  int dims[4];                          /* fine Lx, Ly, Lz, Lt (periodic) */
  int n_levels;                         /* 2 .. WCMG_MAX_LEVELS */
  int block[WCMG_MAX_LEVELS - 1][4];    /* aggregate extents per coarsening */
  int nvec[WCMG_MAX_LEVELS - 1];        /* near-null vectors per coarsening (nbasis = 2 nvec) */
  double m0;                            /* bare mass: D has (4 + m0) on the diagonal */
  double csw;                           /* clover coefficient */
  int smoother_steps;                   /* MR steps of the post-smoother and setup smoother (0 .. 64) */
  int setup_init_sweeps;                /* initial-setup sweeps per level */
  int setup_refine_sweeps;              /* iterative-refinement sweeps */
  int coarse_restart;                   /* GMRES(m) on the coarsest level */
  int coarse_maxiter;
  double coarse_tol;                    /* relative residual of the coarsest solve */
  int outer_restart;                    /* FGMRES(m) outer solver */
  int outer_maxiter;                    /* total outer iterations */
  double outer_tol;                     /* true relative residual ||b - D x|| / ||b|| */
  int inner_prec;                       /* WCMG_F64: all FP64; WCMG_F32: preconditioner,
                                           setup and coarse operators FP32 with FP64
                                           outer residual / orthonormalisation / Hessenberg */
  int coarse_link_prec;                 /* storage of coarse links when inner_prec = F32:
                                           WCMG_F32, WCMG_BF16 or WCMG_F16 (FP32 accumulate) */
  int max_rhs;                          /* largest nrhs of any call */
  int profile;                          /* bitmask of (1 << wcmg_kclass): kernel classes whose
                                           launches are timed with CUDA events (-1: all, 0: none);
                                           launch, byte and flop counts are always kept */
  int use_graphs;                       /* 1: wcmg_solve runs as one CUDA graph with device-side
                                           stopping tests (conditional WHILE / IF nodes), captured
                                           on the second solve with a given nrhs and replayed
                                           after; the first solve runs host-driven.  Plain
                                           multigrid coarse mode only (learned modes run
                                           host-driven).  Kernel-class event timing is not
                                           available inside a replay.  0: host-driven. */
  int autotune;                         /* 1: the first coarse apply of each (level, nrhs, link
                                           storage) times the candidate launch shapes on the
                                           level's own data and keeps the fastest. 0: fixed rule */
  int smoother;                         /* WCMG_SMOOTHER_MR: MR(smoother_steps) (Sec. 2.1);
                                           WCMG_SMOOTHER_GMRES: GMRES with smoother_steps steps,
                                           zero guess, no restart (Sec. 4 comparison runs);
                                           WCMG_SMOOTHER_SAP: Schwarz alternating procedure
                                           (Sec. 4): sap_cycles cycles of two colour passes over
                                           the level's aggregates (coloured by the parity of their
                                           coarse coordinates), each pass r = b - D x on the
                                           blocks of one colour, then smoother_steps MR steps of
                                           the block-local operator D_B (D without the hops that
                                           leave a block) with one step length per block, added
                                           to x.  The same smoother serves the cycle and the
                                           setup sweeps. */
  int kcycle;                           /* 0: V-cycle (one cycle of an intermediate level as its
                                           coarse solve); 1: K-cycle: FGMRES(kcycle_steps) to
                                           kcycle_tol, right-preconditioned by the level's cycle,
                                           on every level between the finest and the coarsest */
  int kcycle_steps;                     /* 1 .. 64 */
  double kcycle_tol;                    /* relative residual of the intermediate FGMRES */
  int sap_cycles;                       /* SAP smoother: cycles (1 .. 16) */
  int sap_eo;                           /* 1: even-odd (red-black) preconditioned SAP block solves on
                                           the fine level (Sec. 4 lists red-black preconditioning
                                           among the missing features): per block, with sites
                                           even / odd by the parity of x + y + z + t,
                                           r^_o = r_o - H_oe C_ee^-1 r_e, smoother_steps MR steps on
                                           the Schur complement C_oo - H_oe C_ee^-1 H_eo (one step
                                           length per block), e_e = C_ee^-1 (r_e - H_eo e_o); H the
                                           hops inside the block, C the clover term, inverted once
                                           per wcmg_set_gauge in FP64.  Fine aggregates of at most
                                           256 sites with an even x extent (else WCMG_ERR_ARG).
                                           Coarse levels keep the plain block solves. */
  int ortho_df;                         /* arithmetic of the block orthonormalisation (Sec. 2.2 Q factor
                                           per aggregate and chirality): 0 FP64; 1 double-float on
                                           the FP32 pipe (each value the unevaluated sum of two
                                           floats, 48-bit significands, compensated dot products),
                                           FP64 input and output.  Same algorithm and stopping rule. */
  int coarse_eo;                        /* 1: even-odd (red-black) preconditioned coarsest solve (Sec. 4
                                           lists red-black preconditioning among the missing features):
                                           with coarse sites even / odd by the parity of x + y + z + t,
                                           b^_o = b_o - A_oe A_ee^-1 b_e, GMRES(coarse_restart) on the
                                           Schur complement S = A_oo - A_oe A_ee^-1 A_eo to coarse_tol
                                           relative to ||b^_o||, x_e = A_ee^-1 (b_e - A_eo x_o); A_ee^-1 =
                                           the inverses of the self blocks A_0 (FP64 Gauss-Jordan, once
                                           per coarse operator).  Needs even extents of the coarsest
                                           lattice (else WCMG_ERR_ARG). */
  int coarse_sigma3;                    /* 1: keep, next to the nine-block links of every coarse operator
                                           that the setup builds (D_c = P^dag D P), a five-block copy
                                           [A_0 | A_{+x} | A_{+y} | A_{+z} | A_{+t}] (Sec. 4: DDalphaAMG's
                                           5 stencil points against Grid's 9): gamma5-hermiticity of D
                                           with gamma5 P = P sigma3 gives A_{-mu}(x) = sigma3
                                           A_{+mu}(x - mu)^dag sigma3, so one-rhs applies may stream 5/9
                                           of the link bytes (launch kind 5, chosen by the autotuner or
                                           set with wcmg_set_coarse_tile).  Links given through
                                           wcmg_set_coarse_links or wcmg_load_setup are not assumed to
                                           have this symmetry and keep the nine-block kernels.
                                           0 (default): nine blocks only. */
} wcmg_params;

typedef enum { WCMG_SMOOTHER_MR = 0, WCMG_SMOOTHER_GMRES = 1, WCMG_SMOOTHER_SAP = 2 } wcmg_smoother;

/* Per-kernel-class counters, filled when params.profile != 0. */
#define WCMG_NKCLASS 12
typedef struct wcmg_kstat {
  long long launches;
  double ms;                            /* summed CUDA-event time of the launches */
  double bytes;                         /* algorithmic bytes moved (per the kernel's model) */
  double flops;                         /* algorithmic flops */
} wcmg_kstat;

typedef struct wcmg_stats {
  int outer_iterations;                 /* FGMRES iterations summed over restarts (max over rhs) */
  int restarts;
  int converged;                        /* 1 if every rhs met outer_tol */
  double true_residual;                 /* max over rhs of ||b - D x|| / ||b|| (FP64) */
  long long coarse_iterations;          /* coarsest-level GMRES iterations, summed */
  long long kernel_launches;            /* CUDA kernels this library launched during the call */
  double ms_setup_init;                 /* wall time of the phases (host clock around synced work) */
  double ms_setup_refine;
  double ms_solve;
  int learned_fallback;                 /* 1 if a learned solve fell back to plain multigrid */
  int learned_cycles;                   /* cycles that used the network */
  int graph;                            /* 1 if the solve ran as a CUDA-graph replay */
  int reserved;
  wcmg_kstat k[WCMG_NKCLASS];           /* index: wcmg_kclass */
} wcmg_stats;

typedef enum {
  WCMG_K_DSLASH = 0, WCMG_K_COARSE = 1, WCMG_K_RESTRICT = 2, WCMG_K_PROLONG = 3,
  WCMG_K_BLAS = 4, WCMG_K_ORTHO = 5, WCMG_K_COARSEN = 6, WCMG_K_CLOVER = 7,
  WCMG_K_PACK = 8, WCMG_K_KRYLOV = 9, WCMG_K_DSLASH64 = 10, WCMG_K_PTC = 11
} wcmg_kclass;

typedef struct wcmg_ctx wcmg_ctx;

/* Fill *p with the defaults of the 4^4 two-level case (blocks 2^4, Nvec 8, MR(4),
 * 3 initial sweeps, GMRES(20) to 0.05 / 100 its, FGMRES(20) to 1e-10, FP64). */
int wcmg_default_params(wcmg_params* p);

/* Validate *p (every extent divisible by its block, nvec <= 32, nbasis even) and
 * allocate the context on the current device.  ERR_ARG, ERR_OOM, ERR_CUDA. */
int wcmg_create(const wcmg_params* p, wcmg_ctx** out);
void wcmg_destroy(wcmg_ctx* ctx);
const char* wcmg_last_error(const wcmg_ctx* ctx);

/* Sec. 2.1 (fine operator D): set U_mu(x).  Builds the FP64 and FP32 internal
 * copies and the clover term C(x) of Sec. 1 "clover" (Sheikholeslami-Wohlert,
 * four-leaf field strength) with params.m0 / params.csw. */
int wcmg_set_gauge(wcmg_ctx* ctx, const void* U, int where, void* stream);

/* Sec. 1 / Sec. 2.1 (Wilson-clover D): rebuild the clover term C(x) from the gauge
 * field already set, with clover coefficient csw (params.m0 unchanged; the context's
 * csw becomes this value).  A setup built before the call still describes the old D:
 * run wcmg_setup (or wcmg_coarsen) again for the hierarchy to follow.  ERR_STATE
 * before wcmg_set_gauge, ERR_ARG for a non-finite csw. */
int wcmg_set_clover(wcmg_ctx* ctx, double csw, void* stream);

/* The same with caller-given site blocks: C is [V][12][12] complex128 (external clover
 * layout, (4 + m0) included, row index 3 * spin + colour), for tests and for clover
 * terms built elsewhere.  The library stores the two chiral 6x6 blocks of a Hermitian
 * C(x) (the SW clover term commutes with gamma5 in the chiral basis), so every site
 * block must be Hermitian and have no entries coupling spins {0, 1} to {2, 3}, to
 * 1e-12 of its largest entry: otherwise (or with a non-finite entry) the call returns
 * ERR_ARG and the context keeps its previous clover term.  As for wcmg_set_clover the
 * setup must be rebuilt.  ERR_STATE before wcmg_set_gauge. */
int wcmg_set_clover_raw(wcmg_ctx* ctx, const void* C, int where, void* stream);

/* Read back C(x) (FP64), external clover layout. */
int wcmg_get_clover(wcmg_ctx* ctx, void* C, int where, void* stream);

/* C(x)^-1 in the layout of wcmg_get_clover (built by wcmg_set_gauge with params.sap_eo;
 * WCMG_ERR_STATE otherwise). */
int wcmg_get_clover_inverse(wcmg_ctx* ctx, void* C, int where, void* stream);

/* out = D in on the fine lattice (Sec. 2.1: MG runs on D itself), nrhs fields. */
int wcmg_apply_D(wcmg_ctx* ctx, const void* in, void* out, int nrhs, int prec, int where, void* stream);

/* Sec. 2.1 / 2.2: give the Nvec raw near-null vectors of level `level`
 * ([nvec][V_level][ncomp] complex128); they are block-orthonormalised per
 * aggregate and chirality (FP64) to form P_level.  Does not coarsen. */
int wcmg_set_nullvecs(wcmg_ctx* ctx, int level, const void* vecs, int where, void* stream);
/* The block-orthonormalised vectors of P_level, same layout. */
int wcmg_get_nullvecs(wcmg_ctx* ctx, int level, void* vecs, int where, void* stream);

/* Sec. 2.1 CoarsenOperator: D_{level+1} = P_level^dag D_level P_level as the
 * nine-block stencil (Sec. 4: 9 stencil points).  Needs P_level and D_level. */
int wcmg_coarsen(wcmg_ctx* ctx, int level, void* stream);
/* Read the coarse links of `level` (external coarse-link layout, FP64): the most
 * precise copy the context holds (FP64, else FP32, else the BF16/FP16 storage). */
int wcmg_get_coarse_links(wcmg_ctx* ctx, int level, void* A, int where, void* stream);
int wcmg_set_coarse_links(wcmg_ctx* ctx, int level, const void* A, int where, void* stream);

/* Sec. 3 blockProject: coarse = P_level^dag fine (level -> level+1). */
int wcmg_restrict(wcmg_ctx* ctx, int level, const void* fine, void* coarse, int nrhs, int prec, int where, void* stream);
/* fine = P_level coarse (level+1 -> level). */
int wcmg_prolong(wcmg_ctx* ctx, int level, const void* coarse, void* fine, int nrhs, int prec, int where, void* stream);
/* Sec. 2.1 Mdiag + 8 x Mdir: out = D_level in, level >= 1. */
int wcmg_apply_coarse(wcmg_ctx* ctx, int level, const void* in, void* out, int nrhs, int prec, int where, void* stream);

/* Sec. 2.1 setup: initial setup on every level from the given random vectors
 * (init_vecs[l] = [nvec_l][V_l][ncomp_l] complex128, concatenated over
 * l = 0 .. n_levels-2), then params.setup_refine_sweeps iterative-refinement
 * sweeps.  Fills every P_l and D_{l+1}. */
int wcmg_setup(wcmg_ctx* ctx, const void* init_vecs, int where, void* stream, wcmg_stats* st);

/* wcmg_setup with the random vectors generated on the device: vector i of level l is
 * the complex Gaussian field of the counter-based generator with (seed, stream
 * 1 + 1000 l + i), element j [site][component] (external order) from the counters
 * 2j, 2j + 1: SplitMix64 finaliser of seed * 0x9E3779B97F4A7C15 + stream *
 * 0xD1B54A32D192ED03 + k, u = (out >> 11) 2^-53, Box-Muller (re, im) = sqrt(-2 log(1 -
 * u_2j)) (cos, sin)(2 pi u_2j+1), the transform in FP32.  The same fields as the host
 * generator of the test inputs (which transforms in FP64) to FP32 rounding.  No host
 * transfer of the Nvec fields. */
int wcmg_setup_seeded(wcmg_ctx* ctx, unsigned long long seed, void* stream, wcmg_stats* st);

/* One application of the multigrid preconditioner M_0 to nrhs fine fields. */
int wcmg_mg_cycle(wcmg_ctx* ctx, const void* r, void* e, int nrhs, int where, void* stream);

/* Krylov solve of D_level x = b at the inner precision: kind 0 = MR(steps,
 * zero guess), kind 1 = GMRES(restart) to tol (relative to ||b||) / maxiter,
 * kind 2 = the SAP smoother (params.sap_cycles cycles, `steps` block-local MR
 * steps; level < n_levels - 1, whose aggregates are the Schwarz blocks).
 * iters_out (nullable) receives the iterations of the slowest rhs. */
int wcmg_krylov(wcmg_ctx* ctx, int level, int kind, const void* b, void* x, int nrhs,
                int steps_or_restart, double tol, int maxiter, int where, void* stream, int* iters_out);

/* Sec. 2.1 outer solver: FGMRES(outer_restart) right-preconditioned by M_0 on D,
 * from a zero initial guess, until ||b - D x|| / ||b|| <= outer_tol (FP64 true
 * residual) for every rhs.  With inner_prec = F32 each restart cycle runs in FP32
 * and the FP64 residual is recomputed at every restart (defect correction).
 * Returns ERR_NOT_CONVERGED (x and *st valid) at outer_maxiter. */
int wcmg_solve(wcmg_ctx* ctx, const void* b, void* x, int nrhs, int where, void* stream, wcmg_stats* st);

/* Options of wcmg_solve_ex. */
typedef struct wcmg_solve_opts {
  int zero_guess;       /* 1: x is output only and the solve starts from x = 0 (wcmg_solve);
                           0: x holds an initial guess x0 on entry (same layout and `where`
                           as the solution) and the solve starts from r = b - D x0; the
                           stopping test stays ||b - D x|| / ||b|| <= outer_tol */
  int reserved[3];      /* set to 0 */
} wcmg_solve_opts;

/* Sec. 2.1 outer solver with options: wcmg_solve with an in/out initial guess
 * (opts->zero_guess = 0).  A guess that already meets outer_tol returns it unchanged
 * with 0 iterations.  With params.use_graphs the CUDA graph is captured separately for
 * the two kinds of start.  ERR_ARG for a null opts or zero_guess not 0 or 1. */
int wcmg_solve_ex(wcmg_ctx* ctx, const void* b, void* x, int nrhs, const wcmg_solve_opts* opts, int where,
                  void* stream, wcmg_stats* st);

/* Batched solve over n independent contexts, e.g. lattices of uneven sizes: each
 * ctxs[i] solves D_i x_i = b_i (nrhs[i] fields, layouts of ctxs[i]) exactly as
 * wcmg_solve with params.use_graphs = 1 would.  All n solves are captured into ONE
 * CUDA graph, one branch per context with device-side stopping tests, and run by
 * a single graph launch on `stream`, so the small lattices fill the SMs that the
 * large one leaves idle.  The first call with a given (contexts, nrhs) runs the n
 * solves host-driven one after another (this allocates every workspace); the
 * second captures; later calls replay.  Every context must have finished its
 * setup, use the plain multigrid coarse mode, and appear once.  st (nullable)
 * is an array of n stats.  Returns the first error of any context
 * (ERR_NOT_CONVERGED if a context stopped at outer_maxiter). */
int wcmg_solve_batch(wcmg_ctx* const* ctxs, int n, const void* const* b, void* const* x, const int* nrhs,
                     int where, void* stream, wcmg_stats* st);

/* Launch shape of the nine-point coarse apply (K4 / K4m).  Fixed rule: one rhs ->
 * the one-rhs kernel (kind 0); several rhs -> the rhs-tile kernel (kind 1); BF16
 * links with >= 8 rhs -> the tcgen05 tensor-core kernel (kind 2).  Kind 3 (one rhs)
 * is a persistent streaming pipeline: each CTA keeps `stages` bulk copies of
 * `parts`-row chunks of the link matrices in flight ahead of the arithmetic.  Kind 4
 * (BF16 links, >= 2 rhs) is the tcgen05 kernel fed by bulk copies: warp-specialised,
 * persistent over (site, rhs tile), `stages` operand stages, MMA M = `threads`.
 * Kind 5 (one rhs) reads the five-block copy of params.coarse_sigma3 (Galerkin
 * operators only). */
typedef struct wcmg_tile {
  int kind;             /* 0 one-rhs kernel, 1 rhs-tile SIMT kernel, 2 tensor-core kernel,
                           3 one-rhs streaming kernel, 4 tensor-core kernel fed by bulk copies,
                           5 one-rhs kernel on the five-block storage, -1 none */
  int rhs_per_cta;      /* kind 1: 1, 4 or 8 rhs per CTA */
  int parts;            /* kinds 0, 1, 5: CTAs sharing one coarse site's rows (kind 1: 0 = automatic);
                           kind 3: link rows per staged chunk; kind 4: TMEM accumulators, 1 or
                           2 (0 = 2) */
  int threads;          /* kinds 0, 3, 5: threads per CTA (kinds 0, 5: 64 .. 512, multiple of 32;
                           kind 3: 128, 256 or 512); kind 4: MMA M, 64 or 128 (>= nbasis) */
  int ntile;            /* kinds 2, 4: rhs per MMA N tile (kind 2: 16, 32, 48 or 64; kind 4: a
                           multiple of 8 up to 64) */
  int source;           /* 0 fixed rule, 1 autotuner, 2 wcmg_set_coarse_tile */
  int candidates;       /* shapes the autotuner timed (fixed rule included) */
  int stages;           /* kinds 0, 5: link rows in flight per warp (0 or 1: one, 2: two);
                           kind 3: chunks in flight (2 .. 8); kind 4: operand stages (2 .. 8) */
  double us;            /* autotuner: time per apply of the chosen shape (back-to-back applies) */
  double us_default;    /* autotuner: time per apply of the fixed rule */
} wcmg_tile;

/* The tile the next full coarse apply of `level` with nrhs rhs at `prec` will use
 * (prec F64: FP64 links; F32: FP32 vectors on the level's params.coarse_link_prec
 * storage).  No GPU work.  ERR_STATE before the level's coarse operator exists. */
int wcmg_get_coarse_tile(wcmg_ctx* ctx, int level, int nrhs, int prec, wcmg_tile* out);

/* Run the autotuner now for (level, nrhs, prec): every candidate shape is timed
 * with CUDA events on the level's own links and the fastest is kept for later
 * applies.  cold = 0: 10 back-to-back applies after 2 warm-up applies (links
 * partly L2-resident, as inside a Krylov loop; the mode of params.autotune);
 * cold = 1: the median of 9 single applies, each after a 256 MiB scratch write
 * that evicts L2 (links streamed from HBM).  Synchronises `stream`. */
int wcmg_tune_coarse(wcmg_ctx* ctx, int level, int nrhs, int prec, int cold, void* stream, wcmg_tile* out);

/* Force a tile for (level, nrhs, prec); t->kind = -1 clears it (back to the
 * fixed rule, or the autotuner when params.autotune = 1).  ERR_ARG if the shape
 * is not valid for the level (e.g. kind 2 without BF16 links, kind 5 without the
 * five-block copy of params.coarse_sigma3). */
int wcmg_set_coarse_tile(wcmg_ctx* ctx, int level, int nrhs, int prec, const wcmg_tile* t);

/* Self-test of the library's bounded device-side waits (every mbarrier wait of the
 * bulk-copy and tensor-core kernels gives up after a fixed number of polls, sets the
 * context's device-wait word and lets its CTA finish; the next call that checks the word
 * returns WCMG_ERR_TIMEOUT and clears it).  Launches one kernel whose single thread waits,
 * at most `polls` (0 .. 2^26) polls, on an mbarrier phase that nothing completes, then
 * checks the word the same way.  Returns WCMG_ERR_TIMEOUT when the mechanism works (the
 * context stays usable), WCMG_ERR_ARG for polls out of range. */
int wcmg_check_bounded_wait(wcmg_ctx* ctx, long long polls, void* stream);

/* Change params.profile of an existing context (no GPU work). */
int wcmg_set_profile(wcmg_ctx* ctx, int mask);
/* Per-kernel-class counters accumulated over the context's lifetime
 * (out: WCMG_NKCLASS entries).  wcmg_setup / wcmg_solve report their own share. */
int wcmg_get_kstats(wcmg_ctx* ctx, wcmg_kstat* out);

/* Operator applications the context has issued from the host since wcmg_create, by
 * kind and level (out: WCMG_NOPC x WCMG_MAX_LEVELS entries, kind-major):
 *   WCMG_OPC_APPLY     D_level applied to one field (the full nine-point operator at
 *                      any precision, the smoother's included; counted per rhs)
 *   WCMG_OPC_RESTRICT  P_level^dag applied to one field (per rhs)
 *   WCMG_OPC_PROLONG   P_level applied to one field (per rhs)
 *   WCMG_OPC_ORTHO     block orthonormalisations of level's near-null vectors (calls)
 *   WCMG_OPC_COARSEN   coarsenings D_{level+1} = P^dag D P (calls; their masked stencils
 *                      and restrictions are not counted under the other kinds)
 * Work inside a replayed CUDA graph is issued by the device and is not counted; a
 * host-driven solve counts every application.  No GPU work. */
#define WCMG_NOPC 5
enum { WCMG_OPC_APPLY = 0, WCMG_OPC_RESTRICT = 1, WCMG_OPC_PROLONG = 2, WCMG_OPC_ORTHO = 3, WCMG_OPC_COARSEN = 4 };
int wcmg_get_opcounts(wcmg_ctx* ctx, long long* out);

/* Allocation-free block orthonormalisation of fine-level near-null vectors.
 * The paper has no counterpart.  It is for callers that cannot allocate device
 * memory: code whose device memory all belongs to another allocator (for example
 * a host framework's caching pool) and that must not call cudaMalloc/cudaFree,
 * which synchronise the whole device and can fail at run time once the pool
 * holds the memory.  Result: what wcmg_set_nullvecs followed by
 * wcmg_get_nullvecs return on the fine level (FP64 Q factor with positive real
 * diag(R) for every aggregate and chirality), with no context.
 *   vecs_in   device pointer, complex128 [nvec][V][4][3], V = product of dims
 *   vecs_out  device pointer, same layout (may equal vecs_in)
 *   dims      host int[4], fine extents Lx, Ly, Lz, Lt
 *   block     host int[4], aggregate extents (each divides its extent)
 * Working memory: a file-scope device array of WCMG_NOALLOC_MAX_ELEMS complex128
 * entries (4 MiB) that every device which loads the library keeps until the
 * process exits; nvec * V * 12 > WCMG_NOALLOC_MAX_ELEMS returns WCMG_ERR_ARG.
 * The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) with the device current.  Every call uses the same array, which keeps
 * the last call's contents: calls whose GPU work overlaps (several streams or
 * host threads) race and must be serialised by the caller.  No cudaMalloc,
 * cudaFree or allocating library routine is called.  Every call ends by copying
 * the rank-check word to a host variable and waiting for `stream` to finish
 * (cudaStreamSynchronize), so it returns only after its GPU work is complete.
 * Errors: WCMG_ERR_ARG (null pointer, sizes, nvec outside 1..32), WCMG_ERR_NAN
 * (rank-deficient aggregate), WCMG_ERR_CUDA. */
#define WCMG_NOALLOC_MAX_ELEMS 262144
int wcmg_block_orthonormalise_noalloc(const void* vecs_in, void* vecs_out, const int dims[4], const int block[4],
                                      int nvec, void* stream);

/* ---- Learned coarse correction (no counterpart in the paper) ----------------
 * A gauge-equivariant parallel-transport convolution (PTC) network N maps a fine
 * residual r to an approximation of the coarse-grid correction P D_c^-1 P^dag r
 * of the multigrid cycle (Sec. 2.1 operators).  Layer:
 *   out_i(x) = sum_j sum_h W_{ijh} (T_h in_j)(x),  h = 0 (identity),
 *   1 + 2 mu: U_mu(x) f(x + mu),  2 + 2 mu: U_mu(x - mu)^dag f(x - mu),
 * W_{ijh} complex 4x4 spin matrices; two linear layers 1 -> 12 -> 1 fields.
 * Weights: complex128 [3456] = W1 [12][1][9][4][4] followed by W2 [1][12][9][4][4].
 * The network runs in FP32 and needs the gauge field (wcmg_set_gauge). */
#define WCMG_PTC_HIDDEN 12
#define WCMG_PTC_NWEIGHTS 3456
int wcmg_ptc_set_weights(wcmg_ctx* ctx, const void* W, int where, void* stream);
int wcmg_ptc_get_weights(wcmg_ctx* ctx, void* W, int where, void* stream);
/* out = N(in) for nrhs fine fields (external fine layout). */
int wcmg_ptc_forward(wcmg_ctx* ctx, const void* in, void* out, int nrhs, int where, void* stream);
/* Given gout = dL/d conj(N(in)) (external fine layout), gin = dL/d conj(in) and
 * gW = dL/d conj(W) (complex128 [3456]) summed over the nrhs fields. */
int wcmg_ptc_backward(wcmg_ctx* ctx, const void* in, const void* gout, void* gin, void* gW, int nrhs, int where,
                      void* stream);

typedef struct wcmg_train_opts {
  int npairs;          /* training pairs held at a time (even split: Gaussian r and residuals
                          r = b - D M_0(b) of one cycle on a Gaussian b) */
  int batch;           /* fields per optimisation step */
  int steps;           /* Adam steps */
  int refresh;         /* > 0: a fresh pool of npairs pairs is generated every `refresh` steps
                          (pairs seen = npairs x pools); 0: one pool */
  double lr;           /* Adam learning rate */
  double target_tol;   /* coarse solves of the targets e = P GMRES(P^dag r) to this tolerance */
  uint64_t seed;       /* counter-based generator seed for the Gaussian fields */
} wcmg_train_opts;
typedef struct wcmg_train_stats {
  double loss_initial; /* mean ||N(r) - e||^2 / ||e||^2 over the first pool before training */
  double loss_final;   /* same over the last training pool after training */
  double ms_generate;  /* wall time of the pair generation */
  double ms_train;     /* wall time of the optimisation */
  double loss_heldout; /* after training, over a fresh pool never trained on */
  long long pairs_total; /* distinct pairs generated for training */
} wcmg_train_stats;
/* Generate training pairs with the current setup (wcmg_setup first; inner_prec
 * F32) and fit the PTC weights with Adam on the loss ||N(r) - e||^2 / ||e||^2
 * (Wirtinger gradients, the real gradient is twice their real/imaginary parts). */
int wcmg_ptc_train(wcmg_ctx* ctx, const wcmg_train_opts* opts, wcmg_train_stats* st, void* stream);

/* Checkpoint of the network: the weights as the network holds them (FP32 complex),
 * written bit for bit after an 8-byte tag "WCMGNET1" and four ints (hidden fields,
 * weight count, bytes per real, 0).  wcmg_load_net accepts only a file of this
 * network's shape (else ERR_ARG) and replaces the context's weights with it.
 * wcmg_save_net: ERR_STATE when the context has no weights. */
int wcmg_save_net(wcmg_ctx* ctx, const char* path);
int wcmg_load_net(wcmg_ctx* ctx, const char* path);

/* Coarse correction used by wcmg_solve's cycle (inner_prec F32 for the learned modes):
 *   WCMG_COARSE_MG          plain multigrid (default)
 *   WCMG_COARSE_WARMSTART   the coarsest GMRES starts from P^dag N(r) instead of 0
 *   WCMG_COARSE_LEARNED     the top-level coarse correction is N(r) (no coarse solve);
 *                           when an outer iteration reduces the residual estimate by
 *                           less than the factor fallback_ratio the solve falls back to
 *                           plain MG for the rest of the solve (fallback_ratio <= 0:
 *                           never; 0.9 is the library's default). */
typedef enum { WCMG_COARSE_MG = 0, WCMG_COARSE_WARMSTART = 1, WCMG_COARSE_LEARNED = 2 } wcmg_coarse_mode;
int wcmg_set_coarse_mode(wcmg_ctx* ctx, int mode, double fallback_ratio);

/* Checkpoint of the setup (near-null vectors and coarse links of every level). */
int wcmg_save_setup(wcmg_ctx* ctx, const char* path);
int wcmg_load_setup(wcmg_ctx* ctx, const char* path);

#ifdef __cplusplus
}
#endif
#endif /* WCMG_H */
