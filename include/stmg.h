/*
 * stmg.h - C ABI of the GB300 hp space-time multigrid library (libstmg.so).
 *
 * The library solves the slab systems of the tensor-product space-time finite element
 * discretisation of the instationary Stokes equations of Margenberg, Bause and Munch,
 * "An hp multigrid approach for tensor-product space-time finite element
 * discretizations of the Stokes equations" (arXiv 2502.09159):
 * Q_{r+1}/P_r^disc in space on a uniform mesh of [0,1]^d (d = 2, 3), DG(k) in time,
 * time marching slab by slab (Problem LocAlg), FGMRES preconditioned by one hp
 * space-time V-cycle (Alg. 1) with cell or vertex-star Vanka smoothing (Eq. vanka).
 * All compute runs in the library's own CUDA kernels for sm_103a.
 *
 * ---------------------------------------------------------------------------------
 * Conventions shared by every call
 * ---------------------------------------------------------------------------------
 * Status.  Every call returns STMG_OK (0) or one of the STMG_ERR_* codes below; no
 *   exception or abort crosses the ABI.  stmg_status_string() names a code.
 *
 * Memory.  Vector arguments are DEVICE pointers on the current CUDA device, owned by
 *   the caller, 256-byte aligned (what cudaMalloc / torch return), not aliasing one
 *   another unless a call says so.  "prec" selects their element type:
 *   STMG_FP64 -> double, STMG_FP32 -> float.  The handle owns its hierarchy, patch
 *   inverses and work vectors; stmg_destroy frees them.  The only host-pointer calls
 *   are stmg_solve_slab_host and stmg_march_host (host vectors in, host vectors out) and
 *   the info/config structs.
 *
 * Streams.  Calls enqueue work on the handle's stream (stmg_set_stream; default: the
 *   legacy default stream) and return without waiting, except stmg_create,
 *   stmg_solve_slab, stmg_solve_slab_host, stmg_march_host and stmg_get_profile, which
 *   synchronise the stream.  A handle must not be used from two host threads at once.
 *
 * Slab vector layout (Eq. DefX / DefSubvec, per slab):
 *     [ V^1 ... V^{k+1} , P^1 ... P^{k+1} ]                      length D
 *   With n_sub > 1 subintervals per system the temporal dofs are numbered subinterval by
 *   subinterval, a = j (k+1) + b, and the vector is [V^1 .. V^{n_sub (k+1)}, P^1 .. ]
 *   (all velocities, then all pressures; the paper's Eq. SubStrGloVec orders the same
 *   unknowns subinterval-major, a permutation of this layout).
 *   V^a  velocity at temporal dof a (Lagrange basis at the right Gauss-Radau points,
 *        Eq. BasYk), component-major: v_x over all velocity nodes, then v_y (, v_z).
 *        Velocity nodes: the ((r+1) n + 1)^d grid of the Q_{r+1} Gauss-Lobatto nodes,
 *        lexicographic with x fastest.
 *   P^a  pressure at temporal dof a, cell-major (cells lexicographic, x fastest),
 *        C(r+d, d) modes per cell: the orthonormal Legendre products
 *        L_i(xi) L_j(eta) (L_l(zeta)) of total degree <= r on the cell,
 *        L_i(xi) = sqrt(2i+1) P_i(2 xi - 1), ordered by total degree, then z degree,
 *        then y degree.
 *   D = (k+1) (d ((r+1) n + 1)^d + C(r+d, d) n^d); boundary velocity dofs included.
 *
 * Slab operator (Eq. InAlg, DefDtauh, with the viscosity of Problem DVP):
 *     S = [ K_tau (x) M_h + M_tau (x) nu A_h    -M_tau (x) B_h^T ]
 *         [ -M_tau (x) B_h                       0               ]
 *   with the boundary velocity rows and columns replaced by the identity (Dirichlet
 *   data; non-homogeneous data enter the right-hand side through stmg_dirichlet_lift).
 *   The continuity rows carry a minus sign (the spatial part is
 *   symmetric); solutions and smoother corrections are unaffected by that choice.
 *   The pressure is determined up to one constant per temporal dof; solutions from
 *   stmg_solve_slab are returned as computed (compare them after removing the mean).
 */
#ifndef STMG_H
#define STMG_H

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define STMG_OK                0
#define STMG_ERR_ARG           1   /* invalid argument (NULL, out of range, bad config)   */
#define STMG_ERR_OOM           2   /* device or host allocation failed / does not fit      */
#define STMG_ERR_NOT_CONVERGED 3   /* FGMRES hit gmres_max_iter before rel_tol            */
#define STMG_ERR_BREAKDOWN     4   /* Arnoldi breakdown without convergence               */
#define STMG_ERR_NONFINITE     5   /* NaN/Inf in the right-hand side or the iteration     */
#define STMG_ERR_CUDA          6   /* a CUDA runtime call failed                           */
#define STMG_ERR_UNIMPLEMENTED 7   /* combination not built (e.g. r > 4 on the GPU)       */
#define STMG_ERR_SINGULAR      8   /* a patch or coarse matrix could not be inverted       */
#define STMG_ERR_TOO_LARGE     9   /* level larger than stmg_smooth_noalloc's fixed scratch */
#define STMG_ERR_TIMEOUT      10   /* a bounded wait inside a kernel expired (device flag)  */

/* precisions */
#define STMG_FP64 0
#define STMG_FP32 1

/* smoother kinds (per level) */
#define STMG_CELL 0   /* cell patches (Eq. vanka0)                                  */
#define STMG_VSP  1   /* vertex-star patches (remark after Eq. vanka)               */

#define STMG_MAX_LEVELS 24

typedef struct stmg_handle stmg_handle;

/* Problem and solver configuration.  stmg_default_config fills every field. */
typedef struct {
  int    dim;              /* 2 or 3                                                     */
  int    n_cells;          /* cells per direction on the finest level (>= 1)             */
  int    r, k;             /* Q_{r+1}/P_r^disc in space (1 <= r <= 4), DG(k) (0 <= k <= 3)*/
  double nu;               /* viscosity                                                  */
  double T;                /* final time; slabs have length tau = T / n_slabs           */
  int    n_slabs;
  /* hierarchy: n_levels = 0 selects the default rule (Alg. 2/3, the reading pinned by
     Table 2(b)); otherwise level_n/r/k[0..n_levels-1] list the levels fine -> coarse.
     Consecutive levels must differ by n -> n/2 (h in space) or r -> r' < r (p in space)
     or neither, and optionally k -> k' <= k (p in time).  The last level is solved
     directly. */
  int    n_levels;
  int    level_n[STMG_MAX_LEVELS], level_r[STMG_MAX_LEVELS], level_k[STMG_MAX_LEVELS];
  int    smoother[STMG_MAX_LEVELS];   /* STMG_CELL or STMG_VSP, per level (fine -> coarse) */
  double omega;            /* Vanka damping (Eq. vanka), default 0.7                     */
  int    nu1, nu2;         /* pre/post smoothing steps, default 1, 1                     */
  int    precond_precision;/* precision of the V-cycle inside stmg_solve_slab            */
  int    precisions;       /* bit mask of precisions to set up: 1 = FP64, 2 = FP32      */
  int    gmres_max_iter;   /* Krylov basis size; no restarts (default 200)               */
  double rel_tol;          /* stop when ||b - S x||_2 <= rel_tol ||b||_2 (default 1e-8) */
  int    use_graphs;       /* capture each V-cycle in a CUDA graph (default 1)           */
  int    sweep_variant;    /* Vanka sweep kernel: 0 = chosen by the tuner (default),
                              1 = one thread block per group of patches,
                              2 = persistent TMA-pipelined (one CTA per SM,
                              cp.async.bulk + mbarrier; patches with B <= 512),
                              3 = pipelined block sweep (the first loads of every row
                              issued before the residual gather, double-buffered rounds;
                              patches with B <= 512, FP32/FP64 inverses)                */
  int    autotune;         /* 1 (default): stmg_create times the candidate launch shapes
                              of every level (see stmg_autotune) and keeps the fastest  */
  int    coarse_n;         /* coarsest mesh of the default hierarchy (Alg. 2's h_0 =
                              1/coarse_n, a power of 2 <= n_cells; default 1, the rule
                              Table 2(b) pins); the coarsest level is solved directly    */
  int    k_min;            /* lowest temporal degree of the default hierarchy's
                              polynomial coarsening in time (Alg. 2's r_0 for k; default
                              1 as in the paper's runs; k_min >= k keeps DG(k) on every
                              level)                                                     */
  int    n_sub;            /* DG(k) subintervals per system (a macro time step, Remark
                              rem:GLSP; default 1 = time marching, Eq. AlgSysTMS); the
                              system of n_sub subintervals is solved at once and the
                              temporal multigrid is p-coarsening per subinterval, with
                              h-coarsening in time by level_nsub / time_h.  tau = T /
                              (n_slabs n_sub); n_sub (k + 1) <= 8                       */
  int    half_inverses;    /* 1: the FP32 V-cycle stores its patch inverses in FP16, each
                              row scaled to [-1, 1] with an FP32 row scale (half the
                              bytes of the dominant stream; the sweep accumulates in
                              FP32).  Default 0 (FP32 inverses).  Not an option of the
                              paper: an extension of its mixed-precision form.          */
  int    transfer_variant; /* grid-transfer kernels: 0 = chosen by the tuner (default),
                              1 = per coarse cell (shared-memory sum factorisation,
                              atomics on shared fine nodes), 2 = gather form, one
                              thread per output value (2D levels only; 3D levels and
                              other shapes keep 1).  Both compute P and P^T exactly
                              (App. A); they differ in rounding order only.             */
  int    apply_variant;    /* operator kernels: 0 = chosen by the tuner (default),
                              1 = one thread block per group of cells (shared-memory sum
                              factorisation, atomics on shared nodes), 2 = node-centred
                              form on tiles of cells, every output written once, 3 =
                              register-resident form, one thread per (cell, temporal dof)
                              (FP32 up to Q5, FP64 up to Q3, k + 1 <= 4), 4 = its
                              pair-split form, two threads per (cell, temporal dof), each
                              with half of the cell's node columns (Q3, k + 1 <= 4).  2, 3
                              and 4 are for 2D levels; 3D levels and shapes that 3 does
                              not cover keep 1 (resp. 1 or 2); levels that 4 does not
                              cover take 3.  Same operator; they differ in rounding order
                              only.                                                      */
  int    persistent;       /* levels below the finest in one persistent kernel (grid-wide
                              barriers between its sweeps, residuals, transfers and the
                              coarse product): 0 = never, 1 = where the tuner finds it
                              faster (default), 2 = from the first level it covers (2D
                              Q2/P1 levels, k + 1 <= 4, patches of <= 256 dofs).  Same
                              V-cycle; rounding order only.                              */
  int    level_nsub[STMG_MAX_LEVELS];  /* explicit hierarchies: subintervals of each level's
                              temporal mesh (0 = n_sub); the first must equal n_sub and each
                              must divide the previous one.  A level of fewer subintervals
                              covers the same system span T / n_slabs with longer ones: the
                              temporal h-coarsening of App. A (Eq. DeftPrRe), transfers =
                              the canonical embedding of the coarser DG(k) function and
                              its transpose                                              */
  int    time_h;           /* default hierarchy with n_sub > 1: 1 = first halve the
                              subintervals on the finest space level (n_sub -> n_sub/2 ->
                              ... -> 1, h in time), then the spatial and temporal-degree
                              levels on one subinterval; 0 (default) = p in time per
                              subinterval only (the paper's choice for macro steps)      */
  int    arnoldi_form;     /* the cooperative Arnoldi step (CGS2) of FGMRES: 0 (default) =
                              the block's rows of w held in registers across its three
                              passes where they fit (at most 16 basis vectors, at most
                              2048 rows per SM), else 1 = the split-pass form that reads w
                              and V from memory in every pass; both give the same sums   */
  int    fuse_transfers;   /* 1 (default): on 2D register-resident levels of the FP32
                              V-cycle, the residual after presmoothing is restricted in
                              the same launch (no fine residual vector), and the
                              prolongation of the coarser level's correction runs inside
                              the first postsmoothing residual (one launch instead of
                              two each way); 0: separate kernels                        */
} stmg_config;

typedef struct {
  int       n, r, k;       /* cells per direction, spatial and temporal degree          */
  int       n_sub;         /* subintervals of the level's temporal mesh in one system     */
  long long size;          /* D of this level                                            */
  long long n_vel;         /* velocity dofs per temporal dof (d ((r+1)n+1)^d)           */
  long long n_pres;        /* pressure dofs per temporal dof (C(r+d,d) n^d)             */
  int       smoother;      /* STMG_CELL / STMG_VSP (coarsest level: -1, direct solve)    */
  int       patch_size;    /* B, dofs per patch (0 on the coarsest level)               */
  long long n_patches;
  int       n_patch_classes;/* distinct patch matrices inverted at setup                 */
  long long inverse_bytes[2]; /* stored patch-inverse bytes for FP64 / FP32 (0: none)    */
  int       sweep_variant[2];            /* per precision: 1 block, 2 TMA, 3 pipelined block */
  int       patches_per_block[2];        /* block sweep launch shape, per precision          */
  int       apply_cells_per_block[2];    /* apply / residual launch shape, per precision:
                                            cells per block (apply_variant 1), threads
                                            per block (3: 64, or fewer so that every SM
                                            gets the same number of items)           */
  int       transfer_cells_per_block[2]; /* transfers to the next coarser level; 0: the
                                            gather form (one thread per value)           */
  int       streaming;     /* 1: the sweep reads the stored inverses with evict-first loads
                              (inverses larger than about a third of L2), so that the
                              coarser levels' inverses stay L2-resident                   */
  int       apply_variant[2]; /* per precision: 1 = one thread block per group of cells
                                 (apply_cells_per_block), 2 = node-centred 2D form on tiles
                                 of apply_tile cells (no atomics), 3 = register-resident
                                 2D form (one thread per cell and temporal dof), 4 = its
                                 pair-split form (two threads per cell and temporal dof) */
  int       apply_tile[2][2]; /* per precision: cells per block in x and y (variant 2)    */
  int       persistent[2];    /* per precision: 1 if the level runs inside the persistent
                                 multigrid kernel (its launch shapes above then unused)    */
  int       sweep_unroll[2];  /* per precision: column chunks per load round of the block
                                 sweeps (4 or 8)                                           */
} stmg_level_info_t;

typedef struct {
  int    iterations;       /* FGMRES iterations (= V-cycles) used                        */
  double rel_residual;     /* true ||b - S x||_2 / ||b||_2 at exit, in FP64             */
  int    status;           /* STMG_OK or STMG_ERR_NOT_CONVERGED / _BREAKDOWN / _NONFINITE */
  double seconds;          /* wall time of the call                                      */
} stmg_solve_info;

/* Per-category device time, the split of Sec. 5.2 (Fig. lid-strong-scale-rel). */
#define STMG_PROF_SMOOTHER    0   /* Vanka sweeps inside the V-cycle                        */
#define STMG_PROF_MG_OTHER    1   /* residuals, transfers, coarse solve inside the V-cycle  */
#define STMG_PROF_OPERATOR    2   /* operator applications outside the V-cycle (FGMRES)     */
#define STMG_PROF_OTHER       3   /* orthogonalisation, vector updates, right-hand sides    */
#define STMG_PROF_FINE_SWEEP  4   /* finest-level sweeps only (subset of SMOOTHER)          */
#define STMG_PROF_N           5

/* ---- setup ----------------------------------------------------------------------- */

/* Fill *cfg with defaults: dim 2, n 8, r 1, k 1, nu 1, T 1, 4 slabs, default hierarchy,
   cell smoothers, omega 0.7, nu1 = nu2 = 1, FP64 preconditioner, both precisions set
   up, 200 iterations, rel_tol 1e-8, graphs on. */
int  stmg_default_config(stmg_config* cfg);

/* Tuning cache: if the environment variable STMG_TUNE_CACHE names a file, stmg_create with
   autotune = 1 reads the launch shapes of an earlier tuning of the same configuration from
   it (and skips the timing), or tunes and appends them to it.  For runs whose timings would
   be distorted, e.g. under a profiler.  A file that cannot be read or written is ignored. */

/* Build the hierarchy (Alg. 2/3 or the explicit list), the level operators, transfers,
   Vanka patch inverses (Eq. vanka0: the global submatrix R_T S R_T^T of every patch,
   inverted in FP64 by Gauss-Jordan elimination with partial pivoting once per distinct
   patch matrix and stored per patch, rounded to FP32 where requested) and the coarsest
   level's bordered inverse.  Synchronous.  On failure *out is NULL. */
int  stmg_create(const stmg_config* cfg, stmg_handle** out);

/* Free everything the handle owns (NULL is accepted). */
void stmg_destroy(stmg_handle* h);

/* Enqueue all further work on `stream` (a cudaStream_t; NULL = legacy default stream). */
int  stmg_set_stream(stmg_handle* h, void* stream);

int  stmg_num_levels(const stmg_handle* h, int* n_levels);

/* Level 0 is the finest, n_levels-1 the coarsest. */
int  stmg_level_info(const stmg_handle* h, int lvl, stmg_level_info_t* info);

/* ---- the hot path ------------------------------------------------------------------ */

/* y = S_lvl x, matrix-free (Sec. 4.5): per cell, sum-factorised Q_{r+1} mass and
   Laplacian, B_h and B_h^T for all k+1 temporal dofs, combined with K_tau and M_tau.
   x, y: length D_lvl, precision prec; must not alias. */
int  stmg_apply(stmg_handle* h, int lvl, int prec, const void* x, void* y);

/* y = S_lvl^T x.  M_h, A_h and M_tau are symmetric and the two B blocks of Eq. InAlg are
   each other's transposes, so S^T is S with K_tau transposed; the boundary identity rows
   and columns are unchanged.  For adjoint (gradient) computations, e.g. training the
   learned initial guess on the residual norm.  x, y must not alias. */
int  stmg_apply_transpose(stmg_handle* h, int lvl, int prec, const void* x, void* y);

/* r = b - S_lvl x (App. B, step 1 of Alg. 4/5).  r must not alias b or x. */
int  stmg_residual(stmg_handle* h, int lvl, int prec, const void* b, const void* x, void* r);

/* `steps` Vanka smoothing iterations x <- x + omega W (b - S x) (Eq. vanka) on level
   lvl (not the coarsest), W = sum_T R_T^T D_T [R_T S R_T^T]^{-1} R_T with the valence
   weights D_T.  x is updated in place. */
int  stmg_smooth(stmg_handle* h, int lvl, int prec, const void* b, void* x, int steps);

/* stmg_smooth for callers that must not have device memory allocated for them while
   they run: a process whose device memory is given out only by its own pool allocator,
   or a time-critical loop that cannot absorb the implicit synchronisation of
   cudaMalloc/cudaFree.  Same arguments and result as stmg_smooth, but the residual lives
   in a fixed device array inside the library (STMG_NOALLOC_MAX_ENTRIES values, 8 MB), so
   the call allocates nothing.  The paper has no counterpart; it is an interface
   convenience.
   - The array's 8 MB are taken on a device when the first handle is created there
     (stmg_create looks up the array's device address once per device, which loads the
     library's module holding it; STMG_ERR_OOM if that fails) and are held until the
     process exits.  Create the handle before any stream capture.  A device reset
     (cudaDeviceReset) invalidates the address, as it invalidates every handle.
   - Levels with more than STMG_NOALLOC_MAX_ENTRIES dofs are rejected with
     STMG_ERR_TOO_LARGE before any work is queued.
   - All calls share the one array and it keeps whatever the last call left in it (each
     step overwrites the whole residual before reading it): calls that can overlap on the
     GPU, from different streams or handles, race with each other; order them on one
     stream.
   - Like stmg_smooth and the other asynchronous calls, it does not report an expired
     bounded wait inside a kernel (the TMA sweep's); stmg_device_status does. */
#define STMG_NOALLOC_MAX_ENTRIES (1 << 20)
int  stmg_smooth_noalloc(stmg_handle* h, int lvl, int prec, const void* b, void* x, int steps);

/* One Vanka correction without the residual: x += omega W res.  (The sweep kernel.) */
int  stmg_vanka_sweep(stmg_handle* h, int lvl, int prec, const void* res, void* x);

/* b_c = T_restrict r_f between level lvl_fine and lvl_fine+1 (App. A: transpose of the
   canonical prolongation, in space (h or p) and in time (p)).  b_c is overwritten. */
int  stmg_restrict(stmg_handle* h, int lvl_fine, int prec, const void* r_f, void* b_c);

/* x_f += T_prolong y_c between level lvl_fine+1 and lvl_fine (App. A, Eq. DeftTps,
   DefoTsl); boundary velocity entries of x_f are left unchanged. */
int  stmg_prolongate_add(stmg_handle* h, int lvl_fine, int prec, const void* y_c, void* x_f);

/* Direct solve on the coarsest level (Alg. 1, step 3): x = G b with the FP64 bordered
   inverse that fixes the pressure mean of every temporal dof; FP32 vectors are
   converted on the fly, the product runs in FP64. */
int  stmg_coarse_solve(stmg_handle* h, int prec, const void* b, void* x);

/* x = V(b): one hp space-time V-cycle (Alg. 1, App. B) from a zero initial guess on the
   finest level; the multigrid runs in precision prec (FP32: b is rounded, x returned in
   FP64).  b, x: FP64, length D_0. */
int  stmg_vcycle(stmg_handle* h, int prec, const double* b, double* x);

/* b = F + (C_tau (x) M_h) V_prev (right-hand side of Eq. AlgSysTMS): interior velocity
   rows of temporal dof a get phi_a(t_{n-1}^+) M_h v_prev, v_prev = the last temporal
   velocity V^{k+1} of x_prev (a full previous-slab vector, boundary values included: the
   jump term couples the whole finite-element function); x_prev = NULL means v_prev = 0.
   Boundary rows of b are copied from F.
   F: the forcing part (Eq. DefFn), FP64, length D_0; b must not alias F or x_prev. */
int  stmg_slab_rhs(stmg_handle* h, const double* F, const double* x_prev, double* b);

/* Non-homogeneous Dirichlet data: y = b - S_{.,D} g on the interior rows (S's columns of
   the boundary velocity dofs applied to the boundary values of g; the interior entries of
   g are not read) and y = g on the boundary rows.  Solving S x = y then gives the
   solution with x = g on the boundary (Eq. InAlg with the boundary values moved to the
   right-hand side).  g, b, y: device FP64, length D_0; y must not alias g or b.  Uses the
   finest level's FP64 operator, which every handle has (FGMRES runs in FP64). */
int  stmg_dirichlet_lift(stmg_handle* h, const double* g, const double* b, double* y);

/* Solve S x = b on the finest level with FGMRES (right preconditioning by one V-cycle
   in cfg.precond_precision, CGS2 orthogonalisation in FP64, no restart).  x: initial
   guess in, solution out (FP64); its boundary entries are first set to b's (the
   boundary rows of S are the identity, and the V-cycle's corrections vanish there).
   Synchronous.  Returns info->status. */
int  stmg_solve_slab(stmg_handle* h, const double* b, double* x, stmg_solve_info* info);

/* Same with HOST vectors (any host memory; pinned memory gives faster copies): copies b
   and x in, solves, copies x out.  For end-to-end measurement and callers without
   device buffers.  Synchronous. */
int  stmg_solve_slab_host(stmg_handle* h, const double* b_host, double* x_host,
                          stmg_solve_info* info);

/* Time marching with HOST buffers (Eq. AlgSysTMS, slab by slab, V_0 = 0): for slab
   s = 0 .. n_slabs-1 the right-hand side is
     kind STMG_MARCH_FORCING:  b_s = F_s + (C_tau (x) M_h) V_{s-1}      (stmg_slab_rhs)
     kind STMG_MARCH_BOUNDARY: b_s = lift of the boundary values g_s (stmg_dirichlet_lift)
                               applied to (C_tau (x) M_h) V_{s-1}, no forcing
   with in_host + s D holding F_s (forcing part, Eq. DefFn) or g_s (slab vector whose
   boundary entries are the Dirichlet values); S x_s = b_s is solved from a zero initial
   guess (stmg_solve_slab) and x_s is written to x_host + s D.  The host-to-device copy of
   slab s+1's input and the device-to-host copy of slab s-1's solution run on an internal
   copy stream while slab s is solved (pinned host memory makes them asynchronous).
   in_host, x_host: host FP64 arrays of n_slabs * D values.  infos: n_slabs entries or
   NULL.  Synchronous.  Stops at the first slab whose solve does not return STMG_OK and
   returns that status; the slabs before it are complete in x_host. */
#define STMG_MARCH_FORCING  0
#define STMG_MARCH_BOUNDARY 1
int  stmg_march_host(stmg_handle* h, int n_slabs, int kind, const double* in_host, double* x_host,
                     stmg_solve_info* infos);

/* ---- forcing (Eq. DefFn) ----------------------------------------------------------- */

/* Number of quadrature points per cell used for the forcing: (r+4)^d Gauss points. */
int  stmg_forcing_npoints(const stmg_handle* h, int* nq_per_cell);

/* Physical coordinates of the forcing quadrature points, device FP64 array
   [cell][q][dim] (cells lexicographic, points x fastest). */
int  stmg_forcing_points(stmg_handle* h, double* xq);

/* Times t_n^a of the n_sub (k+1) Radau points of system `slab` (0-based; subinterval by
   subinterval), host FP64 array. */
int  stmg_slab_times(const stmg_handle* h, int slab, double* t_host);

/* F: (F^a)_i = tau/2 w_a <f(t_n^a), chi_i> by the Gauss rule above, from fq = device FP64
   [a][cell][q][dim] samples of f at the points and times above.  F (device FP64,
   length D_0) is overwritten; boundary and pressure entries are 0. */
int  stmg_assemble_forcing(stmg_handle* h, const double* fq, double* F);

/* ---- cell tensors and temporal extrapolation (learned initial guess, stmg_net.h) ---- */

/* Channels of a cell tensor on level lvl: C = (k+1) (d (r+2)^d + C(r+d, d)). */
int  stmg_cells_channels(const stmg_handle* h, int lvl, int* C);

/* cells[c][ch] = (float)((x - base)[map(c, ch)] * inv_scale[ch]), computed in FP64: one
   row of C channels per cell (cells lexicographic, x fastest).  Channels: the velocity
   values (temporal dof a, component, local node (r+2)^d with x fastest), then the
   pressure modes (temporal dof a, mode), i.e. every slab entry that belongs to the cell;
   a velocity node shared by several cells is copied into each.  x, base: device FP64
   slab vectors of level lvl (base may be NULL = 0); inv_scale: device FP32 [C] (NULL =
   1); cells: device FP32 [n^d][C]. */
int  stmg_cells_gather(stmg_handle* h, int lvl, const double* x, const double* base, const float* inv_scale,
                       float* cells);

/* The same gather into columns channel_offset .. channel_offset + C - 1 of a wider tensor
   with rows of row_stride floats (cells[c * row_stride + channel_offset + ch]), e.g. to
   stack the cell tensors of several slabs along the channels.  row_stride >=
   channel_offset + C, else STMG_ERR_ARG. */
int  stmg_cells_gather_strided(stmg_handle* h, int lvl, const double* x, const double* base,
                               const float* inv_scale, float* cells, long long row_stride, int channel_offset);

/* x += the average over the copies of each entry of scale[ch] * cells[c][ch] (the
   inverse of the gather on consistent tensors), on every non-boundary entry; boundary
   velocity entries of x are left unchanged.  Sums run in FP64 in increasing cell order.
   scale: device FP32 [C] (NULL = 1).  x: device FP64, length D_lvl. */
int  stmg_cells_scatter_add(stmg_handle* h, int lvl, const float* cells, const float* scale, double* x);

/* The adjoint of stmg_cells_scatter_add: every copy of a non-boundary velocity dof g
   receives scale[ch] x[g] / (number of cells holding g); copies of boundary dofs get 0;
   pressure modes get scale[ch] x[g].  Computed in FP64, rounded to FP32.  x: device FP64
   slab vector of level lvl; scale: device FP32 [C] (NULL = 1); cells: device FP32 [n^d][C]. */
int  stmg_cells_gather_adjoint(stmg_handle* h, int lvl, const double* x, const float* scale, float* cells);

/* out[0] = sum_i x_i y_i over n FP64 entries (device pointers), deterministic (fixed-order
   per-block partial sums); asynchronous on the handle's stream. */
int  stmg_dot(stmg_handle* h, long long n, const double* x, const double* y, double* out);

/* x_next = the DG(k) polynomial of x_prev (Lagrange basis at the right Radau points,
   Eq. BasYk) evaluated at the next slab's Radau points, for every velocity and pressure
   entry: x_next^a = sum_b phi_b(s_a + 2) x_prev^b on the reference interval.  Exact for
   data that is polynomial of degree <= k in time.  x_prev, x_next: device FP64, length
   D_lvl, must not alias. */
int  stmg_extrapolate(stmg_handle* h, int lvl, const double* x_prev, double* x_next);

/* Remove the mean pressure of every temporal dof in place (the mode-0 coefficients of
   all cells are shifted by their average; the uniform mesh weights cells equally).  The
   pressure of the slab system is determined up to these constants, so b - S x is
   unchanged.  x: device FP64, length D_lvl. */
int  stmg_remove_pressure_mean(stmg_handle* h, int lvl, double* x);

/* ---- instrumentation ------------------------------------------------------------- */

/* Turn per-category CUDA-event timing on/off (off by default; adds events around
   kernels, so leave it off for headline timings). */
int  stmg_set_profiling(stmg_handle* h, int on);

/* Milliseconds and launch counts per STMG_PROF_* category since the last reset;
   synchronises.  reset != 0 zeroes the counters afterwards. */
int  stmg_get_profile(stmg_handle* h, double* ms, long long* launches, int reset);

/* Launch-parameter tuner: for every level and set-up precision, times the candidate
   launch shapes (sweep: 1/2/4/8 patches per block or the TMA-pipelined variant; apply and
   transfers: 1..32 cells per block) with CUDA events on the handle's own work vectors and
   keeps the fastest; cached V-cycle graphs are recaptured.  Synchronous.  stmg_create
   calls it when cfg.autotune = 1. */
int  stmg_autotune(stmg_handle* h);

/* Synchronise and report device-side failures: STMG_ERR_TIMEOUT if a bounded wait in a
   kernel (the TMA sweep's mbarrier waits) expired since the last check; clears the flag.
   stmg_solve_slab checks the same flag itself. */
int  stmg_device_status(stmg_handle* h);

/* Testing hook for failure handling without a GPU fault: arms the grid barrier of the next
   stmg_solve_slab's first Arnoldi step (the cooperative CGS2 launch) so that it cannot
   complete.  The barrier's bounded waits expire (after about a second), the kernel
   returns, and the solve reports STMG_ERR_TIMEOUT; the handle stays usable and the next
   solve runs normally.  STMG_ERR_UNIMPLEMENTED if the handle does not use the cooperative
   step. */
int  stmg_inject_wait_fault(stmg_handle* h);

/* Total number of this library's kernel launches since the handle was created. */
long long stmg_kernel_launches(const stmg_handle* h);

/* Algorithmic bytes of one Vanka sweep on level lvl in precision prec (stored inverses +
   gathered residual + weights + updated iterate). */
int  stmg_sweep_bytes(const stmg_handle* h, int lvl, int prec, double* bytes);

const char* stmg_status_string(int status);

/* ---- host-side introspection (no GPU needed) ---------------------------------------
 * The setup numerics that stmg_create runs on the host before uploading, callable from
 * a CPU-only process.  Host pointers; sizes as stated; no allocation is returned. */

/* Default level list (Alg. 2/3, the rule pinned by Table 2(b)) with coarsest mesh
   coarse_n and lowest temporal degree k_min (both 1 in the paper's runs):
   levels[3*i..3*i+2] = (n, r, k) fine -> coarse,
   *count levels (<= STMG_MAX_LEVELS). */
int  stmg_host_default_hierarchy(int n, int r, int k, int coarse_n, int k_min, int* levels,
                                 int* count);

/* 1D tables on [0,1] for degree r: Gauss-Lobatto nodes xi[r+2], M1/K1 [(r+2)^2] (mass,
   stiffness of the Lagrange basis), G1/N1 [(r+1)(r+2)] (int L_i ell_p', int L_i ell_p).
   NULL outputs are skipped. */
int  stmg_host_tables_1d(int r, double* xi, double* M1, double* K1, double* G1, double* N1);

/* DG(k) tables (Eq. GF, DefKMC): right Radau nodes/weights on [-1,1] [k+1], K [(k+1)^2]
   row-major, diagonal of M_tau [k+1], phi_a(t_{n-1}^+) [k+1]. */
int  stmg_host_time_tables(int k, double tau, double* nodes, double* weights, double* K,
                           double* Mdiag, double* phi_left);

/* Patch `patch` (STMG_CELL: cells lexicographic; STMG_VSP: vertices lexicographic) of the
   level (dim, n, r, k): dof list (slab indices, -1 boundary, -2 padding) [*B] and its FP64
   inverse [*B x *B] row-major.  dofs = inv = NULL only queries *B, *n_patches and the
   number of distinct patch matrices *n_classes. */
int  stmg_host_patch(int dim, int n, int r, int k, double nu, double tau, int kind,
                     long long patch, int* dofs, double* inv, int* B, long long* n_patches,
                     int* n_classes);

/* Number of patches containing each slab dof [*size]; valence = NULL queries *size. */
int  stmg_host_valence(int dim, int n, int r, int k, int kind, int* valence, long long* size);

/* Bordered coarse inverse of the level (dim, n, r, k) as used by stmg_coarse_solve,
   column-major [*D x *D] (D <= 6000); G = NULL queries *D. */
int  stmg_host_coarse_inverse(int dim, int n, int r, int k, double nu, double tau, double* G,
                              long long* D);

/* In-place inverse of the row-major n x n matrix A (host memory, caller-owned) by the
   routine stmg_create uses for patch matrices and the coarse bordered matrix: Gauss-Jordan
   with partial pivoting in FP64, blocked in panels of 32 columns for n >= 256 with the
   rows split over `threads` threads (0 = the machine's, at most 32).  Returns
   STMG_ERR_SINGULAR, A partly overwritten, when no pivot exceeds 1e-14 max|A|. */
int  stmg_host_invert(double* A, int n, int threads);

#ifdef __cplusplus
}
#endif
#endif /* STMG_H */
