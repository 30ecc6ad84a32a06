/*
 * hh.h - C ABI of the GB300 shifted-HSS Helmholtz solver.
 *
 * The library solves the Q1 finite-element discretisation of the indefinite
 * Helmholtz problem of Cotter, Hope-Collins & Knook (arXiv 2506.18694, Sec. 1,
 * Eq. "helmholtz strong primal"):
 *
 *     (-delta + i k)^2 u - lap u = f   in the unit square (dim 2) or cube (dim 3),
 *     u = 0 on the Dirichlet sides, du/dn - (-delta + i k) u = 0 on the Sommerfeld sides,
 *
 * in its primal weak form b_delta (Sec. 2) on a uniform grid of n cells per axis.
 * The discrete operator is B_delta = K + (-delta + i k)^2 M + (delta - i k) M_Gamma with
 * K the stiffness, M the mass and M_Gamma the boundary mass on Sommerfeld sides.
 *
 * Method: flexible GMRES in FP64 (Sec. 5.1) on B_delta u = b, right-preconditioned by
 * the shifted-HSS operator of Def. 4.1: ceil(k^theta) iterations of
 *     A_L u_{n+1} = (k-1)/(k+1) A_R u_n + 2k/(k+1) r,   u_0 = 0,
 *     A_L = K + (dh^2 - k^2 - 2 i dh k^2) M + (dh - i k^2) M_Gamma,
 *     A_R = -K + (k^2 - dh^2 - 2 i dh k^2) M + (-dh - i k^2) M_Gamma     (dh = delta_hat),
 * each A_L solve approximated by one multigrid V-cycle (scaled Jacobi smoothing,
 * full-weighting restriction R = P^T, bi/trilinear prolongation P) in complex FP32
 * or complex FP64.
 *
 * Batches: one hh_problem holds nb >= 1 independent problems on the same grid, each
 * with its own k, delta and delta_hat (hh_create_batch; hh_create_problem is nb = 1).
 * Every call works on all nb problems at once, in the same kernel launches; a problem
 * whose HSS loop or outer iteration has ended is skipped on the device, so each
 * problem's result is the one a batch of one would give, bit for bit.
 *
 * Data layout (every vector argument): nb consecutive blocks, block b holding problem
 * b's (n_l + 1)^dim complex nodal values of level l (level 0 is the finest,
 * n_l = n / 2^l), lexicographic with x fastest, real and imaginary parts interleaved:
 * double2 for HH_C128, float2 for HH_C64.  Device pointers must be 16-byte (c128) or
 * 8-byte (c64) aligned.  Entries at Dirichlet nodes of inputs are ignored; outputs hold
 * exact zeros there.
 *
 * Ownership: the caller owns every vector it passes; the library owns everything it
 * allocates for a problem (grid hierarchy, Krylov basis, CUDA graphs, streams) and
 * frees it in hh_destroy.  A problem is not thread-safe; distinct problems are
 * independent.  All calls are made on the device that was current at
 * hh_create_problem / hh_create_batch.
 *
 * Errors: every call returns an hh_status; no exception crosses the ABI and no
 * device code traps.  hh_last_error() returns a message for the last failing call
 * of the calling thread.
 */
#ifndef HH_H
#define HH_H

#include <stddef.h>

#if defined(__GNUC__)
#define HH_API __attribute__((visibility("default")))
#else
#define HH_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HH_OK = 0,
    HH_NOT_CONVERGED = 1,   /* max_outer reached; u holds the last iterate           */
    HH_ERR_INVALID = -1,    /* bad argument (see each call)                           */
    HH_ERR_OOM = -2,        /* device allocation failed                               */
    HH_ERR_CUDA = -3,       /* a CUDA runtime call failed                             */
    HH_ERR_NONFINITE = -4,  /* NaN or Inf met in the right side or the iteration      */
    HH_ERR_TIMEOUT = -5     /* a bounded device wait (grid-wide barrier) ran out      */
} hh_status;

/* Boundary tags of Sec. 1: Gamma (radiation condition) and dOmega_0 (u = 0). */
typedef enum { HH_BC_SOMMERFELD = 0, HH_BC_DIRICHLET = 1 } hh_bc;

/* Arithmetic of the multigrid V-cycles (the outer FGMRES is always FP64). */
typedef enum { HH_C128 = 0, HH_C64 = 1 } hh_precision;

/* Outer iteration on B_delta u = b, preconditioned by the shifted-HSS operator: flexible
 * GMRES (Sec. 5.1), or the preconditioned Richardson iteration u += P (b - B_delta u) that
 * the text after Def. 4.1 defines (the stationary iteration of the paper's Richardson
 * tables, Sec. 5.2); restart is ignored for the latter. */
typedef enum { HH_OUTER_FGMRES = 0, HH_OUTER_RICHARDSON = 1 } hh_outer;
/* multigrid smoother (options.smoother) */
typedef enum { HH_SMOOTH_JACOBI = 0, HH_SMOOTH_GMRES = 1 } hh_smoother;
/* discretisation (options.formulation) */
typedef enum { HH_FORM_PRIMAL = 0, HH_FORM_MIXED = 1 } hh_formulation;

/* Operators that hh_apply can apply (coefficient triples of the weak forms). */
typedef enum {
    HH_OP_K = 0,        /* stiffness                                     (Sec. 2) */
    HH_OP_M = 1,        /* mass                                          (Sec. 2) */
    HH_OP_MGAMMA = 2,   /* boundary mass on Sommerfeld sides             (Sec. 2) */
    HH_OP_AL = 3,       /* left HSS operator of Def. 4.1 (delta_hat)              */
    HH_OP_AR = 4,       /* right HSS operator of Def. 4.1 (delta_hat)             */
    HH_OP_B = 5,        /* B_delta of the outer problem                  (Sec. 2) */
    HH_OP_BHAT = 6      /* B_delta_hat, the shifted operator of Sec. 4            */
} hh_operator;

/* Uniform grid of the unit square/cube: dim in {2,3}, n cells per axis. */
typedef struct {
    int dim;
    int n;
} hh_grid;

typedef struct {
    double theta;        /* ceil(k^theta) inner HSS iterations per preconditioning (Def. 4.1) */
    int levels;          /* multigrid levels, coarsening factor 2 (Sec. 5.3 uses 4)           */
    int nu_pre;          /* Jacobi sweeps before restriction                                  */
    int nu_post;         /* Jacobi sweeps after prolongation                                  */
    int nu_coarse;       /* Jacobi sweeps on the coarsest level                               */
    int cycles_per_hss;  /* V-cycles per HSS iteration                                        */
    double omega;        /* Jacobi damping in (0, 2); 0 = automatic: 0.6 in 2D, 0.5 in 3D      */
    int restart;         /* FGMRES restart length                                             */
    int max_outer;       /* FGMRES iteration cap                                              */
    int precision;       /* hh_precision of the V-cycles                                      */
    int use_graphs;      /* 1: replay each preconditioner application from a CUDA graph       */
    int use_pdl;         /* 1: programmatic dependent launch between consecutive kernels      */
    int coarse_cluster_nodes; /* the coarsest level, if it has at most this many nodes and   */
                              /* fits, runs all its sweeps in one launch (coarse_kernel);    */
                              /* 0 = never (one launch per sweep)                            */
    int tile_rows;       /* rows (2D) / z-planes (3D) per warp tile of the stencil kernels:   */
                         /* 2, 4 or 8; 0 = chosen from the grid size                          */
    int autotune;        /* 1: run hh_autotune for `precision` when the problem is created    */
    int fuse_sweeps;     /* 1: in 2D, on levels of at most 600000 nodes (all problems of a     */
                         /* batch together), consecutive steps of the cycle run as one kernel */
                         /* (with V(2,*): the two pre-sweeps, or the HSS right side and them, */
                         /* with the residual restriction; the prolongation with the first    */
                         /* two post-sweeps); same result bit for bit as 0 (one kernel each)  */
    int outer;           /* hh_outer: HH_OUTER_FGMRES (default) or HH_OUTER_RICHARDSON      */
    int cycle_gamma;     /* multigrid cycle index 1..4: 1 V-cycle (default), 2 W-cycle (the    */
                         /* paper's cycle type, Sec. 5.3): each coarse correction is gamma    */
                         /* cycles on the coarse problem, each on the residual left so far    */
    int tile_form;       /* 2D stencil kernels: 0 = chosen from the grid size, 1 = one tile  */
                         /* per warp, 2 = persistent warps walking the tiles (each loads its  */
                         /* next tile while computing the current one); same result bit for  */
                         /* bit; the autotuner's choices override it; ignored in 3D           */
    int smoother;        /* hh_smoother: HH_SMOOTH_JACOBI (default): nu scaled-Jacobi sweeps;  */
                         /* HH_SMOOTH_GMRES: each smoothing step (nu_pre, nu_post, and the     */
                         /* coarsest level's nu_coarse) is nu iterations of GMRES on the       */
                         /* Jacobi-preconditioned level system D^{-1} A_L x = D^{-1} b from    */
                         /* the current iterate (Sec. 5.3's smoother; nu <= 8); the cycle is   */
                         /* then not linear in its right side, which FGMRES allows            */
    int formulation;     /* hh_formulation: HH_FORM_PRIMAL (default): u in Q1, the system     */
                         /* B_delta u = b; HH_FORM_MIXED: (sigma, u) in V_h x Q1 (Sec. 2),     */
                         /* the system A_delta (sigma, u) = (b_sigma, b_u) solved by FGMRES    */
                         /* with the shifted-HSS preconditioner of Def. 4.2 (sigma eliminated; */
                         /* cycles on A_mix = K + k^2 (dh - i)^2 M + k^2 (dh - i) M_Gamma).     */
                         /* V_h: per cell, component a multilinear in the other coordinates    */
                         /* and constant along a (it contains grad Q1).  Vectors of a mixed    */
                         /* problem hold hh_sigma_dofs(grid) sigma entries ((cell x fastest,   */
                         /* component a, vertex s of the other axes) order) and then the       */
                         /* nodes; one problem per object (no batches), no solve server        */
    int persistent;      /* 2D, V(2,2) scaled-Jacobi cycles, one per HSS step: 1: on levels of */
                         /* at most 600000 nodes (all problems of a batch together) the whole  */
                         /* HSS loop of a preconditioner application runs as ONE cooperative  */
                         /* kernel whose CTAs meet at grid-wide barriers between the passes of */
                         /* each cycle; 2: at every size; 0 (default): one kernel per pass,    */
                         /* replayed from a CUDA graph.  Same result bit for bit               */
    long long sync_spin_limit; /* polls a grid-wide barrier wait may take before the kernel     */
                         /* gives up and the call returns HH_ERR_TIMEOUT; 0 = 4194304 (about   */
                         /* a second or more); tiny values make the waits run out on purpose   */
    int stall_cycles;    /* > 0: FGMRES gives a problem up (HH_NOT_CONVERGED, last iterate in u) */
                         /* when stall_cycles restart cycles in a row did not halve its true    */
                         /* residual; 0 (default): only max_outer ends it                       */
    int coarse_kernel;   /* the coarsest level's one-launch solve (see coarse_cluster_nodes): 0    */
                         /* (default) or 1: a thread-block cluster (level in distributed shared  */
                         /* memory, halos exchanged after each group of sweeps: up to four in   */
                         /* 2D, one in 3D); 2 (2D only): bands of rows,                          */
                         /* one CTA each, every sweep in shared memory with the halo rows         */
                         /* recomputed, no exchange between CTAs (what packs and the persistent  */
                         /* loop use).  Same result bit for bit                                  */
} hh_options;

typedef struct {
    int outer_its;          /* outer (FGMRES or Richardson) iterations          */
    long long hss_its;      /* inner HSS iterations                              */
    long long vcycles;      /* V-cycles on the finest level                      */
    double rel_residual;    /* ||b - B_delta u||_2 / ||b||_2 recomputed in FP64   */
    double seconds;         /* wall time of the call                             */
    size_t device_bytes;    /* device memory held by the problem                 */
    long long kernel_launches; /* kernels this call ran (graph replays counted per node) */
    int fallback;           /* solve server only: 1 if the request was solved again with the     */
                            /* server's fallback settings (hh_server_set_fallback)              */
} hh_info;

typedef struct hh_problem hh_problem;

/* Defaults: theta 1, 4 levels, V(2,2), 8 coarse sweeps, omega automatic, restart 30,
 * max_outer 1000, complex FP32 V-cycles, graphs and programmatic launch on,
 * coarse_cluster_nodes 100000, tile shapes from the grid size (no autotuning), fused
 * two-sweep kernels, one kernel per pass (no persistent HSS loop). */
HH_API void hh_options_default(hh_options* opts);

/* Device bytes a problem with this grid and these options allocates for its solves
 * (0 if invalid); building blocks called in the other precision add a second hierarchy. */
HH_API size_t hh_footprint_bytes(const hh_grid* grid, const hh_options* opts);

/* As hh_footprint_bytes for a batch of nb problems (0 if invalid or nb < 1). */
HH_API size_t hh_footprint_batch_bytes(const hh_grid* grid, const hh_options* opts, int nb);

/*
 * Build a problem: validate, compute the operator coefficients of every level and
 * allocate the device hierarchy and the Krylov basis.
 *   k > 0, delta >= 0, delta_hat > 0 (H = 2 delta_hat k M + k M_Gamma must be an inner
 *   product, Sec. 3.1); grid->dim in {2,3}; grid->n >= 2 and divisible by 2^(levels-1);
 *   bc[2*axis + side] in {HH_BC_SOMMERFELD, HH_BC_DIRICHLET} for -x,+x,-y,+y(,-z,+z).
 *   cuda_stream: the caller's stream (NULL = legacy default stream); the library
 *   orders all of its work after the work already queued there and makes that stream
 *   wait for it.
 * Returns HH_ERR_INVALID, HH_ERR_OOM or HH_ERR_CUDA on failure (*out is then NULL).
 */
HH_API hh_status hh_create_problem(const hh_grid* grid, double k, double delta, double delta_hat,
                            const int* bc, const hh_options* opts, void* cuda_stream,
                            hh_problem** out);

/*
 * Build a batch of nb problems on one grid with the same boundary tags and options:
 * k[b], delta[b], delta_hat[b] (host arrays of nb values, each as in hh_create_problem)
 * define problem b; its HSS length is ceil(k[b]^theta).  1 <= nb <= 65535, and in 3D
 * (n + 1) nb <= 65535 (problems share the launch grid's z extent with the planes).
 */
HH_API hh_status hh_create_batch(const hh_grid* grid, int nb, const double* k, const double* delta,
                                 const double* delta_hat, const int* bc, const hh_options* opts,
                                 void* cuda_stream, hh_problem** out);

/* Problems in the batch (0 for NULL). */
HH_API int hh_batch_size(const hh_problem* p);

/*
 * Tile-shape autotuner (a service of this library; the paper has none).  Times every
 * candidate tile shape (rows or planes per warp tile, one tile per warp or persistent
 * warps) of each stencil kernel the solver runs on each level in `precision`, every
 * cluster size of the coarsest-level solve, and the FP64 outer operator, on the problem's
 * own scratch buffers, and keeps the fastest for this problem; later solves use them (the
 * preconditioner graph is captured again).
 * Every shape gives the same result bit for bit.  Choices are remembered per process for
 * (device, dim, level size, batch size, precision, kernel), so problems of the same shape
 * reuse them without timing.  Blocking.  shapes, if not NULL, receives levels x 12 x 2 ints:
 * for level l and kernel m (0 y = op x, 1 axpby, 2 Jacobi, 3 HSS first step, 4 two Jacobi
 * sweeps from 0, 5 prolongation + Jacobi, 6 residual + restriction, 7 prolongation + two
 * sweeps, 8 HSS first step + two sweeps, 9 two sweeps from 0 + residual restriction, 10 HSS
 * first step + two sweeps + residual restriction, 11 coarsest-level solve), {rows, form}
 * (for 9, 10: {coarse rows per tile, 1}; for 11: {cluster size, 0}) at [(l * 12 + m) * 2],
 * 0 where nothing was tuned.
 */
HH_API hh_status hh_autotune(hh_problem* p, int precision, int* shapes);

HH_API void hh_destroy(hh_problem* p);

/*
 * Solve B_delta u = rhs to ||rhs - B_delta u||_2 <= tol ||rhs||_2 (true residual,
 * recomputed in FP64 at the end of every restart cycle) for every problem of the batch.
 * rhs (load vectors), u and the optional initial guess x0 are device complex128 vectors
 * of hh_vector_length(p) entries per problem (nb blocks): level-0 nodes, or for a mixed
 * problem its sigma entries and then the nodes.  Blocking: returns when u is written.  info, if not NULL,
 * points to nb records (kernel_launches is counted for the whole call in info[0]).
 * Returns HH_OK when every problem converged, HH_NOT_CONVERGED when one reached
 * max_outer (u holds the last iterates and info is filled); on errors u is unspecified
 * and every rel_residual is NaN.
 */
HH_API hh_status hh_solve(hh_problem* p, const void* rhs, double tol, void* u, const void* x0,
                   hh_info* info);

/* As hh_solve, but rhs and u are HOST complex128 arrays; the copies are part of the call. */
HH_API hh_status hh_solve_host(hh_problem* p, const void* rhs_host, double tol, void* u_host,
                        hh_info* info);

/* As hh_solve_host, with the nodal values f of the source instead of the load vector:
 * the right side b = M f (Sec. 2, f in Q1) is formed on the device. */
HH_API hh_status hh_solve_host_nodal(hh_problem* p, const void* f_host, double tol, void* u_host,
                                     hh_info* info);

/*
 * Give every problem of the batch new k[b], delta[b], delta_hat[b] (host arrays of nb
 * values, checked as in hh_create_batch) on the same grid: the coefficient tables are
 * rebuilt in place, no device memory is allocated or freed, and the preconditioner graph
 * is captured again at the next solve (or hh_prepare).  Blocking.  A service of this
 * library (the paper has none): it lets a serving loop reuse a problem's hierarchy and
 * Krylov basis for the next request on the same grid.
 */
HH_API hh_status hh_set_params(hh_problem* p, const double* k, const double* delta, const double* delta_hat);

/* Cap, for every problem created or grown afterwards in this process, on the device bytes one
 * problem may hold (0 = no cap, the default).  An allocation past it fails with HH_ERR_OOM
 * before any device call, as a real out-of-memory would (creation then returns NULL, a
 * solve reports the status).  For failure injection and for callers sharing a device. */
HH_API void hh_set_allocation_limit(size_t bytes);

/* sigma entries of a mixed problem on `grid`: n^dim cells x dim components x 2^(dim-1) */
HH_API long long hh_sigma_dofs(const hh_grid* grid);
/* entries of one problem's right side / solution for hh_solve: nodes (primal) or sigma
 * entries and nodes (mixed) */
HH_API long long hh_vector_length(const hh_problem* p);
/* y = the system operator x in FP64 (B_delta, or the mixed A_delta of Sec. 2); x, y: device
 * complex128 vectors of hh_vector_length(p) entries per problem */
HH_API hh_status hh_apply_system(hh_problem* p, const void* x, void* y);

/*
 * Capture the preconditioner graph (and allocate the multigrid buffers) now instead of
 * at the first solve, so that a caller can keep allocations and captures out of the way
 * of work it runs concurrently.  Blocking.
 */
HH_API hh_status hh_prepare(hh_problem* p);

/* Nodes (n_l + 1)^dim of level l, or 0 if l is out of range. */
HH_API long long hh_level_nodes(const hh_problem* p, int level);

/* ---- building blocks (same kernels the solver runs; launched on the problem's stream,
 *      ordered after the caller's stream; non-blocking unless stated) ---- */

/* y = op x on level `level` (Sec. 2 / Def. 4.1 coefficient triples). */
HH_API hh_status hh_apply(hh_problem* p, int level, int op, int precision, const void* x, void* y);

/* One scaled-Jacobi sweep on A_L of level l: x_out = x_in + omega D^{-1} (b - A_L x_in),
 * D = diag(A_L).  x_in == NULL means x_in = 0.  x_out must not alias x_in or b. */
HH_API hh_status hh_jacobi(hh_problem* p, int level, int precision, const void* b, const void* x_in,
                    void* x_out);

/* rc = P^T (b - A_L x): residual on level l restricted to level l+1. */
HH_API hh_status hh_residual_restrict(hh_problem* p, int level, int precision, const void* b,
                               const void* x, void* rc);

/* x += P ec: prolongation of a level-(l+1) correction onto level l. */
HH_API hh_status hh_prolong_correct(hh_problem* p, int level, int precision, const void* ec, void* x);

/* x = one multigrid cycle (V or W, cycle_gamma) on A_L of level 0 from the zero initial guess
 * (cycles_per_hss ignored). */
HH_API hh_status hh_vcycle(hh_problem* p, int precision, const void* b, void* x);

/* rhs = (k-1)/(k+1) A_R u + 2k/(k+1) r on level 0 (Def. 4.1); u == NULL means u = 0. */
HH_API hh_status hh_hss_rhs(hh_problem* p, int precision, const void* u, const void* r, void* rhs);

/* z = shifted-HSS preconditioner applied to r (Def. 4.1; Def. 4.2 for a mixed problem), r
 * and z complex128 vectors of hh_vector_length(p) entries per problem; the inner cycles run
 * in the problem's precision.  Blocking. */
HH_API hh_status hh_precondition(hh_problem* p, const void* r, void* z);

/* b = M f (load vector of a nodal f, Sec. 2), complex128 on level 0. */
HH_API hh_status hh_load_vector(hh_problem* p, const void* f, void* b);

/* out[2b] + i out[2b+1] = x_b^H y_b over the complex128 vectors of problem b
 * (hh_vector_length(p) entries), for every problem of the batch (deterministic order; out
 * holds 2 nb doubles).  Blocking. */
HH_API hh_status hh_dot(hh_problem* p, const void* x, const void* y, double* out);

/*
 * ---- reduction without allocation ----
 * out[i] = V_i^H w for i < nvec (complex128; V_i = V + i*ld entries, each of length n),
 * the same deterministic multi-vector inner product that the outer Krylov iteration
 * runs, but with its block partial sums in a fixed array compiled into the library
 * (nvec <= 64; 304 KiB of device memory that every GPU loading the library holds until
 * the process exits) instead of memory owned by an hh_problem.  It allocates nothing:
 * for callers that must not call cudaMalloc at the point of use (a serving loop whose
 * device memory is all in its own pool, a caller under a budget reserved up front) or
 * that have no hh_problem.  The paper has no counterpart; it is a service of this library.
 *   V, w, out: device pointers (16-byte aligned); out receives nvec complex128 values.
 *   cuda_stream: stream to launch on (NULL = legacy default stream); non-blocking.
 * Returns HH_ERR_INVALID (with a message in hh_last_error) for nvec outside 1..64, n < 0,
 * ld < n or a null pointer, HH_ERR_CUDA if a launch fails.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  The address is kept for the life of
 * the process: after a cudaDeviceReset of a device (which also invalidates every
 * hh_problem on it) the library must not be used on that device again.  All calls share
 * the one array, so calls that overlap on the GPU (different streams, no ordering between
 * them) race.
 */
HH_API hh_status hh_multidot_noalloc(const void* V, long long ld, int nvec, const void* w, long long n,
                                     void* out, void* cuda_stream);

/*
 * ---- packs: problems of different grids in shared launches (a service of this library; the
 *      paper has none) ----
 * A pack runs the FGMRES solves of up to `capacity` problems side by side.  Every outer
 * iteration of a member is the same sequence of operations as in its own hh_solve (same kernels,
 * on the member's own stream), except that the preconditioner applications (Def. 4.1) of all
 * members that need one in the same round run together: each pass of the V-cycle is ONE launch
 * covering the tiles of every member, whatever its grid, replayed from a CUDA graph.  Members
 * join (hh_pack_add) and leave (hh_pack_take) between rounds, so a finished member's slot can be
 * refilled at once while the others go on.  Each member's result equals its own hh_solve's bit
 * for bit.  Members: problems of hh_create_problem (one problem each) in 2D, primal, with
 * V(2,2) scaled-Jacobi cycles, one per HSS step, complex64 cycles, FGMRES, and the same number
 * of levels (2..5); a member problem must not be used otherwise until it is taken.  The pack
 * does not own its members' problems.  Blocking calls; not thread-safe.
 */
typedef struct hh_pack hh_pack;

/* An empty pack for at most `capacity` (1..256) members on the current device. */
HH_API hh_status hh_pack_create(int capacity, hh_pack** out);

/* Add problem p with right side rhs (io 0: device load vector; 1: host load vector; 2: host
 * nodal source f, b = M f), tolerance tol (as hh_solve) and output u (device for io 0, host
 * otherwise; (n + 1)^2 complex128 entries, written when the member finishes).  *slot receives
 * the member's slot.  HH_ERR_INVALID if p cannot be packed, the pack is full or p is in it. */
HH_API hh_status hh_pack_add(hh_pack* k, hh_problem* p, const void* rhs, int io, double tol, void* u, int* slot);

/* Run rounds (every running member advances to its next synchronisation point) until at least
 * one member has finished, no member is running, or max_rounds rounds (> 0) have run; done (room
 * for `capacity` ints) receives the slots of every finished member not yet taken, *ndone their
 * number. */
HH_API hh_status hh_pack_run(hh_pack* k, int max_rounds, int* done, int* ndone);

/* The status and info of the finished member in `slot` (as hh_solve returns them; seconds from
 * hh_pack_add to its end); frees the slot and releases the problem to the caller. */
HH_API hh_status hh_pack_take(hh_pack* k, int slot, hh_info* info);

/* Members in the pack (running or finished and not yet taken). */
HH_API int hh_pack_members(const hh_pack* k);

HH_API void hh_pack_destroy(hh_pack* k);

/*
 * ---- continuous-batching solve server (a service of this library; the paper has none) ----
 * A request loop on the current device: requests of any grid, wavenumber and shifts are
 * queued, admitted in arrival order as worker slots and device memory free up, and solved
 * concurrently, each on its own CUDA stream, so that their kernels overlap on the GPU.
 * Each admitted solve keeps its hierarchy and Krylov basis on the device; finished
 * problems stay pooled and are retargeted (hh_set_params) for later requests on the same
 * grid, and idle problems of other grids are destroyed, least recently used first, when a
 * new request needs their memory.  Every request's result is the one a lone
 * hh_solve_host of the same problem would give.
 */
typedef struct hh_server hh_server;

typedef struct {
    hh_grid grid;           /* unit square / cube, n cells per axis                       */
    double k, delta, delta_hat;
    int bc[6];              /* boundary tags as in hh_create_problem                      */
    double tol;             /* relative residual target of the outer FGMRES               */
    int rhs_kind;           /* 0: rhs is the load vector b; 1: nodal source f, b = M f    */
} hh_request;

typedef struct {
    long long submitted, completed, failed, queued;
    int running;            /* solves on the device now                                   */
    int max_concurrent;     /* most solves on the device at once so far                   */
    size_t budget;          /* device bytes the server may hold in problems               */
    size_t held_bytes;      /* bytes held now (running and pooled problems)               */
    size_t peak_bytes;      /* most bytes held at once so far (never above budget)        */
    long long problems_created, problems_reused, problems_evicted;
} hh_server_stats;

/* Start a server with `slots` worker threads (1..64: at most that many solves run at
 * once) that holds at most device_budget bytes of problems (hh_footprint_bytes of each),
 * all built with *opts.  Returns HH_ERR_INVALID for bad arguments. */
HH_API hh_status hh_server_create(int slots, size_t device_budget, const hh_options* opts, hh_server** out);

/* Queue one solve: rhs_host (load vector or nodal source, complex128, (n+1)^dim entries; see
 * rhs_kind) and u_host (the
 * solution, same size) are host arrays that the caller keeps valid until hh_server_wait
 * returns for *ticket.  HH_ERR_INVALID if the request is invalid or its footprint exceeds
 * the budget (it could never be admitted). */
HH_API hh_status hh_server_submit(hh_server* s, const hh_request* req, const void* rhs_host, void* u_host,
                                  long long* ticket);

/* Wait for a request: returns its solve status and fills info (may be NULL), the time
 * from submission to completion and the time it spent queued (seconds; may be NULL).  A
 * ticket can be waited for once. */
HH_API hh_status hh_server_wait(hh_server* s, long long ticket, hh_info* info, double* latency_s, double* queue_s);

HH_API hh_status hh_server_get_stats(hh_server* s, hh_server_stats* out);

/* Pack the server's 2D requests (before the first request; the server's options must be packable,
 * see hh_pack_create): a dispatcher thread runs up to `capacity` (1..256) of them as members of
 * one pack, so that their preconditioner applications share launches, and admits queued ones
 * between rounds as members finish and device memory frees up (continuous batching).  Only
 * requests with at most max_hss_steps HSS steps (ceil(k^theta); 0: no limit) join the pack: each
 * round advances every member by one FGMRES iteration and lasts as long as the longest member's
 * HSS loop, so long loops are better run apart.  Other requests, and fallback solves, run on the
 * worker slots as before.  Results equal the lone solves bit for bit. */
HH_API hh_status hh_server_set_pack(hh_server* s, int capacity, int max_hss_steps);

/* Fallback for requests that do not converge: a request whose solve ends HH_NOT_CONVERGED (its
 * max_outer reached, or stalled under opts.stall_cycles) is solved once more from zero on a
 * problem built with *opts and this delta_hat (> 0) instead of the request's, and its result,
 * status and info (outer_its, hss_its, vcycles and seconds summed over both attempts, fallback =
 * 1) are those of that second solve.  The solution of B_delta u = b does not depend on delta_hat
 * or the preconditioner; only whether FGMRES reaches it does (e.g. the paper's multigrid, W-cycles
 * with GMRES(5) and Jacobi on every level at delta_hat = 2, Sec. 5.3, where V-cycles with scaled
 * Jacobi at delta_hat = k stall).  opts NULL removes the fallback.  Applies to requests submitted
 * afterwards; the fallback problems count against the same device budget. */
HH_API hh_status hh_server_set_fallback(hh_server* s, const hh_options* opts, double delta_hat);

/* Finish every queued and running request, then free all problems and stop the workers. */
HH_API void hh_server_destroy(hh_server* s);

HH_API const char* hh_status_string(hh_status s);
HH_API const char* hh_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* HH_H */
