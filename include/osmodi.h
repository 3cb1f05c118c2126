/*
 * osmodi -- matrix-based omnidirectional pressure integration on one GB300
 * (Zigunov & Charonko, "A fast, matrix-based method to perform
 * omnidirectional pressure integration", arXiv 2311.16935).
 *
 * C interface.  Every pointer named *_dev is device memory of the calling
 * process's current CUDA device; *_host pointers are host memory.  The caller
 * owns all buffers it passes in; the library never frees them.  Streams are
 * passed as `void*` holding a cudaStream_t (NULL = the legacy default stream).
 *
 * Grids are uniform boxes of nx x ny (2D) or nx x ny x nz (3D) cells stored
 * x fastest: cell (i, j, k) is element (k*ny + j)*nx + i.  Face neighbours are
 * E = +x, W = -x, N = +y, S = -y, F = +z, B = -z.  A gradient field holds ndim
 * such planes back to back (component x first).  Cells outside the box count
 * as missing data (b = 1 in Section 2.2's notation).
 *
 * Error behaviour: every call returns an osmodi_status.  Negative values
 * mean nothing usable was written to the outputs; OSMODI_NOT_CONVERGED means
 * the best iterate was written and the result struct is filled.  No call
 * traps, asserts or aborts on bad input; device-side faults of the inputs
 * (NaN gradients at valid cells) come back as OSMODI_E_NAN_INPUT.
 */
#ifndef OSMODI_H
#define OSMODI_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define OSMODI_API __attribute__((visibility("default")))
#else
#define OSMODI_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct osmodi_plan_s* osmodi_plan; /* opaque, host-owned */

typedef enum {
    OSMODI_OK = 0,
    OSMODI_NOT_CONVERGED = 1, /* max_iter reached or stagnated; best iterate written */
    OSMODI_E_INVALID = -1,    /* bad argument (NULL pointer, bad dims/spacing/dtype/tol) */
    OSMODI_E_UNSUPPORTED = -2,
    OSMODI_E_NOMEM = -3,      /* device allocation at plan creation failed */
    OSMODI_E_CUDA = -4,       /* a CUDA call failed; see osmodi_last_cuda_error() */
    OSMODI_E_DIVERGED = -5,   /* eps_R grew 1e3x above its minimum */
    OSMODI_E_TIMEOUT = -6,    /* a bounded device-side wait ran out */
    OSMODI_E_EMPTY = -7,      /* the mask leaves no valid cell */
    OSMODI_E_NAN_INPUT = -8,  /* non-finite gradient (or initial pressure) at a valid cell */
    OSMODI_E_WORKSPACE = -9   /* workspace pointer NULL, misaligned or too small */
} osmodi_status;

/* element types of caller buffers */
enum { OSMODI_F32 = 0, OSMODI_F64 = 1 };

/* arithmetic of the iterations (Section 2.1 leaves it open; the paper's GPU
 * code used FP64 throughout) */
enum {
    OSMODI_FP64 = 0,        /* every vector and operation in FP64 */
    OSMODI_FP32 = 1,        /* FP32 vectors and sweeps; FP64 only for the residual
                               of the initial guess, norms, dot products and the
                               constant removal */
    OSMODI_FP32_REFINE = 2  /* FP32 sweeps inside an FP64 iterative-refinement loop:
                               r = b - A p in FP64, FP32 correction solve, p += e */
};

/* iteration scheme.  Both reach the same fixed point: Algorithm 1's answer,
 * which solves (I - W^{n+1}_off - W^n) P = S (Eq. MatrixEquation at P^{n+1} =
 * P^n, i.e. a zero momentum residual of Eq. ResidualMomentum). */
enum {
    OSMODI_FPCG = 0,  /* conjugate gradients on (I - W^{n+1}_off - W^n) P = S directly
                         (the boundary term is applied in every iteration) */
    OSMODI_OUTER = 1  /* Algorithm 1 as written: each outer iteration refreshes the
                         boundary term W^n P^n + S and solves Eq. MatrixEquation */
};

/* inner solver of Eq. MatrixEquation in the OUTER scheme */
enum {
    OSMODI_INNER_CG = 0,     /* conjugate gradients on M = I - W^{n+1}_off, warm-started
                                from P^n, as the paper's GPU code (Section 2.1) */
    OSMODI_INNER_JACOBI = 1  /* fixed number of Jacobi sweeps P <- W^{n+1}_off P + RHS
                                (diag M = 1), several fused per pass */
};

typedef struct {
    int precision;       /* OSMODI_FP64 | OSMODI_FP32 | OSMODI_FP32_REFINE (default) */
    int scheme;          /* OSMODI_FPCG (default) | OSMODI_OUTER */
    int inner;           /* OUTER only: OSMODI_INNER_CG (default) | OSMODI_INNER_JACOBI */
    int inner_max;       /* FPCG: max CG iterations per refinement step (default 1<<20);
                            OUTER: max inner iterations (or sweeps) per outer iteration */
    double inner_tol;    /* FP32_REFINE: the FP32 CG runs until its residual has dropped
                            by this factor since the last FP64 residual replacement
                            (default 0.1; 1e-4 with precond = 1, whose few
                            iterations drift little); the search direction carries over
                            ("reliable updates").  OUTER+CG: relative tolerance of
                            each inner solve (default 1e-6) */
    int check_every;     /* iterations between host convergence checks where the
                            host drives the iterations: profile mode,
                            osmodi_solve_noalloc and the fixed-graph comparison
                            mode (0 = default: 64, or 8 with precond = 1); a
                            captured solve otherwise loops on the device */
    int sweeps_per_pass; /* OUTER+JACOBI: Jacobi sweeps fused per pass, 1..4 (default 2) */
    int max_refine;      /* FP32_REFINE: max refinement steps (default 32) */
    int record_history;  /* OUTER: keep eps_R of every outer iteration (osmodi_history) */
    int threads;         /* threads per block of the sweep kernels (0 = tuned) */
    int blocks_per_sm;   /* resident blocks per SM used to size persistent grids (0 = tuned) */
    int profile;         /* 1 = launch the CG iterations one by one (no CUDA graph) with
                            CUDA events around every sweep kernel on the caller's stream;
                            durations readable with osmodi_kernel_stats */
    int slab;            /* z-planes per work item of the tiled 3D sweep kernel (0 = tuned) */
    int flat_sweeps;     /* sweep kernel of the CG on L: 1 (default) flat grid-stride;
                            0 = z-marching tiled; 2 = z-marching with the r / p planes
                            staged in shared memory by bulk tensor (TMA) copies
                            (3D, FP32 inner precision; otherwise falls back to 1) */
    int autotune;        /* 1 = look the launch geometry up in the autotune cache at plan
                            creation (see osmodi_autotune) */
    int accel;           /* OUTER: depth m (0..8) of Anderson mixing of the outer
                            iterates (default 0 = Algorithm 1 unchanged).  Each outer
                            iteration still refreshes the boundary term W^n P^n and
                            solves Eq. MatrixEquation; the new iterate is then
                            x = G(x_k) - sum_i gamma_i dG_i with gamma minimising
                            || f_k - sum_i gamma_i dF_i ||, f = G(x) - x, over the
                            last m differences (Anderson 1965; Walker & Ni 2011).
                            Same fixed point; far fewer outer iterations.  Adds
                            2m + 3 work vectors to the workspace. */
    int precond;         /* FPCG: 1 = multigrid-preconditioned CG (aggregation of 2x2(x2)
                            cells per level, Galerkin coarse weights; symmetric smoothing:
                            3-D red-black SOR, red then black before the coarse correction,
                            black then red after; 2-D damped Jacobi; a fixed symmetric
                            operator, so CG still converges to the same fixed point in far
                            fewer iterations);
                            0 = plain CG.  Built at plan creation (about 2.5 B of device memory per
                            cell); grids of at most 8 cells per axis use plain CG.
                            Not part of the paper's method. */
    int zero_start;      /* 1 = start from P^0 = 0 without reading p: p is output only
                            (saves reading it, e.g. from host memory); 0 = p holds P^0 */
    int mg_sweeps;       /* precond = 1: smoothing sweeps before and after the coarse
                            correction on every level (3-D: red-black sweeps; 2-D: damped
                            Jacobi sweeps), 1..8; 0 = the default, 2 */
    double mg_scale;     /* precond = 1: scale of the coarse correction, (0, 4]; 0 = the
                            default, 2.0.  Any positive scale keeps the preconditioner
                            symmetric positive definite; it changes the iteration count */
    int refine_ff;       /* FP32 precisions: 1 = carry the refinement loop (P, b, the
                            residual r = b - L P, the fold P += e, the output) in
                            float-float arithmetic (pairs of FP32 numbers, about 48
                            bits) at tolerances >= 1e-9, FP64 below; 0 (default) = FP64
                            throughout the refinement loop */
} osmodi_options;

typedef struct {
    int status;              /* osmodi_status of the solve */
    int outer_iters;         /* OUTER: Algorithm 1 iterations; FPCG: refinement steps */
    int64_t inner_iters;     /* CG iterations or Jacobi sweeps, all steps together */
    int refine_steps;        /* FP64 residual evaluations r = b - A p */
    double eps_R;            /* Eq. ResidualMomentum of the returned pressure, in FP64 */
    double eps_P;            /* OUTER: Eq. ResidualPressure of the last outer iteration
                                (FPCG: 0, the scheme has no outer iterates) */
    double ms;               /* wall-clock of the call (host timer around the stream) */
    double point_updates;    /* valid cells x stencil applications (GLUPS numerator) */
    double seed_rel_dist;    /* ||P0 - P|| / ||P|| over valid cells, both gauge-fixed
                                (1 for a zero initial pressure) */
    double kernel_launches;  /* kernels the call issued (including those of a captured
                                chunk that found the iteration already finished) */
} osmodi_result;

/* Fill *opt with the defaults listed above. */
OSMODI_API void osmodi_default_options(osmodi_options* opt);

/*
 * Build a plan for one grid (Section 2.2: the weights depend only on the
 * grid and its mask, "precomputed for a given grid topology").
 *   ndim       2 or 3
 *   dims       {nx, ny, nz} (nz ignored in 2D); each >= 1, nx*ny*nz < 2^40
 *   spacing    {dx, dy, dz} > 0 (dz ignored in 2D).  Unequal 3D spacing uses the
 *              quadrature of Eqs. FarFaceEquation and IAc-ICc; equal spacing the
 *              closed forms of Eqs. ConstantFarFace/ConstantNearFaces.
 *   mask_dev   nx*ny*nz bytes, nonzero = data available; NULL = every cell valid.
 *              Plays the role of the paper's NaN encoding of missing vectors
 *              (Section 2.2, b_j).
 *   opt        NULL = defaults
 *   stream     used for the set-up kernels; the call returns after they finish
 *   out        receives the plan
 * The plan owns the device arrays it allocates here (per-cell neighbour codes
 * and component labels, about 5-9 bytes per cell); osmodi_destroy frees them.
 * Errors: E_INVALID, E_EMPTY (no valid cell), E_NOMEM, E_CUDA.
 */
OSMODI_API osmodi_status osmodi_create(int ndim, const int64_t dims[3], const double spacing[3], const uint8_t* mask_dev,
                            const osmodi_options* opt, void* stream, osmodi_plan* out);

/* Device workspace bytes that osmodi_solve needs for this plan (256-byte
 * aligned start required). */
OSMODI_API size_t osmodi_workspace_bytes(osmodi_plan plan);

/*
 * Solve for the pressure (Algorithm 1's converged answer).
 *   grad_dev    ndim planes of nx*ny*nz values (f = grad P), grad_dtype
 *               OSMODI_F32 or OSMODI_F64.  Values at missing cells are never
 *               read; a non-finite value at a valid cell is E_NAN_INPUT.
 *   p_dev       nx*ny*nz values of p_dtype.  In: initial pressure P^0 (zeros
 *               = the paper's start, Algorithm 1; missing cells ignored).
 *               Out: the pressure with zero mean on every connected component
 *               of valid cells (pressure is defined up to a constant, Eq. 1)
 *               and NaN on missing cells.
 *   tol         threshold on eps_R (Eq. ResidualMomentum, denominator ||S||),
 *               > 0
 *   max_iter    FPCG: total CG iterations; OUTER: outer iterations
 *   workspace   osmodi_workspace_bytes(plan) bytes of device memory
 *   stream      all work is ordered on it; the call synchronises the stream
 *               to read convergence flags and fill *res
 *   res         may be NULL
 * grad_dev and p_dev may be device or managed memory, or page-locked host
 * memory (cudaHostAlloc / cudaHostRegister, unified addressing): the source
 * kernel then reads the gradient and P^0 and the output kernel writes P
 * directly over the host link, with no staging copies.  Any other host
 * pointer is refused with E_INVALID.
 * Returns OK (eps_R <= tol), NOT_CONVERGED, E_NAN_INPUT, E_DIVERGED,
 * E_WORKSPACE, E_INVALID or E_CUDA.  A plan is not thread-safe: one solve at
 * a time per plan.
 */
OSMODI_API osmodi_status osmodi_solve(osmodi_plan plan, const void* grad_dev, int grad_dtype, void* p_dev, int p_dtype,
                           double tol, int max_iter, void* workspace_dev, void* stream, osmodi_result* res);

/*
 * Solve `count` independent problems (many PIV snapshots of uneven sizes and
 * masks) in one persistent cooperative launch that keeps a convergence flag
 * per instance; converged instances drop out while the others continue.
 * All plans must share ndim; precision and scheme come from plans[0]
 * (FP32_REFINE and FP32 supported, scheme FPCG).  grads[i], ps[i] are laid
 * out as for osmodi_solve.  results may be NULL, else count entries.
 * Returns OK when every instance converged, NOT_CONVERGED if any did not, or
 * the first error.
 */
OSMODI_API osmodi_status osmodi_solve_batched(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                   void* const* ps, int p_dtype, double tol, int max_iter, void* workspace_dev,
                                   void* stream, osmodi_result* results);

/*
 * osmodi_solve_noalloc: the same solve as osmodi_solve for callers that
 * cannot allocate device memory at solve time -- for example code running
 * under a host framework whose caching allocator owns the device memory, or
 * a latency-bound acquisition loop where cudaMalloc / cudaFree (which may
 * synchronise the whole device) are not acceptable.  Such callers create
 * their plans during set-up; this call then allocates nothing: no cudaMalloc,
 * no cudaFree, no page-locked host memory, no CUDA graph.  The paper has no
 * counterpart; it is an interface convenience.
 *
 * Its device scratch is one file-scope device array of
 * OSMODI_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads the
 * library keeps until the process exits.  A plan whose
 * osmodi_workspace_bytes() exceeds that size is rejected with
 * OSMODI_E_WORKSPACE (osmodi_last_cuda_error() then says why).  For the
 * default FP32_REFINE / FPCG options that admits grids of up to about
 * 350,000 cells (e.g. 512 x 512 in 2D, 64^3 in 3D).
 *
 * osmodi_create looks the array's device address up on the plan's device
 * (cudaGetSymbolAddress, which also loads the array there) and keeps it, so
 * the solve itself finds the scratch ready; create plans before any stream
 * capture on that device.  (Should that look-up have failed, the first solve
 * on the device retries it.)  All calls share the one array, which keeps
 * the previous call's contents (every value the solve needs zeroed is
 * cleared at the start of each call).  Calls whose GPU work overlaps -- on
 * two streams, from two threads or on plans that share a device -- race on
 * the array and must be serialised by the caller.
 * Arguments, results and error codes are those of osmodi_solve, without the
 * workspace.
 */
#define OSMODI_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
OSMODI_API osmodi_status osmodi_solve_noalloc(osmodi_plan plan, const void* grad_dev, int grad_dtype, void* p_dev,
                                              int p_dtype, double tol, int max_iter, void* stream,
                                              osmodi_result* res);

/*
 * Solve `count` independent problems, each by the single-problem path of
 * osmodi_solve with its own plan's options (so a multigrid-preconditioned
 * plan solves in a few dozen iterations), spread over `streams` (1..64)
 * CUDA streams that as many host threads drive concurrently.  Problem i runs
 * on stream i mod streams with workspaces[i mod streams], which must hold
 * osmodi_workspace_bytes() of every plan assigned to it; a problem's plan is
 * used by one thread only: a plan listed more than once must appear only at
 * indices that map to the same stream (else OSMODI_E_INVALID, nothing run).
 * grads / ps / dtypes as osmodi_solve_batched.
 * Synchronous: returns when every problem has finished.  Returns OK when all
 * converged, NOT_CONVERGED if any did not, NAN_INPUT if one had non-finite
 * input, else the first error (the others stop at their next problem).
 */
OSMODI_API osmodi_status osmodi_solve_many(int count, const osmodi_plan* plans, const void* const* grads, int grad_dtype,
                                           void* const* ps, int p_dtype, double tol, int max_iter, int streams,
                                           void* const* workspaces, osmodi_result* results);

/* Workspace bytes for osmodi_solve_batched over these plans. */
OSMODI_API size_t osmodi_batched_workspace_bytes(int count, const osmodi_plan* plans);

/*
 * The batched solve as a CUDA graph, for a stream of batches over the same
 * geometry (PIV acquisition: fixed masks, new gradients every snapshot).
 *
 * osmodi_batch_graph_create checks its arguments as osmodi_solve_batched
 * does, then captures one solve of the batch -- the upload of the instance
 * and tile tables from page-locked host copies the graph owns, the state
 * resets, the single persistent cooperative launch (a kernel node with the
 * cooperative attribute) and the copy of the per-instance states to
 * page-locked host memory -- and instantiates it.  Because every replay
 * rewrites its tables, the workspace may serve other solves between
 * replays (never while one is in flight).  The graph keeps the addresses it was created with: the
 * plans' codes and labels, grads[i], ps[i] and the workspace must stay alive
 * and unmoved until osmodi_batch_graph_destroy, and the plans must not be
 * destroyed before it.  Between launches the caller writes new gradients
 * into the same buffers and resets (or seeds) ps[i]: as in
 * osmodi_solve_batched, ps[i] holds the initial guess on entry and the
 * solution on exit.
 *
 * osmodi_batch_graph_launch enqueues one replay on `stream` (asynchronous;
 * one replay in flight per graph and per workspace).
 * osmodi_batch_graph_results waits for the last replay and fills `results`
 * (count entries, may be NULL); ms is the replay's device time.  Its return
 * value is that of osmodi_solve_batched for the same solve.
 * OSMODI_E_INVALID: NULL handle, no replay yet, or a launch on another
 * device.  OSMODI_E_CUDA: capture or instantiation refused (the message is in
 * osmodi_last_cuda_error()).
 */
typedef struct osmodi_batch_graph_s* osmodi_batch_graph;
OSMODI_API osmodi_status osmodi_batch_graph_create(int count, const osmodi_plan* plans, const void* const* grads,
                                                   int grad_dtype, void* const* ps, int p_dtype, double tol, int max_iter,
                                                   void* workspace_dev, void* stream, osmodi_batch_graph* out);
OSMODI_API osmodi_status osmodi_batch_graph_launch(osmodi_batch_graph graph, void* stream);
OSMODI_API osmodi_status osmodi_batch_graph_results(osmodi_batch_graph graph, osmodi_result* results);
OSMODI_API void osmodi_batch_graph_destroy(osmodi_batch_graph graph);

/* eps_R of every outer iteration of the plan's last OUTER solve with
 * record_history set; copies min(cap, n) values, returns n.  Entry 0 of each
 * refinement step is the residual of its starting iterate, entry k the
 * residual after k outer iterations of Algorithm 1. */
OSMODI_API int osmodi_history(osmodi_plan plan, double* out_host, int cap);

/* eps_P of Eq. ResidualPressure, ||P^{n+1} - P^n||_2 / ||P^{n+1}||_2 over the
 * valid cells (P ungauged: the refinement's iterate plus the outer iterate),
 * at the same evaluations as osmodi_history; NaN at the first entry of each
 * refinement step (no previous outer iterate).  Copies min(cap, n) values to
 * host memory, returns n. */
OSMODI_API int osmodi_history_pressure(osmodi_plan plan, double* out_host, int cap);

/*
 * Step-level entry points (the pieces of the solve, for checking each one
 * against a CPU evaluation of the paper's formulas).  All synchronous on
 * `stream`; dense nx*ny*nz FP64 arrays.
 *
 * osmodi_ray_counts: per valid cell the 2 + 4*ndim ray counts A_C^n,
 *   A_C^{n+1}, then (A_f^n, A_f^{n+1}) for f = E, W, N, S[, F, B]
 *   (Eqs. Acn, AEnp1, AEn, ANnp1, ANn and the 3D pattern), decoded from the
 *   plan's per-cell neighbour codes; zeros on missing cells.  counts_dev
 *   holds nx*ny*nz*(2+4*ndim) doubles, cell-major.
 * osmodi_source: S of Eq. ExplicitEqn (last sum), 0 on missing cells.
 * osmodi_apply: which = 0: W^{n+1}_off x; 1: W^n x (diagonal included);
 *   2: (I - W^{n+1}_off - W^n) x.  Missing cells of y get 0.
 * osmodi_residual: eps_R of Eq. ResidualMomentum for pressure p (p_dtype).
 */
OSMODI_API osmodi_status osmodi_ray_counts(osmodi_plan plan, double* counts_dev, void* stream);
OSMODI_API osmodi_status osmodi_source(osmodi_plan plan, const void* grad_dev, int grad_dtype, double* S_dev, void* stream);
OSMODI_API osmodi_status osmodi_apply(osmodi_plan plan, int which, const double* x_dev, double* y_dev, void* stream);
OSMODI_API osmodi_status osmodi_residual(osmodi_plan plan, const void* grad_dev, int grad_dtype, const void* p_dev, int p_dtype,
                              double* eps_R_host, void* stream);

/*
 * Source-term front ends: the pressure gradient f that osmodi_solve
 * integrates, computed from velocity data on the plan's grid and mask.  All
 * arrays are FP32 device buffers, dense nx*ny*nz per plane (x fastest),
 * components as consecutive planes; grad_dev receives ndim planes laid out
 * as osmodi_solve's gradient input.  Missing cells of the output get 0.
 * Asynchronous on `stream` (except osmodi_source_compressible, which
 * synchronises to report singular cells).
 *
 * Derivatives (the paper does not fix a scheme): centred where both
 * neighbours along the axis are valid, else the second-order one-sided
 * three-point difference towards the valid side when the cell two steps away
 * is valid too, else the two-point difference, else 0.  Second derivatives:
 * centred, else three-point one-sided, else 0.  Derivatives of products (the
 * conservative terms) difference the product field.
 *
 * osmodi_source_incompressible: Eq. 1 (Section 1),
 *   f = -rho (du/dt + (u . grad) u) + mu lap u.
 *   u_dev: ndim planes at time t.  u_prev_dev / u_next_dev: the snapshots at
 *   t - dt / t + dt, either may be NULL: both given -> centred time
 *   difference, one -> one-sided, none -> steady (du/dt = 0).  dt > 0 when a
 *   neighbour snapshot is given.
 * osmodi_source_rans: Eq. RANS_f (Section 3.3), viscous terms dropped,
 *   f_i = -rho (U_j dU_i/dx_j + d<u_i' u_j'>/dx_j).  u_mean_dev: ndim planes;
 *   stress_dev: the symmetric Reynolds stresses, 3 planes in 2D (xx, yy, xy),
 *   6 in 3D (xx, yy, zz, xy, xz, yz).
 * osmodi_source_compressible: Eq. compressible-pressure (Section 3.4):
 *   per cell the ndim x ndim system (delta_ij + <u_i u_j>/(R T)) g_j =
 *   -(1/(R T)) (d<u_i u_j>/dx_j - <u_i u_j>/T dT/dx_j), <u_i u_j> = U_i U_j +
 *   <u_i' u_j'>, T = T_inf (1 + (gamma - 1)/2 M_inf^2 (1 - |U|^2/V_inf^2)),
 *   solved for g = grad ln(P/P_inf) (written to grad_dev; osmodi_solve then
 *   gives ln(P/P_inf) up to a constant).  temperature_dev (NULL allowed)
 *   receives T.  gamma > 1, mach_inf >= 0, v_inf, t_inf, r_gas > 0.
 *   Returns OSMODI_E_NAN_INPUT when the system was singular at some cell
 *   (only possible for non-physical stresses); those cells hold 0.
 */
OSMODI_API osmodi_status osmodi_source_incompressible(osmodi_plan plan, const float* u_dev, const float* u_prev_dev,
                                                      const float* u_next_dev, double dt, double rho, double mu,
                                                      float* grad_dev, void* stream);
OSMODI_API osmodi_status osmodi_source_rans(osmodi_plan plan, const float* u_mean_dev, const float* stress_dev,
                                            double rho, float* grad_dev, void* stream);
OSMODI_API osmodi_status osmodi_source_compressible(osmodi_plan plan, const float* u_mean_dev, const float* stress_dev,
                                                    double gamma, double mach_inf, double v_inf, double t_inf,
                                                    double r_gas, float* grad_dev, float* temperature_dev,
                                                    void* stream);

/* Device time of the sweep kernels in the plan's last solve with
 * options.profile set, from CUDA events on the solve's stream:
 * out[0] / out[1]: total ms / launches of the CG kernel that applies the
 * stencil (p update, q = A p, x update, p.q); out[2] / out[3]: the CG
 * residual-update kernel (r -= alpha q, r.r); out[4] / out[5]: the FP64
 * residual kernel of the refinement loop; out[6] / out[7]: the multigrid
 * preconditioner (one application z = B r per CG iteration; 0 without it). */
OSMODI_API osmodi_status osmodi_kernel_stats(osmodi_plan plan, double out[8]);

/* Profile mode, multigrid preconditioner: out[0] / out[1] = total ms /
 * launches of the fine-level plain sweep kernel (two launches per V-cycle,
 * z += omega D^-1 (r - L z)); out[2] / out[3] = the fine-level residual
 * kernel (t = r - L z, one per V-cycle).  CUDA events on the solve's stream. */
OSMODI_API osmodi_status osmodi_kernel_stats_precond(osmodi_plan plan, double out[4]);

/*
 * Autotuner.  osmodi_autotune times short bursts of CG iterations on this
 * plan (synthetic right-hand side, the caller's workspace) for every
 * candidate launch geometry -- grid of the stencil kernel (2..5 blocks per
 * SM), grid of the update kernel (4..8 per SM), flat or z-marching stencil
 * kernel -- keeps the fastest in the plan, and records it in the cache file
 * (cache_path, or $OSMODI_AUTOTUNE_CACHE, or ~/.cache/osmodi_autotune.txt;
 * NULL-safe) keyed by GPU name, ndim, log2 of the cell count and precision.
 * Plans created with options.autotune = 1 read that cache.  ms_out (may be
 * NULL) receives the best time per CG iteration.  Synchronous.
 * For an OUTER plan with Jacobi inner sweeps it instead times 24 sweeps of
 * the plan's operator with 1, 2, 3 and 4 sweeps fused per pass, keeps the
 * fastest in options.sweeps_per_pass (ms_out: time per sweep) and caches it
 * the same way.
 *
 * osmodi_autotune_batched picks the tile depth of osmodi_solve_batched (1, 2,
 * 4 or 8 chunks of 4 cells per thread) by timing the batched solve capped at
 * a few iterations on the caller's problems; the choice is stored in
 * plans[0] (the batched solve reads it from there).  The caller's pressure
 * buffers are overwritten.
 */
OSMODI_API osmodi_status osmodi_autotune(osmodi_plan plan, void* workspace_dev, void* stream, const char* cache_path,
                                         double* ms_out);
OSMODI_API osmodi_status osmodi_autotune_batched(int count, const osmodi_plan* plans, const void* const* grads,
                                                 int grad_dtype, void* const* ps, int p_dtype, void* workspace_dev,
                                                 void* stream, int* tile_depth_out);

/* Plan facts: out[0] nx, [1] ny, [2] nz, [3] valid cells, [4] connected
 * components, [5] padded row pitch, [6] padded cells, [7] launch blocks. */
OSMODI_API osmodi_status osmodi_plan_info(osmodi_plan plan, int64_t out[8]);

/* Coarse levels of the plan's multigrid preconditioner (0 when it is off or
 * the grid has at most 8 cells per axis). */
OSMODI_API int osmodi_precond_levels(osmodi_plan plan);

/* The constants the plan uses: c[9] = c_jk row-major (x, y, z), F[3] = face
 * totals, a_tot (Eqs. cxx2D, Atot2D; Section 2.2.2). */
OSMODI_API osmodi_status osmodi_plan_constants(osmodi_plan plan, double c[9], double F[3], double* a_tot);

OSMODI_API void osmodi_destroy(osmodi_plan plan);

/*
 * The seed network (learned initial pressure).  A small 3D convolutional
 * encoder-decoder (4 resolution levels, 16-64 channels, skip additions)
 * maps the gradient field and the mask to a pressure guess P^0 that
 * osmodi_solve then iterates to the usual tolerance (Algorithm 1 starts from
 * any P^0; the answer does not depend on it).  BF16 weights and activations,
 * FP32 accumulation on the tensor cores.  The network is not part of the
 * paper's method; the solve that follows always runs to tolerance, and
 * osmodi_result.seed_rel_dist reports how far the guess started.
 *
 * Inputs: 3D grids whose three sizes are multiples of 8; gradient and target
 * as for osmodi_solve (3 planes, x fastest); mask_dev as for osmodi_create
 * (NULL = all valid); spacing = the (isotropic) grid spacing.
 * Parameters are one FP32 array of osmodi_net_param_count() values: per
 * layer (e0, e1, e1b, e2, e2b, e3, m, m2, u2, u2b, u1, u1b, u0, out) the
 * weights (taps, cin, cout) followed by the biases (cout).
 */
typedef struct osmodi_net_s* osmodi_net;
OSMODI_API size_t osmodi_net_param_count(void);
/* dims = {nx, ny, nz}; train = 1 also allocates gradients, Adam moments and
 * activation gradients.  Parameters start undefined: call set_params. */
OSMODI_API osmodi_status osmodi_net_create(const int64_t dims[3], int train, osmodi_net* out);
OSMODI_API osmodi_status osmodi_net_set_params(osmodi_net net, const float* params_host);
OSMODI_API osmodi_status osmodi_net_get_params(osmodi_net net, float* params_host);
/* accumulated parameter gradients (training nets) */
OSMODI_API osmodi_status osmodi_net_get_grads(osmodi_net net, float* grads_host);
/*
 * One 3x3x3 convolution (stride 1, zero padding) of the seed network's kind,
 * as a step-level entry point for checking the convolution kernels against a
 * reference: y = relu?(conv(x, w) + bias) with x BF16 [D][H][W][cin]
 * (channels last), w BF16 [27][cin][cout] (tap = (dz+1)*9 + (dy+1)*3 +
 * (dx+1)), bias FP32 [cout] (may be NULL), y BF16 [D][H][W][cout].  path 0:
 * tcgen05 with the input tile staged once where the shape allows, else the
 * gathering kernel; 1: warp-level wmma; 2: tcgen05 gathering kernel.  cin a
 * multiple of 8 (paths 0, 2), cout a multiple of 8 and <= 64.  scratch:
 * device memory of scratch_bytes (>= 2 (27 cin + 64) * round_up(cout, 16)
 * suffices) for the rearranged weights; *err_dev (caller-zeroed) is set to 1
 * if a tensor-core wait gave up.  Asynchronous on `stream`; allocates
 * nothing.  No counterpart in the paper.
 */
OSMODI_API osmodi_status osmodi_conv3d(const void* x_dev, const void* w_dev, const float* bias_dev, void* y_dev, int D,
                                       int H, int W, int cin, int cout, int relu, int path, void* scratch_dev,
                                       size_t scratch_bytes, int* err_dev, void* stream);
/* OSMODI_E_TIMEOUT (and the flag cleared) if a tensor-core wait of an
 * earlier network call gave up, else OSMODI_OK; synchronous.  get_output and
 * get_grads report the same. */
OSMODI_API osmodi_status osmodi_net_status(osmodi_net net);
/* the normalised network output of the last forward (nx*ny*nz floats) */
OSMODI_API osmodi_status osmodi_net_get_output(osmodi_net net, float* out_host);
/* P^0 = network output * s into p_dev (0 on missing cells); asynchronous */
OSMODI_API osmodi_status osmodi_net_forward(osmodi_net net, const void* grad_dev, int grad_dtype, const uint8_t* mask_dev,
                                            double spacing, void* p_dev, int p_dtype, void* stream);
/* forward + loss (mean over valid cells of the squared difference of the
 * mean-removed normalised output and target/s) + backward; gradients are
 * added to the accumulated ones.  loss_host may be NULL (else the call
 * synchronises). */
OSMODI_API osmodi_status osmodi_net_backward(osmodi_net net, const void* grad_dev, int grad_dtype, const uint8_t* mask_dev,
                                             double spacing, const double* target_dev, double* loss_host, void* stream);
/* one Adam step with the accumulated gradients divided by `batch`; clears them */
OSMODI_API osmodi_status osmodi_net_adam(osmodi_net net, double lr, double beta1, double beta2, double eps, int batch,
                                         void* stream);
OSMODI_API void osmodi_net_destroy(osmodi_net net);
OSMODI_API const char* osmodi_status_string(int status);
/* Text of the last CUDA error seen by this thread (empty if none). */
OSMODI_API const char* osmodi_last_cuda_error(void);

/*
 * Tensor-core GEMM step (no counterpart in the paper: the contraction the
 * seed network's convolutions are built from, exposed to check it against a
 * reference product): D = A B^T with A 128 x K and B N x K in BF16 (row-major,
 * K contiguous, 16-byte aligned), D 128 x N in FP32 (row-major), on the
 * tcgen05 tensor cores with the accumulator in tensor memory.  N and K
 * multiples of 16, 16 <= N, K <= 256.  *err_dev (device int, caller-zeroed)
 * is set to 1 if the MMAs did not complete within the kernel's bounded wait.
 * Asynchronous on `stream`.
 */
OSMODI_API osmodi_status osmodi_tc_gemm(const void* A_dev, const void* B_dev, float* D_dev, int N, int K,
                                        int* err_dev, void* stream);

/*
 * Measured FP64 arithmetic peak of the current device (no counterpart in
 * the paper; the second roofline of the FP64 refinement kernels): the best
 * of five timed launches (CUDA events on `stream`) of a kernel whose threads
 * run eight independent FP64 fused multiply-add chains, one wave of resident
 * blocks.  *gflops_out = 2 x FMAs / time in GFLOP/s; *ms_out (may be NULL)
 * = that launch's time.  Synchronous; allocates nothing.
 */
OSMODI_API osmodi_status osmodi_probe_fp64(double* gflops_out, double* ms_out, void* stream);

/*
 * The FP32 <-> FP64 conversions the FP64-throughput-bound kernels (the
 * refinement residual, the fold, the output, the float-float source) do on
 * the integer units instead of the conversion instructions (no counterpart
 * in the paper; a check that they are IEEE 754's): for i < n,
 * f_out[i] = d_in[i] rounded to binary32 (to nearest, ties to even) and
 * d_out[i] = f_in[i] as binary64 (exact).  All four are device arrays of n
 * elements, owned by the caller.  OSMODI_E_INVALID: n < 0 or a null array
 * with n > 0.  Asynchronous on `stream`.
 */
OSMODI_API osmodi_status osmodi_probe_convert(const double* d_in_dev, float* f_out_dev, const float* f_in_dev,
                                              double* d_out_dev, int64_t n, void* stream);

/*
 * Test knobs, for exercising the failure statuses without a GPU fault (no
 * counterpart in the paper).  Process-wide; every later call reads them.
 * Returns the previous value; OSMODI_DEBUG_DEFAULT restores the default.
 *
 * OSMODI_DEBUG_BARRIER_SPINS: polls (each followed by a ~64 ns sleep) a grid
 *   barrier of the batched persistent kernel makes before it gives up, sets
 *   the batch's error flag and lets every block return (the call then
 *   reports OSMODI_E_TIMEOUT).  Default (0): 2^25, about 2 s.
 * OSMODI_DEBUG_SKIP_BARRIER_BLOCK: the block of the batched persistent
 *   kernel with this index returns before its first grid barrier, so the
 *   other blocks' barrier runs out of polls.  Default (-1): none.
 * OSMODI_DEBUG_CORRECTION_SCALE: osmodi_solve multiplies each refinement
 *   step's correction by this factor before adding it (0: no scaling); a
 *   large factor makes the residual grow and the solve report
 *   OSMODI_E_DIVERGED.
 * OSMODI_DEBUG_MG_UNFUSED: how the 3-D multigrid preconditioner smooths,
 *   the same arithmetic in each case, for comparisons: 0 (default) fused
 *   one-pass red-black sweeps (every level with packed counts); 1
 *   one-colour half-sweeps in place (two passes per sweep); 2 as 0 with the
 *   fine level's input planes staged by TMA (FP32 plans); 3 as 0 with the
 *   fine sweeps' HBM operands loaded one plane ahead; 4 as 0 with the fine
 *   level's z, r and code planes staged in shared memory by cp.async (FP32
 *   plans).
 * OSMODI_DEBUG_NET_WMMA: which kernels run the seed network's
 *   convolutions, the same products in each case, for comparisons: 0
 *   (default) tcgen05, the forward 3x3x3 layers with their input tile staged
 *   once; 1 the warp-level (wmma) tensor-core path; 2 tcgen05, every layer by
 *   the gathering kernel.
 * OSMODI_DEBUG_BATCH_BOTTOM_CELLS: the batched solve's multigrid runs the
 *   coarse levels of at most this many cells (and the ones below them)
 *   inside one block per instance, the larger ones as grid-wide passes; the
 *   same V-cycle either way.  Default (0): 4096.
 * OSMODI_DEBUG_CG_FIXED_GRAPH: how osmodi_solve's captured CG runs, the same
 *   kernels in the same order, for comparisons: 0 (default) one graph per
 *   CG segment holding a device-side loop (a conditional while node) that
 *   stops at convergence; 1 graphs of check_every iterations relaunched by
 *   the host until the device reports convergence (iterations past it
 *   launch kernels that return at once).
 */
#define OSMODI_DEBUG_BARRIER_SPINS 1
#define OSMODI_DEBUG_SKIP_BARRIER_BLOCK 2
#define OSMODI_DEBUG_CORRECTION_SCALE 3
#define OSMODI_DEBUG_MG_UNFUSED 4
#define OSMODI_DEBUG_NET_WMMA 5
#define OSMODI_DEBUG_BATCH_BOTTOM_CELLS 6
#define OSMODI_DEBUG_CG_FIXED_GRAPH 7
#define OSMODI_DEBUG_DEFAULT (-0x7fffffffffffffffLL)
OSMODI_API long long osmodi_debug_set(int knob, long long value);

#ifdef __cplusplus
}
#endif

#endif /* OSMODI_H */
