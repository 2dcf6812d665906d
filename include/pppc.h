/*
 * pppc.h -- C ABI of the GB300 library for the periodic eddy-current problem
 *
 *     M du/dt + K(u) u = f(t),  t in (0, T),   u(0) = u(T)        (Sec. 2, Eq. 1)
 *
 * solved by the periodic Parareal algorithm with a periodic coarse problem
 * (PP-PC, Eq. 4) whose block-cyclic coarse system (Eqs. 9-10) is solved
 * harmonic by harmonic after a discrete Fourier transform along the time
 * axis (Sec. 3, Eqs. 11-14).
 *
 * Conventions shared by every call
 *  - All calls return a pppc_status; nothing throws across the ABI.  After a
 *    failure, pppc_last_error(h) holds a one-line reason.
 *  - All device work is ordered on the stream given in pppc_config.stream
 *    (a cudaStream_t; NULL means the legacy default stream).  Calls that
 *    return scalars (iterate, solve_periodic, propagate_fine, coarse_update)
 *    synchronise that stream before returning.
 *  - A handle is not thread-safe; separate handles are independent.
 *  - States are FP64, laid out subinterval-major over ALL mesh nodes:
 *    U[n * n_nodes + i] is node i at the coarse point T_n = n T / N,
 *    n = 0..N-1.  Dirichlet nodes are ignored on input and returned as 0.
 *  - "on_device" != 0 means the pointer is CUDA device memory valid on the
 *    handle's stream; 0 means host memory (copied inside the call).  The
 *    caller owns every buffer it passes; the library keeps no pointer to it
 *    after the call returns.
 *  - The handle owns all device workspace; it is allocated by
 *    pppc_set_mesh and released by pppc_destroy.
 */
#ifndef PPPC_H
#define PPPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pppc_status {
    PPPC_OK = 0,
    PPPC_ERR_INVALID_ARG = 1,   /* bad pointer, size, index, degenerate triangle ... */
    PPPC_ERR_CUDA = 2,          /* a CUDA runtime call failed (message in last_error) */
    PPPC_ERR_STATE = 3,         /* call out of order (e.g. no mesh or source yet) */
    PPPC_ERR_NEWTON = 4,        /* a fine-step Newton iteration hit max_newton */
    PPPC_ERR_LINEAR = 5,        /* PCG or COCG hit its iteration cap */
    PPPC_ERR_BREAKDOWN = 6,     /* PCG/COCG breakdown (zero or non-positive curvature) */
    PPPC_ERR_NAN = 7,           /* a non-finite residual appeared */
    PPPC_ERR_TIMEOUT = 8,       /* a device-side grid barrier gave up waiting */
    PPPC_ERR_NOT_CONVERGED = 9, /* solve_periodic reached kmax; state kept, resumable */
    PPPC_ERR_UNSUPPORTED = 10,  /* valid request this build does not provide */
    PPPC_ERR_NOMEM = 11         /* device allocation failed */
} pppc_status;

typedef enum pppc_precision {
    PPPC_FP64 = 0,   /* every operation in FP64 */
    PPPC_MIXED = 1   /* FP32 fine PCG; FP64 Newton residual, jumps, DFT, COCG, update */
} pppc_precision;

typedef enum pppc_coarse_lin {
    /* The paper leaves the coarse matrix of the nonlinear case open (end of
     * Sec. 2).  Within iteration k the coarse stiffness Kbar is frozen as: */
    PPPC_COARSE_AVG_JACOBIAN = 0, /* (1/N) sum_n dK(U)U/dU at U = U_n^k  (default) */
    PPPC_COARSE_AVG_CHORD = 1,    /* (1/N) sum_n K(U_n^k) */
    PPPC_COARSE_ZERO_FIELD = 2    /* dK(U)U/dU at U = 0 */
} pppc_coarse_lin;

/* The frozen coarse stiffness Kbar^k (Eq. 8 with a nonlinear K; the paper
 * leaves it open) is averaged over the N coarse points of the period, taken
 * either at the iterate U_n^k or at the fine results F_n^k.  At the fixed
 * point the two coincide.  The fine results come from physical time
 * stepping, so they keep Kbar meaningful when U^k is far from any
 * physical state (a cold start of a strongly nonlinear cable). */
typedef enum pppc_coarse_at {
    PPPC_COARSE_AT_U = 0,
    PPPC_COARSE_AT_F = 1
} pppc_coarse_at;

typedef enum pppc_method {
    PPPC_METHOD_PPPC = 0, /* periodic coarse problem, multi-harmonic solve (Eq. 4, Eqs. 9-14) */
    PPPC_METHOD_PPIC = 1  /* relaxed periodicity U_0^{k+1} = U_N^k with an initial-value coarse
                             sweep (Eq. 5); the handle also keeps the end-of-period state U_N */
} pppc_method;

typedef enum pppc_nu_model {
    PPPC_NU_LINEAR = 0,  /* constant reluctivity nu */
    PPPC_NU_BRAUER = 1   /* nu(B^2) = k1 exp(k2 B^2) + k3 */
} pppc_nu_model;

/* Material of one region (index = value in the region[] array). */
typedef struct pppc_material {
    double sigma;       /* conductivity [S/m]; > 0 puts the region into M */
    int32_t nu_model;   /* pppc_nu_model */
    double nu;          /* reluctivity [m/H] for PPPC_NU_LINEAR, > 0 */
    double k1, k2, k3;  /* Brauer constants for PPPC_NU_BRAUER, k1,k3 > 0, k2 >= 0 */
    int32_t is_source;  /* 1: carries the impressed current I(t) uniformly */
    double bmax;        /* Brauer only: |B| [T] past which nu(b), b = |B|^2, continues along
                           its tangent at b = bmax^2 instead of exponentially (the fit has
                           no meaning past saturation and overflows on far-off Newton or
                           coarse iterates); nu and nu' stay continuous; 0: no cap */
} pppc_material;

/* Opaque handle: one problem (mesh, materials, source, time grid, state). */
typedef struct pppc_handle pppc_handle;

typedef void* (*pppc_alloc_fn)(size_t bytes, void* ctx);
typedef void (*pppc_free_fn)(void* ptr, void* ctx);

typedef struct pppc_config {
    double T;             /* period [s], > 0 */
    int32_t N;            /* subintervals [T_{n-1}, T_n], even, 2..1024 */
    int32_t n_fine;       /* implicit-Euler steps per subinterval, >= 1 */
    int32_t precision;    /* pppc_precision */
    int32_t coarse_lin;   /* pppc_coarse_lin */
    double tol_newton;    /* fine Newton stop: ||R||_2 <= tol_newton * ||g||_2 * sum_j |amp_j| */
    int32_t max_newton;   /* Newton iteration cap per fine step */
    double tol_lin;       /* smallest PCG forcing term (relative residual of one solve) */
    int32_t max_lin;      /* PCG iteration cap per Newton iteration */
    double tol_coarse;    /* COCG stops harmonic p at ||r_p||^2 <= tol_coarse^2 *
                             max(||b_p||^2, sum_q ||b_q||^2 / (N/2+1)) */
    int32_t max_coarse;   /* COCG iteration cap */
    void* stream;         /* cudaStream_t; NULL = legacy default stream */
    pppc_alloc_fn alloc;  /* optional device allocator (NULL: cudaMalloc) */
    pppc_free_fn free_fn; /* matching free (NULL: cudaFree) */
    void* alloc_ctx;      /* passed to alloc/free_fn */
    double eta0;          /* PCG forcing term of each step's first Newton iteration; later ones
                             follow Eisenstat-Walker, 0.9 (|R_k|/|R_k-1|)^2, within [tol_lin, 0.1] */
    int32_t predictor;    /* Newton start of each fine step: 0 u^m; 1 (default) 2 u^m - u^{m-1};
                             2 3 u^m - 3 u^{m-1} + u^{m-2} (quadratic extrapolation) */
    int32_t method;       /* pppc_method (default PPPC_METHOD_PPPC) */
    int32_t coarse_at;    /* pppc_coarse_at: where the coarse stiffness is frozen (default U^k) */
    int32_t newton_schedule; /* 1: inexact PP-PC, the fine Newton tolerance of iteration k is
                                max(tol_newton, min(1e-6, 1e-3 rel_res(U^{k-1}))): early
                                iterates, whose jumps are large, are propagated less exactly;
                                the last ones at tol_newton (default 0: always tol_newton) */
    int32_t precond;      /* fine PCG preconditioner: 0 Jacobi (default); 1 the tridiagonal part of
                             every 4 consecutive rows, factorised per lane (row order should follow
                             the mesh's strongest couplings, e.g. the rings of a polar mesh);
                             2 one V-cycle of smoothed-aggregation algebraic multigrid: the
                             aggregates and prolongators are built once by pppc_set_mesh from
                             the Newton matrix at zero field, each subinterval's coarse matrices
                             are the Galerkin products of its own Jacobian (rebuilt at the first
                             Newton iteration of every fine step), with l1-Jacobi smoothing on
                             every level, so the
                             preconditioner stays symmetric positive definite for every lane
                             and its iteration count hardly grows with the mesh; a mesh too
                             small to coarsen falls back to Jacobi */
    int32_t lane_team;    /* how the N subintervals of a fine sweep share the GPU.  The sweep's
                             lanes are independent, so they run as teams of lane_team lanes, each
                             team on its own share of the SMs with its own barriers and
                             reductions, never waiting for another team.
                             0 (default): chosen by measurement at the handle's first sweep --
                               every candidate V 2^i (V = 4 lanes in PPPC_MIXED, 2 in PPPC_FP64)
                               dividing the padded N is timed on the sweep's first fine level,
                               and the fastest is kept for every handle of the process with the
                               same precision, padded N, preconditioner and floor(log2 ndof);
                             > 0: that many lanes per team (one of the candidates, else
                               INVALID_ARG from pppc_set_mesh);
                             -1: one team over all lanes.
                             Results agree to rounding whatever the choice; they are bitwise
                             reproducible for a fixed choice. */
} pppc_config;

/* Iteration counts of the most recent iterate / solve / propagate call. */
typedef struct pppc_stats {
    int64_t newton_iters;    /* Newton iterations, summed over steps (max over lanes per step) */
    int64_t pcg_iters;       /* PCG iterations, summed over Newton iterations (lockstep) */
    int64_t cocg_iters;      /* COCG iterations of the coarse solves (lockstep over harmonics) */
    int64_t fine_steps;      /* implicit-Euler steps per lane */
    int32_t pppc_iters;      /* completed PP-PC updates */
    double rel_res;          /* last ||d|| / ||F|| */
    double fine_ms;          /* device time of the fine-propagator launches (CUDA events) */
    double coarse_ms;        /* device time of the coarse kernels (jumps .. update) */
    int64_t launches;        /* kernels this library launched during the call */
    int64_t backtracks;      /* Newton rounds of the fine sweeps in which some lane halved its step
                                because the residual did not drop (0 on well-behaved problems) */
    int64_t pcg_lane_rounds; /* sum over lane teams of PCG rounds x lanes per team: the lane
                                vectors the PCG iterations streamed */
    int64_t pcg_lane_iters;  /* sum over subintervals of the PCG iterations each one needed;
                                1 - pcg_lane_iters / pcg_lane_rounds is the lockstep idle share */
    int64_t newton_lane_rounds; /* sum over lane teams of Newton rounds x lanes per team */
    int64_t graph_launches;  /* CUDA graph launches: with PPPC_METHOD_PPPC and no trace, every
                                iterate / solve iteration is one captured graph (fine sweep, jumps,
                                Kbar, DFT, harmonic solves, inverse DFT + update) and one host sync */
} pppc_stats;

/* Fill *cfg with defaults: T=0.02, N=16, n_fine=20, FP64, averaged Jacobian,
 * tol_newton=1e-10, max_newton=30, tol_lin=1e-6, max_lin=20000,
 * tol_coarse=1e-8, max_coarse=20000, default stream, cudaMalloc,
 * eta0=1e-2, predictor=1.  In PPPC_MIXED the PCG forcing term is at least
 * 1e-4 (an FP32 solve cannot refine further; Newton's FP64 residual does). */
void pppc_config_default(pppc_config* cfg);

/* Create a handle for the time grid of Sec. 2: N subintervals of length
 * dT = T/N (the coarse step, Eq. 8), each marched with n_fine implicit-Euler
 * fine steps of dt = T/(N n_fine) (Eq. 3).  *out is NULL on error.
 * Errors: INVALID_ARG (null pointer, N odd or out of range, T <= 0, ...). */
pppc_status pppc_create(const pppc_config* cfg, pppc_handle** out);

/* Release the handle and all its device memory.  NULL is a no-op. */
void pppc_destroy(pppc_handle* h);

/* Upload the mesh and materials of the space discretisation of Eq. 1
 * (linear triangles, nodal A_z): xy[2*n_nodes] coordinates [m];
 * tri[3*n_tri] node indices; region[n_tri] in [0, n_regions);
 * dirichlet[n_nodes] (1 = A fixed to 0); mat[n_regions].  Builds the sparse
 * pattern and element maps on the host and the matrices K_lin, M and the
 * source shape g on the device.  Host arrays are only read during the call.
 * Resets the state to U = 0.
 * Errors: INVALID_ARG (index out of range, zero-area triangle, nu <= 0, no
 * free node, no source region), NOMEM, CUDA. */
pppc_status pppc_set_mesh(pppc_handle* h, int32_t n_nodes, const double* xy, int32_t n_tri,
                          const int32_t* tri, const int32_t* region, const uint8_t* dirichlet,
                          int32_t n_regions, const pppc_material* mat);

/* Impressed current of the source regions (the excitation f of Eq. 1):
 * I(t) = sum_j amp[j] sin(2 pi freq[j] t + phase[j]), spread uniformly over
 * the discrete source area so that the nodal source sums to I(t).
 * Errors: INVALID_ARG if n_harm < 1 or some freq[j] * T is not an integer
 * (f must be T-periodic, Eq. 1); STATE before set_mesh. */
pppc_status pppc_set_source(pppc_handle* h, int32_t n_harm, const double* amp, const double* freq,
                            const double* phase);

/* Set / read the PP-PC state U_0..U_{N-1} (layout above).  With
 * PPPC_METHOD_PPIC, set_state also sets the end-of-period state U_N to U_0. */
pppc_status pppc_set_state(pppc_handle* h, const double* U, int32_t on_device);
pppc_status pppc_get_state(pppc_handle* h, double* U, int32_t on_device);

/* All N fine propagators at once (Eqs. 2-3): F[j] = F_{j+1}(U[j]) for
 * j = 0..N-1, i.e. subinterval j+1 marched from U_j at T_j to T_{j+1}.
 * U and F use the state layout; they may not alias.  Does not change the
 * handle's state.  Errors: NEWTON, LINEAR, BREAKDOWN, NAN, TIMEOUT, CUDA. */
pppc_status pppc_propagate_fine(pppc_handle* h, const double* U, double* F, int32_t on_device);

/* A window of the fine sweep (Eq. 3 on part of each subinterval): every
 * subinterval j+1 marches `count` implicit-Euler steps from its fine level
 * `first`, i.e. U[j] is the state at t = T_j + first dt and F[j] receives the
 * state at T_j + (first + count) dt, with dt = T / (N n_fine) as in
 * pppc_propagate_fine.  Windows [0, a), [a, b), ..., [c, n_fine) chained
 * through F reproduce pppc_propagate_fine up to the Newton tolerance (each
 * window starts its first step's Newton from u itself, not from an
 * extrapolation).  Layout, aliasing and errors as pppc_propagate_fine, plus
 * INVALID_ARG unless 0 <= first, 1 <= count and first + count <= n_fine. */
pppc_status pppc_propagate_fine_window(pppc_handle* h, const double* U, double* F, int32_t first, int32_t count,
                                       int32_t on_device);

/* The coarse part of one PP-PC iteration (Eq. 4 with the implicit-Euler
 * coarse propagator of Eq. 8, solved through Eqs. 9-14): given U^k and the
 * fine values F[j] = F_{j+1}(U^k_j), write U^{k+1} to U_new and
 * ||d|| / ||F|| of U^k (d_n = F_n - U_{n mod N}) to *rel_res (may be NULL).
 * Does not change the handle's state.  Errors: LINEAR, BREAKDOWN, TIMEOUT,
 * CUDA; UNSUPPORTED with PPPC_METHOD_PPIC (its update also needs U_N). */
pppc_status pppc_coarse_update(pppc_handle* h, const double* U, const double* F, double* U_new,
                               double* rel_res, int32_t on_device);

/* One iteration on the handle's state, U^k -> U^{k+1}: PP-PC (Eq. 4), or
 * PP-IC (Eq. 5) with PPPC_METHOD_PPIC, whose coarse sweep solves
 * Q = M/dT + Kbar once per subinterval in sequence.
 * *rel_res (may be NULL) receives ||d|| / ||F|| of the incoming U^k. */
pppc_status pppc_iterate(pppc_handle* h, double* rel_res);

/* Iterate until rel_res(U^k) <= tol or kmax updates are done.  On success
 * the state is the first U^k that passed and *iters = k (the number of
 * completed updates).  Errors: NOT_CONVERGED (state = U^kmax, resumable),
 * and those of pppc_iterate.  iters and rel_res may be NULL. */
pppc_status pppc_solve_periodic(pppc_handle* h, double tol, int32_t kmax, int32_t* iters,
                                double* rel_res);

/* ---- Allocation-free harmonic solve ---------------------------------------
 * The paper has no counterpart to this call.  It exists for callers that
 * cannot allocate device memory -- for example a plugin that only receives
 * buffers from a host application which owns every allocation, or a loop
 * that cannot afford the device synchronisation cudaMalloc implies.  The
 * handle-based calls above allocate their workspace in pppc_set_mesh, so
 * such callers cannot use them; this call allocates nothing.
 *
 * It solves, for every harmonic p = 0..N/2 at once, the complex symmetric
 * system (K + (1 - exp(-i 2 pi p / N)) C) x_p = b_p with the same batched
 * Jacobi-preconditioned COCG kernel as the coarse solve of pppc_iterate.
 * K and C are real n x n matrices on one CSR pattern (rowptr[n+1], col[nnz],
 * kval[nnz], cval[nnz] with nnz = rowptr[n]; rowptr[0] = 0, rowptr never
 * decreases, every col entry lies in [0, n) and every row holds its diagonal
 * entry).  The pattern is checked on the device before the solve: rowptr
 * first, and col only once rowptr has passed, so a bad pattern returns
 * PPPC_ERR_INVALID_ARG without any out-of-range access.  b and x are
 * complex, interleaved (re, im), laid out [n][N/2+1].  All pointers are
 * device memory owned by the caller; the call stops when every harmonic's
 * ||r_p||^2 <= tol^2 * max(||b_p||^2, sum_q ||b_q||^2 / (N/2+1)) (its own
 * relative tol, or tol times the average right-hand side where its own is
 * smaller; the sum over p of ||r_p||^2 stays within 2 tol^2 times that of
 * ||b_p||^2) or after max_it iterations, writes the
 * iterations done to *iters_out (may be NULL) and synchronises `stream`
 * (a cudaStream_t, NULL = legacy default stream) before returning.
 *
 * Its work vectors live in one static device array of
 * PPPC_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits.  Limits: N even, 2 <= N <= PPPC_NOALLOC_MAX_N, and
 * n * (N/2 + 1) <= PPPC_NOALLOC_MAX_UNKNOWNS; larger requests return
 * PPPC_ERR_INVALID_ARG before any device work.  The first call on each device looks up the array's device
 * address (with that device current); make that first call before any stream
 * capture.  Every call shares the array and clears what must start at zero;
 * calls that overlap on the GPU (other streams or host threads on the same
 * device) race and must be serialised by the caller.
 * Errors: INVALID_ARG, LINEAR, BREAKDOWN, NAN, TIMEOUT, CUDA. */
#define PPPC_NOALLOC_MAX_N 256
#define PPPC_NOALLOC_MAX_UNKNOWNS 65536
#define PPPC_NOALLOC_SCRATCH_BYTES (12u << 20)
pppc_status pppc_harmonic_solve_noalloc(int32_t n, const int32_t* rowptr, const int32_t* col,
                                        const double* kval, const double* cval, int32_t N,
                                        const double* b, double* x, double tol, int32_t max_it,
                                        void* stream, int32_t* iters_out);

/* Iteration counts of the last propagate / coarse / iterate / solve call.
 * newton_iters and pcg_iters are lockstep rounds: per fine sweep the largest
 * count over the lane teams (the sweep's critical path), summed over sweeps. */
pppc_status pppc_get_stats(pppc_handle* h, pppc_stats* out);

/* The lane-team split of the fine sweep in use (pppc_config.lane_team) and
 * what the tuner measured for each candidate. */
typedef struct pppc_fine_plan_info {
    int32_t lanes_per_team;     /* 0: not chosen yet (before the first sweep); -1: one team */
    int32_t teams;
    int32_t threads_per_row;    /* lanes_per_team / lanes per thread (4 FP32, 2 FP64) */
    int32_t blocks_min, blocks_max;  /* blocks (one per SM) per team */
    int32_t n_candidates;
    int32_t candidate_lanes[16];
    double candidate_ms[16];    /* device time of one fine level per candidate, 0 if not timed
                                   by this handle (its bucket had been tuned before) */
    int32_t amg_levels;         /* multigrid levels of precond = 2 (0: not in use) */
    int32_t amg_rows[10];       /* rows of each level, finest first */
} pppc_fine_plan_info;
pppc_status pppc_get_fine_plan(pppc_handle* h, pppc_fine_plan_info* out);

/* Newton trace of the fine propagators (diagnostics).  pppc_set_trace(h, cap)
 * with cap > 0 makes every later fine sweep record up to cap records of
 * 5 doubles: {fine step, Newton iteration, max over subintervals of ||R||_2,
 * subintervals still iterating, PCG iterations of the preceding solve};
 * cap = 0 turns it off.  pppc_get_trace copies at most cap records of the
 * last sweep into out[5*cap] (host memory) and stores the number recorded
 * (which may exceed cap) in *n.  Errors: INVALID_ARG, STATE, NOMEM. */
pppc_status pppc_set_trace(pppc_handle* h, int32_t cap);
pppc_status pppc_get_trace(pppc_handle* h, double* out, int32_t cap, int32_t* n);

/* Number of free nodes (degrees of freedom) after Dirichlet elimination. */
int32_t pppc_ndof(pppc_handle* h);

/* Sizes of the assembled system (for roofline accounting). */
typedef struct pppc_mesh_counts {
    int64_t ndof;             /* free nodes */
    int64_t nnz;              /* entries of the sparse pattern */
    int64_t special_rows;     /* rows touching a nonlinear or conductive element */
    int64_t special_entries;  /* entries of those rows (values stored per lane) */
    int64_t nonlinear_elems;  /* triangles with the Brauer law */
} pppc_mesh_counts;
pppc_status pppc_get_mesh_counts(pppc_handle* h, pppc_mesh_counts* out);

/* One-line description of the last error on h (owned by h), or of the last
 * pppc_create failure when h is NULL. */
const char* pppc_last_error(pppc_handle* h);

/* Static name of a status code. */
const char* pppc_status_string(pppc_status s);

/* ---- Failure detection self-test ------------------------------------------
 * Every device-side wait of the library (grid barriers of the fine sweep and
 * of the harmonic solves) gives up after 2 s of %globaltimer, sets a status
 * word that the host maps to PPPC_ERR_TIMEOUT, and returns, so the context
 * stays usable.  This call runs that path on purpose: one block waits, with
 * the same bounded spin, on a device flag that nothing sets.  It returns
 * PPPC_ERR_TIMEOUT after about 2 s (PPPC_ERR_CUDA if the launch fails) and
 * synchronises `stream` (NULL = legacy default stream).  It allocates 8
 * bytes of device memory and frees them. */
pppc_status pppc_selftest_wait_timeout(void* stream);

/* Target of the device code this library was built with, as the CUDA
 * runtime reports it for the library's kernels (cudaFuncGetAttributes,
 * binaryVersion = 10 major + minor; 103 for GB300's sm_103a).  Needs a
 * device; no device work.  Errors: INVALID_ARG (out NULL), CUDA (no device,
 * or no kernel image for it). */
pppc_status pppc_binary_version(int32_t* out);

/* ---- Periodic adjoint: gradient of the eddy-current loss -------------------
 * Not in the paper; it reuses its method backwards in time.  For the periodic
 * state held by the handle (solve it first, e.g. pppc_solve_periodic to
 * 1e-10 or tighter: the gradient is exact for the discrete periodic solution
 * the state approximates), with the implicit-Euler scheme of the fine
 * propagator (dt = T / (N n_fine), L = N n_fine levels, u^0 = u^L), the
 * period-averaged eddy-current loss is
 *     P = (1/T) sum_m (u^m - u^{m-1})^T M (u^m - u^{m-1}) / dt      [W/m].
 * Its gradient with respect to the conductivity and the Brauer constants of
 * one nonlinear, conducting region r follows from the periodic adjoint
 *     (M/dt + J_m) lam_m = (M/dt) lam_{m+1} + (2/(T dt)) M (du^m - du^{m+1}),
 * a linear periodic problem backwards in time, solved by PP-PC with the
 * multi-harmonic coarse solve (Eq. 4, Eqs. 11-14) run backwards.  Its fine
 * propagators are the fine sweep's kernel in adjoint mode (each level an
 * iteratively refined PCG solve with the handle's preconditioner), with the
 * Jacobians J_m taken at the forward trajectory, which one forward fine
 * sweep from the state recomputes at the start of the call.  Kbar is the
 * forward's.
 *     dP/dsigma_r = P_r / sigma_r - sum_m lam_m^T (M_r / sigma_r) du^m / dt,
 *     dP/dk_i     = - sum_m lam_m^T d(K(u^m) u^m)/dk_i.
 * tol and kmax bound the adjoint PP-PC (rel_res of the adjoint jumps).
 * Errors: INVALID_ARG (region not nonlinear and conducting, tol <= 0),
 * STATE (no mesh/source, or the state's rel_res > 1e-6: not periodic),
 * UNSUPPORTED (PP-IC handle), NOT_CONVERGED, the fine sweep's errors, NOMEM.
 * The handle's state is unchanged. */
typedef struct pppc_adjoint_result {
    double loss;          /* P over all conducting regions [W/m] */
    double grad[4];       /* dP/d(sigma_r, k1_r, k2_r, k3_r) */
    int32_t iterations;   /* adjoint PP-PC updates */
    double rel_res;       /* final adjoint rel_res */
    double forward_rel_res; /* rel_res of the handle's state */
} pppc_adjoint_result;

pppc_status pppc_adjoint(pppc_handle* h, int32_t region, double tol, int32_t kmax, pppc_adjoint_result* out);

/* ---- Many independent problems in one launch ------------------------------
 * The paper solves one problem at a time.  A batch runs PP-PC (Eq. 4 with the
 * multi-harmonic coarse solve, Eqs. 11-14) on many independent problems --
 * cables of different meshes, materials, sources, N and n_fine -- at once.
 * Each batch iteration runs two captured CUDA graphs:
 *   1. one cooperative launch in which every active member's fine sweep runs
 *      on its own team of blocks (each team has its own grid barrier and
 *      reductions), then every member's jumps;
 *   2. every member's coarse linearisation and right-hand side, one
 *      cooperative launch of all members' harmonic solves (again one team per
 *      member), and every member's inverse DFT + update.
 * Every member's fine sweep runs as lane teams (pppc_batch_get_lanes), each
 * team a unit of the block split.  Block counts start from a cost model
 * (rows x lanes x fine steps) and, with autotune = 1, are re-balanced from
 * the per-team times the kernels measure (%globaltimer) whenever that
 * shortens the predicted launch by more than 10%; the graphs are captured
 * again after every change of teams or of the set of active members.
 *
 * Members are handles that already have a mesh, a source and a state, all
 * with the same precision, the PP-PC method, the same stream (cfg.stream)
 * and NB / (4 FP32 or 2 FP64 lanes) a power of two (e.g. N = 16, 32, 64).
 * At most one member per SM.  The batch uses the members' own workspaces and
 * states: pppc_get_state on a member reads its current U^k.  The batch runs
 * its graphs on a stream of its own; each batch call first synchronises the
 * members' stream and returns once its work is complete.  While the batch
 * exists, the members must not be used on their own or in another batch.
 * Destroy the batch before its members.
 *
 * Errors of pppc_batch_create: INVALID_ARG (count < 1, NULL member,
 * duplicate), STATE (member without mesh, source), UNSUPPORTED (mixed
 * precisions or streams, PP-IC, newton_schedule, a lane count that is not a
 * power of two, count > SMs), CUDA, NOMEM.  The message is in pppc_batch_last_error(NULL)
 * after a failed create. */
typedef struct pppc_batch pppc_batch;

typedef struct pppc_batch_stats {
    int32_t iterations;        /* batch iterations run by the last call */
    int32_t retunes;           /* team re-partitions made by the tuner during the last call */
    int64_t graph_launches;    /* CUDA graph launches of the last call */
    int64_t kernel_launches;   /* kernels launched inside those graphs */
    int64_t fine_dof_steps;    /* sum over members and iterations of N * n_fine * ndof */
    double fine_ms;            /* device time of the fine-sweep graphs */
    double coarse_ms;          /* device time of the coarse graphs */
} pppc_batch_stats;

pppc_status pppc_batch_create(pppc_handle* const* members, int32_t count, int32_t autotune, pppc_batch** out);
void pppc_batch_destroy(pppc_batch* b);

/* One PP-PC iteration on every member: rel_res[count] (may be NULL) gets each
 * member's ||d|| / ||F|| of its incoming U^k. */
pppc_status pppc_batch_iterate(pppc_batch* b, double* rel_res);

/* Iterate every member until its rel_res <= tol (its state is then the first
 * U^k that passed and it stops iterating) or kmax updates are done.
 * iters[count] and rel_res[count] (each may be NULL) get every member's
 * update count and final residual.  Returns NOT_CONVERGED if any member did
 * not reach tol (all results are still written), else the first error of
 * any member (the message names it). */
pppc_status pppc_batch_solve_periodic(pppc_batch* b, double tol, int32_t kmax, int32_t* iters, double* rel_res);

pppc_status pppc_batch_get_stats(pppc_batch* b, pppc_batch_stats* out);

/* Current team sizes (blocks) of each member in the fine and coarse
 * launches: fine_blocks[count], cocg_blocks[count] (each may be NULL). */
pppc_status pppc_batch_get_teams(pppc_batch* b, int32_t* fine_blocks, int32_t* cocg_blocks);

/* Lane split of each member's fine sweep in the batch: lanes_per_team[count]
 * and teams[count] (each may be NULL).  A member's lanes run as teams of
 * lanes_per_team lanes -- its size bucket's choice of the single-handle
 * tuner (pppc_config.lane_team), widened while all members' teams outnumber
 * the SMs -- and every team is a unit of the batch's block split. */
pppc_status pppc_batch_get_lanes(pppc_batch* b, int32_t* lanes_per_team, int32_t* teams);

/* Last error on b, or of the last failed pppc_batch_create when b is NULL. */
const char* pppc_batch_last_error(pppc_batch* b);

/* The tuner's split, host only (no device work): blocks[count] for members
 * with costs cost[count] (time x blocks, > 0), caps cap[count] (>= 1) and
 * active[count] (0/1) over `total` blocks, minimising the largest
 * cost / blocks: every active member gets one block, then each further block
 * goes to the active member with the largest cost / blocks below its cap.
 * Inactive members get 0.  *makespan (may be NULL) receives the largest
 * cost / blocks.  Errors: INVALID_ARG (NULL array, count < 1, a cost <= 0
 * or cap < 1 of an active member, fewer blocks than active members). */
pppc_status pppc_batch_plan(const double* cost, const int32_t* cap, const int32_t* active, int32_t count,
                            int32_t total, int32_t* blocks, double* makespan);

#ifdef __cplusplus
}
#endif

#endif /* PPPC_H */
