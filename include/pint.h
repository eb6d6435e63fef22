/*
 * pint.h - C ABI of libpint: the all-at-once preconditioned iteration of the
 * diagonalization-based parallel-in-time (PinT) method of Garai & Mandal,
 * "Diagonalization Based Parallel-in-Time Method for a Class of Fourth Order
 * Time Dependent PDEs" (arXiv 2304.14021), on one NVIDIA GB300 (sm_103a).
 *
 * Equations (paper numbering):
 *   biharmonic heat         u_t = -Lap^2 u                        (Eq. 1.1, 2.1)
 *   linearized Cahn-Hilliard u_t = -beta^2 Lap u - eps^2 Lap^2 u  (Eq. 1.2, 3.1)
 *   Cahn-Hilliard           u_t = Lap(u^3 - u) - eps^2 Lap^2 u    (Eq. 1.3, 4.1)
 * on [0,1] or [0,1]^2, discretized by centred differences (Eq. 2.4) and
 * backward Euler or Crank-Nicolson (the theta-method of Eq. 2.5 with theta = 1 or 1/2; Eq. 4.5).
 *
 * One outer iteration (Sec. 2.1 Eq. 2.6-2.8; Sec. 4.1 Eq. 4.11-4.14, PinT-I)
 * is computed in residual-correction form,
 *     U <- U + P_alpha^{-1} (b - K(U)),
 * with K the alpha = 0 all-at-once operator and P_alpha its alpha-circulant
 * approximation; P_alpha^{-1} is applied by the three steps of Eq. 2.8:
 * alpha-scaled FFT along time, one shifted spatial solve per frequency, inverse
 * FFT and unscaling.  For Cahn-Hilliard the averaged Jacobian of Eq. 4.12 is
 * the scalar mean of 3u^2 over all space-time points, or with
 * PINT_OPT_VARYING_JACOBIAN the paper's time average of 3u^2 at each point.
 *
 * Memory: every pointer named *_dev is a CUDA device pointer in the current
 * device's primary context; *_host pointers are host memory.  Arrays are FP64,
 * C-contiguous, time-major [n][y][x] with x fastest (1-D: ny = 1).  The caller
 * owns all arrays it passes; a handle owns its workspace and tables, allocated
 * in pint_create and freed in pint_destroy.  All device work is issued on the
 * stream given to pint_create.  No function throws; each returns a pint code.
 */
#ifndef PINT_H
#define PINT_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define PINT_OK          0
#define PINT_EINVAL     -1   /* invalid or unsupported problem parameter / argument */
#define PINT_ENOMEM     -2   /* device or host allocation failed */
#define PINT_ECUDA      -3   /* a CUDA runtime call failed */
#define PINT_ENOCONV    -4   /* max_iter reached, or no decrease over three iterations (rounding
                                floor); U holds the last iterate, stats are filled */
#define PINT_EDIVERGED  -5   /* residual non-finite, grew by 1e6 over its first value, or
                                grew monotonically and by 10x over three iterations */

/* PINT_CAHN_HILLIARD:      fully implicit backward Euler (Eq. 4.5), preconditioner of Eq. 4.14 (PinT-I);
 * PINT_CAHN_HILLIARD_EYRE: Eyre's convex-concave splitting, u^3 implicit and the concave -u explicit
 *                          (Sec. 4.2), preconditioner of Eq. 4.25 (PinT-II). */
typedef enum { PINT_BIHARMONIC = 0, PINT_LINEAR_CH = 1, PINT_CAHN_HILLIARD = 2, PINT_CAHN_HILLIARD_EYRE = 3 } pint_equation;

/* Boundary conditions (Sec. 5.1 lists the variants):
 *  SIMPLY_SUPPORTED: u = Lap u = 0, vertex grid of n interior points, h = 1/(n+1);
 *                    spatial solves in the sine basis (DST-I, dense, n <= 1024).
 *  NEUMANN:          d_nu u = d_nu Lap u = 0, cell-centred grid of n cells, h = 1/n;
 *                    spatial solves in the cosine basis (DCT-II): by FFT when n is a
 *                    power of two (x: n <= 4096, y: n <= 1024), else dense (n <= 1024).
 *  NEUMANN_VERTEX:   the same conditions on the vertex grid of Eq. 2.4: n points including
 *                    both ends, h = 1/(n-1), ghosts u_{-1} = u_1; spatial solves in the
 *                    DCT-I basis cos(p pi j/(n-1)) (dense, 3 <= n <= 1024). */
typedef enum { PINT_BC_SIMPLY_SUPPORTED = 0, PINT_BC_NEUMANN = 1, PINT_BC_NEUMANN_VERTEX = 2 } pint_bc;

/* PINT_FP64:     every step in FP64 (the plain form).
 * PINT_MIXED:    residual, alpha-scaling, unscaling and the update in FP64; the
 *                time FFTs and the spatial shifted solves in FP32 / complex64, so
 *                the outer iteration is an iterative refinement.  For the linear
 *                equations on square cells (and in 1-D) the residual and its
 *                alpha-scaling run on the integer pipes in block fixed point: the
 *                FP64 iterate is converted per tile and time level to 64-bit integers
 *                in a common binary unit, the stencil sums are exact, and the
 *                products with the coefficients and with gamma_n/dt use their full
 *                53-bit mantissas, so every rounding lies below 2^-56 of the largest
 *                term (finer than the same sums in FP64); the scaled residual is
 *                rounded once to FP32 (see PINT_OPT_FX_RESIDUAL).
 * PINT_MIXED_FF: as PINT_MIXED, but the iterate and the residual are kept in
 *                float-float (two FP32 words, about 48 significant bits, error-free
 *                stencil sums) on the FP32 pipes, and the alpha-scaling/unscaling is
 *                an FP32 product.  No FP64 arithmetic in the iteration; the FP64
 *                result is assembled once per solve. */
typedef enum { PINT_FP64 = 0, PINT_MIXED = 1, PINT_MIXED_FF = 2 } pint_precision;

/* Problem statement (Eq. 2.1-2.2, 3.1-3.2, 4.1-4.2, the tolerance of Sec. 5). */
typedef struct {
    int    equation;     /* pint_equation */
    int    dim;          /* 1 or 2 */
    int    nx, ny;       /* grid points per axis; ny ignored (treated as 1) when dim == 1 */
    int    bc;           /* pint_bc */
    double eps;          /* interface width epsilon (linear and nonlinear CH) */
    double beta;         /* beta of the linearized CH equation; A = beta|beta| Lap + eps^2 Lap^2, so
                            beta < 0 gives the diffusive second-order term (signed beta^2) */
    double T;            /* final time; dt = T / (nt * n_windows) */
    int    nt;           /* time steps per window, a power of two in [2, 2^20]; above 1024 the number of
                            spatial points must be even (the multi-pass time FFT pairs neighbouring points) */
    int    n_windows;    /* consecutive windows; window w starts from the last step of window w-1 */
    double theta;        /* theta-method parameter (Eq. 2.5): 1 (backward Euler), or 1/2 (Crank-Nicolson)
                            for the linear equations; Cahn-Hilliard is backward Euler (Eq. 4.5) */
    double alpha;        /* PinT parameter alpha in (0, 1) (Eq. 2.2) */
    double tol;          /* stop when ||b - K(U)||_2 / ||b||_2 <= tol */
    int    max_iter;     /* outer iterations per window, 1..PINT_HIST_MAX */
    int    precision;    /* pint_precision */
    int    init_guess;   /* 0: each window starts from U^0 = u0 at every time level;
                            1: the first window starts from the iterate passed in U,
                               later windows as 0;
                            2: each window starts from U^0 = 0 (linear equations; for
                               Cahn-Hilliard this acts as 0, since the scalar Jacobian
                               of a zero iterate misleads the first preconditioner) */
    double tol_update;   /* 0: off.  > 0: a window also stops when the last correction is small,
                            ||delta||_2 / ||U||_2 <= tol_update (an error estimate, in the spirit of
                            the error-based stopping rule of Sec. 5).  For very stiff problems the
                            rounding of any iterate keeps ||b - K(U)|| / ||b|| near
                            eps * dt * max|spectrum of A|, so a residual tolerance alone can be
                            unreachable there while the iterate has converged. */
} pint_problem;

#define PINT_HIST_MAX 256

typedef struct {
    int    status;            /* PINT_OK, PINT_ENOCONV or PINT_EDIVERGED of the last window run */
    int    iters;             /* preconditioner applications, summed over windows */
    int    windows;           /* windows completed */
    int    iters_last;        /* iterations of the last window */
    double rel_residual;      /* final ||r||/||b|| of the last window */
    double contraction;       /* geometric mean of rho_k / rho_{k-1} over the last window */
    double jbar;              /* last averaged Jacobian mean(3u^2) (Cahn-Hilliard), else 0 */
    double hist[PINT_HIST_MAX];  /* rho_0 .. rho_{iters_last} of the last window */
    int    segments;          /* solves run (one per window, more under the adaptive window policy) */
    int    nt_min;            /* shortest segment length used */
    int    retries;           /* segments solved again with half the length (adaptive policy) */
    double update_norm;       /* ||delta||_2 / ||U||_2 of the last correction of the last window
                                 (computed when tol_update > 0, else 0) */
    int    precision;         /* pint_precision the solve ran in.  With amp = 2^-24 dt max|spectrum of A|:
                                 the requested one up to amp 1 (0.1 for Cahn-Hilliard); for the linear
                                 equations PINT_MIXED (FP64 residual and iterate) up to amp 1e3; beyond,
                                 PINT_FP64, where FP32 inner solves cannot be refined */
    int    time_gemm;         /* time transforms on the tensor cores (PINT_OPT_TIME_GEMM): bit 0 Step 1,
                                 bit 1 Step 3, in the last window solved */
    int    fused_spatial;     /* 1: Step 2 ran as one fused 2-D kernel per frequency slice */
    int    tune_cached;       /* 1: the autotuner took this handle's choices from its table */
} pint_stats;

typedef struct pint_handle pint_handle;

/* Validate p, build the eigenvalue / twiddle tables (FP64 on the host) and
 * allocate the workspace on the current device.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  On success *out owns it all.
 * Errors: PINT_EINVAL (bad parameter: dim, sizes, nt not a power of two,
 * NEUMANN with n not a power of two, alpha not in (0,1), theta not 1 or 1/2, ...),
 * PINT_ENOMEM, PINT_ECUDA. */
int pint_create(const pint_problem* p, void* cuda_stream, pint_handle** out);

/* Device bytes pint_create would allocate for p (workspace + tables), or a
 * negative code if p is invalid.  Used for admission by memory footprint. */
long long pint_footprint(const pint_problem* p);

/* Run the PinT iteration over all windows.
 *  u0_dev: initial condition, nx*ny doubles (read only).
 *  U_dev:  nt*nx*ny doubles; on return the iterate of the last window
 *          (time levels 1..nt of that window).  With init_guess = 1 it also
 *          supplies the first window's initial iterate.
 *  st:     may be NULL.
 * Returns PINT_OK when every window reached tol, else PINT_ENOCONV /
 * PINT_EDIVERGED (iteration stopped at that window; U holds its last
 * iterate), or PINT_EINVAL / PINT_ECUDA.  Blocks the host until the stream
 * has finished the solve. */
int pint_solve(pint_handle* h, const double* u0_dev, double* U_dev, pint_stats* st);

/* Solve n independent instances concurrently: instance i is pint_solve(hs[i],
 * u0s[i], Us[i], &st[i]).  Each instance is driven by its own host thread (up to
 * 64 at a time); instances whose handles were created on different streams run
 * concurrently on the GPU, each window's iteration loop as one CUDA graph.
 * Handles may not repeat.  st and rcs (per-instance return codes) may be NULL.
 * Returns PINT_OK, or the first non-zero instance code in index order. */
int pint_solve_batch(pint_handle* const* hs, int n, const double* const* u0s, double* const* Us, pint_stats* st,
                     int* rcs);

/* pint_solve with host buffers: copies u0_host (and U_host if init_guess = 1)
 * to handle-owned device buffers, solves, copies the result to U_host. */
int pint_solve_host(pint_handle* h, const double* u0_host, double* U_host, pint_stats* st);

/* All-at-once residual of one window (Eq. 2.6 / Eq. 4.8 with alpha = 0):
 * r = b - K(U), b = (u0/dt, 0, ..., 0).  r_dev (nt*nx*ny doubles) may be NULL;
 * *rel_res (may be NULL) receives ||r||_2 / ||b||_2.  Computed in FP64
 * arithmetic, or on a PINT_MIXED handle with PINT_OPT_FX_RESIDUAL in exact
 * block fixed point with FP64-accurate products; written in FP64. */
int pint_residual(pint_handle* h, const double* u0_dev, const double* U_dev,
                  double* r_dev, double* rel_res);

/* One application of the diagonalized preconditioner (Eq. 2.8; Eq. 4.14 for
 * Cahn-Hilliard with averaged Jacobian jbar): delta = P_alpha^{-1} r, in the
 * handle's precision.  r_dev, delta_dev: nt*nx*ny doubles (may not alias). */
int pint_precond_apply(pint_handle* h, double jbar, const double* r_dev, double* delta_dev);

/* Per-phase accounting of the kernels a handle launches.  Phases:
 *  0 residual (+ alpha-scaling)      1 convergence check (reduction, status)
 *  2 time FFT (Step 1)               3,4,5 spatial solve stages (Step 2; 1-D uses 3 only)
 *  6 inverse time FFT + unscale + update (Step 3; on 1-D time axes beyond 1024
 *    steps it also carries Step 2's row solves, and phases 3-5 stay empty)
 *  7 window set-up
 * launches[] is always counted; ms[] (device time between CUDA events
 * recorded on the handle's stream around each phase) only while enabled. */
#define PINT_NPHASE 8
typedef struct {
    double    ms[PINT_NPHASE];
    long long launches[PINT_NPHASE];
} pint_profile;

/* Event timing of the phases: on = 1 records events around every phase; on = 2
 * (coarse) records only two spans per iteration, so that no event splits the
 * kernels of one step: the residual with its convergence check, booked to
 * phase 0, and the whole diagonalized step (Steps 1-3), booked to phase 2;
 * phases 1 and 3-6 then read 0 ms.  on = 0 disables.  Timed solves run the
 * host-launched loop (no graph).  Errors: PINT_EINVAL, PINT_ECUDA. */
int pint_profile_enable(pint_handle* h, int on);

/* Copy the accumulated profile into *out; reset = 1 zeroes it afterwards. */
int pint_profile_read(pint_handle* h, pint_profile* out, int reset);

/* Execution options.
 *  PINT_OPT_GRAPHS (default 1): run each window's iteration loop as one CUDA
 *    graph with a device-controlled while-node (no host round trip per
 *    iteration; the graph is built on the first solve and cached).  0 = launch
 *    kernels from the host in chunks of iterations.  While phase timing is
 *    enabled (pint_profile_enable) the host-launched path is used.
 * Errors: PINT_EINVAL for an unknown option or value. */
#define PINT_OPT_GRAPHS 1
/*  PINT_OPT_ADAPTIVE_WINDOWS (default 0): split each window of nt steps into
 *    power-of-two segments (>= 16 steps) chosen before each segment so that
 *    alpha * max_p R_p^L <= 0.1, where R_p = 1/(1 + dt mu_p) and mu_p is the
 *    spectrum of the spatial operator linearized about the segment's initial
 *    data (for Cahn-Hilliard: eps^2 Lam^2 + (1 - mean 3u0^2) Lam).  Growing modes
 *    (spinodal decomposition) make alpha R^L approach 1, where the iteration's
 *    per-mode factor |alpha R^L/(1 - alpha R^L)| (Eq. 2.18) exceeds one; shorter
 *    segments keep it small.  A segment that still diverges or stalls is solved
 *    again from its initial data with half the length (down to 16 steps).
 *    Enabling it builds the tables of the shorter lengths (allocates device
 *    memory); it runs the host-launched loop. */
#define PINT_OPT_ADAPTIVE_WINDOWS 2
/*  PINT_OPT_FUSED_SPATIAL: on square 2-D grids of 64 or 128 cells per side with
 *    Neumann conditions, solve each frequency slice in one kernel (a thread-block
 *    cluster holds the slice in shared memory) instead of three passes over the
 *    spectrum.  Not set: chosen by the autotuner (pint_tune_lookup); 0 or 1: fixed. */
#define PINT_OPT_FUSED_SPATIAL 3
/*  PINT_OPT_KRYLOV (default 0 = off): for the linear equations, wrap the
 *    preconditioner in restarted flexible GMRES(value), 1 <= value <= 30:
 *    right-preconditioned by P_alpha^{-1}, minimizing ||b - K U||_2, with K
 *    applied in FP64 and the basis in FP64 ((2 value + 1) vectors of nt*nx*ny
 *    doubles, allocated here).  The iterate is FP64 in every precision (a
 *    PINT_MIXED_FF handle then runs as PINT_MIXED).  pint_stats.iters counts
 *    preconditioner applications.  Errors: PINT_EINVAL (value out of range, or
 *    Cahn-Hilliard), PINT_ENOMEM. */
#define PINT_OPT_KRYLOV 4
/*  PINT_OPT_VARYING_JACOBIAN (default 0 = off): for Cahn-Hilliard (PinT-I and
 *    PinT-II), Step 2 uses the space-varying averaged Jacobian of Eq. 4.12,
 *    J~(x) = mean over the time levels of 3 u(x)^2, instead of its scalar mean:
 *    one cycle of flexible GMRES(value), 1 <= value <= 30, per outer iteration,
 *    over all frequencies at once, right-preconditioned by the scalar-J divide
 *    and stopped at a relative inner residual of 1e-4.  Work memory: (2 value + 2)
 *    half spectra.  The cycle runs on the device with no host round trip (its
 *    Hessenberg matrix, rotations and stop test in one-CTA kernels), so the
 *    iteration loop is captured in a CUDA graph like the scalar-Jacobian one.
 *    Errors: PINT_EINVAL (value out of range, or a linear equation), PINT_ENOMEM. */
#define PINT_OPT_VARYING_JACOBIAN 5
/*  PINT_OPT_FX_RESIDUAL: on a PINT_MIXED handle of a linear equation with square cells
 *    (or in 1-D), evaluate the residual (and pint_residual) in block fixed point on the
 *    integer pipes; 0 = the FP64 residual kernel.  Default 1 where supported and not stiff
 *    (2^-24 dt max|spectrum| <= 1): for stiffer problems the fixed-point residual reports the
 *    true residual of the FP64-rounded iterate, whose floor can exceed the tolerances, so the
 *    FP64 kernel is the default there.  Errors: PINT_EINVAL for value 1 where unsupported. */
#define PINT_OPT_FX_RESIDUAL 6
/*  PINT_OPT_LOG_INVARIANTS (default 0): after each window (or segment) of a solve,
 *    record for every time level its mass h^d sum_i u_i and its discrete energy
 *    E_h(u) = h^d sum_i (u_i^2 - 1)^2 / 4 + (eps^2/2) h^(d-2) sum over the grid's interior faces
 *    of (u_j - u_i)^2 (the Cahn-Hilliard functional of Sec. 1, Eq. 1.5; both are conserved /
 *    non-increasing along the backward-Euler solution, Sec. 5.3-5.4), reduced on the device in a
 *    fixed order.  Read them with pint_invariants.  Enabling allocates n_windows * nt pairs.
 *    Errors: PINT_EINVAL, PINT_ENOMEM. */
#define PINT_OPT_LOG_INVARIANTS 7
/*  PINT_OPT_TIME_GEMM (default -1): for N_t = 64 or 128 with FP32 transforms and a point count
 *    divisible by 4, Steps 1 and 3 can run as dense DFT matrix products on the tensor cores
 *    (split-FP16 operands, FP32 accumulation, about 2^-22 of each point's largest value) instead
 *    of FFTs.  -1: chosen by measurement on the first pint_solve (each direction timed both
 *    ways on this handle's sizes); 0: FFT; 1: matrix products (Step 3 only for PINT_MIXED, whose
 *    FP64 update it carries).  pint_stats.time_gemm reports the choice.
 *    Errors: PINT_EINVAL (value out of range, or 1 where unsupported). */
#define PINT_OPT_TIME_GEMM 8
int pint_set_option(pint_handle* h, int option, long long value);

/* The project autotuner.  Before a handle's first pint_solve, every Steps 1-3
 * kernel choice that the caller has left open (PINT_OPT_TIME_GEMM = -1, and
 * PINT_OPT_FUSED_SPATIAL not set) is measured on the handle's own buffers (CUDA
 * events; each candidate two warm-up and five timed launches) and the fastest
 * kept.  The choices of a shape go into a process-wide table keyed by
 * (equation, dim, nx, ny, nt, precision as run, bc, theta < 1); a later handle of
 * the same shape takes them from the table without measuring
 * (pint_stats.tune_cached).  If the environment variable PINT_TUNE_FILE names a
 * file, the table is loaded from it at the first lookup and every new entry is
 * appended to it.  The table is mutex-protected. */
typedef struct {
    int   time_fwd_gemm;    /* 1: Step 1 as tensor-core DFT products, 0: FFT */
    int   time_inv_gemm;    /* 1: Step 3 as tensor-core DFT products, 0: FFT */
    int   fused_spatial;    /* 1: Step 2 as one fused 2-D kernel, 0: three passes */
    float ms;               /* measured time of the chosen kernels for one application */
} pint_tune_entry;
/* 1 and *out filled if the table holds p's shape (p as passed to pint_create; its
 * precision is mapped to the one the solve runs in), 0 if not, PINT_EINVAL for an
 * invalid problem. */
int pint_tune_lookup(const pint_problem* p, pint_tune_entry* out);
/* Merge the entries of a table file (format: lines "pint-tune equation dim nx ny
 * nt precision bc half fwd inv fused ms", '#' comments).  Returns the entries
 * read, PINT_EINVAL for a missing file or a malformed line (entries before it
 * are kept). */
int pint_tune_load(const char* path);
/* Write the whole table; returns the entries written or PINT_EINVAL. */
int pint_tune_save(const char* path);
/* Empty the table (a file named by PINT_TUNE_FILE is not read again). */
void pint_tune_clear(void);

/* Copy the invariants recorded by the last pint_solve (PINT_OPT_LOG_INVARIANTS) into
 * mass_host[i], energy_host[i], i = 0 .. min(cap, levels) - 1, for time levels 1, 2, ... of
 * the whole solve (all windows).  Returns the number of levels recorded (>= 0), or PINT_EINVAL
 * (logging not enabled, bad arguments) / PINT_ECUDA.  Synchronizes the handle's stream. */
int pint_invariants(pint_handle* h, double* mass_host, double* energy_host, long long cap);

/* pint_residual_static: the residual of pint_residual for callers that cannot
 * allocate device memory when they need it (a process whose device memory is
 * already reserved by another allocator, a latency path that must not block in
 * cudaMalloc, a program that sizes its memory once at start-up).  No handle,
 * no allocation of any kind: the reduction scratch is a file-scope device array
 * of PINT_STATIC_SCRATCH_BYTES that each GPU which loads the library holds until
 * the process exits.  The paper has no counterpart; this is a deployment aid.
 *  p:           problem (validated as in pint_create)
 *  cuda_stream: cudaStream_t the kernels run on (NULL = legacy default stream)
 *  u0_dev, U_dev: as in pint_residual; r_dev (nt*nx*ny doubles) may be NULL
 *  rel_res_dev: device pointer to one double that receives ||r||_2 / ||b||_2
 * Asynchronous: returns after enqueueing; read rel_res_dev after the stream.
 * The first call on a device looks up the scratch array's device address (with
 * that device current) and caches it; make that first call outside any stream
 * capture.  All calls share the one array: calls whose kernels overlap on a GPU
 * (concurrent streams, threads) race and must be serialized by the caller.
 * Errors: PINT_EINVAL (bad problem or NULL pointer, or a grid whose reduction
 * needs more partial sums than the scratch holds), PINT_ECUDA. */
#define PINT_STATIC_SCRATCH_BYTES 278528
int pint_residual_static(const pint_problem* p, void* cuda_stream, const double* u0_dev, const double* U_dev,
                         double* r_dev, double* rel_res_dev);

/* Free everything the handle owns (NULL is allowed). */
void pint_destroy(pint_handle* h);

/* Static description of a return code. */
const char* pint_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* PINT_H */
