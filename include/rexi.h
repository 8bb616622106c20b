/*
 * rexi.h -- C ABI of the GB300 REXI engine.
 *
 * The engine advances the semi-discrete Schroedinger equation (Eq. (1) of
 * Rittich & Speck, "Time-parallel simulation of the Schroedinger equation",
 * arXiv:1912.03312) by rational approximation of the exponential (Sec. 3.1):
 *
 *     psi(t + tau) ~= alpha_0 psi + sum_{k=1}^{K} alpha_k (tau H - z_k I)^{-1} psi,     (Eq. (5))
 *
 * with H = -(hbar^2/2m) Lap_h + diag(V) on a periodic, second-order
 * finite-difference grid (the B = I discretisation of Sec. 5, scaled by hbar),
 * poles/weights from the Faber-Caratheodory-Fejer construction (Sec. 3.2,
 * Algorithms 1 and 2, conformal map Eq. (9)), and the accuracy condition
 * Eq. (10) met by substeps.  Each pole's system is an independent GMRES solve;
 * all K solves (and, in the batched call, all problems) run in one persistent
 * CUDA launch.
 *
 * Conventions for every call:
 *   - Status: 0 = REXI_OK, negative = error, positive = warning.  No call
 *     aborts or throws.  rexi_status_string() names each code.
 *   - Complex vectors are interleaved (re, im) IEEE doubles ("c128"), the
 *     storage of a torch.complex128 tensor.  Grids are stored x fastest:
 *     index = ix + nx * (iy + ny * iz).
 *   - "device" pointers are CUDA global-memory pointers on the plan's device;
 *     "host" pointers are ordinary CPU memory.  The caller owns every buffer
 *     it passes; the plan owns its own workspace.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   - Calls on one plan must not overlap in time (the workspace is shared).
 */
#ifndef REXI_H
#define REXI_H

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define REXI_OK          0
#define REXI_EINVAL     -1   /* bad argument (size, pointer, NaN/Inf in V, ...) */
#define REXI_ENOMEM     -2   /* device or host allocation failed                 */
#define REXI_ECUDA      -3   /* a CUDA runtime call failed (no device, launch...) */
#define REXI_ENOCONV    -4   /* a pole's GMRES hit max_iters above tolerance     */
#define REXI_ETIMEOUT   -5   /* a bounded device-side wait gave up               */
#define REXI_EPLAN      -6   /* FCF construction failed (root count, spurious pole,
                                non-unique CF approximant)                        */
#define REXI_EBOUNDS    -7   /* an index check of a debug build failed; the access
                                was skipped (rexi_plan_debug_record has the site)  */
#define REXI_WACCURACY   1   /* Eq. (10) violated: tau*W/hbar > R1 (only with
                                allow_substeps = 0, or a potential outside the
                                plan's spectral enclosure)                         */

/* ---- precision forms ----------------------------------------------------- */
#define REXI_FP64   0   /* Krylov basis, matvecs and orthogonalisation in c128   */
#define REXI_MIXED  1   /* Krylov basis/matvecs/orthogonalisation in c64; FP64 for
                           the residual at every restart (iterative refinement),
                           the Hessenberg least squares and the pole sum          */
#define REXI_DF64   2   /* ortho = 2 (Lanczos) only: the recurrence -- stencil,
                           three-term update, inner products and the stored basis
                           -- in double-float (pairs of floats, about 2^-47 per
                           operation) on the FP32 pipe, from the second Krylov
                           vector on; FP64 for the first sweep (any scale of psi),
                           the tridiagonal matrix, every pole's least squares, the
                           combined coefficients and the input state's term of
                           the pole sum.  The recurrence's rounding enters psi'
                           through the combined coefficients sum_k alpha_k y_k,
                           not the individual weights, so its effect stays near
                           1e-13 (the per-pole tolerance and the pole-sum
                           amplification set the step error as in REXI_FP64)     */

#define REXI_MAX_POLES   256
#define REXI_MAX_RESTART 64   /* windowed bases; with full orthogonalisation 31 (delayed
                                 CGS2) or 32 (CGS2) */
#define REXI_MAX_RESTART_FULL 31
#define REXI_MAX_KRYLOV  512  /* ortho = 2 (Lanczos): largest Krylov dimension per substep */

/* Periodic grid: N_d points on [lo_d, hi_d), h_d = (hi_d - lo_d) / N_d,
 * points x_j = lo_d + j h_d.  ndim in {1, 2, 3}; unused n[] entries ignored. */
typedef struct {
    int    ndim;
    int    n[3];
    double lo[3], hi[3];
    double hbar, mass;
} rexi_grid;

typedef struct {
    int    precision;      /* REXI_FP64, REXI_MIXED (default) or REXI_DF64 (ortho = 2 only) */
    int    restart_m;      /* GMRES restart length (default 30): 1..REXI_MAX_RESTART with a
                              window, else 1..REXI_MAX_RESTART_FULL (32 with CGS2); with
                              ortho = 2 the largest Krylov dimension, 1..REXI_MAX_KRYLOV    */
    int    max_iters;      /* Arnoldi iterations per pole solve before ENOCONV (default 2000) */
    double tol;            /* per-pole stop: ||b - A x|| <= tol ||b||; 0 = choose from the
                              pole-sum amplification (see rexi_plan_info.tol)              */
    double inner_tol;      /* REXI_MIXED: relative residual reduction at which an FP32
                              cycle ends and an FP64 residual is formed (default 1e-5)     */
    double R1;             /* half-length of the approximation interval i[-R1, R1] of
                              Eq. (9); 0 = the largest R1 with 2 sigma_{K+1} <= eps_target */
    double eps_target;     /* approximation error target for the default R1 (default 1e-9,
                              the level of Table 1)                                         */
    int    allow_substeps; /* 1 (default): n_sub = ceil(dt W / (hbar R1)) substeps so that
                              Eq. (10) holds; 0: a single rational step, REXI_WACCURACY if
                              Eq. (10) fails                                                 */
    double stabilize_eps;  /* Sec. 3.4: scale every beta_j by (1 - eps); 0 = off (default,
                              as in the paper)                                              */
    int    want_backward;  /* allocate the adjoint workspace at create time (default 0:
                              allocated by the first rexi_step_backward call)               */
    int    device;         /* CUDA device ordinal; -1 = current device (default)          */
    int    shared_first_cycle; /* 1 (default): the first GMRES cycle of every substep runs on
                              one Krylov basis shared by all K poles (the shifted-systems
                              observation of Sec. 5: K(tau H - z_k I, b) is the same space for
                              every k), each pole with its own Hessenberg, rotations and stop;
                              later cycles are per pole.  0: K independent bases throughout  */
    int    ortho;          /* Arnoldi orthogonalisation: 1 (default) delayed classical Gram-
                              Schmidt with reorthogonalisation, one global reduction per step
                              (the previous vector is reorthogonalised and normalised together
                              with the projection of the new one); 0: CGS2, two reductions
                              per step; 2: Lanczos -- REXI_FP64 or REXI_DF64, window 0: every
                              substep builds ONE basis for all K poles (the shifted-systems observation
                              of Sec. 5) by the three-term recurrence of the real symmetric
                              tau (H - c) with real coefficients, one global reduction and one
                              grid barrier per step, no restarts: restart_m (up to
                              REXI_MAX_KRYLOV) is then the largest Krylov dimension, and a pole
                              that has not met its bound by then fails with REXI_ENOCONV.  Each
                              pole solves its least-squares problem on the shared basis (GMRES
                              with the columns orthonormal only locally, so the stop uses the
                              bound |g_{k+1}| L_k >= ||r_k||, L_k = c_k + |s_k| L_{k-1} <= sqrt(k+1)
                              from the rotations) and the pole sum is one
                              pass over the basis.  rexi_step and rexi_solve_poles run on this
                              path; rexi_step_backward runs on the item engine (shared first
                              cycle, window 2, restart min(restart_m, 64)), allocated at its
                              first call; rexi_step_batched runs a batch of such plans as one
                              launch of the Lanczos kernel                                    */
    int    window;         /* with ortho = 1: 0 (default) orthogonalise every new vector against
                              the whole basis; L >= 2: only against the last L vectors (a
                              truncated, quasi-GMRES basis).  H is real symmetric, so tau H - z
                              is a shifted Hermitian operator whose Hessenberg matrix is
                              tridiagonal in exact arithmetic and L >= 2 loses nothing there;
                              in floating point the columns are orthonormal only locally and
                              every residual estimate is taken as sqrt(k+1) |g_{k+1}|, an
                              upper bound of the true residual for unit columns.  Cost per
                              Arnoldi step: O(L) basis vectors instead of O(k).            */
} rexi_options;

/* What a plan computed (host copy, filled by rexi_plan_info). */
typedef struct {
    int    K, n_sub, n_total, restart_m, precision;
    double dt, tau;        /* user step and substep tau = dt / n_sub                       */
    double R1;             /* approximation interval half-length                           */
    double sigma_K1;       /* sigma_{K+1} of Theorem 1 (CF error; the FCF error is <= ~2x)  */
    double E_min, E_max;   /* spectral enclosure of H                                      */
    double c, W;           /* centre and half-width of the enclosure                       */
    double amplification;  /* A = max_{w in i[-R1,R1]} sum |beta_j| / |w - sigma_j|         */
    double tol;            /* per-pole relative residual target in use                     */
    double min_re_sigma;   /* distance of the nearest pole from the approximation interval */
} rexi_plan_info;

/* Per-call statistics (host).  iters/resid are per pole, summed over substeps
 * (iters) and the maximum over substeps (resid, true relative residual). */
typedef struct {
    int    status;                    /* same as the call's return value                */
    int    n_sub;
    int    max_iters_seen;            /* largest per-pole Arnoldi count in one substep   */
    int    total_iters;               /* sum over poles and substeps                     */
    int    total_cycles;              /* restart cycles (FP64 residual evaluations)      */
    int    iters[REXI_MAX_POLES];
    int    cycles[REXI_MAX_POLES];
    int    iters_sq[REXI_MAX_POLES];  /* sum over restart cycles of (cycle length)^2       */
    double resid[REXI_MAX_POLES];
    double bytes;                     /* algorithmic bytes of the launch: every vector a pass
                                         reads or writes (basis, state, x, potential),
                                         counted once per pass by the kernel as it works;
                                         batched: the whole launch, in every entry        */
    double flops64;                   /* FP64 flops of the launch's arithmetic (an FMA is 2),
                                         counted the same way                              */
    double ops32;                     /* FP32-pipe arithmetic instructions per lane of the
                                         Lanczos kernel (compensated sums, double-float
                                         recurrence and final pass), counted the same way;
                                         0 on the item engine                             */
} rexi_stats;

typedef struct rexi_plan rexi_plan;   /* opaque, owned by the library */

/* Fill *opt with the defaults documented above. */
int rexi_options_default(rexi_options* opt);

/* Build a plan for one problem (Sec. 3.1-3.3).
 *   g   : host, the grid.
 *   V   : host, n = prod(n[d]) doubles, the potential, x fastest.  Copied.
 *   dt  : user time step (> 0).
 *   K   : number of poles, 1..REXI_MAX_POLES.
 *   opt : host, NULL = defaults.
 * Computes the spectral enclosure [E_min, E_max] of H (min V; max V plus the
 * exact bound (hbar^2/2m) sum_d 4/h_d^2 of the periodic Laplacian), centres the
 * exponential at c, picks R1 and n_sub (Eq. (10)), builds the FCF poles and
 * weights in double-double arithmetic (Algorithms 1-2), maps them to
 * z_k = tau c + i hbar sigma_k, alpha_k = i hbar beta_k e^{-i tau c / hbar},
 * alpha_0 = 0, and allocates all device workspace (no call below allocates,
 * except the first rexi_step_backward when want_backward = 0).
 * Returns REXI_OK, REXI_WACCURACY (plan usable), or an error (then *out = NULL). */
int rexi_plan_create(rexi_plan** out, const rexi_grid* g, const double* V,
                     double dt, int K, const rexi_options* opt);

void rexi_plan_destroy(rexi_plan* plan);

/* Host copy of the plan's parameters. */
int rexi_plan_get_info(const rexi_plan* plan, rexi_plan_info* info);

/* Per-substep poles and weights of Eq. (5): z[2K], alpha[2K] interleaved
 * (re, im), alpha0[2], n_sub.  Any output pointer may be NULL. */
int rexi_plan_poles(const rexi_plan* plan, double* z, double* alpha, double* alpha0, int* n_sub);

/* FCF poles/weights of exp on i[-R1, R1] (Algorithm 2 output, before the
 * mapping to Eq. (5)): sigma[2K], beta[2K] interleaved.  Host only. */
int rexi_plan_fcf(const rexi_plan* plan, double* sigma, double* beta);

/* Standalone FCF construction (Algorithms 1-2 in double-double), host only:
 * sigma[2K], beta[2K] interleaved; sigma_K1 (Theorem 1), min_re_sigma and
 * amplification may be NULL.  R1 = 0 picks the default radius for eps_target
 * (eps_target <= 0 means 1e-9); *R1_used (may be NULL) receives it. */
int rexi_fcf(int K, double R1, double eps_target, double* sigma, double* beta,
             double* R1_used, double* sigma_K1, double* min_re_sigma, double* amplification);

/* Replace the potential (host or device pointer, n doubles), keeping the
 * plan's c, W, poles and n_sub (for a learnable V).  Returns REXI_WACCURACY if
 * the new potential's enclosure leaves [E_min, E_max] (Eq. (10) may fail). */
int rexi_plan_set_potential(rexi_plan* plan, const double* V, int V_on_device, void* stream);

/* One user step dt (n_sub rational evaluations of Eq. (5)) on the device.
 *   psi_in, psi_out : device c128[n]; psi_in == psi_out allowed.
 *   st              : host, may be NULL.
 * With st == NULL the call only enqueues work on stream and returns launch
 * errors; convergence failures are then reported by rexi_plan_last_status().
 * With st != NULL the call synchronises the stream and returns REXI_ENOCONV /
 * REXI_ETIMEOUT when a pole failed. */
int rexi_step(rexi_plan* plan, const void* psi_in, void* psi_out, void* stream, rexi_stats* st);

/* Same as rexi_step with host buffers (c128[n] each): copies in, steps,
 * copies out and synchronises. */
int rexi_step_host(rexi_plan* plan, const double* psi_in, double* psi_out, void* stream,
                   rexi_stats* st);

/* The Chebyshev propagator the paper compares REXI with (Sec. 4): psi_out =
 * p(Ht) psi_in with p(x) = sum_{k<=N} a_k T_k(x) approximating exp(-i R x) on
 * [-1, 1], Ht = (H - c)/W on the plan's spectral enclosure, R = dt W / hbar,
 * a_k = (2 - delta_k0)(-i)^k J_k(R) exp(-i dt c / hbar) (the Chebyshev
 * coefficients Sec. 4 computes by FFT; here in closed form, Jacobi-Anger),
 * evaluated by the Clenshaw recurrence in one persistent FP64 launch (one grid
 * barrier per degree).  N is the smallest degree >= R with
 * sum_{k>N} |a_k| <= tol (tol = 0: 1e-10), so |p - exp| <= tol on the
 * spectrum; returned in *degree (may be NULL).  One user step dt of the plan,
 * no substeps.  psi_in / psi_out: device c128 of the plan's size, may alias.
 * Uses the plan's two state buffers; asynchronous like rexi_step (status of the
 * bounded barriers via rexi_plan_last_status). */
int rexi_cheb_step(rexi_plan* plan, const void* psi_in, void* psi_out, double tol, void* stream,
                   int* degree);

/* B independent problems (each with its own plan, grid, K and n_sub) in one
 * persistent launch: all problems x all poles share the GPU (the K solves of
 * every problem are the independent tasks of Sec. 3.1).  All plans must be on
 * the same device, distinct, and either all item-engine plans with the same
 * precision, restart length and orthogonalisation, or all Lanczos plans
 * (ortho = 2; REXI_FP64 and REXI_DF64 plans may be mixed, each problem runs in
 * its own arithmetic); B <= 128.  For Lanczos plans the launch divides its CTAs among
 * the problems in proportion to points x substeps (a control CTA and at least one
 * tile CTA each, so B <= the CTAs of the launch / 2), chooses every problem's
 * tile boxes for its share, and each problem synchronises only its own CTAs;
 * every plan's own workspace is used.  The first call with a combination of
 * plans uploads its descriptors (synchronously, into memory owned by plans[0]);
 * later calls with the same plans only launch, so they may be captured in a
 * CUDA graph once the first call has run.
 * psi_in[b], psi_out[b] : device c128 of plan b's size.  st: B entries or NULL
 * (with st the call synchronises and returns the first failing status). */
int rexi_step_batched(rexi_plan* const* plans, int B, const void* const* psi_in,
                      void* const* psi_out, void* stream, rexi_stats* st);

/* Vector-Jacobian product of one user step psi_{n+1} = S(V) psi_n
 * (the step is linear in psi; S^H = sum conj(alpha_k) (tau H - conj(z_k) I)^{-1}
 * because H is real symmetric).
 *   psi_n    : device c128[n], the state the forward step started from.
 *   grad_out : device c128[n], G = 2 dL/dconj(psi_{n+1}) (torch.autograd's
 *              convention for a real loss L).
 *   grad_in  : device c128[n], receives 2 dL/dconj(psi_n) = S^H G.
 *   dLdV     : device double[n], ACCUMULATED: += dL/dV_i =
 *              -tau sum_substeps Re sum_k alpha_k conj(Y_{k,i}) X_{k,i},
 *              X_k = (tau H - z_k)^{-1} psi_s, Y_k = (tau H - conj(z_k))^{-1} G_s.
 *   grad_in may equal grad_out.  Intermediate substep states are recomputed. */
int rexi_step_backward(rexi_plan* plan, const void* psi_n, const void* grad_out, void* grad_in,
                       double* dLdV, void* stream, rexi_stats* st);

/* --- single stages of the hot path, for parity checks and profiling ------- */

/* K1: w_k = (tau H - z_k I) v_k for every pole k, complex FP64.
 * v, w : device c128[K][n] (pole-major).  One substep's tau. */
int rexi_apply_poles(rexi_plan* plan, const void* v, void* w, void* stream);

/* K1-K5: x_k = (tau H - z_k I)^{-1} b for every pole, by the plan's GMRES form
 * (precision, restart, tolerance).  b: device c128[n]; x: device c128[K][n]. */
int rexi_solve_poles(rexi_plan* plan, const void* b, void* x, void* stream, rexi_stats* st);

/* K4b: out = alpha_0 psi + sum_k alpha_k x_k in FP64.  psi, out: device
 * c128[n]; x: device c128[K][n]. */
int rexi_pole_sum(rexi_plan* plan, const void* psi, const void* x, void* out, void* stream);

/* --- allocation-free entry point -------------------------------------------
 * The paper has no counterpart to this call; it exists for callers that cannot
 * allocate device memory: code running inside a custom allocator or memory-pool
 * callback, hosts that reserve all GPU memory for themselves up front, and
 * sandboxes in which cudaMalloc is unavailable.  rexi_plan_create allocates, so
 * these callers use this call instead: one rational evaluation
 *     psi_out = alpha0 psi_in + sum_k alpha_k (tau H - z_k I)^{-1} psi_in,
 * with every byte of engine workspace taken from a fixed 32 MiB array compiled
 * into the library (REXI_STATIC_SCRATCH_BYTES; every GPU that loads the library
 * holds it until the process exits).  Nothing is allocated: no cudaMalloc,
 * cudaFree or allocating library routine.
 *   g            : host, the grid (as rexi_plan_create).
 *   V            : device, n doubles, the potential.
 *   tau, c       : substep length and centre of the spectral enclosure
 *                  (rexi_plan_info.tau and .c of an equivalent plan).
 *   K, z, alpha  : host, K poles z[2K] and weights alpha[2K] (interleaved re, im),
 *                  alpha0[2]; e.g. from rexi_plan_poles.
 *   opt          : host, required (NULL is REXI_EINVAL): precision, restart_m,
 *                  max_iters, tol (finite, > 0: there is no amplification-based
 *                  default here), inner_tol (finite, >= 0), ortho and window
 *                  (the orthogonalisation, validated as in rexi_plan_create)
 *                  are used; every solve has its own basis (no shared cycle).
 *   psi_in, psi_out : device c128[n]; may be the same buffer.
 *   st           : host, may be NULL.  With st the call synchronises and
 *                  returns REXI_ENOCONV / REXI_ETIMEOUT when a solve failed.
 *                  Without st the call only enqueues the work and returns
 *                  argument and launch errors: convergence failures and
 *                  timeouts of that call are then not reported anywhere, so a
 *                  caller that needs them passes st.
 * Returns REXI_EINVAL for a grid of more than 2^30 points, and when the
 * workspace (about K (m+1) n 8 bytes for REXI_MIXED, twice that for REXI_FP64,
 * plus K n 16 bytes) exceeds the static array.
 * The first call on a device looks the array's address up (cudaGetSymbolAddress,
 * done once per device with that device current); make that first call before
 * any stream capture.  All calls share the one array and it keeps the previous
 * call's contents (the call resets what must start at zero), so calls that
 * overlap on the GPU -- on different streams or threads -- race and must not be
 * issued concurrently. */
#define REXI_STATIC_SCRATCH_BYTES (32u << 20)
int rexi_substep_static(const rexi_grid* g, const double* V, double tau, double c, int K,
                        const double* z, const double* alpha, const double* alpha0,
                        const rexi_options* opt, const void* psi_in, void* psi_out, void* stream,
                        rexi_stats* st);

/* Status of the last call on the plan (synchronises the plan's last stream). */
int rexi_plan_last_status(rexi_plan* plan);

/* Index checks.  A library built with REXI_DEBUG defined (librexi_debug.so)
 * checks every indexed access of the Lanczos kernel (ortho = 2) against the
 * extent of the buffer it addresses: shared-memory staging, the halo ring
 * list, the basis, B u, the partial sums, the rows of R, y_k and the
 * coefficients, the states; and, at the start of a launch, that the tile
 * layout fits the dynamic shared memory and the grid fits the partial-sum
 * slots.  A failed check records the first failure, skips the access (nothing
 * outside a buffer is touched), and the launch ends at its next grid barrier
 * with REXI_EBOUNDS.
 * rexi_debug_checks: 1 in such a build, 0 otherwise.
 * rexi_plan_debug_record: rec[0..3] = site (LZ_SITE_* of csrc/lanczos.h; 0 =
 *   no failure), index, extent of the first failed check of the plan's last
 *   Lanczos launch, and the number of failed checks; synchronises the plan's
 *   last stream.  REXI_EINVAL for a plan of a build without checks, or a plan
 *   that is not a Lanczos plan.
 * rexi_plan_debug_trip: make every check of `site` (1 .. 11) fail in the
 *   plan's later launches, 0 = none: the accesses of that site are skipped and
 *   the launch reports REXI_EBOUNDS, which tests the reporting path without an
 *   out-of-range index.  REXI_EINVAL as for rexi_plan_debug_record, or for a
 *   site out of range. */
int rexi_debug_checks(void);
int rexi_plan_debug_record(rexi_plan* plan, long long rec[4]);
int rexi_plan_debug_trip(rexi_plan* plan, int site);

/* Limit of every device-side wait of the plan's launches (grid barriers,
 * bulk-copy completions): seconds > 0, at most 3600; seconds <= 0 restores the
 * default of 4 s.  A wait that runs out sets the launch's error word, every CTA
 * leaves the kernel at its next barrier, and the call (or
 * rexi_plan_last_status) returns REXI_ETIMEOUT; the context stays usable.
 * REXI_EINVAL for a NULL plan, NaN or more than an hour. */
int rexi_plan_set_timeout(rexi_plan* plan, double seconds);

/* Work decomposition of the plan's launches (the autotuner's knobs):
 * pole_tile / group_tile = points per task of pole items / shared-cycle group
 * items, each a multiple of 256 up to 2048; ctas_per_sm caps the resident CTAs
 * per SM of the persistent grid (0 = as many as fit; 1 on an FP64 plan selects
 * the kernel compiled for one CTA per SM, with twice the registers per thread
 * and wider update sweeps).  On a Lanczos plan (ortho = 2) group_tile bounds
 * the interior points of the kernel's box-shaped tiles (the box is chosen to
 * balance the CTAs' work) and ctas_per_sm (0 = 2, at most 8) sets the resident
 * CTAs per SM; pole_tile is not used.  Synchronises the device
 * and rewrites the plan's descriptors; results do not depend on these values
 * beyond floating-point summation order. */
int rexi_plan_set_tiles(rexi_plan* plan, int pole_tile, int group_tile, int ctas_per_sm);

/* Phase tracing.  rexi_plan_set_trace allocates room for `capacity` records
 * (0 disables); afterwards every engine launch of the plan records, at each
 * grid-wide barrier, the phase that ended there and the GPU global timer (ns).
 * Phase codes: 0 substep start, 1 FP64 residual, 2 cycle decision, 3 matvec +
 * first dot sweep, 4 second CGS sweep, 5 CGS update, 6 Givens, 7 x update,
 * 8 pole sum / adjoint accumulation, 9 delayed-CGS2 matvec + dots, 10 delayed-CGS2
 * normalisation + projection + Givens, 99 launch start.
 * rexi_plan_read_trace synchronises the plan's last stream, copies up to cap
 * (phase, ns) pairs of the last launch into out[2*cap] and returns how many
 * were recorded (which may exceed cap), or a negative status. */
int rexi_plan_set_trace(rexi_plan* plan, int capacity);
int rexi_plan_read_trace(rexi_plan* plan, long long* out, int cap);

/* Per-CTA barrier arrivals, for load-balance diagnosis.  After
 * rexi_plan_set_cta_trace(plan, phases) (0 disables) every engine launch of the
 * plan records, for each of its first `phases` grid-wide barriers, the global
 * timer (ns) at which each CTA's threads had all arrived.
 * rexi_plan_read_cta_trace synchronises the plan's last stream, sets *grid to
 * the CTA count of the last launch and copies whole barriers, row by row
 * (row r = barrier r, grid entries), while they fit in out[cap]; it returns the
 * number of barriers recorded (which may exceed what was copied) or a negative
 * status.  Barrier r matches record r of rexi_plan_read_trace, whose time is
 * the barrier's release as seen by CTA 0. */
int rexi_plan_set_cta_trace(rexi_plan* plan, int phases);
int rexi_plan_read_cta_trace(rexi_plan* plan, long long* out, int cap, int* grid);

/* Kernel-counted algorithmic bytes and FP64 flops of the plan's last launch
 * (engine or Chebyshev; the same counts rexi_stats reports).  Synchronises the
 * plan's last stream. */
int rexi_plan_last_work(rexi_plan* plan, double* bytes, double* flops64);

/* Number of CUDA kernel launches issued by the last call on the plan. */
int rexi_plan_last_launches(const rexi_plan* plan);

const char* rexi_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* REXI_H */
