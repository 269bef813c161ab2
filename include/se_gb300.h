/*
 * se_gb300.h -- C ABI of the GB300 (sm_103a) Spectral Ewald k-space library.
 *
 * The library computes the Fourier-space part of the Ewald potential,
 * phi~^{DP,F} of Eq. (fourier_space_ewald), and its gradient, for N point
 * charges in a box [0, L_x) x [0, L_y) x [0, L_z) (Sec. 2: the box need not be
 * a cube) that is periodic in its first D directions (D = 3: x, y, z; D = 2:
 * x, y; D = 1: x; D = 0: none), by the unified
 * Spectral Ewald method of Shamshirgar, Bagge & Tornberg, Alg. 4:
 *   1. gridding (Eq. gridding) with a truncated Gaussian (Eq. gaussian) or a
 *      polynomial Kaiser-Bessel window (PKB, Sec. 4.1) of P^3 support,
 *   2. FFT; for D = 1, 2 the adaptive FFT of Alg. 1, for D = 0 a zero-padded
 *      (2 M~)^3 FFT,
 *   3. scaling by e^{-|k|^2/4xi^2} W^(k)^{-2} G^{DP}(k) (Eq. scale) with the
 *      truncated Green's functions of Eqs. (G_hat_3d)-(G_hat_0d) and, for
 *      D = 0, the precomputed G^{0P}_R of Alg. 3,
 *   4. inverse FFT / AIFT (Alg. 2),
 *   5. gathering (Eq. complete_integral) and, for forces, the window
 *      gradient gather of Eq. (force-method-1).
 *
 * Conventions that hold for every entry point:
 *  - Precision.  A plan is created for SE_F32 or SE_F64; every array passed
 *    to it holds float or double accordingly.  Positions x are row-major
 *    [N][3], charges q and potentials phi are [N], forces F are [N][3].
 *  - Memory.  Unless SE_HOST_IO is given, x, q and every output are DEVICE
 *    pointers owned by the caller.  The plan owns its grids, FFT plans, tables
 *    and particle workspace; the workspace grows on demand (cudaMalloc) or
 *    once up front through se_plan_reserve.
 *  - Streams.  Work is issued on the plan's stream (se_plan_set_stream;
 *    default: the legacy stream) and is asynchronous: a returned SE_OK means
 *    the work was validated and launched.  Errors detected on the device
 *    (coordinates outside the box in a free direction, non-finite input) are
 *    latched in the plan and reported by se_plan_check (which synchronises)
 *    or at the end of a call made with SE_SYNC_CHECK.
 *  - Errors.  Every function returns an se_status; se_status_str names it.
 *    Nothing aborts the process.  A failed call leaves the plan usable.
 *  - Threads.  A plan must not be used by two host threads at once.
 */
#ifndef SE_GB300_H
#define SE_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct se_plan_s *se_plan_t;

typedef enum { SE_WIN_GAUSSIAN = 0, SE_WIN_PKB = 1 } se_window;
typedef enum { SE_F32 = 0, SE_F64 = 1 } se_dtype;

typedef enum {
    SE_OK = 0,
    SE_EINVAL = 1,        /* an argument is out of range (message: se_last_error) */
    SE_ENONNEUTRAL = 2,   /* SE_CHECK_NEUTRAL: |sum q| > 1e-12 sum |q| */
    SE_EOUTOFBOX = 3,     /* a coordinate in a free direction is outside [0, L) */
    SE_ENOMEM = 4,        /* device allocation failed */
    SE_ECUDA = 5,         /* a CUDA runtime call failed */
    SE_ECUFFT = 6,        /* a cuFFT call failed */
    SE_ETIMEOUT = 7,      /* reserved for bounded device-side waits */
    SE_ENOTFINITE = 8,    /* a position or charge is NaN or infinite */
    SE_ECAPACITY = 9      /* the request exceeds a fixed capacity of the entry point */
} se_status;

/* Call flags (bitwise OR). */
#define SE_ADD_SELF      1u  /* add phi^self_m = -2 xi / sqrt(pi) q_m (Sec. 2) to phi */
#define SE_CHECK_NEUTRAL 2u  /* verify sum q = 0 first (synchronises the stream) */
#define SE_SYNC_CHECK    4u  /* synchronise at the end and report device-side input errors */
#define SE_HOST_IO       8u  /* x, q and the outputs are HOST pointers; the call copies
                                them to and from the device on the plan's stream and
                                returns after the results are in host memory (page-locked
                                x and q are read in place by the binning's first kernel,
                                which writes the device copies, so the transfer overlaps
                                the counting; without SE_CHECK_NEUTRAL).  With
                                page-locked buffers (and without SE_CHECK_NEUTRAL or
                                profiling) the call -- copies included -- is captured
                                into a CUDA graph the first time and replayed while the
                                same call (N, pointers, flags) repeats; keep such
                                buffers allocated while the plan may replay them */

/* Optional overrides of the paper's parameter rules (Sec. 6).  A field left at
 * its "unset" value (given in brackets) takes the paper's default. */
typedef struct {
    double lambda;   /* [<= 0] extension factor, M~ = 2 ceil((M + lambda P)/2); Table (lambda) */
    double s0;       /* [<= 0] zero-mode / free-space upsampling: 2 (D=2), 2.5 (D=1), 2.8 (D=0) */
    int    s_mt;     /* [<= 0] s M~ of the upsampled modes of the set I, Eq. (estimate-s) */
    int    n_l;      /* [< 0]  size of the set I, Eq. (estimate-nl) */
    int    nu;       /* [<= 0] PKB polynomial degree, min(P/2 + 2, 9) */
    double shape;    /* [<= 0] alpha = (pi/2) P 0.91 (Gaussian) or beta = 2.5 P (PKB) */
    double aft_eps;  /* [<= 0] relative tolerance in Eqs. (estimate-s), (estimate-nl):
                        1e-5 for SE_F32 plans, 1e-10 for SE_F64 plans */
    int    tile;     /* [<= 0] edge of the gridding tile in grid cells (4, 8 or 16) */
    int    spread_mode; /* [<= 0] gridding kernel: 1 shared-memory atomics, one CTA per tile;
                           2 the same split over a thread-block cluster of `split` CTAs whose
                           blocks are summed through distributed shared memory; 3 per-warp
                           private blocks without atomics (bit-reproducible) */
    int    gather_mode; /* [<= 0] gathering kernel: 1 tile block staged in shared memory,
                           `split` CTAs per tile; 2 direct reads of the grid; 3 (FP32, tiles of
                           edge 8, P = 8 or 10) the staged block with four particles per warp
                           over chunks of at most 256 particles; 4 (FP32, same conditions) the
                           staged block with one particle per warp over the same chunks, which
                           by default FP32 plans of that kind with 32 or more particles per tile
                           take (the others mode 2) */
    int    split;       /* [<= 0] CTAs per tile for spread_mode 2 / gather_mode 1 (1..8) */
    int    force_method; /* [<= 0 -> 1] how se_force differentiates (Sec. 7.2): 1 gathers with
                           the window's derivative, Eq. (force-method-1); 2 multiplies the
                           scaling by i k per direction and runs the inverse transform and a
                           gathering with W three more times (the plan then holds three more
                           spectra and grids).  se_potential and se_vjp are unaffected. */
    int    fft_mode;    /* [<= 0] D = 0 transform: the z-direction FFT, scaling and inverse
                           FFT fused into one kernel per column when 2 M~ is a power of two
                           from 16 to 1024 (cuFFT otherwise); 1 cuFFT for every stage;
                           2 (D = 1 plans; method 1) the free-direction transforms of every
                           class, their padding (Alg. 1, Alg. 2) and the scaling as three
                           line-transform launches (padded rows and columns that are zero or
                           cut are never transformed) between cuFFT's x transforms, when
                           every free-direction length is at most 1024; otherwise as 0 */
    int    fft_sizes;   /* [<= 0] free-direction transform lengths: the smallest the rules of
                           Sec. 3.3 and Sec. 6 allow; 1 each of M~_i, s0 M~_i and s M~_i rounded
                           up to the next even length whose prime factors are 2, 3, 5 and 7
                           (more extension and upsampling, never less; faster FFTs) */
} se_opts;

/* Derived parameters of a plan (read-only report). */
typedef struct {
    int D, M, P, nu, Mt, s0_mt, s_mt, n_l;
    int grid[3];          /* real grid n_x, n_y, n_z (M or M~ per axis) */
    int tile[3];          /* gridding tile edge per axis */
    int n_tiles;
    double h, L, Lt, R, delta_L, xi, shape;
    int64_t capacity;     /* particles the workspace holds now */
    int64_t device_bytes; /* device memory held by the plan */
    int column_fft;       /* 1: the D = 0 z-direction FFT, scaling and inverse FFT run fused
                             in one kernel; 2: the D = 1 free-direction transforms and scaling
                             run as line transforms (se_opts.fft_mode) */
    /* per axis (non-cubic boxes; the scalar fields above are the cube's values:
       M of x, M~ / s0 M~ / s M~ of the first free axis, n_l of x) */
    int M_v[3];           /* grid intervals L_i / h */
    int Mt_v[3];          /* extended grid M~_i on free axes (M_i on periodic ones) */
    int s0_mt_v[3];       /* zero-mode / free-space transform lengths of the free axes */
    int s_mt_v[3];        /* set-I transform lengths of the free axes */
    int n_I[3];           /* half-width of the set I in mode indices, periodic axes */
    double L_v[3];        /* box sides */
} se_plan_info_t;

/* Fill *o with the "unset" values. */
void se_opts_default(se_opts *o);

/* Create a plan.  box[3] = side lengths along x, y, z (Sec. 2: the box need
 * not be a cube); D = number of periodic directions (the first D axes);
 * xi = Ewald splitting parameter (Eq. gamma); M = grid intervals along x
 * (even): the grid spacing h = box[0] / M is used on every axis, and every
 * side must be an even multiple of h; P = window support in grid intervals
 * (even, 2 <= P <= 16, P <= M and <= the grid of every periodic side);
 * w, dt = window and precision; opts may be NULL.  Sec. 3.3, Alg. 4 step 0,
 * Sec. 6, with the per-axis rules of the non-cubic box (the extended free
 * sides, R = length of the extended free sides, s0 raised to 1 + R / L~_i
 * where larger, s and n_l per free axis, the set I a box in k).  For D = 0
 * the call also runs the precomputation of Alg. 3 on the current device
 * (FP64).  Errors: SE_EINVAL (arguments), SE_ENOMEM, SE_ECUDA, SE_ECUFFT. */
se_status se_plan_create(se_plan_t *out, const double box[3], int D, double xi, int M, int P,
                         se_window w, se_dtype dt, const se_opts *opts);

/* Release every resource of the plan (NULL is accepted). */
se_status se_plan_destroy(se_plan_t plan);

/* Issue all later work of the plan on this CUDA stream (a cudaStream_t). */
se_status se_plan_set_stream(se_plan_t plan, void *stream);

/* Grow the particle workspace to hold n_max particles now, so that later calls
 * with N <= n_max allocate nothing (required before capturing a CUDA graph). */
se_status se_plan_reserve(se_plan_t plan, int64_t n_max);

/* Report the derived parameters. */
se_status se_plan_get_info(se_plan_t plan, se_plan_info_t *info);

/* Synchronise the plan's stream and report (then clear) the device-side input
 * errors latched since the last check: SE_EOUTOFBOX or SE_ENOTFINITE. */
se_status se_plan_check(se_plan_t plan);

/* phi~^{DP,F}(x_m), m = 1..N: Alg. 4 steps 1-5 (Eq. fourier_space_ewald).
 * x [N][3], q [N] in, phi [N] out.  Periodic coordinates may take any value
 * (they are wrapped into [0, L)); free coordinates must lie in [0, L).
 * flags: SE_ADD_SELF, SE_CHECK_NEUTRAL, SE_SYNC_CHECK, SE_HOST_IO.
 * N = 0 is a no-op.  Errors: SE_EINVAL, SE_ENONNEUTRAL, SE_EOUTOFBOX,
 * SE_ENOTFINITE, SE_ENOMEM, SE_ECUDA, SE_ECUFFT. */
se_status se_potential(se_plan_t plan, int64_t N, const void *x, const void *q, void *phi,
                       unsigned flags);

/* Fourier-space forces F_m = -q_m grad phi~(x_m) (Sec. 7.2).  Method 1 (the
 * default, Eq. force-method-1): one inverse transform, gradient gather with the
 * exact derivative of the window.  Method 2 (se_opts.force_method = 2): the
 * scaled spectrum times i k_a for a = x, y, z, four inverse transforms, and a
 * gathering of the four grids with W; i k_a is zero at the Nyquist index of an
 * even-length transform.  F [N][3] out; phi [N] out if non-NULL;
 * energy (DEVICE pointer to one double, may be NULL) receives
 * E = 1/2 sum_m q_m phi_m accumulated in FP64 (with SE_ADD_SELF the self
 * term is part of phi and of E).  Flags and errors as se_potential. */
se_status se_force(se_plan_t plan, int64_t N, const void *x, const void *q, void *F, void *phi,
                   double *energy, unsigned flags);

/* Vector-Jacobian product of phi = A(x) q (the adjoint of se_potential):
 * given g = dL/dphi [N], returns g_q = dL/dq = A g [N] and
 * g_x = dL/dx [N][3] = g_m grad_m (A q)_m + q_m grad_m (A g)_m.  The operator
 * A = S^T G S is symmetric because the scaling is real and even in k, so
 * the adjoint re-runs the forward pipeline on g (reverse spread/gather
 * through the same grid).  Either output may be NULL.  Device pointers. */
se_status se_vjp(se_plan_t plan, int64_t N, const void *x, const void *q, const void *g_phi,
                 void *g_x, void *g_q);

/* Stage profiling (measurement aid).  While enabled, every se_potential /
 * se_force call records CUDA events between its stages on the plan's stream,
 * waits for the call to finish, and adds each stage's duration to per-plan
 * accumulators.  Stages (index into ms[]):
 *   0 binning (tile counts, scan, sorted records)   1 gridding (per-tile blocks)
 *   2 block merge into the FFT input                3 forward FFT / AFT
 *   4 scaling                                       5 inverse FFT / AIFT
 *   6 gathering (phi, forces)                       7 energy reduction
 * se_plan_get_profile copies SE_N_STAGES accumulated milliseconds into ms,
 * the number of profiled calls into *calls and the number of kernels the
 * library launched itself (cuFFT's kernels excluded) since the plan was
 * created into *launches; any pointer may be NULL.  Enabling resets the
 * accumulators. */
#define SE_N_STAGES 8
se_status se_plan_set_profiling(se_plan_t plan, int enable);
se_status se_plan_get_profile(se_plan_t plan, double *ms, int64_t *calls, int64_t *launches);

/* Potential of se_potential, computed without allocating device memory.
 * The paper has no counterpart: this entry point serves callers that must not
 * call cudaMalloc while they run (a fixed memory budget handed out at start-up,
 * a loop where cudaMalloc's implicit device synchronisation is unacceptable, a
 * framework whose allocator owns all device memory during a step).  Create the
 * plan and call se_plan_reserve(plan, n_max) at set-up; afterwards this call
 * allocates nothing.  The per-tile gridding blocks live in a fixed array of
 * SE_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads the
 * library holds until the process exits.
 *  - se_plan_reserve looks up that array's device address on the plan's device
 *    (the first lookup on a device is when the driver allocates the array).  A
 *    plan whose workspace grew through other calls, without se_plan_reserve,
 *    does that lookup in its first call here instead: make that first call
 *    before any CUDA stream capture.
 *  - All calls share the array and it keeps the last call's contents; calls
 *    whose work overlaps on the GPU (several streams or plans at once) race.
 *  - Arguments as se_potential (device pointers; SE_ADD_SELF, SE_CHECK_NEUTRAL,
 *    SE_SYNC_CHECK).  Errors: SE_ECAPACITY when N exceeds the reserved
 *    capacity or the plan's gridding blocks exceed the fixed array;
 *    SE_EINVAL for SE_HOST_IO (it needs staging memory) or bad arguments. */
#define SE_NOALLOC_SCRATCH_BYTES (32u << 20)
se_status se_potential_noalloc(se_plan_t plan, int64_t N, const void *x, const void *q, void *phi,
                               unsigned flags);

/* Real-space part of the Ewald sum, Eq. (real_space_ewald): phi^R_m = sum over
 * images p in P_D (the plan's periodicity) and sources n, excluding n = m at
 * p = 0, of q_n erfc(xi r)/r for r = |x_m - x_n + p| < rc, with the plan's xi,
 * box and precision; F^R_m = -q_m grad phi^R_m.  Together with se_force and
 * SE_ADD_SELF this gives the full potential of Eq. (potential_split).  Cell
 * list of edge >= rc (rc < L/2 in periodic directions).  phi [N] and F [N][3]
 * (device; either may be NULL) are overwritten, or added to with
 * SE_ACCUMULATE.  The workspace grows on demand.  Errors: SE_EINVAL, SE_ENOMEM,
 * SE_ECUDA; with SE_SYNC_CHECK also the latched input errors. */
#define SE_ACCUMULATE 16u
se_status se_real_space(se_plan_t plan, int64_t N, const void *x, const void *q, double rc, void *phi, void *F,
                        unsigned flags);

/* ---- Batched evaluation of many independent systems ------------------------
 * nsys systems, system i with N[i] particles in a cubic box of side L[i],
 * periodic in its first D[i] directions, splitting parameter xi[i].  Each
 * system's grid M_i (Eq. KP_kinf) and support P_i (the approximation-error
 * estimate of Sec. 5.2 with the error-pollution rule, Sec. 6) start from the
 * absolute tolerance eps_rel * B_i, B_i = sqrt(Q_i) f_c(xi_i L_i) / L_i
 * (Eq. fc-expression; Q = NULL takes Q_i = N_i / 3, the mean for charges
 * uniform in [-1, 1]), with P_i + 2 for the forces (Sec. 7.2) and M_i rounded
 * up to an FFT-friendly size; the AFT of D = 1, 2 systems gets eps_rel / 4.
 * With autotuning, the first call then measures, on its own inputs, the
 * relative rms errors of phi and F of (M, P) candidates around that rule
 * against an FP64 reference of each system and keeps, among the candidates
 * whose errors are both within eps_rel / 2 (se_batch_get_accuracy reports
 * them), the one of least work: N P^3 window updates (doubled for P > 10)
 * plus 64 per grid point.  The window is w for all systems.  Every call replays one CUDA graph (captured on
 * first use and whenever the pointers change) in one of three forms:
 *  - single pipeline (SE_BATCH_LINES; every system D = 3 or 2, force method 1):
 *    binning, gridding, block merge and gathering of all systems as one kernel
 *    launch per stage and class of systems with equal support P_i (Alg. 4
 *    steps 1 and 5), and the transforms and scaling of all systems (steps 2-4,
 *    with the adaptive transform of Alg. 1 / Alg. 2 for D = 2) in five
 *    launches, each a list of line transforms of every system; no cuFFT call;
 *  - multi-system (SE_BATCH_FUSED): the same stages, each system's transforms
 *    and scaling (cuFFT) in parallel graph branches;
 *  - per-system (SE_BATCH_BRANCHES): each system's whole pipeline in parallel
 *    graph branches.
 * Unless SE_BATCH_NO_AUTOTUNE is given, the first se_batch_force call times the
 * gridding tile (4, 8, 16) and kernel variants per system on the real inputs,
 * then the forms as captured graphs (the two multi-system ones with 1, 2, 4 or
 * 8 CTAs per gridding tile, also with tiles of edge 4 for systems of more than
 * 512 particles per tile), and keeps the fastest; without autotuning the
 * form is the multi-system one unless a form flag is given.
 * Arrays x [sum N][3], q [sum N], F [sum N][3], phi [sum N] (may be NULL) are
 * concatenated in system order (device pointers); energy [nsys] (device, may be
 * NULL) receives E_i = 1/2 sum q phi per system.  The first call synchronises
 * (autotuning); later calls are asynchronous on the batch stream. */
#define SE_BATCH_NO_AUTOTUNE 1u
#define SE_BATCH_BRANCHES    2u   /* use the per-system form only */
#define SE_BATCH_FUSED       4u   /* use the multi-system form only */
#define SE_BATCH_LINES       8u   /* use the single-pipeline form only */
typedef struct se_batch_s *se_batch_t;
se_status se_batch_create(se_batch_t *out, int nsys, const int64_t *N, const int *D, const double *L,
                          const double *xi, const double *Q, double eps_rel, se_window w, se_dtype dt,
                          unsigned flags);
se_status se_batch_destroy(se_batch_t batch);
se_status se_batch_set_stream(se_batch_t batch, void *stream);
se_status se_batch_force(se_batch_t batch, const void *x, const void *q, void *F, void *phi, double *energy);
/* The same result with one plain se_force call per system on the batch stream
 * (no graph): the per-system baseline the batched form is measured against. */
se_status se_batch_force_each(se_batch_t batch, const void *x, const void *q, void *F, void *phi,
                              double *energy);
/* Relative rms errors of system i's phi and F that the autotuner measured for
 * the chosen (M, P) against its FP64 reference on the first call's inputs
 * (host outputs, either may be NULL; -1 when the batch was not autotuned or
 * before the first call).  Batching has no counterpart in the paper.  Errors:
 * SE_EINVAL for a bad batch or index. */
se_status se_batch_get_accuracy(se_batch_t batch, int i, double *err_phi, double *err_F);
/* Derived parameters of system i. */
se_status se_batch_get_system(se_batch_t batch, int i, se_plan_info_t *info);
/* Form of the captured graph (1 per-system, 2 multi-system, 3 single
 * pipeline) and the number of library kernels one call launches (cuFFT's own
 * kernels excluded; the single pipeline launches none; valid after the first
 * se_batch_force).  Batching has no counterpart in the paper.  Either
 * pointer (host memory, written by the call) may be NULL.  Errors: SE_EINVAL
 * for a NULL batch. */
se_status se_batch_get_form(se_batch_t batch, int *form, int64_t *kernels_per_call);

/* Sec. 6: grid size M (= 2 k_inf, Eq. KP_kinf) and window support P (from the
 * approximation-error estimates of Sec. 5.2, rounded up to even, with the
 * error-pollution rule of Eq. error_pollution: M up 5 % and P + 4 when
 * P > f_W(M / (xi L))) for the relative rms tolerance eps_rel, i.e. the
 * absolute tolerance eps_rel B with B = sqrt(Q) f_c(xi L) / L
 * (Eq. fc-expression).  Q = sum q^2; Q <= 0 takes N / 3 (the mean for charges
 * uniform in [-1, 1]).  box[3] = the sides (host memory); the estimates are the
 * cube's, taken with L = box[0], whose M intervals set the spacing h of every
 * axis; M is then raised to the smallest even value (up to 4x) for which every
 * side is an even multiple of h, as se_plan_create requires.  D (0..3) is
 * checked; the rules of Sec. 6 for M and P are the same for every D (the AFT
 * sizes that depend on D are set by se_plan_create).  The result may exceed
 * the plan limits (P <= 16).  *M, *P: host outputs.  Errors: SE_EINVAL
 * (arguments, or no admissible M for the box). */
se_status se_params_from_tolerance(double eps_rel, double xi, int64_t N, double Q, const double box[3], int D,
                                   se_window w, int *M, int *P);

/* Measured throughput ceilings of the units the gridding and gathering kernels
 * run on, for roofline reports (a measurement aid; the paper has no
 * counterpart).  kind: 0 FP32 fused multiply-add, 1 FP64 fused multiply-add
 * (*ops_per_s in flop/s, 2 flop per FMA, 8 independent chains per thread);
 * 2 shared-memory 32-bit integer atomic adds, 3 shared-memory FP32 atomic
 * adds (*ops_per_s in updates/s; every lane of a warp on its own word and bank).
 * One kernel fills every SM of the current device with resident warps and runs
 * `iters` iterations of its loop (128 FMA or 16 atomic adds per thread each);
 * *ms (may be NULL) receives its CUDA-event duration.  Synchronises the
 * device; allocates 1 MiB for the duration of the call.  Errors: SE_EINVAL,
 * SE_ECUDA. */
se_status se_measure_peak(int kind, int64_t iters, double *ops_per_s, double *ms);

/* Testing aid for callers' error paths (the paper has no counterpart): arm a
 * host-side allocation failure.  From this call on, the k-th device allocation
 * the library makes itself (plan grids, tables and workspace, batch workspace;
 * in any plan or batch and any thread; cuFFT's own work areas are not counted)
 * fails with SE_ENOMEM without calling cudaMalloc, exactly as a real
 * out-of-memory would be reported; later allocations proceed normally.
 * k <= 0 disarms.  Nothing on the GPU is touched.  Always returns SE_OK. */
se_status se_debug_fail_alloc(int64_t k);

/* Name of a status code; text of the last error raised in this thread. */
const char *se_status_str(se_status s);
const char *se_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SE_GB300_H */
