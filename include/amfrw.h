/*
 * amfrw.h -- C ABI of the GB300 (sm_103a) AMFR-W2 sparse-grid solver for the
 * SABR-LMM pricing PDE.
 *
 * Method: J.G. Lopez-Salas, S. Perez-Rodriguez, C. Vazquez, "AMFR-W numerical
 * methods for solving high dimensional SABR/LIBOR PDE models"
 * (arXiv 2408.00559).  The library computes, for each pricing instance:
 *   - the component grids of the standard (eq. standardCombTechnique, psi = 0)
 *     or modified (eq. modifiedCombTechnique, psi >= 1) combination technique,
 *     or one full grid;
 *   - on every grid, the finite-difference semi-discretisation of Sec. 3
 *     (Sketch 1: central differences, Dirichlet data on the lower faces,
 *     homogeneous Neumann conditions on the upper faces, eq. bound1);
 *   - n_steps AMFR-W2 steps (Sec. 4.1, eqs. row-s, Wmat1, amfrw, coef_W2),
 *     each stage made of explicit evaluations of F and the directional
 *     tridiagonal solves of Lemma ls / Algorithm 1;
 *   - multilinear interpolation of every grid at the spot point and the
 *     combination sum  price = discount * sum_l c_l u_l(x*).
 * All arithmetic runs in CUDA kernels on the device; the host only validates
 * parameters, enumerates grids and launches.
 *
 * Conventions for every entry point
 *   - Axes: the paper's F_1..F_{N-1} (forward rates) are axes 0..N-2, the
 *     volatility V = F_N is axis N-1.  N = n_rates + 1, 2 <= N <= 8.
 *   - Ownership: the caller owns every pointer it passes.  Inputs are copied
 *     (to the device) before the call returns; no input pointer is retained.
 *     Device memory the library allocates belongs to the handle that
 *     allocated it and is released by the matching destroy call.
 *   - Streams: cuda_stream is a cudaStream_t (NULL = legacy default stream).
 *     Work is stream-ordered.  Calls that write host memory synchronise the
 *     stream before returning.
 *   - Errors: every int-returning call returns an AMFRW_* status; nothing is
 *     thrown across the ABI.  On error, output arguments are left untouched
 *     and *out handles are set to NULL.  amfrw_status_string() names a status
 *     and amfrw_last_error() gives a one-line detail for the calling thread.
 *   - Device: the current CUDA device of the calling thread at create time.
 */
#ifndef AMFRW_H
#define AMFRW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AMFRW_MAX_DIM 8

enum amfrw_status {
    AMFRW_OK = 0,
    AMFRW_EINVAL = 1,     /* invalid argument (range, NULL, non-finite input)  */
    AMFRW_ENOTPSD = 2,    /* correlation of (F_1..F_{N-1}, V) not PSD          */
    AMFRW_ENOMEM = 3,     /* device or host allocation failed                 */
    AMFRW_ECUDA = 4,      /* a CUDA runtime call failed                       */
    AMFRW_ETIMEOUT = 5,   /* reserved: a bounded device wait gave up          */
    AMFRW_ENONFINITE = 6, /* a computed price is NaN or infinite              */
    AMFRW_ETOOBIG = 7     /* a grid or a problem exceeds the supported size   */
};

enum amfrw_payoff {
    AMFRW_CAPLET = 0,   /* (F_1 - K)^+ (Sec. 2; tau and discounting via discount) */
    AMFRW_SWAPTION = 1  /* max{sum_i tau_i (F_i - K) / prod_{l<=i}(1+tau_l F_l), 0} (Sec. 2) */
};

enum amfrw_precision {
    AMFRW_FP64 = 0,  /* every operation in double precision                      */
    AMFRW_MIXED = 1  /* F and the line solves in FP32; stage accumulation of Y,
                        the evaluation of F on the payoff, interpolation and the
                        combination sum in FP64                                 */
};

/*
 * Problem statement of one pricing instance (Sec. 2 and Sec. 6).
 *   n_rates   N-1 >= 1 forward rates; the PDE has N = n_rates + 1 axes.
 *   alpha     [n_rates]  alpha_i >= 0, instantaneous volatility coefficients.
 *   phi       [n_rates]  rate/volatility correlations phi_i in [-1, 1].
 *   rho       [n_rates*n_rates] row-major rate correlations rho_ij, symmetric,
 *             unit diagonal; [[rho, phi],[phi^T, 1]] must be PSD.
 *   tau       [n_rates]  accrual fractions tau_i > 0 (drift eq. coef_adv and
 *             swaption payoff).
 *   F0        [n_rates]  spot forward rates, 0 <= F0_i <= Fmax_i.
 *   Fmax      [n_rates]  upper domain bounds F_i^max > 0 (Neumann faces).
 *   sigma     volatility of the volatility (>= 0).
 *   beta      elasticity in [0, 1].
 *   V0, Vmax  spot volatility and its upper bound, 0 <= V0 <= Vmax, Vmax > 0.
 *   K, T      strike and maturity T > 0.
 *   discount  price = discount * sum_l c_l u_l(x*)  (e.g. P(0,T_1)).
 *   n_steps   uniform AMFR-W2 steps over [0, T] (dt = T / n_steps), >= 1.
 *   level     combination level n >= 0 (or the full-grid level).
 *   psi       0: standard combination; >= 1: modified combination.
 *   full_grid nonzero: one full grid with `level` on every axis.
 *   precision AMFRW_FP64 or AMFRW_MIXED.
 *   flags     bitwise or of
 *             AMFRW_FLAG_GLOBAL_GRIDS: solve every component grid with its
 *               state in global memory, the path that grids too large for
 *               shared memory (or with lines of more than 256 rows) always
 *               take; the result is the same to rounding;
 *             AMFRW_FLAG_DIRICHLET: the earlier boundary conditions of eq.
 *               bound1_0 instead of the Neumann faces of eq. bound1 on the
 *               rate axes: u = payoff on the upper face F_i = F_i^max of every
 *               rate (the lower faces and V = 0 keep their Dirichlet data,
 *               V = V^max its Neumann condition); a rate line then has
 *               M_i - 1 Inner nodes;
 *             other bits: EINVAL.
 *   theta     W-method parameter; AMFR-W2 has order 3 for (3+sqrt(3))/6.
 *   nu_amf    AMF parameter nu > 0 of eq. (Wmat1) (the paper's nu; named so
 *             apart from the volatility of volatility).
 */
#define AMFRW_FLAG_GLOBAL_GRIDS 1
#define AMFRW_FLAG_DIRICHLET 2

typedef struct amfrw_params {
    int32_t n_rates;
    int32_t payoff;
    int32_t n_steps;
    int32_t level;
    int32_t psi;
    int32_t full_grid;
    int32_t precision;
    int32_t flags;
    const double *alpha;
    const double *phi;
    const double *rho;
    const double *tau;
    const double *F0;
    const double *Fmax;
    double sigma;
    double beta;
    double V0;
    double Vmax;
    double K;
    double T;
    double discount;
    double theta;
    double nu_amf;
} amfrw_params;

typedef struct amfrw_problem amfrw_problem;
typedef struct amfrw_batch amfrw_batch;

/* Validate *p, enumerate its component grids, copy the parameters to the
 * device and set every grid to the payoff (eq. icNd).  No time step is taken.
 * Errors: EINVAL, ENOTPSD, ETOOBIG (a grid has more than 2^22 Inner nodes),
 * ENOMEM, ECUDA. */
int amfrw_problem_create(const amfrw_params *p, void *cuda_stream, amfrw_problem **out);

/* Advance every component grid by n_steps AMFR-W2 steps of size T/p->n_steps
 * (eq. amfrw with eq. coef_W2), then interpolate each grid at the spot.  The
 * grid functions stay on the device, so repeated calls continue in time.
 * Asynchronous on the handle's stream.  Errors: EINVAL (NULL, n_steps < 0),
 * ECUDA. */
int amfrw_step(amfrw_problem *h, int32_t n_steps);

/* price = discount * sum_l c_l u_l(x*) in FP64 in a fixed grid order
 * (eq. standardCombTechnique / modifiedCombTechnique).  Synchronises.  (A
 * mixed-precision problem is not re-solved in FP64 when its sum cancels; the
 * batch entry points do that, see amfrw_batch_set_kappa_max.)
 * Errors: EINVAL, ECUDA, ENONFINITE. */
int amfrw_combine(amfrw_problem *h, double *price_out);

/* Number of component grids and the dimension N. */
int amfrw_problem_num_grids(const amfrw_problem *h, int32_t *n_grids, int32_t *dim);

/* Grid levels [n_grids * N] (log2 M_i per axis) and coefficients c_l
 * [n_grids], in the library's grid order.  Host outputs, caller-allocated. */
int amfrw_problem_grid_info(const amfrw_problem *h, int32_t *levels_out, double *coefs_out);

/* Interpolated values u_l(x*) after the last amfrw_step [n_grids], host
 * output.  Synchronises. */
int amfrw_problem_grid_values(amfrw_problem *h, double *u_out);

/* The grid function Y of grid `grid` on its Inner nodes (all j_i >= 1),
 * prod_i M_i doubles in lexicographic order with axis 0 fastest (the paper's
 * theta_1 order, Sec. 3).  Outer nodes are not returned (they hold the
 * payoff).  Host output.  Synchronises.  Errors: EINVAL, ECUDA. */
int amfrw_problem_read_grid(amfrw_problem *h, int32_t grid, double *Y_out);

void amfrw_problem_destroy(amfrw_problem *h);

/* Price n independent instances in one go: upload, one persistent launch per
 * kernel class over all their component grids, combination, download.
 * prices_out: host array [n].  Synchronises.  Errors as create/combine.
 * Plan reuse: the calling thread keeps the batch of its last call (grid
 * list, device buffers, captured graph; about what amfrw_batch_create
 * allocates).  A following call on the same device and stream whose
 * instances have, one by one, the same n_rates, payoff, n_steps, level, psi,
 * full_grid, precision and flags validates its parameters, uploads only the
 * instance records and replays the graph; any other call releases it and
 * plans afresh.  amfrw_solve_batch_release frees it (so does thread exit).
 * After an ECUDA error nothing is kept. */
int amfrw_solve_batch(const amfrw_params *ps, int32_t n, double *prices_out, void *cuda_stream);

/* Bytes the calling thread's last amfrw_solve_batch call copied host->device
 * (everything a fresh plan uploads, or the instance records alone when the
 * plan was reused) and device->host (prices and the non-finite flag); 0
 * before any call.  Errors: EINVAL (NULL). */
int amfrw_solve_batch_io(int64_t *h2d_bytes, int64_t *d2h_bytes);

/* Free the plan amfrw_solve_batch keeps for the calling thread (no-op if
 * none). */
void amfrw_solve_batch_release(void);

/* The same split in two: amfrw_batch_create validates, enumerates and uploads
 * everything once; amfrw_batch_run prices all instances with device-resident
 * inputs and writes the prices to the DEVICE array d_prices_out [n]
 * (asynchronous, stream-ordered; the array must stay valid until the stream
 * reaches that point).  amfrw_batch_run may be called any number of times;
 * its first call captures the solve and the combination into a CUDA graph
 * (on a private stream) that later calls replay. */
int amfrw_batch_create(const amfrw_params *ps, int32_t n, void *cuda_stream, amfrw_batch **out);
int amfrw_batch_run(amfrw_batch *b, double *d_prices_out);
/* Number of kernel launches one amfrw_batch_run issues (for accounting). */
int amfrw_batch_launches(const amfrw_batch *b, int32_t *n_launches);

/* Kernel timing (tracing).  With timing on, every amfrw_batch_run records a
 * CUDA event pair around each solver launch: one persistent multi-class
 * launch per (N, precision) for all grids of at most 64 Inner nodes (when
 * that strategy is selected), and one launch per remaining (N, precision,
 * grid class).  amfrw_batch_kernel_times synchronises and writes, for the
 * last run, the device milliseconds of each solver launch to
 * ms_out[0..*n_out-1] (at most cap entries), the Inner-node-steps it advanced
 * (sum over its grids of Inner nodes x steps) to node_steps_out (may be NULL)
 * and its N to dims_out (may be NULL). */
int amfrw_batch_enable_timing(amfrw_batch *b, int32_t on);
int amfrw_batch_kernel_times(amfrw_batch *b, float *ms_out, double *node_steps_out,
                             int32_t *dims_out, int32_t cap, int32_t *n_out);

/* Autotuning of the launch strategy, of the warp groups' width and of where
 * grid states live (the paper has no counterpart; its CPU code schedules
 * grids with OpenMP's dynamic schedule).  Times, on this batch and device
 * (`trials` solves each after a warm-up): (1) per-class launches against one
 * persistent multi-class launch for the warp-solved grids; (2) the warp
 * groups' width: each grid on its natural number of lanes (two nodes per
 * lane) against twice as many (one node per lane, one more level of parallel
 * cyclic reduction and fewer Thomas rows per line); (3) for every CTA class
 * (grids in shared memory) its launch with the grid states in shared memory
 * against in global memory, class by class.  Keeps the faster choices (the
 * single persistent launch unless the per-class launches are more than 10 %
 * faster) and caches them in-process under the batch's class signature (and, if the
 * environment variable AMFRW_TUNE_CACHE names a file, appends them there),
 * so later batches with the same classes start with them.  *use_multi_out
 * (may be NULL) receives choice (1).  Prices change by rounding only.
 * Synchronises. */
int amfrw_batch_autotune(amfrw_batch *b, int32_t trials, int32_t *use_multi_out);
/* FP64 re-solve of ill-conditioned mixed-precision instances (the paper has no
 * counterpart: it computes in FP64 only).  A mixed-precision price carries an
 * error that is a small multiple of the combination's scale
 * sum_l |c_l u_l| (about 3e-11 of it, measured against FP64), so where the
 * combination sum cancels, kappa = sum_l |c_l u_l| / |sum_l c_l u_l| large,
 * the relative error of the price grows by kappa.  Every amfrw_batch_run (and
 * amfrw_solve_batch) computes kappa per instance in its combination kernel;
 * mixed instances with kappa > kappa_max are re-solved in FP64 and
 * recombined inside the same CUDA graph, by a conditional node that runs only
 * when some instance is above the bound.  Default kappa_max: 1e5.
 *   set_kappa_max  kappa_max <= 0 turns the re-solve off; takes effect at the
 *                  next amfrw_batch_run.  Errors: EINVAL.
 *   promoted       after a run: *n_promoted = instances re-solved in FP64 by
 *                  the last run, kappa_out [n] (may be NULL) = each instance's
 *                  kappa from that run's mixed or FP64 solve (0 when the
 *                  re-solve is off or the batch has no mixed instance).
 *                  Synchronises.  Errors: EINVAL, ECUDA. */
int amfrw_batch_set_kappa_max(amfrw_batch *b, double kappa_max);
int amfrw_batch_promoted(amfrw_batch *b, int32_t *n_promoted, double *kappa_out);

/* Launch classes of a batch by work-group kind: warp groups, CTA groups
 * (grids in shared memory), global-memory groups.  Any pointer may be NULL. */
int amfrw_batch_classes(const amfrw_batch *b, int32_t *n_warp, int32_t *n_cta, int32_t *n_global);

/* Bytes one amfrw_solve_batch call of this problem set copies host->device
 * (instance records, grid list, coefficients) and device->host (prices and
 * the non-finite flag). */
int amfrw_batch_io_bytes(const amfrw_batch *b, int64_t *h2d_bytes, int64_t *d2h_bytes);
void amfrw_batch_destroy(amfrw_batch *b);

/* ------------------------------------------------------------------------
 * Surrogate network building block (the paper has no counterpart; the
 * surrogate is an addition to the method).  C[M x N] = A[M x K] * B[N x K]^T
 * on the tensor cores (tcgen05, BF16 operands, FP32 accumulation).  A, B:
 * DEVICE, row-major BF16 with leading dimensions lda, ldb (multiples of 8,
 * >= K, 16-byte aligned); C: DEVICE FP32 row-major with leading dimension
 * ldc >= N.  Requires N a multiple of 16 (and of 256 when above 256), K a
 * multiple of 16.  Synchronises.  Errors: EINVAL, ENOMEM, ECUDA, ETIMEOUT
 * (a bounded wait inside the kernel gave up; the result is not valid). */
int amfrw_tc_gemm_bf16(const void *dA, int32_t lda, const void *dB, int32_t ldb, float *dC,
                       int32_t ldc, int32_t M, int32_t N, int32_t K, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Surrogate pricing with solver fallback (the paper has no counterpart; it is
 * an addition to the method).  An ensemble of MLPs 8 -> 256 -> 256 -> 256 -> 1
 * with GELU, BF16 weights and activations on the tensor cores (tcgen05) and
 * FP32 accumulation maps the features of an instance to its price.  One
 * surrogate serves one instance family, fixed by the training set:
 *   - N, payoff, n_steps, level, psi, full_grid, precision, F0, Fmax, tau, V0,
 *     Vmax, discount, theta and nu_amf equal to the training set's;
 *   - one alpha shared by all rates; rate correlations
 *     rho_ik = exp(-lambda |i - k|); rate/vol correlations phi_i linear in the
 *     rate index between phi_1 and phi_{N-1}.
 * The features (alpha, sigma, beta, K, T, lambda, phi_1, phi_{N-1}), in this
 * order, then determine the instance (lambda = 0 when N = 2).  A feature that
 * takes between 2 and 32 distinct values in the training set (for instance
 * strikes on a lattice) is a lattice feature: queries off its training values
 * are outside the box and fall back.  The ensemble
 * spread times a calibration factor estimates the error; eval answers from
 * the network where that estimate is within rel_bound * |price| and falls
 * back to the batched solver (amfrw_solve_batch) for every other query,
 * including queries outside the family or outside the trained feature box.
 * All arrays are host memory; calls synchronise.  Errors are reported by
 * amfrw_surrogate_last_error().
 *   create     n_members in [1, 16] networks, He initialisation from `seed`.
 *   fit        on n >= 1024 instances and their solver prices: the target
 *              g is the log price when every price is positive (so squared
 *              errors are relative), else the price.  A least-squares cubic
 *              in the normalised features (165 monomials) is the control
 *              variate; every member learns the standardised residual of g
 *              (Adam, cosine-decayed learning rate, batches of 1024, mean
 *              squared error); the members train concurrently, each on a
 *              stream of its own, joined to cuda_stream before returning.  *final_loss_out (may be NULL) = mean loss of
 *              the last epoch, in standardised units.
 *   calibrate  on an audit sample judged by the solver: the factor is the
 *              `quantile` of |error| / spread; stores rel_bound.
 *   predict    ensemble mean and spread (price units) per instance;
 *              in_domain_out (may be NULL) = 1 inside the family and box.
 *   predict_features  the same for raw feature rows [n x 8]; in_box_out
 *              (may be NULL) = 1 inside the trained feature box.
 *   eval       prices_out [n] (network or solver), fell_back_out [n] (may be
 *              NULL): 1 where the solver priced the instance.
 *   eval_features  the same for queries given as raw features [n x 8]
 *              (row-major, the order above) of the family's instances; a
 *              fallback query is solved as the family instance with those
 *              features (EINVAL if that instance is not valid).
 *   save/load  plain binary file (magic AMFRWSG3, scaling, family,
 *              lattices, FP32 weights).
 *   params     FP32 parameters of one member (136193 floats: W1 [256 x 16]
 *              (inputs 8..15 are padding), b1 [256], W2 [256 x 256], b2, W3,
 *              b3, w4 [256], b4), read to params_out and/or set from
 *              params_in (either may be NULL).
 *   grad       loss 1/2 mean (y - t)^2 and its gradient (same layout) for one
 *              batch of `rows` (multiple of 16, <= 1024) normalised feature
 *              rows x_norm [rows x 8] and targets [rows]; no update. */
typedef struct amfrw_surrogate amfrw_surrogate;
int amfrw_surrogate_create(int32_t n_members, uint64_t seed, void *cuda_stream, amfrw_surrogate **out);
int amfrw_surrogate_fit(amfrw_surrogate *s, const amfrw_params *ps, const double *prices, int64_t n,
                        int32_t epochs, float lr, float *final_loss_out);
int amfrw_surrogate_calibrate(amfrw_surrogate *s, const amfrw_params *ps, const double *prices, int64_t n,
                              double rel_bound, double quantile, double *calib_out);
int amfrw_surrogate_predict(amfrw_surrogate *s, const amfrw_params *ps, int64_t n, double *mean_out,
                            double *spread_out, uint8_t *in_domain_out);
int amfrw_surrogate_predict_features(amfrw_surrogate *s, const double *features, int64_t n, double *mean_out,
                                     double *spread_out, uint8_t *in_box_out);
int amfrw_surrogate_eval(amfrw_surrogate *s, const amfrw_params *ps, int64_t n, double *prices_out,
                         uint8_t *fell_back_out, void *cuda_stream);
int amfrw_surrogate_eval_features(amfrw_surrogate *s, const double *features, int64_t n, double *prices_out,
                                  uint8_t *fell_back_out, void *cuda_stream);
int amfrw_surrogate_save(const amfrw_surrogate *s, const char *path);
int amfrw_surrogate_load(const char *path, void *cuda_stream, amfrw_surrogate **out);
int amfrw_surrogate_params(amfrw_surrogate *s, int32_t member, float *params_out, const float *params_in);
int amfrw_surrogate_grad(amfrw_surrogate *s, int32_t member, const float *x_norm, const float *targets,
                         int32_t rows, float *grad_out, float *loss_out);
void amfrw_surrogate_destroy(amfrw_surrogate *s);
const char *amfrw_surrogate_last_error(void);

/* ------------------------------------------------------------------------
 * Pricing without device allocation.  The paper has no counterpart: this is
 * an integration entry point of the library.
 *
 * Every other entry point obtains its device buffers with cudaMalloc.  Some
 * callers cannot: programs whose device memory belongs to another allocator
 * (a framework's caching pool, or a fixed budget reserved at start-up), and
 * latency-sensitive loops that must not pay for cudaMalloc/cudaFree, since a
 * free synchronises the whole device and stalls every other stream.
 * amfrw_solve_noalloc prices the n instances of ps like amfrw_solve_batch,
 * but its device working memory is one fixed array compiled into the library
 * (AMFRW_NOALLOC_SCRATCH_BYTES); it calls no cudaMalloc, cudaFree or other
 * allocating routine.  Host side it only uses small temporary host buffers
 * for validation and the grid list.
 *   - d_prices_out: DEVICE array [n] owned by the caller; written
 *     asynchronously on cuda_stream (like amfrw_batch_run).
 *   - Limit: the instance records, grid list, per-grid values, counters and
 *     line-solve factors must fit in AMFRW_NOALLOC_SCRATCH_BYTES (about 2000
 *     instances of the d=4 level-5 problem, or one d=6 modified level-6
 *     problem); larger problems are rejected with AMFRW_ETOOBIG and a message
 *     giving the bytes needed.  All instances must share n_steps (EINVAL).
 *   - The array is reserved on every GPU that loads the library, for the life
 *     of the process, and is shared by all calls: calls whose work overlaps
 *     on the GPU (different streams, or host threads) race and give wrong
 *     prices; serialise them.  The array keeps the previous call's contents;
 *     each call rewrites everything it reads and zeroes its counters.
 *   - Each call looks up the array's device address for the calling thread's
 *     current device (cheap once the library's module is loaded; nothing is
 *     cached, so a device reset between calls is harmless).
 *   - The call must not be recorded into a CUDA graph: it copies its records
 *     from temporary host buffers that are freed when it returns.  A call
 *     while cuda_stream is being captured returns EINVAL.
 *   - The prices are not checked for finiteness (there is no host copy of
 *     them to inspect without a synchronisation); the caller tests them.
 *     Mixed-precision instances whose combination sum cancels are not
 *     re-solved in FP64 (amfrw_batch_set_kappa_max describes that re-solve of
 *     the allocating batch entry points).
 * Errors: EINVAL, ENOTPSD, ETOOBIG, ECUDA. */
#define AMFRW_NOALLOC_SCRATCH_BYTES (16u << 20)
int amfrw_solve_noalloc(const amfrw_params *ps, int32_t n, double *d_prices_out, void *cuda_stream);

/* ------------------------------------------------------------------------
 * Arithmetic peak of the current device (a measurement utility; the paper has
 * no counterpart).  The solver kernels keep their grids in shared memory and
 * are bound by the FP64 or FP32 pipes, whose rates are not among the copy and
 * GEMM peaks measured elsewhere, so the library measures them itself: every
 * resident thread of the device runs 8 independent FMA chains of `iters`
 * dependent FMAs (precision AMFRW_FP64, or 2 for FP32), timed with CUDA events
 * on cuda_stream (the best of 5 launches after a warm-up).
 * *tflops_out = 2 x FMAs / time, in TFLOP/s.  Synchronises.
 * Errors: EINVAL (NULL, iters < 1, unknown precision), ECUDA. */
int amfrw_peak_probe(int32_t precision, int32_t iters, double *tflops_out, void *cuda_stream);

const char *amfrw_status_string(int status);
const char *amfrw_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* AMFRW_H */
