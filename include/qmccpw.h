/*
 * qmccpw — QMC conditional-pathwise (QMC-CPW) Greeks on NVIDIA GB300 (sm_103a).
 *
 * C-ABI of the hot path of Bilokon, Kucherenko & Williams, "Quasi-Monte Carlo
 * methods for calculating derivatives sensitivities on the GPU" (arXiv
 * 2209.11337).  Per point of a randomised Sobol' set the library builds the
 * separated GBM path S~(t_1..t_d) (Sec. 3.3.1), integrates the first Gaussian
 * out in closed form (Sec. 3.3, eq. QmcCpwNewTargetDefinition), evaluates the
 * conditional price and its pathwise delta, vega and gamma (Sec. 3.3.2,
 * Sec. 4.5) and reduces them to one estimate per randomised replicate; the
 * reported estimate is the mean over replicates and its standard error
 * (Sec. 5).  Everything runs in CUDA kernels; no path leaves the GPU.
 *
 * Conventions shared by every entry point
 *   - Dates are equally spaced: t_j = j*T/d, j = 1..d.  n = d-1 Gaussians are
 *     sampled per point; the first Gaussian x_1 is integrated out.
 *   - Value order of every 4-vector: price, delta (d/dS0), vega (d/dsigma,
 *     per unit of sigma, not per 1%), gamma (d^2/dS0^2).
 *   - Point k (0-based) of replicate r uses Sobol' index g(k) = k ^ (k >> 1)
 *     (Gray-code order), so for N = 2^m the point set is the first 2^m points.
 *   - All host pointers are caller-owned and only read/written during the
 *     call.  Device pointers are CUDA global-memory addresses of the plan's
 *     device.
 *   - Every function returns a qmccpw_status; QMCCPW_OK is 0.  On failure no
 *     output is written unless stated, and qmccpw_last_error() describes it.
 *   - One plan may be used by one host thread at a time.
 */
#ifndef QMCCPW_H
#define QMCCPW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
typedef enum {
    QMCCPW_OK = 0,
    QMCCPW_ERR_INVALID_ARG = 1, /* an argument is out of range or NULL */
    QMCCPW_ERR_OOM = 2,         /* device or host memory (or the plan's workspace budget) exhausted */
    QMCCPW_ERR_CUDA = 3,        /* a CUDA runtime call failed; last_error names it */
    QMCCPW_ERR_TIMEOUT = 4,     /* a bounded wait expired */
    QMCCPW_NOT_READY = 5,       /* asynchronous result not yet available (not an error) */
    QMCCPW_ERR_UNSUPPORTED = 6  /* combination not provided (e.g. tensor-core precision with the bridge) */
} qmccpw_status;

/* ---- limits -------------------------------------------------------------- */
#define QMCCPW_D_LIMIT 1024          /* largest number of monitoring dates d of any plan */
#define QMCCPW_R_LIMIT 4096          /* largest number of replicates R of any plan */

/* ---- products (Sec. 4.2, 4.5) -------------------------------------------- */
typedef enum {
    QMCCPW_ARITH_ASIAN_CALL = 0,     /* (mean_j S(t_j) - K)^+                          (Sec. 4.5.2) */
    QMCCPW_BINARY_ASIAN = 1,         /* 1{mean_j S(t_j) > K}                            (Sec. 3.3.2, 4.5.1) */
    QMCCPW_LOOKBACK_FIXED_CALL = 2,  /* (max_j S(t_j) - K)^+                           (Sec. 4.5.3) */
    QMCCPW_GEOMETRIC_ASIAN_CALL = 3  /* (geomean_j S(t_j) - K)^+: same separated form, closed-form price */
} qmccpw_option_type;

/* ---- path construction of W~ = A z with A A^T = Sigma (eq. WboldTilde) -- */
typedef enum {
    QMCCPW_BB = 0,                   /* Brownian bridge, Sec. 4.4: terminal value, then midpoints breadth first */
    QMCCPW_PCA = 1,                  /* principal components of Sigma (named in Sec. 6 as the next reduction) */
    QMCCPW_STD = 2,                  /* standard construction, one increment per step (the path of the
                                        simulation listing, Sec. 4.1-4.2): W~(s_i) = W~(s_{i-1}) + sqrt(dt) z_i */
    QMCCPW_BB_LEAD = 3,              /* the whole path of the d dates by the bridge, its leading coordinate
                                        (the terminal value) integrated out instead of the first increment;
                                        switch point by Newton's method (Sec. 6-7 name this reduction);
                                        the lookback by the upper envelope of the dates' exponentials */
    QMCCPW_PCA_LEAD = 4              /* the same with the PCA of the d dates, its first component integrated out */
} qmccpw_construction;

/* ---- arithmetic precision ----------------------------------------------- */
typedef enum {
    QMCCPW_FP64 = 0,                 /* every step in double precision */
    QMCCPW_MIXED = 1,                /* inverse normal and path in float; switch point psi and the
                                        per-point values in float-float (about 44 bits); tile and
                                        replicate sums in double */
    QMCCPW_MIXED_TC_BF16X3 = 2,      /* MIXED with the PCA product on tensor cores in bf16: z in two
                                        parts, Ahat in three, the leading parts on fixed grids
                                        (exact hi x hi accumulation), five products (d <= 257);
                                        bridge contracts run as MIXED */
    QMCCPW_MIXED_TC_TF32X3 = 3       /* the same in tf32: z and Ahat in two parts, three products
                                        (d <= 257); bridge contracts run as MIXED */
} qmccpw_precision;

typedef struct qmccpw_plan_s *qmccpw_plan_t;
typedef struct qmccpw_batch_s *qmccpw_batch_t;

/* Plan descriptor (read once by qmccpw_plan). */
typedef struct {
    int32_t device;            /* CUDA device ordinal */
    int32_t d_max;             /* largest d this plan accepts, 1..QMCCPW_D_LIMIT */
    int32_t r_max;             /* largest R this plan accepts, 2..QMCCPW_R_LIMIT */
    int32_t reserved;          /* must be 0 */
    uint64_t seed;             /* key of the random linear scrambles and digital shifts */
    void *stream;              /* cudaStream_t to run on; NULL: the plan creates and owns one */
    uint64_t workspace_bytes;  /* device scratch budget in bytes; 0: 1 GiB */
} qmccpw_plan_desc;

typedef struct {
    int32_t type;              /* qmccpw_option_type */
    int32_t d;                 /* monitoring dates, 1..plan d_max */
    double K;                  /* strike, > 0 */
    double T;                  /* maturity in years, > 0 */
} qmccpw_option;

typedef struct {
    double S0;                 /* spot, > 0 */
    double r;                  /* risk-free rate (continuous), finite */
    double sigma;              /* volatility, > 0 */
} qmccpw_market;

typedef struct {
    double mean[4];            /* estimate: mean over replicates of (price, delta, vega, gamma) */
    double se[4];              /* standard error of that mean: sd of replicate estimates / sqrt(R) */
    double *per_replicate;     /* optional caller-owned host array of R*4 doubles (replicate-major);
                                  NULL to skip */
} qmccpw_result;

typedef struct {
    qmccpw_option option;
    qmccpw_market market;
    uint64_t N;                /* points per replicate, 1..2^32 (powers of two recommended) */
    int32_t R;                 /* replicates, 2..plan r_max */
    int32_t construction;      /* qmccpw_construction */
    int32_t first_replicate;   /* the contract uses replicates first_replicate .. first_replicate+R-1
                                  of the plan's randomisation (first_replicate + R <= r_max); 0 for
                                  the usual estimate.  Replicate r is the same set of points whichever
                                  call, batch or GPU computes it, so a contract split into replicate
                                  ranges (plans with the same seed) gives per-replicate estimates
                                  bit-identical to one call over the whole range; mean and SE are
                                  those of the call's own R replicates */
    uint32_t first_point;      /* the contract uses Sobol' points first_point .. first_point+N-1 of
                                  each replicate (first_point + N <= 2^32); 0 for the usual estimate.
                                  The Sobol' sequence extends (Sec. 2.2.2: the first 2^m points of
                                  2^(m+1) are the 2^m-point set), so a run of N1 points from 0 and a
                                  run of N2 points from N1 give, per replicate, (N1 e1 + N2 e2) /
                                  (N1 + N2) = the estimate of N1 + N2 points from 0 (up to the order
                                  of the sums): an estimate can be refined without recomputing the
                                  points it already has */
} qmccpw_contract;

/*
 * Create a plan: selects the device, builds the Sobol' direction numbers
 * (Sec. 2.2.2: primitive polynomials in increasing degree and value, initial
 * odd m_i < 2^i drawn by SplitMix64 under a fixed key) and the scrambled
 * tables of replicates 0..r_max-1 for d_max-1 dimensions (Sec. 2.2.3: unit
 * lower-triangular GF(2) matrix and digital shift, bits drawn by SplitMix64
 * under `seed`), and reserves the scratch workspace.
 * *out receives an opaque handle owned by the caller until qmccpw_free.
 * Errors: INVALID_ARG (NULL, d_max or r_max out of range, reserved != 0),
 * CUDA (device selection or allocation), OOM.
 */
int qmccpw_plan(qmccpw_plan_t *out, const qmccpw_plan_desc *desc);

/*
 * Estimate price, delta, vega and gamma of one contract with N points per
 * replicate and R replicates.  Synchronous: the result is in *out when the
 * call returns.  Path construction per `construction`, arithmetic per
 * `precision` (a tensor-core precision applies to PCA contracts with
 * d <= 257 and runs bridge contracts as MIXED).
 * Errors: INVALID_ARG (d, R outside the plan; N = 0 or > 2^32; S0, K, T,
 * sigma not positive and finite; r not finite), UNSUPPORTED, OOM (workspace
 * budget), CUDA.
 */
int qmccpw_greeks(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market,
                  uint64_t N, int32_t R, int32_t construction, int32_t precision, qmccpw_result *out);

/*
 * Batched form: `count` contracts of any mix of products, d, N and R, run in
 * one persistent launch sequence (one grid over every (contract, replicate,
 * run of tiles) work item; the runs depend on the contract alone).  out[i]
 * receives contract i's result; each out[i].per_replicate may be NULL.
 * Results equal those of qmccpw_greeks for the same contract (same points,
 * same tiles, same order of the sums).
 */
int qmccpw_greeks_batch(qmccpw_plan_t plan, const qmccpw_contract *contracts, int32_t count,
                        int32_t precision, qmccpw_result *out);

/*
 * Prepared batch for device-resident repetition: qmccpw_batch_create uploads
 * the contract descriptors and the work list once; qmccpw_batch_launch
 * enqueues the kernels on `stream` (NULL: the plan's stream) and returns
 * without waiting; results stay on the device until qmccpw_batch_results
 * (synchronises, copies, fills out[0..count-1]).  qmccpw_batch_device_results
 * exposes the device arrays: per_replicate (sum over contracts of R*4
 * doubles, contract-major) and stats (count*8 doubles: mean[4], se[4]).
 */
int qmccpw_batch_create(qmccpw_plan_t plan, const qmccpw_contract *contracts, int32_t count,
                        int32_t precision, qmccpw_batch_t *out);
int qmccpw_batch_launch(qmccpw_batch_t batch, void *stream);
int qmccpw_batch_results(qmccpw_batch_t batch, qmccpw_result *out);
int qmccpw_batch_device_results(qmccpw_batch_t batch, const double **per_replicate,
                                const double **stats);
/* number of CUDA kernel launches one qmccpw_batch_launch enqueues */
int qmccpw_batch_launch_count(qmccpw_batch_t batch, int32_t *launches);
/*
 * Kernel timing (measurement aid, no counterpart in the paper): with
 * capacity > 0, every following qmccpw_batch_launch records a CUDA event
 * pair on its stream around the fused kernel (up to `capacity` launches are
 * kept).  qmccpw_batch_timing waits for those events, returns the summed
 * fused-kernel time in milliseconds and the number of launches it covers,
 * and clears the record.  capacity = 0 turns timing off.
 */
int qmccpw_batch_set_timing(qmccpw_batch_t batch, int32_t capacity);
int qmccpw_batch_timing(qmccpw_batch_t batch, float *fused_ms, int32_t *launches);
/*
 * The same record split by launch segment, without clearing it (call before
 * qmccpw_batch_timing): segment_ms[0] bridge contracts, [1] standard
 * construction, [2] PCA on the streamed tensor-core kernel (d > 65), [3] the
 * other PCA contracts, [4] and [5] the leading-coordinate bridge and PCA,
 * each the summed milliseconds from the end of the previous segment (a
 * segment a batch does not have reads about 0).  Graph replays record no
 * segments (*launches = 0).  segment_ms has 6 entries.
 * Errors: INVALID_ARG (NULL argument), CUDA.
 */
int qmccpw_batch_segment_timing(qmccpw_batch_t batch, float *segment_ms, int32_t *launches);
/*
 * CUDA-graph replay (launch-bound small batches; no counterpart in the
 * paper): with enable != 0 the next qmccpw_batch_launch captures the batch's
 * launch sequence (counter resets, fused grids, reduction, statistics) into
 * a CUDA graph on a private stream, and every launch then replays it with
 * one graph launch on the caller's stream.  The work and its results are
 * the same as without the graph; timing events, if on, bracket the whole
 * replay.  enable = 0 waits for the device and drops the graph.
 * Errors: INVALID_ARG (NULL batch), CUDA (capture or instantiation failed).
 */
int qmccpw_batch_use_graph(qmccpw_batch_t batch, int32_t enable);
int qmccpw_batch_free(qmccpw_batch_t batch);

/*
 * Self-test of the failure path of the tensor-core kernels' waits (no
 * counterpart in the paper): launches on `device` one CTA that waits, with
 * the kernels' own bounded poll loop and a limit of `limit_us`
 * microseconds, on an mbarrier that nothing arrives at.  The wait must give
 * up and the kernel exit normally: *kernel_status = QMCCPW_ERR_TIMEOUT (what
 * the kernels record on expiry), QMCCPW_OK if the barrier completed (a
 * defect).  The context stays usable.  Errors: INVALID_ARG (NULL status,
 * limit outside 1..1e6), OOM, CUDA.
 */
int qmccpw_selftest_bounded_wait(int32_t device, int32_t limit_us, int32_t *kernel_status);

/*
 * Diagnostics for bit-exact checks.  qmccpw_sobol_points writes the 32-bit
 * scrambled Sobol' integers of points k0..k0+count-1 (Gray index g(k)) of
 * replicate `replicate`, dimensions 0..ndims-1, row-major into the host
 * array out[count*ndims], produced by the same device code as the fused
 * kernel.  qmccpw_point_values writes the per-point values (price, delta,
 * vega, gamma) of those points into out[count*4] (host), also from the fused
 * kernel's device code.  count <= 2^20 per call.
 */
int qmccpw_sobol_points(qmccpw_plan_t plan, uint32_t replicate, int32_t ndims, uint64_t k0,
                        uint64_t count, uint32_t *out);
int qmccpw_point_values(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market,
                        int32_t construction, int32_t precision, uint32_t replicate, uint64_t k0,
                        uint64_t count, double *out);

/*
 * Allocation-free form of qmccpw_greeks (the paper has no counterpart: this
 * is a deployment aid).  Some callers must not allocate device memory per
 * request: latency-critical services (cudaMalloc can block and cudaFree
 * synchronises the whole device), and hosts whose device memory is owned by
 * another allocator such as a framework's caching pool, where a stray
 * cudaMalloc competes with that pool for the same memory.  This entry point
 * performs no cudaMalloc,
 * cudaFree or other device-memory allocation: every per-call device array
 * (work-item partial sums, the contract descriptor, the bridge or PCA tables) is
 * placed in one fixed 16 MiB array compiled into the library, which every
 * GPU that loads the library holds until the process exits.  The plan (made
 * beforehand with qmccpw_plan, which does allocate) supplies the Sobol'
 * tables.
 *   out: caller-owned device memory of (R + 2) * 4 doubles, written as the R
 *        per-replicate estimates (replicate-major, 4 values each), then
 *        mean[4], then se[4] (same meaning as qmccpw_result).
 *   stream: cudaStream_t to enqueue on (NULL: the plan's stream).  The call
 *        returns once the work is enqueued; read `out` after synchronising
 *        that stream.
 * All calls on a device share the one array and it keeps the previous
 * call's contents (nothing in it needs to start at zero: every slot a call
 * reads, the same call writes first).  Calls that can overlap on the GPU
 * (issued on different streams without ordering between them) race on the
 * array; serialise them on one stream.  The first call on each device looks
 * up the array's device address (cudaGetSymbolAddress) and caches it: make
 * that first call before any stream capture begins.
 * Errors: as qmccpw_greeks; OOM when the work of this call (32 bytes per
 * work item and replicate: about 32 * R * N / (P * g) bytes, P = 256 points
 * per tile for d <= 65 in MIXED, g = 1..16 tiles per item as N / P grows
 * past 512, plus the d-dependent tables) exceeds the 16 MiB array;
 * UNSUPPORTED for the tensor-core precisions and the leading-coordinate
 * constructions.
 */
int qmccpw_greeks_noalloc(qmccpw_plan_t plan, const qmccpw_option *option, const qmccpw_market *market,
                          uint64_t N, int32_t R, int32_t construction, int32_t precision, double *out,
                          void *stream);

/* ---- tile tuning (a deployment aid; the paper has a fixed 64-thread block)
 * The CUDA-core kernels (FP64, MIXED) process tiles of P points per CTA; by
 * default P is the largest power of two <= 256 whose z/W tile fits 65 KiB of
 * shared memory (three CTAs per SM).  qmccpw_autotune times the fused kernel
 * with CUDA events on a workload of about 2^24 point-dates (2^21 in FP64)
 * for every distinct (construction, d) of `sample`, over P from twice the
 * default down to a quarter of it (>= 32), and keeps the fastest in the
 * plan; every later call on the plan uses it.  qmccpw_tuning_get reads the
 * P in use; qmccpw_tuning_set stores one (a power of two in 32..256; 0
 * restores the default), so a caller can persist and reload a tuning.
 * Different tiles regroup the per-tile partial sums, so FP64 results can
 * differ from the untuned ones in the last bits. */
int qmccpw_autotune(qmccpw_plan_t plan, const qmccpw_contract *sample, int32_t count, int32_t precision);
int qmccpw_tuning_get(qmccpw_plan_t plan, int32_t precision, int32_t construction, int32_t d, int32_t *points_per_tile);
int qmccpw_tuning_set(qmccpw_plan_t plan, int32_t precision, int32_t construction, int32_t d, int32_t points_per_tile);

/* ---- serving: a device-resident request loop ------------------------------
 * Sec. 7 proposes wrapping the estimator in a microservice; this is its GPU
 * side.  A persistent kernel runs on the plan's device while work arrives.
 * Requests (contracts) are written into a ring of pinned, host-mapped
 * entries and published through two host-written counters; one CTA of the
 * kernel copies each new entry into device memory and republishes it there,
 * and the other CTAs take the published requests' work items (replicate,
 * run of tiles) in publication order from one device counter, so a request that
 * arrives while others run fills the SMs as they free up; the CTA that
 * finishes a request's last item reduces it on the device and raises the
 * request's completion flag in host-mapped memory.  Admission is in arrival order,
 * while the admitted requests' device scratch (32 bytes per work item and
 * replicate: about 32 * R * N / (P * g) bytes, P the points per tile, g =
 * 1..16 the tiles per item) fits
 * `max_inflight_bytes` and at most `max_inflight` requests are on the
 * device; the rest wait on the host.  Every wait of the kernel is bounded by
 * %globaltimer: after `idle_limit_us` without a published work item its CTAs
 * leave (the launch ends with an idle status, counted in idle_exits) and the
 * host launches it again when a request arrives; the work items a leaving
 * CTA held are handed out first by that launch.  A host thread watches the
 * flags and relaunches; qmccpw_submit, qmccpw_poll and qmccpw_wait do the
 * same steps themselves.  A request's result does not depend on what else
 * runs: its tiles and their reduction order are those of qmccpw_greeks
 * (bit-identical).  Precisions FP64 and MIXED; the tensor-core precisions
 * return UNSUPPORTED (their PCA kernel is a batch kernel).  While a server
 * runs, the plan must not be used by the other entry points. */
typedef struct {
    int32_t precision;             /* QMCCPW_FP64 or QMCCPW_MIXED for every request */
    int32_t max_inflight;          /* requests on the device at once, 1..4096 (0: 1024); fewer when
                                      r_max * 32 + 64 bytes of host-mapped results per request
                                      would pass 256 MiB */
    int32_t idle_limit_us;         /* the kernel leaves after this long without work, 1..10^7 (0: 20000) */
    int32_t constructions;         /* accepted constructions, bit c for qmccpw_construction c (0: all);
                                      MIXED without QMCCPW_PCA runs a kernel that fits three CTAs per SM
                                      instead of two; other requests return UNSUPPORTED */
    uint64_t max_inflight_bytes;   /* device scratch of the requests on the device (0: 256 MiB) */
} qmccpw_server_desc;

typedef struct {
    uint64_t submitted, completed, failed;
    uint64_t launches;             /* serving-kernel launches: the first and one per return from idle */
    uint64_t idle_exits;           /* launches that ended on the idle limit */
    uint64_t point_dates;          /* sum of N * R * d over completed requests */
    uint64_t pending;              /* requests waiting for admission */
    uint64_t inflight;             /* requests on the device, not yet collected by the host */
    uint64_t running;              /* 1 while a serving kernel runs */
} qmccpw_server_stats;

/* Start the service on a plan (INVALID_ARG if one already runs). */
int qmccpw_server_start(qmccpw_plan_t plan, const qmccpw_server_desc *desc);
/* Queue one contract; *ticket identifies it.  Validation as qmccpw_greeks;
 * OOM if the contract alone needs more than max_inflight_bytes. */
int qmccpw_submit(qmccpw_plan_t plan, const qmccpw_contract *contract, uint64_t *ticket);
/* Non-blocking: OK and the result (per_replicate filled if non-NULL, R*4
 * doubles) once finished, QMCCPW_NOT_READY before; a collected ticket is
 * forgotten. */
int qmccpw_poll(qmccpw_plan_t plan, uint64_t ticket, qmccpw_result *out);
/* Blocking form of qmccpw_poll, at most timeout_ms milliseconds (TIMEOUT). */
int qmccpw_wait(qmccpw_plan_t plan, uint64_t ticket, int32_t timeout_ms, qmccpw_result *out);
int qmccpw_server_get_stats(qmccpw_plan_t plan, qmccpw_server_stats *out);
/* Finish every queued request, then stop the kernel and the host thread
 * (no-op without a server). */
int qmccpw_server_stop(qmccpw_plan_t plan);

/* ---- baskets: several underlying assets (Sec. 6) ----------------------------
 * Sec. 6 notes that the simulation extends to options on several underlying
 * assets by redefining the path and the payoff formulas; this is that
 * extension for a basket average of m <= QMCCPW_ASSETS_MAX correlated GBM
 * assets:
 *   S_i(t) = spot[i] * S0 * exp(omega_i t + sigma_i W_i(t)),
 *   sigma_i = vol[i] * sigma, omega_i = r - sigma_i^2 / 2,
 *   W = L B, L the lower Cholesky factor of corr (L_11 = 1), B independent
 *   standard Brownian motions,
 *   X = sum_i weight[i] * (1/d) sum_j S_i(t_j),  t_j = j T / d.
 * Products: QMCCPW_ARITH_ASIAN_CALL pays (X - K)^+, QMCCPW_BINARY_ASIAN pays
 * 1{X > K}.  Each factor B_k is its first increment sqrt(t_1) x_k plus the
 * bridge of Sec. 4.4 over t_2..t_d (n = d - 1 nodes, the order of the
 * single-asset bridge); x_1, the first increment of factor 1, is integrated
 * out as in Sec. 3.3.1.  Then X(x_1) = sum_i C_i exp(b_i x_1) with
 * b_i = sigma_i L_i1 sqrt(t_1) > 0, and the switch point x* of X(x*) = K is
 * found per point by Newton's method on ln X - ln K; price and Greeks follow
 * in closed form (E[e^{b x}; x > x*] = e^{b^2/2} Phi(b - x*)).  Greeks:
 * delta and gamma with respect to the spot scale S0 (every spot moves with
 * it), vega with respect to the volatility scale sigma (every volatility
 * moves with it).  Sobol' dimension b*m + k (b = 0..d-2, k = 0..m-1) drives
 * bridge node b of factor k+1, dimension (d-1)*m + k-1 the first increment of
 * factor k+1 (k = 1..m-1): m*d - 1 dimensions, at most the plan's d_max - 1.
 * With m = 1 the basket is the single-asset contract with the bridge, point
 * for point. */
#define QMCCPW_ASSETS_MAX 8
typedef struct {
    int32_t type;              /* QMCCPW_ARITH_ASIAN_CALL or QMCCPW_BINARY_ASIAN, on the basket average */
    int32_t d;                 /* monitoring dates; m * d <= plan d_max */
    int32_t m;                 /* assets, 1..QMCCPW_ASSETS_MAX */
    int32_t reserved;          /* must be 0 */
    double K, T;               /* strike > 0, maturity > 0 */
    double S0, r, sigma;       /* spot scale > 0, rate (finite), volatility scale > 0 */
    double weight[QMCCPW_ASSETS_MAX];   /* w_i >= 0, w_0 > 0 */
    double spot[QMCCPW_ASSETS_MAX];     /* relative spots > 0: S_i(0) = spot[i] * S0 */
    double vol[QMCCPW_ASSETS_MAX];      /* relative volatilities > 0: sigma_i = vol[i] * sigma */
    double corr[QMCCPW_ASSETS_MAX * QMCCPW_ASSETS_MAX];  /* m x m correlation, row-major with row
                                                             stride m (the first m*m entries), symmetric
                                                             positive definite, unit diagonal,
                                                             corr[i] > 0 (every asset positively
                                                             correlated with asset 1) */
} qmccpw_basket;

/*
 * Estimate price, delta, vega, gamma of a basket with N points per replicate
 * and R replicates (replicates 0..R-1 of the plan's randomisation).
 * Synchronous, like qmccpw_greeks; precision QMCCPW_FP64 (every step in
 * double) or QMCCPW_MIXED (inverse normal, bridges and exponentials in float
 * with the float path's own polynomials; per-asset sums, switch point and the
 * per-point values in double; tile and replicate sums in double).
 * Errors: INVALID_ARG (NULL, a field out of range, a correlation matrix that
 * is not positive definite), UNSUPPORTED (another type or precision), OOM
 * (workspace budget), CUDA.
 */
int qmccpw_basket_greeks(qmccpw_plan_t plan, const qmccpw_basket *basket, uint64_t N, int32_t R,
                         int32_t precision, qmccpw_result *out);
/* Per-point values (price, delta, vega, gamma) of points k0..k0+count-1 of
 * replicate `replicate` into the host array out[count*4], from the same
 * device code (diagnostics; count <= 2^20). */
int qmccpw_basket_point_values(qmccpw_plan_t plan, const qmccpw_basket *basket, int32_t precision,
                               uint32_t replicate, uint64_t k0, uint64_t count, double *out);

/* Release a plan after waiting for its work; NULL is accepted (no-op). */
int qmccpw_free(qmccpw_plan_t plan);

/* Thread-local description of the last failure of this thread ("" if none).
 * The string stays valid until the thread's next qmccpw call. */
const char *qmccpw_last_error(void);

/*
 * Splitting a job over several GPUs (a deployment aid; the paper runs one GPU).
 * Replicates are independent (Sec. 5: the estimate is the mean of R
 * independently randomised replicate estimates), so a contract's replicates
 * can be split into ranges (qmccpw_contract.first_replicate) computed on
 * different GPUs with plans of the same seed, and a book's contracts split
 * among GPUs.  The only exchange is the R x 4 replicate estimates of each
 * contract.
 *
 * qmccpw_batch_scatter_replicates: after every later launch of `batch`, copy
 * the R x 4 replicate estimates of its contract i (caller's order) to rows
 * first_row[i] .. first_row[i] + R_i - 1 of the device array `dst` (4 doubles
 * a row), on the launch's stream, by a kernel.  first_row is a host array of
 * the batch's count entries, read during the call; dst is caller-owned device
 * memory of the batch's device and must stay valid while launches use it.
 * dst = NULL turns the copy off.  The call waits for the device to be idle.
 * Errors: INVALID_ARG (NULL batch, NULL first_row with dst, negative row),
 * OOM, CUDA.
 *
 * qmccpw_replicate_stats: mean and standard error over replicates (as
 * qmccpw_result: mean of the R replicate estimates and sd / sqrt(R) with the
 * (R - 1) sample variance, both sums compensated, in replicate order) of
 * `count` contracts whose replicate estimates sit in the device array
 * per_replicate: contract i's R[i] rows of 4 doubles from row first_row[i].
 * first_row (int64), R (int32, each >= 2) and stats (count x 8 doubles:
 * mean[4] then se[4] per contract) are device arrays; the kernel is enqueued
 * on `stream` (a cudaStream_t of the current device, NULL: the default
 * stream) and the call returns without waiting.  It allocates nothing.
 * With the rows of every range of a split contract in place, the result is
 * bit-identical to one call over all of its replicates.
 * Errors: INVALID_ARG (NULL array, count < 1), CUDA.
 */
int qmccpw_batch_scatter_replicates(qmccpw_batch_t batch, double *dst, const int64_t *first_row);
int qmccpw_replicate_stats(const double *per_replicate, const int64_t *first_row, const int32_t *R,
                           int32_t count, double *stats, void *stream);

/*
 * Pipe micro-benchmarks (a measurement aid; the paper reports no pipe rates):
 * the issue rates that bound the kernels, measured on `device` with CUDA
 * events (best of five launches after a warm-up), each from long chains of
 * independent operations of one kind over every SM.  The roofline of the
 * float path divides by the FP32 and SFU rates, that of the FP64 path by the
 * FP64 rate, and that of the tensor-core PCA product by the tcgen05 rates.
 *   fp32_fma_tflops:  FFMA, 2 flops per lane and instruction
 *   fp32_fma2_tflops: packed two-lane FFMA2, 4 flops per lane and instruction
 *   fp64_fma_tflops:  DFMA, 2 flops
 *   sfu_*_gops:       ex2.approx, lg2.approx, rcp.approx results per second / 1e9
 *   tc_*_tflops:      dense tcgen05.mma kind::f16 (bf16) and kind::tf32,
 *                     M = 128, N = 256, FP32 accumulation in tensor memory
 * The call allocates a few bytes of device memory, runs about 0.1 s of
 * kernels and changes no device setting.  Errors: CUDA; TIMEOUT if the
 * bounded wait for the tensor-core products expired.
 */
typedef struct {
    double fp32_fma_tflops, fp32_fma2_tflops, fp64_fma_tflops;
    double sfu_ex2_gops, sfu_lg2_gops, sfu_rcp_gops;
    double tc_bf16_tflops, tc_tf32_tflops;
} qmccpw_pipe_peaks;
int qmccpw_measure_pipe_peaks(int32_t device, qmccpw_pipe_peaks *out);

/* Library version string, e.g. "qmccpw 0.1 sm_103a". */
const char *qmccpw_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QMCCPW_H */
