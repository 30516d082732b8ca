/*
 * smc2.h -- C ABI of the GB300 CRN particle filter and gradient-enhanced SMC^2
 * (arXiv 2407.17296, "Enhanced SMC^2: Leveraging Gradient Information from
 * Differentiable Particle Filters Within Langevin Proposals").
 *
 * Plain C99.  No C++ or torch types cross this boundary; device pointers are
 * plain addresses in the current CUDA context and streams are passed as
 * `void*` holding a cudaStream_t.
 *
 * Error convention.  Every function returns an int: SMC2_OK (0), SMC2_PENDING
 * (1, only smc2_poll) or a negative SMC2_E_* code.  smc2_last_error() returns a
 * thread-local message describing the last failure on the calling thread.  No
 * exception crosses the ABI; device-side trouble is reported through status
 * words, never through a device fault.
 *
 * Notation follows the paper: N samples theta (the outer SMC sampler, Sec. III),
 * M particles x per filter (N_x in Sec. II), T observations y_{1:T}, D = |theta|.
 */
#ifndef SMC2_H
#define SMC2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
#define SMC2_OK 0
#define SMC2_PENDING 1
#define SMC2_E_INVAL (-1)    /* bad argument or unsupported configuration */
#define SMC2_E_NOMEM (-2)    /* device memory or HBM budget exhausted */
#define SMC2_E_CUDA (-3)     /* a CUDA runtime call failed */
#define SMC2_E_TIMEOUT (-4)  /* a bounded wait expired */
#define SMC2_E_NOTFOUND (-5) /* unknown job id */
#define SMC2_E_BUSY (-6)     /* resource in use */

/* State-space model families (Sec. II, Eqs. xt and yt).
 *  SMC2_LG_DIAG: theta = (a[d_x], log q[d_x], log r[d_y]), D = 2 d_x + d_y;
 *    x_0 ~ N(0, I), x_t = diag(a) x_{t-1} + diag(q) v_t, y_t = H x_t + diag(r) w_t.
 *    Supported shapes (d_x, d_y): (1,1), (4,2), (16,16) with H = identity.
 *  SMC2_SV: theta = (mu, atanh phi, log sigma), D = 3, d_x = d_y = 1;
 *    x_0 = mu + sigma/sqrt(1-phi^2) eps, x_t = mu + phi (x_{t-1} - mu) + sigma eta_t,
 *    y_t = exp(x_t / 2) eps_t.
 *  SMC2_LG_OPT: the linear-Gaussian model of Sec. IV-A, theta = (mu, phi, sigma), D = 3,
 *    d_x = d_y = 1; x_0 ~ N(0, 1), x_t ~ N(mu x_{t-1}, phi^2), y_t ~ N(x_t, sigma^2),
 *    filtered with the "optimal" proposal N(rho^2 (y_t/sigma^2 + mu x_{t-1}/phi^2), rho^2),
 *    1/rho^2 = 1/phi^2 + 1/sigma^2, and weights p(y_t | x_{t-1}) = N(y_t; mu x_{t-1},
 *    phi^2 + sigma^2). */
enum { SMC2_LG_DIAG = 0, SMC2_SV = 1, SMC2_LG_OPT = 2 };
/* Outer proposals (Sec. III-D): SMC0 random walk, SMC1 Langevin, and HMC and NUTS (the
 * extensions Sec. V names).  HMC: hmc_steps leapfrog steps whose single step is the SMC1
 * move, with momentum v ~ N(0, gamma^2 I) and the momentum-reversal L-kernel, i.e. the weight
 * pi(theta_L) N(v_L; 0, gamma^2 I) / (pi(theta_0) N(v_0; 0, gamma^2 I)).  NUTS: the same
 * leapfrog, run forwards or backwards in time, doubles a trajectory in random directions
 * until it makes a U-turn ((theta+ - theta-) . v < 0 at an end of a sub-trajectory), a point
 * diverges (H - H_0 > 1000, H = -log pi + |v|^2 / (2 gamma^2), or a non-finite estimate) or
 * the depth reaches nuts_max_depth; the new sample is drawn from the trajectory with weights
 * exp(-H) (uniform progressive sampling inside a new sub-trajectory, biased progressive
 * sampling when it is merged).  Its L-kernel (nuts_weight): SMC2_NUTS_REVERSAL, the NUTS
 * kernel's own reversal, which leaves log w unchanged (exact for a fixed target; the
 * default), or SMC2_NUTS_MOMENTUM_REVERSAL, the HMC weight above at the selected point and
 * its momentum.  Random numbers: Philox stream 5 of the sample's key (direction of doubling
 * j: top bit of word 0 of counter (j, 0, 5, 0); merge uniform: word 2 of that counter;
 * selection uniform of point n of doubling j: word 1 of counter (j, n, 5, 0)); momentum:
 * stream 3 as HMC.  The trajectory points of all samples are built in lockstep: every
 * iteration runs 2^nuts_max_depth - 1 leapfrog points, each a forward + adjoint pass of the
 * N particle filters with the iteration's CRN keys (samples whose trajectory has stopped
 * ignore theirs). */
enum { SMC2_RW = 0, SMC2_LANGEVIN = 1, SMC2_HMC = 2, SMC2_NUTS = 3 };
enum { SMC2_NUTS_REVERSAL = 0, SMC2_NUTS_MOMENTUM_REVERSAL = 1 };
/* Particle-filter resampler (Sec. II-B, App. B). */
enum { SMC2_SYSTEMATIC = 0, SMC2_MULTINOMIAL = 1 };
/* Prior on theta: Gaussian N(prior_mean, diag(prior_std^2)), or uniform on the box
 * [prior_mean[d], prior_std[d]] (Sec. IV-A), whose iteration-1 draws map the sampler's
 * normals through the standard normal CDF. */
enum { SMC2_PRIOR_GAUSSIAN = 0, SMC2_PRIOR_UNIFORM = 1 };

typedef struct smc2_config {
    uint32_t struct_size;       /* sizeof(smc2_config): versioning */
    int32_t model_family;       /* SMC2_LG_DIAG or SMC2_SV */
    int32_t d_x, d_y;
    const float* H;             /* host, d_y x d_x row-major; NULL = identity; copied */
    const float* y;             /* T x d_y row-major observations; copied */
    int32_t y_on_device;        /* nonzero: y is a device pointer */
    int32_t T, N, M, D;         /* D must equal the family's parameter count */
    const double* prior_mean;   /* host [D] or NULL (zeros); prior N(mean, diag(std^2)) */
    const double* prior_std;    /* host [D] or NULL (ones) */
    int32_t proposal;           /* SMC2_RW, SMC2_LANGEVIN or SMC2_HMC */
    double gamma;               /* step size, Gamma = gamma^2 I */
    int32_t K_iters;            /* iterations for a served job (smc2_submit) */
    int32_t pf_resample;        /* SMC2_SYSTEMATIC or SMC2_MULTINOMIAL */
    float ess_frac;             /* resample the filter when ESS < ess_frac * M (0.5 in the paper) */
    uint64_t seed;              /* CRN seed: key (seed_lo ^ k, seed_hi ^ i) per sample i, iteration k */
    int32_t ckpt_every;         /* adjoint checkpoint interval in steps; 0 = automatic, 1 = store all */
    int32_t particles_per_thread; /* 0 = automatic (autotuned), else 1, 2, 4 or 8 */
    void* stream;               /* cudaStream_t for all work of the handle; NULL = a private stream */
    int32_t prior_kind;         /* SMC2_PRIOR_GAUSSIAN (default) or SMC2_PRIOR_UNIFORM */
    int32_t hmc_steps;          /* SMC2_HMC: leapfrog steps per move, 1..64 (1 = the SMC1 move) */
    int32_t nuts_max_depth;     /* SMC2_NUTS: maximum number of doublings, 1..6 */
    int32_t nuts_weight;        /* SMC2_NUTS: SMC2_NUTS_REVERSAL or SMC2_NUTS_MOMENTUM_REVERSAL */
} smc2_config;

/* Fill defaults: struct_size, ess_frac 0.5, K_iters 10, systematic, Langevin, gamma 0.1,
 * hmc_steps 1, nuts_max_depth 3, nuts_weight SMC2_NUTS_REVERSAL. */
void smc2_config_init(smc2_config* cfg);

typedef struct smc2_handle smc2_handle;

/* Per-iteration statistics of smc2_step (Sec. III-A..C). */
typedef struct smc2_stats {
    int32_t k;                /* iteration just completed, 1-based */
    int32_t resampled;        /* outer resampling happened at the end of k */
    double ess;               /* N_eff of the outer weights before resampling (Eq. ess_smc2) */
    double l_k;               /* recycling statistic (Eq. recycling_I) */
    double max_logw;          /* largest outer log-weight (diagnostic) */
    double* mean;             /* caller host storage [D] or NULL: f~_k = sum_i w~_i theta_i (Eq. realised_estimates) */
    double* recycled_mean;    /* caller host storage [D] or NULL: sum_k c_k f~_k over iterations so far (Sec. III-C) */
    /* Near-ties of iteration k (App. B: the ancestor index counts the cumulative weights below a
     * threshold, so a weight within rounding of a threshold decides it only up to rounding).
     * pf_near_ties: over the N filters, systematic resampling counts the cumulative weights
     * c_j (j < M-1) within 1e-6 of a threshold (i + nu)/M, multinomial the thresholds nu_i
     * within 1e-6 of the cumulative weights next to their index; evaluated in FP32.
     * pf_resample_steps: filter steps that resampled (the decisions those ties come from).
     * outer_near_ties: outer resampling thresholds within 1e-6 of a cumulative weight (FP64),
     * 0 when the outer sampler did not resample. */
    int64_t pf_near_ties;
    int64_t pf_resample_steps;
    int64_t outer_near_ties;
} smc2_stats;

/*
 * smc2_create: validate cfg, copy y and H, allocate the device-resident state of
 * one inference job (theta [N][D], log-weights, log pi-hat, gradients, particle
 * checkpoints and the ancestor tape).  The library owns every allocation it makes.
 * Sizes: 1 <= N <= 16384 samples, 1 <= M <= 4096 particles (less where a model's block would
 * not fit), T >= 1.
 * Errors: SMC2_E_INVAL (bad or unsupported cfg), SMC2_E_NOMEM, SMC2_E_CUDA.
 * Problem statement: Sec. II (f, g, y_{1:T}, M) and Sec. III (prior, N, step size).
 */
int smc2_create(const smc2_config* cfg, smc2_handle** out);

/*
 * pf_loglik_grad: the hot path.  For rows i = 0..n-1 of theta_dev ([n][D] row-major
 * FP64, device) run one CRN particle filter each with Philox key
 * (seed_lo ^ iter, seed_hi ^ i) and write log p-hat(y|theta_i) to loglik_dev[i]
 * (FP64, device; the log of Eq. likelihood_pf_) and, if grad_dev is not NULL, its
 * gradient d log p-hat / d theta (Eq. dloglik, App. A/B, computed by a reverse-time
 * adjoint) to grad_dev[i*D..] (FP64, device).  A filter whose weights all vanish
 * or overflow reports log p-hat = -inf and a zero gradient.
 * Caller owns all buffers; n <= N of the handle.  Asynchronous on the handle's
 * stream.  When a gradient is requested, the handle's N filters exceed what the GPU holds
 * at once and n is above half of N, the rows run as two halves, the second on a stream of the handle's own that
 * is forked from and joined back into the handle's stream (work queued on that stream
 * afterwards still waits for every row).  Errors: SMC2_E_INVAL, SMC2_E_CUDA.
 */
int pf_loglik_grad(smc2_handle* h, const double* theta_dev, int n, uint32_t iter,
                   double* loglik_dev, double* grad_dev);

/* As pf_loglik_grad with the Philox row index starting at row0 (rows row0..row0+n-1),
 * for callers that shard the N samples of one iteration across launches or devices. */
int pf_loglik_grad_rows(smc2_handle* h, const double* theta_dev, int n, uint32_t iter,
                        uint32_t row0, double* loglik_dev, double* grad_dev);

/* As pf_loglik_grad with HOST buffers: copies theta in, runs, copies loglik/grad out,
 * and synchronises the handle's stream before returning. */
int pf_loglik_grad_host(smc2_handle* h, const double* theta_host, int n, uint32_t iter,
                        double* loglik_host, double* grad_host);

/*
 * smc2_step: one SMC^2 iteration k (k counts from 1 per handle).
 *  k = 1: theta ~ prior (Eq. init_sample), PF, w = pi/q_1 (Eq. init_weights).
 *  k > 1: Langevin or random-walk move (Sec. III-D), PF at the new theta, weight with
 *         the L-kernel (Eq. l_weights, Sec. III-E); with SMC2_HMC, hmc_steps leapfrog steps
 *         (a PF forward + adjoint at every point) and the momentum-reversal weight; with
 *         SMC2_NUTS, a no-U-turn trajectory of up to 2^nuts_max_depth - 1 points.
 *  then normalise, estimate, recycling statistic, ESS and, if N_eff < N/2,
 *  systematic resampling (Sec. III-A..C).  Fills *out (may be NULL) on the host:
 *  this call synchronises the handle's stream.
 * Errors: SMC2_E_INVAL, SMC2_E_CUDA.
 */
int smc2_step(smc2_handle* h, smc2_stats* out);

/* K SMC^2 iterations back to back (asynchronous on the handle's stream; no host
 * round trip between them), then fills *out (may be NULL) with the statistics of the last
 * one, synchronising once.  Equivalent to K calls of smc2_step.  Errors as smc2_step. */
int smc2_run(smc2_handle* h, int K, smc2_stats* out);

/* Filter-pass timing.  With timing on, iterations record CUDA events on the handle's stream
 * around the forward and adjoint passes (iterations after the first replay the captured step
 * graph with three event-record nodes, re-targeted to a ring of events before each launch, so
 * the timed iterations run as production ones do); smc2_get_step_timing returns the mean
 * device time of the
 * passes over the iterations run since timing was switched on or last queried (up to the
 * last 512): ms[0] forward, ms[1] adjoint (waits for them to finish).  A handle whose N
 * filters exceed what the GPU holds at once runs them as two halves on two streams, the
 * forward pass of one overlapping the adjoint of the other: then ms[0] is the time of both
 * passes together and ms[1] is -1.  SMC2_E_INVAL if no timed iteration ran since then. */
int smc2_set_step_timing(smc2_handle* h, int on);
int smc2_get_step_timing(smc2_handle* h, float* ms);

/*
 * One SMC^2 iteration split in two calls, for a job whose N particle filters are spread
 * over several devices or processes (the filters of an iteration are independent: the
 * importance-sampling and gradient rows of Table I scale with N/P; only the O(N D) outer
 * update couples the samples).  Every participant holds a replica of the outer state
 * (a handle created from the same cfg) and:
 *   smc2_step_filters  proposes theta' for all N samples (Sec. III-D; the same Philox keys on
 *                      every replica, so the proposals agree) and runs the particle filters
 *                      of rows row0 .. row0+n-1 only, with the Philox keys of those rows,
 *                      writing log p-hat to loglik_dev [n] and its gradient to grad_dev
 *                      [n][D] (caller-owned device buffers, FP64).  Asynchronous on the
 *                      handle's stream.
 *   (the caller exchanges the rows, e.g. one all-gather, so each replica has all N)
 *   smc2_step_update   takes loglik_all_dev [N] and grad_all_dev [N][D] (device, caller-owned,
 *                      row i = sample i) and completes the iteration exactly as smc2_step:
 *                      L-kernel weight, normalise, estimate, recycling statistic, ESS,
 *                      resampling (Sec. III-A..E).  Fills *out (may be NULL); synchronises.
 * Replicas that pass the same N rows to smc2_step_update stay identical, and equal to one
 * handle running smc2_step.  The two calls must alternate; smc2_step_update without a
 * preceding smc2_step_filters, or n < 0, row0 < 0, row0 + n > N, or NULL buffers with n > 0:
 * SMC2_E_INVAL; so is a handle with the SMC2_HMC or SMC2_NUTS proposal (their leapfrog
 * needs every sample's filters at each point).  Launch failures: SMC2_E_CUDA.
 */
int smc2_step_filters(smc2_handle* h, int row0, int n, double* loglik_dev, double* grad_dev);
int smc2_step_update(smc2_handle* h, const double* loglik_all_dev, const double* grad_all_dev,
                     smc2_stats* out);

/*
 * Fused iterations of several jobs (persistent multi-job filter kernels).  smc2_batch_step runs
 * one SMC^2 iteration of each of the n handles, exactly as smc2_step on each would (the same
 * results, bit for bit), but the particle-filter passes of handles that share a kernel variant
 * (model shape, particles per thread, register cap), a block size and an adjoint ring are fused
 * into one forward and one adjoint launch over all their filters: a persistent grid whose blocks
 * take (job, filter) items from a device counter, longest filters first, so jobs of different
 * T, N, parameters and data fill the GPU together (Table I: the filters of an iteration are the
 * O(N/P) work).  Each handle's proposal and update run on its own stream; a group's fused passes
 * run on the stream of its longest job, which first waits for the others' proposals, and their
 * streams wait for the passes.  A handle alone in its group, and an HMC move after the first
 * iteration (its leapfrog points need several filter passes), step as smc2_step does.
 * stats: [n] caller storage or NULL; the call synchronises every handle's stream.
 * smc2_batch_create allocates the device descriptors for up to max_jobs handles (1..4096) on the
 * current device; a batch serves one call at a time.  Errors: SMC2_E_INVAL (n outside
 * [0, max_jobs], NULL or repeated handles, a split step pending), SMC2_E_NOMEM, SMC2_E_CUDA,
 * SMC2_E_TIMEOUT as smc2_step.
 */
typedef struct smc2_batch smc2_batch;
int smc2_batch_create(int max_jobs, smc2_batch** out);
int smc2_batch_step(smc2_batch* b, smc2_handle* const* handles, int n, smc2_stats* stats);
int smc2_batch_destroy(smc2_batch* b);

/* Copy the current samples to host: theta_host [N][D] and logw_host [N] (either may be NULL). */
int smc2_get_samples(smc2_handle* h, double* theta_host, double* logw_host);

/* Copy per-sample log-likelihood estimates and gradients of the log posterior to host
 * (loglik_host [N], gradpi_host [N][D]; either may be NULL). */
int smc2_get_state(smc2_handle* h, double* loglik_host, double* gradpi_host);

/*
 * smc2_get_trace: decisions taken during the last particle-filter launch and the last
 * outer step, for verification: pf_anc [N][T][M] (ancestor of particle i before step
 * t, row t-1; rows of steps without resampling are unspecified), pf_flag [N][T]
 * (1 if the filter resampled before step t), outer_anc [N] (ancestor of each sample if
 * the last smc2_step resampled).  Any pointer may be NULL.  Host buffers.
 */
int smc2_get_trace(smc2_handle* h, uint16_t* pf_anc, uint8_t* pf_flag, int32_t* outer_anc,
                   int32_t* outer_resampled);

/*
 * smc2_get_nuts_trace: the decisions of each sample's NUTS move in the last smc2_step (host
 * buffers [N], any may be NULL), for verification.  Points are numbered s = 2^j - 1 + n (point
 * n of doubling j).  sel: bit s set where point s became its sub-trajectory's candidate;
 * merge: bit j set where doubling j's candidate replaced the selected point; stop_point and
 * stop_kind: where and why the trajectory stopped (kind 0: maximum depth, at the last point;
 * 1: U-turn inside a sub-trajectory; 2: divergent or non-finite point; 3: U-turn of the whole
 * trajectory, at the last point of a doubling; 4: not moved, stop_point -1, because the
 * sample's log pi or gradient is not finite).  SMC2_E_INVAL if the handle's proposal is not
 * SMC2_NUTS or no NUTS move ran yet.  Synchronises the handle's stream.
 */
int smc2_get_nuts_trace(smc2_handle* h, uint64_t* sel, uint32_t* merge, int32_t* stop_point,
                        int32_t* stop_kind);

/*
 * Per-point tapes, for verification of moves with several leapfrog points (HMC, NUTS).
 * smc2_set_point_trace(h, on): with on, every later iteration also keeps the ancestor tape and
 * resampling flags of the filter launch at each of its leapfrog points (device copies; the
 * first call allocates 2 bytes x points x N x T x M rounded up to 8, plus points x N x T bytes;
 * while on, iterations run without the captured graph).  smc2_get_point_trace(h, point, pf_anc,
 * pf_flag) copies point `point` (0-based, in launch order; NUTS: s = 2^j - 1 + n) of the last
 * iteration to host buffers laid out as smc2_get_trace's.  SMC2_E_INVAL if tracing was never on
 * or point is out of range; SMC2_E_NOMEM if the allocation fails.
 */
int smc2_set_point_trace(smc2_handle* h, int on);
int smc2_get_point_trace(smc2_handle* h, int point, uint16_t* pf_anc, uint8_t* pf_flag);

/*
 * pf_loglik_grad_static: pf_loglik_grad for callers that cannot allocate device memory
 * (for example code inside a framework that owns all device memory through its own
 * pool, latency-critical loops where cudaMalloc/cudaFree would synchronise the device,
 * or plug-ins that must not grow the device footprint after start-up).  The paper has
 * no counterpart; this is a deployment variant of the same computation.
 *
 * No handle and no allocation: cfg describes the model and sizes (model_family, d_x,
 * d_y, H (host, copied), y (DEVICE pointer, y_on_device must be 1), T, M, D,
 * pf_resample, ess_frac, seed, ckpt_every, particles_per_thread, stream); cfg->N is
 * ignored (the size checks use n) and n rows of theta_dev ([n][D] FP64, device, n <= 4096)
 * are filtered with Philox rows
 * row0..row0+n-1 and iteration iter.  Outputs as for pf_loglik_grad (loglik_dev [n],
 * grad_dev [n][D] or NULL), caller-owned device buffers.  Work is enqueued on
 * cfg->stream (NULL: the legacy default stream).
 *
 * Working memory (checkpoints, ancestor tape, per-step scalars, a copy of H) comes from
 * one static device array of 64 MiB that every GPU loading this library holds until the
 * process exits.  With ckpt_every = 0 the checkpoint interval is the smallest power of
 * two whose working set fits; a problem that does not fit even then is rejected with
 * SMC2_E_INVAL and a message giving the bytes it needs.  The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  All calls share the one array and it keeps the last
 * call's contents (each call clears the status word it uses; nothing else needs to start at
 * zero): calls whose work overlaps on
 * the GPU race with each other, so serialise them (one stream, or events).
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine.
 * Errors: SMC2_E_INVAL, SMC2_E_CUDA.  The call is asynchronous: a bounded wait that expires
 * inside its kernels is reported by pf_static_get_status afterwards (SMC2_E_TIMEOUT).
 */
int pf_loglik_grad_static(const smc2_config* cfg, const double* theta_dev, int n, uint32_t iter,
                          uint32_t row0, double* loglik_dev, double* grad_dev);

/* Status word of the last pf_loglik_grad_static call on the current device (it lives in the
 * same static array; each call clears it before its kernels run): 0, or kernel error bits
 * (1: a bounded wait inside a filter kernel expired, so that call's outputs are invalid and
 * the call should be treated as failed with SMC2_E_TIMEOUT).  Copies the word with
 * cudaMemcpyAsync on `stream` (the stream the call used; NULL: the legacy default stream) and
 * synchronises that stream; clear != 0 resets a nonzero word.  Allocates nothing.
 * Errors: SMC2_E_INVAL (status NULL), SMC2_E_CUDA. */
int pf_static_get_status(void* stream, int* status, int clear);

/* The cudaStream_t (as void*) on which the handle enqueues its work: cfg->stream, or the
 * handle's private stream.  Callers that mix the handle's work with work on other streams
 * (e.g. a framework's current stream) order the two with events on this stream. */
int smc2_get_stream(const smc2_handle* h, void** stream);

/* Read the handle's device status word (synchronises its stream): 0, or kernel error bits
 * (1: a bounded wait inside a filter kernel expired; that launch's results are invalid).
 * clear != 0 resets it.  smc2_step and pf_loglik_grad_host report a set status as
 * SMC2_E_TIMEOUT. */
int smc2_get_status(smc2_handle* h, int* status, int clear);

/* Failure detection without a fault: runs one block whose warps wait on a barrier that
 * nothing completes, with the filter kernels' bounded wait cut to `polls` polls; the wait
 * gives up, the block records the timeout in a device status word and finishes.  Sets
 * *timed_out to 1 when the status word says so.  The CUDA context stays usable.  No
 * counterpart in the paper.  Errors: SMC2_E_INVAL (polls < 1, NULL), SMC2_E_NOMEM,
 * SMC2_E_CUDA. */
int smc2_selftest_bounded_wait(int polls, int* timed_out);

/* The common random numbers of the filter kernels, for verification against an independent
 * implementation of the same generator (Philox4x32-10, Salmon et al., SC'11; Sec. I and
 * Sec. II-A use one fixed stream of numbers per sample and iteration).  For i = 0..n-1 (device
 * buffers): key_dev[i] = (seed_lo, seed_hi, iter, row) gives the kernels' key
 * (seed_lo ^ iter, seed_hi ^ row); ctr_dev[i] = the 4 counter words (the kernels use
 * (t, call, stream, 0)).  Writes words_dev[i][4] (the block's 4 output words), u_dev[i][4]
 * (the map to (0,1]: ((w >> 8) + 1) 2^-24) and z_dev[i][4] (Box-Muller normals of the word
 * pairs (0,1) and (2,3)); any output may be NULL.  Runs on `stream` (NULL: the legacy default
 * stream) and synchronises it.  No counterpart in the paper.  Errors: SMC2_E_INVAL, SMC2_E_CUDA. */
int smc2_selftest_crn(const uint32_t* ctr_dev, const uint32_t* key_dev, int n, uint32_t* words_dev, float* u_dev,
                      float* z_dev, void* stream);

/* Replace the observations (T x d_y FP32, host) of an existing handle; the copy is
 * stream-ordered on the handle's stream. */
int smc2_set_observations(smc2_handle* h, const float* y_host);

/* Bytes of device memory the handle holds (the footprint used for admission). */
int smc2_footprint(const smc2_config* cfg, size_t* bytes);

int smc2_destroy(smc2_handle* h);

/* Launch-configuration choice for a model shape (the autotuner): for the forward pass and
 * the adjoint separately, the particles-per-thread / register-cap variant, then the
 * checkpoint interval, each picked by timing the candidates with CUDA events on the
 * current device over a 64-step prefix of y, once per (device, family, d_x, d_y, M, N, T,
 * resampler), and cached in-process; later smc2_create calls with particles_per_thread = 0
 * and ckpt_every = 0 use it.  theta_host ([N][D] FP64, host) are the parameters to time
 * with (NULL: every row at the prior mean); representative values matter because the
 * resampling rate, and so the cost, depends on them.  Writes the forward pass's particles
 * per thread to *ppt and the checkpoint interval to *ckpt (either may be NULL). */
int smc2_autotune(const smc2_config* cfg, const double* theta_host, int* ppt, int* ckpt);

/* The launch choice of a handle: out[0..4] = forward particles per thread, forward
 * register cap, adjoint particles per thread, adjoint register cap, checkpoint interval. */
int smc2_get_launch(const smc2_handle* h, int* out);

/* Pin the launch choice for cfg's shape (the key smc2_autotune caches under: device,
 * family, d_x, d_y, M, N, T, resampling scheme), in the layout of smc2_get_launch, for
 * handles created afterwards.  No device work.  SMC2_E_INVAL if no compiled kernel variant
 * has those particles per thread and register cap for this shape, or the checkpoint
 * interval is outside [1, T]. */
int smc2_set_launch(const smc2_config* cfg, const int* launch);

/* Number of kernels this library launched since load (a device-work counter). */
uint64_t smc2_kernel_launches(void);

const char* smc2_last_error(void);

/* ---------------------------------------------------------------- serving */

typedef struct smc2_server smc2_server;

typedef struct smc2_result {
    int32_t status;            /* SMC2_OK or an error code of the job */
    int32_t K;                 /* iterations run */
    double latency_s;          /* submit -> completion wall time */
    double queue_s;            /* submit -> admission wall time */
    double* theta;             /* caller host storage [N][D] or NULL: final samples */
    double* logw;              /* caller host storage [N] or NULL: final log-weights */
    double* recycled_mean;     /* caller host storage [D] or NULL */
} smc2_result;

/*
 * smc2_server_create: a continuous-batching request loop on the current device.
 * Jobs are admitted while their footprint (smc2_footprint) fits hbm_budget bytes and
 * fewer than max_active jobs run; each admitted job keeps its state on the device and
 * advances one SMC^2 iteration at a time on its own stream, so iterations of
 * different jobs overlap on the GPU.  A worker thread drives the loop.
 */
int smc2_server_create(size_t hbm_budget, int max_active, smc2_server** out);

/* Fused batching on (default) or off: with it on, the jobs ready for their next iteration at the
 * same moment step together through smc2_batch_step (their filter passes fused into persistent
 * multi-job launches where they share a kernel variant and block size); off, every job steps on
 * its own stream.  Results are the same either way.  Errors: SMC2_E_INVAL. */
int smc2_server_set_fused(smc2_server* s, int on);

/* Queue a job (cfg and y are copied; cfg->K_iters iterations).  Returns immediately.
 * Admission (in arrival order) takes the job's own checkpoint interval when its footprint fits
 * the memory left; with ckpt_every = 0 it may instead take a longer interval whose footprint
 * fits (fewer stored steps, more recomputation: the job starts now instead of waiting).
 * SMC2_E_NOMEM only if the job can never fit the budget (at the longest interval). */
int smc2_submit(smc2_server* s, const smc2_config* cfg, uint64_t* job_id);

/* SMC2_PENDING while queued or running; SMC2_OK once finished (fills *out and
 * releases the job's result); SMC2_E_NOTFOUND for unknown ids. */
int smc2_poll(smc2_server* s, uint64_t job_id, smc2_result* out);

/* Drop a job that has not finished.  SMC2_E_NOTFOUND for unknown ids. */
int smc2_cancel(smc2_server* s, uint64_t job_id);

/* Stop the worker (running jobs are cancelled) and free everything. */
int smc2_server_destroy(smc2_server* s);

#ifdef __cplusplus
}
#endif

#endif /* SMC2_H */
