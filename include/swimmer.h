/*
 * swimmer.h -- C ABI of the GB300 (sm_103a) batched Brinkmanlet swimmer library.
 *
 * Method: Larson, Olson & Matzavinos, "Bayesian uncertainty quantification for
 * micro-swimmers with fully resolved hydrodynamics" (arXiv 1910.12007).
 *   - forward model g(theta|M): Sec. 2 (Eqs. eqnblob, BrV, Fenergy) and the Appendix
 *     (Eqs. EFB, curva, EFT; forward Euler);
 *   - Gaussian likelihood: Sec. 3.1, Eqs. (likelihood), (fitness);
 *   - TMCMC: Sec. 3.2, Algorithm 1.
 *
 * Conventions for every entry point
 *   - Return value: 0 on success, a negative SWIMMER_E* code otherwise.  Arguments are
 *     validated on the host before anything is launched; on error nothing is launched
 *     and no output is written.  swimmer_last_error() gives a message for the last
 *     failure on the calling thread.
 *   - Arrays are caller-owned DEVICE pointers unless stated otherwise ("host" below),
 *     row-major, FP64 unless stated.  The library never frees caller memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *     are asynchronous on that stream unless stated otherwise.
 *   - theta rows are (alpha, log10 K_C, a): Brinkman resistance, curvature stiffness,
 *     beat amplitude.  All other physical parameters come from swimmer_config.
 *   - Per-sample status codes: SWIMMER_OK, SWIMMER_DIVERGED (non-finite velocity, a
 *     point moving more than ds in one step, or a segment stretched beyond 20 %),
 *     SWIMMER_BAD_SAMPLE (parameters outside the supported range).  A sample that is not
 *     OK has log-likelihood -inf and NaN outputs.
 */
#ifndef SWIMMER_H
#define SWIMMER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    SWIMMER_OK = 0,
    SWIMMER_DIVERGED = 1,
    SWIMMER_BAD_SAMPLE = 2
};

enum {
    SWIMMER_E_ARG = -1,      /* invalid argument (NULL pointer, size out of range) */
    SWIMMER_E_CUDA = -2,     /* a CUDA runtime call failed */
    SWIMMER_E_CAPACITY = -3, /* batch larger than the handle's capacity */
    SWIMMER_E_STATE = -4     /* inconsistent TMCMC state (e.g. all samples diverged) */
};

enum { SWIMMER_FP64 = 0, SWIMMER_FP32C = 1 };

/* Launch-shape flags (FP32C only, at most one), OR-ed into a threads-per-sample value: the
 * pair sum takes two (WIDE) or four (QUAD) blocks of 32 targets per warp against one block of
 * sources, so each source load and shuffle serves two or four pair evaluations.  QUAD units
 * need 128 registers a thread: a launch whose shared memory allows more than 64K / 128
 * registers' worth of threads per SM runs WIDE units instead. */
#define SWIMMER_SHAPE_WIDE 0x10000
#define SWIMMER_SHAPE_QUAD 0x20000

/* Physical and numerical parameters (Table Tab:param fields).  POD, host memory. */
typedef struct swimmer_config {
    int n_max;              /* largest number of points per sample (3 .. 1024) */
    int b_max;              /* largest batch this handle serves (1 .. 65536) */
    double length;          /* flagellum length L when ds_fixed == 0 */
    double ds_fixed;        /* > 0: per-sample length = (n - 1) * ds_fixed (uneven N) */
    double mu;              /* viscosity */
    double delta_over_ds;   /* blob width delta in units of ds */
    double dt;              /* forward Euler step */
    double k_t;             /* tension stiffness K_T */
    double eta;             /* wavenumber */
    double omega;           /* angular frequency */
    long long steps;        /* time steps per forward run, 1 .. 2^31 - 2 */
    long long obs_every;    /* observation of the head point every obs_every steps */
    int precision;          /* SWIMMER_FP64 or SWIMMER_FP32C */
    /* Full sperm model (Appendix, Table Tab:param): a circular head of n_head points joined
     * to the flagellum's proximal point by five neck springs and a neck-angle energy.
     * n_head = 0 is the flagellum alone.  Points per sample = n (flagellum) + n_head <=
     * n_max; head and gap sizes in units of ds (0 selects n_head / (2 pi) and 1). */
    int n_head;             /* head points N_H: 0, or even in [4, 256] */
    double head_radius_over_ds;  /* H_r / ds */
    double neck_gap_over_ds;     /* dN / ds: initial gap between flagellum end and head */
    double k_head_tens;     /* K_{H,tens}: head membrane and diametral springs */
    double k_head_c;        /* K_{H,C}: head bending toward curvature 1/H_r */
    double k_neck_tens;     /* K_{N,tens}: the five neck springs */
    double k_neck_ang;      /* K_{N,ang}: neck angle energy K (z1 . z2)^2 */
    int obs_kind;           /* SWIMMER_OBS_HEAD_POINT: proximal flagellum point (x, y);
                               SWIMMER_OBS_HEAD_VELOCITY: head-centre velocity (x, y), the
                               centre's displacement over each observation interval / its
                               duration (n_head > 0);
                               SWIMMER_OBS_PAIR_DISTANCES: (distance between the tail tips,
                               distance between the head centres) of two swimmers */
    /* Two swimmers per sample (Sec. 4.2): the same swimmer twice, the second displaced by
     * swimmer_distance along y; the fluid couples them (one pair sum over all points).
     * Points per sample = n_swimmers (n + n_head) <= n_max. */
    int n_swimmers;         /* 1 or 2 (2 needs n_head > 0) */
    double swimmer_distance;  /* initial vertical separation d (length units) */
    double sigma_ratio;     /* noise of the second observed component / the first (sigma_h /
                               sigma_t for two swimmers); 0 means 1 */
    /* Unknowns per sample: 3 = theta (alpha, log10 K_C, a); 4 adds the noise level as an
     * unknown (Sec. 3.1, sigma/beta inferred): a sample's sigma is theta[3] times the sigma
     * passed to the likelihood calls.  theta rows have n_params entries in every call of
     * the handle.  0 means 3. */
    int n_params;
} swimmer_config;

enum { SWIMMER_OBS_HEAD_POINT = 0, SWIMMER_OBS_HEAD_VELOCITY = 1, SWIMMER_OBS_PAIR_DISTANCES = 2 };

typedef struct swimmer_handle swimmer_handle;

/* Create a handle on the current CUDA device: allocates the per-sample kernel tables,
 * the work queues and the TMCMC workspace for b_max samples (device memory owned by the
 * handle).  Synchronous.  *out receives the handle. */
int swimmer_init(const swimmer_config *cfg, swimmer_handle **out);

/* Free everything the handle owns.  Synchronizes the device first. */
int swimmer_destroy(swimmer_handle *h);

/* Message for the last error on the calling thread (static storage). */
const char *swimmer_last_error(void);

/* Opt-in profiling.  mode 1: time every forward-kernel (K2) launch with CUDA events
 * recorded on its stream and count all kernel launches of this handle; mode 0: stop;
 * mode 2: wait for the recorded events, write out[5] = {total K2 milliseconds, K2
 * launches, kernel launches, pair evaluations K2 executed (sum of n^2 x steps run, so
 * skipped and early-stopped samples count what they did), the part of those a
 * one-step-at-a-time TMCMC also performs (pre-fetched runs off the realized chain paths
 * excluded)} (host array) and reset.  Synchronous. */
int swimmer_profile(swimmer_handle *h, int mode, double *out);

/* The K2 launches recorded since profiling started or was last reset (mode 2 of
 * swimmer_profile), oldest first: ms[i] = device time of launch i (CUDA events),
 * samples[i] = its batch size, for i < min(cap, recorded); *count = recorded.  Host
 * arrays of cap entries (may be NULL when cap = 0).  Waits for the events; resets nothing.
 * Diagnostic only (not part of the method). */
int swimmer_profile_launches(swimmer_handle *h, int cap, double *ms, int *samples, int *count);

/* Kernel functions of the regularized Brinkmanlet (Sec. 2.1, Eq. BrV):
 * g1(r) = B''(r) and g2(r) = (r B''(r) - B'(r))/r^3 for (Lap - alpha^2) B = G, Lap G =
 * phi_delta (Eq. eqnblob), evaluated through the same per-sample table the forward
 * kernels use.  r[m], g1[m], g2[m]: device arrays; precision selects the FP64 (Chebyshev
 * degree 9) or the FP32 (quadratic, built the way FP32 handles build it) table.  For
 * testing the table build (step A1). */
int swimmer_kernel_eval(swimmer_handle *h, double alpha, double delta, double r_max, int m,
                        const double *r, double *g1, double *g2, int precision, void *stream);

/* Allocation-free variant of swimmer_kernel_eval, for callers that cannot allocate device
 * memory (for example services whose device-memory budget is fixed at start-up, or code that
 * must not grow the process's allocations per request).  No
 * handle: the table build of the one sample runs on scratch held in file-scope device
 * arrays (about 98 KB, kept by every GPU that loads the library until the process exits).
 * The paper has no counterpart; this is an interface convenience.
 *   - Same arguments and results as swimmer_kernel_eval; r, g1, g2 stay caller-owned.
 *   - Limit: r_max/delta < 4000 (24 octaves of u), alpha * r_max <= 600; larger sizes are
 *     rejected with SWIMMER_E_ARG and a message.
 *   - Allocates nothing (no cudaMalloc, cudaFree or allocating library routine).
 *   - The first call on a device does a one-time set-up on that device (device addresses of
 *     the arrays, constant tables, kernel attributes, loading of the kernels); later calls
 *     on that device only launch kernels.
 *   - Every call on a device shares the arrays, which keep the last call's contents; calls
 *     that overlap on the GPU (different streams, no ordering) race and give wrong results. */
int swimmer_kernel_eval_noalloc(double alpha, double delta, double r_max, int m, const double *r,
                                double *g1, double *g2, int precision, void *stream);

/* Batched forward model (Sec. 2; Appendix): for each sample b, B in 1..b_max,
 *   theta[b*3 + 0..2]   (alpha, log10 K_C, a),
 *   n_pts[b]            points (3..n_max) or n_pts == NULL for n_max everywhere,
 * runs cfg.steps forward Euler steps from the straight filament X_k = (k ds, 0) and writes
 *   head_traj[b][o][0..1]  head point (k = n-1) after every obs_every steps
 *                          (n_obs = steps / obs_every rows; may be NULL),
 *   mean_speed[b]          centroid x-displacement / (steps * dt)   (may be NULL),
 *   status[b]              per-sample status code (required).
 * One persistent launch for the whole batch (plus the table build). */
int forward_batch(swimmer_handle *h, int B, const double *theta, const int *n_pts,
                  double *head_traj, double *mean_speed, int *status, void *stream);

/* Autotuner for the forward kernel's launch shape.  The persistent kernel's time is set by
 * the number of samples each SM holds, so batch sizes fall into buckets k = 0..16 of
 * k + 1 samples per SM (ceil(B / SMs) - 1, capped at 16).  For each bucket up to b_max it
 * times the kernel on B = min((k + 1) SMs, b_max) samples (handle's precision, `steps` Euler
 * steps) with every admissible number of threads per sample (a
 * power of two from the smallest that covers n_max up to 1024 or the shared-memory limit;
 * the extra threads take more pair units in FP32 and split the source loop in FP64) and
 * stores the fastest in the handle (in FP32C each threads value is timed plain, with
 * SWIMMER_SHAPE_WIDE and with SWIMMER_SHAPE_QUAD; a flagged shape must be 2 % faster than the
 * best so far to be kept; the stored shape may carry a flag).  The samples are the caller's theta (device, [n_theta][3]
 * FP64, rows repeated as needed) when given: batches whose runs differ in length (runs that
 * diverge and stop early) favour shapes with fewer resident samples, whose work queue
 * rebalances the SMs.  With theta NULL, b_max copies of a mid-prior swimmer are timed.
 * out_threads (host array of 17, may be NULL) receives the choice per measured bucket, 0
 * after the last.  Synchronous; allocates and frees
 * temporary device memory; must not run during stream capture.  Untuned handles use a
 * heuristic. */
int swimmer_autotune(swimmer_handle *h, int steps, const double *theta, int n_theta, int *out_threads);

/* Read (set = 0) or replace (set = 1) the handle's launch-shape table for one precision
 * (SWIMMER_FP64 or SWIMMER_FP32C): threads[k] = threads per sample for batches holding
 * k + 1 samples per SM (ceil(B / SMs) = k + 1; k = 16 also takes larger batches), host
 * array of 17.  0 means "use the heuristic".  Set
 * entries must be 0 or a power of two from 32 to 1024 whose shared memory fits the
 * device, in FP32C optionally OR-ed with SWIMMER_SHAPE_WIDE or SWIMMER_SHAPE_QUAD, else
 * SWIMMER_E_ARG and nothing changes.  Lets a caller keep autotuned shapes
 * across handles or processes. */
int swimmer_tuning(swimmer_handle *h, int precision, int *threads, int set);

/* forward_batch that also returns each run's final state: final_state (device
 * [B][n_max][4] FP64) = (x, y, F_x, F_y) of every point at t = steps dt, the forces
 * recomputed there (Eq. Fenergy); rows past a sample's points and runs that stopped early are
 * NaN.  Points: flagellum 0..n-1, then the head, then the second swimmer's.  Used for the
 * flow field below.  Errors as forward_batch. */
int forward_batch_state(swimmer_handle *h, int B, const double *theta, const int *n_pts, double *head_traj,
                        double *mean_speed, int *status, double *final_state, void *stream);

/* Velocity and pressure at target points (Eqs. BrP, BrV with targets x away from the
 * swimmer): vel[g] = (1/mu) sum_j [-F_j g1(r) + (F_j . d) d g2(r)], pres[g] = sum_j (F_j . d)
 * G_delta'(r)/r, d = x_g - X_j, from the n points of state (device [n][4] (x, y, F_x, F_y),
 * e.g. one sample of forward_batch_state) for the kernel of (alpha, delta).  grid: device
 * [G][2]; vel: device [G][2]; pres: device [G] (either may be NULL, not both).  r_max bounds
 * every target-to-point distance (the FP64 table is built to it; farther distances are
 * clamped).  Builds the table in the handle's sample slot 0.  Asynchronous on stream;
 * SWIMMER_E_ARG on bad sizes or parameters (alpha r_max beyond the table's reach gives NaN). */
int swimmer_flow_field(swimmer_handle *h, double alpha, double delta, double r_max, int n, const double *state,
                       int G, const double *grid, double *vel, double *pres, void *stream);

/* Batched log-likelihood (Sec. 3.1, Eqs. likelihood/fitness with Sigma = sigma^2 I):
 *   loglik[b] = -(m/2) ln(2 pi sigma^2) - sum_o |D_o - head_o(theta_b)|^2 / (2 sigma^2),
 * m = 2 n_obs, obs = D [n_obs][2] on the device, shared by all samples.  The residuals
 * are accumulated in FP64 inside the forward kernel; no trajectory is stored. */
int loglik_batch(swimmer_handle *h, int B, const double *theta, const int *n_pts,
                 const double *obs, double sigma, double *loglik, int *status, void *stream);

/* ---------------------------------------------------------------------------------------
 * TMCMC (Sec. 3.2, Algorithm 1) on the device.
 * ------------------------------------------------------------------------------------- */
typedef struct tmcmc_state {
    int B;                 /* samples per stage (<= b_max) */
    double *theta;         /* device [B][P] current samples (updated in place), P = n_params */
    double *loglik;        /* device [B] their log-likelihoods (updated in place) */
    int *status;           /* device [B] */
    const int *n_pts;      /* ignored: every TMCMC sample uses n_max points */
    const double *obs;     /* device [n_obs][2] observations D */
    double sigma;          /* noise standard deviation (the scale beta when n_params = 4) */
    double prior_lo[4];    /* host: box-uniform prior bounds (first P used) */
    double prior_hi[4];
    double q;              /* host: annealing exponent q_j of the current samples */
    int stage;             /* host: stage index j */
    /* host outputs of the last stage */
    double log_s;          /* log S_j (evidence factor) */
    double mu[4];          /* weighted sample mean mu_j (first P) */
    double sigma_prop[16]; /* scaled covariance b^2 Sigma_j (P x P, row-major, row stride 4) */
    int unique;            /* number of distinct resampled samples (chains) */
    int max_chain;         /* longest chain */
    int n_exact;           /* forward-model runs executed this stage (pre-fetched runs included) */
    int n_screened;        /* surrogate evaluations this stage (delayed acceptance) */
    int n_accept;          /* accepted proposals this stage */
    int n_exact_path;      /* forward-model runs the chains used (what one-step-at-a-time needs) */
    double *surr_loglik;   /* device [B] surrogate log-likelihoods (delayed acceptance) */
    double log_evidence;   /* host: sum of log S_j over the stages run with this state, the
                              estimate of log p(D | M) once q = 1 (Sec. 3.2, model evidence;
                              start it at 0) */
    int surrogate_used;    /* host: 1 when the last stage screened proposals with the surrogate */
    double surrogate_error; /* host: the plain model's judgement of the surrogate in the last stage,
                               q_{j+1} sd(l - l~) in nats over the proposals both evaluated (NaN
                               without one); above 1 the next stage runs plain Metropolis */
} tmcmc_state;

/* Summary record of one stage (device FP64 array of SWIMMER_STAGE_SUMMARY entries written by
 * tmcmc_stage_async): status (0 ok; 1 every log-likelihood is -inf; 2 the proposal covariance
 * is not positive definite; a failed stage leaves the population unchanged), the exponent q_j
 * it started from and q_{j+1}, log S_j, mu_j [4], b^2 Sigma_j [4][4], the number of chains
 * (distinct resampled samples), the longest chain, accepted proposals, surrogate evaluations,
 * forward-model runs executed and those on the realized chain paths; with delayed acceptance,
 * whether this stage screened with the surrogate (1) and the plain model's judgement of the
 * surrogate: q_{j+1} times the spread (standard deviation) of l - l~ over the proposals both
 * evaluated, in nats (NaN without a judgement). */
enum {
    SWIMMER_STAGE_STATUS = 0,
    SWIMMER_STAGE_Q_IN = 1,
    SWIMMER_STAGE_Q = 2,
    SWIMMER_STAGE_LOG_S = 3,
    SWIMMER_STAGE_MU = 4,
    SWIMMER_STAGE_SIGMA = 8,
    SWIMMER_STAGE_UNIQUE = 24,
    SWIMMER_STAGE_MAX_CHAIN = 25,
    SWIMMER_STAGE_ACCEPT = 26,
    SWIMMER_STAGE_SCREENED = 27,
    SWIMMER_STAGE_EXACT = 28,
    SWIMMER_STAGE_EXACT_PATH = 29,
    SWIMMER_STAGE_SURR_USED = 30,
    SWIMMER_STAGE_SURR_ERR = 31,
    SWIMMER_STAGE_SUMMARY = 32
};

/* One TMCMC stage enqueued on `stream` without any host synchronization (Sec. 3.2,
 * Algorithm 1; the same stage as tmcmc_stage_shard, rank and world as there).  The state's
 * device arrays (theta, loglik, status, surr_loglik) and its sigma, obs and prior box are
 * used; its host fields are neither read nor written.  Instead:
 *   q       device FP64 scalar, in/out: the annealing exponent q_j of the current samples,
 *           replaced by q_{j+1} when the stage succeeds (a stage enqueued at q = 1 runs
 *           another Metropolis pass at the posterior);
 *   summary device FP64 [SWIMMER_STAGE_SUMMARY]: the stage's summary record (above).
 * The Metropolis chains' pre-fetch rounds run as a loop whose condition the device sets, so a
 * stage's length needs no host decision; each round's forward launch takes the launch shape
 * and CTAs per SM of the rows that run in it (a conditional switch node, set on the device,
 * with one branch per bucket of runs per SM).  When `stream` is being captured into a CUDA graph
 * the stage becomes part of that graph (a conditional while node holds the rounds) and every
 * replay runs a whole stage; otherwise the stage builds, launches and releases a graph of its
 * own.  Uses the handle's internal streams for the capture: one stage of a handle at a time. */
int tmcmc_stage_async(swimmer_handle *h, const tmcmc_state *st, const double *uniforms, const double *normals,
                      int use_surrogate, int rank, int world, double *q, double *summary, void *stream);

/* One TMCMC stage: analyze (q_{j+1} by bisection on COV(w) = 1, w_bar, S_j, mu_j,
 * Sigma_j = b^2 sum w_bar (theta - mu)(theta - mu)^T, b = 0.2), multinomial resample
 * (64-bit fixed-point inverse CDF), and the Metropolis chains of length n_{j+1,k} with
 * target f_{j+1} and Gaussian proposal N(theta, Sigma_j).
 *   uniforms: device [3][B]: row 0 resampling, row 1 acceptance, row 2 second-step
 *             acceptance (delayed acceptance only);
 *   normals:  device [B][3] proposal normals (chain c, step s uses row off_c + s).
 *   use_surrogate: 1 = delayed acceptance through the surrogate set with
 *             swimmer_surrogate_set (requires st->surr_loglik), 0 = plain.  The plain model
 *             judges the surrogate on every proposal both evaluate: a stage screens only while
 *             the previous one found q_{j+1} sd(l - l~) <= 1 nat (the first stage, from
 *             q_j = 0, and a surrogate set anew are trusted); otherwise it runs plain Metropolis with row 1's uniforms, still
 *             evaluating the surrogate so that it can be trusted again.
 * Each launch pre-fetches the forward runs of the live chains' next steps along a best-first
 * tree of pending accept decisions, so several chain steps resolve per launch with results
 * identical to the one-step-at-a-time chain.  Runs tmcmc_stage_async and synchronizes
 * `stream` once, at the end, to fill the state's host fields (q, stage, log_s,
 * log_evidence, mu, sigma_prop and the counters). */
int tmcmc_stage(swimmer_handle *h, tmcmc_state *st, const double *uniforms, const double *normals,
                int use_surrogate, void *stream);

/* tmcmc_stage for one of `world` processes that share one population (one GPU each).
 * Every rank passes the same state and random numbers and runs the same analysis and
 * resampling; rank `rank` then runs only the Metropolis chains whose output rows lie in its
 * block: chain c (chains in ascending sample order, output rows off_c .. off_c + len_c - 1)
 * belongs to rank floor((2 off_c + len_c) world / (2 B)).  On return st->theta, st->loglik
 * (and st->surr_loglik) hold this rank's rows and zeros elsewhere, so a SUM all-reduce over
 * the ranks assembles the population (the caller's one exchange per stage); the counters
 * n_accept, n_exact, n_screened and n_exact_path count this rank's work.  world = 1 is
 * tmcmc_stage.  Errors as tmcmc_stage, plus SWIMMER_E_ARG for rank outside [0, world). */
int tmcmc_stage_shard(swimmer_handle *h, tmcmc_state *st, const double *uniforms, const double *normals,
                      int use_surrogate, int rank, int world, void *stream);

/* The decision tree tmcmc_stage pre-fetches for each live chain (host only, no device
 * work): the root plus M - 1 nodes chosen best-first by the probability that a chain
 * accepting each proposal with probability p_accept follows the path to them, depth below
 * depth_cap (1..31).  nodes (host, 4 M ints): per node {parent (-1 for the root),
 * 2 depth + (1 if it is its parent's accept child), accept child, reject child} (-1 when
 * absent); *count = nodes built (fewer than M when the depth cap runs out). */
int tmcmc_tree_template(int M, double p_accept, int depth_cap, int *nodes, int *count);

/* The FP32 pair sum's work list for a sample of nb blocks of 32 points (host only, no
 * device work; 1 <= nb <= 32).  Each unordered pair of points is evaluated once (Eq. BrV is
 * even in the separation, so one kernel lookup serves both points).  A unit is 16 steps of
 * a warp: lane l holds target I*32 + l (and I2*32 + l, ... in a multi-target unit) and at
 * step d = d0 .. d0 + 15 meets source J*32 + (l + d) mod 32.  Packing (5-bit fields):
 * I | J << 5 | I2 << 10 | I3 << 15 | I4 << 20 | code << 25 | kind << 27, code 0: d0 = 0,
 * 1: d0 = 16, 2: a diagonal unit (I = J, d = 1 .. 16, lanes < 16 only at d = 16); kind 0, 1,
 * 2: 1, 2 or 4 target blocks.  An off-diagonal block pair is two units (d0 = 0, 16).
 * mode 0: nb diagonal units, then every block pair {I, J} as one-target units in circulant
 * order.  mode 1 (2): block pairs grouped two (four) at a time around a shared source block
 * J, the rest as pairs, at most one left as a one-target pair, then the diagonal units; below
 * 8 blocks mode 2 gives the mode 1 list.
 * out: host, at least nb^2 unsigned; *count = units written.  SWIMMER_E_ARG on bad
 * arguments. */
int swimmer_pair_units(int nb, int mode, unsigned *out, int *count);

/* Stage pieces, exposed for testing (Algorithm 1 'Analyze' and 'Resample'):
 * tmcmc_analyze: from loglik[B] (device), theta[B][P] (device, P = n_params) and q (host)
 *   compute on the device: out_w[B] = exp(dq (l - l_max)) (0 for -inf), and stats[64]
 *   (device FP64) = {dq, q_next, log_S, l_max, mu[4], Sigma[4][4], L[4][4] (lower Cholesky
 *   factor of Sigma; the first P rows and columns used), status (0 ok, 1 every
 *   log-likelihood is -inf, 2 Sigma not positive definite), ...}.
 * tmcmc_resample: idx[B] (device int) = min{i : C_i > floor(u_k C_B)}, C = inclusive
 *   prefix of floor(w_i 2^40); also counts[B] (device int).  Integer results are exact. */
int tmcmc_analyze(swimmer_handle *h, int B, const double *theta, const double *loglik, double q,
                  double *out_w, double *stats, void *stream);
int tmcmc_resample(swimmer_handle *h, int B, const double *w, const double *u, int *idx,
                   int *counts, void *stream);

/* ---------------------------------------------------------------------------------------
 * Learned surrogate (not in the paper): MLP 5 -> 256 -> 256 -> 256 -> 80, GELU, BF16
 * weights with FP32 accumulation; inputs are normalized (alpha, log10 K_C, a, log10 K_T,
 * omega), outputs normalized head positions at 40 times.
 * ------------------------------------------------------------------------------------- */
#define SWIMMER_MLP_IN 5
#define SWIMMER_MLP_HIDDEN 256
#define SWIMMER_MLP_OUT 80
#define SWIMMER_MLP_NPARAM (5 * 256 + 256 + 256 * 256 + 256 + 256 * 256 + 256 + 256 * 80 + 80)

/* Bytes of device workspace mlp_forward / mlp_backward need for a batch of n samples
 * (hidden pre-activations and activations, outputs and their gradients). */
size_t mlp_workspace_bytes(int n);

/* Forward pass: x[n][5] (device FP32) -> y[n][80] (device FP32).  params (device FP32
 * master copy, NPARAM floats, layout W1,b1,W2,b2,W3,b3,W4,b4 with W[out][in]).  Weights are
 * rounded to BF16 as they enter a product and every product accumulates in FP32; the three
 * 256-wide layers run on the tensor cores, with their activations (and, in mlp_backward,
 * the output gradients) rounded to BF16 as they enter, while the first layer keeps its 5
 * inputs in FP32.  workspace: device buffer of mlp_workspace_bytes(n) bytes, owned by the
 * caller. */
int mlp_forward(int n, const float *params, const float *x, float *y, float *workspace, void *stream);

/* Loss and gradient: loss_out[0] = mean over n x 80 of (y - t)^2 and grad[NPARAM] = its
 * gradient with respect to params (the forward above differentiated with its rounded
 * factors, the rounding taken as the identity), both device FP32 and overwritten.
 * Deterministic (no atomics). */
int mlp_backward(int n, const float *params, const float *x, const float *t, float *grad,
                 float *loss_out, float *workspace, void *stream);

/* Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected; step counts from 1) in place
 * on the FP32 master params with moments m, v (device FP32, NPARAM each). */
int mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, void *stream);

/* Surrogate log-likelihood for delayed acceptance: attaches trained parameters and the
 * normalization (host arrays: in_lo[5], in_hi[5] map inputs to [-1,1]; out_mean[80],
 * out_std[80]) to the handle, plus the observation subsampling (obs_stride: surrogate
 * output o corresponds to observation row o * obs_stride + obs_stride - 1).  The handle
 * copies everything; params is a device pointer. */
int swimmer_surrogate_set(swimmer_handle *h, const float *params, const double *in_lo,
                          const double *in_hi, const double *out_mean, const double *out_std,
                          int obs_stride, double log10_kt, double omega);

/* Surrogate log-likelihood of B samples against obs/sigma (device arrays as in
 * loglik_batch; uses the 40 subsampled observation rows and rescales J by the ratio of
 * observation counts). */
int surrogate_loglik_batch(swimmer_handle *h, int B, const double *theta, const double *obs,
                           double sigma, double *loglik, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SWIMMER_H */
