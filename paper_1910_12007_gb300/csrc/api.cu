// C-ABI entry points: handle lifetime, argument validation, forward model and likelihood.
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include <algorithm>

#include "common.cuh"

static thread_local char g_err[512] = "";

struct ProfileEvents {
    std::vector<cudaEvent_t> start, stop;
    std::vector<int> samples;
    size_t used = 0;
};

void prof_count(swimmer_handle *h, int launches) { h->n_launch += launches; }

void prof_k2_begin(swimmer_handle *h, cudaStream_t s, int samples) {
    if (!h->profile) return;
    ProfileEvents *p = h->prof;
    if (p->used == p->start.size()) {
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        p->start.push_back(a);
        p->stop.push_back(b);
        p->samples.push_back(0);
    }
    p->samples[p->used] = h->prof_rows > 0 ? h->prof_rows : samples;
    cudaEventRecord(p->start[p->used], s);
}

void prof_k2_end(swimmer_handle *h, cudaStream_t s) {
    if (!h->profile) return;
    ProfileEvents *p = h->prof;
    cudaEventRecord(p->stop[p->used], s);
    p->used += 1;
}

extern "C" int swimmer_profile_launches(swimmer_handle *h, int cap, double *ms, int *samples, int *count) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(cap >= 0, "cap must be >= 0");
    ARG_CHECK(cap == 0 || (ms != nullptr && samples != nullptr), "ms or samples is NULL");
    ARG_CHECK(count != nullptr, "count is NULL");
    ProfileEvents *p = h->prof;
    for (size_t i = 0; i < p->used && i < (size_t)cap; ++i) {
        CUDA_TRY(cudaEventSynchronize(p->stop[i]));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, p->start[i], p->stop[i]));
        ms[i] = t;
        samples[i] = p->samples[i];
    }
    *count = (int)p->used;
    return 0;
}

extern "C" int swimmer_profile(swimmer_handle *h, int mode, double *out) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(mode >= 0 && mode <= 2, "mode must be 0, 1 or 2");
    ProfileEvents *p = h->prof;
    if (mode == 2) {
        ARG_CHECK(out != nullptr, "out is NULL");
        double ms = 0.0, samples = 0.0;
        for (size_t i = 0; i < p->used; ++i) {
            CUDA_TRY(cudaEventSynchronize(p->stop[i]));
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, p->start[i], p->stop[i]));
            ms += t;
            samples += p->samples[i];
        }
        unsigned long long work[2] = {0, 0};
        CUDA_TRY(cudaMemcpy(work, h->work, sizeof(work), cudaMemcpyDeviceToHost));
        out[0] = ms;
        out[1] = (double)p->used;
        out[2] = (double)h->n_launch;
        out[3] = (double)work[0];
        out[4] = (double)work[1];
        p->used = 0;
        h->n_launch = 0;
        CUDA_TRY(cudaMemset(h->work, 0, sizeof(work)));
        return 0;
    }
    h->profile = mode;
    p->used = 0;
    h->n_launch = 0;
    CUDA_TRY(cudaDeviceSynchronize());
    CUDA_TRY(cudaMemset(h->work, 0, 2 * sizeof(unsigned long long)));
    return 0;
}

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

extern "C" const char *swimmer_last_error(void) { return g_err; }

static int check_config(const swimmer_config *c) {
    ARG_CHECK(c != nullptr, "config is NULL");
    ARG_CHECK(c->n_max >= 3 && c->n_max <= N_PTS_MAX, "n_max %d outside [3, %d]", c->n_max, N_PTS_MAX);
    ARG_CHECK(c->b_max >= 1 && c->b_max <= 65536, "b_max %d outside [1, 65536]", c->b_max);
    ARG_CHECK(c->ds_fixed > 0.0 || c->length > 0.0, "length must be > 0 (or ds_fixed > 0)");
    ARG_CHECK(c->mu > 0.0, "mu must be > 0");
    ARG_CHECK(c->delta_over_ds > 0.0, "delta_over_ds must be > 0");
    ARG_CHECK(c->dt > 0.0, "dt must be > 0");
    ARG_CHECK(c->k_t >= 0.0, "k_t must be >= 0");
    ARG_CHECK(c->steps >= 1 && c->steps < (1LL << 31) - 1, "steps must be in [1, 2^31 - 1)");
    ARG_CHECK(c->obs_every >= 1, "obs_every must be >= 1");
    ARG_CHECK(c->precision == SWIMMER_FP64 || c->precision == SWIMMER_FP32C, "precision must be 0 or 1");
    ARG_CHECK(c->n_head == 0 || (c->n_head >= 4 && c->n_head <= 256 && c->n_head % 2 == 0),
              "n_head must be 0 or even in [4, 256]");
    ARG_CHECK(c->n_head == 0 || c->n_max - c->n_head >= 3, "n_max must leave at least 3 flagellum points");
    ARG_CHECK(c->head_radius_over_ds >= 0.0 && c->neck_gap_over_ds >= 0.0, "head sizes must be >= 0");
    ARG_CHECK(c->k_head_tens >= 0.0 && c->k_head_c >= 0.0 && c->k_neck_tens >= 0.0 && c->k_neck_ang >= 0.0,
              "head and neck stiffnesses must be >= 0");
    ARG_CHECK(c->n_swimmers == 1 || (c->n_swimmers == 2 && c->n_head > 0), "n_swimmers must be 1, or 2 with a head");
    ARG_CHECK(c->n_swimmers == 1 || c->swimmer_distance > 0.0, "swimmer_distance must be > 0");
    ARG_CHECK(c->n_max - c->n_swimmers * c->n_head >= 3 * c->n_swimmers, "n_max too small for the swimmers");
    ARG_CHECK(c->sigma_ratio >= 0.0, "sigma_ratio must be >= 0");
    ARG_CHECK(c->n_params == 0 || c->n_params == 3 || c->n_params == 4, "n_params must be 0, 3 or 4");
    ARG_CHECK(c->obs_kind == SWIMMER_OBS_HEAD_POINT || (c->obs_kind == SWIMMER_OBS_HEAD_VELOCITY && c->n_head > 0) ||
                  (c->obs_kind == SWIMMER_OBS_PAIR_DISTANCES && c->n_swimmers == 2),
              "obs_kind must be HEAD_POINT, HEAD_VELOCITY with a head, or PAIR_DISTANCES with two swimmers");
    return 0;
}

#define ALLOC(ptr, count)                                                       \
    do {                                                                        \
        cudaError_t _e = cudaMalloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count)); \
        if (_e != cudaSuccess) {                                                \
            set_error("cudaMalloc of %s (%zu bytes) failed: %s", #ptr,           \
                      sizeof(*(ptr)) * (size_t)(count), cudaGetErrorString(_e)); \
            swimmer_destroy(h);                                                 \
            return SWIMMER_E_CUDA;                                              \
        }                                                                       \
    } while (0)

extern "C" int swimmer_init(const swimmer_config *cfg, swimmer_handle **out) {
    int rc = check_config(cfg);
    if (rc) return rc;
    ARG_CHECK(out != nullptr, "out is NULL");
    *out = nullptr;
    swimmer_handle *h = (swimmer_handle *)calloc(1, sizeof(swimmer_handle));
    ARG_CHECK(h != nullptr, "out of host memory");
    h->cfg = *cfg;
    h->prof = new ProfileEvents();
    CUDA_TRY(cudaGetDevice(&h->device));
    CUDA_TRY(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device));
    CUDA_TRY(cudaDeviceGetAttribute(&h->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device));
    CUDA_TRY(cudaDeviceGetAttribute(&h->regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, h->device));
    const int B = cfg->b_max;
    ALLOC(h->tab64, (size_t)B * TAB64_STRIDE);
    ALLOC(h->k1_scratch, (size_t)B * K1_SCRATCH);
    ALLOC(h->tab32, (size_t)B * TAB32_STRIDE);
    ALLOC(h->pq, (size_t)B * cfg->n_max);
    ALLOC(h->sp, B);
    ALLOC(h->order, B);
    ALLOC(h->queue, 4);
    ALLOC(h->speed_tmp, B);
    ALLOC(h->w, B);
    ALLOC(h->stats, 64);
    ALLOC(h->idx, B);
    ALLOC(h->counts, B);
    ALLOC(h->chain_id, B);
    ALLOC(h->chain_off, B);
    ALLOC(h->chain_len, B);
    ALLOC(h->aux, B + 64);
    ALLOC(h->cur_theta, P_MAX * B);
    ALLOC(h->cur_ll, B);
    ALLOC(h->cur_sl, B);
    ALLOC(h->prop_theta, P_MAX * B);
    ALLOC(h->prop_ll, B);
    ALLOC(h->prop_sl, B);
    ALLOC(h->out_theta, P_MAX * B);
    ALLOC(h->out_ll, B);
    ALLOC(h->out_sl, B);
    ALLOC(h->prop_status, B);
    ALLOC(h->live, B);
    ALLOC(h->chain_pos, B);
    ALLOC(h->tmpl, B);
    ALLOC(h->stage_q, 1);
    ALLOC(h->stage_summary, SWIMMER_STAGE_SUMMARY);
    ALLOC(h->surr_dstat, 3);
    ALLOC(h->surr_trust, 1);
    ALLOC(h->cum, B);
    ALLOC(h->info, 128);
    ALLOC(h->work, 2);
    CUDA_TRY(cudaMemset(h->work, 0, 2 * sizeof(unsigned long long)));
    ALLOC(h->run_work, B);
    ALLOC(h->surr_norm, 2 * SWIMMER_MLP_OUT);
    ALLOC(h->surr_params, SWIMMER_MLP_NPARAM);
    ALLOC(h->surr_x, (size_t)B * SWIMMER_MLP_IN);
    ALLOC(h->surr_y, (size_t)B * SWIMMER_MLP_OUT);
    {
        cudaError_t e1 = cudaMallocHost((void **)&h->host_pinned, (B + 128) * sizeof(int));
        cudaError_t e2 = cudaMallocHost((void **)&h->host_pinned_d, 64 * sizeof(double));
        cudaError_t e3 = cudaStreamCreateWithFlags(&h->side_stream, cudaStreamNonBlocking);
        cudaError_t e4 = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
        cudaError_t e5 = cudaStreamCreateWithFlags(&h->shape_stream, cudaStreamNonBlocking);
        if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess || e4 != cudaSuccess || e5 != cudaSuccess) {
            set_error("cudaMallocHost or cudaStreamCreate failed");
            swimmer_destroy(h);
            return SWIMMER_E_CUDA;
        }
    }
    rc = gl_init();
    if (!rc) rc = upload_pair_units(h);
    if (!rc) rc = tmcmc_templates_init(h);
    if (rc) {
        swimmer_destroy(h);
        return rc;
    }
    CUDA_TRY(cudaDeviceSynchronize());
    *out = h;
    return 0;
}

extern "C" int swimmer_destroy(swimmer_handle *h) {
    if (!h) return 0;
    cudaDeviceSynchronize();
    void *ptrs[] = {h->tab64, h->k1_scratch, h->tab32, h->pq, h->sp, h->order, h->queue, h->speed_tmp, h->w, h->stats,
                    h->idx, h->counts, h->chain_id, h->chain_off, h->chain_len, h->aux,
                    h->cur_theta, h->cur_ll, h->cur_sl, h->prop_theta, h->prop_ll, h->prop_sl,
                    h->out_theta, h->out_ll, h->out_sl, h->prop_status, h->live, h->chain_pos, h->tmpl,
                    h->tmpl_master, h->tmpl_map, h->p_accept_dev, h->stage_q, h->stage_summary, h->surr_dstat,
                    h->surr_trust, h->cum, h->info,
                    h->work, h->run_work,
                    h->surr_norm, h->surr_params, h->surr_x, h->surr_y, h->surr_ws, h->units};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (h->host_pinned) cudaFreeHost(h->host_pinned);
    if (h->host_pinned_d) cudaFreeHost(h->host_pinned_d);
    if (h->side_stream) cudaStreamDestroy(h->side_stream);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    if (h->shape_stream) cudaStreamDestroy(h->shape_stream);
    if (h->prof) {
        for (cudaEvent_t e : h->prof->start) cudaEventDestroy(e);
        for (cudaEvent_t e : h->prof->stop) cudaEventDestroy(e);
        delete h->prof;
    }
    free(h);
    return 0;
}

extern "C" int swimmer_kernel_eval(swimmer_handle *h, double alpha, double delta, double r_max, int m,
                                   const double *r, double *g1, double *g2, int precision, void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(m >= 0, "m must be >= 0");
    ARG_CHECK(m == 0 || (r && g1 && g2), "r, g1, g2 must be device pointers");
    ARG_CHECK(alpha >= 0.0 && delta > 0.0 && r_max > 0.0, "need alpha >= 0, delta > 0, r_max > 0");
    ARG_CHECK(r_max / delta < 4000.0, "r_max/delta beyond the table range");
    ARG_CHECK(alpha * r_max <= X_MAX, "alpha * r_max beyond %g", X_MAX);
    ARG_CHECK(precision == SWIMMER_FP64 || precision == SWIMMER_FP32C, "precision must be 0 or 1");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_set_sample(h, alpha, delta, r_max, s);
    if (!rc) rc = launch_table_build(h, 1, precision == SWIMMER_FP64 ? 2 : 3, s);
    if (!rc && m > 0) rc = launch_kernel_eval(h, m, r, g1, g2, precision, s);
    return rc;
}

static int check_batch(swimmer_handle *h, int B, const double *theta, const int *status) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B = %d outside [1, b_max = %d]", B, h ? h->cfg.b_max : 0);
    ARG_CHECK(theta != nullptr, "theta is NULL");
    ARG_CHECK(status != nullptr, "status is NULL");
    return 0;
}

int run_forward(swimmer_handle *h, int B, const double *theta, const int *n_pts, const double *obs,
                double sigma, double *loglik, double *head_traj, double *mean_speed, int *status,
                cudaStream_t s, int speculative, double *final_state, int threads_override) {
    int rc = launch_prepare(h, B, theta, n_pts, s);
    if (!rc) rc = launch_table_build(h, B, h->cfg.precision == SWIMMER_FP64, s);
    if (!rc)
        rc = launch_forward(h, B, obs, sigma, loglik, head_traj, mean_speed, status, h->cfg.precision, s,
                            threads_override, speculative, final_state);
    return rc;
}

// Autotuner: for batch sizes B = 1, 2, 4, ... up to b_max, time the forward kernel on
// `steps` Euler steps with every admissible threads-per-sample and keep the fastest.
extern "C" int swimmer_tuning(swimmer_handle *h, int precision, int *threads, int set) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(threads != nullptr, "threads is NULL");
    ARG_CHECK(precision == SWIMMER_FP64 || precision == SWIMMER_FP32C, "precision must be FP64 or FP32C");
    int *tab = h->tune_threads[precision == SWIMMER_FP64 ? 0 : 1];
    if (!set) {
        for (int k = 0; k < 17; ++k) threads[k] = tab[k];
        return 0;
    }
    for (int k = 0; k < 17; ++k) {
        const int t = threads[k] & SHAPE_THREADS;
        const int flags = threads[k] & ~SHAPE_THREADS;
        ARG_CHECK(flags == 0 || (precision != SWIMMER_FP64 && (flags == SHAPE_WIDE || flags == SHAPE_QUAD)),
                  "threads[%d] = %d: flags must be none, SWIMMER_SHAPE_WIDE or SWIMMER_SHAPE_QUAD (FP32C only)", k,
                  threads[k]);
        ARG_CHECK(threads[k] == 0 || (t >= forward_min_threads(h, precision) && t <= 1024 && (t & (t - 1)) == 0),
                  "threads[%d] = %d is not 0 or a power of two in [%d, 1024]", k, t, forward_min_threads(h, precision));
        ARG_CHECK(t == 0 || forward_fits(h, t, precision), "threads[%d] = %d needs more shared memory than the device has", k, t);
    }
    for (int k = 0; k < 17; ++k) tab[k] = threads[k];
    return 0;
}

extern "C" int swimmer_autotune(swimmer_handle *h, int steps, const double *theta_in, int n_theta,
                                int *out_threads) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(steps >= 1, "steps must be >= 1");
    ARG_CHECK(theta_in == nullptr || n_theta >= 1, "n_theta must be >= 1 with theta");
    const int bmax = h->cfg.b_max;
    double *theta = nullptr;
    int *status = nullptr;
    const int np = n_params(h->cfg);
    CUDA_TRY(cudaMalloc((void **)&theta, sizeof(double) * np * bmax));
    CUDA_TRY(cudaMalloc((void **)&status, sizeof(int) * bmax));
    if (theta_in) {
        // the caller's representative samples, repeated to b_max rows
        for (int off = 0; off < bmax; off += n_theta) {
            const int rows = std::min(n_theta, bmax - off);
            CUDA_TRY(cudaMemcpy(theta + np * off, theta_in, sizeof(double) * np * rows, cudaMemcpyDeviceToDevice));
        }
    } else {
        double *ht = (double *)malloc(sizeof(double) * np * bmax);
        for (int b = 0; b < bmax; ++b) {
            ht[np * b] = 1.0 + 0.001 * (b % 17);
            ht[np * b + 1] = 0.0;
            ht[np * b + 2] = 0.1;
            if (np == 4) ht[np * b + 3] = 1.0;
        }
        cudaMemcpy(theta, ht, sizeof(double) * np * bmax, cudaMemcpyHostToDevice);
        free(ht);
    }
    const long long saved_steps = h->cfg.steps, saved_obs = h->cfg.obs_every;
    h->cfg.steps = steps;
    h->cfg.obs_every = steps;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int rc = 0, k = 0;
    const int prec = h->cfg.precision;
    const int T0 = forward_min_threads(h, prec);
    // one batch per bucket: k + 1 samples per SM (the last one b_max)
    for (int per = 1; per <= 17 && !rc; ++per, ++k) {
        const int B = (int)std::min<long long>((long long)per * h->num_sms, bmax);
        rc = launch_prepare(h, B, theta, nullptr, 0);
        if (!rc) rc = launch_table_build(h, B, 1, 0);
        float best = 1e30f;
        int bestT = T0;
        for (int T = T0; T <= 1024 && !rc; T <<= 1) {
            if (!forward_fits(h, T, prec)) break;
            for (int mode = 0; mode <= (prec == SWIMMER_FP64 ? 0 : 2) && !rc; ++mode) {
                const int shape = T | (mode == 1 ? SHAPE_WIDE : mode == 2 ? SHAPE_QUAD : 0);
                float ms = 0.f;
                for (int rep = 0; rep < 2 && !rc; ++rep) {  // first run warms up
                    cudaEventRecord(e0, 0);
                    rc = launch_forward(h, B, nullptr, 0.0, nullptr, nullptr, nullptr, status, prec, 0, shape);
                    cudaEventRecord(e1, 0);
                    cudaEventSynchronize(e1);
                    cudaEventElapsedTime(&ms, e0, e1);
                }
                // a shape with more target blocks per unit has to win by 2 % (timing noise)
                if (mode == 0 ? ms < best : ms < 0.98f * best) {
                    best = ms;
                    bestT = shape;
                }
            }
        }
        h->tune_threads[prec == SWIMMER_FP64 ? 0 : 1][tune_bucket(h, B)] = bestT;
        if (out_threads) out_threads[k] = bestT;
        if (B == bmax) {
            ++k;
            break;
        }
    }
    // buckets beyond b_max keep the largest measured choice
    for (int j = tune_bucket(h, bmax) + 1; j < 17; ++j)
        h->tune_threads[prec == SWIMMER_FP64 ? 0 : 1][j] = h->tune_threads[prec == SWIMMER_FP64 ? 0 : 1][j - 1];
    for (int j = k; j < 17; ++j)
        if (out_threads) out_threads[j] = 0;
    h->cfg.steps = saved_steps;
    h->cfg.obs_every = saved_obs;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(theta);
    cudaFree(status);
    CUDA_TRY(cudaDeviceSynchronize());
    return rc;
}

extern "C" int forward_batch(swimmer_handle *h, int B, const double *theta, const int *n_pts,
                             double *head_traj, double *mean_speed, int *status, void *stream) {
    int rc = check_batch(h, B, theta, status);
    if (rc) return rc;
    return run_forward(h, B, theta, n_pts, nullptr, 0.0, nullptr, head_traj, mean_speed, status,
                       (cudaStream_t)stream, 0, nullptr, 0);
}

extern "C" int forward_batch_state(swimmer_handle *h, int B, const double *theta, const int *n_pts,
                                   double *head_traj, double *mean_speed, int *status, double *final_state,
                                   void *stream) {
    int rc = check_batch(h, B, theta, status);
    if (rc) return rc;
    ARG_CHECK(final_state != nullptr, "final_state is NULL");
    return run_forward(h, B, theta, n_pts, nullptr, 0.0, nullptr, head_traj, mean_speed, status,
                       (cudaStream_t)stream, 0, final_state, 0);
}

extern "C" int loglik_batch(swimmer_handle *h, int B, const double *theta, const int *n_pts,
                            const double *obs, double sigma, double *loglik, int *status, void *stream) {
    int rc = check_batch(h, B, theta, status);
    if (rc) return rc;
    ARG_CHECK(obs != nullptr, "obs is NULL");
    ARG_CHECK(loglik != nullptr, "loglik is NULL");
    ARG_CHECK(sigma > 0.0, "sigma must be > 0");
    ARG_CHECK(h->cfg.steps / h->cfg.obs_every >= 1, "no observation within steps");
    return run_forward(h, B, theta, n_pts, obs, sigma, loglik, nullptr, nullptr, status, (cudaStream_t)stream, 0,
                       nullptr, 0);
}
