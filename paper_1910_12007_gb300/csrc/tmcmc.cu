// K3/K4: transitional MCMC stage on the device (Sec. 3.2, Algorithm 1).
//
// K3 analyze (one CTA): l_max, then bisection on dq in (0, 1 - q_j] for COV(w) = 1 with
//   w_k = exp(dq (l_k - l_max)) (population standard deviation over mean, two-pass, FP64,
//   fixed-order block reductions), q_{j+1}, log S_j, w_bar, mu_j,
//   Sigma_j = b^2 sum w_bar (theta - mu)(theta - mu)^T (b = 0.2) and its Cholesky factor.
// K4 resample (one CTA): W_k = floor(w_k 2^40) (exact: w_k in [0, 1]), inclusive 64-bit
//   prefix C, t_k = min(floor(u_k C_B), C_B - 1), index_k = min{i : C_i > t_k} by binary
//   search; integer results are independent of summation order.
// Chains: the unique resampled indices in ascending order; chain c owns output rows
//   off_c .. off_c + n_c - 1 (off = exclusive prefix of the counts) and its step s uses
//   normals / uniforms of row off_c + s.  Chains are processed longest first so that the
//   chains alive at step s are a prefix of the list; each step is one batched forward
//   launch (K1 + K2) of the proposals, followed by the Metropolis accept with target
//   f_{j+1} (uniform box prior: proposals outside are rejected without a model run).
// Delayed acceptance (not in the paper): the surrogate screens proposals first (step 1
//   with min(1, exp(q (l~' - l~)))); only survivors run the forward model and face step 2
//   with min(1, exp(q (l' - l) - q (l~' - l~))).
#include <math.h>

#include "common.cuh"

int run_forward(swimmer_handle *h, int B, const double *theta, const int *n_pts, const double *obs,
                double sigma, double *loglik, double *head_traj, double *mean_speed, int *status,
                cudaStream_t s);
int run_surrogate_loglik(swimmer_handle *h, int B, const double *theta, const double *obs, double sigma,
                         double *loglik, cudaStream_t s);

namespace {

constexpr int T1 = 1024;
constexpr double B_SCALE = 0.2;
constexpr double COV_TARGET = 1.0;
constexpr double FIXED_SCALE = 1099511627776.0;  // 2^40

// stats layout
enum { S_DQ = 0, S_QN, S_LOGS, S_LMAX, S_MU, S_SIG = S_MU + 3, S_L = S_SIG + 9, S_STATUS = S_L + 9,
       S_U, S_MAXLEN, S_COUNT };

// fixed-order block sum of one double per thread (T1 threads); result to all threads
__device__ double block_sum(double v, double *red) {
    const int tid = threadIdx.x;
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (tid < 32) {
        t = red[tid];
        for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (tid == 0) red[32] = t;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double *red) {
    const int tid = threadIdx.x;
    for (int o = 16; o >= 1; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((tid & 31) == 0) red[tid >> 5] = v;
    __syncthreads();
    if (tid < 32) {
        double t = red[tid];
        for (int o = 16; o >= 1; o >>= 1) t = fmax(t, __shfl_xor_sync(0xffffffffu, t, o));
        if (tid == 0) red[32] = t;
    }
    __syncthreads();
    double r = red[32];
    __syncthreads();
    return r;
}

// COV of w(dq) with the two-pass population variance
__device__ double cov_of(int B, const double *__restrict__ ll, double lmax, double dq, double *red) {
    double s = 0.0;
    for (int k = threadIdx.x; k < B; k += T1) {
        double l = ll[k];
        s += isfinite(l) ? exp(dq * (l - lmax)) : 0.0;
    }
    double m = block_sum(s, red) / B;
    double v = 0.0;
    for (int k = threadIdx.x; k < B; k += T1) {
        double l = ll[k];
        double w = isfinite(l) ? exp(dq * (l - lmax)) : 0.0;
        v += (w - m) * (w - m);
    }
    double var = block_sum(v, red) / B;
    return sqrt(var) / m;
}

__global__ void __launch_bounds__(T1) analyze_kernel(int B, const double *__restrict__ theta,
                                                    const double *__restrict__ ll, double q,
                                                    double *__restrict__ w_out, double *__restrict__ st) {
    __shared__ double red[40];
    const int tid = threadIdx.x;
    double lm = -INFINITY;
    for (int k = tid; k < B; k += T1)
        if (isfinite(ll[k])) lm = fmax(lm, ll[k]);
    const double lmax = block_max(lm, red);
    if (!isfinite(lmax)) {
        if (tid == 0) st[S_STATUS] = 1.0;
        return;
    }
    double hi = 1.0 - q, dq;
    if (cov_of(B, ll, lmax, hi, red) <= COV_TARGET) {
        dq = hi;
    } else {
        double lo = 0.0;
        for (int it = 0; it < 200; ++it) {
            double mid = 0.5 * (lo + hi);
            if (cov_of(B, ll, lmax, mid, red) > COV_TARGET)
                hi = mid;
            else
                lo = mid;
            if (hi - lo < 1e-15) break;
        }
        dq = 0.5 * (lo + hi);
    }
    // weights and statistics
    double sw = 0.0;
    for (int k = tid; k < B; k += T1) {
        double l = ll[k];
        double w = isfinite(l) ? exp(dq * (l - lmax)) : 0.0;
        w_out[k] = w;
        sw += w;
    }
    const double W = block_sum(sw, red);
    double mu[3];
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int k = tid; k < B; k += T1) s += (w_out[k] / W) * theta[3 * k + a];
        mu[a] = block_sum(s, red);
    }
    double sig[6];
    const int ia[6] = {0, 1, 2, 1, 2, 2}, ib[6] = {0, 0, 0, 1, 1, 2};
    for (int e = 0; e < 6; ++e) {
        double s = 0.0;
        for (int k = tid; k < B; k += T1) {
            double wb = w_out[k] / W;
            s += wb * (theta[3 * k + ia[e]] - mu[ia[e]]) * (theta[3 * k + ib[e]] - mu[ib[e]]);
        }
        sig[e] = B_SCALE * B_SCALE * block_sum(s, red);
    }
    if (tid == 0) {
        st[S_DQ] = dq;
        st[S_QN] = (q + dq >= 1.0 - 1e-15) ? 1.0 : q + dq;
        st[S_LOGS] = dq * lmax + log(W / B);
        st[S_LMAX] = lmax;
        for (int a = 0; a < 3; ++a) st[S_MU + a] = mu[a];
        double S[3][3];
        for (int e = 0; e < 6; ++e) S[ia[e]][ib[e]] = S[ib[e]][ia[e]] = sig[e];
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) st[S_SIG + 3 * a + c] = S[a][c];
        // Cholesky S = L L^T
        double L[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
        int ok = 1;
        for (int a = 0; a < 3; ++a) {
            for (int c = 0; c <= a; ++c) {
                double s = S[a][c];
                for (int k = 0; k < c; ++k) s -= L[a][k] * L[c][k];
                if (a == c) {
                    if (!(s > 0.0)) ok = 0;
                    L[a][a] = sqrt(fmax(s, 0.0));
                } else {
                    L[a][c] = L[c][c] > 0.0 ? s / L[c][c] : 0.0;
                }
            }
        }
        for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c) st[S_L + 3 * a + c] = L[a][c];
        st[S_STATUS] = ok ? 0.0 : 2.0;
    }
}

// exclusive scan of one 64-bit value per thread (T1 threads), returns the exclusive prefix
// and writes the total to *total
__device__ unsigned long long block_exscan(unsigned long long v, unsigned long long *sm, unsigned long long *total) {
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sm[wid] = x;
    __syncthreads();
    if (wid == 0) {
        unsigned long long t = sm[lane];
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        sm[32 + lane] = t;  // inclusive over warps
    }
    __syncthreads();
    unsigned long long base = wid ? sm[32 + wid - 1] : 0ull;
    *total = sm[32 + 31];
    __syncthreads();
    return base + x - v;
}

__global__ void __launch_bounds__(T1) resample_kernel(int B, const double *__restrict__ w, const double *__restrict__ u,
                                                     unsigned long long *__restrict__ cum, int *__restrict__ idx,
                                                     int *__restrict__ counts) {
    __shared__ unsigned long long sm[64];
    const int tid = threadIdx.x;
    const int chunk = (B + T1 - 1) / T1;
    const int lo = tid * chunk, hi = min(B, lo + chunk);
    unsigned long long s = 0;
    for (int k = lo; k < hi; ++k) s += (unsigned long long)floor(w[k] * FIXED_SCALE);
    unsigned long long total;
    unsigned long long run = block_exscan(s, sm, &total);
    for (int k = lo; k < hi; ++k) {
        run += (unsigned long long)floor(w[k] * FIXED_SCALE);
        cum[k] = run;
    }
    for (int k = tid; k < B; k += T1) counts[k] = 0;
    __syncthreads();
    for (int k = tid; k < B; k += T1) {
        double tt = floor(u[k] * (double)total);
        unsigned long long t = (unsigned long long)tt;
        if (t > total - 1) t = total - 1;
        int a = 0, b = B - 1;  // first i with cum[i] > t
        while (a < b) {
            int m = (a + b) >> 1;
            if (cum[m] > t)
                b = m;
            else
                a = m + 1;
        }
        idx[k] = a;
        atomicAdd(&counts[a], 1);
    }
}

// chains: ids/offsets/lengths in ascending sample order, a longest-first processing order,
// per-step alive counts (host-visible) and the chains' starting states
__global__ void __launch_bounds__(T1) chains_kernel(int B, const int *__restrict__ counts,
                                                   const double *__restrict__ theta, const double *__restrict__ ll,
                                                   const double *__restrict__ sl, int *__restrict__ chain_off,
                                                   int *__restrict__ chain_len, int *__restrict__ order,
                                                   int *__restrict__ hist, double *__restrict__ cur_theta,
                                                   double *__restrict__ cur_ll, double *__restrict__ cur_sl,
                                                   int *__restrict__ host_info, int host_cap) {
    __shared__ unsigned long long sm[64];
    __shared__ int s_max;
    const int tid = threadIdx.x;
    const int chunk = (B + T1 - 1) / T1;
    const int lo = tid * chunk, hi = min(B, lo + chunk);
    // exclusive prefix of (count > 0) -> chain index; prefix of counts -> output offset
    unsigned long long nz = 0, cs = 0;
    for (int k = lo; k < hi; ++k) {
        nz += counts[k] > 0;
        cs += counts[k];
    }
    unsigned long long tot_u, tot_c;
    unsigned long long cidx = block_exscan(nz, sm, &tot_u);
    unsigned long long off = block_exscan(cs, sm, &tot_c);
    const int U = (int)tot_u;
    if (tid == 0) s_max = 0;
    for (int k = tid; k <= B; k += T1) hist[k] = 0;
    __syncthreads();
    // chain c -> sample index via chain_off/chain_len arrays indexed by chain number
    for (int k = lo; k < hi; ++k) {
        int n = counts[k];
        if (n > 0) {
            chain_off[cidx] = (int)off;
            chain_len[cidx] = n;
            cur_theta[3 * cidx + 0] = theta[3 * k + 0];
            cur_theta[3 * cidx + 1] = theta[3 * k + 1];
            cur_theta[3 * cidx + 2] = theta[3 * k + 2];
            cur_ll[cidx] = ll[k];
            cur_sl[cidx] = sl ? sl[k] : 0.0;
            atomicAdd(&hist[n], 1);
            atomicMax(&s_max, n);
            ++cidx;
        }
        off += n;
    }
    __syncthreads();
    const int maxlen = s_max;
    // alive(s) = #chains with length > s; bucket start for length n (longest first)
    if (tid == 0) {
        int acc = 0;
        for (int n = maxlen; n >= 1; --n) {
            int c = hist[n];
            hist[n] = acc;  // start position of length-n chains in the order
            acc += c;
        }
        host_info[0] = U;
        host_info[1] = maxlen;
    }
    __syncthreads();
    for (int c = tid; c < U; c += T1) {
        int pos = atomicAdd(&hist[chain_len[c]], 1);
        order[pos] = c;
    }
    __syncthreads();
    // alive counts for the host: alive(s) = start of the bucket of length s (exclusive)
    // i.e. number of chains with length >= s + 1 = hist_end(s+1)
    if (tid == 0) {
        for (int s = 0; s < host_cap - 2; ++s) host_info[2 + s] = 0;
    }
    __syncthreads();
    for (int c = tid; c < U; c += T1) {
        int n = chain_len[c];
        for (int s = 0; s < n && s < host_cap - 2; ++s) atomicAdd(&host_info[2 + s], 1);
    }
}

__global__ void propose_kernel(int active, int s, const int *__restrict__ order, const int *__restrict__ chain_off,
                               const double *__restrict__ cur_theta, const double *__restrict__ st,
                               const double *__restrict__ normals, double lo0, double lo1, double lo2, double hi0,
                               double hi1, double hi2, double *__restrict__ prop) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= active) return;
    int c = order[k];
    int pos = chain_off[c] + s;
    const double *L = st + S_L;
    double z0 = normals[3 * pos], z1 = normals[3 * pos + 1], z2 = normals[3 * pos + 2];
    double t0 = cur_theta[3 * c] + L[0] * z0 + L[1] * z1 + L[2] * z2;
    double t1 = cur_theta[3 * c + 1] + L[3] * z0 + L[4] * z1 + L[5] * z2;
    double t2 = cur_theta[3 * c + 2] + L[6] * z0 + L[7] * z1 + L[8] * z2;
    bool in = t0 >= lo0 && t0 <= hi0 && t1 >= lo1 && t1 <= hi1 && t2 >= lo2 && t2 <= hi2;
    // outside the prior box: NaN alpha makes the forward launch skip it (rejected)
    prop[3 * k] = in ? t0 : nan("");
    prop[3 * k + 1] = t1;
    prop[3 * k + 2] = t2;
}

// delayed acceptance step 1: keep proposals that pass the surrogate screen, mark others
__global__ void screen_kernel(int active, int s, const int *__restrict__ order, const int *__restrict__ chain_off,
                             const double *__restrict__ cur_sl, const double *__restrict__ prop_sl,
                             const double *__restrict__ st, const double *__restrict__ u1,
                             double *__restrict__ prop, int *__restrict__ counter) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= active) return;
    int c = order[k];
    int pos = chain_off[c] + s;
    double qn = st[S_QN];
    bool valid = !isnan(prop[3 * k]);
    bool pass = valid && log(u1[pos]) < qn * (prop_sl[k] - cur_sl[c]);
    if (!pass) prop[3 * k] = nan("");
    if (pass) atomicAdd(counter, 1);
}

__global__ void accept_kernel(int active, int s, int delayed, const int *__restrict__ order,
                              const int *__restrict__ chain_off, double *__restrict__ cur_theta,
                              double *__restrict__ cur_ll, double *__restrict__ cur_sl,
                              const double *__restrict__ prop, const double *__restrict__ prop_ll,
                              const double *__restrict__ prop_sl, const int *__restrict__ prop_status,
                              const double *__restrict__ st, const double *__restrict__ u_acc,
                              double *__restrict__ out_theta, double *__restrict__ out_ll,
                              double *__restrict__ out_sl, int *__restrict__ counter) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= active) return;
    int c = order[k];
    int pos = chain_off[c] + s;
    double qn = st[S_QN];
    bool valid = !isnan(prop[3 * k]) && prop_status[k] == SWIMMER_OK;
    double thr = qn * (prop_ll[k] - cur_ll[c]);
    if (delayed) thr -= qn * (prop_sl[k] - cur_sl[c]);
    if (valid && log(u_acc[pos]) < thr) {
        cur_theta[3 * c] = prop[3 * k];
        cur_theta[3 * c + 1] = prop[3 * k + 1];
        cur_theta[3 * c + 2] = prop[3 * k + 2];
        cur_ll[c] = prop_ll[k];
        if (delayed) cur_sl[c] = prop_sl[k];
        atomicAdd(counter, 1);
    }
    out_theta[3 * pos] = cur_theta[3 * c];
    out_theta[3 * pos + 1] = cur_theta[3 * c + 1];
    out_theta[3 * pos + 2] = cur_theta[3 * c + 2];
    out_ll[pos] = cur_ll[c];
    out_sl[pos] = cur_sl[c];
}

}  // namespace

extern "C" int tmcmc_analyze(swimmer_handle *h, int B, const double *theta, const double *loglik, double q,
                             double *out_w, double *stats, void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(theta && loglik && out_w && stats, "NULL device pointer");
    ARG_CHECK(q >= 0.0 && q < 1.0, "q must be in [0, 1)");
    analyze_kernel<<<1, T1, 0, (cudaStream_t)stream>>>(B, theta, loglik, q, out_w, stats);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

extern "C" int tmcmc_resample(swimmer_handle *h, int B, const double *w, const double *u, int *idx, int *counts,
                              void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(w && u && idx && counts, "NULL device pointer");
    resample_kernel<<<1, T1, 0, (cudaStream_t)stream>>>(B, w, u, (unsigned long long *)h->cum, idx, counts);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

extern "C" int tmcmc_stage(swimmer_handle *h, tmcmc_state *st, const double *uniforms, const double *normals,
                           int use_surrogate, void *stream) {
    ARG_CHECK(h != nullptr && st != nullptr, "NULL handle or state");
    const int B = st->B;
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(st->theta && st->loglik && st->status && st->obs, "NULL device pointer in the state");
    ARG_CHECK(uniforms && normals, "NULL uniforms/normals");
    ARG_CHECK(st->sigma > 0.0, "sigma must be > 0");
    ARG_CHECK(st->q >= 0.0 && st->q < 1.0, "stage already at q = 1");
    ARG_CHECK(!use_surrogate || (h->surr_ready && st->surr_loglik), "surrogate not set up");
    for (int a = 0; a < 3; ++a) ARG_CHECK(st->prior_lo[a] <= st->prior_hi[a], "prior box is empty");
    cudaStream_t s = (cudaStream_t)stream;
    const int cap = 64;
    analyze_kernel<<<1, T1, 0, s>>>(B, st->theta, st->loglik, st->q, h->w, h->stats);
    CUDA_TRY(cudaGetLastError());
    resample_kernel<<<1, T1, 0, s>>>(B, h->w, uniforms, (unsigned long long *)h->cum, h->idx, h->counts);
    CUDA_TRY(cudaGetLastError());
    const double *sl = use_surrogate ? st->surr_loglik : nullptr;
    chains_kernel<<<1, T1, 0, s>>>(B, h->counts, st->theta, st->loglik, sl, h->chain_off, h->chain_len,
                                   h->chain_id, h->aux, h->cur_theta, h->cur_ll, h->cur_sl, h->info, cap);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 3);
    CUDA_TRY(cudaMemcpyAsync(h->host_pinned, h->info, cap * sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(h->host_pinned_d, h->stats, 32 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    const double *hs = h->host_pinned_d;
    if (hs[S_STATUS] != 0.0) {
        set_error(hs[S_STATUS] == 1.0 ? "every sample has log-likelihood -inf" : "proposal covariance is not positive definite");
        return SWIMMER_E_STATE;
    }
    const int U = h->host_pinned[0], maxlen = h->host_pinned[1];
    int alive[64];
    for (int i = 0; i < cap - 2; ++i) alive[i] = h->host_pinned[2 + i];
    const double qn = hs[S_QN];
    CUDA_TRY(cudaMemsetAsync(h->info + cap, 0, 2 * sizeof(int), s));  // accept / screen counters
    int n_exact = 0, n_screened = 0;
    for (int step = 0; step < maxlen; ++step) {
        int active;
        if (step < cap - 2) {
            active = alive[step];
        } else {
            // rare: a chain longer than the host-visible table; count on the host
            CUDA_TRY(cudaMemcpyAsync(h->host_pinned, h->chain_len, sizeof(int) * U, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            active = 0;
            for (int c = 0; c < U; ++c) active += h->host_pinned[c] > step;
        }
        if (active <= 0) break;
        int grid = (active + 127) / 128;
        propose_kernel<<<grid, 128, 0, s>>>(active, step, h->chain_id, h->chain_off, h->cur_theta, h->stats, normals,
                                            st->prior_lo[0], st->prior_lo[1], st->prior_lo[2], st->prior_hi[0],
                                            st->prior_hi[1], st->prior_hi[2], h->prop_theta);
        CUDA_TRY(cudaGetLastError());
        prof_count(h, 2 + (use_surrogate ? 1 : 0));
        if (use_surrogate) {
            int rc = run_surrogate_loglik(h, active, h->prop_theta, st->obs, st->sigma, h->prop_sl, s);
            if (rc) return rc;
            n_screened += active;
            screen_kernel<<<grid, 128, 0, s>>>(active, step, h->chain_id, h->chain_off, h->cur_sl, h->prop_sl,
                                               h->stats, uniforms + B, h->prop_theta, h->info + cap + 1);
            CUDA_TRY(cudaGetLastError());
        }
        int rc = run_forward(h, active, h->prop_theta, nullptr, st->obs, st->sigma, h->prop_ll, nullptr, nullptr,
                             h->prop_status, s);
        if (rc) return rc;
        if (!use_surrogate) n_exact += active;
        accept_kernel<<<grid, 128, 0, s>>>(active, step, use_surrogate, h->chain_id, h->chain_off, h->cur_theta,
                                           h->cur_ll, h->cur_sl, h->prop_theta, h->prop_ll, h->prop_sl,
                                           h->prop_status, h->stats, uniforms + (use_surrogate ? 2 * B : B),
                                           h->out_theta, h->out_ll, h->out_sl, h->info + cap);
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(cudaMemcpyAsync(st->theta, h->out_theta, 3 * sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(st->loglik, h->out_ll, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    if (use_surrogate)
        CUDA_TRY(cudaMemcpyAsync(st->surr_loglik, h->out_sl, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemsetAsync(st->status, 0, sizeof(int) * B, s));
    CUDA_TRY(cudaMemcpyAsync(h->host_pinned, h->info + cap, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    st->q = qn;
    st->stage += 1;
    st->log_s = hs[S_LOGS];
    for (int a = 0; a < 3; ++a) st->mu[a] = hs[S_MU + a];
    for (int e = 0; e < 9; ++e) st->sigma_prop[e] = hs[S_SIG + e];
    st->unique = U;
    st->max_chain = maxlen;
    st->n_accept = h->host_pinned[0];
    st->n_screened = n_screened;
    st->n_exact = use_surrogate ? h->host_pinned[1] : n_exact;
    return 0;
}
