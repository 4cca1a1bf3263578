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
                cudaStream_t s, int speculative);
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

// ---------------------------------------------------------------------------------
// Metropolis chain steps with pre-fetching.  A chain at step s will either move to its
// proposal or stay; the proposal of step s+1 is base + L z[row s+1] for whichever base that
// decision leaves.  Evaluating the forward model for every node of the decision tree of depth
// k (2^(k+1) - 1 candidates) in one batched launch lets one launch resolve k + 1 chain steps
// exactly as the sequential chain would (the random inputs of each row are fixed in
// advance).  Node q of a tree: level l = floor(log2(q + 1)), decision bits b = q + 1 - 2^l,
// first decision most significant.  k = 0 is the plain one-step-per-launch chain.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ int node_level(int q) { return 31 - __clz(q + 1); }

__device__ __forceinline__ void add_step(const double *L, const double *z, const double *base, double *out) {
    out[0] = base[0] + L[0] * z[0] + L[1] * z[1] + L[2] * z[2];
    out[1] = base[1] + L[3] * z[0] + L[4] * z[1] + L[5] * z[2];
    out[2] = base[2] + L[6] * z[0] + L[7] * z[1] + L[8] * z[2];
}

struct Box {
    double lo[3], hi[3];
    __device__ bool in(const double *t) const {
        return t[0] >= lo[0] && t[0] <= hi[0] && t[1] >= lo[1] && t[1] <= hi[1] && t[2] >= lo[2] && t[2] <= hi[2];
    }
};

// candidates of all nodes: prop[(slot*NC + q)*3].  Unreachable nodes (an accepted decision on
// the path whose candidate lies outside the prior box), nodes beyond the chain's length and
// candidates outside the box get a NaN alpha, which the forward launch skips.
__global__ void spec_propose_kernel(int A, int s, int k, const int *__restrict__ order, const int *__restrict__ chain_off,
                                    const int *__restrict__ chain_len, const double *__restrict__ cur_theta,
                                    const double *__restrict__ st, const double *__restrict__ normals, Box box,
                                    double *__restrict__ prop, int *__restrict__ counter) {
    const int NC = (2 << k) - 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= A * NC) return;
    const int slot = idx / NC, q = idx % NC;
    const int c = order[slot];
    const int l = node_level(q), b = q + 1 - (1 << l);
    const int off = chain_off[c];
    const double *L = st + S_L;
    double base[3] = {cur_theta[3 * c], cur_theta[3 * c + 1], cur_theta[3 * c + 2]};
    bool ok = s + l < chain_len[c];
    double cand[3];
    for (int i = 0; i < l && ok; ++i) {
        add_step(L, normals + 3 * (off + s + i), base, cand);
        if ((b >> (l - 1 - i)) & 1) {
            if (!box.in(cand)) ok = false;  // that acceptance cannot happen
            base[0] = cand[0];
            base[1] = cand[1];
            base[2] = cand[2];
        }
    }
    add_step(L, normals + 3 * (off + s + l), base, cand);
    ok = ok && box.in(cand);
    prop[3 * idx] = ok ? cand[0] : nan("");
    prop[3 * idx + 1] = cand[1];
    prop[3 * idx + 2] = cand[2];
    if (ok) atomicAdd(counter, 1);
}

// surrogate log-likelihood of the base state of node (l, b): the candidate of the deepest
// accepted decision on the path, else the chain's current state
__device__ __forceinline__ double base_value(int slot, int NC, int l, int b, const double *node_val, double cur) {
    for (int i = l - 1; i >= 0; --i)
        if ((b >> (l - 1 - i)) & 1) {
            int qi = (1 << i) - 1 + (b >> (l - i));
            return node_val[slot * NC + qi];
        }
    return cur;
}

// delayed acceptance step 1 for every node: proposals failing the surrogate screen against
// their base are marked NaN (not run)
__global__ void spec_screen_kernel(int A, int s, int k, const int *__restrict__ order, const int *__restrict__ chain_off,
                                   const double *__restrict__ cur_sl, const double *__restrict__ prop_sl,
                                   const double *__restrict__ st, const double *__restrict__ u1, double *__restrict__ prop,
                                   int *__restrict__ counter) {
    const int NC = (2 << k) - 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= A * NC) return;
    const int slot = idx / NC, q = idx % NC;
    const int c = order[slot];
    const int l = node_level(q), b = q + 1 - (1 << l);
    const int pos = chain_off[c] + s + l;
    if (isnan(prop[3 * idx])) return;
    double bsl = base_value(slot, NC, l, b, prop_sl, cur_sl[c]);
    bool pass = log(u1[pos]) < st[S_QN] * (prop_sl[idx] - bsl);
    if (!pass) prop[3 * idx] = nan("");
    else atomicAdd(counter, 1);
}

// walk each chain's tree along the decisions it actually takes
__global__ void spec_resolve_kernel(int A, int s, int k, int delayed, const int *__restrict__ order,
                                    const int *__restrict__ chain_off, const int *__restrict__ chain_len,
                                    double *__restrict__ cur_theta, double *__restrict__ cur_ll,
                                    double *__restrict__ cur_sl, const double *__restrict__ prop,
                                    const double *__restrict__ prop_ll, const double *__restrict__ prop_sl,
                                    const int *__restrict__ prop_status, const double *__restrict__ st,
                                    const double *__restrict__ u_acc, double *__restrict__ out_theta,
                                    double *__restrict__ out_ll, double *__restrict__ out_sl, int *__restrict__ counter,
                                    const unsigned long long *__restrict__ run_work,
                                    unsigned long long *__restrict__ useful) {
    const int NC = (2 << k) - 1;
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= A) return;
    const int c = order[slot];
    const double qn = st[S_QN];
    int b = 0, acc = 0, ran = 0;
    unsigned long long work = 0;
    for (int l = 0; l <= k && s + l < chain_len[c]; ++l) {
        const int idx = slot * NC + (1 << l) - 1 + b;
        const int pos = chain_off[c] + s + l;
        bool run = !isnan(prop[3 * idx]);  // the one-step chain would have run this proposal
        ran += run;
        if (run) work += run_work[idx];
        bool valid = run && prop_status[idx] == SWIMMER_OK;
        double thr = qn * (prop_ll[idx] - cur_ll[c]);
        if (delayed) thr -= qn * (prop_sl[idx] - cur_sl[c]);
        bool accept = valid && log(u_acc[pos]) < thr;
        if (accept) {
            cur_theta[3 * c] = prop[3 * idx];
            cur_theta[3 * c + 1] = prop[3 * idx + 1];
            cur_theta[3 * c + 2] = prop[3 * idx + 2];
            cur_ll[c] = prop_ll[idx];
            if (delayed) cur_sl[c] = prop_sl[idx];
            ++acc;
        }
        out_theta[3 * pos] = cur_theta[3 * c];
        out_theta[3 * pos + 1] = cur_theta[3 * c + 1];
        out_theta[3 * pos + 2] = cur_theta[3 * c + 2];
        out_ll[pos] = cur_ll[c];
        out_sl[pos] = cur_sl[c];
        b = 2 * b + (accept ? 1 : 0);
    }
    if (acc) atomicAdd(counter, acc);
    if (ran) atomicAdd(counter + 3, ran);
    if (work) atomicAdd(useful, work);
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
    // counters: accepted, screen passes (runs with delayed acceptance), proposals run (plain),
    // runs on the realized chain paths
    CUDA_TRY(cudaMemsetAsync(h->info + cap, 0, 4 * sizeof(int), s));
    int n_screened = 0;
    Box box;
    for (int a = 0; a < 3; ++a) {
        box.lo[a] = st->prior_lo[a];
        box.hi[a] = st->prior_hi[a];
    }
    // pre-fetch depth: resolve several chain steps per launch while few chains are alive,
    // keeping each launch within about two samples per SM (and within b_max)
    const int spec_cap = min(h->cfg.b_max, 2 * h->num_sms);
    for (int step = 0; step < maxlen;) {
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
        int k = 0;
        while (k < 5 && step + k + 1 < maxlen && active * ((4 << k) - 1) <= spec_cap) ++k;
        const int NC = (2 << k) - 1, n = active * NC;
        const int grid = (n + 127) / 128;
        spec_propose_kernel<<<grid, 128, 0, s>>>(active, step, k, h->chain_id, h->chain_off, h->chain_len,
                                                 h->cur_theta, h->stats, normals, box, h->prop_theta,
                                                 h->info + cap + 2);
        CUDA_TRY(cudaGetLastError());
        prof_count(h, 2);
        if (use_surrogate) {
            int rc = run_surrogate_loglik(h, n, h->prop_theta, st->obs, st->sigma, h->prop_sl, s);
            if (rc) return rc;
            n_screened += n;
            spec_screen_kernel<<<grid, 128, 0, s>>>(active, step, k, h->chain_id, h->chain_off, h->cur_sl,
                                                    h->prop_sl, h->stats, uniforms + B, h->prop_theta,
                                                    h->info + cap + 1);
            CUDA_TRY(cudaGetLastError());
            prof_count(h, 1);
        }
        int rc = run_forward(h, n, h->prop_theta, nullptr, st->obs, st->sigma, h->prop_ll, nullptr, nullptr,
                             h->prop_status, s, 1);
        if (rc) return rc;
        spec_resolve_kernel<<<(active + 127) / 128, 128, 0, s>>>(
            active, step, k, use_surrogate, h->chain_id, h->chain_off, h->chain_len, h->cur_theta, h->cur_ll,
            h->cur_sl, h->prop_theta, h->prop_ll, h->prop_sl, h->prop_status, h->stats,
            uniforms + (use_surrogate ? 2 * B : B), h->out_theta, h->out_ll, h->out_sl, h->info + cap, h->run_work,
            h->work + 1);
        CUDA_TRY(cudaGetLastError());
        step += k + 1;
    }
    CUDA_TRY(cudaMemcpyAsync(st->theta, h->out_theta, 3 * sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(st->loglik, h->out_ll, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    if (use_surrogate)
        CUDA_TRY(cudaMemcpyAsync(st->surr_loglik, h->out_sl, sizeof(double) * B, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemsetAsync(st->status, 0, sizeof(int) * B, s));
    CUDA_TRY(cudaMemcpyAsync(h->host_pinned, h->info + cap, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
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
    st->n_exact = use_surrogate ? h->host_pinned[1] : h->host_pinned[2];
    st->n_exact_path = h->host_pinned[3];
    return 0;
}
