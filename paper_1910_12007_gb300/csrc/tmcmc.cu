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

#include <algorithm>
#include <vector>

#include "common.cuh"

int run_forward(swimmer_handle *h, int B, const double *theta, const int *n_pts, const double *obs,
                double sigma, double *loglik, double *head_traj, double *mean_speed, int *status,
                cudaStream_t s, int speculative, double *final_state, int threads_override);
int run_surrogate_loglik(swimmer_handle *h, int B, const double *theta, const double *obs, double sigma,
                         double *loglik, cudaStream_t s);

namespace {

constexpr int T1 = 1024;

// a host value into device memory, in stream order (no host buffer to race on)
__global__ void set_double_kernel(double *dst, double v) { dst[0] = v; }

constexpr double B_SCALE = 0.2;
constexpr double COV_TARGET = 1.0;
constexpr double FIXED_SCALE = 1099511627776.0;  // 2^40

// stats layout
// (P <= P_MAX unknowns: mean [P_MAX], covariance and its Cholesky factor [P_MAX][P_MAX], row-major
// with row stride P_MAX)
enum { S_DQ = 0, S_QN, S_LOGS, S_LMAX, S_MU, S_SIG = S_MU + P_MAX, S_L = S_SIG + P_MAX * P_MAX,
       S_STATUS = S_L + P_MAX * P_MAX, S_U, S_MAXLEN, S_COUNT };

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

__global__ void __launch_bounds__(T1) analyze_kernel(int B, int P, const double *__restrict__ theta,
                                                    const double *__restrict__ ll, const double *__restrict__ q_in,
                                                    double *__restrict__ w_out, double *__restrict__ st,
                                                    int *__restrict__ trust) {
    __shared__ double red[40];
    const int tid = threadIdx.x;
    const double q = q_in[0];
    // a run from the prior (q = 0) trusts the surrogate anew: no earlier stage has judged it
    if (trust && tid == 0 && q == 0.0) trust[0] = 1;
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
    double mu[P_MAX] = {0, 0, 0, 0};
    for (int a = 0; a < P; ++a) {
        double s = 0.0;
        for (int k = tid; k < B; k += T1) s += (w_out[k] / W) * theta[P * k + a];
        mu[a] = block_sum(s, red);
    }
    // lower triangle of the weighted covariance, b^2 scaled
    double S[P_MAX][P_MAX];
    for (int a = 0; a < P; ++a)
        for (int c = 0; c <= a; ++c) {
            double s = 0.0;
            for (int k = tid; k < B; k += T1) {
                double wb = w_out[k] / W;
                s += wb * (theta[P * k + a] - mu[a]) * (theta[P * k + c] - mu[c]);
            }
            S[a][c] = S[c][a] = B_SCALE * B_SCALE * block_sum(s, red);
        }
    if (tid == 0) {
        st[S_DQ] = dq;
        st[S_QN] = (q + dq >= 1.0 - 1e-15) ? 1.0 : q + dq;
        st[S_LOGS] = dq * lmax + log(W / B);
        st[S_LMAX] = lmax;
        for (int a = 0; a < P_MAX; ++a) st[S_MU + a] = a < P ? mu[a] : 0.0;
        for (int a = 0; a < P_MAX; ++a)
            for (int c = 0; c < P_MAX; ++c) st[S_SIG + P_MAX * a + c] = a < P && c < P ? S[a][c] : 0.0;
        // Cholesky S = L L^T
        double L[P_MAX][P_MAX];
        for (int a = 0; a < P_MAX; ++a)
            for (int c = 0; c < P_MAX; ++c) L[a][c] = 0.0;
        int ok = 1;
        for (int a = 0; a < P; ++a) {
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
        for (int a = 0; a < P_MAX; ++a)
            for (int c = 0; c < P_MAX; ++c) st[S_L + P_MAX * a + c] = L[a][c];
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
__global__ void __launch_bounds__(T1) chains_kernel(int B, int P, const double *__restrict__ st,
                                                   const int *__restrict__ counts,
                                                   const double *__restrict__ theta, const double *__restrict__ ll,
                                                   const double *__restrict__ sl, int *__restrict__ chain_off,
                                                   int *__restrict__ chain_len, int *__restrict__ order,
                                                   int *__restrict__ hist, double *__restrict__ cur_theta,
                                                   double *__restrict__ cur_ll, double *__restrict__ cur_sl,
                                                   int *__restrict__ host_info, int host_cap) {
    __shared__ unsigned long long sm[64];
    __shared__ int s_max;
    const int tid = threadIdx.x;
    if (st[S_STATUS] != 0.0) {  // the analysis failed: no chains, the stage changes nothing
        if (tid == 0) {
            host_info[0] = 0;
            host_info[1] = 0;
        }
        return;
    }
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
            for (int a = 0; a < P; ++a) cur_theta[P * cidx + a] = theta[P * k + a];
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
// Metropolis chain steps with pre-fetching.  A chain at step s either moves to its proposal
// or stays; the proposal of step s+1 is base + L z[row s+1] for whichever base that decision
// leaves.  Evaluating the forward model for several nodes of this decision tree in one
// batched launch lets one launch resolve several chain steps exactly as the sequential
// chain would (the random inputs of every row are fixed in advance).  The host picks the
// nodes: a template tree shared by all live chains, grown best-first by the probability
// that the chain's actual path reaches a node (acceptance rate estimated from the stage so
// far).  Template node v: x = parent (-1 for the root), y = 2 depth + (1 if v is the
// parent's accept child), z = accept child, w = reject child (-1 when absent).  Chains
// advance by different numbers of steps; chain_pos holds each chain's progress.
// ---------------------------------------------------------------------------------
constexpr int TREE_DEPTH_MAX = 31;

// proposal base + L z (L lower triangular, row stride P_MAX), summed left to right
__device__ __forceinline__ void add_step(int P, const double *L, const double *z, const double *base, double *out) {
    for (int a = 0; a < P; ++a) {
        double v = base[a];
        for (int c = 0; c < P; ++c) v += L[P_MAX * a + c] * z[c];
        out[a] = v;
    }
}

struct Box {
    int P;
    double lo[P_MAX], hi[P_MAX];
    __device__ bool in(const double *t) const {
        bool ok = true;
        for (int a = 0; a < P; ++a) ok = ok && t[a] >= lo[a] && t[a] <= hi[a];
        return ok;
    }
};

// path of template node v from the root: path[0] = root, path[depth] = v
__device__ __forceinline__ int tree_path(const int4 *__restrict__ tmpl, int v, int *path) {
    const int depth = tmpl[v].y >> 1;
    for (int d = depth, u = v; d >= 0; --d) {
        path[d] = u;
        u = tmpl[u].x;
    }
    return depth;
}

// Chain c belongs to rank floor((2 off_c + len_c) world / (2 B)): the ranks own contiguous
// blocks of output positions (chains in ascending sample order), balanced by chain length.
__device__ __forceinline__ bool chain_owned(int off, int len, int B, int rank, int world) {
    return world == 1 || (int)(((2ll * off + len) * world) / (2ll * B)) == rank;
}

// live chains of this rank (chain_pos < chain_len) in the longest-first order, their
// number, the largest remaining length, and the rank's accepted / decided steps so far
__global__ void __launch_bounds__(T1) live_kernel(const int *__restrict__ U_in, int B, int rank, int world,
                                                  const int *__restrict__ order, const int *__restrict__ chain_off,
                                                  const int *__restrict__ chain_len, const int *__restrict__ chain_pos,
                                                  int *__restrict__ live, const int *__restrict__ counter,
                                                  int *__restrict__ host_info, cudaGraphConditionalHandle cond,
                                                  int use_cond) {
    __shared__ unsigned long long sm[64];
    __shared__ int s_rem, s_dec;
    const int tid = threadIdx.x;
    const int U = U_in[0];
    if (tid == 0) {
        s_rem = 0;
        s_dec = 0;
    }
    const int chunk = (U + T1 - 1) / T1;
    const int lo = min(U, tid * chunk), hi = min(U, lo + chunk);
    unsigned long long cnt = 0;
    int rem = 0, dec = 0;
    for (int i = lo; i < hi; ++i) {
        const int c = order[i];
        if (!chain_owned(chain_off[c], chain_len[c], B, rank, world)) continue;
        const int r = chain_len[c] - chain_pos[c];
        cnt += r > 0;
        rem = max(rem, r);
        dec += chain_pos[c];
    }
    unsigned long long total;
    unsigned long long at = block_exscan(cnt, sm, &total);
    atomicMax(&s_rem, rem);
    atomicAdd(&s_dec, dec);
    for (int i = lo; i < hi; ++i) {
        const int c = order[i];
        if (chain_len[c] > chain_pos[c] && chain_owned(chain_off[c], chain_len[c], B, rank, world)) live[at++] = c;
    }
    __syncthreads();
    if (tid == 0) {
        host_info[0] = (int)total;
        host_info[1] = s_rem;
        host_info[2] = counter[0];  // accepted so far
        host_info[3] = s_dec;       // decided so far
        // the stage's while loop runs another round only while chains remain after this one
        // (this round's own work follows in the same loop body)
        if (use_cond) cudaGraphSetConditional(cond, total > 0 ? 1u : 0u);
    }
}

// The round's pre-fetch tree: the best-first order of M nodes for the acceptance rate
// estimated so far, from the master orders made on the host (one per bin of that rate, nodes in
// best-first order with children after their parents).  Best-first growth under a depth cap
// takes, in order, the master nodes shallower than the cap, so the tree is the first
// M = max(1, slots / A) of those, renumbered.  Writes am = {A, M, A M, 0} for the round's
// kernels; am[3] then counts the rows that will run (candidates and screen below).
constexpr int TMPL_BINS = 32;
__global__ void __launch_bounds__(T1) template_kernel(int slots, const int *__restrict__ live_info,
                                                      const double *__restrict__ p_prev,
                                                      const int4 *__restrict__ master, int *__restrict__ map,
                                                      int4 *__restrict__ tmpl, int *__restrict__ am,
                                                      int *__restrict__ screened, int use_surrogate) {
    __shared__ unsigned long long sm[64];
    const int tid = threadIdx.x;
    const int A = live_info[0];
    if (A <= 0) {
        if (tid == 0) am[0] = am[1] = am[2] = am[3] = 0;
        return;
    }
    const int cap = min(live_info[1], TREE_DEPTH_MAX);
    // acceptance rate: this stage's decisions so far, shrunk towards the previous stages'
    const double p = ((double)live_info[2] + 20.0 * p_prev[0]) / ((double)live_info[3] + 20.0);
    const int bin = min(TMPL_BINS - 1, max(0, (int)(p * TMPL_BINS)));
    const int want = max(1, slots / A);
    const int4 *mo = master + (size_t)bin * slots;
    const int chunk = (slots + T1 - 1) / T1;
    const int lo = min(slots, tid * chunk), hi = min(slots, lo + chunk);
    unsigned long long c = 0;
    for (int i = lo; i < hi; ++i) c += (mo[i].y >> 1) < cap;
    unsigned long long total;
    unsigned long long at = block_exscan(c, sm, &total);
    for (int i = lo; i < hi; ++i) {
        const bool shallow = (mo[i].y >> 1) < cap;
        map[i] = shallow && at < (unsigned long long)want ? (int)at : -1;
        at += shallow;
    }
    __syncthreads();
    for (int i = lo; i < hi; ++i) {
        const int j = map[i];
        if (j < 0) continue;
        const int4 m = mo[i];
        tmpl[j] = make_int4(m.x >= 0 ? map[m.x] : -1, m.y, m.z >= 0 ? map[m.z] : -1, m.w >= 0 ? map[m.w] : -1);
    }
    if (tid == 0) {
        const int M = (int)min(total, (unsigned long long)want);
        am[0] = A;
        am[1] = M;
        am[2] = A * M;
        am[3] = 0;
        if (use_surrogate) screened[0] += A * M;
    }
}

// The forward launch of a round inside a graph: a switch node with one branch per bucket of
// runs per SM, ceil(n / SMs) - 1 for the n rows that run (none when n = 0).
struct ShapeSwitch {
    int sms;      // SMs of the device
    int buckets;  // branches: the buckets of 1 .. rows runs
};
__global__ void select_kernel(const int *__restrict__ runs, ShapeSwitch sw, cudaGraphConditionalHandle h) {
    const int n = runs[0];
    cudaGraphSetConditional(h, n > 0 ? min(sw.buckets - 1, (n + sw.sms - 1) / sw.sms - 1) : sw.buckets);
}

// candidates of every (live chain, template node): prop[(slot*M + v)*3].  Unreachable nodes
// (an accepted decision on the path whose candidate lies outside the prior box), nodes
// beyond the chain's length and candidates outside the box get a NaN alpha, which the
// forward launch skips.
__global__ void tree_propose_kernel(int rows, const int *__restrict__ am, const int *__restrict__ live,
                                    const int *__restrict__ chain_off, const int *__restrict__ chain_len,
                                    const int *__restrict__ chain_pos, const double *__restrict__ cur_theta,
                                    const double *__restrict__ st, const double *__restrict__ normals, Box box,
                                    const int4 *__restrict__ tmpl, double *__restrict__ prop,
                                    int *__restrict__ counter, int *__restrict__ runs) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows) return;
    const int M = am[1];
    if (idx >= am[2]) {  // a row this round does not use: the forward launch skips it
        prop[box.P * idx] = nan("");
        return;
    }
    const int slot = idx / M, v = idx % M;
    const int c = live[slot];
    const int row = chain_off[c] + chain_pos[c];  // normals row of the chain's next step
    const int P = box.P;
    int path[TREE_DEPTH_MAX + 1];
    const int depth = tree_path(tmpl, v, path);
    const double *L = st + S_L;
    double base[P_MAX], cand[P_MAX];
    for (int a = 0; a < P; ++a) base[a] = cur_theta[P * c + a];
    bool ok = chain_pos[c] + depth < chain_len[c];
    for (int i = 0; i < depth && ok; ++i) {
        add_step(P, L, normals + P * (row + i), base, cand);
        if (tmpl[path[i + 1]].y & 1) {  // the path accepts at depth i
            if (!box.in(cand)) ok = false;
            for (int a = 0; a < P; ++a) base[a] = cand[a];
        }
    }
    add_step(P, L, normals + P * (row + depth), base, cand);
    ok = ok && box.in(cand);
    prop[P * idx] = ok ? cand[0] : nan("");
    for (int a = 1; a < P; ++a) prop[P * idx + a] = cand[a];
    if (ok) {
        atomicAdd(counter, 1);
        atomicAdd(runs, 1);
    }
}

// delayed acceptance step 1: along the path of each node, every decision is screened by the
// surrogate against its base (the candidate of the deepest accepted decision above it, else
// the chain's state).  A node is not run when its own candidate fails the screen or when its
// path accepts a candidate that fails it (that path cannot happen).
__global__ void tree_screen_kernel(int rows, const int *__restrict__ am, int P, const int *__restrict__ live,
                                   const int *__restrict__ chain_off, const int *__restrict__ chain_pos,
                                   const double *__restrict__ cur_sl, const double *__restrict__ prop_sl,
                                   const double *__restrict__ st, const double *__restrict__ u1,
                                   const int4 *__restrict__ tmpl, double *__restrict__ prop,
                                   int *__restrict__ counter, const int *__restrict__ trust,
                                   int *__restrict__ runs) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows || idx >= am[2] || !trust[0]) return;  // no screen while the surrogate is not trusted
    if (isnan(prop[P * idx])) return;
    const int M = am[1];
    const int slot = idx / M, v = idx % M;
    const int c = live[slot];
    const int row = chain_off[c] + chain_pos[c];
    const double qn = st[S_QN];
    int path[TREE_DEPTH_MAX + 1];
    const int depth = tree_path(tmpl, v, path);
    double bsl = cur_sl[c];
    bool reach = true;
    for (int i = 0; i < depth && reach; ++i) {
        const double a_sl = prop_sl[slot * M + path[i]];
        if (tmpl[path[i + 1]].y & 1) {
            if (!(log(u1[row + i]) < qn * (a_sl - bsl))) reach = false;
            bsl = a_sl;
        }
    }
    const bool pass = reach && log(u1[row + depth]) < qn * (prop_sl[idx] - bsl);
    if (!pass) {
        prop[P * idx] = nan("");
        atomicSub(runs, 1);
    } else {
        atomicAdd(counter, 1);
    }
}

// walk each live chain down the template along the decisions it actually takes
__global__ void tree_resolve_kernel(const int *__restrict__ am, int P, int use_surrogate,
                                    const int *__restrict__ trust, double *__restrict__ dstat,
                                    const int *__restrict__ live,
                                    const int *__restrict__ chain_off, const int *__restrict__ chain_len,
                                    int *__restrict__ chain_pos, double *__restrict__ cur_theta,
                                    double *__restrict__ cur_ll, double *__restrict__ cur_sl,
                                    const double *__restrict__ prop, const double *__restrict__ prop_ll,
                                    const double *__restrict__ prop_sl, const int *__restrict__ prop_status,
                                    const double *__restrict__ st, const double *__restrict__ u_plain,
                                    const double *__restrict__ u_second, const int4 *__restrict__ tmpl,
                                    double *__restrict__ out_theta,
                                    double *__restrict__ out_ll, double *__restrict__ out_sl, int *__restrict__ counter,
                                    const unsigned long long *__restrict__ run_work,
                                    unsigned long long *__restrict__ useful) {
    int slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= am[0]) return;
    const int M = am[1];
    const int c = live[slot];
    const double qn = st[S_QN];
    const int len = chain_len[c];
    const bool delayed = use_surrogate && trust[0];
    const double *u_acc = delayed ? u_second : u_plain;  // the second step's row, or plain Metropolis
    int p = chain_pos[c];
    int v = 0, acc = 0, ran = 0;
    double d1 = 0.0, d2 = 0.0, dn = 0.0;  // the plain model's judgement of the surrogate
    unsigned long long work = 0;
    while (v >= 0 && p < len) {
        const int idx = slot * M + v;
        const int pos = chain_off[c] + p;
        const bool run = !isnan(prop[P * idx]);  // the one-step chain would have run this proposal
        ran += run;
        if (run) work += run_work[idx];
        const bool valid = run && prop_status[idx] == SWIMMER_OK;
        if (use_surrogate && valid) {
            const double d = prop_ll[idx] - prop_sl[idx];
            d1 += d;
            d2 += d * d;
            dn += 1.0;
        }
        double thr = qn * (prop_ll[idx] - cur_ll[c]);
        if (delayed) thr -= qn * (prop_sl[idx] - cur_sl[c]);
        const bool accept = valid && log(u_acc[pos]) < thr;
        if (accept) {
            for (int q = 0; q < P; ++q) cur_theta[P * c + q] = prop[P * idx + q];
            cur_ll[c] = prop_ll[idx];
            if (use_surrogate) cur_sl[c] = prop_sl[idx];
            ++acc;
        }
        for (int q = 0; q < P; ++q) out_theta[P * pos + q] = cur_theta[P * c + q];
        out_ll[pos] = cur_ll[c];
        out_sl[pos] = cur_sl[c];
        ++p;
        v = accept ? tmpl[v].z : tmpl[v].w;
    }
    chain_pos[c] = p;
    if (acc) atomicAdd(counter, acc);
    if (ran) atomicAdd(counter + 3, ran);
    if (work) atomicAdd(useful, work);
    if (dn > 0.0) {
        atomicAdd(dstat, d1);
        atomicAdd(dstat + 1, d2);
        atomicAdd(dstat + 2, dn);
    }
}

// Best-first decision tree of M nodes (host): the root, then repeatedly the candidate child
// with the largest probability of lying on the chain's path, an accepted step having
// probability p.  Depth < depth_cap.  Ties go to the earlier candidate.
int build_template(int M, double p, int depth_cap, int4 *t) {
    struct Cand {
        double prob;
        int parent, accept, seq;
    };
    std::vector<Cand> heap;
    auto less = [](const Cand &a, const Cand &b) { return a.prob < b.prob || (a.prob == b.prob && a.seq > b.seq); };
    std::vector<double> prob(M);
    int seq = 0;
    t[0] = make_int4(-1, 0, -1, -1);
    prob[0] = 1.0;
    auto push_children = [&](int v) {
        if ((t[v].y >> 1) + 1 >= depth_cap) return;
        heap.push_back({prob[v] * p, v, 1, seq++});
        std::push_heap(heap.begin(), heap.end(), less);
        heap.push_back({prob[v] * (1.0 - p), v, 0, seq++});
        std::push_heap(heap.begin(), heap.end(), less);
    };
    push_children(0);
    int n = 1;
    while (n < M && !heap.empty()) {
        std::pop_heap(heap.begin(), heap.end(), less);
        Cand cd = heap.back();
        heap.pop_back();
        const int depth = (t[cd.parent].y >> 1) + 1;
        t[n] = make_int4(cd.parent, 2 * depth + cd.accept, -1, -1);
        prob[n] = cd.prob;
        if (cd.accept) t[cd.parent].z = n;
        else t[cd.parent].w = n;
        push_children(n);
        ++n;
    }
    return n;
}

}  // namespace

extern "C" int tmcmc_tree_template(int M, double p_accept, int depth_cap, int *nodes, int *count) {
    ARG_CHECK(M >= 1, "M must be >= 1");
    ARG_CHECK(p_accept > 0.0 && p_accept < 1.0, "p_accept must be in (0, 1)");
    ARG_CHECK(depth_cap >= 1 && depth_cap <= TREE_DEPTH_MAX, "depth_cap must be in [1, %d]", TREE_DEPTH_MAX);
    ARG_CHECK(nodes != nullptr && count != nullptr, "NULL output");
    std::vector<int4> t(M);
    const int n = build_template(M, p_accept, depth_cap, t.data());
    for (int v = 0; v < n; ++v) {
        nodes[4 * v] = t[v].x;
        nodes[4 * v + 1] = t[v].y;
        nodes[4 * v + 2] = t[v].z;
        nodes[4 * v + 3] = t[v].w;
    }
    *count = n;
    return 0;
}

extern "C" int tmcmc_analyze(swimmer_handle *h, int B, const double *theta, const double *loglik, double q,
                             double *out_w, double *stats, void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(theta && loglik && out_w && stats, "NULL device pointer");
    ARG_CHECK(q >= 0.0 && q < 1.0, "q must be in [0, 1)");
    set_double_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(h->stage_q, q);
    analyze_kernel<<<1, T1, 0, (cudaStream_t)stream>>>(B, n_params(h->cfg), theta, loglik, h->stage_q, out_w, stats,
                                                       nullptr);
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

namespace {

// ---------------------------------------------------------------------------------
// One stage, enqueued without host synchronization.  Device counters (ints at info + 64):
// [0] accepted, [1] screen passes, [2] proposals run, [3] runs on the realized paths,
// [4] surrogate evaluations; [8..11] the round's live chains, largest remaining length,
// accepted and decided so far; [16..19] the round's A, M, A M and rows that run.
// ---------------------------------------------------------------------------------
constexpr int CNT = 64, LIVE = CNT + 8, AM = CNT + 16;
constexpr double SURR_ERR_MAX = 1.0;    // nats: spread of l - l~ allowed for screening
constexpr double SURR_MIN_JUDGED = 10;  // proposals both models evaluated, for a judgement

// The chains' outputs become the population (when the analysis succeeded); the annealing
// exponent and the acceptance estimate advance; the stage summary (SWIMMER_STAGE_* layout) is
// written.
__global__ void finalize_kernel(int B, int P, int use_surrogate, const double *__restrict__ st,
                                const int *__restrict__ info, const double *__restrict__ out_theta,
                                const double *__restrict__ out_ll, const double *__restrict__ out_sl,
                                double *__restrict__ theta, double *__restrict__ ll, double *__restrict__ sl,
                                int *__restrict__ status, double *__restrict__ q_io, double *__restrict__ p_accept,
                                double *__restrict__ summary, const double *__restrict__ dstat,
                                int *__restrict__ trust) {
    const bool ok = st[S_STATUS] == 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
        if (ok) {
            for (int a = 0; a < P; ++a) theta[P * i + a] = out_theta[P * i + a];
            ll[i] = out_ll[i];
            if (use_surrogate) sl[i] = out_sl[i];
        }
        status[i] = 0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const int *cnt = info + CNT;
        summary[SWIMMER_STAGE_STATUS] = st[S_STATUS];
        summary[SWIMMER_STAGE_Q_IN] = q_io[0];
        summary[SWIMMER_STAGE_Q] = ok ? st[S_QN] : q_io[0];
        summary[SWIMMER_STAGE_LOG_S] = ok ? st[S_LOGS] : 0.0;
        for (int a = 0; a < P_MAX; ++a) summary[SWIMMER_STAGE_MU + a] = ok ? st[S_MU + a] : 0.0;
        for (int a = 0; a < P_MAX * P_MAX; ++a) summary[SWIMMER_STAGE_SIGMA + a] = ok ? st[S_SIG + a] : 0.0;
        summary[SWIMMER_STAGE_UNIQUE] = info[0];
        summary[SWIMMER_STAGE_MAX_CHAIN] = info[1];
        summary[SWIMMER_STAGE_ACCEPT] = cnt[0];
        summary[SWIMMER_STAGE_SCREENED] = cnt[4];
        const bool screened = use_surrogate && trust[0];
        summary[SWIMMER_STAGE_EXACT] = screened ? cnt[1] : cnt[2];
        summary[SWIMMER_STAGE_EXACT_PATH] = cnt[3];
        summary[SWIMMER_STAGE_SURR_USED] = screened ? 1.0 : 0.0;
        summary[SWIMMER_STAGE_SURR_ERR] = nan("");
        if (ok) {
            q_io[0] = st[S_QN];
            p_accept[0] = 0.5 * p_accept[0] + 0.5 * (double)cnt[0] / (double)B;
        }
        // delayed acceptance (not in the paper): the plain model judges the surrogate on the
        // proposals both evaluated.  A constant offset of l - l~ cancels in the screen's ratio;
        // its spread, in nats at this stage's exponent, must stay within SURR_ERR_MAX for the
        // next stage to screen, else that stage runs plain Metropolis (the surrogate is still
        // evaluated, so it can be trusted again)
        if (use_surrogate && ok && dstat[2] >= SURR_MIN_JUDGED) {
            const double m = dstat[0] / dstat[2];
            const double err = st[S_QN] * sqrt(fmax(dstat[1] / dstat[2] - m * m, 0.0));
            summary[SWIMMER_STAGE_SURR_ERR] = err;
            trust[0] = err <= SURR_ERR_MAX ? 1 : 0;
        }
    }
}

// the host-checked arguments of a stage
struct StageArgs {
    const tmcmc_state *st;
    const double *uniforms, *normals;
    int use_surrogate, rank, world, B, P;
    double *q_dev, *summary;
    Box box;
};

// analysis, resampling, chains; counters and the outputs of other ranks' rows cleared
int enqueue_prefix(swimmer_handle *h, const StageArgs &a, cudaStream_t s) {
    const tmcmc_state *st = a.st;
    analyze_kernel<<<1, T1, 0, s>>>(a.B, a.P, st->theta, st->loglik, a.q_dev, h->w, h->stats, h->surr_trust);
    CUDA_TRY(cudaGetLastError());
    resample_kernel<<<1, T1, 0, s>>>(a.B, h->w, a.uniforms, (unsigned long long *)h->cum, h->idx, h->counts);
    CUDA_TRY(cudaGetLastError());
    const double *sl = a.use_surrogate ? st->surr_loglik : nullptr;
    chains_kernel<<<1, T1, 0, s>>>(a.B, a.P, h->stats, h->counts, st->theta, st->loglik, sl, h->chain_off,
                                   h->chain_len, h->chain_id, h->aux, h->cur_theta, h->cur_ll, h->cur_sl, h->info,
                                   CNT);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 3);
    CUDA_TRY(cudaMemsetAsync(h->info + CNT, 0, 8 * sizeof(int), s));
    CUDA_TRY(cudaMemsetAsync(h->surr_dstat, 0, 3 * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(h->chain_pos, 0, sizeof(int) * a.B, s));
    if (a.world > 1) {  // rows of other ranks' chains stay zero, so a SUM over ranks assembles them
        CUDA_TRY(cudaMemsetAsync(h->out_theta, 0, a.P * sizeof(double) * a.B, s));
        CUDA_TRY(cudaMemsetAsync(h->out_ll, 0, sizeof(double) * a.B, s));
        CUDA_TRY(cudaMemsetAsync(h->out_sl, 0, sizeof(double) * a.B, s));
    }
    return 0;
}

// Pre-fetch slots per round: as many forward models as the GPU holds at once at the smallest
// launch shape.  Filling the resident capacity beat smaller budgets and a cost-per-resolved-step
// choice in simulations of the stage with measured launch costs.
int stage_slots(const swimmer_handle *h) { return min(h->cfg.b_max, forward_slots(h, h->cfg.precision)); }

// Launch shape of a round of forward runs in bucket b of samples per SM: the autotuned shape
// of that bucket, else the heuristic's at the bucket's largest batch (at most the round's rows).
// Both the graph's switch node and the host-driven rounds take it, so they run alike.
int round_shape(const swimmer_handle *h, int b, int rows) {
    return forward_threads(h, min(rows, (b + 1) * h->num_sms), h->cfg.precision);
}

// The switch over the buckets of 1 .. rows runs: one branch per bucket (its launch shape, and
// as many CTAs per SM as the bucket has runs per SM: the running rows, dealt first by the
// queue, then go one per CTA and spread over the SMs).
ShapeSwitch round_shapes(const swimmer_handle *h, int rows) { return ShapeSwitch{h->num_sms, tune_bucket(h, rows) + 1}; }

// one pre-fetch round: live chains (and the loop condition), the tree, candidates, the
// surrogate screen, the forward runs, the walk down the trees.  Every size comes from device
// memory; the launches cover the round's capacity and idle past the round's rows.  The
// candidate and screen kernels count the rows that will run; inside a graph (body != nullptr:
// the while node's body) the forward launch is a switch node with one branch per bucket of that
// count, selected on the device.  Driven from the host, the round reads the count back (its one
// synchronization) and stops when no chain is live.
int enqueue_round(swimmer_handle *h, const StageArgs &a, cudaStream_t s, cudaGraph_t body,
                  cudaGraphConditionalHandle cond, bool *done) {
    const tmcmc_state *st = a.st;
    const int slots = h->tmpl_slots;
    // a round has A M <= max(slots, B) tree nodes (M = 1 once the live chains outnumber the
    // slots); the launches cover that many rows, of which the counted ones run
    const int rows = max(slots, a.B);
    int *runs = h->info + AM + 3;
    live_kernel<<<1, T1, 0, s>>>(h->info, a.B, a.rank, a.world, h->chain_id, h->chain_off, h->chain_len, h->chain_pos,
                                 h->live, h->info + CNT, h->info + LIVE, cond, body != nullptr);
    CUDA_TRY(cudaGetLastError());
    template_kernel<<<1, T1, 0, s>>>(slots, h->info + LIVE, h->p_accept_dev, h->tmpl_master, h->tmpl_map, h->tmpl,
                                     h->info + AM, h->info + CNT + 4, a.use_surrogate);
    CUDA_TRY(cudaGetLastError());
    const int grid = (rows + 127) / 128;
    tree_propose_kernel<<<grid, 128, 0, s>>>(rows, h->info + AM, h->live, h->chain_off, h->chain_len, h->chain_pos,
                                             h->cur_theta, h->stats, a.normals, a.box, h->tmpl, h->prop_theta,
                                             h->info + CNT + 2, runs);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 3);
    if (a.use_surrogate) {
        int rc = run_surrogate_loglik(h, rows, h->prop_theta, st->obs, st->sigma, h->prop_sl, s);
        if (rc) return rc;
        tree_screen_kernel<<<grid, 128, 0, s>>>(rows, h->info + AM, a.P, h->live, h->chain_off, h->chain_pos,
                                                h->cur_sl, h->prop_sl, h->stats, a.uniforms + a.B, h->tmpl,
                                                h->prop_theta, h->info + CNT + 1, h->surr_trust, runs);
        CUDA_TRY(cudaGetLastError());
        prof_count(h, 1);
    }
    const ShapeSwitch sw = round_shapes(h, rows);
    cudaGraphConditionalHandle sw_handle = 0;
    int n_run = 0;
    if (body) {
        CUDA_TRY(cudaGraphConditionalHandleCreate(&sw_handle, body, 0, cudaGraphCondAssignDefault));
        select_kernel<<<1, 1, 0, s>>>(runs, sw, sw_handle);
        CUDA_TRY(cudaGetLastError());
        prof_count(h, 1);
    } else {
        CUDA_TRY(cudaMemcpyAsync(h->host_pinned, h->info + AM, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (h->host_pinned[0] <= 0) {
            *done = true;
            return 0;
        }
        n_run = h->host_pinned[3];
    }
    int rc = launch_prepare(h, rows, h->prop_theta, nullptr, s);
    if (!rc) rc = launch_table_build(h, rows, h->cfg.precision == SWIMMER_FP64, s);
    if (rc) return rc;
    if (body) {
        cudaStreamCaptureStatus cs;
        cudaGraph_t g;
        const cudaGraphNode_t *deps = nullptr;
        const cudaGraphEdgeData *edges = nullptr;
        size_t nd = 0;
        CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd));
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = sw_handle;
        cp.conditional.type = cudaGraphCondTypeSwitch;
        cp.conditional.size = (unsigned)sw.buckets;
        cudaGraphNode_t node;
        CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, nd, &cp));
        for (int k = 0; k < sw.buckets; ++k) {
            CUDA_TRY(cudaStreamBeginCaptureToGraph(h->shape_stream, cp.conditional.phGraph_out[k], nullptr, nullptr,
                                                   0, cudaStreamCaptureModeRelaxed));
            rc = launch_forward(h, rows, st->obs, st->sigma, h->prop_ll, nullptr, nullptr, h->prop_status,
                                h->cfg.precision, h->shape_stream, round_shape(h, k, rows), 1, nullptr,
                                (k + 1) * h->num_sms);
            cudaGraph_t captured = nullptr;
            cudaError_t e = cudaStreamEndCapture(h->shape_stream, &captured);
            if (rc) return rc;
            CUDA_TRY(e);
        }
        CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    } else if (n_run > 0) {
        const int bucket = tune_bucket(h, n_run);
        h->prof_rows = n_run;  // the profile records the runs, not the rows the launch covers
        rc = launch_forward(h, rows, st->obs, st->sigma, h->prop_ll, nullptr, nullptr, h->prop_status,
                            h->cfg.precision, s, round_shape(h, bucket, rows), 1, nullptr, (bucket + 1) * h->num_sms);
        h->prof_rows = 0;
        if (rc) return rc;
    }
    tree_resolve_kernel<<<grid, 128, 0, s>>>(h->info + AM, a.P, a.use_surrogate, h->surr_trust, h->surr_dstat,
                                             h->live, h->chain_off, h->chain_len,
                                             h->chain_pos, h->cur_theta, h->cur_ll, h->cur_sl, h->prop_theta,
                                             h->prop_ll, h->prop_sl, h->prop_status, h->stats,
                                             a.uniforms + a.B, a.uniforms + 2 * a.B, h->tmpl, h->out_theta,
                                             h->out_ll, h->out_sl, h->info + CNT, h->run_work, h->work + 1);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
    return 0;
}

int enqueue_finalize(swimmer_handle *h, const StageArgs &a, cudaStream_t s) {
    const tmcmc_state *st = a.st;
    finalize_kernel<<<(a.B + 255) / 256, 256, 0, s>>>(a.B, a.P, a.use_surrogate, h->stats, h->info, h->out_theta,
                                                       h->out_ll, h->out_sl, st->theta, st->loglik, st->surr_loglik,
                                                       st->status, a.q_dev, h->p_accept_dev, a.summary, h->surr_dstat,
                                                       h->surr_trust);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
    return 0;
}

// The rounds as a while node of the graph that stream s is capturing: its body, one round, is
// captured on the handle's side stream; live_kernel sets the condition on the device.
int enqueue_rounds_in_capture(swimmer_handle *h, const StageArgs &a, cudaStream_t s) {
    cudaStreamCaptureStatus cs;
    cudaGraph_t g;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edges = nullptr;
    size_t nd = 0;
    CUDA_TRY(cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd));
    if (cs != cudaStreamCaptureStatusActive) {
        set_error("stream is not capturing");
        return SWIMMER_E_CUDA;
    }
    cudaGraphConditionalHandle cond;
    CUDA_TRY(cudaGraphConditionalHandleCreate(&cond, g, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = cond;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    CUDA_TRY(cudaGraphAddNode(&node, g, deps, edges, nd, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    CUDA_TRY(cudaStreamBeginCaptureToGraph(h->side_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    bool done = false;
    int rc = enqueue_round(h, a, h->side_stream, body, cond, &done);
    cudaGraph_t captured = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->side_stream, &captured);
    if (rc) return rc;
    CUDA_TRY(e);
    CUDA_TRY(cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    return 0;
}

int stage_enqueue(swimmer_handle *h, const StageArgs &a, cudaStream_t s) {
    if (h->profile) {
        // profiling: rounds driven from the host (event records per forward launch cannot sit
        // inside a graph's while node); the same kernels, one host synchronization per round
        int rc = enqueue_prefix(h, a, s);
        for (bool done = false; !rc && !done;) rc = enqueue_round(h, a, s, nullptr, 0, &done);
        return rc ? rc : enqueue_finalize(h, a, s);
    }
    cudaStreamCaptureStatus cs;
    CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    if (cs == cudaStreamCaptureStatusActive) {  // the caller is capturing: become part of its graph
        int rc = enqueue_prefix(h, a, s);
        if (!rc) rc = enqueue_rounds_in_capture(h, a, s);
        if (!rc) rc = enqueue_finalize(h, a, s);
        return rc;
    }
    // otherwise the stage's own graph, captured on the handle's capture stream, launched on s
    cudaStream_t c = h->cap_stream;
    CUDA_TRY(cudaStreamBeginCapture(c, cudaStreamCaptureModeRelaxed));
    int rc = enqueue_prefix(h, a, c);
    if (!rc) rc = enqueue_rounds_in_capture(h, a, c);
    if (!rc) rc = enqueue_finalize(h, a, c);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(c, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    CUDA_TRY(e);
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    CUDA_TRY(e);
    e = cudaGraphLaunch(x, s);
    cudaGraphExecDestroy(x);  // freed once the launch completes
    CUDA_TRY(e);
    return 0;
}

int check_stage(swimmer_handle *h, const tmcmc_state *st, const double *uniforms, const double *normals,
                int use_surrogate, int rank, int world, StageArgs *a) {
    ARG_CHECK(h != nullptr && st != nullptr, "NULL handle or state");
    ARG_CHECK(world >= 1 && rank >= 0 && rank < world, "rank %d outside [0, world %d)", rank, world);
    const int B = st->B;
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(st->theta && st->loglik && st->status && st->obs, "NULL device pointer in the state");
    ARG_CHECK(uniforms && normals, "NULL uniforms/normals");
    ARG_CHECK(st->sigma > 0.0, "sigma must be > 0");
    ARG_CHECK(!use_surrogate || (h->surr_ready && st->surr_loglik), "surrogate not set up");
    const int P = n_params(h->cfg);
    for (int q = 0; q < P; ++q) ARG_CHECK(st->prior_lo[q] <= st->prior_hi[q], "prior box is empty");
    a->st = st;
    a->uniforms = uniforms;
    a->normals = normals;
    a->use_surrogate = use_surrogate ? 1 : 0;
    a->rank = rank;
    a->world = world;
    a->B = B;
    a->P = P;
    a->box.P = P;
    for (int q = 0; q < P_MAX; ++q) {
        a->box.lo[q] = q < P ? st->prior_lo[q] : 0.0;
        a->box.hi[q] = q < P ? st->prior_hi[q] : 0.0;
    }
    return 0;
}

}  // namespace

// master pre-fetch orders for the handle (once, at creation): per bin of the acceptance rate
int tmcmc_templates_init(swimmer_handle *h) {
    const int slots = stage_slots(h);
    h->tmpl_slots = slots;
    std::vector<int4> all((size_t)TMPL_BINS * slots, make_int4(-1, 2 * 63, -1, -1));
    for (int b = 0; b < TMPL_BINS; ++b) build_template(slots, (b + 0.5) / TMPL_BINS, TREE_DEPTH_MAX, &all[(size_t)b * slots]);
    CUDA_TRY(cudaMalloc((void **)&h->tmpl_master, sizeof(int4) * all.size()));
    CUDA_TRY(cudaMalloc((void **)&h->tmpl_map, sizeof(int) * slots));
    CUDA_TRY(cudaMemcpy(h->tmpl_master, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
    const double p0 = 0.8;  // first guess of the acceptance rate
    CUDA_TRY(cudaMalloc((void **)&h->p_accept_dev, sizeof(double)));
    CUDA_TRY(cudaMemcpy(h->p_accept_dev, &p0, sizeof(double), cudaMemcpyHostToDevice));
    return 0;
}

extern "C" int tmcmc_stage_async(swimmer_handle *h, const tmcmc_state *st, const double *uniforms,
                                 const double *normals, int use_surrogate, int rank, int world, double *q,
                                 double *summary, void *stream) {
    StageArgs a;
    int rc = check_stage(h, st, uniforms, normals, use_surrogate, rank, world, &a);
    if (rc) return rc;
    ARG_CHECK(q != nullptr && summary != nullptr, "NULL q or summary");
    a.q_dev = q;
    a.summary = summary;
    return stage_enqueue(h, a, (cudaStream_t)stream);
}

extern "C" int tmcmc_stage(swimmer_handle *h, tmcmc_state *st, const double *uniforms, const double *normals,
                           int use_surrogate, void *stream) {
    return tmcmc_stage_shard(h, st, uniforms, normals, use_surrogate, 0, 1, stream);
}

extern "C" int tmcmc_stage_shard(swimmer_handle *h, tmcmc_state *st, const double *uniforms, const double *normals,
                                 int use_surrogate, int rank, int world, void *stream) {
    StageArgs a;
    int rc = check_stage(h, st, uniforms, normals, use_surrogate, rank, world, &a);
    if (rc) return rc;
    ARG_CHECK(st->q >= 0.0 && st->q < 1.0, "stage already at q = 1");
    cudaStream_t s = (cudaStream_t)stream;
    // the exponent in, the stage, its summary out: one synchronization, at the end
    set_double_kernel<<<1, 1, 0, s>>>(h->stage_q, st->q);
    CUDA_TRY(cudaGetLastError());
    a.q_dev = h->stage_q;
    a.summary = h->stage_summary;
    rc = stage_enqueue(h, a, s);
    if (rc) return rc;
    double *hs = h->host_pinned_d + 1;
    CUDA_TRY(cudaMemcpyAsync(hs, h->stage_summary, sizeof(double) * SWIMMER_STAGE_SUMMARY, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hs[SWIMMER_STAGE_STATUS] != 0.0) {
        set_error(hs[SWIMMER_STAGE_STATUS] == 1.0 ? "every sample has log-likelihood -inf"
                                                   : "proposal covariance is not positive definite");
        return SWIMMER_E_STATE;
    }
    const int P = a.P;
    st->q = hs[SWIMMER_STAGE_Q];
    st->stage += 1;
    st->log_s = hs[SWIMMER_STAGE_LOG_S];
    st->log_evidence += hs[SWIMMER_STAGE_LOG_S];
    for (int i = 0; i < 4; ++i) st->mu[i] = i < P ? hs[SWIMMER_STAGE_MU + i] : 0.0;
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) st->sigma_prop[4 * i + j] = i < P && j < P ? hs[SWIMMER_STAGE_SIGMA + 4 * i + j] : 0.0;
    st->unique = (int)hs[SWIMMER_STAGE_UNIQUE];
    st->max_chain = (int)hs[SWIMMER_STAGE_MAX_CHAIN];
    st->n_accept = (int)hs[SWIMMER_STAGE_ACCEPT];
    st->n_screened = (int)hs[SWIMMER_STAGE_SCREENED];
    st->n_exact = (int)hs[SWIMMER_STAGE_EXACT];
    st->n_exact_path = (int)hs[SWIMMER_STAGE_EXACT_PATH];
    st->surrogate_used = (int)hs[SWIMMER_STAGE_SURR_USED];
    st->surrogate_error = hs[SWIMMER_STAGE_SURR_ERR];
    return 0;
}
