// Shared definitions of the sm_103a swimmer library (handle, limits, error helpers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "swimmer.h"

// ---- table layout ------------------------------------------------------------------
// Both tables cover u = 1 + r^2/delta^2 in [1, 2^n_oct): octave e = floor(log2 u), each
// octave cut into equal panels.  The kernel functions are analytic in u except at u = 0,
// so short panels far from 0 make low-degree polynomials accurate.
constexpr int N_OCT_MAX = 24;          // u < 2^24 (r/delta < 4096)
constexpr int F64_SUB_LOG2 = 3;        // 8 panels per octave
constexpr int F64_SUB = 1 << F64_SUB_LOG2;
constexpr int F64_DEG = 9;             // Chebyshev degree 9 per panel (10 nodes)
constexpr int F64_NODES = F64_DEG + 1;
constexpr int F32_SUB_LOG2 = 6;        // 64 panels per octave (quadratic)
constexpr int F32_SUB = 1 << F32_SUB_LOG2;
constexpr int F64_PANELS_MAX = N_OCT_MAX * F64_SUB;
constexpr int F32_PANELS_MAX = N_OCT_MAX * F32_SUB;
constexpr int NODES_MAX = F64_PANELS_MAX * F64_NODES;   // 1920
// FP64 table per sample: [2][F64_PANELS_MAX][F64_NODES] Chebyshev coefficients
constexpr int TAB64_STRIDE = 2 * F64_PANELS_MAX * F64_NODES;
// FP32 table per sample (float4 units): part A [F32_PANELS_MAX] float4 = (g1 c0, g1 c1,
// g1 c2, h c0) then part B [F32_PANELS_MAX] float2 = (h c1, h c2), h = delta^2 g2: monomial
// quadratic coefficients in G = 1 + f / F32_SUB, f in [0, 1) the local panel coordinate
// (G is u's mantissa with the panel bits cleared)
constexpr int TAB32_STRIDE = F32_PANELS_MAX + F32_PANELS_MAX / 2;
constexpr int TAIL_MAX = 64;           // pieces of the integral of K0 phi s beyond the last node
constexpr int K1_SCRATCH = 2 * NODES_MAX + TAIL_MAX;  // doubles of table-build scratch per sample
constexpr double R_MAX_OVER_L = 1.25;  // table reach in units of the flagellum length
constexpr double STRETCH_MAX = 0.20;   // segment stretch beyond which a run counts as diverged
constexpr int N_PTS_MAX = 1024;
// FP32 pair units (see forward.cu): one list per block count nb = ceil(n / 32) and per mode
// (0: one target block per unit, 1: two target blocks sharing a source block, 2: four); the
// handle's device buffer starts with [UNIT_MODES][UNIT_NB_MAX + 1] offsets (list nb of mode m
// spans [hdr[m][nb - 1], hdr[m][nb]) after the header), at most nb^2 units a list
constexpr int UNIT_NB_MAX = N_PTS_MAX / 32;
constexpr int UNIT_MODES = 3;
constexpr int UNIT_HDR = UNIT_MODES * (UNIT_NB_MAX + 1);
constexpr int SHAPE_WIDE = SWIMMER_SHAPE_WIDE;  // launch-shape flag: two-target pair units
constexpr int SHAPE_QUAD = SWIMMER_SHAPE_QUAD;  // launch-shape flag: four-target pair units
constexpr int SHAPE_THREADS = SHAPE_WIDE - 1;
// unit packing: I [0, 5), J [5, 10), I2, I3, I4 [10, 25), step code [25, 27) (0: d0 = 0,
// 1: d0 = 16, 2: diagonal block, d = 1 .. 16), kind [27, 29) (0, 1, 2: 1, 2, 4 target blocks)
__host__ __device__ inline unsigned unit_pack(int kind, int code, int J, int I, int I2 = 0, int I3 = 0, int I4 = 0) {
    return (unsigned)I | ((unsigned)J << 5) | ((unsigned)I2 << 10) | ((unsigned)I3 << 15) | ((unsigned)I4 << 20) |
           ((unsigned)code << 25) | ((unsigned)kind << 27);
}
constexpr int P_THETA = 3;
constexpr double X_MAX = 600.0;        // largest alpha * r the Bessel evaluations accept

// per-sample derived parameters written by the table builder and read by the forward kernel
struct SampleParams {
    double alpha, kc, amp, length, ds, delta;
    int n, n_oct, status, nh;  // flagellum points, table octaves, status, head points
    double sig;                // noise scale of the sample (theta[3] with 4 unknowns, else 1)
};

// head model geometry in units of ds (defaults: head points spaced like the flagellum's, a
// gap of one ds), and the largest distance between two points of a straight swimmer of n
// flagellum points (flagellum, neck gap, head diameter), in units of ds
__host__ __device__ inline double head_radius_over_ds(const swimmer_config &c) {
    return c.head_radius_over_ds > 0.0 ? c.head_radius_over_ds : c.n_head / (2.0 * 3.14159265358979323846);
}
__host__ __device__ inline double neck_gap_over_ds(const swimmer_config &c) {
    return c.neck_gap_over_ds > 0.0 ? c.neck_gap_over_ds : 1.0;
}
__host__ __device__ inline double reach_over_ds(const swimmer_config &c, int n_flag) {
    return (n_flag - 1) + (c.n_head > 0 ? neck_gap_over_ds(c) + 2.0 * head_radius_over_ds(c) : 0.0);
}
// unknowns per sample (rows of theta)
__host__ __device__ inline int n_params(const swimmer_config &c) { return c.n_params == 4 ? 4 : 3; }
constexpr int P_MAX = 4;

// flagellum points per swimmer when a sample does not give its own
__host__ __device__ inline int default_flagellum_points(const swimmer_config &c) {
    const int ns = c.n_swimmers == 2 ? 2 : 1;
    return c.n_max / ns - c.n_head;
}
// the largest distance between two points of a sample (two swimmers add their separation)
__host__ __device__ inline double sample_reach(const swimmer_config &c, int n_flag, double ds) {
    return reach_over_ds(c, n_flag) * ds + (c.n_swimmers == 2 ? c.swimmer_distance : 0.0);
}

struct ProfileEvents;

struct swimmer_handle {
    swimmer_config cfg;
    // opt-in profiling: CUDA events around every forward-kernel launch, launch counter
    int profile;
    long long n_launch;
    ProfileEvents *prof;
    int prof_rows;          // rows a speculative launch actually runs (profiling record), 0 = all
    unsigned long long *work;  // device counters: [0] pair evaluations executed by the forward
                               // kernel, [1] those a one-step-at-a-time TMCMC would also run
    unsigned long long *run_work;  // [b_max] pair evaluations of each run of the last launch
    // autotuned threads per sample for batch sizes in [2^k, 2^(k+1)), per precision; 0 = heuristic
    int tune_threads[2][17];  // [FP64, FP32C][samples per SM - 1, capped at 16]; launch shapes
    unsigned *units;          // device: FP32 pair-unit lists (UNIT_HDR offsets, then the lists)
    int device;
    int num_sms;
    int max_smem;  // opt-in shared memory per block (bytes)
    int regs_per_sm;  // 32-bit registers per SM
    // per-sample workspace (b_max samples)
    double *tab64;          // [b_max][TAB64_STRIDE]
    double *k1_scratch;     // [b_max][K1_SCRATCH] interval integrals of the table build
    float4 *tab32;          // [b_max][TAB32_STRIDE]
    float2 *pq;             // [b_max][n_max] FP32 kernel: preferred-curvature coefficients
    SampleParams *sp;       // [b_max]
    int *order;             // [b_max] processing order (longest first)
    int *queue;             // [4] work counters
    double *speed_tmp;      // [b_max]
    // TMCMC workspace
    double *w;              // [b_max]
    double *stats;          // [64]
    int *idx, *counts, *chain_id, *chain_off, *chain_len, *aux;  // [b_max] each, aux [b_max+64]
    double *cur_theta, *cur_ll, *cur_sl, *prop_theta, *prop_ll, *prop_sl, *out_theta, *out_ll, *out_sl;
    int *prop_status, *live, *chain_pos;  // [b_max] each
    int4 *tmpl;                           // device [b_max]: the round's pre-fetch template tree
    int4 *tmpl_master;                    // device [32][tmpl_slots]: best-first orders per rate bin
    int *tmpl_map;                        // device [tmpl_slots]: master node -> round node
    int tmpl_slots;                       // forward runs per pre-fetch round
    double *p_accept_dev;                 // device: running Metropolis acceptance rate estimate
    double *stage_q, *stage_summary;      // device: tmcmc_stage's exponent and summary record
    double *surr_dstat;                   // device [3]: sum, sum of squares, count of l - l~
    int *surr_trust;                      // device: 1 while the surrogate may screen proposals
    cudaStream_t side_stream, cap_stream, shape_stream;  // capture streams of the stage graph
    unsigned long long *cum;  // [b_max] fixed-point prefix sums
    int *info;              // [128] device counters / host-visible summary
    int *host_pinned;       // pinned host scratch (b_max + 128 ints)
    double *host_pinned_d;  // pinned host scratch (64 doubles)
    // surrogate
    float *surr_params;     // device copy of the trained parameters (NPARAM)
    double surr_in_lo[5], surr_in_hi[5];
    double *surr_norm;      // device [2][80] out_mean, out_std
    int surr_obs_stride;
    double surr_log10_kt, surr_omega;
    int surr_ready;
    float *surr_x, *surr_y; // [b_max][5], [b_max][80]
    float *surr_ws;         // MLP workspace for b_max samples (allocated by swimmer_surrogate_set)
};

// ---- error reporting -----------------------------------------------------------------
void set_error(const char *fmt, ...);

#define CUDA_TRY(expr)                                                               \
    do {                                                                             \
        cudaError_t _e = (expr);                                                     \
        if (_e != cudaSuccess) {                                                     \
            set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), __FILE__, \
                      __LINE__);                                                     \
            return SWIMMER_E_CUDA;                                                   \
        }                                                                            \
    } while (0)

#define ARG_CHECK(cond, ...)                                                         \
    do {                                                                             \
        if (!(cond)) {                                                               \
            set_error(__VA_ARGS__);                                                  \
            return SWIMMER_E_ARG;                                                    \
        }                                                                            \
    } while (0)

// profiling hooks (api.cu): count a kernel launch; bracket a forward-kernel launch
void prof_count(swimmer_handle *h, int launches);
void prof_k2_begin(swimmer_handle *h, cudaStream_t s, int samples);
void prof_k2_end(swimmer_handle *h, cudaStream_t s);

// ---- launchers implemented in the kernel translation units ----------------------------
int launch_prepare(swimmer_handle *h, int B, const double *theta, const int *n_pts, cudaStream_t s);
int launch_table_build(swimmer_handle *h, int B, int need64, cudaStream_t s);
int launch_forward(swimmer_handle *h, int B, const double *obs, double sigma, double *loglik,
                   double *head_traj, double *mean_speed, int *status, int precision,
                   cudaStream_t s, int threads_override = 0, int speculative = 0, double *final_state = nullptr,
                   int max_runs = 0);
int forward_threads(const swimmer_handle *h, int B, int precision);
int tune_bucket(const swimmer_handle *h, int B);
int forward_min_threads(const swimmer_handle *h, int precision);
bool forward_fits(const swimmer_handle *h, int threads, int precision);
int forward_slots(const swimmer_handle *h, int precision);
int tmcmc_templates_init(swimmer_handle *h);
int upload_pair_units(swimmer_handle *h);
int launch_kernel_eval(swimmer_handle *h, int m, const double *r, double *g1, double *g2,
                       int precision, cudaStream_t s);
int gl_init();
// octaves the tables need for the largest sample a handle serves
int handle_octaves(const swimmer_handle *h);
int launch_set_sample(swimmer_handle *h, double alpha, double delta, double r_max, cudaStream_t s);
