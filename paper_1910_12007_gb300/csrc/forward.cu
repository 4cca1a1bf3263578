// K2: fused persistent forward model + log-likelihood, one CTA per sample at a time.
//
// Per time step (Appendix, last paragraph; Sec. 2.1):
//   A  segment vectors e_k = X_{k+1} - X_k and spring tension 2 K_T (|e_k|/ds - 1)/|e_k|
//      (Eq. EFT read as Hookean springs).  The strain comes from |e|^2/ds^2 - 1 evaluated
//      without cancellation (FP64 in the FP64 kernel; error-free FP32 transformations on
//      the double-float positions in the FP32 kernel);
//   B  (same pass) nonlinear curvature zeta_k (Eq. curva) from central differences,
//      preferred curvature zeta^_k(t), and c_k d zeta_k / d X_{k-1,k,k+1} with
//      c_k = 2 K_C ds (zeta - zeta^) (gradient of Eq. EFB).  The FP32 kernel takes the
//      second differences from the double-float segments before rounding them, uses the
//      hardware reciprocal square root, and forms zeta^_k = P_k cos(omega t) +
//      Q_k sin(omega t) from per-run FP64 coefficients and an FP64 rotation of the phase;
//   C  point forces F = -dE/dX (Eq. Fenergy) gathered from the stencils;
//   D  Brinkmanlet pair sum (Eq. BrV) v_i = (1/mu) sum_j [-F_j g1 + (F_j . d) d g2],
//      d = X_i - X_j, with g1, g2 from the per-sample shared-memory table (quadratic in
//      G = 1 + f/64 in FP32, Chebyshev degree 9 in FP64).
//      FP32: every unordered pair once.  g1, g2 and (F . d) d are even in d, so one table
//      lookup serves v_i and v_j.  The points form blocks of 32; a warp takes a block pair
//      (I, J) along diagonals: lane l holds target I*32 + l and meets source
//      J*32 + (l + d) mod 32 at step d, so all lanes look up nearly the same table panel
//      (|d| ds apart on a smooth filament) and the loads broadcast, while the source-side
//      sums travel down the lanes with warp shuffles.  Two consecutive steps run together
//      in the packed FP32 instructions (fma/mul .f32x2: two FMAs per issued instruction),
//      the sources (x/delta, y/delta, Fx, Fy) stored as pair records of a point and its
//      successor in the block; a pair's term is the symmetric 2x2 mobility
//      M = delta^2 g2 e e^T - g1 I (e = d/delta) applied to F_j and to F_i.  Launch
//      shapes may group two or four block pairs {I, J} that share the source block J into
//      one unit (each source load and rotation then serves two or four targets per lane);
//      the host builds the unit lists per block count.  Per-warp partial sums are combined
//      in a fixed order with TwoSum, so results do not depend on scheduling.  Launches
//      whose shared memory holds an SM to one CTA of at most 512 threads use an
//      instantiation compiled for 128 registers a thread.
//      FP64: target i meets source i + d at step d (the point list stored twice), the S
//      threads of a target splitting the sources and combining with warp shuffles;
//   E  forward Euler X += dt v: FP64 positions in the FP64 kernel, double-float (hi + lo
//      FP32, about 48 significant bits) positions updated by TwoSum in the FP32 kernel;
//      every obs_every steps the head point is compared with the observations and the
//      squared residual accumulated in FP64 (Eq. fitness).
// A run stops early, with status DIVERGED, when a velocity is not finite, a point moves
// more than ds in one step, or a segment stretches beyond STRETCH_MAX.
#include <limits.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "table_eval.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;

struct FwdArgs {
    int B;
    const SampleParams *sp;
    const int *order;
    int *queue;
    const double *tab64;
    const float4 *tab32;
    float2 *pq;  // FP32 kernel: [B][n_max] preferred-curvature coefficients (P_k, Q_k) per run
    double mu, dt, kt, eta, omega;
    double hr_over_ds, gap_over_ds, k_head_tens, k_head_c, k_neck_tens, k_neck_ang;  // head model
    int obs_kind;
    double swim_d;        // two swimmers: initial separation along y
    double sigma_ratio;   // noise of the second observed component / the first
    long long steps, obs_every;
    const double *obs;
    double sigma;
    double *loglik;
    double *head_traj;
    double *speed;
    double *final_state;  // optional [B][n_max][4]: (x, y, Fx, Fy) at the end of the run
    int *status;
    unsigned long long *work;      // [0] executed, [1] useful pair evaluations
    unsigned long long *run_work;  // per-run pair evaluations (speculative launches)
    int speculative;               // 1: the caller decides later which runs were useful
    int n_max;
    int threads;
    int tab_panels;  // panels of the shared-memory table region (handle's octaves x panels/octave)
    const unsigned *units;  // FP32 pair-unit lists (offsets header, then the lists)
    int mode;               // FP32 pair units: 0 one-, 1 two-, 2 four-target
};

struct __align__(32) dbl4 {
    double x, y, z, w;
};

template <bool F64>
struct Types;
template <>
struct Types<false> {
    typedef float R;
    typedef float4 R4;
};
template <>
struct Types<true> {
    typedef double R;
    typedef dbl4 R4;
};

// error-free transformations (Knuth TwoSum, Dekker Fast2Sum)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e) {
    s = a + b;
    e = b - (s - a);
}
// compensated accumulation: (s, e) += b
__device__ __forceinline__ void acc_two_sum(float &s, float &e, float b) {
    float t, err;
    two_sum(s, b, t, err);
    e += err;
    s = t;
}

// X_j - X_i of double-float coordinates (hi, lo) as a double-float (dh, dl)
__device__ __forceinline__ void df_sub(const float *h, const float *l, int i, int j, float &dh, float &dl) {
    float s, e;
    two_sum(h[j], -h[i], s, e);
    fast_two_sum(s, e + (l[j] - l[i]), dh, dl);
}

// A Hookean spring E = K (l/l0 - 1)^2 l0 (Eq. EFT's form): rest length l0 (and l0^2 as a
// double-float), 2 K.  spring_*(i, j) returns t with force on i = t (X_j - X_i),
// t = 2 K (l/l0 - 1)/l, and the strain l/l0 - 1 (from l^2/l0^2 - 1, without cancellation).
struct RestF32 {
    float l0, l02_hi, l02_lo, inv_l02, k2;
};
struct RestF64 {
    double l0, inv_l02, k2;
};

__host__ __device__ inline RestF32 rest_f32(double l0, double k) {
    RestF32 r;
    r.l0 = (float)l0;
    r.l02_hi = (float)(l0 * l0);
    r.l02_lo = (float)(l0 * l0 - (double)r.l02_hi);
    r.inv_l02 = (float)(1.0 / (l0 * l0));
    r.k2 = (float)(2.0 * k);
    return r;
}

__host__ __device__ inline RestF64 rest_f64(double l0, double k) {
    RestF64 r;
    r.l0 = l0;
    r.inv_l02 = 1.0 / (l0 * l0);
    r.k2 = 2.0 * k;
    return r;
}

__device__ __forceinline__ float spring_f32(const float *xh, const float *xl, const float *yh, const float *yl, int i,
                                            int j, const RestF32 &r, float &ex, float &ey, float &exl_out,
                                            float &eyl_out, float &strain) {
    float exh, exl, eyh, eyl;
    df_sub(xh, xl, i, j, exh, exl);
    df_sub(yh, yl, i, j, eyh, eyl);
    // |e|^2 - l0^2 without cancellation: exact squares of the hi parts
    float pxx = exh * exh, qxx = fmaf(exh, exh, -pxx);
    float pyy = eyh * eyh, qyy = fmaf(eyh, eyh, -pyy);
    float sp, spe;
    two_sum(pxx, pyy, sp, spe);
    float rest = ((spe + qxx + qyy) + 2.0f * (exh * exl + eyh * eyl)) - r.l02_lo;
    float s2 = ((sp - r.l02_hi) + rest) * r.inv_l02;  // l^2/l0^2 - 1
    float one = 1.0f + s2;
    float root = one * rsqrtf(one);                   // l/l0
    strain = __fdividef(s2, 1.0f + root);            // l/l0 - 1
    float ell = r.l0 * (1.0f + strain);
    ex = exh;
    ey = eyh;
    exl_out = exl;
    eyl_out = eyl;
    return __fdividef(r.k2 * strain, ell);
}

__device__ __forceinline__ double spring_f64(const double *sx, const double *sy, int i, int j, const RestF64 &r,
                                             double &ex, double &ey, double &strain) {
    ex = sx[j] - sx[i];
    ey = sy[j] - sy[i];
    double s2 = fma(fma(ex, ex, ey * ey), r.inv_l02, -1.0);  // l^2/l0^2 - 1
    strain = s2 / (1.0 + sqrt(1.0 + s2));
    double ell = r.l0 * (1.0 + strain);
    return r.k2 * strain / ell;
}

// table region in shared memory: FP32: float4 part A [P] then float2 part B [P] (24 bytes a
// panel), or with MERGED one 32-byte record per panel [P][2] float4, so that one address serves
// both loads of a lookup (the 128-register instantiation, whose launches are held to one or two
// CTAs per SM by other limits, so the larger table costs no occupancy there);
// FP64: Chebyshev coefficients of g1 [P][10] then of g2 [P][10]
template <bool F64, bool MERGED = false>
__host__ __device__ size_t table_bytes(int P) {
    return F64 ? sizeof(double) * 2 * P * F64_NODES : (MERGED ? 2 * sizeof(float4) : sizeof(float4) + sizeof(float2)) * P;
}

__host__ __device__ inline size_t align32(size_t b) { return (b + 31) & ~size_t(31); }

// Warps of a CTA that take part in the FP32 pair sum: one per pair unit at most (a sample of
// n points has ceil(n/32)^2 units of 16 diagonal steps).  Splitting units further for more
// warps was measured slower: lone samples at 1024 threads with 8-step units took 3.9 us per
// step against 3.4 us at 512 threads (more partial sums to combine, more per-unit work).
__host__ __device__ inline int pair_warps(int n_max, int threads) {
    const int nbm = (n_max + 31) / 32;
    const int W = threads / 32;
    return W < nbm * nbm ? W : nbm * nbm;
}

// Per-step state in shared memory.
// FP64: positions sx, sy [n_max] (double); sources (x, y, Fx, Fy) [2 n_max] (the point list
//   twice in a row); tension vectors tx, ty [n_max]; six bending terms [6][n_max].
// FP32: positions xh, xl, yh, yl [n_max]; sources per block of 32 points as two planes of
//   pair records ([nbm][2][32] float4, plane_a / plane_b); tension vectors and bending terms
//   [8][n_max], which
//   during the pair sum hold the per-warp partial velocities [pair warps][nbm * 32] (float2)
//   instead, the region growing when those need more room.
template <bool F64>
__host__ __device__ size_t state_bytes(int n_max, int threads) {
    if (F64) return align32(16 * (size_t)n_max) + 2 * 32 * (size_t)n_max + 8 * 8 * (size_t)n_max;
    const size_t nbm = (n_max + 31) / 32;
    size_t forces = 32 * (size_t)n_max, part = 256 * nbm * (size_t)pair_warps(n_max, threads);
    // (the same bytes are the pair-unit assignment's scratch at the start of a sample)
    const size_t assign = 4 * (2 * nbm * nbm + 2 * 32);
    size_t region = forces > part ? forces : part;
    if (assign > region) region = assign;
    return align32(16 * (size_t)n_max) + 1024 * nbm + align32(region);
}

// FP32: the sample's pair units (unit_pack), at most ceil(n_max/32)^2 ints after the table
template <bool F64, bool MERGED = false>
__host__ __device__ size_t smem_bytes(int n_max, int P, int threads) {
    const size_t nbm = (n_max + 31) / 32;
    return state_bytes<F64>(n_max, threads) + table_bytes<F64, MERGED>(P) + (F64 ? 0 : 4 * nbm * nbm);
}


// -g1 and h = delta^2 g2 from the FP32 table: quadratic in G = 1 + f / 64, f in [0, 1) the
// position of u within its panel.  The table holds -g1, the sign g1 takes in the mobility.
// tab: part A (or the merged records), tB: part B (unused with MERGED).
template <bool MERGED>
__device__ __forceinline__ void kern_f32(const float4 *__restrict__ tab, const float2 *__restrict__ tB, int pmax,
                                         float u, float &gn, float &h) {
    // u >= 1: the panel is (exponent - 127) * panels per octave + top mantissa bits; the
    // exponent bias is subtracted after the clamp, where it folds into the load offsets.  G
    // is u's mantissa with the panel bits cleared (one logic operation).
    constexpr int BIAS = 127 << F32_SUB_LOG2;
    const unsigned bits = __float_as_uint(u);
    const int p = (int)min(bits >> (23 - F32_SUB_LOG2), (unsigned)(pmax + BIAS));
    const float G = __uint_as_float(0x3f800000u | (bits & ((1u << (23 - F32_SUB_LOG2)) - 1u)));
    float4 a;
    float2 c;
    if (MERGED) {
        const float4 *rec = tab + 2 * (p - BIAS);  // (-g1 c0, c1, c2, h c0), (h c1, h c2, ., .)
        a = rec[0];
        c = *(const float2 *)(rec + 1);
    } else {
        a = tab[p - BIAS];
        c = tB[p - BIAS];
    }
    gn = fmaf(G, fmaf(G, a.z, a.y), a.x);
    h = fmaf(G, fmaf(G, c.y, c.x), a.w);
}

__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// Sources of the FP32 pair sum, per block of 32 points, in two planes of pair records:
// plane A entry i holds (x_i, x_{i+1}, y_i, y_{i+1}) and plane B (Fx_i, Fx_{i+1}, Fy_i,
// Fy_{i+1}), positions in units of delta, i + 1 taken modulo 32 within the block.  One 16-byte
// load brings the two sources a lane meets on two consecutive steps of the diagonal walk,
// already paired for the packed FP32 instructions (two FMAs per instruction).
__device__ __forceinline__ int plane_a(int k) { return ((k >> 5) << 6) + (k & 31); }
__device__ __forceinline__ int plane_b(int k) { return ((k >> 5) << 6) + 32 + (k & 31); }
__device__ __forceinline__ int plane_prev(int k) { return (k & ~31) | ((k - 1) & 31); }

// One FP32 pair unit of 16 diagonal steps: lane l holds targets I_r*32 + l, r < R (the I_r
// and J distinct blocks, or R = 1 and I = J for a diagonal block), and at step d = d0 ..
// d0+15 meets source J*32 + (l + d) mod 32; one source load serves R pair evaluations.  Two
// consecutive steps run together in the two halves of the packed FP32 instructions: half 0
// is step d, half 1 step d + 1.  Each pair's term is the symmetric 2x2 mobility
// M = h e e^T - g1 I (e = d / delta, h = delta^2 g2), even in e (Eq. BrV): v_i += M F_j and
// v_j += M F_i.  The source-side sums travel with their sources: after each pair of steps
// both halves move two lanes down, so lane l always holds, in half 0, the sum (over the even
// steps) of the source it meets next on an even step and, in half 1, the odd-step sum of the
// source after it; at the end each source's two sums are brought to its own lane.  A
// diagonal block runs d = 1 .. 16, and at d = 16 only lanes < 16 count (lanes l and l + 16
// meet the same pair there).  Adds the unit's sums into the warp's partial array.
template <int R, bool DIAG, bool MERGED>
__device__ __forceinline__ void pair_unit(const float4 *__restrict__ s4, const float4 *__restrict__ tab,
                                          const float2 *__restrict__ tB, int pmax, int lane, int I0, int I1, int I2,
                                          int I3, int Jb, int d0, float2 *__restrict__ mypart) {
    const int I[4] = {I0, I1, I2, I3};
    const float2 one = dup2(1.f), neg1 = dup2(-1.f);
    float2 mx[R], my[R], mz[R], mw[R], vx[R], vy[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const float4 A = s4[(I[r] << 6) + lane], Bf = s4[(I[r] << 6) + 32 + lane];
        mx[r] = dup2(A.x);
        my[r] = dup2(A.z);
        mz[r] = dup2(Bf.x);
        mw[r] = dup2(Bf.z);
        vx[r] = dup2(0.f);
        vy[r] = dup2(0.f);
    }
    const float4 *srcJ = s4 + (Jb << 6);
    const int nxt2 = (lane + 2) & 31;
    float2 ax = dup2(0.f), ay = dup2(0.f);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int j = (lane + d0 + 2 * k) & 31;
        const float4 qa = srcJ[j], qb = srcJ[32 + j];
        const float2 qx = make_float2(qa.x, qa.y), qy = make_float2(qa.z, qa.w);
        const float2 qz = make_float2(qb.x, qb.y), qw = make_float2(qb.z, qb.w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float2 ex = __ffma2_rn(qx, neg1, mx[r]), ey = __ffma2_rn(qy, neg1, my[r]);
            const float2 u = __ffma2_rn(ex, ex, __ffma2_rn(ey, ey, one));
            float2 gn, h;
            kern_f32<MERGED>(tab, tB, pmax, u.x, gn.x, h.x);
            kern_f32<MERGED>(tab, tB, pmax, u.y, gn.y, h.y);
            if (DIAG && k == 7 && lane >= 16) {  // step 16 of a diagonal block: lanes < 16 only
                gn.y = 0.f;
                h.y = 0.f;
            }
            const float2 hx = __fmul2_rn(h, ex), hy = __fmul2_rn(h, ey);
            const float2 m11 = __ffma2_rn(hx, ex, gn), m12 = __fmul2_rn(hx, ey), m22 = __ffma2_rn(hy, ey, gn);
            vx[r] = __ffma2_rn(m11, qz, __ffma2_rn(m12, qw, vx[r]));
            vy[r] = __ffma2_rn(m12, qz, __ffma2_rn(m22, qw, vy[r]));
            ax = __ffma2_rn(m11, mz[r], __ffma2_rn(m12, mw[r], ax));
            ay = __ffma2_rn(m12, mz[r], __ffma2_rn(m22, mw[r], ay));
        }
        ax.x = __shfl_sync(0xffffffffu, ax.x, nxt2);
        ax.y = __shfl_sync(0xffffffffu, ax.y, nxt2);
        ay.x = __shfl_sync(0xffffffffu, ay.x, nxt2);
        ay.y = __shfl_sync(0xffffffffu, ay.y, nxt2);
    }
    // lane l now holds the even-step sum of source (l + d0 + 16) mod 32 and the odd-step sum
    // of source (l + d0 + 17) mod 32: bring both sums of source l to lane l
    const int from0 = (lane - d0 - 16) & 31, from1 = (lane - d0 - 17) & 31;
    const float sx = __shfl_sync(0xffffffffu, ax.x, from0) + __shfl_sync(0xffffffffu, ax.y, from1);
    const float sy = __shfl_sync(0xffffffffu, ay.x, from0) + __shfl_sync(0xffffffffu, ay.y, from1);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        float2 pv = mypart[(I[r] << 5) + lane];
        pv.x += vx[r].x + vx[r].y;
        pv.y += vy[r].x + vy[r].y;
        if (DIAG) {
            pv.x += sx;
            pv.y += sy;
        }
        mypart[(I[r] << 5) + lane] = pv;
    }
    if (!DIAG) {
        float2 pa = mypart[(Jb << 5) + lane];
        pa.x += sx;
        pa.y += sy;
        mypart[(Jb << 5) + lane] = pa;
    }
}

// The sample's pair units over its n_pw pair warps, longest processing time first: the list
// runs from the heaviest kind down and each unit goes to the least loaded warp (ties to the
// lower warp); the list is then regrouped warp by warp and wstart[w] .. wstart[w + 1] are warp
// w's units.  A fixed assignment, so results stay independent of scheduling.  Costs: a unit's
// pair evaluations per step relative to a one-target unit, as measured (two targets 1.8, four
// 3.4).  scratch (shared memory): 2 n_units + 2 n_pw words.  One thread, once per sample.
__device__ __forceinline__ void assign_units(unsigned *units, int n_units, int n_pw, unsigned *scratch,
                                             int *wstart) {
    unsigned *own = scratch, *tmp = scratch + n_units;
    float *load = (float *)(tmp + n_units);
    int *cnt = (int *)(load + n_pw);
    for (int w = 0; w < n_pw; ++w) {
        load[w] = 0.f;
        cnt[w] = 0;
    }
    for (int u = 0; u < n_units; ++u) {
        const int kind = (units[u] >> 27) & 3;
        int best = 0;
        for (int w = 1; w < n_pw; ++w)
            if (load[w] < load[best]) best = w;
        load[best] += kind == 0 ? 1.0f : kind == 1 ? 1.8f : 3.4f;
        own[u] = best;
        ++cnt[best];
    }
    wstart[0] = 0;
    for (int w = 0; w < n_pw; ++w) {
        wstart[w + 1] = wstart[w] + cnt[w];
        cnt[w] = wstart[w];  // next slot of warp w
    }
    for (int u = 0; u < n_units; ++u) tmp[cnt[own[u]]++] = units[u];
    for (int u = 0; u < n_units; ++u) units[u] = tmp[u];
}

// observations computed by warp 0 after a step (head-centre velocities, two-swimmer
// distances) rather than by the thread that updates the proximal point
__device__ __forceinline__ bool vel_obs(const FwdArgs &a, int nh) {
    return (a.obs_kind == SWIMMER_OBS_HEAD_VELOCITY || a.obs_kind == SWIMMER_OBS_PAIR_DISTANCES) && nh > 0;
}

// Mean of the head points (FP64 sums over one warp, fixed order); all lanes of warp 0 call
// it, lane 0 gets the result.
template <bool F64>
__device__ __forceinline__ void head_centre(const double *sx, const double *sy, const float *xh, const float *xl,
                                            const float *yh, const float *yl, int nf, int nh, int lane, double &cx,
                                            double &cy) {
    cx = 0.0;
    cy = 0.0;
    for (int m = lane; m < nh; m += 32) {
        const int k = nf + m;
        cx += F64 ? sx[k] : (double)xh[k] + (double)xl[k];
        cy += F64 ? sy[k] : (double)yh[k] + (double)yl[k];
    }
    for (int o = 16; o >= 1; o >>= 1) {
        cx += __shfl_xor_sync(0xffffffffu, cx, o);
        cy += __shfl_xor_sync(0xffffffffu, cy, o);
    }
    cx /= nh;
    cy /= nh;
}

// MODEL 0: the flagellum; 1: the full sperm model (head points and neck); 2: two sperm models
// coupled by the fluid.  Code for models a launch does not run compiles out.  BIG: compiled
// for at most 512 threads and one CTA per SM (up to 128 registers a thread), for launches
// whose shared memory already holds them to that few threads per SM (large N): the pair
// loop then keeps more loads in flight.
template <bool F64, int MODEL, bool BIG = false>
__global__ void __launch_bounds__(BIG ? 512 : 1024, 1) forward_kernel(FwdArgs a) {
    constexpr bool HEAD = MODEL >= 1, TWO = MODEL == 2;
    constexpr bool MERGED = !F64 && BIG;  // the FP32 table as 32-byte records (see table_bytes)
    typedef typename Types<F64>::R R;
    typedef typename Types<F64>::R4 R4;
    extern __shared__ __align__(32) unsigned char smraw[];
    const int n_max = a.n_max;
    // positions: FP64 kernel sx, sy (double); FP32 kernel xh, xl, yh, yl (float)
    double *sx = (double *)smraw;
    double *sy = sx + n_max;
    float *xh = (float *)smraw, *xl = xh + n_max, *yh = xl + n_max, *yl = yh + n_max;
    const int nbm = (n_max + 31) >> 5;
    R4 *src = (R4 *)(smraw + align32(16 * (size_t)n_max));  // FP64 [2 n_max]; FP32 [nbm][64]
    R *tvx = (R *)(src + (F64 ? 2 * n_max : 64 * nbm));    // tension vectors, then bending
    R *tvy = tvx + n_max;
    R *bend = tvy + n_max;  // [6][n_max]
    float2 *part = (float2 *)tvx;  // FP32 pair sum: per-warp partial velocities
    unsigned char *tabraw = smraw + state_bytes<F64>(n_max, blockDim.x);
    __shared__ int s_work;
    // the sample's model constants: [0, 18) the springs (flagellum segment, head membrane,
    // diametral, neck A (end to H(pi +- dth)), neck B (next-to-end to H(pi +- dth)), neck
    // gap (end to H(pi))) as RestF64 or RestF32 records; then 1/(2 ds_H), 1/ds_H^2, 1/H_r,
    // 2 K_HC ds_H, 2 K_NA; [23, 25) the head centre at the previous observation
    __shared__ double s_model[26];
    // FP32 kernel: the sample's single-precision constants (see below)
    enum { F_DS, F_INV2DS, F_INVDS2, F_KC2DS, F_INVDELTA, F_DTMU, F_COUNT };
    __shared__ float s_f32[F64 ? 1 : 16];
    // FP32 kernel: (cos, sin)(omega t) of the current step, and the FP64 rotation state
    // (cos, sin)(omega step dt), (cos, sin)(omega dt) that thread 0 advances once per step
    __shared__ float s_rot[2];
    __shared__ double s_rot64[4];
    // FP32 pair sum: warp w processes units [s_wstart[w], s_wstart[w + 1]) of the sample's list
    __shared__ int s_wstart[F64 ? 1 : 33];
    static_assert(F_COUNT <= 16, "s_f32 holds 16 constants");
    const RestF32 *rest32 = (const RestF32 *)s_model;
    const RestF64 *rest64 = (const RestF64 *)s_model;
    enum { M_I2H = 18, M_IH2, M_IHR, M_KHC, M_KANG, M_CX, M_CY };

    const int tid = threadIdx.x, T = blockDim.x;
    const int lane = tid & 31;

    for (;;) {
        if (tid == 0) s_work = atomicAdd(a.queue, 1);
        __syncthreads();
        const int w = s_work;
        if (w >= a.B) break;
        const int b = a.order[w];
        const SampleParams p = a.sp[b];
        const int nf = p.n, nh = HEAD ? p.nh : 0, h2 = nh >> 1;
        const int nsw = nf + nh;            // points per swimmer: flagellum, then head
        const int n = TWO ? 2 * nsw : nsw;  // all points of the sample
        const long long n_obs = a.steps / a.obs_every;
        if (p.status != SWIMMER_OK) {
            if (tid == 0) {
                a.status[b] = p.status;
                if (a.loglik) a.loglik[b] = -INFINITY;
                if (a.speed) a.speed[b] = nan("");
                if (a.speculative) a.run_work[b] = 0;
            }
            if (a.head_traj)
                for (long long o = tid; o < 2 * n_obs; o += T) a.head_traj[(size_t)b * 2 * n_obs + o] = nan("");
            __syncthreads();
            continue;
        }
        // ---- table into shared memory
        const int P = a.tab_panels;
        const int npan = min(P, p.n_oct * (F64 ? F64_SUB : F32_SUB));
        if (F64) {
            const double *g = a.tab64 + (size_t)b * TAB64_STRIDE;
            double *t = (double *)tabraw;
            for (int i = tid; i < npan * F64_NODES; i += T) {
                t[i] = g[i];
                t[(size_t)P * F64_NODES + i] = g[F64_PANELS_MAX * F64_NODES + i];
            }
        } else {
            const float4 *g = a.tab32 + (size_t)b * TAB32_STRIDE;
            const float2 *gb = (const float2 *)(g + F32_PANELS_MAX);
            float4 *t = (float4 *)tabraw;
            float2 *tb = (float2 *)(t + P);
            for (int i = tid; i < npan; i += T) {
                if (MERGED) {
                    t[2 * i] = g[i];
                    t[2 * i + 1] = make_float4(gb[i].x, gb[i].y, 0.f, 0.f);
                } else {
                    t[i] = g[i];
                    tb[i] = gb[i];
                }
            }
            // the sample's pair units, from the handle's list for its block count
            const int nbs = (n + 31) >> 5;
            const unsigned *hdr = a.units + a.mode * (UNIT_NB_MAX + 1);
            const unsigned *ul = a.units + UNIT_HDR + hdr[nbs - 1];
            unsigned *units = (unsigned *)(tabraw + table_bytes<F64, MERGED>(P));
            for (int un = tid; un < (int)(hdr[nbs] - hdr[nbs - 1]); un += T) units[un] = ul[un];
        }
        // ---- initial straight filament X_k = (k ds, 0), stored relative to (L/2, 0); the
        //      head circle's centre H_r + dN to the right of the proximal point, head point m
        //      at angle 2 pi m / N_H (Appendix)
        const double ds = p.ds, L = p.length;
        const double xref = 0.5 * L;
        {
        const double hr = a.hr_over_ds * ds, gap = a.gap_over_ds * ds;
        const double dth = nh ? 2.0 * PI / nh : 0.0, dsh = hr * dth;
        for (int k = tid; k < n; k += T) {
            const int sw = TWO && k >= nsw;  // second swimmer: displaced by d along y
            const int kl = k - sw * nsw;
            double x0, y0;
            if (kl < nf) {
                x0 = kl * ds - xref;
                y0 = 0.0;
            } else {
                double sn, cs;
                sincos((kl - nf) * dth, &sn, &cs);
                x0 = L + gap + hr + hr * cs - xref;
                y0 = hr * sn;
            }
            if (sw) y0 += a.swim_d;
            if (F64) {
                sx[k] = x0;
                sy[k] = y0;
            } else {
                float h = (float)x0;
                xh[k] = h;
                xl[k] = (float)(x0 - (double)h);
                h = (float)y0;
                yh[k] = h;
                yl[k] = (float)(y0 - (double)h);
            }
        }
        if (tid == 0) {
            const double c1 = hr * (1.0 - cos(dth)), s1 = hr * sin(dth);
            const double l0[6] = {ds, 2.0 * hr * sin(0.5 * dth), 2.0 * hr, hypot(gap + c1, s1), hypot(ds + gap + c1, s1),
                                  gap};
            const double kk[6] = {a.kt, a.k_head_tens, a.k_head_tens, a.k_neck_tens, a.k_neck_tens, a.k_neck_tens};
            for (int q = 0; q < 6; ++q) {
                const double lq = l0[q] > 0.0 ? l0[q] : 1.0;  // unused without a head
                if (F64)
                    ((RestF64 *)s_model)[q] = rest_f64(lq, kk[q]);
                else
                    ((RestF32 *)s_model)[q] = rest_f32(lq, kk[q]);
            }
            s_model[M_I2H] = nh ? 0.5 / dsh : 0.0;
            s_model[M_IH2] = nh ? 1.0 / (dsh * dsh) : 0.0;
            s_model[M_IHR] = nh ? 1.0 / hr : 0.0;
            s_model[M_KHC] = 2.0 * a.k_head_c * dsh;
            s_model[M_KANG] = 2.0 * a.k_neck_ang;
        }
        }
        if (!F64) {  // pad the last block with force-free sources at the origin
            const int npad = ((n + 31) >> 5) << 5;
            for (int k = n + tid; k < npad; k += T) {
                src[plane_a(k)] = R4{0, 0, 0, 0};
                src[plane_b(k)] = R4{0, 0, 0, 0};
            }
            if (n < npad && tid == 0) {  // the last point's entries pair it with the first pad
                const int kp = plane_prev(n);
                src[plane_a(kp)].y = 0;
                src[plane_a(kp)].w = 0;
                src[plane_b(kp)].y = 0;
                src[plane_b(kp)].w = 0;
            }
        }
        // FP32 kernel: the sample's single-precision constants, made once here in FP64 and read
        // from shared memory in the step loop (where, short of registers, the compiler would
        // otherwise recompute them from the FP64 parameters every step)
        if (!F64 && tid == 0) {
            s_f32[F_DS] = (float)ds;
            s_f32[F_INV2DS] = (float)(0.5 / ds);
            s_f32[F_INVDS2] = (float)(1.0 / (ds * ds));
            s_f32[F_KC2DS] = (float)(2.0 * p.kc * ds);
            s_f32[F_INVDELTA] = (float)(1.0 / p.delta);
            s_f32[F_DTMU] = (float)(a.dt / a.mu);
            // (cos, sin)(omega t) at t = 0 and the rotation by omega dt per step
            double sw, cw;
            sincos(a.omega * a.dt, &sw, &cw);
            s_rot64[0] = 1.0;
            s_rot64[1] = 0.0;
            s_rot64[2] = cw;
            s_rot64[3] = sw;
            s_rot[0] = 1.f;
            s_rot[1] = 0.f;
        }
        if (!F64) {
            // the preferred curvature of flagellum point k (Appendix: y^ = a (1 - s/L)
            // sin(eta s - omega t), zeta^ = d^2 y^/ds^2) split as
            // zeta^_k(t) = P_k cos(omega t) + Q_k sin(omega t), made in FP64 once per run
            float2 *pq = a.pq + (size_t)b * n_max;
            for (int k = tid; k < nf; k += T) {
                const double sk = k * ds;
                double sn, cs;
                sincos(a.eta * sk, &sn, &cs);
                const double c1 = 2.0 * a.eta / L, c2 = (1.0 - sk / L) * a.eta * a.eta;
                pq[k] = make_float2((float)(-p.amp * (c1 * cs + c2 * sn)), (float)(-p.amp * (c1 * sn - c2 * cs)));
            }
        }
        const double dt_mu = a.dt / a.mu;
        // FP64 pair sum: thread -> (target, source split of S lanes)
        int S = 1;
        while (S < 32 && 2 * S * n <= T) S <<= 1;
        const int slot = tid / S, split = tid % S;
        const int tgt = slot;  // one target per slot
        const bool owner = (split == 0) && (tgt < n);
        // FP32 pair sum: the sample's units of 16 steps over the pair warps
        const unsigned *uhdr = a.units + a.mode * (UNIT_NB_MAX + 1);
        const int nb = (n + 31) >> 5, n_units = F64 ? 0 : (int)(uhdr[nb] - uhdr[nb - 1]);
        const int n_pw = F64 ? 0 : min(pair_warps(n_max, T), (int)(uhdr[nbm] - uhdr[nbm - 1]));
        // the thread that keeps the log-likelihood: thread 0 for head-centre velocities (one
        // warp reduces the head after each observation step), else the one that updates the
        // proximal flagellum point nf - 1 (the observed point)
        const bool head_thread = vel_obs(a, nh) ? tid == 0 : F64 ? (owner && tgt == nf - 1) : (tid == (nf - 1) % T);
        double J = 0.0;
        int status = SWIMMER_OK;
        long long steps_done = a.steps;
        __syncthreads();
        if (!F64 && tid == 0)
            assign_units((unsigned *)(tabraw + table_bytes<F64, MERGED>(P)), n_units, n_pw, (unsigned *)part, s_wstart);
        __syncthreads();
        const R r_ds = F64 ? (R)ds : (R)s_f32[F_DS], r_inv2ds = F64 ? (R)(0.5 / ds) : (R)s_f32[F_INV2DS];
        const R r_invds2 = F64 ? (R)(1.0 / (ds * ds)) : (R)s_f32[F_INVDS2];
        const R kc2ds = F64 ? (R)(2.0 * p.kc * ds) : (R)s_f32[F_KC2DS];
        const R r_amp = (R)p.amp, r_eta = (R)a.eta, r_omega = (R)a.omega, r_L = (R)L;  // (FP64 kernel)
        const R inv_d2 = (R)(1.0 / (p.delta * p.delta));
        if (vel_obs(a, nh) && tid < 32) {  // head centre at the previous observation
            double cx, cy;
            head_centre<F64>(sx, sy, xh, xl, yh, yl, nf, nh, lane, cx, cy);
            if (tid == 0) {
                s_model[M_CX] = cx;
                s_model[M_CY] = cy;
            }
        }
        float g10 = 0.f;  // FP32: -g1 at r = 0 (self term)
        if (!F64) {
            float g2unused;
            kern_f32<MERGED>((const float4 *)tabraw, (const float2 *)((const float4 *)tabraw + P), npan - 1, 1.0f,
                             g10, g2unused);
        }

        // with a final state requested, one more pass of the force phases at t = steps dt
        const long long last = a.steps + (a.final_state ? 1 : 0);
        // 32-bit step count (steps < 2^31 - 1 by the argument checks), observation steps by a
        // countdown (no 64-bit division in the loop), and the FP32 kernel's time in FP32, so
        // that the loop issues no FP64 instruction outside observation steps
        const int obs_every = (int)min(a.obs_every, (long long)INT_MAX);  // > steps: no observation
        int obs_left = obs_every, obs_idx = 0;
        for (int step = 0; step < (int)last; ++step) {
            const double tR = (double)step * a.dt;  // (FP64 kernel; the FP32 kernel rotates s_rot)
            const bool obs_step = --obs_left == 0;
            int bad = 0;
            // ---- A+B: segments, tension, curvature stencils, relative positions.  Thread k
            //      forms e_k (tension of the segment to its next point) and again e_{k-1}
            //      (for the curvature at k), which saves a barrier.  Flagellum points
            //      k < nf form an open chain; head points a closed one (periodic stencils).
            for (int k = tid; k < n; k += T) {
                const int base = (TWO && k >= nsw) ? nsw : 0;  // the point's swimmer
                const int kl = k - base;
                const bool hd = HEAD && kl >= nf;
                const int m = kl - nf;
                const int next = hd ? base + nf + (m + 1 == nh ? 0 : m + 1) : (kl + 1 < nf ? k + 1 : -1);
                const int prev = hd ? base + nf + (m == 0 ? nh - 1 : m - 1) : k - 1;
                const bool center = hd || (kl >= 1 && kl + 1 < nf);
                R qx, qy, epx = 0, epy = 0, emx = 0, emy = 0, tk = 0;
                float d2x = 0.f, d2y = 0.f;  // FP32: e_k - e_{k-1} from the double-float segments
                if (F64) {
                    if (next >= 0) {
                        double ex, ey, strain;
                        tk = (R)spring_f64(sx, sy, k, next, rest64[hd ? 1 : 0], ex, ey, strain);
                        epx = (R)ex;
                        epy = (R)ey;
                        if (!(fabs(strain) <= STRETCH_MAX)) bad = 1;
                    }
                    if (center) {
                        emx = (R)(sx[k] - sx[prev]);
                        emy = (R)(sy[k] - sy[prev]);
                    }
                    qx = (R)sx[k];
                    qy = (R)sy[k];
                } else {
                    float epxl = 0.f, epyl = 0.f;
                    if (next >= 0) {
                        float strain, ex, ey;
                        tk = (R)spring_f32(xh, xl, yh, yl, k, next, rest32[hd ? 1 : 0], ex, ey, epxl, epyl, strain);
                        epx = (R)ex;
                        epy = (R)ey;
                        if (!(fabsf(strain) <= (float)STRETCH_MAX)) bad = 1;
                    }
                    if (center) {
                        // e_{k-1} as a double-float (s, lo); the second difference e_k - e_{k-1}
                        // subtracts the high parts first (neighbouring segments are close, so
                        // that difference is exact) and then the low parts: rounding the
                        // segments to FP32 before subtracting would leave it an error of
                        // about 6e-8 ds, amplified by 1/ds^2 in the curvature
                        float s, e, lo;
                        two_sum(xh[k], -xh[prev], s, e);
                        lo = e + (xl[k] - xl[prev]);
                        emx = (R)(s + lo);
                        d2x = (epx - s) + (epxl - lo);
                        two_sum(yh[k], -yh[prev], s, e);
                        lo = e + (yl[k] - yl[prev]);
                        emy = (R)(s + lo);
                        d2y = (epy - s) + (epyl - lo);
                    }
                    // the pair sum measures separations in units of delta
                    qx = (R)((xh[k] + xl[k]) * s_f32[F_INVDELTA]);
                    qy = (R)((yh[k] + yl[k]) * s_f32[F_INVDELTA]);
                }
                if (next >= 0) {  // tension force vector of segment (k, next)
                    tvx[k] = tk * epx;
                    tvy[k] = tk * epy;
                }
                if (F64) {  // the point list stored twice
                    src[k].x = qx;
                    src[k].y = qy;
                    src[k + n].x = qx;
                    src[k + n].y = qy;
                } else {  // plane A: own entry, and the previous entry's second half
                    const int ka = plane_a(k), kp = plane_a(plane_prev(k));
                    src[ka].x = qx;
                    src[ka].z = qy;
                    src[kp].y = qx;
                    src[kp].w = qy;
                }
                if (center) {
                    const R i2h = hd ? (R)s_model[M_I2H] : r_inv2ds, ih2 = hd ? (R)s_model[M_IH2] : r_invds2;
                    R A = (emx + epx) * i2h, Bv = (emy + epy) * i2h;
                    R C = (F64 ? epx - emx : (R)d2x) * ih2, D = (F64 ? epy - emy : (R)d2y) * ih2;
                    R S2 = A * A + Bv * Bv;
                    R rs;
                    if (F64) {
                        rs = (R)(1.0 / sqrt((double)S2));
                    } else {
                        // the hardware estimate plus one Newton step: its ~2 ulp error would
                        // otherwise enter zeta and the stencils, which multiply it by 1/ds^2
                        const float r0 = rsqrtf((float)S2);
                        rs = (R)fmaf(r0 * 0.5f, fmaf(-(float)S2 * r0, r0, 1.0f), r0);
                    }
                    R S15 = rs * rs * rs;
                    R S25 = S15 * rs * rs;
                    R cross = A * D - Bv * C;
                    R zeta = cross * S15;
                    R zhat;
                    if (hd) {
                        zhat = (R)s_model[M_IHR];  // preferred head curvature 1/H_r
                    } else {
                        if (F64) {
                            const R s = (R)kl * r_ds;
                            const R ph = r_eta * s - r_omega * tR;
                            double sd, cd;
                            sincos((double)ph, &sd, &cd);
                            zhat = -r_amp * ((R)2 * r_eta / r_L * (R)cd + ((R)1 - s / r_L) * r_eta * r_eta * (R)sd);
                        } else {
                            // zeta^_k(t) = P_k cos(omega t) + Q_k sin(omega t) (made in FP64 for the
                            // run); (cos, sin)(omega t) is advanced in FP64 once per step
                            const float2 c = a.pq[(size_t)b * n_max + kl];
                            zhat = (R)fmaf(c.x, s_rot[0], c.y * s_rot[1]);
                        }
                    }
                    R ck = (hd ? (R)s_model[M_KHC] : kc2ds) * (zeta - zhat);
                    R za = D * S15 - (R)3 * A * cross * S25;
                    R zb = -C * S15 - (R)3 * Bv * cross * S25;
                    R zc = -Bv * S15, zd = A * S15;
                    bend[0 * n_max + k] = ck * (-za * i2h + zc * ih2);
                    bend[1 * n_max + k] = ck * (-zb * i2h + zd * ih2);
                    bend[2 * n_max + k] = ck * ((R)-2 * zc * ih2);
                    bend[3 * n_max + k] = ck * ((R)-2 * zd * ih2);
                    bend[4 * n_max + k] = ck * (za * i2h + zc * ih2);
                    bend[5 * n_max + k] = ck * (zb * i2h + zd * ih2);
                }
            }
            __syncthreads();
            // (cos, sin)(omega t) of the next step, rotated in FP64 by the last thread, which
            // has the fewest points here (this step's values were read before the barrier)
            if (!F64 && tid == T - 1) {
                const double c = s_rot64[0], sn = s_rot64[1], wc = s_rot64[2], ws = s_rot64[3];
                const double nc = fma(c, wc, -sn * ws), ns = fma(sn, wc, c * ws);
                s_rot64[0] = nc;
                s_rot64[1] = ns;
                s_rot[0] = (float)nc;
                s_rot[1] = (float)ns;
            }
            // ---- C: point forces, gathered per point (no atomics): segment tensions, the
            //      bending stencils of the centres k-1, k, k+1, and for the head model the
            //      diametral and neck springs and the neck angle (Appendix)
            for (int k = tid; k < n; k += T) {
                const int base = (TWO && k >= nsw) ? nsw : 0;  // the point's swimmer
                const int kl = k - base;
                const bool hd = HEAD && kl >= nf;
                const int m = kl - nf;
                const int next = hd ? base + nf + (m + 1 == nh ? 0 : m + 1) : (kl + 1 < nf ? k + 1 : -1);
                const int prev = hd ? base + nf + (m == 0 ? nh - 1 : m - 1) : (kl >= 1 ? k - 1 : -1);
                R fx = 0, fy = 0;
                if (next >= 0) {
                    fx += tvx[k];
                    fy += tvy[k];
                }
                if (prev >= 0) {
                    fx -= tvx[prev];
                    fy -= tvy[prev];
                }
                if (hd || kl >= 2) {  // centre prev acts on k as its next neighbour
                    fx -= bend[4 * n_max + prev];
                    fy -= bend[5 * n_max + prev];
                }
                if (hd || (kl >= 1 && kl + 1 < nf)) {
                    fx -= bend[2 * n_max + k];
                    fy -= bend[3 * n_max + k];
                }
                if (hd || kl + 2 < nf) {  // centre next acts on k as its previous neighbour
                    fx -= bend[0 * n_max + next];
                    fy -= bend[1 * n_max + next];
                }
                if (HEAD && nh > 0) {
                    // springs (k, j): force on k = t e, e = X_j - X_k; up to three per point
                    for (int q = 0; q < 3; ++q) {
                        int j = -1, kind = 0;  // kind: 0 diametral, 1 neck A, 2 neck B, 3 neck gap
                        if (hd) {
                            if (q == 0) {
                                j = nf + (m + h2 >= nh ? m + h2 - nh : m + h2);
                            } else if (m == h2 - 1 || m == h2 + 1) {
                                j = q == 1 ? nf - 1 : nf - 2;
                                kind = q;
                            } else if (m == h2 && q == 1) {
                                j = nf - 1;
                                kind = 3;
                            }
                        } else if (kl == nf - 1) {
                            j = nf + h2 - 1 + q;
                            kind = q == 1 ? 3 : 1;
                        } else if (kl == nf - 2 && q < 2) {
                            j = nf + h2 - 1 + 2 * q;
                            kind = 2;
                        }
                        if (j < 0) continue;
                        j += base;
                        if (F64) {
                            const RestF64 &r = rest64[2 + kind];
                            double ex, ey, strain;
                            double t = spring_f64(sx, sy, k, j, r, ex, ey, strain);
                            fx += (R)(t * ex);
                            fy += (R)(t * ey);
                            if (!(fabs(strain) <= STRETCH_MAX)) bad = 1;
                        } else {
                            const RestF32 &r = rest32[2 + kind];
                            float ex, ey, exl, eyl, strain;
                            float t = spring_f32(xh, xl, yh, yl, k, j, r, ex, ey, exl, eyl, strain);
                            fx += (R)(t * ex);
                            fy += (R)(t * ey);
                            if (!(fabsf(strain) <= (float)STRETCH_MAX)) bad = 1;
                        }
                    }
                    // neck angle E = K (z1 . z2)^2, z1 = H(pi) - X_{nf-1}, z2 = H(pi+dth) - H(pi-dth)
                    const int ihp = base + nf + h2, iplus = ihp + 1, iminus = ihp - 1, iend = base + nf - 1;
                    if (k == ihp || k == iplus || k == iminus || k == iend) {
                        R z1x, z1y, z2x, z2y;
                        if (F64) {
                            z1x = (R)(sx[ihp] - sx[iend]);
                            z1y = (R)(sy[ihp] - sy[iend]);
                            z2x = (R)(sx[iplus] - sx[iminus]);
                            z2y = (R)(sy[iplus] - sy[iminus]);
                        } else {
                            float h, l;
                            df_sub(xh, xl, iend, ihp, h, l);
                            z1x = (R)(h + l);
                            df_sub(yh, yl, iend, ihp, h, l);
                            z1y = (R)(h + l);
                            df_sub(xh, xl, iminus, iplus, h, l);
                            z2x = (R)(h + l);
                            df_sub(yh, yl, iminus, iplus, h, l);
                            z2y = (R)(h + l);
                        }
                        const R w = (R)s_model[M_KANG] * (z1x * z2x + z1y * z2y);
                        if (k == ihp) {
                            fx -= w * z2x;
                            fy -= w * z2y;
                        } else if (k == iend) {
                            fx += w * z2x;
                            fy += w * z2y;
                        } else if (k == iplus) {
                            fx -= w * z1x;
                            fy -= w * z1y;
                        } else {
                            fx += w * z1x;
                            fy += w * z1y;
                        }
                    }
                }
                if (F64) {
                    src[k].z = fx;
                    src[k].w = fy;
                    src[k + n].z = fx;
                    src[k + n].w = fy;
                } else {  // plane B
                    const int kb = plane_b(k), kp = plane_b(plane_prev(k));
                    src[kb].x = fx;
                    src[kb].z = fy;
                    src[kp].y = fx;
                    src[kp].w = fy;
                }
            }
            __syncthreads();
            if (step == a.steps) {  // final state: positions and the forces there
                for (int k = tid; k < n; k += T) {
                    double *o = a.final_state + ((size_t)b * n_max + k) * 4;
                    o[0] = (F64 ? sx[k] : (double)xh[k] + (double)xl[k]) + xref;
                    o[1] = F64 ? sy[k] : (double)yh[k] + (double)yl[k];
                    o[2] = F64 ? (double)src[k].z : (double)src[plane_b(k)].x;
                    o[3] = F64 ? (double)src[k].w : (double)src[plane_b(k)].z;
                }
                break;
            }
            // ---- D: pair sum
            double vxd = 0.0, vyd = 0.0;
            if (F64) {
                // FP64: target tgt meets source tgt + d at step d (d = split, split + S, ...)
                if (tgt < n) {
                    const R4 me = src[tgt];
                    const double xi = (double)me.x, yi = (double)me.y;
                    const double *tab = (const double *)tabraw;
                    double vx = 0.0, vy = 0.0;
                    const R4 *sp = src + tgt + split;
                    for (int d = split; d < n; d += S, sp += S) {
                        R4 q = *sp;
                        double dx = xi - (double)q.x, dy = yi - (double)q.y;
                        double u = fma(fma(dx, dx, dy * dy), (double)inv_d2, 1.0);
                        double g1, g2;
                        kern_f64(tab, P, npan - 1, u, g1, g2);
                        double fd = fma((double)q.z, dx, (double)q.w * dy);
                        double wv = fd * g2;
                        vx = fma(wv, dx, fma(-(double)q.z, g1, vx));
                        vy = fma(wv, dy, fma(-(double)q.w, g1, vy));
                    }
                    vxd = vx;
                    vyd = vy;
                }
                // combine the S source splits (lanes of one warp)
                for (int o = S >> 1; o >= 1; o >>= 1) {
                    vxd += __shfl_xor_sync(0xffffffffu, vxd, o);
                    vyd += __shfl_xor_sync(0xffffffffu, vyd, o);
                }
            } else if ((tid >> 5) < n_pw) {
                // FP32: each unordered pair {i, j} once.  g1(r) and g2(r) are even in
                // d = X_i - X_j and (F . d) d is even too, so one table lookup gives both
                // v_i += -F_j g1 + (F_j . d) d g2 and v_j += -F_i g1 + (F_i . d) d g2.
                // Unit (I, J, d0): lane l takes target I*32 + l and, at step d = d0 .. d0+15,
                // source J*32 + (l + d) mod 32.  The source-side sum rotates one lane down
                // per step, so lane l always holds the sum of the source it meets.
                // Diagonal units (I = J) run d = 1 .. 16 (at d = 16 only lanes < 16, since
                // lanes l and l + 16 meet the same pair); off-diagonal blocks run d = 0 .. 31
                // as two units.  A two- or four-target unit (wide and quad launch shapes)
                // walks the block pairs {I, J}, {I2, J} (, {I3, J}, {I4, J}) together, sharing
                // the source loads and rotations.  Units go to warps by the sample's fixed
                // longest-processing-time assignment (above).  Each
                // warp adds its units' sums into its own partial array, in a fixed order, so
                // the result does not depend on scheduling.
                const float4 *s4 = (const float4 *)src;
                const float4 *tab = (const float4 *)tabraw;
                const float2 *tB = (const float2 *)(tab + P);
                const int warp = tid >> 5;
                float2 *mypart = part + warp * (nb << 5);
                for (int k = lane; k < (nb << 5); k += 32) mypart[k] = make_float2(0.f, 0.f);
                const unsigned *units = (const unsigned *)(tabraw + table_bytes<F64, MERGED>(P));
                for (int un = s_wstart[warp]; un < s_wstart[warp + 1]; ++un) {
                    const unsigned pk = units[un];
                    const int I = pk & 31, Jb = (pk >> 5) & 31, code = (pk >> 25) & 3, kind = (pk >> 27) & 3;
                    const int d0 = code == 2 ? 1 : code << 4;
                    const int I2 = (pk >> 10) & 31, I3 = (pk >> 15) & 31, I4 = (pk >> 20) & 31;
                    if (kind == 0) {
                        if (I == Jb)
                            pair_unit<1, true, MERGED>(s4, tab, tB, npan - 1, lane, I, 0, 0, 0, Jb, d0, mypart);
                        else
                            pair_unit<1, false, MERGED>(s4, tab, tB, npan - 1, lane, I, 0, 0, 0, Jb, d0, mypart);
                    } else if (BIG && kind == 2) {
                        pair_unit<4, false, MERGED>(s4, tab, tB, npan - 1, lane, I, I2, I3, I4, Jb, d0, mypart);
                    } else {
                        pair_unit<2, false, MERGED>(s4, tab, tB, npan - 1, lane, I, I2, 0, 0, Jb, d0, mypart);
                        // the host gives four-target lists to the 128-register instantiation
                        // only; a run that meets one here ends as diverged, not with pairs missing
                        if (kind == 2) bad = 1;
                    }
                }
            }
            if (!F64) __syncthreads();
            // ---- E: Euler step, divergence, observations
            for (int k = F64 ? (owner ? tgt : n) : tid; k < n; k += F64 ? n : T) {
                if (F64) {
                    double dx = vxd * dt_mu, dy = vyd * dt_mu;  // displacement this step
                    if (!isfinite(dx) || !isfinite(dy) || fmax(fabs(dx), fabs(dy)) > ds) bad = 1;
                    sx[k] += dx;
                    sy[k] += dy;
                } else {
                    // v_k = self term + the pair warps' partial sums, compensated
                    const float4 fk = ((const float4 *)src)[plane_b(k)];  // (Fx, ., Fy, .)
                    float hx = fk.x * g10, lx = 0.f, hy = fk.z * g10, ly = 0.f;
                    for (int w = 0; w < n_pw; ++w) {
                        const float2 pv = part[w * (nb << 5) + k];
                        acc_two_sum(hx, lx, pv.x);
                        acc_two_sum(hy, ly, pv.y);
                    }
                    float dx = (hx + lx) * s_f32[F_DTMU], dy = (hy + ly) * s_f32[F_DTMU];
                    if (!isfinite(dx) || !isfinite(dy) || fmaxf(fabsf(dx), fabsf(dy)) > s_f32[F_DS]) bad = 1;
                    float s, e, nh, nl;
                    two_sum(xh[k], dx, s, e);
                    two_sum(s, xl[k] + e, nh, nl);
                    xh[k] = nh;
                    xl[k] = nl;
                    two_sum(yh[k], dy, s, e);
                    two_sum(s, yl[k] + e, nh, nl);
                    yh[k] = nh;
                    yl[k] = nl;
                }
                // the head point's observation: squared residual into J (FP64), trajectory row;
                // obs_step is the same for every thread, so other steps branch around it
                if (obs_step) {
                    if (!vel_obs(a, nh) && k == nf - 1) {
                        double hxo = F64 ? sx[k] : (double)xh[k] + (double)xl[k];
                        const double hyo = F64 ? sy[k] : (double)yh[k] + (double)yl[k];
                        const long long o = obs_idx;
                        hxo += xref;
                        if (a.obs) {
                            double rx = a.obs[2 * o] - hxo, ry = (a.obs[2 * o + 1] - hyo) / a.sigma_ratio;
                            J = fma(rx, rx, fma(ry, ry, J));
                        }
                        if (a.head_traj) {
                            a.head_traj[((size_t)b * n_obs + o) * 2] = hxo;
                            a.head_traj[((size_t)b * n_obs + o) * 2 + 1] = hyo;
                        }
                    }
                }
            }
            if (__syncthreads_or(bad)) {
                status = SWIMMER_DIVERGED;
                steps_done = step + 1;
                break;
            }
            if (vel_obs(a, nh) && obs_step && tid < 32) {
                double ox, oy;
                if (TWO && a.obs_kind == SWIMMER_OBS_PAIR_DISTANCES) {
                    // distances between the tail tips and between the head centres (Sec. 4.2)
                    double c0x, c0y, c1x, c1y;
                    head_centre<F64>(sx, sy, xh, xl, yh, yl, nf, nh, lane, c0x, c0y);
                    head_centre<F64>(sx, sy, xh, xl, yh, yl, nsw + nf, nh, lane, c1x, c1y);
                    double tx, ty;
                    if (F64) {
                        tx = sx[nsw] - sx[0];
                        ty = sy[nsw] - sy[0];
                    } else {
                        float hh, ll;
                        df_sub(xh, xl, 0, nsw, hh, ll);
                        tx = (double)hh + (double)ll;
                        df_sub(yh, yl, 0, nsw, hh, ll);
                        ty = (double)hh + (double)ll;
                    }
                    ox = sqrt(tx * tx + ty * ty);
                    oy = sqrt((c1x - c0x) * (c1x - c0x) + (c1y - c0y) * (c1y - c0y));
                } else {
                    // head-centre velocity over the observation interval (Sec. 4.1)
                    double cx, cy;
                    head_centre<F64>(sx, sy, xh, xl, yh, yl, nf, nh, lane, cx, cy);
                    const double inv = 1.0 / ((double)a.obs_every * a.dt);
                    ox = (cx - s_model[M_CX]) * inv;
                    oy = (cy - s_model[M_CY]) * inv;
                    __syncwarp();
                    if (tid == 0) {
                        s_model[M_CX] = cx;
                        s_model[M_CY] = cy;
                    }
                }
                if (tid == 0) {
                    const long long o = obs_idx;
                    if (a.obs) {
                        const double rx = a.obs[2 * o] - ox, ry = (a.obs[2 * o + 1] - oy) / a.sigma_ratio;
                        J = fma(rx, rx, fma(ry, ry, J));
                    }
                    if (a.head_traj) {
                        a.head_traj[((size_t)b * n_obs + o) * 2] = ox;
                        a.head_traj[((size_t)b * n_obs + o) * 2 + 1] = oy;
                    }
                }
            }
            if (obs_step) {
                obs_left = obs_every;
                ++obs_idx;
            }
        }
        // ---- outputs
        if (a.final_state) {  // rows past the sample's points, or of a run that stopped: NaN
            const int k0 = status == SWIMMER_OK ? n : 0;
            for (int k = k0 + tid; k < n_max; k += T)
                for (int c = 0; c < 4; ++c) a.final_state[((size_t)b * n_max + k) * 4 + c] = nan("");
        }
        if (a.speed && tid < 32) {
            // mean speed: x-displacement of the flagellum's centroid (which starts at 0 in the
            // stored coordinates) or, with a head, of the head centre, over the run's duration;
            // one warp sums in a fixed order
            // (the first swimmer's, with two)
            const int k0 = nh > 0 ? nf : 0;
            double cx = 0.0;
            for (int k = k0 + lane; k < nsw; k += 32) cx += F64 ? sx[k] : (double)xh[k] + (double)xl[k];
            for (int o = 16; o >= 1; o >>= 1) cx += __shfl_xor_sync(0xffffffffu, cx, o);
            if (tid == 0) {
                const double c0 = nh > 0 ? L + (a.gap_over_ds + a.hr_over_ds) * ds - xref : 0.0;
                a.speed[b] = status == SWIMMER_OK ? (cx / (nsw - k0) - c0) / (a.steps * a.dt) : nan("");
            }
        }
        if (tid == 0) {
            unsigned long long wk = (unsigned long long)n * (unsigned long long)n * (unsigned long long)steps_done;
            atomicAdd(a.work, wk);
            if (a.speculative)
                a.run_work[b] = wk;
            else
                atomicAdd(a.work + 1, wk);
        }
        if (head_thread) {
            a.status[b] = status;
            if (a.loglik) {
                // Sigma = diag(sigma^2, (sigma_ratio sigma)^2) per observation (Sec. 3.1; two
                // noise levels, Sec. 4.2): residuals of the second component are divided by
                // sigma_ratio in J
                const double sg = a.sigma * p.sig;  // the sample's noise level
                double s2 = sg * sg;
                a.loglik[b] = status == SWIMMER_OK
                                  ? -(double)n_obs * (log(2.0 * PI * s2) + log(a.sigma_ratio)) - 0.5 * J / s2
                                  : -INFINITY;
            }
            if (status != SWIMMER_OK && a.head_traj) {
                // observations after the divergence were never taken
                for (long long o = steps_done / a.obs_every; o < n_obs; ++o) {
                    a.head_traj[((size_t)b * n_obs + o) * 2] = nan("");
                    a.head_traj[((size_t)b * n_obs + o) * 2 + 1] = nan("");
                }
            }
        }
        __syncthreads();
    }
}

typedef void (*ForwardKernel)(FwdArgs);

ForwardKernel forward_kernel_for(bool f64, const swimmer_config &c, bool big = false) {
    const int model = c.n_swimmers == 2 ? 2 : c.n_head > 0 ? 1 : 0;
    if (f64) return model == 2 ? forward_kernel<true, 2> : model == 1 ? forward_kernel<true, 1> : forward_kernel<true, 0>;
    if (big)
        return model == 2 ? forward_kernel<false, 2, true>
               : model == 1 ? forward_kernel<false, 1, true>
                            : forward_kernel<false, 0, true>;
    return model == 2 ? forward_kernel<false, 2> : model == 1 ? forward_kernel<false, 1> : forward_kernel<false, 0>;
}

}  // namespace

// The pair-unit list of nb blocks (packing and order as swimmer_pair_units documents).
// Multi-target lists group the off-diagonal block pairs (edges of the complete graph on the
// blocks) around a shared block: blocks are visited from the last down, each takes its edges
// to lower blocks plus those handed to it, and when their number is odd it hands one edge to
// a lower block whose own count would otherwise be odd, so at most one edge stays alone, at
// block 0.  Mode 2 (from 8 blocks on) hands edges down until a block's count is a multiple of
// four (as far as its own edges to lower blocks allow) and takes them four at a time, the rest
// in pairs and alone.
static std::vector<unsigned> build_pair_units(int nb, int mode) {
    // below 8 blocks the edges of a block are too few to form four-target units; there mode 2
    // takes the two-target list
    if (mode == 2 && nb < 8) mode = 1;
    std::vector<unsigned> out;
    if (mode == 0) {
        for (int i = 0; i < nb; ++i) out.push_back(unit_pack(0, 2, i, i));
        // off-diagonal block pairs in circulant order: {r, r + k} for k = 1 .. (nb - 1) / 2,
        // then {r, r + nb / 2} for r < nb / 2 (even nb)
        for (int k = 1; k <= (nb - 1) / 2; ++k)
            for (int r = 0; r < nb; ++r)
                for (int c = 0; c < 2; ++c) out.push_back(unit_pack(0, c, (r + k) % nb, r));
        if (nb % 2 == 0)
            for (int r = 0; r < nb / 2; ++r)
                for (int c = 0; c < 2; ++c) out.push_back(unit_pack(0, c, r + nb / 2, r));
        return out;
    }
    std::vector<std::vector<int>> handed(nb);
    std::vector<unsigned> quad, pair, single;
    for (int J = nb - 1; J >= 0; --J) {
        std::vector<int> other;  // the other blocks of the edges grouped at J
        for (int i = 0; i < J; ++i) other.push_back(i);
        for (int x : handed[J]) other.push_back(x);
        if (mode == 1 && other.size() % 2 == 1 && J > 0) {
            int pick = 0;
            for (int i = J - 1; i >= 0; --i)
                if ((i + handed[i].size()) % 2 == 1) {
                    pick = i;
                    break;
                }
            other.erase(std::find(other.begin(), other.end(), pick));
            handed[pick].push_back(J);
        }
        // mode 2: hand edges down until the count is a multiple of four, each to the lower
        // block whose own count comes closest to a multiple of four by it
        for (int hand = mode == 2 && J > 0 ? (int)(other.size() % 4) : 0; hand > 0; --hand) {
            int pick = -1, best = -1;
            for (int i = J - 1; i >= 0; --i) {
                if (std::find(other.begin(), other.end(), i) == other.end()) continue;  // handed already
                const int score = (int)((i + handed[i].size()) % 4);  // 3 is best: +1 makes 0 mod 4
                if (score > best) {
                    best = score;
                    pick = i;
                }
            }
            if (pick < 0) break;
            other.erase(std::find(other.begin(), other.end(), pick));
            handed[pick].push_back(J);
        }
        size_t k = 0;
        if (mode == 2)
            for (; k + 3 < other.size(); k += 4)
                for (int c = 0; c < 2; ++c)
                    quad.push_back(unit_pack(2, c, J, other[k], other[k + 1], other[k + 2], other[k + 3]));
        for (; k + 1 < other.size(); k += 2)
            for (int c = 0; c < 2; ++c) pair.push_back(unit_pack(1, c, J, other[k], other[k + 1]));
        if (k < other.size())
            for (int c = 0; c < 2; ++c) single.push_back(unit_pack(0, c, J, other[k]));
    }
    out.insert(out.end(), quad.begin(), quad.end());
    out.insert(out.end(), pair.begin(), pair.end());
    out.insert(out.end(), single.begin(), single.end());
    for (int i = 0; i < nb; ++i) out.push_back(unit_pack(0, 2, i, i));
    return out;
}

extern "C" int swimmer_pair_units(int nb, int mode, unsigned *out, int *count) {
    ARG_CHECK(nb >= 1 && nb <= UNIT_NB_MAX, "nb must be in [1, %d]", UNIT_NB_MAX);
    ARG_CHECK(mode >= 0 && mode < UNIT_MODES, "mode must be 0, 1 or 2");
    ARG_CHECK(out != nullptr && count != nullptr, "out or count is NULL");
    const std::vector<unsigned> u = build_pair_units(nb, mode);
    std::copy(u.begin(), u.end(), out);
    *count = (int)u.size();
    return 0;
}

// Device copy of every mode's lists for every block count up to the handle's n_max.
int upload_pair_units(swimmer_handle *h) {
    const int nbm = (h->cfg.n_max + 31) / 32;
    std::vector<unsigned> all(UNIT_HDR, 0u), body;
    for (int m = 0; m < UNIT_MODES; ++m) {
        for (int nb = 1; nb <= nbm; ++nb) {
            const std::vector<unsigned> u = build_pair_units(nb, m);
            if ((int)u.size() > nb * nb) {
                set_error("pair-unit list of %d blocks has %zu units", nb, u.size());
                return SWIMMER_E_ARG;
            }
            all[m * (UNIT_NB_MAX + 1) + nb - 1] = (unsigned)body.size();
            body.insert(body.end(), u.begin(), u.end());
        }
        all[m * (UNIT_NB_MAX + 1) + nbm] = (unsigned)body.size();
    }
    all.insert(all.end(), body.begin(), body.end());
    CUDA_TRY(cudaMalloc((void **)&h->units, sizeof(unsigned) * all.size()));
    CUDA_TRY(cudaMemcpy(h->units, all.data(), sizeof(unsigned) * all.size(), cudaMemcpyHostToDevice));
    return 0;
}

// Threads per sample: at least one per target (FP64) or one warp per pair unit (FP32);
// more when the batch is too small to fill the GPU, so that the per-step latency of a lone
// sample shrinks, as long as the shared memory fits; FP32 pair units as measured best for
// the sample size.  The autotuned choice wins.
bool forward_fits(const swimmer_handle *h, int threads, int precision) {
    const bool f64 = precision == SWIMMER_FP64;
    const int P = handle_octaves(h) * (f64 ? F64_SUB : F32_SUB);
    size_t smem = f64 ? smem_bytes<true>(h->cfg.n_max, P, threads) : smem_bytes<false>(h->cfg.n_max, P, threads);
    return smem + 1024 <= (size_t)h->max_smem;  // static shared memory of the kernel
}

// Samples the forward kernel holds at once on the device at its smallest launch shape (the
// most resident samples); at least one per SM.
int forward_slots(const swimmer_handle *h, int precision) {
    const bool f64 = precision == SWIMMER_FP64;
    const int T = forward_min_threads(h, precision);
    const int P = handle_octaves(h) * (f64 ? F64_SUB : F32_SUB);
    size_t smem = f64 ? smem_bytes<true>(h->cfg.n_max, P, T) : smem_bytes<false>(h->cfg.n_max, P, T);
    auto kern = forward_kernel_for(f64, h->cfg);
    int per_sm = 0;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();  // clear the error state a failed query leaves
        per_sm = 1;
    }
    return per_sm * h->num_sms;
}

// Launch-shape bucket of a batch: samples per SM, ceil(B / SMs) - 1, capped at 16.  The
// persistent kernel's time is set by how many samples each SM holds.
int tune_bucket(const swimmer_handle *h, int B) {
    const long long per_sm = ((long long)B + h->num_sms - 1) / h->num_sms;
    return (int)(per_sm < 1 ? 0 : (per_sm > 17 ? 16 : per_sm - 1));
}

// Smallest launch shape: FP64 needs a thread per target, FP32 a few warps for the O(N) phases.
int forward_min_threads(const swimmer_handle *h, int precision) {
    int T = 128;
    if (precision == SWIMMER_FP64)
        while (T < h->cfg.n_max && T < 1024) T <<= 1;
    return T;
}

int forward_threads(const swimmer_handle *h, int B, int precision) {
    const int bucket = tune_bucket(h, B);
    const int tuned = h->tune_threads[precision == SWIMMER_FP64 ? 0 : 1][bucket];
    const int tT = tuned & SHAPE_THREADS;
    int T = forward_min_threads(h, precision);
    if (tT >= T && tT <= 1024 && forward_fits(h, tT, precision)) return tuned;
    int cap = 1024;
    if (precision != SWIMMER_FP64) {  // warps beyond the pair units only help the O(N) phases
        const int nbm = (h->cfg.n_max + 31) / 32;
        while (cap > T && cap / 2 >= 32 * nbm * nbm) cap /= 2;
    }
    while (T < cap && (long long)B * T * 2 <= (long long)h->num_sms * 1024 && forward_fits(h, 2 * T, precision))
        T <<= 1;
    // two-target units (measured): from 8 blocks of 32 points at every thread count, and from 4
    // blocks when the batch fills the GPU (the heuristic stays at 128 threads only then)
    const int nbm = (h->cfg.n_max + 31) / 32;
    if (precision != SWIMMER_FP64 && (nbm >= 8 || (nbm >= 4 && T == 128))) return T | SHAPE_WIDE;
    return T;
}

int launch_forward(swimmer_handle *h, int B, const double *obs, double sigma, double *loglik,
                   double *head_traj, double *mean_speed, int *status, int precision, cudaStream_t s,
                   int threads_override, int speculative, double *final_state, int max_runs) {
    FwdArgs a;
    a.B = B;
    a.sp = h->sp;
    a.order = h->order;
    a.queue = h->queue;
    a.tab64 = h->tab64;
    a.tab32 = h->tab32;
    a.pq = h->pq;
    a.mu = h->cfg.mu;
    a.dt = h->cfg.dt;
    a.kt = h->cfg.k_t;
    a.hr_over_ds = head_radius_over_ds(h->cfg);
    a.gap_over_ds = neck_gap_over_ds(h->cfg);
    a.k_head_tens = h->cfg.k_head_tens;
    a.k_head_c = h->cfg.k_head_c;
    a.k_neck_tens = h->cfg.k_neck_tens;
    a.k_neck_ang = h->cfg.k_neck_ang;
    a.obs_kind = h->cfg.obs_kind;
    a.swim_d = h->cfg.swimmer_distance;
    a.sigma_ratio = h->cfg.sigma_ratio > 0.0 ? h->cfg.sigma_ratio : 1.0;
    a.eta = h->cfg.eta;
    a.omega = h->cfg.omega;
    a.steps = h->cfg.steps;
    a.obs_every = h->cfg.obs_every;
    a.obs = obs;
    a.sigma = sigma;
    a.loglik = loglik;
    a.head_traj = head_traj;
    a.speed = mean_speed;
    a.final_state = final_state;
    a.status = status;
    a.work = h->work;
    a.run_work = h->run_work;
    a.speculative = speculative;
    a.n_max = h->cfg.n_max;
    const int shape = threads_override > 0 ? threads_override : forward_threads(h, B, precision);
    const int T = shape & SHAPE_THREADS;
    a.threads = T;
    const bool f64 = precision == SWIMMER_FP64;
    a.units = h->units;
    a.mode = f64 ? 0 : (shape & SHAPE_QUAD) ? 2 : (shape & SHAPE_WIDE) ? 1 : 0;
    a.tab_panels = handle_octaves(h) * (f64 ? F64_SUB : F32_SUB);
    size_t smem = f64 ? smem_bytes<true>(a.n_max, a.tab_panels, T) : smem_bytes<false>(a.n_max, a.tab_panels, T);
    auto kern = forward_kernel_for(f64, h->cfg);
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  cudaSharedmemCarveoutMaxShared));
    int per_sm = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, T, smem));
    // CTAs per SM: no more than the launch has runs per SM.  A speculative launch over B rows of
    // which at most max_runs are real (the others skip as bad samples, queued last) counts
    // those: the real runs, queued first, are then taken one per CTA as the CTAs start, spread
    // over the SMs, instead of landing two or three on some SMs
    const int runs = max_runs > 0 && max_runs < B ? max_runs : B;
    if (per_sm > 1) per_sm = min(per_sm, (runs + h->num_sms - 1) / h->num_sms);
    // FP32 with shared memory for so few threads per SM that each could hold 128 registers:
    // the instantiation compiled for that register budget (same CTAs per SM)
    // (with the table as 32-byte records, if that still fits)
    const size_t smem_big = smem_bytes<false, true>(a.n_max, a.tab_panels, T);
    if (!f64 && T <= 512 && per_sm >= 1 && (long long)per_sm * T * 128 <= h->regs_per_sm &&
        smem_big + 1024 <= (size_t)h->max_smem) {
        auto big = forward_kernel_for(f64, h->cfg, true);
        int per_big = 0;
        CUDA_TRY(cudaFuncSetAttribute(big, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_big));
        CUDA_TRY(cudaFuncSetAttribute(big, cudaFuncAttributePreferredSharedMemoryCarveout,
                                      cudaSharedmemCarveoutMaxShared));
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_big, big, T, smem_big));
        if (per_big >= per_sm) {
            kern = big;
            smem = smem_big;
        }
    }
    // four-target units need the 128-register budget; elsewhere the launch runs two-target ones
    if (a.mode == 2 && kern == forward_kernel_for(f64, h->cfg)) a.mode = 1;
    if (per_sm < 1) {
        set_error("forward kernel does not fit on an SM (threads %d, smem %zu)", T, smem);
        return SWIMMER_E_CUDA;
    }
    int grid = per_sm * h->num_sms;
    if (grid > B) grid = B;
    CUDA_TRY(cudaMemsetAsync(h->queue, 0, sizeof(int), s));
    prof_k2_begin(h, s, B);
    kern<<<grid, T, smem, s>>>(a);
    CUDA_TRY(cudaGetLastError());
    prof_k2_end(h, s);
    prof_count(h, 1);
    return 0;
}
