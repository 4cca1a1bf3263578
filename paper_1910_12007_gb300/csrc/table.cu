// K1: per-sample tables of the regularized Brinkmanlet kernel functions (FP64 build).
//
// For each sample (alpha, delta) this builds, on the device,
//   g1(r) = B''(r),  g2(r) = (r B''(r) - B'(r))/r^3     (Sec. 2.1, Eq. BrV)
// with (Lap - alpha^2) B = G and Lap G = phi_delta (Eq. eqnblob).  With
//   M0(r) = int_0^r phi s ds = (1 - delta^3/R^3)/(2 pi)            (closed form)
//   A1(r) = int_0^r (I0(alpha s) - 1) phi s ds
//   C(r)  = int_r^inf K0(alpha s) phi s ds
// and x = alpha r, the solution of the radial problem by variation of parameters
// (Green's function -K0(alpha |x|)/(2 pi), averaged over circles) gives
//   g1 = [1/x^2 - W] M0 - W A1 - (I0 + I2) C / 2,             W = (K0 + K2)/2
//   g2 = [(2/x^2 - K2) M0 - K2 A1 - I2 C] / r^2
// where the bracketed differences are evaluated from their power series for x <= 2.
// alpha = 0 is the regularized Stokeslet in closed form (Cortez 2001).
//
// Numerics (all FP64): Bessel I by power series (x <= 30) or the Hankel asymptotic
// series; Bessel K by the A&S 9.6.11/9.6.13 series for x <= 2 and otherwise by the
// trapezoid rule on K_nu(x) e^x = int_0^inf exp(-x (cosh t - 1)) cosh(nu t) dt, whose
// error decays like exp(-2 pi d/h) for the strip half-width d = acos(1 - 1/x).  A1 and C
// at the table nodes come from 16-point Gauss-Legendre integrals between consecutive
// nodes, a warp prefix (A1) / suffix (C) sum and a geometric tail for C.
//
// Output per sample: FP64 Chebyshev coefficients (8 panels per octave of
// u = 1 + r^2/delta^2, degree 9) and, derived from them, FP32 quadratic coefficients in
// the mantissa F in [1, 2) of u (64 panels per octave).
#include <math.h>
#include <stdio.h>

#include <mutex>

#include "common.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double EGAMMA = 0.57721566490153286061;
constexpr int GL_N = 16;
__constant__ double c_gl_x[GL_N];   // 16-point Gauss-Legendre on [-1, 1]
__constant__ double c_gl_w[GL_N];
__constant__ double c_gl8_x[8];     // 8-point rule (FP32 handles: the table only feeds FP32)
__constant__ double c_gl8_w[8];
constexpr int NSER = 160;
__constant__ double c_inv_k[NSER];          // 1/k (index 0 unused)
__constant__ double c_inv_kk[2][NSER];      // 1/((k+1)(k+1+nu)) for nu = 0, 2
__constant__ double c_cheb_t[F64_NODES];    // ascending Chebyshev nodes of the FP64 panels
__constant__ double c_dct[F64_NODES][F64_NODES];  // (2/n) cos(pi k (i + 1/2)/n), k = 0 halved
// FP32 handles: the intermediate FP64 table needs only ~1e-9 (it feeds an FP32 table), so
// its panels carry degree-5 series fitted at 6 nodes
constexpr int LITE_NODES = 6;
__constant__ double c_cheb_t6[LITE_NODES];
__constant__ double c_dct6[LITE_NODES][LITE_NODES];
__constant__ double c_node3[3];             // Chebyshev nodes for the FP32 quadratic fit
__constant__ double c_dct3[3][3];

// ---------------------------------------------------------------------------------
// Bessel functions
// ---------------------------------------------------------------------------------
// I_nu(x), nu in {0, 2}: power series for x <= 30, Hankel asymptotic expansion beyond.
__device__ double bessel_i(int nu, double x) {
    if (x <= 30.0) {
        double y = 0.25 * x * x;
        double term = nu == 0 ? 1.0 : 0.5;  // 1/nu!
        const double *inv = c_inv_kk[nu == 0 ? 0 : 1];
        double s = 0.0;
        for (int k = 0; k < NSER; ++k) {
            s += term;
            term *= y * inv[k];
            if (term < 1e-18 * s) break;
        }
        return s * (nu == 0 ? 1.0 : y);  // (x/2)^2 = y for nu = 2
    }
    double mu = 4.0 * nu * nu;
    double s = 1.0, term = 1.0, inv8x = 0.125 / x;
    for (int k = 1; k < 60; ++k) {
        double a = (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) * c_inv_k[k] * inv8x;
        double nt = -term * a;
        if (fabs(nt) > fabs(term)) break;
        term = nt;
        s += term;
        if (fabs(term) < 1e-18 * fabs(s)) break;
    }
    return exp(x) / sqrt(2.0 * PI * x) * s;
}

// I0(x) - 1 without cancellation
__device__ double bessel_i0m1(double x) {
    if (x > 1.0) return bessel_i(0, x) - 1.0;
    double y = 0.25 * x * x, term = y, s = 0.0;
    for (int k = 1; k < 60; ++k) {
        s += term;
        term *= y * c_inv_kk[0][k];  // 1/((k+1)^2)
        if (term < 1e-18 * s) break;
    }
    return s;
}

struct BesselSet {
    double i0, i2, k0, k2, t2k2, ix2w;  // t2k2 = 2/x^2 - K2, ix2w = 1/x^2 - (K0+K2)/2
};

// K0(x) e^x and K1(x) e^x for x > 2 by the trapezoid rule on the integral representation
__device__ void bessel_k01_scaled(double x, double *k0e, double *k1e) {
    double d = acos(1.0 - 1.0 / x);
    double h = d / 6.5;
    double s0 = 0.5, s1 = 0.5;
    const double eh = exp(h), emh = 1.0 / eh;
    double ep = 1.0, em = 1.0;  // e^{m h}, e^{-m h}
    for (int m = 1; m < 4000; ++m) {
        ep *= eh;
        em *= emh;
        double c = 0.5 * (ep + em);  // cosh(m h)
        double e = exp(-x * (c - 1.0));
        s0 += e;
        s1 += e * c;
        if (e < 1e-19 * s0) break;
    }
    *k0e = h * s0;
    *k1e = h * s1;
}

__device__ BesselSet bessel_set(double x) {
    BesselSet b;
    b.i0 = bessel_i(0, x);
    b.i2 = bessel_i(2, x);
    if (x <= 2.0) {
        double y = 0.25 * x * x;
        double lx = log(0.5 * x) + EGAMMA;
        // K0 = -lx I0 + sum_{k>=1} H_k y^k/(k!)^2
        double term = 1.0, hk = 0.0, tail = 0.0;
        for (int k = 1; k < 60; ++k) {
            term *= y * c_inv_kk[0][k - 1];  // 1/k^2
            hk += c_inv_k[k];
            tail += hk * term;
            if (term < 1e-19) break;
        }
        b.k0 = -lx * b.i0 + tail;
        // 2/x^2 - K2 = 1/2 + y sum_k [lx - (H_k + H_{k+2})/2] y^k/(k!(k+2)!)
        double s = 0.0;
        term = 0.5;
        double hk0 = 0.0, hk2 = 1.5;  // H_0, H_2
        for (int k = 0; k < 60; ++k) {
            s += (lx - 0.5 * (hk0 + hk2)) * term;
            term *= y * c_inv_kk[1][k];  // 1/((k+1)(k+3))
            hk0 += c_inv_k[k + 1];
            hk2 += c_inv_k[k + 3];
            if (term < 1e-20) break;
        }
        b.t2k2 = 0.5 + y * s;
        b.k2 = 2.0 / (x * x) - b.t2k2;
        b.ix2w = 0.5 * b.t2k2 - 0.5 * b.k0;
    } else {
        double k0e, k1e;
        bessel_k01_scaled(x, &k0e, &k1e);
        double ex = exp(-x);
        b.k0 = k0e * ex;
        double k1 = k1e * ex;
        b.k2 = b.k0 + 2.0 * k1 / x;
        b.t2k2 = 2.0 / (x * x) - b.k2;
        b.ix2w = 1.0 / (x * x) - 0.5 * (b.k0 + b.k2);
    }
    return b;
}

__device__ double bessel_k0(double x) {
    if (x <= 2.0) {
        // K0 = -(ln(x/2) + gamma) I0 + sum_{k>=1} H_k y^k/(k!)^2, y = x^2/4 (one pass)
        double y = 0.25 * x * x, term = 1.0, i0 = 1.0, hk = 0.0, tail = 0.0;
        for (int k = 1; k < 60; ++k) {
            term *= y * c_inv_kk[0][k - 1];
            hk += c_inv_k[k];
            i0 += term;
            tail += hk * term;
            if (term < 1e-19 * i0) break;
        }
        return -(log(0.5 * x) + EGAMMA) * i0 + tail;
    }
    double k0e, k1e;
    bessel_k01_scaled(x, &k0e, &k1e);
    return k0e * exp(-x);
}

// ---------------------------------------------------------------------------------
// integrands and panel integrals
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double blob(double s, double delta) {
    double R2 = s * s + delta * delta;
    return 3.0 * delta * delta * delta / (2.0 * PI * R2 * R2 * sqrt(R2));
}

__device__ double m0_closed(double r, double delta) {
    double R = sqrt(r * r + delta * delta);
    return (r * r / (R + delta)) * (R * R + R * delta + delta * delta) / (R * R * R) / (2.0 * PI);
}

// int_a^b f(s) ds with f = (I0(alpha s)-1) phi s (which = 0) or K0(alpha s) phi s (which = 1),
// split so that no piece is wider than 0.5/alpha or half the distance scale max(a, delta/4)
__device__ double panel_integral(int which, double a, double b, double alpha, double delta, bool gl8) {
    if (b <= a) return 0.0;
    double w = b - a;
    int n = (int)ceil(fmax(alpha * w / 0.5, w / (0.5 * fmax(a, 0.25 * delta))));
    if (n < 1) n = 1;
    if (n > 4096) n = 4096;
    const int ng = gl8 ? 8 : GL_N;
    const double *gx = gl8 ? c_gl8_x : c_gl_x, *gw = gl8 ? c_gl8_w : c_gl_w;
    double hw = 0.5 * w / n, tot = 0.0;
    for (int p = 0; p < n; ++p) {
        double c = a + (2 * p + 1) * hw, acc = 0.0;
        for (int g = 0; g < ng; ++g) {
            double s = c + hw * gx[g];
            double f = (which == 0 ? bessel_i0m1(alpha * s) : bessel_k0(alpha * s)) * blob(s, delta) * s;
            acc += gw[g] * f;
        }
        tot += acc * hw;
    }
    return tot;
}

__device__ __forceinline__ double node_u(int m, int np) {
    // node m -> (octave, panel, ascending Chebyshev index); np nodes per panel
    int panel = m / np, ii = m % np;
    int e = panel >> F64_SUB_LOG2, j = panel & (F64_SUB - 1);
    double f = 0.5 * ((np == F64_NODES ? c_cheb_t[ii] : c_cheb_t6[ii]) + 1.0);
    return ldexp(1.0 + (j + f) / F64_SUB, e);
}

__device__ void stokes_g(double r, double delta, double *g1, double *g2) {
    double R = sqrt(r * r + delta * delta);
    *g1 = (log(R + delta) - delta * (R + 2.0 * delta) / (R * (R + delta))) / (4.0 * PI);
    *g2 = (R + 2.0 * delta) / (4.0 * PI * R * (R + delta) * (R + delta));
}

// ---------------------------------------------------------------------------------
// per-sample parameters from theta
// ---------------------------------------------------------------------------------
__global__ void prepare_kernel(int B, const double *__restrict__ theta, const int *__restrict__ n_pts,
                               swimmer_config cfg, SampleParams *__restrict__ sp, int *__restrict__ order) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    SampleParams p;
    p.n = n_pts ? n_pts[b] : default_flagellum_points(cfg);
    p.nh = cfg.n_head;
    const int np = n_params(cfg);
    p.alpha = theta[np * b + 0];
    p.kc = pow(10.0, theta[np * b + 1]);
    p.amp = theta[np * b + 2];
    p.sig = np == 4 ? theta[np * b + 3] : 1.0;
    p.length = cfg.ds_fixed > 0.0 ? (p.n - 1) * cfg.ds_fixed : cfg.length;
    p.status = SWIMMER_OK;
    if (p.n < 3 || (cfg.n_swimmers == 2 ? 2 : 1) * (p.n + p.nh) > cfg.n_max) {
        p.n = 3;
        p.status = SWIMMER_BAD_SAMPLE;
    }
    p.ds = p.length / (p.n - 1);
    p.delta = cfg.delta_over_ds * p.ds;
    double rho = R_MAX_OVER_L * sample_reach(cfg, p.n, p.ds) / p.delta;  // r_max/delta, as handle_octaves()
    int n_oct = (int)floor(log2(1.0 + rho * rho)) + 1;
    if (n_oct > N_OCT_MAX) {
        n_oct = N_OCT_MAX;
        p.status = SWIMMER_BAD_SAMPLE;
    }
    p.n_oct = n_oct;
    if (!(p.sig > 0.0) || !isfinite(p.sig)) p.status = SWIMMER_BAD_SAMPLE;
    if (!(p.alpha >= 0.0) || p.alpha * R_MAX_OVER_L * sample_reach(cfg, p.n, p.ds) > X_MAX || !isfinite(p.kc) ||
        !isfinite(p.amp) || !(p.kc > 0.0))
        p.status = SWIMMER_BAD_SAMPLE;
    sp[b] = p;
    order[b] = b;
}

// Longest-first processing order for the persistent work queue (the classic LPT rule):
// batches of uneven size by n, largest first (a run costs n^2 per step); batches of one size
// by ascending bending stiffness K_C, whose growth lowers forward Euler's stability limit, so
// that the runs likely to stop early (DIVERGED) come last and the queue, which deals runs to
// the SMs in turn, spreads them over the SMs.  Counting sort in one CTA (log10 K_C in 1024
// buckets over [-5, 5]); samples with a bad status go last (they do no work).
constexpr int SORT_THREADS = 1024;
__device__ __forceinline__ int order_key(const SampleParams &p, bool by_kc) {
    if (p.status != SWIMMER_OK) return N_PTS_MAX + 1;
    if (by_kc) return min(max((int)floor((log10(p.kc) + 5.0) * 102.4), 0), N_PTS_MAX);
    return N_PTS_MAX + 1 - min(max(p.n, 0), N_PTS_MAX);
}
__global__ void __launch_bounds__(SORT_THREADS) order_kernel(int B, const SampleParams *__restrict__ sp,
                                                           int *__restrict__ order, int by_kc) {
    __shared__ int cnt[N_PTS_MAX + 2];
    __shared__ int start[N_PTS_MAX + 2];
    const int tid = threadIdx.x;
    for (int i = tid; i < N_PTS_MAX + 2; i += SORT_THREADS) cnt[i] = 0;
    __syncthreads();
    for (int b = tid; b < B; b += SORT_THREADS) atomicAdd(&cnt[order_key(sp[b], by_kc)], 1);
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int k = 0; k < N_PTS_MAX + 2; ++k) {
            start[k] = acc;
            acc += cnt[k];
        }
    }
    __syncthreads();
    for (int b = tid; b < B; b += SORT_THREADS) order[atomicAdd(&start[order_key(sp[b], by_kc)], 1)] = b;
}

// ---------------------------------------------------------------------------------
// K1a: interval integrals, one thread per node interval or tail piece (all samples)
// ---------------------------------------------------------------------------------
constexpr int K1_THREADS = 256;
constexpr int K1A_THREADS = 128;

__device__ __forceinline__ int node_count(const SampleParams &p, int NP, int max_oct) {
    return min(p.n_oct, max_oct) * F64_SUB * NP;
}

// tail piece k beyond r_last: widths double from the blob scale up to 2/alpha, then stay;
// the last piece ends at s_end.  Returns false when piece k does not exist.
__device__ bool tail_piece(int k, double r_last, double s_end, double alpha, double delta, double *lo, double *hi) {
    double s = r_last;
    for (int i = 0; i < TAIL_MAX; ++i) {
        if (s >= s_end) return false;
        double w = fmin(fmax(s, 0.25 * delta), 2.0 / alpha);
        double e = (i == TAIL_MAX - 1) ? s_end : fmin(s + w, s_end);
        if (i == k) {
            *lo = s;
            *hi = e;
            return true;
        }
        s = e;
    }
    return false;
}

__global__ void __launch_bounds__(K1A_THREADS)
table_integrals_kernel(int B, const SampleParams *__restrict__ sp, double *__restrict__ scratch, int gl8,
                       int max_oct) {
    const int b = blockIdx.x;
    const SampleParams p = sp[b];
    if (p.status != SWIMMER_OK || !(p.alpha > 0.0)) return;
    const int NP = gl8 ? LITE_NODES : F64_NODES;
    const int M = node_count(p, NP, max_oct);
    const int q = blockIdx.y * blockDim.x + threadIdx.x;
    const double alpha = p.alpha, delta = p.delta;
    double *IA = scratch + (size_t)b * K1_SCRATCH, *IC = IA + NODES_MAX, *IT = IC + NODES_MAX;
    if (q < M) {
        double r = delta * sqrt(node_u(q, NP) - 1.0);
        double rprev = q ? delta * sqrt(node_u(q - 1, NP) - 1.0) : 0.0;
        IA[q] = panel_integral(0, rprev, r, alpha, delta, gl8);
        IC[q] = q + 1 < M ? panel_integral(1, r, delta * sqrt(node_u(q + 1, NP) - 1.0), alpha, delta, gl8) : 0.0;
    } else if (q < M + TAIL_MAX) {
        const int k = q - M;
        double r_last = delta * sqrt(node_u(M - 1, NP) - 1.0);
        double s_end = fmin(r_last + 60.0 / alpha, 1e6 * delta);
        double lo, hi;
        IT[k] = tail_piece(k, r_last, s_end, alpha, delta, &lo, &hi) ? panel_integral(1, lo, hi, alpha, delta, gl8) : 0.0;
    }
}

// ---------------------------------------------------------------------------------
// K1b: per sample (one CTA): prefix/suffix sums, node values, Chebyshev and FP32 fits
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(K1_THREADS)
table_build_kernel(int B, SampleParams *__restrict__ sp, const double *__restrict__ scratch,
                   double *__restrict__ tab64, float4 *__restrict__ tab32, int gl8, int max_oct) {
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    if (b >= B) return;
    SampleParams p = sp[b];
    if (p.n_oct > max_oct) {  // never beyond the shared-memory node arrays
        p.n_oct = max_oct;
        __syncthreads();
        if (threadIdx.x == 0) sp[b].n_oct = max_oct;
    }
    const int NP = gl8 ? LITE_NODES : F64_NODES;  // nodes per FP64 panel
    const int M = p.n_oct * F64_SUB * NP;
    double *nodeA = sm;            // [M] interval integrals -> A1 prefix
    double *nodeC = sm + M;        // [M] interval integrals -> C suffix
    double *g1s = sm + 2 * M;      // [M]
    double *g2s = sm + 3 * M;      // [M]
    const int tid = threadIdx.x;
    const double alpha = p.alpha, delta = p.delta;
    const bool stokes = !(alpha > 0.0);
    double *t64 = tab64 + (size_t)b * TAB64_STRIDE;
    float4 *t32 = tab32 + (size_t)b * TAB32_STRIDE;

    if (p.status != SWIMMER_OK) {
        // keep the tables finite so that a stray read cannot produce garbage
        for (int i = tid; i < TAB64_STRIDE; i += blockDim.x) t64[i] = 0.0;
        for (int i = tid; i < TAB32_STRIDE; i += blockDim.x) t32[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }

    if (!stokes) {
        const double *IA = scratch + (size_t)b * K1_SCRATCH, *IC = IA + NODES_MAX, *IT = IC + NODES_MAX;
        for (int m = tid; m < M; m += blockDim.x) {
            nodeA[m] = IA[m];
            nodeC[m] = IC[m];
        }
        __syncthreads();
        if (tid == 0) {
            double tail = 0.0;
            for (int k = TAIL_MAX - 1; k >= 0; --k) tail += IT[k];  // far (small) pieces first
            nodeC[M - 1] = tail;
        }
        __syncthreads();
        // prefix (A1) and suffix (C) sums by warp 0: lanes own contiguous chunks
        if (tid < 32) {
            int chunk = (M + 31) / 32;
            int lo = tid * chunk, hi = min(M, lo + chunk);
            double sa = 0.0, sc = 0.0;
            for (int m = lo; m < hi; ++m) sa += nodeA[m];
            for (int m = lo; m < hi; ++m) sc += nodeC[m];
            // exclusive scans of the chunk totals (A: from the left, C: from the right)
            double pa = sa, pc = sc;
            for (int o = 1; o < 32; o <<= 1) {
                double va = __shfl_up_sync(0xffffffffu, pa, o);
                double vc = __shfl_down_sync(0xffffffffu, pc, o);
                if (tid >= o) pa += va;
                if (tid + o < 32) pc += vc;
            }
            double offa = pa - sa, offc = pc - sc;
            double run = offa;
            for (int m = lo; m < hi; ++m) {
                run += nodeA[m];
                nodeA[m] = run;
            }
            run = offc;
            for (int m = hi - 1; m >= lo; --m) {
                run += nodeC[m];
                nodeC[m] = run;
            }
        }
        __syncthreads();
    }

    // kernel function values at the nodes
    for (int m = tid; m < M; m += blockDim.x) {
        double r = delta * sqrt(node_u(m, NP) - 1.0);
        double g1, g2;
        if (stokes) {
            stokes_g(r, delta, &g1, &g2);
        } else {
            double x = alpha * r;
            BesselSet bs = bessel_set(x);
            double M0 = m0_closed(r, delta), A = nodeA[m], C = nodeC[m];
            double w = 0.5 * (bs.k0 + bs.k2);
            g1 = bs.ix2w * M0 - w * A - 0.5 * (bs.i0 + bs.i2) * C;
            g2 = (bs.t2k2 * M0 - bs.k2 * A - bs.i2 * C) / (r * r);
        }
        g1s[m] = g1;
        g2s[m] = g2;
    }
    __syncthreads();

    // Chebyshev coefficients per FP64 panel: a_k = (2/n) sum_i g(t_i) T_k(t_i), a_0 halved
    const int np64 = p.n_oct * F64_SUB;
    for (int q = tid; q < 2 * np64 * F64_NODES; q += blockDim.x) {
        int f = q / (np64 * F64_NODES);
        int rem = q % (np64 * F64_NODES);
        int panel = rem / F64_NODES, k = rem % F64_NODES;
        const double *g = (f == 0 ? g1s : g2s) + panel * NP;
        double s = 0.0;
        if (NP == F64_NODES) {
            for (int ii = 0; ii < F64_NODES; ++ii) s += g[ii] * c_dct[k][ii];
        } else if (k < LITE_NODES) {
            for (int ii = 0; ii < LITE_NODES; ++ii) s += g[ii] * c_dct6[k][ii];
        }
        t64[(f * F64_PANELS_MAX + panel) * F64_NODES + k] = s;
    }
    __syncthreads();

    // FP32 quadratic per eighth of an FP64 panel from the FP64 series (Chebyshev fit at 3
    // nodes, then monomial coefficients in G = 1 + f / F32_SUB, f in [0, 1) across the
    // panel); the FP32 table holds -g1 (the sign the pair sum's mobility -g1 I + h e e^T
    // takes) and h = delta^2 g2, for separations measured in units of delta
    const int np32 = p.n_oct * F32_SUB;
    constexpr int SPLIT = F32_SUB / F64_SUB;  // FP32 panels per FP64 panel
    float2 *t32b = (float2 *)(t32 + F32_PANELS_MAX);
    for (int q = tid; q < np32; q += blockDim.x) {
        int e = q >> F32_SUB_LOG2, jj = q & (F32_SUB - 1);
        int panel64 = e * F64_SUB + jj / SPLIT;
        double cf[2][3];
        for (int fn = 0; fn < 2; ++fn) {
            const double *c = t64 + (fn * F64_PANELS_MAX + panel64) * F64_NODES;
            double vals[3];
            for (int i = 0; i < 3; ++i) {
                double f32 = 0.5 * (c_node3[i] + 1.0);  // node of the FP32 panel
                double f64 = ((jj % SPLIT) + f32) / SPLIT;
                double t = 2.0 * f64 - 1.0;
                double b1 = 0.0, b2 = 0.0;
                for (int k = F64_DEG; k >= 1; --k) {
                    double b0 = 2.0 * t * b1 - b2 + c[k];
                    b2 = b1;
                    b1 = b0;
                }
                vals[i] = t * b1 - b2 + c[0];
            }
            double a[3];
            for (int k = 0; k < 3; ++k) a[k] = vals[0] * c_dct3[k][0] + vals[1] * c_dct3[k][1] + vals[2] * c_dct3[k][2];
            // p(t) = a0 + a1 t + a2 (2 t^2 - 1), t = 2 f - 1: p = m0 + m1 f + m2 f^2.  The kernel
            // reads G = 1 + f / S (S = F32_SUB) straight from the low mantissa bits of u, so
            // p = c0 + c1 G + c2 G^2 with f = S (G - 1)
            const double m0 = a[0] - a[1] + a[2], m1 = 2.0 * a[1] - 8.0 * a[2], m2 = 8.0 * a[2];  // in f
            const double S = F32_SUB, sc = fn == 1 ? p.delta * p.delta : -1.0;  // -g1; delta^2 g2
            cf[fn][0] = sc * (m0 - S * m1 + S * S * m2);
            cf[fn][1] = sc * (S * m1 - 2.0 * S * S * m2);
            cf[fn][2] = sc * (S * S * m2);
        }
        t32[q] = make_float4((float)cf[0][0], (float)cf[0][1], (float)cf[0][2], (float)cf[1][0]);
        t32b[q] = make_float2((float)cf[1][1], (float)cf[1][2]);
    }
}

__global__ void set_sample_kernel(SampleParams *sp, double alpha, double delta, double r_max) {
    SampleParams p;
    p.alpha = alpha;
    p.kc = 1.0;
    p.amp = 0.0;
    p.length = r_max / R_MAX_OVER_L;
    p.n = 3;
    p.nh = 0;
    p.sig = 1.0;
    p.ds = p.length / 2;
    p.delta = delta;
    double rho = r_max / delta;
    int n_oct = (int)floor(log2(1.0 + rho * rho)) + 1;
    p.status = SWIMMER_OK;
    if (n_oct > N_OCT_MAX || !(alpha >= 0.0) || alpha * r_max > X_MAX) p.status = SWIMMER_BAD_SAMPLE;
    p.n_oct = min(n_oct, N_OCT_MAX);
    sp[0] = p;
}

// ---------------------------------------------------------------------------------
// kernel-function evaluation through the tables (testing entry point)
// ---------------------------------------------------------------------------------
__global__ void kernel_eval_kernel(int m, const double *__restrict__ r, double *__restrict__ g1,
                                   double *__restrict__ g2, const SampleParams *__restrict__ sp,
                                   const double *__restrict__ tab64, const float4 *__restrict__ tab32,
                                   int precision) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const SampleParams p = sp[0];
    double rr = r[i];
    if (precision == SWIMMER_FP64) {
        double u = 1.0 + rr * rr / (p.delta * p.delta);
        unsigned long long bits = (unsigned long long)__double_as_longlong(u);
        unsigned long long panel = (bits >> (52 - F64_SUB_LOG2)) - (1023ull << F64_SUB_LOG2);
        if (!(u >= 1.0) || panel >= (unsigned long long)(p.n_oct * F64_SUB)) {
            g1[i] = g2[i] = nan("");
            return;
        }
        double f = __longlong_as_double(0x3ff0000000000000LL | (long long)((bits << F64_SUB_LOG2) & 0x000fffffffffffffull)) - 1.0;
        double t = 2.0 * f - 1.0;
        for (int fn = 0; fn < 2; ++fn) {
            const double *c = tab64 + (fn * F64_PANELS_MAX + panel) * F64_NODES;
            double b1 = 0.0, b2 = 0.0;
            for (int k = F64_DEG; k >= 1; --k) {
                double b0 = 2.0 * t * b1 - b2 + c[k];
                b2 = b1;
                b1 = b0;
            }
            (fn == 0 ? g1 : g2)[i] = t * b1 - b2 + c[0];
        }
    } else {
        float inv_d2 = (float)(1.0 / (p.delta * p.delta));
        float r2 = (float)(rr * rr);
        float u = fmaf(r2, inv_d2, 1.0f);
        unsigned bits = __float_as_uint(u);
        unsigned panel = (bits >> (23 - F32_SUB_LOG2)) - (127u << F32_SUB_LOG2);
        if (!(u >= 1.0f) || panel >= (unsigned)(p.n_oct * F32_SUB)) {
            g1[i] = g2[i] = nan("");
            return;
        }
        float G = __uint_as_float(0x3f800000u | (bits & ((1u << (23 - F32_SUB_LOG2)) - 1u)));
        float4 a = tab32[panel];
        float2 c = ((const float2 *)(tab32 + F32_PANELS_MAX))[panel];
        g1[i] = -fmaf(G, fmaf(G, a.z, a.y), a.x);           // the table holds -g1
        g2[i] = fmaf(G, fmaf(G, c.y, c.x), a.w) * inv_d2;  // and delta^2 g2
    }
}

}  // namespace

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_n (host).
static void gauss_legendre(int n, double *x, double *w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) {
            double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

// constant tables for the table builder (host; constant memory is per device, so once
// per device)
int gl_init() {
    static bool done[256] = {};
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) {
        set_error("device ordinal %d out of range", dev);
        return SWIMMER_E_ARG;
    }
    if (done[dev]) return 0;
    double x[GL_N], w[GL_N];
    for (int i = 0; i < GL_N; ++i) {
        double z = cos(PI * (i + 0.75) / (GL_N + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= GL_N; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = GL_N * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    CUDA_TRY(cudaMemcpyToSymbol(c_gl_x, x, sizeof(x)));
    CUDA_TRY(cudaMemcpyToSymbol(c_gl_w, w, sizeof(w)));
    {
        double x8[8], w8[8];
        gauss_legendre(8, x8, w8);
        CUDA_TRY(cudaMemcpyToSymbol(c_gl8_x, x8, sizeof(x8)));
        CUDA_TRY(cudaMemcpyToSymbol(c_gl8_w, w8, sizeof(w8)));
    }
    double ik[NSER], ikk[2][NSER];
    for (int k = 0; k < NSER; ++k) {
        ik[k] = k ? 1.0 / k : 0.0;
        ikk[0][k] = 1.0 / ((k + 1.0) * (k + 1.0));
        ikk[1][k] = 1.0 / ((k + 1.0) * (k + 3.0));
    }
    CUDA_TRY(cudaMemcpyToSymbol(c_inv_k, ik, sizeof(ik)));
    CUDA_TRY(cudaMemcpyToSymbol(c_inv_kk, ikk, sizeof(ikk)));
    double ct[F64_NODES], dct[F64_NODES][F64_NODES];
    for (int ii = 0; ii < F64_NODES; ++ii) {
        int i = F64_NODES - 1 - ii;  // ascending node ii is Chebyshev index i
        ct[ii] = cos(PI * (i + 0.5) / F64_NODES);
        for (int k = 0; k < F64_NODES; ++k)
            dct[k][ii] = (2.0 / F64_NODES) * cos(PI * k * (i + 0.5) / F64_NODES) * (k == 0 ? 0.5 : 1.0);
    }
    CUDA_TRY(cudaMemcpyToSymbol(c_cheb_t, ct, sizeof(ct)));
    CUDA_TRY(cudaMemcpyToSymbol(c_dct, dct, sizeof(dct)));
    double ct6[LITE_NODES], dct6[LITE_NODES][LITE_NODES];
    for (int ii = 0; ii < LITE_NODES; ++ii) {
        int i = LITE_NODES - 1 - ii;
        ct6[ii] = cos(PI * (i + 0.5) / LITE_NODES);
        for (int k = 0; k < LITE_NODES; ++k)
            dct6[k][ii] = (2.0 / LITE_NODES) * cos(PI * k * (i + 0.5) / LITE_NODES) * (k == 0 ? 0.5 : 1.0);
    }
    CUDA_TRY(cudaMemcpyToSymbol(c_cheb_t6, ct6, sizeof(ct6)));
    CUDA_TRY(cudaMemcpyToSymbol(c_dct6, dct6, sizeof(dct6)));
    double n3[3], d3[3][3];
    for (int i = 0; i < 3; ++i) {
        n3[i] = cos(PI * (i + 0.5) / 3.0);
        for (int k = 0; k < 3; ++k) d3[k][i] = (2.0 / 3.0) * cos(PI * k * (i + 0.5) / 3.0) * (k == 0 ? 0.5 : 1.0);
    }
    CUDA_TRY(cudaMemcpyToSymbol(c_node3, n3, sizeof(n3)));
    CUDA_TRY(cudaMemcpyToSymbol(c_dct3, d3, sizeof(d3)));
    done[dev] = true;
    return 0;
}

int handle_octaves(const swimmer_handle *h) {
    // the sample with the most flagellum points and, for two swimmers, the smallest ds
    const int nfm = default_flagellum_points(h->cfg);
    const double ds = h->cfg.ds_fixed > 0.0 ? h->cfg.ds_fixed : h->cfg.length / (nfm - 1);
    double rho = R_MAX_OVER_L * sample_reach(h->cfg, nfm, ds) / (h->cfg.delta_over_ds * ds);
    int n_oct = (int)floor(log2(1.0 + rho * rho)) + 1;
    return n_oct > N_OCT_MAX ? N_OCT_MAX : n_oct;
}

int launch_prepare(swimmer_handle *h, int B, const double *theta, const int *n_pts, cudaStream_t s) {
    prepare_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, theta, n_pts, h->cfg, h->sp, h->order);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
    {  // longest first: by n for uneven sizes, else by K_C
        order_kernel<<<1, SORT_THREADS, 0, s>>>(B, h->sp, h->order, n_pts ? 0 : 1);
        CUDA_TRY(cudaGetLastError());
        prof_count(h, 1);
    }
    return 0;
}

int launch_table_build(swimmer_handle *h, int B, int need64, cudaStream_t s) {
    // node arrays for the handle's octaves (kernel_eval may need the full range)
    // need64: 0 = FP32 handle build, 1 = FP64 build, 2/3 = the same over the full range
    const int oct = need64 >= 2 ? N_OCT_MAX : handle_octaves(h);
    const bool lite = need64 == 0 || need64 == 3;
    const int M = oct * F64_SUB * (lite ? LITE_NODES : F64_NODES);
    size_t smem = 4 * (size_t)M * sizeof(double);
    CUDA_TRY(cudaFuncSetAttribute(table_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(4 * (size_t)NODES_MAX * sizeof(double))));
    dim3 ga(B, (M + TAIL_MAX + K1A_THREADS - 1) / K1A_THREADS);
    table_integrals_kernel<<<ga, K1A_THREADS, 0, s>>>(B, h->sp, h->k1_scratch, lite ? 1 : 0, oct);
    CUDA_TRY(cudaGetLastError());
    table_build_kernel<<<B, K1_THREADS, smem, s>>>(B, h->sp, h->k1_scratch, h->tab64, h->tab32, lite ? 1 : 0, oct);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 2);
    return 0;
}

int launch_set_sample(swimmer_handle *h, double alpha, double delta, double r_max, cudaStream_t s) {
    set_sample_kernel<<<1, 1, 0, s>>>(h->sp, alpha, delta, r_max);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

int launch_kernel_eval(swimmer_handle *h, int m, const double *r, double *g1, double *g2,
                       int precision, cudaStream_t s) {
    kernel_eval_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, r, g1, g2, h->sp, h->tab64, h->tab32, precision);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------------------------
// Allocation-free kernel-function evaluation
// ---------------------------------------------------------------------------------
// Some callers may not allocate device memory at all: services that fix their device-memory
// budget at start-up and must not grow it per request.  For them the
// table build of one sample (the kernels above that use scratch memory) runs on scratch
// that lives in file-scope device arrays: every GPU that loads this library holds these
// ~98 KB until the process exits, and every call on a device shares them.
namespace {
__device__ __align__(256) double g_noalloc_scratch[K1_SCRATCH];
__device__ __align__(256) double g_noalloc_tab64[TAB64_STRIDE];
__device__ __align__(256) float4 g_noalloc_tab32[TAB32_STRIDE];
__device__ __align__(256) SampleParams g_noalloc_sp[1];

struct NoallocPtrs {
    double *scratch, *tab64;
    float4 *tab32;
    SampleParams *sp;
    bool ready;
};
NoallocPtrs g_noalloc[256];
std::mutex g_noalloc_mutex;

// once per device, with that device current: the device addresses of the arrays (their names
// are host-side stand-ins in host code), constant tables and kernel attributes
int noalloc_setup(int dev, NoallocPtrs *out) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoallocPtrs &p = g_noalloc[dev];
    if (!p.ready) {
        int rc = gl_init();
        if (rc) return rc;
        CUDA_TRY(cudaGetSymbolAddress((void **)&p.scratch, g_noalloc_scratch));
        CUDA_TRY(cudaGetSymbolAddress((void **)&p.tab64, g_noalloc_tab64));
        CUDA_TRY(cudaGetSymbolAddress((void **)&p.tab32, g_noalloc_tab32));
        CUDA_TRY(cudaGetSymbolAddress((void **)&p.sp, g_noalloc_sp));
        CUDA_TRY(cudaFuncSetAttribute(table_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)(4 * (size_t)NODES_MAX * sizeof(double))));
        // load every kernel of the call now: with lazy module loading a kernel first launched
        // later (kernel_eval_kernel after calls with m = 0) would load its code then
        cudaFuncAttributes fa;
        CUDA_TRY(cudaFuncGetAttributes(&fa, set_sample_kernel));
        CUDA_TRY(cudaFuncGetAttributes(&fa, table_integrals_kernel));
        CUDA_TRY(cudaFuncGetAttributes(&fa, table_build_kernel));
        CUDA_TRY(cudaFuncGetAttributes(&fa, kernel_eval_kernel));
        p.ready = true;
    }
    *out = p;
    return 0;
}
}  // namespace

extern "C" int swimmer_kernel_eval_noalloc(double alpha, double delta, double r_max, int m, const double *r,
                                           double *g1, double *g2, int precision, void *stream) {
    ARG_CHECK(m >= 0, "m must be >= 0");
    ARG_CHECK(m == 0 || (r && g1 && g2), "r, g1, g2 must be device pointers");
    ARG_CHECK(alpha >= 0.0 && delta > 0.0 && r_max > 0.0, "need alpha >= 0, delta > 0, r_max > 0");
    ARG_CHECK(r_max / delta < 4000.0, "r_max/delta = %g beyond the maximum 4000 of the static tables",
              r_max / delta);
    ARG_CHECK(alpha * r_max <= X_MAX, "alpha * r_max beyond %g", X_MAX);
    ARG_CHECK(precision == SWIMMER_FP64 || precision == SWIMMER_FP32C, "precision must be 0 or 1");
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    ARG_CHECK(dev >= 0 && dev < 256, "device ordinal %d out of range", dev);
    NoallocPtrs p;
    int rc = noalloc_setup(dev, &p);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const bool lite = precision != SWIMMER_FP64;  // as FP32 handles build their table
    const int M = N_OCT_MAX * F64_SUB * (lite ? LITE_NODES : F64_NODES);
    set_sample_kernel<<<1, 1, 0, s>>>(p.sp, alpha, delta, r_max);
    CUDA_TRY(cudaGetLastError());
    dim3 ga(1, (M + TAIL_MAX + K1A_THREADS - 1) / K1A_THREADS);
    table_integrals_kernel<<<ga, K1A_THREADS, 0, s>>>(1, p.sp, p.scratch, lite ? 1 : 0, N_OCT_MAX);
    CUDA_TRY(cudaGetLastError());
    table_build_kernel<<<1, K1_THREADS, 4 * (size_t)M * sizeof(double), s>>>(1, p.sp, p.scratch, p.tab64, p.tab32,
                                                                           lite ? 1 : 0, N_OCT_MAX);
    CUDA_TRY(cudaGetLastError());
    if (m > 0) {
        kernel_eval_kernel<<<(m + 127) / 128, 128, 0, s>>>(m, r, g1, g2, p.sp, p.tab64, p.tab32, precision);
        CUDA_TRY(cudaGetLastError());
    }
    return 0;
}
