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
// u = 1 + r^2/delta^2, degree 9) and, derived from them, FP32 cubic coefficients in the
// local panel coordinate f in [0, 1) (16 panels per octave).
#include <math.h>
#include <stdio.h>

#include "common.cuh"

namespace {

constexpr double PI = 3.14159265358979323846;
constexpr double EGAMMA = 0.57721566490153286061;
constexpr int GL_N = 16;
__constant__ double c_gl_x[GL_N];
__constant__ double c_gl_w[GL_N];

// ---------------------------------------------------------------------------------
// Bessel functions
// ---------------------------------------------------------------------------------
// I_nu(x), nu in {0, 2}: power series for x <= 30, Hankel asymptotic expansion beyond.
__device__ double bessel_i(int nu, double x) {
    if (x <= 30.0) {
        double y = 0.25 * x * x;
        double term = 1.0;
        for (int m = 1; m <= nu; ++m) term /= m;  // 1/nu!
        double s = 0.0;
        for (int k = 0; k < 400; ++k) {
            s += term;
            term *= y / ((k + 1.0) * (k + 1.0 + nu));
            if (term < 1e-18 * s) break;
        }
        return s * (nu == 0 ? 1.0 : y);  // (x/2)^2 = y for nu = 2
    }
    double mu = 4.0 * nu * nu;
    double s = 1.0, term = 1.0;
    for (int k = 1; k < 60; ++k) {
        double a = (mu - (2.0 * k - 1.0) * (2.0 * k - 1.0)) / (k * 8.0 * x);
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
        term *= y / ((k + 1.0) * (k + 1.0));
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
    for (int m = 1; m < 4000; ++m) {
        double t = m * h;
        double c = cosh(t);
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
            term *= y / ((double)k * k);
            hk += 1.0 / k;
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
            term *= y / ((k + 1.0) * (k + 3.0));
            hk0 += 1.0 / (k + 1.0);
            hk2 += 1.0 / (k + 3.0);
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
    if (x <= 2.0) return bessel_set(x).k0;
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
__device__ double panel_integral(int which, double a, double b, double alpha, double delta) {
    if (b <= a) return 0.0;
    double w = b - a;
    int n = (int)ceil(fmax(alpha * w / 0.5, w / (0.5 * fmax(a, 0.25 * delta))));
    if (n < 1) n = 1;
    if (n > 4096) n = 4096;
    double hw = 0.5 * w / n, tot = 0.0;
    for (int p = 0; p < n; ++p) {
        double c = a + (2 * p + 1) * hw, acc = 0.0;
        for (int g = 0; g < GL_N; ++g) {
            double s = c + hw * c_gl_x[g];
            double f = (which == 0 ? bessel_i0m1(alpha * s) : bessel_k0(alpha * s)) * blob(s, delta) * s;
            acc += c_gl_w[g] * f;
        }
        tot += acc * hw;
    }
    return tot;
}

__device__ __forceinline__ double node_u(int m) {
    // node m -> (octave, panel, ascending Chebyshev index)
    int panel = m / F64_NODES, ii = m % F64_NODES;
    int e = panel >> F64_SUB_LOG2, j = panel & (F64_SUB - 1);
    double t = -cos(PI * (ii + 0.5) / F64_NODES);  // ascending in ii
    double f = 0.5 * (t + 1.0);
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
    p.n = n_pts ? n_pts[b] : cfg.n_max;
    p.alpha = theta[3 * b + 0];
    p.kc = pow(10.0, theta[3 * b + 1]);
    p.amp = theta[3 * b + 2];
    p.length = cfg.ds_fixed > 0.0 ? (p.n - 1) * cfg.ds_fixed : cfg.length;
    p.status = SWIMMER_OK;
    if (p.n < 3 || p.n > cfg.n_max) {
        p.n = 3;
        p.status = SWIMMER_BAD_SAMPLE;
    }
    p.ds = p.length / (p.n - 1);
    p.delta = cfg.delta_over_ds * p.ds;
    double rho = R_MAX_OVER_L * p.length / p.delta;
    int n_oct = (int)floor(log2(1.0 + rho * rho)) + 1;
    if (n_oct > N_OCT_MAX) {
        n_oct = N_OCT_MAX;
        p.status = SWIMMER_BAD_SAMPLE;
    }
    p.n_oct = n_oct;
    if (!(p.alpha >= 0.0) || p.alpha * R_MAX_OVER_L * p.length > X_MAX || !isfinite(p.kc) ||
        !isfinite(p.amp) || !(p.kc > 0.0))
        p.status = SWIMMER_BAD_SAMPLE;
    sp[b] = p;
    order[b] = b;
}

// ---------------------------------------------------------------------------------
// K1: one CTA per sample
// ---------------------------------------------------------------------------------
constexpr int K1_THREADS = 256;

__global__ void __launch_bounds__(K1_THREADS)
table_build_kernel(int B, const SampleParams *__restrict__ sp, double *__restrict__ tab64,
                   float4 *__restrict__ tab32) {
    extern __shared__ double sm[];
    const int b = blockIdx.x;
    if (b >= B) return;
    const SampleParams p = sp[b];
    const int M = p.n_oct * F64_SUB * F64_NODES;
    double *nodeA = sm;            // [M] interval integrals -> A1 prefix
    double *nodeC = sm + M;        // [M] interval integrals -> C suffix
    double *g1s = sm + 2 * M;      // [M]
    double *g2s = sm + 3 * M;      // [M]
    __shared__ double red[K1_THREADS];
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
        // interval integrals between consecutive nodes
        double tail = 0.0;
        for (int m = tid; m < M; m += blockDim.x) {
            double r = delta * sqrt(node_u(m) - 1.0);
            double rprev = m ? delta * sqrt(node_u(m - 1) - 1.0) : 0.0;
            nodeA[m] = panel_integral(0, rprev, r, alpha, delta);
            if (m + 1 < M) nodeC[m] = panel_integral(1, r, delta * sqrt(node_u(m + 1) - 1.0), alpha, delta);
        }
        // geometric tail beyond the last node, spread over the block, fixed-order reduction
        {
            double r_last = delta * sqrt(node_u(M - 1) - 1.0);
            double s_end = fmin(r_last + 60.0 / alpha, 1e6 * delta);
            // piece k covers [s_k, s_{k+1}], s_{k+1} = s_k + min(max(s_k, delta/4), 0.5/alpha)
            // computed serially for boundaries (cheap), integrated in parallel
            double acc = 0.0;
            double s = r_last;
            for (int k = 0; s < s_end && k < 100000; ++k) {
                double w = fmin(fmax(s, 0.25 * delta), 0.5 / alpha);
                double e = fmin(s + w, s_end);
                if (k % blockDim.x == tid) acc += panel_integral(1, s, e, alpha, delta);
                s = e;
            }
            red[tid] = acc;
            __syncthreads();
            for (int o = blockDim.x / 2; o > 0; o >>= 1) {
                if (tid < o) red[tid] += red[tid + o];
                __syncthreads();
            }
            tail = red[0];
        }
        if (tid == 0) nodeC[M - 1] = tail;
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
        double r = delta * sqrt(node_u(m) - 1.0);
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
        const double *g = (f == 0 ? g1s : g2s) + panel * F64_NODES;
        double s = 0.0;
        for (int ii = 0; ii < F64_NODES; ++ii) {
            int i = F64_NODES - 1 - ii;  // descending Chebyshev index of ascending node ii
            s += g[ii] * cos(PI * k * (i + 0.5) / F64_NODES);
        }
        s *= 2.0 / F64_NODES;
        if (k == 0) s *= 0.5;
        t64[(f * F64_PANELS_MAX + panel) * F64_NODES + k] = s;
    }
    __syncthreads();

    // FP32 cubic per half panel from the FP64 series (Chebyshev fit at 4 nodes, then
    // monomial coefficients in f in [0, 1))
    const int np32 = p.n_oct * F32_SUB;
    for (int q = tid; q < 2 * np32; q += blockDim.x) {
        int f = q / np32, panel32 = q % np32;
        int e = panel32 >> F32_SUB_LOG2, jj = panel32 & (F32_SUB - 1);
        int panel64 = e * F64_SUB + (jj >> 1);
        const double *c = t64 + (f * F64_PANELS_MAX + panel64) * F64_NODES;
        double vals[4];
        for (int i = 0; i < 4; ++i) {
            double tl = cos(PI * (i + 0.5) / 4.0);        // in [-1, 1] of the FP32 panel
            double f32 = 0.5 * (tl + 1.0);
            double f64 = 0.5 * ((jj & 1) + f32);
            double t = 2.0 * f64 - 1.0;
            double b1 = 0.0, b2 = 0.0;
            for (int k = F64_DEG; k >= 1; --k) {
                double b0 = 2.0 * t * b1 - b2 + c[k];
                b2 = b1;
                b1 = b0;
            }
            vals[i] = t * b1 - b2 + c[0];
        }
        double a[4];
        for (int k = 0; k < 4; ++k) {
            double s = 0.0;
            for (int i = 0; i < 4; ++i) s += vals[i] * cos(PI * k * (i + 0.5) / 4.0);
            a[k] = s * 0.5 * (k == 0 ? 0.5 : 1.0);
        }
        // p(t) = a0 + a1 T1 + a2 T2 + a3 T3, t = 2 f - 1
        double c0 = a[0] - a[1] + a[2] - a[3];
        double c1 = 2.0 * a[1] - 8.0 * a[2] + 18.0 * a[3];
        double c2 = 8.0 * a[2] - 48.0 * a[3];
        double c3 = 32.0 * a[3];
        t32[f * F32_PANELS_MAX + panel32] = make_float4((float)c0, (float)c1, (float)c2, (float)c3);
    }
}

__global__ void set_sample_kernel(SampleParams *sp, double alpha, double delta, double r_max) {
    SampleParams p;
    p.alpha = alpha;
    p.kc = 1.0;
    p.amp = 0.0;
    p.length = r_max / R_MAX_OVER_L;
    p.n = 3;
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
        float f = __uint_as_float(0x3f800000u | ((bits << F32_SUB_LOG2) & 0x7fffffu)) - 1.0f;
        float4 a = tab32[panel], c = tab32[F32_PANELS_MAX + panel];
        g1[i] = fmaf(f, fmaf(f, fmaf(f, a.w, a.z), a.y), a.x);
        g2[i] = fmaf(f, fmaf(f, fmaf(f, c.w, c.z), c.y), c.x);
    }
}

}  // namespace

// Gauss-Legendre nodes/weights on [-1, 1] by Newton's method on P_16 (host, once).
int gl_init() {
    static bool done = false;
    if (done) return 0;
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
    done = true;
    return 0;
}

int launch_prepare(swimmer_handle *h, int B, const double *theta, const int *n_pts, cudaStream_t s) {
    prepare_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, theta, n_pts, h->cfg, h->sp, h->order);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
    return 0;
}

int launch_table_build(swimmer_handle *h, int B, int need64, cudaStream_t s) {
    (void)need64;
    size_t smem = 4 * (size_t)NODES_MAX * sizeof(double);
    static bool attr = false;
    if (!attr) {
        CUDA_TRY(cudaFuncSetAttribute(table_build_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    table_build_kernel<<<B, K1_THREADS, smem, s>>>(B, h->sp, h->tab64, h->tab32);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
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
