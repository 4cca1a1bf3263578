/*
 * Plain FP64 forward Euler time loop of the elastic flagellum in a Brinkman fluid
 * (oracle; test infrastructure only -- the CUDA product path never links this file).
 *
 * The arithmetic is the one oracle/swimmer.py states (Appendix Eqs. EFB, curva, EFT;
 * Eq. Fenergy; Eq. BrV; forward Euler), written as straightforward loops.  The kernel
 * functions g1 = B'', g2 = (r B'' - B')/r^3 come from the oracle's Chebyshev table over
 * u = 1 + r^2/delta^2 (oracle/brinkmanlet.py, KernelTable): octave e = floor(log2 u),
 * panel j of n_sub equal panels per octave, local t in [-1, 1].
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int n_oct, n_sub, deg;
    const double *coef; /* [2][n_oct*n_sub][deg+1] */
} table_t;

/* g1, g2 at squared distance r2 from the Chebyshev table. Returns 0, or -1 if out of range. */
static int table_eval(const table_t *T, double inv_delta2, double r2, double *g1, double *g2)
{
    double u = 1.0 + r2 * inv_delta2;
    int e;
    double m = frexp(u, &e); /* u = m 2^e, m in [0.5, 1) -> octave e-1 */
    e -= 1;
    if (e < 0) e = 0;
    if (e >= T->n_oct) return -1;
    double base = ldexp(1.0, e);
    int j = (int)floor((u / base - 1.0) * T->n_sub);
    if (j < 0) j = 0;
    if (j >= T->n_sub) j = T->n_sub - 1;
    double ua = base * (1.0 + (double)j / T->n_sub);
    double w = base / T->n_sub;
    double t = 2.0 * (u - ua) / w - 1.0;
    int npan = T->n_oct * T->n_sub, p = e * T->n_sub + j;
    (void)m;
    for (int f = 0; f < 2; ++f) {
        const double *c = T->coef + ((size_t)f * npan + p) * (T->deg + 1);
        double b1 = 0.0, b2 = 0.0;
        for (int k = T->deg; k >= 1; --k) {
            double b0 = 2.0 * t * b1 - b2 + c[k];
            b2 = b1;
            b1 = b0;
        }
        double val = t * b1 - b2 + c[0];
        if (f == 0) *g1 = val; else *g2 = val;
    }
    return 0;
}

/* zeta^_k(t) = -a [ (2 eta / L) cos(eta s - omega t) + (1 - s/L) eta^2 sin(eta s - omega t) ] */
static double pref_curv(double s, double L, double a, double eta, double omega, double t)
{
    double ph = eta * s - omega * t;
    return -a * (2.0 * eta / L * cos(ph) + (1.0 - s / L) * eta * eta * sin(ph));
}

/* F = -dE/dX for E = K_T sum (l/ds - 1)^2 ds + K_C sum_{interior} (zeta - zeta^)^2 ds */
static void forces(int n, const double *x, const double *y, double ds, double L, double KT,
                   double KC, double a, double eta, double omega, double t, double *fx, double *fy)
{
    for (int k = 0; k < n; ++k) fx[k] = fy[k] = 0.0;
    for (int k = 0; k + 1 < n; ++k) {
        double sx = x[k + 1] - x[k], sy = y[k + 1] - y[k];
        double l = sqrt(sx * sx + sy * sy);
        double c = 2.0 * KT * (l / ds - 1.0) / l;
        fx[k + 1] -= c * sx; fy[k + 1] -= c * sy;
        fx[k] += c * sx;     fy[k] += c * sy;
    }
    for (int k = 1; k + 1 < n; ++k) {
        double A = (x[k + 1] - x[k - 1]) / (2.0 * ds);
        double Bv = (y[k + 1] - y[k - 1]) / (2.0 * ds);
        double C = (x[k + 1] - 2.0 * x[k] + x[k - 1]) / (ds * ds);
        double D = (y[k + 1] - 2.0 * y[k] + y[k - 1]) / (ds * ds);
        double S = A * A + Bv * Bv;
        double S15 = pow(S, -1.5), S25 = pow(S, -2.5);
        double cross = A * D - Bv * C;
        double zeta = cross * S15;
        double ck = 2.0 * KC * ds * (zeta - pref_curv(k * ds, L, a, eta, omega, t));
        double za = D * S15 - 3.0 * A * cross * S25;
        double zb = -C * S15 - 3.0 * Bv * cross * S25;
        double zc = -Bv * S15;
        double zd = A * S15;
        fx[k - 1] -= ck * (-za / (2.0 * ds) + zc / (ds * ds));
        fx[k]     -= ck * (-2.0 * zc / (ds * ds));
        fx[k + 1] -= ck * (za / (2.0 * ds) + zc / (ds * ds));
        fy[k - 1] -= ck * (-zb / (2.0 * ds) + zd / (ds * ds));
        fy[k]     -= ck * (-2.0 * zd / (ds * ds));
        fy[k + 1] -= ck * (zb / (2.0 * ds) + zd / (ds * ds));
    }
}

/* One sample: returns status (0 ok, 1 diverged, 2 table range exceeded). */
static int forward_one(int n, double L, double mu, double delta_over_ds, double dt, double KT,
                       double KC, double a, double eta, double omega, long steps, long obs_every,
                       const table_t *T, double *obs, double *Xf, double *xc)
{
    double ds = L / (n - 1), delta = delta_over_ds * ds, inv_d2 = 1.0 / (delta * delta);
    double *x = calloc(n, sizeof(double)), *y = calloc(n, sizeof(double));
    double *fx = calloc(n, sizeof(double)), *fy = calloc(n, sizeof(double));
    double *vx = calloc(n, sizeof(double)), *vy = calloc(n, sizeof(double));
    int status = 0;
    long o = 0;
    for (int k = 0; k < n; ++k) { x[k] = k * ds; y[k] = 0.0; }
    double c0 = 0.0;
    for (int k = 0; k < n; ++k) c0 += x[k];
    xc[0] = c0 / n;
    for (long step = 0; step < steps && status == 0; ++step) {
        double t = step * dt;
        forces(n, x, y, ds, L, KT, KC, a, eta, omega, t, fx, fy);
        double vmax = 0.0;
        for (int i = 0; i < n && status == 0; ++i) {
            double sx = 0.0, sy = 0.0;
            for (int j = 0; j < n; ++j) {
                double dx = x[i] - x[j], dy = y[i] - y[j];
                double g1, g2;
                if (table_eval(T, inv_d2, dx * dx + dy * dy, &g1, &g2)) { status = 2; break; }
                double fd = fx[j] * dx + fy[j] * dy;
                sx += -fx[j] * g1 + fd * dx * g2;
                sy += -fy[j] * g1 + fd * dy * g2;
            }
            vx[i] = sx / mu;
            vy[i] = sy / mu;
            if (!isfinite(vx[i]) || !isfinite(vy[i])) status = 1;
            double m = fabs(vx[i]) > fabs(vy[i]) ? fabs(vx[i]) : fabs(vy[i]);
            if (m > vmax) vmax = m;
        }
        if (status) break;
        if (vmax * dt > ds) { status = 1; break; }
        for (int i = 0; i < n; ++i) { x[i] += dt * vx[i]; y[i] += dt * vy[i]; }
        if ((step + 1) % obs_every == 0) {
            obs[2 * o] = x[n - 1];
            obs[2 * o + 1] = y[n - 1];
            ++o;
        }
    }
    double c1 = 0.0;
    for (int k = 0; k < n; ++k) { c1 += x[k]; Xf[2 * k] = x[k]; Xf[2 * k + 1] = y[k]; }
    xc[1] = c1 / n;
    free(x); free(y); free(fx); free(fy); free(vx); free(vy);
    return status;
}

int oracle_forward_batch(int B, const int *n, const double *L, double mu, double delta_over_ds,
                         double dt, double KT, double eta, double omega, long steps, long obs_every,
                         const double *alpha, const double *KC, const double *amp,
                         int n_sub, int deg, const int *n_oct, const double *coef, const long *coef_off,
                         double *obs, double *Xf, double *xc, int *status, int threads)
{
    int n_max = 0;
    (void)alpha;
    for (int b = 0; b < B; ++b) {
        if (n[b] < 3) return -1;
        if (n[b] > n_max) n_max = n[b];
    }
    long n_obs = steps / obs_every;
    if (n_obs < 1) n_obs = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int b = 0; b < B; ++b) {
        table_t T = {n_oct[b], n_sub, deg, coef + coef_off[b]};
        status[b] = forward_one(n[b], L[b], mu, delta_over_ds, dt, KT, KC[b], amp[b], eta, omega,
                                steps, obs_every, &T, obs + (size_t)b * n_obs * 2,
                                Xf + (size_t)b * n_max * 2, xc + 2 * b);
    }
    return 0;
}
