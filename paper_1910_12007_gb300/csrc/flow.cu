// Flow and pressure at target points (Eqs. BrP, BrV with targets x other than the
// swimmer's points): v(x) = (1/mu) sum_j [-F_j g1(r) + (F_j . d) d g2(r)] and
// p(x) = sum_j F_j . grad G_delta = sum_j (F_j . d) G_delta'(r)/r, d = x - X_j, with
// G_delta'(r)/r = (R^2 + R delta + delta^2) / (2 pi R^3 (R + delta)), R = sqrt(r^2 + delta^2)
// (the blob's moment over r^2, finite at r = 0).  One thread per target point, FP64, the
// sample's full-range FP64 table from global memory.
#include <math.h>

#include "common.cuh"
#include "table_eval.cuh"

int launch_set_sample(swimmer_handle *h, double alpha, double delta, double r_max, cudaStream_t s);
int launch_table_build(swimmer_handle *h, int B, int need64, cudaStream_t s);

namespace {

__global__ void flow_kernel(int n, const double *__restrict__ state, const double *__restrict__ tab,
                            const SampleParams *__restrict__ sp, double mu, int G, const double *__restrict__ grid,
                            double *__restrict__ vel, double *__restrict__ pres) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= G) return;
    const SampleParams p = sp[0];
    if (p.status != SWIMMER_OK) {
        if (vel) vel[2 * g] = vel[2 * g + 1] = nan("");
        if (pres) pres[g] = nan("");
        return;
    }
    const double delta = p.delta, inv_d2 = 1.0 / (delta * delta);
    const int pmax = p.n_oct * F64_SUB - 1;
    const double x = grid[2 * g], y = grid[2 * g + 1];
    double vx = 0.0, vy = 0.0, pr = 0.0;
    for (int j = 0; j < n; ++j) {
        const double *q = state + 4 * (size_t)j;
        const double dx = x - q[0], dy = y - q[1];
        const double r2 = fma(dx, dx, dy * dy);
        double g1, g2;
        kern_f64(tab, F64_PANELS_MAX, pmax, fma(r2, inv_d2, 1.0), g1, g2);
        const double fd = fma(q[2], dx, q[3] * dy);
        vx = fma(fd * g2, dx, fma(-q[2], g1, vx));
        vy = fma(fd * g2, dy, fma(-q[3], g1, vy));
        const double R = sqrt(r2 + delta * delta);
        pr = fma(fd, (R * R + R * delta + delta * delta) / (2.0 * 3.14159265358979323846 * R * R * R * (R + delta)), pr);
    }
    if (vel) {
        vel[2 * g] = vx / mu;
        vel[2 * g + 1] = vy / mu;
    }
    if (pres) pres[g] = pr;
}

}  // namespace

extern "C" int swimmer_flow_field(swimmer_handle *h, double alpha, double delta, double r_max, int n,
                                  const double *state, int G, const double *grid, double *vel, double *pres,
                                  void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(alpha >= 0.0 && delta > 0.0 && r_max > 0.0, "need alpha >= 0, delta > 0, r_max > 0");
    ARG_CHECK(n >= 1 && G >= 0, "need n >= 1 points and G >= 0 targets");
    ARG_CHECK(state != nullptr && (G == 0 || grid != nullptr), "NULL device pointer");
    ARG_CHECK(vel != nullptr || pres != nullptr, "no output requested");
    if (G == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = launch_set_sample(h, alpha, delta, r_max, s);
    if (!rc) rc = launch_table_build(h, 1, 2, s);  // full-range FP64 table in sample slot 0
    if (rc) return rc;
    flow_kernel<<<(G + 127) / 128, 128, 0, s>>>(n, state, h->tab64, h->sp, h->cfg.mu, G, grid, vel, pres);
    CUDA_TRY(cudaGetLastError());
    prof_count(h, 1);
    return 0;
}
