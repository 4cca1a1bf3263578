// K5/K6: the learned surrogate, an MLP 5 -> 256 -> 256 -> 256 -> 80 with GELU hidden
// activations (not in the paper).  Weights are kept as an FP32 master copy and rounded to
// BF16 when they enter a product; every product accumulates in FP32.
//
// The products of the three 256-wide layers (forward, weight gradient, input gradient) run on
// the tensor cores: BF16 operands, FP32 accumulation, warp-level m16n8k16 MMA over 64 x 64
// output tiles.  The first layer (5 inputs, which stay FP32) runs through a tiled FP32 GEMM
// (64 x 64 tiles, 16-deep K panels, 4 x 4 outputs per thread).  Both carry fused epilogues:
// bias + GELU for the forward pass, the GELU derivative for the backward pass.  Weight
// gradients reduce over the batch in up to 16 slices of the batch (split K, so that the 16
// output tiles of a 256 x 256 gradient fill the GPU), whose partial products are then summed
// in a fixed order (no atomics), so gradients are deterministic.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"

namespace {

constexpr int IN = SWIMMER_MLP_IN, HID = SWIMMER_MLP_HIDDEN, OUT = SWIMMER_MLP_OUT;
constexpr int NLAYER = 4;
__host__ __device__ constexpr int fan_in(int l) { return l == 0 ? IN : HID; }
__host__ __device__ constexpr int fan_out(int l) { return l == NLAYER - 1 ? OUT : HID; }
__host__ __device__ constexpr int w_off(int l) {
    return l == 0 ? 0 : w_off(l - 1) + fan_in(l - 1) * fan_out(l - 1) + fan_out(l - 1);
}
__host__ __device__ constexpr int b_off(int l) { return w_off(l) + fan_in(l) * fan_out(l); }
static_assert(b_off(NLAYER - 1) + OUT == SWIMMER_MLP_NPARAM, "parameter layout");

enum Epi { EPI_PLAIN = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_DGELU = 3 };

constexpr float INV_SQRT2 = 0.70710678118654752f;
constexpr float INV_SQRT2PI = 0.39894228040143268f;

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * INV_SQRT2)); }
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * INV_SQRT2)) + z * expf(-0.5f * z * z) * INV_SQRT2PI;
}
__device__ __forceinline__ float bf16r(float w) { return __bfloat162float(__float2bfloat16_rn(w)); }

// C[m][n] = epi( sum_k A(m, k) B(k, n) ),  A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn]
// round_b: B holds weights, rounded to BF16 on load.  Split K (gridDim.z > 1, EPI_PLAIN):
// CTA z sums k in [z kc, (z + 1) kc) into the partial plane C + z M ldc.
constexpr int TM = 64, TN = 64, TK = 16;
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, int kc, const float *__restrict__ A, int sam,
                                                  int sak, const float *__restrict__ B, int sbk, int sbn, int round_b,
                                                  float *__restrict__ C, int ldc, int epi,
                                                  const float *__restrict__ bias, const float *__restrict__ Z,
                                                  int ldz, float *__restrict__ C2) {
    __shared__ float As[TK][TM + 1];
    __shared__ float Bs[TK][TN + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    C += (size_t)blockIdx.z * M * ldc;
    float acc[4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += TK) {
        for (int e = threadIdx.x; e < TM * TK; e += 256) {
            int mm = e / TK, kk = e % TK;
            int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < ke) ? A[(size_t)m * sam + (size_t)k * sak] : 0.f;
        }
        for (int e = threadIdx.x; e < TK * TN; e += 256) {
            int kk = e / TN, nn = e % TN;
            int k = k0 + kk, n = n0 + nn;
            float v = (k < ke && n < N) ? B[(size_t)k * sbk + (size_t)n * sbn] : 0.f;
            Bs[kk][nn] = round_b ? bf16r(v) : v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < TK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        int m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            float v = acc[i][j];
            if (epi == EPI_BIAS || epi == EPI_BIAS_GELU) v += bias[n];
            if (epi == EPI_DGELU) v *= gelu_grad(Z[(size_t)m * ldz + n]);
            C[(size_t)m * ldc + n] = v;
            if (epi == EPI_BIAS_GELU) C2[(size_t)m * ldc + n] = gelu(v);
        }
    }
}

// The same product on the tensor cores: BF16 operands (both rounded to nearest as they are
// staged), FP32 accumulation, warp-level m16n8k16 MMA.  A 64 x 64 output tile per CTA of four
// warps (2 x 2, each 32 x 32: 2 x 4 MMA tiles), K panels of 32 staged in shared memory as
// [row][k] BF16 with rows padded to 40 elements (80 bytes: the fragment loads of a warp fall
// in distinct banks).  Operands are read with any strides and zero-filled past M, N, K.
constexpr int TC_TM = 64, TC_TN = 64, TC_TK = 32, TC_LD = TC_TK + 8;
__device__ __forceinline__ unsigned pack_bf16(float lo, float hi) {
    const unsigned a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const unsigned b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}
// stage rows [r0, r0 + 64) x k [k0, k0 + 32) of X(r, k) = X[r*sr + k*sk] into S[row][k] as BF16
// pairs; the loop runs along whichever index has unit stride, so global reads coalesce
__device__ __forceinline__ void tc_stage(unsigned *S, const float *__restrict__ X, int R, int K, int r0, int k0,
                                         int sr, int sk) {
    if (sk == 1) {
        for (int e = threadIdx.x; e < TC_TM * TC_TK / 2; e += 128) {
            const int rr = e / (TC_TK / 2), kk = 2 * (e % (TC_TK / 2));
            const int r = r0 + rr, k = k0 + kk;
            const float v0 = (r < R && k < K) ? X[(size_t)r * sr + k] : 0.f;
            const float v1 = (r < R && k + 1 < K) ? X[(size_t)r * sr + k + 1] : 0.f;
            S[rr * (TC_LD / 2) + kk / 2] = pack_bf16(v0, v1);
        }
    } else {
        for (int e = threadIdx.x; e < TC_TM * TC_TK / 2; e += 128) {
            const int rr = e % TC_TM, kk = 2 * (e / TC_TM);
            const int r = r0 + rr, k = k0 + kk;
            const float v0 = (r < R && k < K) ? X[(size_t)r * sr + (size_t)k * sk] : 0.f;
            const float v1 = (r < R && k + 1 < K) ? X[(size_t)r * sr + (size_t)(k + 1) * sk] : 0.f;
            S[rr * (TC_LD / 2) + kk / 2] = pack_bf16(v0, v1);
        }
    }
}
// C[m][n] = epi( sum_k A(m, k) B(k, n) ), A(m, k) = A[m*sam + k*sak], B(k, n) = B[k*sbk + n*sbn];
// split K as in gemm_kernel (kc a multiple of the 32-deep panel)
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, int kc, const float *__restrict__ A,
                                                     int sam, int sak, const float *__restrict__ B, int sbk, int sbn,
                                                     float *__restrict__ C, int ldc, int epi,
                                                     const float *__restrict__ bias, const float *__restrict__ Z,
                                                     int ldz, float *__restrict__ C2) {
    __shared__ unsigned As[TC_TM * TC_LD / 2];  // [m][k] BF16 pairs
    __shared__ unsigned Bs[TC_TN * TC_LD / 2];  // [n][k] BF16 pairs
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gid = lane >> 2, tig = lane & 3;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int m0 = blockIdx.y * TC_TM, n0 = blockIdx.x * TC_TN;
    const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
    C += (size_t)blockIdx.z * M * ldc;
    float acc[2][4][4] = {};
    for (int k0 = kb; k0 < ke; k0 += TC_TK) {
        tc_stage(As, A, M, ke, m0, k0, sam, sak);
        tc_stage(Bs, B, N, ke, n0, k0, sbn, sbk);
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < TC_TK; ks += 16) {
            unsigned af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + 16 * i + gid, c = (ks >> 1) + tig;
                af[i][0] = As[r * (TC_LD / 2) + c];
                af[i][1] = As[(r + 8) * (TC_LD / 2) + c];
                af[i][2] = As[r * (TC_LD / 2) + c + 4];
                af[i][3] = As[(r + 8) * (TC_LD / 2) + c + 4];
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = wn + 8 * j + gid, c = (ks >> 1) + tig;
                bf[j][0] = Bs[r * (TC_LD / 2) + c];
                bf[j][1] = Bs[r * (TC_LD / 2) + c + 4];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16_16816(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + wm + 16 * i + gid + (q >= 2 ? 8 : 0);
                const int n = n0 + wn + 8 * j + 2 * tig + (q & 1);
                if (m >= M || n >= N) continue;
                float v = acc[i][j][q];
                if (epi == EPI_BIAS || epi == EPI_BIAS_GELU) v += bias[n];
                if (epi == EPI_DGELU) v *= gelu_grad(Z[(size_t)m * ldz + n]);
                C[(size_t)m * ldc + n] = v;
                if (epi == EPI_BIAS_GELU) C2[(size_t)m * ldc + n] = gelu(v);
            }
}

// column sums (bias gradients): out[n] = sum_m X[m][n] in a fixed order: 32 columns per CTA,
// row group g (of 32) sums rows g, g + 32, ..., then the groups add in order
__global__ void __launch_bounds__(1024) colsum_kernel(int M, int N, const float *__restrict__ X, int ldx,
                                                      float *__restrict__ out) {
    __shared__ float red[32][33];
    const int c = threadIdx.x & 31, gr = threadIdx.x >> 5;
    const int n = blockIdx.x * 32 + c;
    float s = 0.f;
    if (n < N)
        for (int m = gr; m < M; m += 32) s += X[(size_t)m * ldx + n];
    red[gr][c] = s;
    __syncthreads();
    if (gr == 0 && n < N) {
        float t = 0.f;
        for (int g = 0; g < 32; ++g) t += red[g][c];
        out[n] = t;
    }
}

// split-K partial planes P[z][m][n] (z < S) summed in order into C[m][n]
__global__ void splitk_reduce_kernel(int M, int N, int S, const float *__restrict__ P, float *__restrict__ C, int ldc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M * N) return;
    float t = 0.f;
    for (int z = 0; z < S; ++z) t += P[(size_t)z * M * N + i];
    C[(size_t)(i / N) * ldc + i % N] = t;
}

// dY = 2 (Y - T)/(M N) and per-row squared error (for the loss)
__global__ void dloss_kernel(int M, int N, const float *__restrict__ Y, const float *__restrict__ T,
                             float *__restrict__ dY, float *__restrict__ rowerr) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    float s = 0.f, sc = 2.0f / ((float)M * (float)N);
    for (int n = 0; n < N; ++n) {
        float d = Y[(size_t)m * N + n] - T[(size_t)m * N + n];
        dY[(size_t)m * N + n] = sc * d;
        s = fmaf(d, d, s);
    }
    rowerr[m] = s;
}

__global__ void loss_reduce_kernel(int M, int N, const float *__restrict__ rowerr, float *__restrict__ loss) {
    __shared__ float red[256];
    float s = 0.f;
    for (int m = threadIdx.x; m < M; m += 256) s += rowerr[m];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[0] = red[0] / ((float)M * (float)N);
}

__global__ void adam_kernel(int n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float gi = g[i];
    float mi = b1 * m[i] + (1.f - b1) * gi;
    float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// tensor_core: BF16 operands on the tensor cores (the 256-wide layers); else the FP32 SIMT
// product with BF16 weights (the first layer, whose 5 inputs stay unrounded)
// part: scratch for split-K partial planes (SPLIT_MAX x M x N floats), or nullptr for no split.
// A long K over few output tiles (the weight gradients: K = the batch, 16 tiles of 256 x 256)
// is split so that about two CTAs per SM run; the planes are summed in a fixed order.
constexpr int SPLIT_MAX = 16, SPLIT_MIN_K = 256;
int gemm(cudaStream_t s, bool tensor_core, int M, int N, int K, const float *A, int sam, int sak, const float *B,
         int sbk, int sbn, int round_b, float *C, int ldc, int epi, const float *bias = nullptr,
         const float *Z = nullptr, int ldz = 0, float *C2 = nullptr, float *part = nullptr) {
    const int tm = tensor_core ? TC_TM : TM, tn = tensor_core ? TC_TN : TN, tk = tensor_core ? TC_TK : TK;
    const int tiles = ((N + tn - 1) / tn) * ((M + tm - 1) / tm);
    int split = 1;
    if (part && epi == EPI_PLAIN) {
        int dev = 0, sms = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        split = (2 * sms + tiles - 1) / tiles;
        split = max(1, min(split, min(SPLIT_MAX, K / SPLIT_MIN_K)));
    }
    int kc = (K + split - 1) / split;
    kc = (kc + tk - 1) / tk * tk;
    split = (K + kc - 1) / kc;
    float *dst = split > 1 ? part : C;
    const int ldd = split > 1 ? N : ldc;
    dim3 grid((N + tn - 1) / tn, (M + tm - 1) / tm, split);
    if (tensor_core)
        gemm_tc_kernel<<<grid, 128, 0, s>>>(M, N, K, kc, A, sam, sak, B, sbk, sbn, dst, ldd, epi, bias, Z, ldz, C2);
    else
        gemm_kernel<<<grid, 256, 0, s>>>(M, N, K, kc, A, sam, sak, B, sbk, sbn, round_b, dst, ldd, epi, bias, Z, ldz,
                                         C2);
    CUDA_TRY(cudaGetLastError());
    if (split > 1) {
        splitk_reduce_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(M, N, split, part, C, ldc);
        CUDA_TRY(cudaGetLastError());
    }
    return 0;
}

// workspace layout for n samples: Z[l] and H[l] for the 3 hidden layers (n x 256 each),
// Y (n x 80), dY (n x 80), two gradient buffers (n x 256), row errors (n), then the split-K
// partial planes of the weight gradients (SPLIT_MAX x 256 x 256)
struct Ws {
    float *Z[3], *H[3], *Y, *dY, *G0, *G1, *rowerr, *part;
};
Ws carve(float *w, int n) {
    Ws s;
    size_t o = 0;
    for (int l = 0; l < 3; ++l) {
        s.Z[l] = w + o;
        o += (size_t)n * HID;
        s.H[l] = w + o;
        o += (size_t)n * HID;
    }
    s.Y = w + o;
    o += (size_t)n * OUT;
    s.dY = w + o;
    o += (size_t)n * OUT;
    s.G0 = w + o;
    o += (size_t)n * HID;
    s.G1 = w + o;
    o += (size_t)n * HID;
    s.rowerr = w + o;
    o += (size_t)n;
    s.part = w + o;
    return s;
}

int forward_all(cudaStream_t s, int n, const float *P, const float *x, float *y, const Ws &w) {
    const float *in = x;
    for (int l = 0; l < NLAYER; ++l) {
        const int fi = fan_in(l), fo = fan_out(l);
        const float *W = P + w_off(l), *b = P + b_off(l);
        int rc;
        if (l < NLAYER - 1)
            rc = gemm(s, l > 0, n, fo, fi, in, fi, 1, W, 1, fi, 1, w.Z[l], fo, EPI_BIAS_GELU, b, nullptr, 0, w.H[l]);
        else
            rc = gemm(s, l > 0, n, fo, fi, in, fi, 1, W, 1, fi, 1, y, fo, EPI_BIAS, b);
        if (rc) return rc;
        in = l < NLAYER - 1 ? w.H[l] : nullptr;
    }
    return 0;
}

}  // namespace

extern "C" size_t mlp_workspace_bytes(int n) {
    return sizeof(float) * ((size_t)n * (6 * HID + 2 * OUT + 2 * HID) + n + (size_t)SPLIT_MAX * HID * HID);
}

extern "C" int mlp_forward(int n, const float *params, const float *x, float *y, float *workspace, void *stream) {
    ARG_CHECK(n >= 1, "n must be >= 1");
    ARG_CHECK(params && x && y && workspace, "NULL device pointer");
    Ws w = carve(workspace, n);
    return forward_all((cudaStream_t)stream, n, params, x, y, w);
}

extern "C" int mlp_backward(int n, const float *params, const float *x, const float *t, float *grad,
                            float *loss_out, float *workspace, void *stream) {
    ARG_CHECK(n >= 1, "n must be >= 1");
    ARG_CHECK(params && x && t && grad && loss_out && workspace, "NULL device pointer");
    cudaStream_t s = (cudaStream_t)stream;
    Ws w = carve(workspace, n);
    int rc = forward_all(s, n, params, x, w.Y, w);
    if (rc) return rc;
    dloss_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, OUT, w.Y, t, w.dY, w.rowerr);
    CUDA_TRY(cudaGetLastError());
    loss_reduce_kernel<<<1, 256, 0, s>>>(n, OUT, w.rowerr, loss_out);
    CUDA_TRY(cudaGetLastError());
    // backward through layers 3 .. 0; dZ of layer l lives in `dz` (n x fan_out(l))
    const float *dz = w.dY;
    float *bufs[2] = {w.G0, w.G1};
    for (int l = NLAYER - 1; l >= 0; --l) {
        const int fi = fan_in(l), fo = fan_out(l);
        const float *W = params + w_off(l);
        const float *hin = l > 0 ? w.H[l - 1] : x;
        // dW[o][i] = sum_s dZ[s][o] H[s][i]   (M = fo, N = fi, K = n)
        rc = gemm(s, l > 0, fo, fi, n, dz, 1, fo, hin, fi, 1, 0, grad + w_off(l), fi, EPI_PLAIN, nullptr, nullptr, 0,
                  nullptr, w.part);
        if (rc) return rc;
        colsum_kernel<<<(fo + 31) / 32, 1024, 0, s>>>(n, fo, dz, fo, grad + b_off(l));
        CUDA_TRY(cudaGetLastError());
        if (l > 0) {
            // dZ_{l-1}[s][i] = (sum_o dZ[s][o] W[o][i]) * gelu'(Z_{l-1}[s][i])
            float *dst = bufs[l & 1];
            rc = gemm(s, true, n, fi, fo, dz, fo, 1, W, fi, 1, 1, dst, fi, EPI_DGELU, nullptr, w.Z[l - 1], HID);
            if (rc) return rc;
            dz = dst;
        }
    }
    return 0;
}

extern "C" int mlp_adam(float *params, const float *grad, float *m, float *v, int step, float lr, void *stream) {
    ARG_CHECK(params && grad && m && v, "NULL device pointer");
    ARG_CHECK(step >= 1, "step counts from 1");
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(SWIMMER_MLP_NPARAM + 255) / 256, 256, 0, (cudaStream_t)stream>>>(SWIMMER_MLP_NPARAM, params, grad, m,
                                                                                   v, lr, b1, b2, eps, c1, c2);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

// ---------------------------------------------------------------------------------
// surrogate log-likelihood for delayed acceptance
// ---------------------------------------------------------------------------------
namespace {

__global__ void surr_input_kernel(int B, int np, const double *__restrict__ theta, float *__restrict__ x, double lo0,
                                  double lo1, double lo2, double lo3, double lo4, double hi0, double hi1, double hi2,
                                  double hi3, double hi4, double log10_kt, double omega) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    double v[5] = {theta[np * b], theta[np * b + 1], theta[np * b + 2], log10_kt, omega};
    double lo[5] = {lo0, lo1, lo2, lo3, lo4}, hi[5] = {hi0, hi1, hi2, hi3, hi4};
    for (int k = 0; k < 5; ++k) {
        double span = hi[k] - lo[k];
        x[5 * b + k] = span > 0.0 ? (float)(2.0 * (v[k] - lo[k]) / span - 1.0) : 0.f;
    }
}

__global__ void surr_loglik_kernel(int B, int np, const double *__restrict__ theta, const float *__restrict__ y,
                                   const double *__restrict__ norm, const double *__restrict__ obs, int stride,
                                   long long n_obs, double sigma, double *__restrict__ ll) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    // the sample's noise level: theta[3] times sigma with 4 unknowns
    const double sg = np == 4 ? sigma * theta[np * b + 3] : sigma;
    if (isnan(theta[np * b]) || !(sg > 0.0)) {
        ll[b] = -INFINITY;
        return;
    }
    double J = 0.0;
    for (int o = 0; o < OUT / 2; ++o) {
        long long row = (long long)o * stride + stride - 1;
        double px = norm[2 * o] + norm[OUT + 2 * o] * (double)y[OUT * b + 2 * o];
        double py = norm[2 * o + 1] + norm[OUT + 2 * o + 1] * (double)y[OUT * b + 2 * o + 1];
        double rx = obs[2 * row] - px, ry = obs[2 * row + 1] - py;
        J = fma(rx, rx, fma(ry, ry, J));
    }
    J *= (double)n_obs / (double)(OUT / 2);
    double s2 = sg * sg;
    ll[b] = -(double)n_obs * log(2.0 * 3.14159265358979323846 * s2) - 0.5 * J / s2;
}

}  // namespace

int run_surrogate_loglik(swimmer_handle *h, int B, const double *theta, const double *obs, double sigma,
                         double *loglik, cudaStream_t s) {
    const double *lo = h->surr_in_lo, *hi = h->surr_in_hi;
    const int np = n_params(h->cfg);
    surr_input_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, np, theta, h->surr_x, lo[0], lo[1], lo[2], lo[3], lo[4], hi[0],
                                                     hi[1], hi[2], hi[3], hi[4], h->surr_log10_kt, h->surr_omega);
    CUDA_TRY(cudaGetLastError());
    Ws w = carve(h->surr_ws, B);
    int rc = forward_all(s, B, h->surr_params, h->surr_x, h->surr_y, w);
    if (rc) return rc;
    surr_loglik_kernel<<<(B + 127) / 128, 128, 0, s>>>(B, np, theta, h->surr_y, h->surr_norm, obs, h->surr_obs_stride,
                                                       h->cfg.steps / h->cfg.obs_every, sigma, loglik);
    CUDA_TRY(cudaGetLastError());
    return 0;
}

extern "C" int swimmer_surrogate_set(swimmer_handle *h, const float *params, const double *in_lo, const double *in_hi,
                                     const double *out_mean, const double *out_std, int obs_stride, double log10_kt,
                                     double omega) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(params && in_lo && in_hi && out_mean && out_std, "NULL pointer");
    ARG_CHECK(obs_stride >= 1, "obs_stride must be >= 1");
    ARG_CHECK((long long)(OUT / 2) * obs_stride <= h->cfg.steps / h->cfg.obs_every,
              "surrogate outputs beyond the observation record");
    if (!h->surr_ws) {
        size_t bytes = mlp_workspace_bytes(h->cfg.b_max);
        CUDA_TRY(cudaMalloc((void **)&h->surr_ws, bytes));
    }
    for (int k = 0; k < 5; ++k) {
        h->surr_in_lo[k] = in_lo[k];
        h->surr_in_hi[k] = in_hi[k];
    }
    CUDA_TRY(cudaMemcpy(h->surr_params, params, sizeof(float) * SWIMMER_MLP_NPARAM, cudaMemcpyDeviceToDevice));
    CUDA_TRY(cudaMemcpy(h->surr_norm, out_mean, sizeof(double) * OUT, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(h->surr_norm + OUT, out_std, sizeof(double) * OUT, cudaMemcpyHostToDevice));
    const int trusted = 1;  // a surrogate set anew may screen until the plain model judges it
    CUDA_TRY(cudaMemcpy(h->surr_trust, &trusted, sizeof(int), cudaMemcpyHostToDevice));
    h->surr_obs_stride = obs_stride;
    h->surr_log10_kt = log10_kt;
    h->surr_omega = omega;
    h->surr_ready = 1;
    return 0;
}

extern "C" int surrogate_loglik_batch(swimmer_handle *h, int B, const double *theta, const double *obs, double sigma,
                                      double *loglik, void *stream) {
    ARG_CHECK(h != nullptr, "handle is NULL");
    ARG_CHECK(h->surr_ready, "surrogate not set (swimmer_surrogate_set)");
    ARG_CHECK(B >= 1 && B <= h->cfg.b_max, "B outside [1, b_max]");
    ARG_CHECK(theta && obs && loglik, "NULL device pointer");
    ARG_CHECK(sigma > 0.0, "sigma must be > 0");
    return run_surrogate_loglik(h, B, theta, obs, sigma, loglik, (cudaStream_t)stream);
}
