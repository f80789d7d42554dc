// Cost-model network on the GPU: forward pass, per-CTA partial gradients of the mean squared
// error, and the reduction of those partials fused with the Adam update (Kingma & Ba, 2015).
//
// Network: x (16) -> relu(W1 x + b1) (64) -> relu(W2 h1 + b2) (64) -> w3 . h2 + b3.  Flat
// parameter layout: W1 (64 x 16 row-major), b1, W2 (64 x 64 row-major), b2, w3, b3.
//
// One warp works on one sample at a time; lane l owns hidden units l and l + 32 of both layers.
// Weight rows are staged in shared memory with odd strides (17, 65) so that the lanes of a warp
// reading one column of W1 or W2 hit distinct banks.  Gradients are accumulated per CTA (each
// lane owns its rows, no atomics) and summed over CTAs in a fixed order, so a training step is
// deterministic for a given grid.
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int NIN = 16, NH = 64;
constexpr int P_W1 = 0, P_B1 = NH * NIN, P_W2 = P_B1 + NH, P_B2 = P_W2 + NH * NH, P_W3 = P_B2 + NH, P_B3 = P_W3 + NH;
constexpr int NPARAM = P_B3 + 1;
// padded shared layout
constexpr int S1 = NIN + 1, S2 = NH + 1;
constexpr int Q_W1 = 0, Q_B1 = NH * S1, Q_W2 = Q_B1 + NH, Q_B2 = Q_W2 + NH * S2, Q_W3 = Q_B2 + NH, Q_B3 = Q_W3 + NH;
constexpr int NSHARED = Q_B3 + 1;
static_assert(NPARAM == 5313, "parameter layout");

__device__ __forceinline__ void stage_params(float *sp, const float *__restrict__ P) {
    for (int k = threadIdx.x; k < NH * NIN; k += blockDim.x) sp[Q_W1 + (k / NIN) * S1 + k % NIN] = P[P_W1 + k];
    for (int k = threadIdx.x; k < NH * NH; k += blockDim.x) sp[Q_W2 + (k / NH) * S2 + k % NH] = P[P_W2 + k];
    for (int k = threadIdx.x; k < NH; k += blockDim.x) {
        sp[Q_B1 + k] = P[P_B1 + k];
        sp[Q_B2 + k] = P[P_B2 + k];
        sp[Q_W3 + k] = P[P_W3 + k];
    }
    if (threadIdx.x == 0) sp[Q_B3] = P[P_B3];
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Forward pass of one sample by one warp.  h1 (64 floats, shared) receives the first layer;
// returns y on every lane and leaves a1, a2 of the lane's units in registers.
__device__ __forceinline__ float fwd_warp(const float *sp, const float *x, float *h1, float (&a1)[2], float (&a2)[2],
                                          float (&h2)[2]) {
    const int lane = threadIdx.x & 31;
    const float xv = lane < NIN ? x[lane] : 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int u = lane + 32 * k;
        float a = sp[Q_B1 + u];
#pragma unroll
        for (int f = 0; f < NIN; ++f) a = fmaf(sp[Q_W1 + u * S1 + f], __shfl_sync(0xffffffffu, xv, f), a);
        a1[k] = a;
        h1[u] = fmaxf(a, 0.f);
    }
    __syncwarp();
    float part = 0.f;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int u = lane + 32 * k;
        float a = sp[Q_B2 + u];
#pragma unroll 16
        for (int i = 0; i < NH; ++i) a = fmaf(sp[Q_W2 + u * S2 + i], h1[i], a);
        a2[k] = a;
        h2[k] = fmaxf(a, 0.f);
        part = fmaf(sp[Q_W3 + u], h2[k], part);
    }
    return warp_sum(part) + sp[Q_B3];
}

__global__ void __launch_bounds__(256) k_mlp_fwd(const float *__restrict__ P, const float *__restrict__ X, int64_t B,
                                                 float *__restrict__ Y) {
    __shared__ float sp[NSHARED];
    __shared__ float sh1[8][NH];
    stage_params(sp, P);
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t s = (int64_t)blockIdx.x * 8 + warp; s < B; s += (int64_t)gridDim.x * 8) {
        float a1[2], a2[2], h2[2];
        const float y = fwd_warp(sp, X + s * NIN, sh1[warp], a1, a2, h2);
        if (lane == 0) Y[s] = y;
        __syncwarp();
    }
}

// Partial gradient of L = (1/B) sum (y - t)^2 over the samples idx[start + j], j = blockIdx.x,
// blockIdx.x + gridDim.x, ... < B.  One warp per CTA; part[blockIdx.x] gets the CTA's sum in the
// flat layout, lpart[blockIdx.x] its share of the loss.
__global__ void __launch_bounds__(32) k_mlp_grad(const float *__restrict__ P, const float *__restrict__ X,
                                                 const float *__restrict__ T, const int32_t *__restrict__ idx,
                                                 int64_t start, int64_t B, float *__restrict__ part,
                                                 double *__restrict__ lpart) {
    __shared__ float sp[NSHARED];
    __shared__ float sg[NSHARED];
    __shared__ float sh1[NH], sd2[NH];
    stage_params(sp, P);
    for (int k = threadIdx.x; k < NSHARED; k += 32) sg[k] = 0.f;
    __syncwarp();
    const int lane = threadIdx.x;
    const float inv_b = 1.f / (float)B;
    double lsum = 0.0;
    for (int64_t j = blockIdx.x; j < B; j += gridDim.x) {
        const int64_t s = idx ? idx[start + j] : start + j;
        const float *x = X + s * NIN;
        float a1[2], a2[2], h2[2];
        const float y = fwd_warp(sp, x, sh1, a1, a2, h2);
        const float err = y - T[s];
        const float dy = 2.f * err * inv_b;
        if (lane == 0) {
            lsum += (double)err * (double)err / (double)B;
            sg[Q_B3] += dy;
        }
        float d2[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int u = lane + 32 * k;
            sg[Q_W3 + u] = fmaf(dy, h2[k], sg[Q_W3 + u]);
            d2[k] = a2[k] > 0.f ? dy * sp[Q_W3 + u] : 0.f;
            sg[Q_B2 + u] += d2[k];
            sd2[u] = d2[k];
#pragma unroll 16
            for (int i = 0; i < NH; ++i) sg[Q_W2 + u * S2 + i] = fmaf(d2[k], sh1[i], sg[Q_W2 + u * S2 + i]);
        }
        __syncwarp();
        const float xv = lane < NIN ? x[lane] : 0.f;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int i = lane + 32 * k;
            float acc = 0.f;
#pragma unroll 16
            for (int u = 0; u < NH; ++u) acc = fmaf(sp[Q_W2 + u * S2 + i], sd2[u], acc);
            const float d1 = a1[k] > 0.f ? acc : 0.f;
            sg[Q_B1 + i] += d1;
#pragma unroll
            for (int f = 0; f < NIN; ++f)
                sg[Q_W1 + i * S1 + f] = fmaf(d1, __shfl_sync(0xffffffffu, xv, f), sg[Q_W1 + i * S1 + f]);
        }
        __syncwarp();
    }
    float *out = part + (size_t)blockIdx.x * NPARAM;
    for (int k = lane; k < NH * NIN; k += 32) out[P_W1 + k] = sg[Q_W1 + (k / NIN) * S1 + k % NIN];
    for (int k = lane; k < NH * NH; k += 32) out[P_W2 + k] = sg[Q_W2 + (k / NH) * S2 + k % NH];
    for (int k = lane; k < NH; k += 32) {
        out[P_B1 + k] = sg[Q_B1 + k];
        out[P_B2 + k] = sg[Q_B2 + k];
        out[P_W3 + k] = sg[Q_W3 + k];
    }
    if (lane == 0) {
        out[P_B3] = sg[Q_B3];
        lpart[blockIdx.x] = lsum;
    }
}

// g = sum of the nblk partials (fixed order).  mode 0: write g to `grad`; mode 1: Adam update
// of P with moments M, V (c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)).  Thread 0 also sums the
// loss partials into *loss.
__global__ void k_mlp_reduce(const float *__restrict__ part, int nblk, const double *__restrict__ lpart, double *loss,
                             int mode, float *__restrict__ grad, float *__restrict__ P, float *__restrict__ M,
                             float *__restrict__ V, float lr, float c1, float c2) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0) {
        double l = 0.0;
        for (int b = 0; b < nblk; ++b) l += lpart[b];
        *loss = l;
    }
    if (p >= NPARAM) return;
    float g = 0.f;
    for (int b = 0; b < nblk; ++b) g += part[(size_t)b * NPARAM + p];
    if (mode == 0) {
        grad[p] = g;
        return;
    }
    const float m = 0.9f * M[p] + 0.1f * g;
    const float v = 0.999f * V[p] + 0.001f * g * g;
    M[p] = m;
    V[p] = v;
    P[p] -= lr * (m * c1) / (sqrtf(v * c2) + 1e-8f);
}

}  // namespace

int mlp_param_count() { return NPARAM; }

void launch_mlp_fwd(const float *P, const float *X, int64_t B, float *Y, cudaStream_t st) {
    if (B <= 0) return;
    const int grid = (int)std::min<int64_t>((B + 7) / 8, 4 * (int64_t)num_sms());
    k_mlp_fwd<<<grid, 256, 0, st>>>(P, X, B, Y);
    check_cuda(cudaGetLastError(), "mlp forward launch");
}

int mlp_grad_blocks(int64_t B) { return (int)std::max<int64_t>(1, std::min<int64_t>(B, 128)); }

void launch_mlp_grad(const float *P, const float *X, const float *T, const int32_t *idx, int64_t start, int64_t B,
                     float *part, double *lpart, cudaStream_t st) {
    k_mlp_grad<<<mlp_grad_blocks(B), 32, 0, st>>>(P, X, T, idx, start, B, part, lpart);
    check_cuda(cudaGetLastError(), "mlp gradient launch");
}

void launch_mlp_reduce(const float *part, int nblk, const double *lpart, double *loss, int mode, float *grad, float *P,
                       float *M, float *V, float lr, float c1, float c2, cudaStream_t st) {
    k_mlp_reduce<<<(NPARAM + 255) / 256, 256, 0, st>>>(part, nblk, lpart, loss, mode, grad, P, M, V, lr, c1, c2);
    check_cuda(cudaGetLastError(), "mlp reduce launch");
}

}  // namespace sv
