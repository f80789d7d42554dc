// Readouts with FP64 accumulation: probabilities |a_i|^2 (Sec. II.A), norm, Pauli-word
// expectation values and the two device steps of inverse-CDF sampling (per-range sums, then
// the in-range scan for each shot).
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kThreads = 256;

template <typename T2>
__device__ __forceinline__ double p2(const T2 &v) {
    return (double)v.x * (double)v.x + (double)v.y * (double)v.y;
}

template <typename T2>
__global__ void k_probs(const T2 *__restrict__ a, double *__restrict__ out, int64_t first, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = p2(a[first + i]);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NT>
__device__ __forceinline__ double block_sum(double v) {
    __shared__ double red[NT / 32];
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double s = 0;
    if (threadIdx.x < 32) {
        s = threadIdx.x < NT / 32 ? red[threadIdx.x] : 0.0;
        s = warp_sum(s);
    }
    __syncthreads();
    return s;
}

// Each CTA sums a contiguous range of the state (the partials are added in CTA order, so the
// result does not depend on scheduling).  complex64: threads read 16-byte vectors (two
// amplitudes); squares are summed in FP32 over runs of 8 vectors per thread (16 terms, all
// non-negative) and the runs accumulated in FP64 -- FP64 arithmetic on every element would
// make this pass FP64-bound instead of HBM-bound on GB300.  complex128: FP64 throughout.
__global__ void __launch_bounds__(kThreads) k_partial_norm_c64(const float4 *__restrict__ v, int64_t nv,
                                                               double *partials) {
    const int64_t per = (nv + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < nv ? lo + per : nv;
    double s = 0;
    for (int64_t base = lo + threadIdx.x; base < hi; base += 8 * kThreads) {
        float f = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int64_t i = base + (int64_t)k * kThreads;
            if (i < hi) {
                const float4 q = v[i];
                f = fmaf(q.x, q.x, fmaf(q.y, q.y, fmaf(q.z, q.z, fmaf(q.w, q.w, f))));
            }
        }
        s += (double)f;
    }
    s = block_sum<kThreads>(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_partial_norm_c128(const double2 *__restrict__ a, int64_t len,
                                                                double *partials) {
    const int64_t per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < len ? lo + per : len;
    double s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) s += p2(a[i]);
    s = block_sum<kThreads>(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// Norm restoration after a tensor-core circuit: d = sqrt(n_in / n_out) - 1 from the two sets of
// norm partials (input at part[0, nb), output at part[nb, 2 nb)), applied only when every fused
// group was unitary (*flag != 0).
__global__ void k_renorm_factor(const double *__restrict__ part, int nb, const int *__restrict__ flag,
                                float *__restrict__ out) {
    double nin = 0, nout = 0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        nin += part[b];
        nout += part[nb + b];
    }
    nin = block_sum<kThreads>(nin);
    nout = block_sum<kThreads>(nout);
    if (threadIdx.x == 0) out[0] = (*flag != 0 && nout > 0) ? (float)(sqrt(nin / nout) - 1.0) : 0.f;
}

// a <- a (1 + d), applied as a small correction so that the factor's FP32 rounding next to 1
// does not become the error.
template <typename V>
__global__ void __launch_bounds__(kThreads) k_renorm_apply(V *__restrict__ v, int64_t nv, const float *__restrict__ dp) {
    const float d = *dp;
    if (d == 0.f) return;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < nv; i += (int64_t)gridDim.x * kThreads) {
        V q = v[i];
        q.x = fmaf(q.x, d, q.x);
        q.y = fmaf(q.y, d, q.y);
        q.z = fmaf(q.z, d, q.z);
        q.w = fmaf(q.w, d, q.w);
        v[i] = q;
    }
}

// sum_j conj(a_{j^x}) a_j (-1)^{popc(j & z)}; the phase i^{popc(x&z)} is applied on the host.
template <typename T2>
__global__ void __launch_bounds__(kThreads) k_partial_expval(const T2 *__restrict__ a, int64_t len, uint64_t x,
                                                             uint64_t z, double *partials) {
    const int64_t per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < len ? lo + per : len;
    double sr = 0, si = 0;
    for (int64_t j = lo + threadIdx.x; j < hi; j += kThreads) {
        const T2 u = a[(uint64_t)j ^ x], v = a[j];
        // conj(u) * v
        double tr = (double)u.x * (double)v.x + (double)u.y * (double)v.y;
        double ti = (double)u.x * (double)v.y - (double)u.y * (double)v.x;
        if (__popcll((unsigned long long)j & z) & 1) { tr = -tr; ti = -ti; }
        sr += tr;
        si += ti;
    }
    sr = block_sum<kThreads>(sr);
    si = block_sum<kThreads>(si);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sr;
        partials[2 * blockIdx.x + 1] = si;
    }
}

// sums[b] = sum of |a_i|^2 over i in [b 2^sb, (b+1) 2^sb), one warp per range, summed in
// index order within each lane then across lanes.
template <typename T2>
__global__ void __launch_bounds__(kThreads) k_block_sums(const T2 *__restrict__ a, int sb, int64_t nb, double *sums) {
    const int64_t w = ((int64_t)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nb) return;
    const int64_t lo = w << sb;
    const int64_t len = int64_t(1) << sb;
    double s = 0;
    for (int64_t i = lane; i < len; i += 32) s += p2(a[lo + i]);
    s = warp_sum(s);
    if (lane == 0) sums[w] = s;
}

// Shot k: scan range shot_block[k] in index order from prefix[k] until the running sum
// exceeds target[k]; returns the first index that does (or the range's last non-zero index
// if rounding never lets it).
template <typename T2>
__global__ void k_sample_within(const T2 *__restrict__ a, int sb, const double *__restrict__ prefix,
                                const int64_t *__restrict__ blk, const double *__restrict__ target, int64_t shots,
                                uint64_t *out) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= shots) return;
    const int64_t lo = blk[k] << sb, len = int64_t(1) << sb;
    double acc = prefix[k];
    const double t = target[k];
    int64_t last_nz = lo;
    int64_t found = -1;
    for (int64_t i = 0; i < len; ++i) {
        const double p = p2(a[lo + i]);
        if (p > 0) last_nz = lo + i;
        acc += p;
        if (acc > t) { found = lo + i; break; }
    }
    out[k] = (uint64_t)(found >= 0 ? found : last_nz);
}

}  // namespace

void launch_probs(int dtype, const void *state, int n, double *out, int64_t first, int64_t count, cudaStream_t st) {
    (void)n;
    const int grid = (int)std::min<int64_t>((count + kThreads - 1) / kThreads, (int64_t)num_sms() * 16);
    if (dtype == SV_C64)
        k_probs<float2><<<grid, kThreads, 0, st>>>((const float2 *)state, out, first, count);
    else
        k_probs<double2><<<grid, kThreads, 0, st>>>((const double2 *)state, out, first, count);
    check_cuda(cudaGetLastError(), "probabilities kernel launch");
}

void launch_partial_norm(int dtype, const void *state, int n, double *partials, int nblocks, cudaStream_t st) {
    const int64_t len = int64_t(1) << n;
    if (dtype == SV_C64)  // n >= 1: an even number of amplitudes
        k_partial_norm_c64<<<nblocks, kThreads, 0, st>>>((const float4 *)state, len / 2, partials);
    else
        k_partial_norm_c128<<<nblocks, kThreads, 0, st>>>((const double2 *)state, len, partials);
    check_cuda(cudaGetLastError(), "norm kernel launch");
}

void launch_renorm(int dtype, void *state, int n, const double *partials, int nblocks, const int *flag, float *d,
                   cudaStream_t st) {
    k_renorm_factor<<<1, kThreads, 0, st>>>(partials, nblocks, flag, d);
    check_cuda(cudaGetLastError(), "renorm factor launch");
    const int64_t nv = (int64_t(1) << n) / (dtype == SV_C64 ? 2 : 1);
    const int grid = (int)std::min<int64_t>((nv + kThreads - 1) / kThreads, (int64_t)num_sms() * 8);
    if (dtype == SV_C64)
        k_renorm_apply<float4><<<grid, kThreads, 0, st>>>((float4 *)state, nv, d);
    else
        fail(SV_ERR_UNSUPPORTED, "norm restoration is for complex64 tensor-core circuits");
    check_cuda(cudaGetLastError(), "renorm launch");
}

void launch_partial_expval(int dtype, const void *state, int n, uint64_t x, uint64_t z, double *partials, int nblocks,
                           cudaStream_t st) {
    const int64_t len = int64_t(1) << n;
    if (dtype == SV_C64)
        k_partial_expval<float2><<<nblocks, kThreads, 0, st>>>((const float2 *)state, len, x, z, partials);
    else
        k_partial_expval<double2><<<nblocks, kThreads, 0, st>>>((const double2 *)state, len, x, z, partials);
    check_cuda(cudaGetLastError(), "expval kernel launch");
}

void launch_block_sums(int dtype, const void *state, int n, int sb, double *sums, cudaStream_t st) {
    const int64_t nb = int64_t(1) << (n - sb);
    const int grid = (int)((nb * 32 + kThreads - 1) / kThreads);
    if (dtype == SV_C64)
        k_block_sums<float2><<<grid, kThreads, 0, st>>>((const float2 *)state, sb, nb, sums);
    else
        k_block_sums<double2><<<grid, kThreads, 0, st>>>((const double2 *)state, sb, nb, sums);
    check_cuda(cudaGetLastError(), "block-sum kernel launch");
}

void launch_sample_within(int dtype, const void *state, int n, int sb, const double *prefix, const int64_t *blk,
                          const double *target, int64_t shots, uint64_t *out, cudaStream_t st) {
    (void)n;
    const int grid = (int)((shots + 127) / 128);
    if (dtype == SV_C64)
        k_sample_within<float2><<<grid, 128, 0, st>>>((const float2 *)state, sb, prefix, blk, target, shots, out);
    else
        k_sample_within<double2><<<grid, 128, 0, st>>>((const double2 *)state, sb, prefix, blk, target, shots, out);
    check_cuda(cudaGetLastError(), "sampling kernel launch");
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output s of the stream seeded with `seed`
// mixes seed + (s+1) * 0x9E3779B97F4A7C15; the uniform takes its top 53 bits.
double splitmix_uniform(uint64_t seed, uint64_t s) {
    uint64_t z = seed + (s + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

}  // namespace sv
