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

// Each CTA sums a contiguous range of 2^n / gridDim.x amplitudes (the partials are added on
// the host in CTA order, so the result does not depend on scheduling).
template <typename T2>
__global__ void __launch_bounds__(kThreads) k_partial_norm(const T2 *__restrict__ a, int64_t len, double *partials) {
    const int64_t per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < len ? lo + per : len;
    double s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) s += p2(a[i]);
    s = block_sum<kThreads>(s);
    if (threadIdx.x == 0) partials[blockIdx.x] = s;
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
    if (dtype == SV_C64)
        k_partial_norm<float2><<<nblocks, kThreads, 0, st>>>((const float2 *)state, len, partials);
    else
        k_partial_norm<double2><<<nblocks, kThreads, 0, st>>>((const double2 *)state, len, partials);
    check_cuda(cudaGetLastError(), "norm kernel launch");
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
