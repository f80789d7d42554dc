// Pauli expectation value that allocates no memory (sv_expval_pauli_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a readout: code running
// under a memory pool or budget they do not own, real-time loops where cudaMalloc/cudaFree
// would synchronise the device, or hosts that hand this library a pre-sized arena and forbid
// allocations afterwards.  This entry point computes the same quantity as sv_expval_pauli
// but keeps its partial sums in a fixed array compiled into the library instead of the
// handle's lazily allocated scratch buffer.
//
// The array lives in device memory for as long as the library is loaded, on every GPU that
// loads it.  Its host-side name is only a stand-in, so the host fetches the device address
// with cudaGetSymbolAddress once per device (on the first call made on that device, with that
// device current) and passes it to the kernels.  All calls share the array: two calls whose
// kernels overlap on the GPU (for example on different streams) race on it.
#include <array>
#include <mutex>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxPartials = 4096;  // up to 4096 CTAs of partial sums (64 KiB of scratch)
constexpr int kMaxDevices = 64;

// (re, im) partial sums of up to kMaxPartials CTAs, then the final (re, im) pair.
static __device__ __align__(256) double g_expval_scratch[2 * kMaxPartials + 2];

std::mutex g_mu;
std::array<double *, kMaxDevices> g_addr{};

double *scratch_address(int dev) {
    if (dev < 0 || dev >= kMaxDevices) fail(SV_ERR_UNSUPPORTED, "sv_expval_pauli_noalloc: device index too large");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        double *p = nullptr;
        check_cuda(cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_expval_scratch),
                   "cudaGetSymbolAddress(expval scratch)");
        g_addr[dev] = p;
    }
    return g_addr[dev];
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// CTA b sums conj(a_{j^x}) a_j (-1)^{popc(j&z)} over its contiguous range of j and writes
// (re, im) to scratch[2b], scratch[2b+1]; every CTA overwrites its own slots, so nothing has
// to start at zero.
template <typename T2>
__global__ void __launch_bounds__(kThreads) k_expval_partials_noalloc(const T2 *__restrict__ a, int64_t len,
                                                                      uint64_t x, uint64_t z, double *scratch) {
    __shared__ double red[2][kThreads / 32];
    const int64_t per = (len + gridDim.x - 1) / gridDim.x;
    const int64_t lo = (int64_t)blockIdx.x * per, hi = lo + per < len ? lo + per : len;
    double sr = 0, si = 0;
    for (int64_t j = lo + threadIdx.x; j < hi; j += kThreads) {
        const T2 u = a[(uint64_t)j ^ x], v = a[j];
        double tr = (double)u.x * (double)v.x + (double)u.y * (double)v.y;
        double ti = (double)u.x * (double)v.y - (double)u.y * (double)v.x;
        if (__popcll((unsigned long long)j & z) & 1) { tr = -tr; ti = -ti; }
        sr += tr;
        si += ti;
    }
    sr = warp_sum(sr);
    si = warp_sum(si);
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        double r = threadIdx.x < kThreads / 32 ? red[0][threadIdx.x] : 0.0;
        double i = threadIdx.x < kThreads / 32 ? red[1][threadIdx.x] : 0.0;
        r = warp_sum(r);
        i = warp_sum(i);
        if (threadIdx.x == 0) {
            scratch[2 * blockIdx.x] = r;
            scratch[2 * blockIdx.x + 1] = i;
        }
    }
}

// One thread adds the partials in CTA order into the final pair.
__global__ void k_expval_final_noalloc(double *scratch, int nparts) {
    double r = 0, i = 0;
    for (int b = 0; b < nparts; ++b) {
        r += scratch[2 * b];
        i += scratch[2 * b + 1];
    }
    scratch[2 * kMaxPartials] = r;
    scratch[2 * kMaxPartials + 1] = i;
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_expval_pauli_noalloc(sv_handle h, uint64_t x, uint64_t z, double *out) {
    try {
        if (!h || !out) fail(SV_ERR_ARG, "sv_expval_pauli_noalloc: null argument");
        if ((x >> h->n) || (z >> h->n)) fail(SV_ERR_ARG, "sv_expval_pauli_noalloc: Pauli mask outside the register");
        int dev = -1;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        if (dev != h->device) fail(SV_ERR_ARG, "sv_expval_pauli_noalloc: the handle's device is not current");
        const int64_t len = int64_t(1) << h->n;
        const int64_t nb = std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8, len / 256));
        if (nb > kMaxPartials)
            fail(SV_ERR_UNSUPPORTED, "sv_expval_pauli_noalloc: needs " + std::to_string(nb) +
                                         " partial sums, more than the fixed scratch holds (4096)");
        double *scratch = scratch_address(dev);
        if (h->dtype == SV_C64)
            k_expval_partials_noalloc<float2><<<(unsigned)nb, kThreads, 0, h->stream>>>((const float2 *)h->amp, len, x,
                                                                                        z, scratch);
        else
            k_expval_partials_noalloc<double2><<<(unsigned)nb, kThreads, 0, h->stream>>>((const double2 *)h->amp, len,
                                                                                         x, z, scratch);
        check_cuda(cudaGetLastError(), "expval (no-alloc) kernel launch");
        k_expval_final_noalloc<<<1, 1, 0, h->stream>>>(scratch, (int)nb);
        check_cuda(cudaGetLastError(), "expval (no-alloc) final kernel launch");
        double res[2] = {0, 0};
        check_cuda(cudaMemcpyAsync(res, scratch + 2 * kMaxPartials, sizeof(res), cudaMemcpyDeviceToHost, h->stream),
                   "cudaMemcpyAsync(expval result)");
        // synchronise and report a failure an earlier kernel on this handle left in its error word
        check_dev_error(h);
        double sr = res[0], si = res[1];
        switch (__builtin_popcountll(x & z) & 3) {  // times i^{popc(x & z)}
            case 1: { const double t = sr; sr = -si; si = t; break; }
            case 2: sr = -sr; si = -si; break;
            case 3: { const double t = sr; sr = si; si = -t; break; }
            default: break;
        }
        out[0] = sr;
        out[1] = si;
        return SV_OK;
    } catch (const sv::Error &e) {
        sv::set_error(e.msg);
        return e.code;
    }
}
