// Half-state gather and scatter for exchanges between pieces of a partitioned state (Sec. II.B:
// the state is divided on its top qubits over processes; Sec. IV.C, Fig. 10 case (a): a
// chunk_swap of a local qubit s with a partition qubit moves the half of each piece whose bit s
// differs from the piece's own value of the partition qubit to the partner piece, whose matching
// half comes back into the same places).  Pack copies the amplitudes with bit `bit` equal to
// `value`, in index order, into a contiguous buffer; unpack writes such a buffer back.
#include "sv_internal.h"

namespace sv {
namespace {

template <typename T2>
__global__ void k_pack_half(const T2 *__restrict__ a, int bit, int value, int64_t half, T2 *__restrict__ out) {
    const int64_t lo = (int64_t(1) << bit) - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = ((k & ~lo) << 1) | (int64_t(value) << bit) | (k & lo);
        out[k] = a[i];
    }
}

template <typename T2>
__global__ void k_unpack_half(T2 *__restrict__ a, int bit, int value, int64_t half, const T2 *__restrict__ in) {
    const int64_t lo = (int64_t(1) << bit) - 1;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < half; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = ((k & ~lo) << 1) | (int64_t(value) << bit) | (k & lo);
        a[i] = in[k];
    }
}

template <typename T2>
void launch_half(bool pack, void *state, int n, int bit, int value, void *buf, cudaStream_t st) {
    const int64_t half = int64_t(1) << (n - 1);
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((half + threads - 1) / threads, (int64_t)num_sms() * 16);
    if (pack)
        k_pack_half<T2><<<(unsigned)blocks, threads, 0, st>>>((const T2 *)state, bit, value, half, (T2 *)buf);
    else
        k_unpack_half<T2><<<(unsigned)blocks, threads, 0, st>>>((T2 *)state, bit, value, half, (const T2 *)buf);
    check_cuda(cudaGetLastError(), "half-state copy launch");
}

}  // namespace

void launch_shard_half(bool pack, int dtype, void *state, int n, int bit, int value, void *buf, cudaStream_t st) {
    if (dtype == SV_C64) launch_half<float2>(pack, state, n, bit, value, buf, st);
    else launch_half<double2>(pack, state, n, bit, value, buf, st);
}

}  // namespace sv
