// Batched execution: many independent states (noisy trajectories, parameter sets of a circuit
// family) advanced by ONE persistent kernel launch.
//
// Each state is planned with gathered chunks (Sec. IV.A transpiler without data movement);
// a state whose qubits fit one chunk has a single section and runs its whole circuit in one
// shared-memory residency.  The launch drains a global work queue of (state, section, chunk)
// items.  Items are ordered section level by section level, round-robin over the states, so a
// state's section o+1 is queued after all of its section o.  A CTA that takes a chunk of
// section o waits (bounded) until every chunk of the state's earlier sections is done; since
// every earlier item was taken by a CTA that is running and never waits on a later item, the
// queue always drains.  Completion counters use release/acquire ordering and chunk data goes
// through L2 (ld.global.cg / st.global.cg) so that no stale L1 line is read.
#include "ptx.cuh"
#include "sv_internal.h"

namespace sv {
namespace {

constexpr uint64_t kWaitLimitNs = 4000000000ull;
constexpr int NCB = 256;  // threads per CTA
constexpr int RB = 4;     // register-group width

__device__ __forceinline__ int ld_acquire(const int *p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void cmul_acc(float &yr, float &yi, float mr, float mi, float xr, float xi) {
    yr = fmaf(mr, xr, yr);
    yr = fmaf(-mi, xi, yr);
    yi = fmaf(mr, xi, yi);
    yi = fmaf(mi, xr, yi);
}

// Dense / diagonal / permutation gates on a register group of 16 amplitudes (runtime bits).
template <int A>
__device__ __forceinline__ void g1(float (&r)[16], float (&i)[16], const DevGate<float> &g) {
    const float *m = g.m;
#pragma unroll
    for (int x = 0; x < 16; ++x) {
        if (x & (1 << A)) continue;
        const int y = x | (1 << A);
        const float ar = r[x], ai = i[x], br = r[y], bi = i[y];
        float pr = 0, pi = 0, qr = 0, qi = 0;
        if (g.op == OP_DENSE1) {
            cmul_acc(pr, pi, m[0], m[1], ar, ai);
            cmul_acc(pr, pi, m[2], m[3], br, bi);
            cmul_acc(qr, qi, m[4], m[5], ar, ai);
            cmul_acc(qr, qi, m[6], m[7], br, bi);
        } else {
            cmul_acc(pr, pi, m[0], m[1], ar, ai);
            cmul_acc(qr, qi, m[2], m[3], br, bi);
        }
        r[x] = pr; i[x] = pi; r[y] = qr; i[y] = qi;
    }
}

template <int A, int B>
__device__ __forceinline__ void g2(float (&r)[16], float (&i)[16], const DevGate<float> &g) {
    float mm[32];
    if (g.op == OP_DENSE2) {
#pragma unroll
        for (int k = 0; k < 32; ++k) mm[k] = g.m[k];
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) mm[k] = 0.f;
        if (g.op == OP_DIAG2) {
#pragma unroll
            for (int q = 0; q < 4; ++q) { mm[2 * (5 * q)] = g.m[2 * q]; mm[2 * (5 * q) + 1] = g.m[2 * q + 1]; }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) mm[2 * (4 * q + cc)] = ((int)g.m[q] == cc) ? 1.f : 0.f;
        }
    }
#pragma unroll
    for (int x = 0; x < 16; ++x) {
        if (x & ((1 << A) | (1 << B))) continue;
        const int id[4] = {x, x | (1 << A), x | (1 << B), x | (1 << A) | (1 << B)};
        float xr[4], xi[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) { xr[k] = r[id[k]]; xi[k] = i[id[k]]; }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float yr = 0, yi = 0;
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) cmul_acc(yr, yi, mm[2 * (4 * q + cc)], mm[2 * (4 * q + cc) + 1], xr[cc], xi[cc]);
            r[id[q]] = yr;
            i[id[q]] = yi;
        }
    }
}

__device__ __forceinline__ void apply(float (&r)[16], float (&i)[16], const DevGate<float> &g) {
    if (g.op == OP_DENSE1 || g.op == OP_DIAG1) {
        switch (g.code) {
            case 0: g1<0>(r, i, g); break;
            case 1: g1<1>(r, i, g); break;
            case 2: g1<2>(r, i, g); break;
            default: g1<3>(r, i, g); break;
        }
    } else {
        switch (g.code) {
            case 0 * 8 + 1: g2<0, 1>(r, i, g); break;
            case 0 * 8 + 2: g2<0, 2>(r, i, g); break;
            case 0 * 8 + 3: g2<0, 3>(r, i, g); break;
            case 1 * 8 + 2: g2<1, 2>(r, i, g); break;
            case 1 * 8 + 3: g2<1, 3>(r, i, g); break;
            default: g2<2, 3>(r, i, g); break;
        }
    }
}

__device__ __forceinline__ int64_t deposit(int64_t v, const int8_t *bits, int nbits) {
    int64_t x = 0;
    for (int k = 0; k < nbits; ++k)
        if ((v >> k) & 1) x |= int64_t(1) << bits[k];
    return x;
}

// Shared-memory slot of chunk-local amplitude i: the low four bits are XORed with the higher
// nibbles, so that 16 consecutive threads whose indices differ outside a register group hit
// distinct banks whichever four bits the group holds.
__device__ __forceinline__ int slot(int i) { return i ^ (((i >> 4) ^ (i >> 8) ^ (i >> 12)) & 15); }

__global__ void __launch_bounds__(NCB) k_batch(const BatchOp *__restrict__ ops, int nops,
                                               const unsigned char *__restrict__ progs, float2 *const *amps,
                                               int *ops_done, int *chunks_done, unsigned long long *next,
                                               int64_t total, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *chunk = reinterpret_cast<float2 *>(smem);
    unsigned char *sprog = smem + (size_t(1) << kBatchMaxChunkBits) * sizeof(float2);
    __shared__ int64_t s_item;
    __shared__ int s_op, s_cached, s_abort;
    __shared__ BatchOp s_bop;
    if (threadIdx.x == 0) { s_cached = -1; s_abort = 0; }
    __syncthreads();
    while (true) {
        if (threadIdx.x == 0) {
            s_item = (int64_t)atomicAdd(next, 1ull);
            int k = -1;
            if (s_item < total) {  // last op with first <= item
                int lo = 0, hi = nops - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) / 2;
                    if (ops[mid].first <= s_item) lo = mid; else hi = mid - 1;
                }
                k = lo;
                // earlier sections of this state must be complete
                const BatchOp &op = ops[k];
                const uint64_t t0 = ptx::globaltimer();
                while (ld_acquire(&ops_done[op.state]) < op.op) {
                    if (ptx::globaltimer() - t0 > kWaitLimitNs || *(volatile int *)err) {
                        atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                        s_abort = 1;
                        break;
                    }
                    __nanosleep(256);
                }
            }
            s_op = k;
            if (k >= 0) s_bop = ops[k];
        }
        __syncthreads();
        if (s_item >= total || s_abort) break;
        const BatchOp &op = s_bop;
        const int64_t j = s_item - op.first;
        const int ce = op.ce;
        // section program (register groups + gates) into shared memory, once per section
        if (s_cached != s_op) {
            const int bytes = op.prog_bytes;
            for (int k = threadIdx.x * 16; k < bytes; k += NCB * 16)
                *reinterpret_cast<uint4 *>(sprog + k) = *reinterpret_cast<const uint4 *>(progs + op.prog_off + k);
        }
        // gather chunk j: local index = (high bits | low run); state index = outer(j) | high | low
        float2 *amp = amps[op.state];
        const int64_t obase = deposit(j, op.outer, op.nouter);
        const int low = op.low;
        for (int e = threadIdx.x; e < (1 << ce); e += NCB) {
            const int r = e >> low, l = e & ((1 << low) - 1);
            const int64_t gidx = obase | deposit(r, op.high, op.nhigh) | l;
            chunk[slot(e)] = __ldcg(amp + gidx);
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cached = s_op;
        const DevSeg *segs = reinterpret_cast<const DevSeg *>(sprog);
        const DevGate<float> *gates =
            reinterpret_cast<const DevGate<float> *>(sprog + ((op.nseg * sizeof(DevSeg) + 15) & ~size_t(15)));
        for (int si = 0; si < op.nseg; ++si) {
            const DevSeg &sg = segs[si];
            const int G = 1 << (ce - RB);
            for (int g = threadIdx.x; g < G; g += NCB) {
                // natural layout throughout: group base = bits of g inserted around the group bits
                int base = g;
#pragma unroll
                for (int q = 0; q < RB; ++q) {
                    const int p = sg.pos[q];
                    base = ((base >> p) << (p + 1)) | (base & ((1 << p) - 1));
                }
                int off[16];
#pragma unroll
                for (int b = 0; b < 16; ++b) {
                    int o = 0;
#pragma unroll
                    for (int q = 0; q < RB; ++q)
                        if (b & (1 << q)) o |= 1 << sg.pos[q];
                    off[b] = base | o;
                }
                float re[16], im[16];
#pragma unroll
                for (int b = 0; b < 16; ++b) { const float2 v = chunk[slot(off[b])]; re[b] = v.x; im[b] = v.y; }
                for (int gi = sg.g0; gi < sg.g1; ++gi) apply(re, im, gates[gi]);
#pragma unroll
                for (int b = 0; b < 16; ++b) chunk[slot(off[b])] = make_float2(re[b], im[b]);
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < (1 << ce); e += NCB) {
            const int r = e >> low, l = e & ((1 << low) - 1);
            const int64_t gidx = obase | deposit(r, op.high, op.nhigh) | l;
            __stcg(amp + gidx, chunk[slot(e)]);
        }
        __threadfence();
        __syncthreads();
        if (threadIdx.x == 0) {
            if (atomicAdd(&chunks_done[s_op], 1) == op.nchunks - 1) {
                __threadfence();
                atomicAdd(&ops_done[op.state], 1);  // section complete: release the state's next one
            }
        }
    }
}

}  // namespace

void launch_batch(const void *dev_ops, int nops, const void *dev_progs, void *const *dev_amps, int *dev_ops_done,
                  int *dev_chunks_done, unsigned long long *dev_next, int64_t total, int *dev_err, cudaStream_t st) {
    const size_t smem = (size_t(1) << kBatchMaxChunkBits) * sizeof(float2) + kBatchMaxProgBytes;
    check_cuda(cudaFuncSetAttribute(k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "cudaFuncSetAttribute(batch)");
    int per_sm = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch, NCB, smem), "occupancy(batch)");
    if (per_sm < 1) per_sm = 1;
    // every CTA resident at once: a waiting CTA only ever waits for items already taken
    const int grid = num_sms() * per_sm;
    k_batch<<<grid, NCB, smem, st>>>((const BatchOp *)dev_ops, nops, (const unsigned char *)dev_progs,
                                     (float2 *const *)dev_amps, dev_ops_done, dev_chunks_done, dev_next, total,
                                     dev_err);
    check_cuda(cudaGetLastError(), "batch kernel launch");
}

}  // namespace sv
