// Batched execution: many independent states (noisy trajectories, parameter sets of a circuit
// family) advanced by ONE persistent kernel launch.
//
// Each state is planned with gathered chunks (Sec. IV.A transpiler without data movement);
// a state whose qubits fit one chunk has a single section and runs its whole circuit in one
// shared-memory residency (a long program is streamed through shared memory in pieces).  The launch drains a global work queue of (state, section, chunk)
// items.  Items are ordered section level by section level, round-robin over the states, so a
// state's section o+1 is queued after all of its section o.  A CTA that takes a chunk of
// section o waits (bounded) until every chunk of the state's earlier sections is done; since
// every earlier item was taken by a CTA that is running and never waits on a later item, the
// queue always drains.  Completion counters use release/acquire ordering and chunk data goes
// through L2 (cp.async.cg / st.global.cg) so that no stale L1 line is read.  Inside a chunk the
// section's register groups run on the same engine as the single-state blocking kernel.
#include "block_core.cuh"
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

__device__ __forceinline__ int64_t deposit(int64_t v, const int8_t *bits, int nbits) {
    int64_t x = 0;
    for (int k = 0; k < nbits; ++k)
        if ((v >> k) & 1) x |= int64_t(1) << bits[k];
    return x;
}

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void *g) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Last op whose first item is <= item, searching forward from `k` (a CTA's items increase).
__device__ __forceinline__ int find_op(const BatchOp *ops, int nops, int64_t item, int k) {
    if (ops[k].first > item) k = 0;
    int step = 1, hi = k;
    while (hi + step < nops && ops[hi + step].first <= item) {
        hi += step;
        step <<= 1;
    }
    int lo = hi, top = min(nops - 1, hi + step - 1);
    while (lo < top) {
        const int mid = (lo + top + 1) / 2;
        if (ops[mid].first <= item) lo = mid; else top = mid - 1;
    }
    return lo;
}

constexpr int kMaxRuns = 1 << (kBatchMaxChunkBits - 4);  // chunk runs above a low run of >= 4 bits

__device__ __forceinline__ void copy_prog(unsigned char *dst, const unsigned char *src, int bytes) {
    for (int k = threadIdx.x * 16; k < bytes; k += NCB * 16)
        *reinterpret_cast<uint4 *>(dst + k) = *reinterpret_cast<const uint4 *>(src + k);
}  // chunk runs above a low run of >= 4 bits

__global__ void __launch_bounds__(NCB) k_batch(const BatchOp *__restrict__ ops, int nops,
                                               const unsigned char *__restrict__ progs, float2 *const *amps,
                                               int *ops_done, int *chunks_done, unsigned long long *next,
                                               int64_t total, int from_zero, int *err) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *chunk = reinterpret_cast<float2 *>(smem);
    const uint32_t chunk_s = ptx::smem_addr(chunk);
    unsigned char *sprog = smem + (size_t(1) << kBatchMaxChunkBits) * sizeof(float2);
    __shared__ int64_t s_item, s_next;
    __shared__ int s_op, s_cached, s_abort;
    __shared__ BatchOp s_bop;
    __shared__ int64_t s_dep[kMaxRuns];  // state-index bits of each run of the chunk
    if (threadIdx.x == 0) {
        s_cached = -1;
        s_abort = 0;
        s_op = 0;
        s_next = (int64_t)atomicAdd(next, 1ull);
    }
    __syncthreads();
    while (true) {
        if (threadIdx.x == 0) {
            const int64_t item = s_next;
            s_item = item;
            if (item < total) {
                const int k = find_op(ops, nops, item, s_op);
                if (k != s_op || s_cached < 0) s_bop = ops[k];
                s_op = k;
                // take the next index now; its lookup and wait happen after this item
                s_next = (int64_t)atomicAdd(next, 1ull);
                // earlier sections of this state must be complete
                const int st = s_bop.state, need = s_bop.op;
                if (ld_acquire(&ops_done[st]) < need) {
                    const uint64_t t0 = ptx::globaltimer();
                    while (ld_acquire(&ops_done[st]) < need) {
                        if (ptx::globaltimer() - t0 > kWaitLimitNs || *(volatile int *)err) {
                            atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                            s_abort = 1;
                            break;
                        }
                        __nanosleep(200);
                    }
                }
            }
        }
        __syncthreads();
        if (s_item >= total || s_abort) break;
        const BatchOp &op = s_bop;
        const int64_t j = s_item - op.first;
        const int ce = op.ce, low = op.low;
        const bool fresh = s_cached != s_op;
        // run table once per section; a one-piece program stays in shared memory across chunks
        if (fresh) {
            for (int r = threadIdx.x; r < (1 << (ce - low)); r += NCB) s_dep[r] = deposit(r, op.high, op.nhigh);
            if (op.npiece == 1) copy_prog(sprog, progs + op.prog_off, op.prog_bytes);
            __syncthreads();
        }
        float2 *amp = amps[op.state];
        const int64_t obase = deposit(j, op.outer, op.nouter);
        const int lmask = (1 << low) - 1, npairs = 1 << (ce - 1);
        if (from_zero && op.op == 0) {
            // first section of a state started from |0..0>: the chunk holding index 0 is e_0
            for (int f = threadIdx.x; f < npairs; f += NCB)
                *reinterpret_cast<float4 *>(chunk + 2 * f) = make_float4((j == 0 && f == 0) ? 1.f : 0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll 4
            for (int f = threadIdx.x; f < npairs; f += NCB) {
                const int e = 2 * f;
                const int64_t gidx = obase | s_dep[e >> low] | (e & lmask);
                cp_async16(chunk_s + 8u * (uint32_t)e, amp + gidx);
            }
            cp_async_wait_all();
        }
        __syncthreads();
        if (threadIdx.x == 0) s_cached = s_op;
        // register groups, piece by piece: the first group reads the natural layout, the last
        // writes it back natural
        uint32_t poff = op.prog_off;
        for (int pc = 0; pc < op.npiece; ++pc) {
            const int4 hd = *reinterpret_cast<const int4 *>(progs + poff);
            if (op.npiece > 1) {
                copy_prog(sprog, progs + poff, hd.z);
                __syncthreads();
            }
            const uint32_t seg_s = ptx::smem_addr(sprog) + 16u;
            const uint32_t gate_s = seg_s + (uint32_t)((hd.x * sizeof(DevSeg) + 15) & ~size_t(15));
            for (int si = 0; si < hd.x; ++si) {
                run_segment<float, RB, NCB, 1>(chunk_s, seg_s + (uint32_t)(si * sizeof(DevSeg)), gate_s, threadIdx.x,
                                               c_swz64, ce, obase);
                __syncthreads();
            }
            poff += (uint32_t)hd.z;
        }
#pragma unroll 4
        for (int f = threadIdx.x; f < npairs; f += NCB) {
            const int e = 2 * f;
            const int64_t gidx = obase | s_dep[e >> low] | (e & lmask);
            __stcg(reinterpret_cast<float4 *>(amp + gidx), *reinterpret_cast<const float4 *>(chunk + e));
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
                  int *dev_chunks_done, unsigned long long *dev_next, int64_t total, int from_zero, int *dev_err,
                  cudaStream_t st) {
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
                                     from_zero, dev_err);
    check_cuda(cudaGetLastError(), "batch kernel launch");
}

}  // namespace sv
