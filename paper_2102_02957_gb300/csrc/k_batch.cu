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

// Threads per CTA: 256 for SIMT-only batches, 128 (one 128-row tensor-core tile) when sections
// run on the tensor cores.
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


template <int NT>
__device__ __forceinline__ void copy_prog(unsigned char *dst, const unsigned char *src, int bytes, int ctid) {
    for (int k = ctid * 16; k < bytes; k += NT * 16)
        *reinterpret_cast<uint4 *>(dst + k) = *reinterpret_cast<const uint4 *>(src + k);
}

// A CTA holds POOLS independent workers ("pools") of NT threads; each drains the queue on its
// own with its own chunk and program buffers and its own named barrier.  SIMT batches: one pool
// of 256 threads, two CTAs per SM.  Tensor-core batches: pools of 128 threads (one 128-row tile
// each) in one CTA per SM sharing its 512 tensor-memory columns: two pools of two tile buffers
// for chunks of up to 13 bits, or three of one buffer for chunks of up to 12 bits (more
// independent tile chains in flight; the smaller chunk buffers make room for the third).
template <int NT, int POOLS>
__device__ __forceinline__ void pool_sync(int p) {
    if constexpr (POOLS == 1) __syncthreads();
    else ptx::named_bar_sync(1 + p, NT);
}

template <int NT, int POOLS, int NB>
__global__ void __launch_bounds__(NT * POOLS, POOLS >= 2 ? 1 : 2) k_batch(const BatchOp *__restrict__ ops, int nops,
                                                      const unsigned char *__restrict__ progs, float2 *const *amps,
                                                      int *ops_done, int *chunks_done, unsigned long long *next,
                                                      int64_t total, int from_zero, int prog_cap, int *err,
                                                      uint64_t wait_ns, int stall_state) {
    constexpr bool TC = POOLS >= 2;  // the tensor-core configurations
    constexpr int kCapBits = POOLS == 3 ? kBatchTc3ChunkBits : kBatchMaxChunkBits;  // chunk buffer
    constexpr int kMaxRuns = 1 << (kCapBits - 4);  // chunk runs above a low run of >= 4 bits
    extern __shared__ __align__(16) unsigned char smem[];
    const int p = threadIdx.x / NT, ctid = threadIdx.x % NT;
    const size_t pool_bytes = (size_t(1) << kCapBits) * sizeof(float2) + (size_t)prog_cap;
    float2 *chunk = reinterpret_cast<float2 *>(smem + (size_t)p * pool_bytes);
    const uint32_t chunk_s = ptx::smem_addr(chunk);
    unsigned char *sprog = reinterpret_cast<unsigned char *>(chunk) + (size_t(1) << kCapBits) * sizeof(float2);
    __shared__ int64_t s_item[POOLS], s_next[POOLS];
    __shared__ int s_op[POOLS], s_cached[POOLS], s_abort[POOLS];
    __shared__ BatchOp s_bop[POOLS];
    __shared__ int64_t s_dep[POOLS][kMaxRuns];  // state-index bits of each run of the chunk
    __shared__ uint64_t s_mma[POOLS][2];        // tensor-core tile buffers: MMAs complete
    __shared__ uint32_t s_tmem;
    __shared__ int s_tc_abort[POOLS];
    __shared__ uint64_t s_wait_ns;  // the wait bound, read where a wait gives up
    if (threadIdx.x == 0) s_wait_ns = wait_ns;
    if (ctid == 0) {
        s_cached[p] = -1;
        s_abort[p] = 0;
        s_op[p] = 0;
        s_tc_abort[p] = 0;
        if constexpr (TC) {
            ptx::mbar_init(&s_mma[p][0], 1);
            ptx::mbar_init(&s_mma[p][1], 1);
            ptx::fence_mbar_init();
        }
        s_next[p] = (int64_t)atomicAdd(next, 1ull);
    }
    // tensor memory only in the tensor-core configuration (a SIMT batch carries no tcgen05 code)
    if constexpr (TC) {
        if (threadIdx.x < 32) ptx::tmem_alloc(ptx::smem_addr(&s_tmem), 512);
        ptx::tc_fence_before();
    }
    __syncthreads();
    if constexpr (TC) ptx::tc_fence_after();
    static_assert(!TC || POOLS * NB * TcGeom<4>::COLS <= 512, "tile buffers exceed tensor memory");
    const uint32_t tmem_pool = TC ? s_tmem + (uint32_t)(p * NB * TcGeom<4>::COLS) : 0u;
    uint32_t mma_phase[2] = {0, 0};
    BatchOp &op = s_bop[p];
    while (true) {
        if (ctid == 0) {
            const int64_t item = s_next[p];
            s_item[p] = item;
            if (item < total) {
                const int k = find_op(ops, nops, item, s_op[p]);
                if (k != s_op[p] || s_cached[p] < 0) s_bop[p] = ops[k];
                s_op[p] = k;
                // take the next index now; its lookup and wait happen after this item
                s_next[p] = (int64_t)atomicAdd(next, 1ull);
                // earlier sections of this state must be complete
                const int st = s_bop[p].state, need = s_bop[p].op;
                if (ld_acquire(&ops_done[st]) < need) {
                    const int64_t t0 = clock64(), lim = ptx::wait_cycles(wait_ns);
                    while (ld_acquire(&ops_done[st]) < need) {
                        if (clock64() - t0 > lim || *(volatile int *)err) {
                            atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                            s_abort[p] = 1;
                            break;
                        }
                        __nanosleep(200);
                    }
                }
            }
        }
        pool_sync<NT, POOLS>(p);
        if (s_item[p] >= total || s_abort[p]) break;
        const int64_t j = s_item[p] - op.first;
        const int ce = op.ce, low = op.low;
        const bool fresh = s_cached[p] != s_op[p];
        // run table once per section; a one-piece program stays in shared memory across chunks
        if (fresh) {
            for (int r = ctid; r < (1 << (ce - low)); r += NT) s_dep[p][r] = deposit(r, op.high, op.nhigh);
            if (op.npiece == 1) copy_prog<NT>(sprog, progs + op.prog_off, op.prog_bytes, ctid);
            if (op.tc) ptx::fence_proxy_async_smem();  // B operands, read by the tensor cores
            pool_sync<NT, POOLS>(p);
        }
        float2 *amp = amps[op.state];
        const int64_t obase = deposit(j, op.outer, op.nouter);
        const int lmask = (1 << low) - 1, npairs = 1 << (ce - 1);
        if (from_zero && op.op == 0) {
            // first section of a state started from |0..0>: the chunk holding index 0 is e_0
            for (int f = ctid; f < npairs; f += NT)
                *reinterpret_cast<float4 *>(chunk + 2 * f) = make_float4((j == 0 && f == 0) ? 1.f : 0.f, 0.f, 0.f, 0.f);
        } else {
#pragma unroll 4
            for (int f = ctid; f < npairs; f += NT) {
                const int e = 2 * f;
                const int64_t gidx = obase | s_dep[p][e >> low] | (e & lmask);
                cp_async16(chunk_s + 8u * (uint32_t)e, amp + gidx);
            }
            cp_async_wait_all();
        }
        pool_sync<NT, POOLS>(p);
        if (ctid == 0) s_cached[p] = s_op[p];
        // register groups, piece by piece: the first group reads the natural layout, the last
        // writes it back natural
        uint32_t poff = op.prog_off;
        bool tc_failed = false;
        for (int pc = 0; pc < op.npiece && !tc_failed; ++pc) {
            const int4 hd = *reinterpret_cast<const int4 *>(progs + poff);
            if (op.npiece > 1) {
                copy_prog<NT>(sprog, progs + poff, hd.z, ctid);
                if (op.tc) ptx::fence_proxy_async_smem();
                pool_sync<NT, POOLS>(p);
            }
            const uint32_t seg_s = ptx::smem_addr(sprog) + 16u;
            const uint32_t body_s = seg_s + (uint32_t)((hd.x * sizeof(DevSeg) + 15) & ~size_t(15));
            for (int si = 0; si < hd.x; ++si) {
                if (op.tc) {
                    // fused group on the tensor cores, unbiased per row (the batch has no
                    // per-circuit norm restoration); the return value is uniform over the pool
                    if constexpr (TC) {
                        if (!run_segment_tc<4, NT, true, NB>(chunk_s, seg_s + (uint32_t)(si * sizeof(DevSeg)),
                                                      body_s + (uint32_t)(si * kBatchTcGroupBytes), ctid, c_swz64, ce,
                                                      tmem_pool, 1 + p, s_mma[p], mma_phase, &s_tc_abort[p],
                                                      &s_wait_ns)) {
                            tc_failed = true;
                            break;
                        }
                    }
                } else {
                    run_segment<float, RB, NT, 1>(chunk_s, seg_s + (uint32_t)(si * sizeof(DevSeg)), body_s, ctid,
                                                  c_swz64, ce, obase);
                }
                pool_sync<NT, POOLS>(p);
            }
            poff += (uint32_t)hd.z;
        }
        if (tc_failed) {
            if (ctid == 0) atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
            break;
        }
#pragma unroll 4
        for (int f = ctid; f < npairs; f += NT) {
            const int e = 2 * f;
            const int64_t gidx = obase | s_dep[p][e >> low] | (e & lmask);
            __stcg(reinterpret_cast<float4 *>(amp + gidx), *reinterpret_cast<const float4 *>(chunk + e));
        }
        __threadfence();
        pool_sync<NT, POOLS>(p);
        if (ctid == 0) {
            if (atomicAdd(&chunks_done[s_op[p]], 1) == op.nchunks - 1) {
                __threadfence();
                // section complete: release the state's next one (except the stall test's section)
                if (!(op.state == stall_state && op.op == 0)) atomicAdd(&ops_done[op.state], 1);
            }
        }
    }
    // both pools are done with tensor memory before the allocating warp frees it
    if constexpr (TC) {
        ptx::tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) {
            ptx::tc_fence_after();
            ptx::tmem_dealloc(s_tmem, 512);
        }
    }
}

}  // namespace

void launch_batch(const void *dev_ops, int nops, const void *dev_progs, void *const *dev_amps, int *dev_ops_done,
                  int *dev_chunks_done, unsigned long long *dev_next, int64_t total, int from_zero, int use_tc,
                  int *dev_err, cudaStream_t st, uint64_t wait_ns, int stall_state) {
    const int prog_cap = use_tc == 2 ? kBatchMaxProgBytesTc3 : use_tc ? kBatchMaxProgBytesTc : kBatchMaxProgBytes;
    const int pools = use_tc == 2 ? 3 : use_tc ? 2 : 1, nt = use_tc ? 128 : 256;
    const int cap_bits = use_tc == 2 ? kBatchTc3ChunkBits : kBatchMaxChunkBits;
    const size_t smem = (size_t)pools * ((size_t(1) << cap_bits) * sizeof(float2) + (size_t)prog_cap);
    auto kern = use_tc == 2 ? k_batch<128, 3, 1> : use_tc ? k_batch<128, 2, 2> : k_batch<256, 1, 1>;
    check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
               "cudaFuncSetAttribute(batch)");
    int per_sm = 0;
    check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, nt * pools, smem), "occupancy(batch)");
    if (per_sm < 1) per_sm = 1;
    // a tensor-core CTA takes all 512 tensor-memory columns of its SM (its shared memory
    // already keeps a second CTA off)
    if (use_tc && per_sm > 1) fail(SV_ERR_UNSUPPORTED, "batch kernel occupancy exceeds tensor memory");
    // every CTA resident at once: a waiting pool only ever waits for items already taken
    const int grid = num_sms() * per_sm;
    kern<<<grid, nt * pools, smem, st>>>((const BatchOp *)dev_ops, nops, (const unsigned char *)dev_progs,
                                         (float2 *const *)dev_amps, dev_ops_done, dev_chunks_done, dev_next, total,
                                         from_zero, prog_cap, dev_err, wait_ns, stall_state);
    check_cuda(cudaGetLastError(), "batch kernel launch");
}

}  // namespace sv
