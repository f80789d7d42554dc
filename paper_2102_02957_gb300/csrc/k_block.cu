// Blocking section: one HBM sweep applies every gate of the section to every chunk
// (Sec. IV.C, Listing 4: for all chunks, fetch the chunk, apply each gate of the section, write
// it back).  On one GPU the chunk of 2^c amplitudes is the unit staged from HBM into shared
// memory: either the contiguous chunk j (physical bits 0..c-1 after the paper's chunk_swap
// rounds) or a gathered chunk (any c bits including the low pinned ones, fetched in place by
// rank <= 5 tensor copies).  The transpiler (Sec. IV.A) guarantees that every gate of the section
// acts on chunk bits only -- except diagonal gates planned with diag_outside, whose outside bits
// are read off the chunk's origin index.
//
// Kernel organisation (persistent, warp-specialised):
//  * warp 0 is the producer (produce_chunks): it streams the CTA's chunks
//    j = blockIdx.x + t*gridDim.x into a ring of shared-memory buffers with bulk or tensor
//    asynchronous copies (TMA engine) completing on "full" mbarriers, each lane issuing its own
//    boxes of a gathered chunk (lane 0 does the mbarrier bookkeeping);
//  * G consumer groups of NC threads (two; four for tensor-core sections of chunks up to 12 bits)
//    take chunks in turn, so one group's shared-memory and barrier phases overlap another's
//    arithmetic.  For each chunk a group runs the section's
//    register groups -- SIMT (run_segment: each thread loads the 2^R amplitudes spanned by the
//    group's R chunk bits into registers, applies every gate of the group there, stores them
//    back) or tensor cores (run_segment_tc: the group's fused unitary applied to 128-row tiles
//    with tcgen05 MMAs) -- then hand it to the store warp through a "done" mbarrier;
//  * warp 1 is the store warp (store_chunks): it writes the chunks back in order, a box or piece
//    per lane, and releases each buffer to the producer through an "empty" mbarrier once the
//    copies have read it.
//
// Shared-memory layout of a chunk while it is being worked on: amplitude i sits in slot
// i ^ F(i), where F XORs a fixed non-zero pattern V[k] into the low slot bits for every set
// bit k >= SB of i (SB = log2 of the amplitudes per 128-byte row).  The copies move the natural
// layout, so the first group reads and the last group writes unswizzled slots.  For every group
// the host picks which chunk bits the lanes of a half-warp (quarter-warp for complex128)
// enumerate so that their slots fall in distinct banks.
//
// Every wait is bounded (SM clock cycles); on expiry the kernel records DEV_ERR_TIMEOUT in the
// error word and stops.
#include <cuda.h>

#include <cstdlib>
#include <cstring>
#include <mutex>

#include "block_core.cuh"
#include "ptx.cuh"
#include "sv_internal.h"

namespace sv {
namespace {

// Amplitude index of the first element of copy t of gathered chunk j.
__device__ __forceinline__ int64_t gather_origin(const GatherArgs &ga, int64_t j, int t) {
    int64_t x = 0;
    for (int k = 0; k < ga.nouter; ++k)
        if ((j >> k) & 1) x |= int64_t(1) << ga.outer[k];
    for (int k = 0; k < ga.nloop; ++k)
        if ((t >> k) & 1) x |= int64_t(1) << ga.loop[k];
    return x;
}

// Chunk data moves with the TMA engine: one producer thread (tensor copies of the gathered layout,
// or 16 KiB bulk copies of a contiguous chunk) and one store thread.
constexpr int kSvcThreads = 64;
constexpr int kPiece = 16384;  // bytes per bulk copy instruction

// Tensor coordinates of the box that holds amplitude index x (box bits of x are zero).
template <typename T2>
__device__ __forceinline__ void gather_coords(const GatherArgs &ga, int64_t x, int *coord) {
    for (int d = 0; d < ga.rank; ++d) {
        const int w = ga.s[d + 1] - ga.s[d];
        int64_t v = (x >> ga.s[d]) & ((int64_t(1) << w) - 1);
        if (d == 0 && sizeof(T2) == 16) v *= 2;  // complex128: two doubles per amplitude
        coord[d] = (int)v;
    }
    for (int d = ga.rank; d < 5; ++d) coord[d] = 0;
}

// Producer (one warp): stream this CTA's chunks j = blockIdx.x + it * gridDim.x into the ring
// of nbuf shared-memory buffers (bulk copies for contiguous chunks, tensor copies for gathered
// ones), each completing on full[slot]; a slot is reused once the store warp released it on
// empty[slot].  A gathered chunk with more runs of bits than a tensor map has dimensions takes
// several boxes; each lane issues its own, since one thread issuing them in sequence waits on
// every box in turn.
template <typename T2>
__device__ __forceinline__ void produce_chunks(T2 *state, int c, int64_t count, int nbuf, T2 *bufs, uint64_t *full,
                                               uint64_t *empty, volatile int *abort_flag, int *err,
                                               const GatherArgs &ga, const CUtensorMap *tmap, uint64_t wait_ns) {
    const int lane = threadIdx.x & 31;
    const int chunk_amps = 1 << c;
    const uint32_t chunk_bytes = (uint32_t)chunk_amps * (uint32_t)sizeof(T2);
    int64_t issued = 0;
    for (int64_t it = 0; it < count; ++it) {
        const int s = (int)(it % nbuf);
        bool ok = true;
        if (it >= nbuf) ok = ptx::mbar_wait(&empty[s], (uint32_t)((it / nbuf - 1) & 1), wait_ns) && !*abort_flag;
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            break;
        }
        const int64_t j = blockIdx.x + it * gridDim.x;
        unsigned char *dst = reinterpret_cast<unsigned char *>(bufs + (size_t)s * chunk_amps);
        if (lane == 0) ptx::mbar_arrive_expect_tx(&full[s], chunk_bytes);
        __syncwarp();
        if (ga.rank > 0) {
            for (int t = lane; t < (1 << ga.nloop); t += 32) {
                int coord[5];
                gather_coords<T2>(ga, gather_origin(ga, j, t), coord);
                ptx::tensor_g2s(dst + (size_t)t * ga.box_amps * sizeof(T2), tmap, coord, ga.rank, &full[s]);
            }
        } else {
            const unsigned char *src = reinterpret_cast<const unsigned char *>(state + j * chunk_amps);
            for (uint32_t o = (uint32_t)lane * kPiece; o < chunk_bytes; o += 32u * kPiece) {
                const uint32_t b = chunk_bytes - o < (uint32_t)kPiece ? chunk_bytes - o : (uint32_t)kPiece;
                ptx::bulk_g2s(dst + o, src + o, b, &full[s]);
            }
        }
        ++issued;
    }
    // do not leave while copies into this CTA's shared memory are still in flight
    for (int64_t it = issued > nbuf ? issued - nbuf : 0; it < issued; ++it)
        (void)ptx::mbar_wait(&full[it % nbuf], (uint32_t)((it / nbuf) & 1), wait_ns);
}

// Issue the copies that write chunk j back from shared memory (lane `lane` of the store warp
// takes every 32nd box or piece).
template <typename T2>
__device__ __forceinline__ void write_chunk(T2 *state, int c, int64_t j, const T2 *buf, const GatherArgs &ga,
                                            const CUtensorMap *tmap, int lane) {
    const int chunk_amps = 1 << c;
    const uint32_t chunk_bytes = (uint32_t)chunk_amps * (uint32_t)sizeof(T2);
    const unsigned char *srcs = reinterpret_cast<const unsigned char *>(buf);
    if (ga.rank > 0) {
        for (int t = lane; t < (1 << ga.nloop); t += 32) {
            int coord[5];
            gather_coords<T2>(ga, gather_origin(ga, j, t), coord);
            ptx::tensor_s2g(tmap, coord, ga.rank, srcs + (size_t)t * ga.box_amps * sizeof(T2));
        }
    } else {
        unsigned char *dstg = reinterpret_cast<unsigned char *>(state + j * chunk_amps);
        for (uint32_t o = (uint32_t)lane * kPiece; o < chunk_bytes; o += 32u * kPiece) {
            const uint32_t b = chunk_bytes - o < (uint32_t)kPiece ? chunk_bytes - o : (uint32_t)kPiece;
            ptx::bulk_s2g(dstg + o, srcs + o, b);
        }
    }
}

// Store warp: write the CTA's chunks back in order as their consumers finish them (done[slot])
// and release each slot to the producer (empty[slot]) as soon as the copies have read it.
// (Keeping two write-backs in flight, releasing chunk it - 1 after chunk it's copies are issued,
// was measured slower: the slot is held longer and the prefetch depth shrinks.)
template <typename T2>
__device__ __forceinline__ void store_chunks(T2 *state, int c, int64_t count, int nbuf, const T2 *bufs, uint64_t *done,
                                             uint64_t *empty, volatile int *abort_flag, int *err,
                                             const GatherArgs &ga, const CUtensorMap *tmap, uint64_t wait_ns) {
    const int lane = threadIdx.x & 31;
    const int chunk_amps = 1 << c;
    for (int64_t it = 0; it < count; ++it) {
        const int s = (int)(it % nbuf);
        // use it / nbuf of done[s]: the previous use (chunk it - nbuf) was waited for here
        const bool ok = ptx::mbar_wait(&done[s], (uint32_t)((it / nbuf) & 1), wait_ns) && !*abort_flag;
        if (__any_sync(0xFFFFFFFFu, !ok)) {
            if (lane == 0) {
                atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
                *abort_flag = 1;
            }
            break;
        }
        write_chunk<T2>(state, c, blockIdx.x + it * gridDim.x, bufs + (size_t)s * chunk_amps, ga, tmap, lane);
        ptx::bulk_commit();
        ptx::bulk_wait_read<0>();
        __syncwarp();
        if (lane == 0) ptx::mbar_arrive(&empty[s]);
    }
    ptx::bulk_wait<0>();
}

constexpr int CG2 = 2;  // consumer groups per CTA (default)

// G consumer groups per CTA; tensor-core groups keep NB tile buffers each
// (G * NB * TcGeom<R>::COLS <= 512 TMEM columns).
template <typename T, int R, int NC, int KU, bool TC, int G, int NB>
__device__ __forceinline__ void block_body(typename V2<T>::type *__restrict__ state, int c, int64_t nchunks, int nbuf,
                                           const unsigned char *__restrict__ prog, int nseg, int ngate, int *err,
                                           const CUtensorMap &tmap, const GatherArgs &ga_in, uint64_t wait_ns) {
    using T2 = typename V2<T>::type;
    __shared__ GatherArgs ga;  // gathered chunks (rank > 0); rank 0 = contiguous chunk j
    if (threadIdx.x == 0) ga = ga_in;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int chunk_amps = 1 << c;
    const uint32_t chunk_bytes = (uint32_t)chunk_amps * (uint32_t)sizeof(T2);
    T2 *bufs = reinterpret_cast<T2 *>(smem);
    // block program copied into shared memory: register groups, then gate records (SIMT) or the
    // groups' B operands (tensor cores), 16-byte aligned
    const int seg_bytes = (int)((nseg * sizeof(DevSeg) + 15) & ~size_t(15));
    constexpr int kBBytes = TcGeom<(R < 3 ? 3 : R)>::B_BYTES;  // B operand of one tensor-core group
    const int prog_bytes = seg_bytes + (TC ? nseg * kBBytes : ngate * (int)sizeof(DevGate<T>));
    unsigned char *sprog = smem + (size_t)nbuf * chunk_bytes;
    const DevSeg *segs = reinterpret_cast<const DevSeg *>(sprog);
    const DevGate<T> *gates = reinterpret_cast<const DevGate<T> *>(sprog + seg_bytes);
    uint64_t *full = reinterpret_cast<uint64_t *>(sprog + ((prog_bytes + 15) & ~15));
    uint64_t *empty = full + nbuf;
    uint64_t *done = empty + nbuf;
    uint64_t *mma_bar = done + nbuf;  // two per consumer group (tensor-core path)
    volatile int *abort_flag = reinterpret_cast<volatile int *>(mma_bar + 2 * G);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_bar + 2 * G) + 1;
    __shared__ int swz[24];
    // the wait bound lives in shared memory: waits are rare, a register for it in every thread is not
    __shared__ uint64_t s_wait_ns;
    constexpr uint32_t kTmemCols = 512;  // G consumer groups x NB tile buffers x TcGeom<R>::COLS

    for (int k = threadIdx.x * 16; k < prog_bytes; k += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(sprog + k) = *reinterpret_cast<const uint4 *>(prog + k);
    if (threadIdx.x < 24) swz[threadIdx.x] = sizeof(T2) == 8 ? c_swz64[threadIdx.x] : c_swz128[threadIdx.x];
    if (threadIdx.x == 0) {
        s_wait_ns = wait_ns;
        for (int s = 0; s < nbuf; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], 1);
            ptx::mbar_init(&done[s], 1);
        }
        for (int g = 0; g < 2 * G; ++g) ptx::mbar_init(&mma_bar[g], 1);
        *abort_flag = 0;
        ptx::fence_mbar_init();
    }
    constexpr int kTmemWarp = kSvcThreads / 32;  // the first consumer warp allocates tensor memory
    if (TC && (threadIdx.x >> 5) == kTmemWarp) ptx::tmem_alloc(ptx::smem_addr(tmem_slot), kTmemCols);
    if (TC) {
        ptx::fence_proxy_async_smem();  // B operands written by generic stores, read by the tensor cores
        ptx::tc_fence_before();
    }
    __syncthreads();
    if (TC) ptx::tc_fence_after();
    const uint32_t tmem_base = TC ? *tmem_slot : 0u;

    const int64_t count = blockIdx.x < nchunks ? (nchunks - 1 - blockIdx.x) / gridDim.x + 1 : 0;

    if (threadIdx.x < kSvcThreads) {
        // ------------------------------------------------- producer (warp 0), store (warp 1)
        if (threadIdx.x < 32)
            produce_chunks<T2>(state, c, count, nbuf, bufs, full, empty, abort_flag, err, ga, &tmap, wait_ns);
        else
            store_chunks<T2>(state, c, count, nbuf, bufs, done, empty, abort_flag, err, ga, &tmap, wait_ns);
        return;
    }

    // -------------------------------------------------------------- consumers
    // G consumer groups of NC threads take alternate chunks, so one group's shared-memory phases
    // overlap another group's arithmetic; each group synchronises on its own named barrier.
    // (Two groups sharing a chunk, each with half of its tiles, was measured slower: the shared
    // barriers between register groups cost more than the deeper prefetch gained.)
    const int cg = (threadIdx.x - kSvcThreads) / NC;
    const int ctid = (threadIdx.x - kSvcThreads) % NC;
    const int bar_id = 1 + cg;
    uint32_t mma_phase[2] = {0, 0};
    // A parity wait cannot tell this chunk's load (use u = it / nbuf of slot s) from the slot's
    // previous, still incomplete one (another group's chunk it - nbuf).  So a group first waits
    // for that previous chunk's write-back (empty[s], use u - 1), which follows its load: then
    // full[s] is at use u.  That wait is itself unambiguous: use u - 2 of empty[s] was observed
    // by the producer before it issued this group's previous chunk.  The argument needs every
    // group's previous chunk to be at most nbuf back, so at most nbuf groups take chunks.
    const int geff = G < nbuf ? G : nbuf;
    for (int64_t it = cg; cg < geff && it < count; it += geff) {
        const int s = (int)(it % nbuf);
        const int64_t u = it / nbuf;
        const int64_t j = blockIdx.x + it * gridDim.x;
        const uint64_t *wl = &s_wait_ns;
        const bool bad = (u > 0 && !ptx::mbar_wait(&empty[s], (uint32_t)((u - 1) & 1), *(volatile const uint64_t *)wl)) ||
                         !ptx::mbar_wait(&full[s], (uint32_t)(u & 1), *(volatile const uint64_t *)wl);
        if (bad) {
            atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
            *abort_flag = 1;
        }
        // every thread of the group leaves together (the flag is read before the barrier)
        if (ptx::named_bar_or(bar_id, NC, bad || *abort_flag)) break;
        T2 *buf = bufs + (size_t)s * chunk_amps;
        // state index of the chunk's first amplitude (its bits outside the chunk are the chunk's)
        const int64_t origin = ga.rank > 0 ? gather_origin(ga, j, 0) : j << c;
        bool failed = false;
        for (int si = 0; si < nseg; ++si) {
            const uint32_t seg_addr = ptx::smem_addr(segs) + (uint32_t)(si * sizeof(DevSeg));
            [[maybe_unused]] bool ok = true;
            if constexpr (TC) {
                ok = run_segment_tc<R, NC, false, NB>(ptx::smem_addr(buf), seg_addr,
                                                      ptx::smem_addr(sprog + seg_bytes) + (uint32_t)(si * kBBytes), ctid,
                                                      swz, c, tmem_base + (uint32_t)(cg * NB * TcGeom<R>::COLS), bar_id,
                                                      &mma_bar[2 * cg], mma_phase, abort_flag, &s_wait_ns);
            } else {
                run_segment<T, R, NC, KU>(ptx::smem_addr(buf), seg_addr, ptx::smem_addr(gates), ctid, swz, c, origin);
            }
            if (si == nseg - 1) ptx::fence_proxy_async_smem();  // the store copies read the chunk
            if constexpr (TC) {
                if (ptx::named_bar_or(bar_id, NC, !ok)) {  // a group leaves together
                    failed = true;
                    break;
                }
            } else {
                ptx::named_bar_sync(bar_id, NC);  // SIMT groups have no waits that can fail
            }
        }
        if (failed) {
            atomicCAS(err, DEV_OK, DEV_ERR_TIMEOUT);
            break;
        }
        if (nseg == 0) ptx::fence_proxy_async_smem();
        // hand the chunk to the store thread (the group's last barrier ordered all its writes)
        if (ctid == 0) ptx::mbar_arrive(&done[s]);
    }
    if constexpr (TC) {
        // every consumer is done with tensor memory before the allocating warp frees it
        ptx::tc_fence_before();
        ptx::named_bar_sync(1 + G, G * NC);
        if ((threadIdx.x >> 5) == kTmemWarp) {
            ptx::tc_fence_after();
            ptx::tmem_dealloc(tmem_base, kTmemCols);
        }
    }
}

// SIMT sections: launch bounds let the compiler fit two 256-thread consumer groups.
template <typename T, int R, int NC, int KU, bool TC, int G = CG2, int NB = 2>
__global__ void __launch_bounds__(G * NC + kSvcThreads, 1)
    k_block(typename V2<T>::type *__restrict__ state, int c, int64_t nchunks, int nbuf,
            const unsigned char *__restrict__ prog, int nseg, int ngate, int *err,
            const __grid_constant__ CUtensorMap tmap, const GatherArgs ga_in, uint64_t wait_ns) {
    block_body<T, R, NC, KU, TC, G, NB>(state, c, nchunks, nbuf, prog, nseg, ngate, err, tmap, ga_in, wait_ns);
}

// Tensor-core sections: one CTA per SM (it takes all of the SM's tensor memory).  The register
// file is split over the SM's four sub-partitions (16384 registers each) and a CTA's warps are
// spread over them in turn, so a thread may use 16384 / (32 * ceil(warps / 4)) registers
// (rounded down to a multiple of 8).
constexpr int tc_max_regs(int threads) {
    return (16384 / (32 * (((threads + 31) / 32 + 3) / 4))) / 8 * 8 > 248
               ? 248
               : (16384 / (32 * (((threads + 31) / 32 + 3) / 4))) / 8 * 8;
}
static_assert(tc_max_regs(576) == 96 && tc_max_regs(320) == 168, "register budget per thread");

template <typename T, int R, int NC, int KU, bool TC, int G, int NB>
__global__ void __maxnreg__(tc_max_regs(G * NC + kSvcThreads))
    k_block_tc(typename V2<T>::type *__restrict__ state, int c, int64_t nchunks, int nbuf,
               const unsigned char *__restrict__ prog, int nseg, int ngate, int *err,
               const __grid_constant__ CUtensorMap tmap, const GatherArgs ga_in, uint64_t wait_ns) {
    block_body<T, R, NC, KU, TC, G, NB>(state, c, nchunks, nbuf, prog, nseg, ngate, err, tmap, ga_in, wait_ns);
}

template <typename T, int R, int NC, int KU, bool TC = false, int G = CG2, int NB = 2>
void launch_typed(void *state, int n, int ce, const void *prog, int nseg, int ngate, int *err, cudaStream_t st,
                  const CUtensorMap &tmap, const GatherArgs &ga, uint64_t wait_ns) {
    if (ce - R - 5 > kMaxRest) fail(SV_ERR_UNSUPPORTED, "chunk too wide for the register-group layout");
    using T2 = typename V2<T>::type;
    const size_t chunk_bytes = (size_t(1) << ce) * sizeof(T2);
    const int64_t nchunks = int64_t(1) << (n - ce);
    const size_t seg_bytes = (nseg * sizeof(DevSeg) + 15) & ~size_t(15);
    const size_t prog_bytes =
        (seg_bytes + (TC ? (size_t)nseg * TcGeom<(R < 3 ? 3 : R)>::B_BYTES : ngate * sizeof(DevGate<T>)) + 15) &
        ~size_t(15);
    if (TC && G * NB * TcGeom<(R < 3 ? 3 : R)>::COLS > 512) fail(SV_ERR_UNSUPPORTED, "tile buffers exceed tensor memory");
    int nbuf = TC ? G + 2 : 3;  // tensor cores: every consumer group holds a chunk, plus prefetch
    // program + mbarriers (full, empty, done per buffer; two per consumer group), abort flag,
    // TMEM address
    const size_t extra = prog_bytes + (size_t)(3 * nbuf + 2 * G) * 8 + 16;
    const size_t max_smem = 227 * 1024 - 1024;  // minus the static swizzle table (1 KiB aligned)
    while (nbuf > 1 && nbuf * chunk_bytes + extra > max_smem) --nbuf;
    size_t smem = nbuf * chunk_bytes + extra;
    if (smem > max_smem) fail(SV_ERR_UNSUPPORTED, "chunk and section program do not fit in shared memory");
    // a tensor-core CTA takes all of its SM's tensor memory: reserve over half the shared memory
    // so that the scheduler never places two on one SM
    if (TC && smem < 120 * 1024) smem = 120 * 1024;
    auto grid_of = [&](auto kern) -> unsigned {
        check_cuda(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(block)");
        int per_sm = 0;
        check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, G * NC + kSvcThreads, smem),
                   "occupancy(block)");
        if (per_sm < 1) per_sm = 1;
        if (TC) per_sm = 1;  // each CTA allocates all 512 tensor-memory columns of its SM
        return (unsigned)std::min<int64_t>(nchunks, (int64_t)num_sms() * per_sm);
    };
    if constexpr (TC) {
        auto kern = k_block_tc<T, R, NC, KU, TC, G, NB>;
        kern<<<grid_of(kern), G * NC + kSvcThreads, smem, st>>>((T2 *)state, ce, nchunks, nbuf, (const unsigned char *)prog, nseg,
                                                     ngate, err, tmap, ga, wait_ns);
    } else {
        auto kern = k_block<T, R, NC, KU, TC, G, NB>;
        kern<<<grid_of(kern), G * NC + kSvcThreads, smem, st>>>((T2 *)state, ce, nchunks, nbuf, (const unsigned char *)prog, nseg,
                                                     ngate, err, tmap, ga, wait_ns);
    }
    check_cuda(cudaGetLastError(), "block kernel launch");
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        check_cuda(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q),
                   "cudaGetDriverEntryPointByVersion(cuTensorMapEncodeTiled)");
        if (q != cudaDriverEntryPointSuccess || !p) fail(SV_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
        fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// Tensor map of the whole state viewed with the gathered layout's dimensions: dimension d
// covers index bits [s[d], s[d+1]), its box the chunk run at its bottom.
CUtensorMap make_gather_map(void *state, const GatherLayout &lay, int elem_bytes) {
    const GatherArgs &ga = lay.args;
    cuuint64_t dims[5], strides[4];
    cuuint32_t box[5], estr[5];
    const int dup = elem_bytes == 16 ? 2 : 1;  // complex128 as two doubles
    for (int d = 0; d < ga.rank; ++d) {
        dims[d] = (cuuint64_t(1) << (ga.s[d + 1] - ga.s[d])) * (d == 0 ? dup : 1);
        box[d] = (cuuint32_t(1) << lay.box_len[d]) * (d == 0 ? dup : 1);
        estr[d] = 1;
        if (d > 0) strides[d - 1] = (cuuint64_t(1) << ga.s[d]) * (cuuint64_t)elem_bytes;
    }
    CUtensorMap m;
    const CUresult r = encode_tiled()(&m, elem_bytes == 16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_INT64,
                                      (cuuint32_t)ga.rank, state, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) fail(SV_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return m;
}

}  // namespace

size_t devgate_bytes(int dtype) { return dtype == SV_C64 ? sizeof(DevGate<float>) : sizeof(DevGate<double>); }

// Threads per consumer group: 2^4-amplitude groups need ~96 registers (2 x 256 threads fit the
// register file), 2^5-amplitude and complex128 groups ~170 (2 x 128 threads).
// Threads per consumer group: complex64 with 2^4-amplitude register groups runs 2 x 256
// consumers (17 warps, <= 96 registers a thread); 2^5-amplitude groups and complex128 run
// 2 x 128 (9 warps, <= 168 registers).  Each thread holds one register group at a time.
int block_threads(int ce, int seg_bits, int dtype) {
    (void)ce;
    return (dtype == SV_C64 && seg_bits == 4) ? 256 : 128;
}

static void dispatch(int dtype, int r, int nc, void *state, int n, int ce, const void *prog, int nseg, int ngates,
                     int *err, cudaStream_t st, const CUtensorMap &m, const GatherArgs &ga, uint64_t wait_ns) {
    (void)nc;
    if (dtype == SV_C64) {
        if (r == 4) launch_typed<float, 4, 256, 1>(state, n, ce, prog, nseg, ngates, err, st, m, ga, wait_ns);
        else launch_typed<float, 5, 128, 1>(state, n, ce, prog, nseg, ngates, err, st, m, ga, wait_ns);
    } else {
        launch_typed<double, 4, 128, 1>(state, n, ce, prog, nseg, ngates, err, st, m, ga, wait_ns);
    }
}

void launch_block(int dtype, void *state, int n, int c, const void *dev_prog, int nseg, int ngates, int *dev_err,
                  int seg_bits, cudaStream_t st, uint64_t wait_ns) {
    const int ce = c < n ? c : n;
    if (ce < 4) fail(SV_ERR_UNSUPPORTED, "blocked path needs a chunk of at least 4 bits");
    const int r = seg_bits < ce ? seg_bits : ce;  // the register groups were built with this width
    GatherArgs ga{};  // rank 0: contiguous chunk j
    CUtensorMap none;
    std::memset(&none, 0, sizeof(none));
    dispatch(dtype, r, block_threads(ce, r, dtype), state, n, ce, dev_prog, nseg, ngates, dev_err, st, none, ga,
             wait_ns);
}

void launch_block_gather(int dtype, void *state, int n, const GatherLayout &lay, const void *dev_prog, int nseg,
                         int ngates, int *dev_err, int seg_bits, cudaStream_t st, uint64_t wait_ns) {
    const int ce = lay.ce;
    if (ce < 4) fail(SV_ERR_UNSUPPORTED, "blocked path needs a chunk of at least 4 bits");
    if (reinterpret_cast<uintptr_t>(state) % 16) fail(SV_ERR_ARG, "state buffer not 16-byte aligned");
    const int elem = dtype == SV_C64 ? 8 : 16;
    // every tensor copy lands on a 128-byte boundary of the chunk buffer
    if ((size_t)lay.args.box_amps * elem < 128)
        fail(SV_ERR_UNSUPPORTED, "gathered chunk boxes smaller than 128 bytes (pin more low bits)");
    const CUtensorMap m = make_gather_map(state, lay, elem);
    const int r = seg_bits < ce ? seg_bits : ce;
    dispatch(dtype, r, block_threads(ce, r, dtype), state, n, ce, dev_prog, nseg, ngates, dev_err, st, m, lay.args,
             wait_ns);
}

}  // namespace sv

namespace sv {

void launch_block_tc(void *state, int n, int c, const GatherLayout *lay, const void *dev_prog, int nseg, int *dev_err,
                     int seg_bits, cudaStream_t st, uint64_t wait_ns) {
    const int ce = lay ? lay->ce : (c < n ? c : n);
    if (seg_bits < 3 || seg_bits > 5) fail(SV_ERR_UNSUPPORTED, "tensor-core register groups have 3, 4 or 5 bits");
    if (ce < seg_bits + 7) fail(SV_ERR_UNSUPPORTED, "tensor-core sections need chunks of at least 2^(r+7) amplitudes");
    GatherArgs ga{};  // rank 0: contiguous chunk j
    CUtensorMap m;
    std::memset(&m, 0, sizeof(m));
    if (lay) {
        if ((size_t)lay->args.box_amps * 8 < 128)
            fail(SV_ERR_UNSUPPORTED, "gathered chunk boxes smaller than 128 bytes (pin more low bits)");
        m = make_gather_map(state, *lay, 8);
        ga = lay->args;
    }
    // tile buffers in the SM's 512 TMEM columns (TcGeom<R>::COLS each): four consumer groups with
    // one buffer each where the chunks are small, two with two buffers otherwise; 5-bit groups
    // (256 columns a buffer) run two groups with one buffer
    if (seg_bits == 3)
        launch_typed<float, 3, 128, 1, true, 4, 2>(state, n, ce, dev_prog, nseg, 0, dev_err, st, m, ga, wait_ns);
    else if (seg_bits == 5)
        launch_typed<float, 5, 128, 1, true, 2, 1>(state, n, ce, dev_prog, nseg, 0, dev_err, st, m, ga, wait_ns);
    else if (ce <= 12)
        launch_typed<float, 4, 128, 1, true, 4, 1>(state, n, ce, dev_prog, nseg, 0, dev_err, st, m, ga, wait_ns);
    else
        launch_typed<float, 4, 128, 1, true, 2, 2>(state, n, ce, dev_prog, nseg, 0, dev_err, st, m, ga, wait_ns);
}

}  // namespace sv
