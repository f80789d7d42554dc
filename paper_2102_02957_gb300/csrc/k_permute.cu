// chunk_swap round as one in-place HBM pass (Sec. IV.C, Fig. 10).
//
// A round is a set of disjoint bit transpositions (p_j, q_j).  The index permutation P it
// induces is an involution, and the pass sets a'[i] = a[P(i)] in place.  On one GPU the
// paper's exchange of chunk halves between memory spaces (case (a): p < nc <= q) and of whole
// chunks (case (b): both >= nc, output reordering) are the same data movement: amplitudes
// trade places inside HBM.
//
// Layout of the pass: the index bits are split into a tile part V and an outer part.  V holds
// the low L0 bits (a 128-byte line: 16 complex64 or 8 complex128) plus the partner q_j of every
// pair whose p_j is one of those low bits, so V is closed under P.  Pairs with p_j >= L0 act
// only on the outer part.  For an outer index o with partner o' = P_high(o), the CTA loads both
// tiles (whole 128-byte lines, 16-byte vector accesses), and writes tile o' from tile o and
// tile o from tile o' with the tile bits permuted through shared memory.  Outer indices with
// o' < o are done by their partner; tiles that P leaves fixed are not touched.
#include "sv_internal.h"

namespace sv {
namespace {

constexpr int kThreads = 256;
constexpr int kUnitsPerCta = 512;   // 16-byte units per side and batch staged in shared memory
constexpr int kMaxItems = 128;      // outer items per batch (tiles are at least 8 units)

struct PermArgs {
    int vbits;        // |V|
    int L0;           // contiguous low bits in V
    int nextra;       // |V| - L0
    int nlow, nhigh;
    int64_t nitems;   // 2^(n - |V|)
    int ib;           // outer items per CTA batch
    int vpos[16];     // V bits: 0 .. L0-1 then the extras ascending (physical positions)
    int vsorted[16];  // the same bits in ascending order
    int lp[16], lq[16];  // low pairs in V coordinates
    int hp[32], hq[32];  // high pairs (physical positions)
};

__device__ __forceinline__ int64_t insert0(int64_t x, int p) {
    const int64_t low = x & ((int64_t(1) << p) - 1);
    return ((x >> p) << (p + 1)) | low;
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Byte offset of tile unit ut (its first amplitude v0 = ut * apu in V coordinates) from the tile
// base: the low bits stay, the extra V bits are deposited at their physical positions.
__device__ __forceinline__ int64_t unit_offset(const PermArgs &P, int v0) {
    int64_t off = v0 & ((1 << P.L0) - 1);
    for (int j = 0; j < P.nextra; ++j) off |= int64_t((v0 >> (P.L0 + j)) & 1) << P.vpos[P.L0 + j];
    return off;
}

// Batches b = blockIdx.x, + gridDim.x, ... in two shared-memory buffers: while batch b is
// permuted and written back from one buffer, batch b + gridDim.x is already in flight into the
// other (cp.async), so loads and stores overlap.  The grid is 32 times the resident CTAs:
// batches differ in work (pairs whose partner comes first are skipped), and many short-lived
// CTAs keep the SMs evenly loaded (measured: 3.55 ms per n = 30 pass against 4.78 ms with one
// wave of persistent CTAs and 5.92 ms with one buffer).
template <typename T2>
__global__ void __launch_bounds__(kThreads, 6) k_permute(T2 *a, PermArgs P) {
    constexpr int apu = 16 / sizeof(T2);  // amplitudes per 16-byte unit
    extern __shared__ __align__(16) unsigned char smem[];
    T2 *sA = reinterpret_cast<T2 *>(smem);            // [2][kUnitsPerCta * apu]
    T2 *sB = sA + 2 * kUnitsPerCta * apu;             // [2][kUnitsPerCta * apu]
    __shared__ int64_t s_base[2][kMaxItems], s_base2[2][kMaxItems];
    __shared__ int s_mode[2][kMaxItems];  // 0 skip, 1 self, 2 exchange

    const int T = 1 << P.vbits;
    const int lg_upt = P.vbits - (apu == 2 ? 1 : 0);
    const int upt = 1 << lg_upt;  // units per tile (T / apu)
    const int units = P.ib * upt;
    const int64_t nbatch = (P.nitems + P.ib - 1) / P.ib;

    // items of batch `batch` into slot k (threads < ib), then (after a barrier) its loads
    auto describe = [&](int64_t batch, int k) {
        for (int it = threadIdx.x; it < P.ib; it += kThreads) {
            const int64_t o = batch * P.ib + it;
            int mode = 0;
            int64_t base = 0, base2 = 0;
            if (o < P.nitems) {
                // deposit o into the bits outside V (zero bits inserted at V, ascending)
                base = o;
                for (int j = 0; j < P.vbits; ++j) base = insert0(base, P.vsorted[j]);
                base2 = base;
                for (int j = 0; j < P.nhigh; ++j) {
                    const int64_t d = ((base2 >> P.hp[j]) ^ (base2 >> P.hq[j])) & 1;
                    base2 ^= (d << P.hp[j]) | (d << P.hq[j]);
                }
                if (base2 > base) mode = 2;
                else if (base2 == base && P.nlow > 0) mode = 1;
            }
            s_base[k][it] = base;
            s_base2[k][it] = base2;
            s_mode[k][it] = mode;
        }
    };
    auto load = [&](int k) {
        const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(sA + (size_t)k * kUnitsPerCta * apu);
        const uint32_t b0 = (uint32_t)__cvta_generic_to_shared(sB + (size_t)k * kUnitsPerCta * apu);
        for (int u = threadIdx.x; u < units; u += kThreads) {
            const int it = u >> lg_upt, ut = u & (upt - 1);
            const int mode = s_mode[k][it];
            if (!mode) continue;
            const int64_t off = unit_offset(P, ut * apu);
            cp_async16(a0 + (uint32_t)u * 16u, a + s_base[k][it] + off);
            if (mode == 2) cp_async16(b0 + (uint32_t)u * 16u, a + s_base2[k][it] + off);
        }
    };

    int64_t batch = blockIdx.x;
    if (batch < nbatch) {
        describe(batch, 0);
        __syncthreads();
        load(0);
    }
    cp_async_commit();
    for (int k = 0; batch < nbatch; batch += gridDim.x, k ^= 1) {
        const int64_t next = batch + gridDim.x;
        if (next < nbatch) {
            describe(next, k ^ 1);
            __syncthreads();
            load(k ^ 1);
        }
        cp_async_commit();
        cp_async_wait<1>();  // this batch's copies (the next one's may still be in flight)
        __syncthreads();
        const T2 *A = sA + (size_t)k * kUnitsPerCta * apu, *B = sB + (size_t)k * kUnitsPerCta * apu;
        for (int u = threadIdx.x; u < units; u += kThreads) {
            const int it = u >> lg_upt, ut = u & (upt - 1);
            const int mode = s_mode[k][it];
            if (!mode) continue;
            const int v0 = ut * apu;
            const int64_t off = unit_offset(P, v0);
            T2 outA[apu], outB[apu];
#pragma unroll
            for (int e = 0; e < apu; ++e) {
                int v = v0 + e;
                for (int j = 0; j < P.nlow; ++j) {
                    const int d = ((v >> P.lp[j]) ^ (v >> P.lq[j])) & 1;
                    v ^= (d << P.lp[j]) | (d << P.lq[j]);
                }
                const size_t src = (size_t)it * T + v;
                outA[e] = mode == 2 ? B[src] : A[src];  // a'[(o, v)]  = a[(o', P_low(v))]
                outB[e] = A[src];                       // a'[(o', v)] = a[(o, P_low(v))]
            }
            *reinterpret_cast<uint4 *>(a + s_base[k][it] + off) = *reinterpret_cast<const uint4 *>(outA);
            if (mode == 2) *reinterpret_cast<uint4 *>(a + s_base2[k][it] + off) = *reinterpret_cast<const uint4 *>(outB);
        }
        __syncthreads();  // slot k is free for the batch after next
    }
    cp_async_wait<0>();
}

}  // namespace

void launch_permute(int dtype, void *state, int n, const std::vector<std::pair<int32_t, int32_t>> &pairs,
                    cudaStream_t st) {
    if (pairs.empty()) return;
    const int apu = dtype == SV_C64 ? 2 : 1;
    const int lg_apu = dtype == SV_C64 ? 1 : 0;
    if (n < lg_apu + 1) fail(SV_ERR_ARG, "state too small to permute");
    PermArgs A{};
    uint64_t used = 0;
    for (auto pq : pairs) {
        int p = std::min(pq.first, pq.second), q = std::max(pq.first, pq.second);
        if (p < 0 || q >= n || p == q) fail(SV_ERR_ARG, "permute: bit out of range");
        if (((used >> p) & 1) || ((used >> q) & 1)) fail(SV_ERR_ARG, "permute: pairs not disjoint");
        used |= (1ull << p) | (1ull << q);
    }
    if ((size_t(1) << n) * (dtype == SV_C64 ? 8 : 16) <= (size_t)kUnitsPerCta * 16) {
        // the whole state is one tile
        A.L0 = n;
        A.vbits = n;
        A.nextra = 0;
        for (int j = 0; j < n; ++j) A.vpos[j] = j;
        for (auto pq : pairs) {
            A.lp[A.nlow] = std::min(pq.first, pq.second);
            A.lq[A.nlow] = std::max(pq.first, pq.second);
            ++A.nlow;
        }
    } else {
        A.L0 = dtype == SV_C64 ? 4 : 3;
        std::vector<int> extras;
        for (auto pq : pairs) {
            const int p = std::min(pq.first, pq.second), q = std::max(pq.first, pq.second);
            if (p < A.L0 && q >= A.L0) extras.push_back(q);
        }
        std::sort(extras.begin(), extras.end());
        A.nextra = (int)extras.size();
        A.vbits = A.L0 + A.nextra;
        for (int j = 0; j < A.L0; ++j) A.vpos[j] = j;
        for (int j = 0; j < A.nextra; ++j) A.vpos[A.L0 + j] = extras[j];
        for (auto pq : pairs) {
            const int p = std::min(pq.first, pq.second), q = std::max(pq.first, pq.second);
            if (p < A.L0) {
                int vq = q;
                if (q >= A.L0) vq = A.L0 + (int)(std::find(extras.begin(), extras.end(), q) - extras.begin());
                A.lp[A.nlow] = p;
                A.lq[A.nlow] = vq;
                ++A.nlow;
            } else {
                if (A.nhigh >= 32) fail(SV_ERR_ARG, "permute: too many pairs");
                A.hp[A.nhigh] = p;
                A.hq[A.nhigh] = q;
                ++A.nhigh;
            }
        }
    }
    const int upt = (1 << A.vbits) / apu;
    if (upt > kUnitsPerCta) fail(SV_ERR_UNSUPPORTED, "permute: tile too large");
    A.ib = std::min(kMaxItems, std::max(1, kUnitsPerCta / upt));
    for (int j = 0; j < A.vbits; ++j) A.vsorted[j] = A.vpos[j];
    std::sort(A.vsorted, A.vsorted + A.vbits);
    A.nitems = int64_t(1) << (n - A.vbits);
    if (A.ib > A.nitems) A.ib = (int)A.nitems;
    const int64_t nbatch = (A.nitems + A.ib - 1) / A.ib;
    // two slots x two sides of kUnitsPerCta 16-byte units: 32 KiB, six CTAs per SM
    const size_t smem = (size_t)4 * kUnitsPerCta * 16;
    int per_sm = 0;
    if (dtype == SV_C64) {
        check_cuda(cudaFuncSetAttribute(k_permute<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(permute)");
        check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_permute<float2>, kThreads, smem),
                   "occupancy(permute)");
    } else {
        check_cuda(cudaFuncSetAttribute(k_permute<double2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem),
                   "cudaFuncSetAttribute(permute)");
        check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_permute<double2>, kThreads, smem),
                   "occupancy(permute)");
    }
    if (per_sm < 1) per_sm = 1;
    const int grid = (int)std::min<int64_t>(nbatch, (int64_t)num_sms() * per_sm * 32);
    if (dtype == SV_C64)
        k_permute<float2><<<grid, kThreads, smem, st>>>((float2 *)state, A);
    else
        k_permute<double2><<<grid, kThreads, smem, st>>>((double2 *)state, A);
    check_cuda(cudaGetLastError(), "permute kernel launch");
}

}  // namespace sv
