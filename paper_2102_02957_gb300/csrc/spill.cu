// Host-resident states: the GPU as a cache for chunks in host memory (Sec. IV.C: chunks that do
// not fit in GPU memory are kept in host memory and staged through the GPU; Sec. V.B runs 33-35
// qubits that way).  The state's 2^n amplitudes stay in host memory (pinned, so the copies run
// at the link's rate); a plan of the paper's layout (contiguous chunks, chunk_swap rounds) runs in
// passes, and every pass streams the whole state through a device work buffer once.
//
// A pass is a run of consecutive plan ops.  Its sub-state is m + |H| qubits: the state's low m
// bits (m >= c, so every chunk of a section lies inside) and H, the set of the pass's swap-pair
// bits at or above m.  The sub-states of a pass are the 2^(n - m - |H|) values of the remaining
// high bits; each is gathered from 2^|H| host slabs of 2^m contiguous amplitudes into the buffer
// (slab e of the sub-state at offset e << m, sub-state bit m + t = state bit H[t]), every op of
// the pass runs on it with the library's section and permutation kernels (pairs renumbered), and
// it is written back.  A run may be extended while c + |{pair bits >= c}| <= M (2^M amplitudes fit
// half the buffer: two sub-states are in flight, on two streams, so one's copies overlap the
// other's kernels); m is then the largest value with m + |{pair bits >= m}| <= M.  A round whose
// pairs alone do not fit is split into several items (its transpositions commute).
#include <algorithm>
#include <cstring>
#include <vector>

#include "sv_internal.h"

namespace sv {
namespace {

// Slab copies by a kernel, for host memory the GPU can address directly (pinned and mapped):
// sub-state amplitude j = (slab e << m) | w lives in host amplitude base | dep(e) | w, dep(e)
// depositing e's bit t at state bit high[t].  One 16-byte unit per thread and step; IN copies
// host -> sub-state, else sub-state -> host.  Used where the slabs are small, so that a pass is a
// few launches instead of thousands of tiny copies.
struct SlabArgs {
    int m, nh, lg_apu;  // slab bits, |H|, log2 amplitudes per 16-byte unit
    int8_t high[64];
    int64_t base;       // state index of the sub-state's first amplitude
    int64_t units;      // 16-byte units of the sub-state
};

template <bool IN>
__global__ void __launch_bounds__(256) k_slab_copy(uint4 *__restrict__ dev, uint4 *__restrict__ host, SlabArgs a) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < a.units; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = u << a.lg_apu;  // sub-state amplitude of the unit's first element
        const int64_t e = j >> a.m;
        int64_t x = a.base | (j & ((int64_t(1) << a.m) - 1));
        for (int t = 0; t < a.nh; ++t)
            if ((e >> t) & 1) x |= int64_t(1) << a.high[t];
        const int64_t hu = x >> a.lg_apu;
        if (IN) dev[u] = host[hu];
        else host[hu] = dev[u];
    }
}

constexpr size_t kKernelSlabBytes = size_t(1) << 20;  // slabs below 1 MiB go through k_slab_copy

struct PassItem {
    int op;                                          // plan op
    std::vector<std::pair<int32_t, int32_t>> pairs;  // swap pairs of this item (rounds only)
};

struct Pass {
    std::vector<PassItem> items;
    int m = 0;               // low bits of every slab
    std::vector<int> high;   // H: state bits >= m carried by the sub-state, ascending
};

// Distinct pair bits >= lo of a set of items.
int count_high(const std::vector<PassItem> &items, int lo, std::vector<int> *bits = nullptr) {
    std::vector<char> seen(64, 0);
    int k = 0;
    for (const PassItem &it : items)
        for (const auto &pq : it.pairs)
            for (int b : {pq.first, pq.second})
                if (b >= lo && !seen[b]) {
                    seen[b] = 1;
                    ++k;
                }
    if (bits) {
        bits->clear();
        for (int b = 0; b < 64; ++b)
            if (seen[b]) bits->push_back(b);
    }
    return k;
}

std::vector<Pass> make_passes(const sv_plan &plan, int M) {
    const int c = std::min(plan.c, plan.n);
    std::vector<PassItem> work;  // ops, with over-wide rounds split into items that fit
    for (int oi = 0; oi < (int)plan.ops.size(); ++oi) {
        const PlanOp &op = plan.ops[(size_t)oi];
        if (op.kind == 2) {
            work.push_back(PassItem{oi, {}});
            continue;
        }
        PassItem cur{oi, {}};
        for (const auto &pq : op.pairs) {
            PassItem trial = cur;
            trial.pairs.push_back(pq);
            if (!cur.pairs.empty() && c + count_high({trial}, c) > M) {
                work.push_back(cur);
                cur = PassItem{oi, {pq}};
            } else {
                cur = trial;
            }
        }
        if (!cur.pairs.empty()) work.push_back(cur);
    }
    std::vector<Pass> passes;
    for (size_t i = 0; i < work.size();) {
        Pass p;
        p.items.push_back(work[i++]);
        while (i < work.size()) {
            std::vector<PassItem> trial = p.items;
            trial.push_back(work[i]);
            if (c + count_high(trial, c) > M) break;
            p.items.push_back(work[i++]);
        }
        // the largest m in [c, M] whose sub-state (m + |pair bits >= m|) fits
        p.m = c;
        for (int m = std::min(M, plan.n); m >= c; --m)
            if (m + count_high(p.items, m) <= M) {
                p.m = m;
                break;
            }
        count_high(p.items, p.m, &p.high);
        passes.push_back(std::move(p));
    }
    return passes;
}

// Run one pass: for every value of the state bits >= m outside H, gather the sub-state's 2^|H|
// slabs, run the pass's items on it, write it back.  Sub-states alternate between the two halves
// of the work buffer and the two streams.
void run_pass(const Pass &p, const sv_plan &plan, int dtype, unsigned char *host, unsigned char *host_dev,
              unsigned char *work, size_t half_bytes, const unsigned char *prog, const SimtPrograms &sp, int *dev_err,
              cudaStream_t *st, uint64_t wait_ns) {
    const int n = plan.n, m = p.m, nh = (int)p.high.size(), nsub = m + nh;
    const size_t elem = dtype == SV_C64 ? 8 : 16;
    const size_t slab_bytes = (size_t(1) << m) * elem;
    if ((size_t(1) << nsub) * elem > half_bytes) fail(SV_ERR_ARG, "host-resident pass does not fit the work buffer");
    std::vector<int> outer;  // state bits >= m not in H: they number the sub-states
    for (int b = m; b < n; ++b)
        if (std::find(p.high.begin(), p.high.end(), b) == p.high.end()) outer.push_back(b);
    // the items' pairs in sub-state bit numbers
    auto local_bit = [&](int b) {
        if (b < m) return b;
        return m + (int)(std::find(p.high.begin(), p.high.end(), b) - p.high.begin());
    };
    std::vector<std::vector<std::pair<int32_t, int32_t>>> pairs(p.items.size());
    for (size_t i = 0; i < p.items.size(); ++i)
        for (const auto &pq : p.items[i].pairs) pairs[i].emplace_back(local_bit(pq.first), local_bit(pq.second));
    const int64_t nsubs = int64_t(1) << outer.size();
    // small slabs (passes that carry many high swap bits) move by kernel when the host memory is
    // mapped into the device's address space
    const bool by_kernel = host_dev && slab_bytes < kKernelSlabBytes;
    SlabArgs sa{};
    sa.m = m;
    sa.nh = nh;
    sa.lg_apu = elem == 8 ? 1 : 0;
    for (int t = 0; t < nh; ++t) sa.high[t] = (int8_t)p.high[(size_t)t];
    sa.units = (int64_t)(((size_t(1) << nsub) * elem) / 16);
    const unsigned grid = (unsigned)std::min<int64_t>((sa.units + 255) / 256, (int64_t)num_sms() * 8);
    for (int64_t o = 0; o < nsubs; ++o) {
        const int k = (int)(o & 1);
        unsigned char *buf = work + (size_t)k * half_bytes;
        int64_t base = 0;  // state index of the sub-state's first amplitude
        for (size_t t = 0; t < outer.size(); ++t)
            if ((o >> t) & 1) base |= int64_t(1) << outer[t];
        auto slab_host = [&](int e) {
            int64_t x = base;
            for (int t = 0; t < nh; ++t)
                if ((e >> t) & 1) x |= int64_t(1) << p.high[(size_t)t];
            return host + (size_t)x * elem;
        };
        sa.base = base;
        if (by_kernel) {
            k_slab_copy<true><<<grid, 256, 0, st[k]>>>(reinterpret_cast<uint4 *>(buf), reinterpret_cast<uint4 *>(host_dev), sa);
            check_cuda(cudaGetLastError(), "slab gather launch");
        } else {
            for (int e = 0; e < (1 << nh); ++e)
                check_cuda(cudaMemcpyAsync(buf + (size_t)e * slab_bytes, slab_host(e), slab_bytes, cudaMemcpyHostToDevice,
                                           st[k]),
                           "cudaMemcpyAsync(host slab in)");
        }
        for (size_t i = 0; i < p.items.size(); ++i) {
            const int op = p.items[i].op;
            if (plan.ops[(size_t)op].kind == 2) {
                const SimtPrograms::Prog *pr = nullptr;
                for (const auto &q : sp.progs)
                    if (q.op_index == op) pr = &q;
                if (!pr) fail(SV_ERR_PLAN, "no program for a blocking section");
                launch_block(dtype, buf, nsub, plan.c, prog + pr->off, pr->nseg, pr->ngate, dev_err, sp.seg_bits, st[k],
                             wait_ns);
            } else if (!pairs[i].empty()) {
                launch_permute(dtype, buf, nsub, pairs[i], st[k]);
            }
        }
        if (by_kernel) {
            k_slab_copy<false><<<grid, 256, 0, st[k]>>>(reinterpret_cast<uint4 *>(buf), reinterpret_cast<uint4 *>(host_dev), sa);
            check_cuda(cudaGetLastError(), "slab scatter launch");
        } else {
            for (int e = 0; e < (1 << nh); ++e)
                check_cuda(cudaMemcpyAsync(slab_host(e), buf + (size_t)e * slab_bytes, slab_bytes, cudaMemcpyDeviceToHost,
                                           st[k]),
                           "cudaMemcpyAsync(host slab out)");
        }
    }
}

}  // namespace
}  // namespace sv

using namespace sv;

extern "C" sv_status sv_apply_circuit_host(int32_t n, int32_t dtype, void *host_amps, const sv_gate *gates,
                                           int64_t n_gates, sv_plan_h plan, void *dev_work, size_t work_bytes,
                                           void *cuda_stream, int32_t *passes_out) {
    void *owned = nullptr;
    void *progbuf = nullptr;
    int *dev_err = nullptr;
    cudaStream_t st[2] = {nullptr, nullptr};
    cudaEvent_t ev = nullptr;
    sv_status status = SV_OK;
    try {
        if (!host_amps || !plan || (n_gates > 0 && !gates)) fail(SV_ERR_ARG, "null argument");
        if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_ARG, "unknown dtype");
        if (n < 1 || n > 40 || plan->n != n) fail(SV_ERR_PLAN, "plan was made for another qubit count");
        if (plan->pinned) fail(SV_ERR_UNSUPPORTED, "host-resident states need a contiguous-chunk plan (gather_pinned = 0)");
        if ((int64_t)plan->keys.size() != n_gates) fail(SV_ERR_PLAN, "plan was made for another gate list");
        for (int64_t i = 0; i < n_gates; ++i) {
            const GateKey key{gates[i].nq, gates[i].q[0], gates[i].nq == 2 ? gates[i].q[1] : -1, gates[i].flags};
            if (!(key == plan->keys[(size_t)i])) fail(SV_ERR_PLAN, "gate list differs from the planned one");
        }
        const size_t elem = dtype == SV_C64 ? 8 : 16;
        const int c = std::min(plan->c, n);
        int M = 0;  // 2^M amplitudes per half of the work buffer
        while (M < n && (size_t(2) << (M + 1)) * elem <= work_bytes) ++M;
        if (M < n && M < c + 2)
            fail(SV_ERR_ARG, "work buffer too small: it must hold two sub-states of 2^(c+2) amplitudes");
        const size_t half_bytes = (size_t(1) << M) * elem;
        if (!dev_work) {
            check_cuda(cudaMalloc(&owned, 2 * half_bytes), "cudaMalloc(work buffer)");
            dev_work = owned;
        }
        SimtPrograms sp;
        build_simt_programs(plan, gates, dtype, sp);
        check_cuda(cudaMalloc(&progbuf, std::max<size_t>(sp.host.size(), 256)), "cudaMalloc(programs)");
        check_cuda(cudaMalloc(&dev_err, sizeof(int)), "cudaMalloc(error word)");
        const cudaStream_t caller = (cudaStream_t)cuda_stream;
        check_cuda(cudaMemsetAsync(dev_err, 0, sizeof(int), caller), "cudaMemsetAsync");
        if (!sp.host.empty())
            check_cuda(cudaMemcpyAsync(progbuf, sp.host.data(), sp.host.size(), cudaMemcpyHostToDevice, caller),
                       "upload programs");
        for (auto &s : st) check_cuda(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "cudaStreamCreate");
        check_cuda(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "cudaEventCreate");
        auto join = [&](cudaStream_t from, cudaStream_t to) {
            check_cuda(cudaEventRecord(ev, from), "cudaEventRecord");
            check_cuda(cudaStreamWaitEvent(to, ev, 0), "cudaStreamWaitEvent");
        };
        join(caller, st[0]);
        join(caller, st[1]);
        const uint64_t wait_ns = plan->wait_limit_ms > 0 ? (uint64_t)plan->wait_limit_ms * 1000000ull : kDefaultWaitNs;
        // the device's address of the host state, if the GPU can address it directly (pinned and
        // mapped host memory); else every slab goes through a copy
        unsigned char *host_dev = nullptr;
        {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, host_amps) == cudaSuccess && at.type == cudaMemoryTypeHost &&
                at.devicePointer != nullptr && (reinterpret_cast<uintptr_t>(at.devicePointer) % 16) == 0)
                host_dev = static_cast<unsigned char *>(at.devicePointer);
            cudaGetLastError();  // an unregistered pointer leaves an error state; clear it
        }
        const std::vector<Pass> passes = make_passes(*plan, M);
        for (const Pass &p : passes) {
            run_pass(p, *plan, dtype, static_cast<unsigned char *>(host_amps), host_dev, static_cast<unsigned char *>(dev_work),
                     half_bytes, static_cast<const unsigned char *>(progbuf), sp, dev_err, st, wait_ns);
            // the next pass reads what either stream wrote back
            join(st[0], st[1]);
            join(st[1], st[0]);
        }
        join(st[0], caller);
        join(st[1], caller);
        int e = 0;
        check_cuda(cudaMemcpyAsync(&e, dev_err, sizeof(int), cudaMemcpyDeviceToHost, caller), "read error word");
        check_cuda(cudaStreamSynchronize(caller), "cudaStreamSynchronize");
        if (e == DEV_ERR_TIMEOUT) fail(SV_ERR_TIMEOUT, "a bounded device wait expired");
        if (e != DEV_OK) fail(SV_ERR_CUDA, "device error word set");
        if (passes_out) *passes_out = (int32_t)passes.size();
    } catch (const sv::Error &err) {
        sv::set_error(err.msg);
        status = err.code;
    } catch (const std::bad_alloc &) {
        sv::set_error("host allocation failed");
        status = SV_ERR_OOM;
    }
    for (auto &s : st)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (ev) cudaEventDestroy(ev);
    if (owned) cudaFree(owned);
    if (progbuf) cudaFree(progbuf);
    if (dev_err) cudaFree(dev_err);
    return status;
}
