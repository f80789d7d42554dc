// C ABI entry points (include/sv.h): state handles, planning, execution and readouts.
#include <algorithm>
#include <cstring>
#include <atomic>
#include <mutex>
#include <thread>

#include "sv_internal.h"

namespace sv {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

void fail(sv_status code, const std::string &msg) { throw Error{code, msg}; }

void check_cuda(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(SV_ERR_OOM, std::string(what) + ": " + cudaGetErrorString(e));
    fail(SV_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int num_sms() {
    static int cached = 0;
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (!cached) {
        int dev = 0;
        check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
        check_cuda(cudaDeviceGetAttribute(&cached, cudaDevAttrMultiProcessorCount, dev), "cudaDeviceGetAttribute");
    }
    return cached;
}

static size_t amp_bytes(int dtype) { return dtype == SV_C64 ? 8 : 16; }

static int reduce_blocks(int n) {
    const int64_t len = int64_t(1) << n;
    return (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8, len / 256));
}

static void ensure_scratch(sv_state *h, size_t bytes) {
    if (h->scratch_bytes >= bytes) return;
    if (h->scratch) {
        check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        cudaFree(h->scratch);
        h->scratch = nullptr;
        h->scratch_bytes = 0;
    }
    check_cuda(cudaMalloc(&h->scratch, bytes), "cudaMalloc(scratch)");
    h->scratch_bytes = bytes;
}

void check_dev_error(sv_state *h) {
    int e = 0;
    check_cuda(cudaMemcpyAsync(&e, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream), "read error word");
    check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    if (e != DEV_OK) {
        int zero = 0;
        cudaMemcpy(h->dev_err, &zero, sizeof(int), cudaMemcpyHostToDevice);
        if (e == DEV_ERR_TIMEOUT) fail(SV_ERR_TIMEOUT, "a bounded device wait expired");
        fail(SV_ERR_CUDA, "device error word set");
    }
}

static void validate_gates(int n, const sv_gate *gates, int64_t n_gates) {
    if (n_gates < 0 || (n_gates > 0 && !gates)) fail(SV_ERR_ARG, "bad gate list");
    for (int64_t i = 0; i < n_gates; ++i) {
        const sv_gate &g = gates[i];
        if (g.nq != 1 && g.nq != 2) fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": nq must be 1 or 2");
        for (int j = 0; j < g.nq; ++j)
            if (g.q[j] < 0 || g.q[j] >= n) fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": qubit out of range");
        if (g.nq == 2 && g.q[0] == g.q[1]) fail(SV_ERR_ARG, "gate " + std::to_string(i) + ": repeated qubit");
    }
}

// Device program of one blocking section: register groups, then gate records, laid out as
// the kernel copies them into shared memory.
struct BlockProg {
    size_t off;
    int nseg, ngate;
    int r = 0;         // tensor-core register-group width of the sweep
    GatherLayout lay;  // gathered sections only
    int op_index = -1;
    bool gathered = false;
};

// Runs fn(0..count-1) on up to 8 host threads (on the calling thread alone for small counts).
// fn must not throw except std::bad_alloc, which is passed on to the caller.
template <typename F>
static void parallel_for(int count, F fn) {
    const unsigned hw = std::thread::hardware_concurrency();
    const int nth = (int)std::max(1u, std::min(8u, std::min(hw ? hw : 1u, (unsigned)(count / 4))));
    if (nth <= 1) {
        for (int i = 0; i < count; ++i) fn(i);
        return;
    }
    std::atomic<bool> oom{false};
    auto work = [&](int t) {
        try {
            for (int i = t; i < count; i += nth) fn(i);
        } catch (const std::bad_alloc &) {
            oom = true;
        }
    };
    std::vector<std::thread> pool;
    int started = 1;
    try {
        pool.reserve((size_t)nth);
        for (; started < nth; ++started) pool.emplace_back(work, started);
    } catch (...) {
        // threads that could not start: their shares run on this thread
    }
    for (int t = started; t < nth; ++t) work(t);
    work(0);
    for (std::thread &th : pool) th.join();
    if (oom) throw std::bad_alloc();
}

// Tensor-core programs: every register group (r bits) of a section becomes one fused unitary.  A
// section whose B operands (tc_b_bytes(r) per group: 2, 8 or 32 KiB) would not fit next to the
// chunk ring in shared memory is split into consecutive sweeps of at most max_tc_segs(r) groups.
// A section's width is its own where the plan chose one (steered plans), else the plan's.
// Appended after the section programs: the composer's work lists, one per width (3, 4, 5 bits),
// and the FP64 gate records they read.
static int max_tc_segs(int r) { return r == 3 ? 24 : r == 4 ? 11 : 3; }

static void build_programs_tc(const sv_plan *plan, const sv_gate *gates, int r_plan, std::vector<unsigned char> &host,
                              std::vector<BlockProg> &progs, size_t (&cs_off)[3], int (&ncs)[3], size_t &g_off,
                              size_t &flag_off) {
    host.clear();
    progs.clear();
    auto align = [&](size_t a) {
        while (host.size() % a) host.push_back(0);
    };
    std::vector<ComposeSeg> cs[3];  // per width 3, 4, 5
    std::vector<DevGate<double>> dg;
    // each section's chunk layout, local gates and checks, in section order
    struct Section {
        size_t oi;
        int r, width;
        GatherLayout lay;
        std::vector<BlockGate> gates;
        std::vector<HostSeg> segs;
    };
    std::vector<Section> secs;
    for (size_t oi = 0; oi < plan->ops.size(); ++oi) {
        const PlanOp &op0 = plan->ops[oi];
        if (op0.kind != 2 && op0.kind != 4) continue;
        Section sc{};
        sc.oi = oi;
        sc.r = op0.seg_bits ? op0.seg_bits : r_plan;
        if (sc.r < 3 || sc.r > 5) fail(SV_ERR_PLAN, "tensor-core register groups have 3, 4 or 5 bits");
        sc.width = std::min(plan->c, plan->n);
        if (op0.kind == 4) {
            sc.lay = gather_layout(op0.mask, plan->n, 8);
            sc.gates = localize_gates(op0, plan->n, plan->c, &sc.lay);
            sc.width = sc.lay.ce;
        } else {
            sc.gates = localize_gates(op0, plan->n, plan->c, nullptr);
        }
        for (const BlockGate &g : sc.gates)
            if (g.ext[0] >= 0 || g.ext[1] >= 0) fail(SV_ERR_PLAN, "tensor-core sections take no gates outside the chunk");
        if (sc.width - plan->reserve < sc.r + 7) fail(SV_ERR_PLAN, "a section's chunk is too small for its register-group width");
        secs.push_back(std::move(sc));
    }
    // register groups of every section (independent searches, spread over host threads; each
    // section's result is its own, so the program does not depend on the threading)
    parallel_for((int)secs.size(), [&](int i) {
        Section &sc = secs[(size_t)i];
        sc.segs = segment_block(sc.gates, sc.width, sc.r, 8);
    });
    for (const Section &sc : secs) {
        const size_t oi = sc.oi;
        const PlanOp &op0 = plan->ops[oi];
        const int r = sc.r;
        const int kMaxTcSegs = max_tc_segs(r);
        const int b_bytes = tc_b_bytes(r);
        const GatherLayout &lay = sc.lay;
        const std::vector<HostSeg> &segs = sc.segs;
        for (size_t p0 = 0; p0 < segs.size(); p0 += kMaxTcSegs) {
            const size_t p1 = std::min(segs.size(), p0 + (size_t)kMaxTcSegs);
            BlockProg bp{};
            bp.lay = lay;
            bp.gathered = op0.kind == 4;
            bp.op_index = (int)oi;
            bp.r = r;
            align(256);
            bp.off = host.size();
            bp.nseg = (int)(p1 - p0);
            bp.ngate = 0;
            for (size_t k = p0; k < p1; ++k) {
                const HostSeg &s = segs[k];
                DevSeg d;
                std::memset(&d, 0, sizeof(d));
                d.r = (int8_t)s.r;
                for (int q = 0; q < s.r; ++q) d.pos[q] = (int8_t)s.pos[q];
                for (int q = 0; q < 5; ++q) d.lane[q] = (int8_t)s.lane[q];
                d.nrest = (int8_t)s.nrest;
                for (int q = 0; q < s.nrest; ++q) d.rest[q] = (int8_t)s.rest[q];
                d.flags = (int8_t)((k == p0 ? 1 : 0) | (k + 1 == p1 ? 2 : 0));
                const unsigned char *p = reinterpret_cast<const unsigned char *>(&d);
                host.insert(host.end(), p, p + sizeof(d));
            }
            align(16);
            const size_t b_base = host.size();
            host.resize(host.size() + (size_t)bp.nseg * b_bytes, 0);
            for (size_t k = p0; k < p1; ++k) {
                ComposeSeg c{};
                c.flag_off = kNoFlag;
                c.g0 = (int32_t)dg.size();
                for (int32_t gi : segs[k].gates) {
                    DevGate<double> g;
                    const BlockGate &bg = sc.gates[gi];
                    encode_gate<double>(gates[bg.gi], bg, segs[k], g);
                    dg.push_back(g);
                }
                c.g1 = (int32_t)dg.size();
                c.b_off = (uint32_t)(b_base + (k - p0) * b_bytes);
                cs[r - 3].push_back(c);
            }
            progs.push_back(bp);
        }
    }
    const unsigned char *p = nullptr;
    for (int w = 0; w < 3; ++w) {
        align(256);
        cs_off[w] = host.size();
        ncs[w] = (int)cs[w].size();
        p = reinterpret_cast<const unsigned char *>(cs[w].data());
        host.insert(host.end(), p, p + cs[w].size() * sizeof(ComposeSeg));
    }
    align(256);
    g_off = host.size();
    p = reinterpret_cast<const unsigned char *>(dg.data());
    host.insert(host.end(), p, p + dg.size() * sizeof(DevGate<double>));
    align(256);
    // "every fused group is unitary", set here and cleared by the compose kernel
    flag_off = host.size();
    const int32_t one[4] = {1, 0, 0, 0};
    p = reinterpret_cast<const unsigned char *>(one);
    host.insert(host.end(), p, p + sizeof(one));
}

template <typename T>
static void build_programs(const sv_plan *plan, const sv_gate *gates, int seg_bits, std::vector<unsigned char> &host,
                           std::vector<BlockProg> &progs) {
    host.clear();
    progs.clear();
    auto align = [&](size_t a) {
        while (host.size() % a) host.push_back(0);
    };
    for (const PlanOp &op0 : plan->ops) {
        if (op0.kind != 2 && op0.kind != 4) continue;
        int width = std::min(plan->c, plan->n);
        BlockProg bp{};
        PlanOp local;
        const PlanOp *opp = &op0;
        local = op0;
        if (op0.kind == 4) {  // gate bits -> chunk-local bits of the gathered layout
            bp.lay = gather_layout(op0.mask, plan->n, (int)(2 * sizeof(T)));
            local.gates = localize_gates(op0, plan->n, plan->c, &bp.lay);
            width = bp.lay.ce;
            bp.gathered = true;
        } else {
            local.gates = localize_gates(op0, plan->n, plan->c, nullptr);
        }
        opp = &local;
        bp.op_index = (int)(&op0 - plan->ops.data());
        const PlanOp &op = *opp;
        std::vector<HostSeg> segs = segment_block(op.gates, width, seg_bits, (int)(2 * sizeof(T)));
        std::vector<DevSeg> dsegs;
        std::vector<DevGate<T>> dgates;
        for (const HostSeg &s : segs) {
            DevSeg d;
            std::memset(&d, 0, sizeof(d));
            d.r = (int8_t)s.r;
            for (int k = 0; k < s.r; ++k) d.pos[k] = (int8_t)s.pos[k];
            for (int k = 0; k < 5; ++k) d.lane[k] = (int8_t)s.lane[k];
            d.nrest = (int8_t)s.nrest;
            for (int k = 0; k < s.nrest; ++k) d.rest[k] = (int8_t)s.rest[k];
            d.flags = (int8_t)s.flags;
            d.g0 = (int16_t)dgates.size();
            for (int32_t gi : s.gates) {
                DevGate<T> dg;
                const BlockGate &bg = op.gates[gi];
                encode_gate<T>(gates[bg.gi], bg, s, dg);
                dgates.push_back(dg);
            }
            if (dgates.size() > 32767) fail(SV_ERR_UNSUPPORTED, "too many gates in one blocking section");
            d.g1 = (int16_t)dgates.size();
            dsegs.push_back(d);
        }
        align(256);
        bp.off = host.size();
        bp.nseg = (int)dsegs.size();
        bp.ngate = (int)dgates.size();
        const unsigned char *p = reinterpret_cast<const unsigned char *>(dsegs.data());
        host.insert(host.end(), p, p + dsegs.size() * sizeof(DevSeg));
        align(16);
        p = reinterpret_cast<const unsigned char *>(dgates.data());
        host.insert(host.end(), p, p + dgates.size() * sizeof(DevGate<T>));
        align(16);
        progs.push_back(bp);
    }
    align(256);
}

void build_simt_programs(const sv_plan *plan, const sv_gate *gates, int dtype, SimtPrograms &out) {
    out.seg_bits = (dtype == SV_C64 && plan->seg_bits == 5) ? 5 : 4;
    std::vector<BlockProg> progs;
    if (dtype == SV_C64) build_programs<float>(plan, gates, out.seg_bits, out.host, progs);
    else build_programs<double>(plan, gates, out.seg_bits, out.host, progs);
    out.progs.clear();
    for (const BlockProg &bp : progs) out.progs.push_back(SimtPrograms::Prog{bp.off, bp.nseg, bp.ngate, bp.op_index});
}

static void upload_program(sv_state *h, const std::vector<unsigned char> &host) {
    const size_t bytes = std::max<size_t>(host.size(), 256);
    if (h->prog_event) check_cuda(cudaEventSynchronize(h->prog_event), "cudaEventSynchronize");
    if (h->prog_host_bytes < bytes) {
        if (h->prog_host) cudaFreeHost(h->prog_host);
        h->prog_host = nullptr;
        check_cuda(cudaHostAlloc(&h->prog_host, bytes, cudaHostAllocDefault), "cudaHostAlloc(program)");
        h->prog_host_bytes = bytes;
    }
    if (h->prog_bytes < bytes) {
        if (h->prog) {
            check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
            cudaFree(h->prog);
        }
        h->prog = nullptr;
        check_cuda(cudaMalloc(&h->prog, bytes), "cudaMalloc(program)");
        h->prog_bytes = bytes;
    }
    if (!host.empty()) {
        std::memcpy(h->prog_host, host.data(), host.size());
        check_cuda(cudaMemcpyAsync(h->prog, h->prog_host, host.size(), cudaMemcpyHostToDevice, h->stream),
                   "upload program");
    }
    if (!h->prog_event) check_cuda(cudaEventCreateWithFlags(&h->prog_event, cudaEventDisableTiming), "cudaEventCreate");
    check_cuda(cudaEventRecord(h->prog_event, h->stream), "cudaEventRecord");
}

}  // namespace sv

using namespace sv;

#define SV_API_BEGIN try {
#define SV_API_END                  \
    return SV_OK;                   \
    }                               \
    catch (const sv::Error &e) {    \
        sv::set_error(e.msg);       \
        return e.code;              \
    }                               \
    catch (const std::bad_alloc &) { \
        sv::set_error("host allocation failed"); \
        return SV_ERR_OOM;          \
    }                               \
    catch (...) {                   \
        sv::set_error("unexpected exception"); \
        return SV_ERR_CUDA;         \
    }

extern "C" {

const char *sv_last_error(void) { return g_last_error.c_str(); }

void sv_options_default(sv_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->chunk_bits = 13;
    o->reserve = 0;
    o->restore_layout = 1;
    o->seg_bits = 4;
    o->use_tc = 0;
    o->use_model = 0;
    o->threads = 0;
}

sv_status sv_create(int32_t n, int32_t dtype, void *dev_buf, size_t bytes, void *cuda_stream, sv_handle *out) {
    SV_API_BEGIN
    if (!out) fail(SV_ERR_ARG, "sv_create: out is null");
    *out = nullptr;
    if (n < 1 || n > 34) fail(SV_ERR_ARG, "sv_create: n must be in [1, 34]");
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_ARG, "sv_create: unknown dtype");
    const size_t need = (size_t(1) << n) * amp_bytes(dtype);
    std::unique_ptr<sv_state> h(new sv_state());
    h->n = n;
    h->dtype = dtype;
    h->stream = (cudaStream_t)cuda_stream;
    check_cuda(cudaGetDevice(&h->device), "cudaGetDevice");
    if (dev_buf) {
        if (bytes < need) fail(SV_ERR_ARG, "sv_create: buffer smaller than 2^n amplitudes");
        if (reinterpret_cast<uintptr_t>(dev_buf) % 256) fail(SV_ERR_ARG, "sv_create: buffer not 256-byte aligned");
        h->amp = dev_buf;
        h->owns_amp = false;
    } else {
        check_cuda(cudaMalloc(&h->amp, need), "cudaMalloc(state)");
        h->owns_amp = true;
    }
    check_cuda(cudaMalloc(&h->dev_err, sizeof(int)), "cudaMalloc(error word)");
    check_cuda(cudaMemsetAsync(h->dev_err, 0, sizeof(int), h->stream), "cudaMemsetAsync");
    *out = h.release();
    SV_API_END
}

sv_status sv_destroy(sv_handle h) {
    SV_API_BEGIN
    if (!h) return SV_OK;
    cudaStreamSynchronize(h->stream);
    if (h->owns_amp && h->amp) cudaFree(h->amp);
    if (h->dev_err) cudaFree(h->dev_err);
    if (h->scratch) cudaFree(h->scratch);
    if (h->prog) cudaFree(h->prog);
    if (h->prog_host) cudaFreeHost(h->prog_host);
    if (h->prog_event) cudaEventDestroy(h->prog_event);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    SV_API_END
}

sv_status sv_init_basis(sv_handle h, uint64_t basis) {
    SV_API_BEGIN
    if (!h) fail(SV_ERR_ARG, "null handle");
    if (basis >> h->n) fail(SV_ERR_ARG, "sv_init_basis: index out of range");
    launch_init_basis(h->dtype, h->amp, h->n, basis, h->stream);
    SV_API_END
}

sv_status sv_get_state(sv_handle h, void *host_out) {
    SV_API_BEGIN
    if (!h || !host_out) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    check_cuda(cudaMemcpyAsync(host_out, h->amp, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(D2H)");
    check_dev_error(h);
    SV_API_END
}

sv_status sv_set_state(sv_handle h, const void *host_in) {
    SV_API_BEGIN
    if (!h || !host_in) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    check_cuda(cudaMemcpyAsync(h->amp, host_in, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(H2D)");
    check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    SV_API_END
}

sv_status sv_get_state_async(sv_handle h, void *host_out) {
    SV_API_BEGIN
    if (!h || !host_out) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    check_cuda(cudaMemcpyAsync(host_out, h->amp, bytes, cudaMemcpyDeviceToHost, h->stream), "cudaMemcpyAsync(D2H)");
    SV_API_END
}

sv_status sv_set_state_async(sv_handle h, const void *host_in) {
    SV_API_BEGIN
    if (!h || !host_in) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    check_cuda(cudaMemcpyAsync(h->amp, host_in, bytes, cudaMemcpyHostToDevice, h->stream), "cudaMemcpyAsync(H2D)");
    SV_API_END
}

sv_status sv_device_ptr(sv_handle h, void **p) {
    SV_API_BEGIN
    if (!h || !p) fail(SV_ERR_ARG, "null argument");
    *p = h->amp;
    SV_API_END
}

sv_status sv_synchronize(sv_handle h) {
    SV_API_BEGIN
    if (!h) fail(SV_ERR_ARG, "null handle");
    check_dev_error(h);
    SV_API_END
}

sv_status sv_plan_blocking(int32_t n, const sv_gate *gates, int64_t n_gates, const sv_options *opts, sv_plan_h *out) {
    SV_API_BEGIN
    if (!out) fail(SV_ERR_ARG, "out is null");
    *out = nullptr;
    sv_options o;
    if (opts) o = *opts; else sv_options_default(&o);
    *out = plan_blocking(n, gates, n_gates, o);
    SV_API_END
}

sv_status sv_plan_free(sv_plan_h p) {
    SV_API_BEGIN
    delete p;
    SV_API_END
}

sv_status sv_plan_get_info(sv_plan_h p, sv_plan_info *info) {
    SV_API_BEGIN
    if (!p || !info) fail(SV_ERR_ARG, "null argument");
    std::memset(info, 0, sizeof(*info));
    info->n = p->n;
    info->chunk_bits = p->c;
    info->reserve = p->reserve;
    info->restore_layout = p->restore;
    for (const PlanOp &op : p->ops) {
        if (op.kind == 1) ++info->n_swap_rounds;
        if (op.kind == 2 || op.kind == 4) { ++info->n_blocks; info->n_gates_emitted += (int64_t)op.gates.size(); }
        if (op.kind == 3) ++info->n_unpermute_rounds;
    }
    info->n_segments = plan_segment_count(*p);
    for (int q = 0; q < p->n && q < 64; ++q) info->final_map[q] = p->final_map[q];
    SV_API_END
}

sv_status sv_plan_get_widths(sv_plan_h p, int32_t *out, int64_t cap, int64_t *count) {
    SV_API_BEGIN
    if (!p || !count || cap < 0) fail(SV_ERR_ARG, "null argument");
    int64_t k = 0;
    for (const PlanOp &op : p->ops) {
        if (op.kind != 2 && op.kind != 4) continue;
        if (out && k < cap) out[k] = op.seg_bits ? op.seg_bits : p->seg_bits;
        ++k;
    }
    *count = k;
    SV_API_END
}

sv_status sv_plan_serialize(sv_plan_h p, int64_t *buf, int64_t cap, int64_t *len) {
    SV_API_BEGIN
    if (!p || !len) fail(SV_ERR_ARG, "null argument");
    std::vector<int64_t> v{p->n, p->c, p->reserve, p->restore, (int64_t)p->ops.size()};
    for (const PlanOp &op : p->ops) {
        v.push_back(op.kind);
        if (op.kind == 2 || op.kind == 4) {
            if (op.kind == 4) v.push_back((int64_t)op.mask);
            v.push_back((int64_t)op.gates.size());
            for (const BlockGate &g : op.gates) {
                v.push_back(g.gi);
                v.push_back(g.nq);
                if (g.nq == 1) {
                    v.push_back(g.phys[0]);
                    v.push_back(-1);
                } else {  // ascending logical (label) order
                    const bool swap = g.label[0] > g.label[1];
                    v.push_back(swap ? g.phys[1] : g.phys[0]);
                    v.push_back(swap ? g.phys[0] : g.phys[1]);
                }
            }
        } else {
            v.push_back((int64_t)op.pairs.size());
            for (auto pq : op.pairs) {
                v.push_back(pq.first);
                v.push_back(pq.second);
            }
        }
    }
    for (int32_t x : p->final_map) v.push_back(x);
    *len = (int64_t)v.size();
    if (buf && cap > 0) std::memcpy(buf, v.data(), sizeof(int64_t) * (size_t)std::min<int64_t>(cap, *len));
    SV_API_END
}

// Timing marks around launches (profiling mode): kind 0 = per-gate, 1 = block, 2 = permute.
static void mark_begin(sv_state *h, int kind, int op = -1) {
    if (!h->profiling) return;
    const size_t need = 2 * (h->ev_marks.size() + 1);
    while (h->ev_pool.size() < need) {
        cudaEvent_t e;
        check_cuda(cudaEventCreate(&e), "cudaEventCreate");
        h->ev_pool.push_back(e);
    }
    const int idx = (int)(2 * h->ev_marks.size());
    check_cuda(cudaEventRecord(h->ev_pool[idx], h->stream), "cudaEventRecord");
    h->ev_marks.push_back(sv_state::Mark{kind, idx, op});
}

static void mark_end(sv_state *h) {
    if (!h->profiling) return;
    check_cuda(cudaEventRecord(h->ev_pool[h->ev_marks.back().ev + 1], h->stream), "cudaEventRecord");
}

sv_status sv_set_profiling(sv_handle h, int32_t on) {
    SV_API_BEGIN
    if (!h) fail(SV_ERR_ARG, "null handle");
    h->profiling = on != 0;
    SV_API_END
}

sv_status sv_apply_circuit(sv_handle h, const sv_gate *gates, int64_t n_gates, sv_plan_h plan) {
    SV_API_BEGIN
    if (!h) fail(SV_ERR_ARG, "null handle");
    validate_gates(h->n, gates, n_gates);
    if (h->profiling && !h->ev_marks.empty() && !h->stats_timed)
        check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");  // events about to be reused
    h->ev_marks.clear();
    h->stats_timed = false;
    sv_apply_stats st{};
    const double sweep = 2.0 * (double)(int64_t(1) << h->n) * (double)amp_bytes(h->dtype);
    if (!plan) {
        for (int64_t i = 0; i < n_gates; ++i) {
            mark_begin(h, 0);
            launch_gate(h->dtype, h->amp, h->n, gates[i], h->stream);
            mark_end(h);
            ++st.kernel_launches;
            ++st.sweeps_gate;
        }
    } else {
        if (plan->n != h->n) fail(SV_ERR_PLAN, "plan was made for another qubit count");
        if ((int64_t)plan->keys.size() != n_gates) fail(SV_ERR_PLAN, "plan was made for another gate list");
        for (int64_t i = 0; i < n_gates; ++i) {
            const GateKey k{gates[i].nq, gates[i].q[0], gates[i].nq == 2 ? gates[i].q[1] : -1, gates[i].flags};
            if (!(k == plan->keys[(size_t)i])) fail(SV_ERR_PLAN, "gate " + std::to_string(i) + " differs from the planned list");
        }
        std::vector<unsigned char> host;
        std::vector<BlockProg> progs;
        // SIMT register groups: 4 bits, or 5 for complex64
        const int seg_bits = (h->dtype == SV_C64 && plan->seg_bits == 5) ? 5 : 4;
        // tensor cores: complex64 with chunks of at least 128 rows of the plan's r-bit groups
        const int tc_bits = plan->seg_bits;
        const bool tc = plan->use_tc && h->dtype == SV_C64 && std::min(plan->c, plan->n) - plan->reserve >= tc_bits + 7;
        size_t cs_off[3] = {0, 0, 0}, g_off = 0, flag_off = 0;
        int ncs[3] = {0, 0, 0};
        // Tensor-core sections accumulate in FP32 with truncation, which shrinks every group's
        // result by a few units in the last place, the same way each time: a bias that compounds
        // over the circuit (norm 0.99981 after 450 quantum-volume gates at n = 30).  A unitary
        // circuit keeps the norm, so when every fused group is unitary the state is rescaled to its
        // input norm at the end: the radial error is removed, the unbiased rest stays.  The input
        // norm is taken first, so that it runs while the host builds the programs.
        const int nb_norm = reduce_blocks(h->n);
        const bool renorm = tc && !plan->tc_no_renorm;
        if (tc) ensure_scratch(h, (size_t)(2 * nb_norm + 2) * sizeof(double));
        if (renorm) {
            launch_partial_norm(h->dtype, h->amp, h->n, h->scratch, nb_norm, h->stream);
            ++st.kernel_launches;
        }
        if (tc) build_programs_tc(plan, gates, tc_bits, host, progs, cs_off, ncs, g_off, flag_off);
        else if (h->dtype == SV_C64) build_programs<float>(plan, gates, seg_bits, host, progs);
        else build_programs<double>(plan, gates, seg_bits, host, progs);
        upload_program(h, host);
        const unsigned char *base = static_cast<const unsigned char *>(h->prog);
        int *unitary_flag = tc ? reinterpret_cast<int *>(static_cast<unsigned char *>(h->prog) + flag_off) : nullptr;
        if (tc) {  // fuse every register group into its B operand, in FP64 on the GPU
            for (int w = 0; w < 3; ++w)
                if (ncs[w]) {
                    launch_compose(base + cs_off[w], ncs[w], base + g_off, h->prog, unitary_flag, w + 3, h->stream);
                    ++st.kernel_launches;
                }
        }
        const uint64_t wait_ns = plan->wait_limit_ms > 0 ? (uint64_t)plan->wait_limit_ms * 1000000ull : kDefaultWaitNs;
        size_t bi = 0;
        for (size_t oi = 0; oi < plan->ops.size(); ++oi) {
            const PlanOp &op = plan->ops[oi];
            if (op.kind == 2 || op.kind == 4) {
                for (; bi < progs.size() && progs[bi].op_index == (int)oi; ++bi) {
                    const BlockProg &bp = progs[bi];
                    mark_begin(h, 1, (int)oi);
                    if (tc)
                        launch_block_tc(h->amp, h->n, plan->c, bp.gathered ? &bp.lay : nullptr, base + bp.off, bp.nseg,
                                        h->dev_err, bp.r, h->stream, wait_ns);
                    else if (!bp.gathered)
                        launch_block(h->dtype, h->amp, h->n, plan->c, base + bp.off, bp.nseg, bp.ngate, h->dev_err,
                                     seg_bits, h->stream, wait_ns);
                    else
                        launch_block_gather(h->dtype, h->amp, h->n, bp.lay, base + bp.off, bp.nseg, bp.ngate,
                                            h->dev_err, seg_bits, h->stream, wait_ns);
                    mark_end(h);
                    ++st.sweeps_block;
                    ++st.kernel_launches;
                }
                continue;
            } else {
                mark_begin(h, 2, (int)oi);
                launch_permute(h->dtype, h->amp, h->n, op.pairs, h->stream);
                mark_end(h);
                ++st.sweeps_permute;
            }
            ++st.kernel_launches;
        }
        if (renorm) {
            launch_partial_norm(h->dtype, h->amp, h->n, h->scratch + nb_norm, nb_norm, h->stream);
            launch_renorm(h->dtype, h->amp, h->n, h->scratch, nb_norm, unitary_flag,
                          reinterpret_cast<float *>(h->scratch + 2 * nb_norm), h->stream);
            st.kernel_launches += 3;
        }
    }
    st.algorithmic_bytes = sweep * (double)(st.sweeps_block + st.sweeps_permute + st.sweeps_gate);
    h->stats = st;
    SV_API_END
}

sv_status sv_apply_plan_ops(sv_handle h, const sv_gate *gates, int64_t n_gates, sv_plan_h plan, int32_t op_begin,
                            int32_t op_end) {
    SV_API_BEGIN
    if (!h || !plan) fail(SV_ERR_ARG, "null argument");
    if (plan->pinned) fail(SV_ERR_UNSUPPORTED, "sv_apply_plan_ops: plans with gathered chunks are not split into pieces");
    if (plan->n < h->n) fail(SV_ERR_PLAN, "sv_apply_plan_ops: the plan has fewer qubits than the state");
    if (std::min(plan->c, plan->n) > h->n) fail(SV_ERR_PLAN, "sv_apply_plan_ops: the chunk is wider than the state piece");
    if (op_begin < 0 || op_end < op_begin || op_end > (int32_t)plan->ops.size()) fail(SV_ERR_ARG, "op range out of bounds");
    validate_gates(plan->n, gates, n_gates);
    if ((int64_t)plan->keys.size() != n_gates) fail(SV_ERR_PLAN, "plan was made for another gate list");
    for (int64_t i = 0; i < n_gates; ++i) {
        const GateKey k{gates[i].nq, gates[i].q[0], gates[i].nq == 2 ? gates[i].q[1] : -1, gates[i].flags};
        if (!(k == plan->keys[(size_t)i])) fail(SV_ERR_PLAN, "gate " + std::to_string(i) + " differs from the planned list");
    }
    std::vector<unsigned char> host;
    std::vector<BlockProg> progs;
    const int seg_bits = (h->dtype == SV_C64 && plan->seg_bits == 5) ? 5 : 4;
    if (h->dtype == SV_C64) build_programs<float>(plan, gates, seg_bits, host, progs);
    else build_programs<double>(plan, gates, seg_bits, host, progs);
    upload_program(h, host);
    const unsigned char *base = static_cast<const unsigned char *>(h->prog);
    const uint64_t wait_ns = plan->wait_limit_ms > 0 ? (uint64_t)plan->wait_limit_ms * 1000000ull : kDefaultWaitNs;
    size_t bi = 0;  // programs are in op order
    for (int32_t oi = op_begin; oi < op_end; ++oi) {
        const PlanOp &op = plan->ops[(size_t)oi];
        if (op.kind == 2) {
            while (bi < progs.size() && progs[bi].op_index < oi) ++bi;
            if (bi == progs.size() || progs[bi].op_index != oi) fail(SV_ERR_PLAN, "no program for a blocking section");
            const BlockProg &bp = progs[bi];
            launch_block(h->dtype, h->amp, h->n, plan->c, base + bp.off, bp.nseg, bp.ngate, h->dev_err, seg_bits,
                         h->stream, wait_ns);
        } else {
            // pairs inside the piece; the others move data between pieces and are the caller's
            std::vector<std::pair<int32_t, int32_t>> local;
            for (const auto &pq : op.pairs)
                if (pq.first < h->n && pq.second < h->n) local.push_back(pq);
            if (!local.empty()) launch_permute(h->dtype, h->amp, h->n, local, h->stream);
        }
    }
    SV_API_END
}

sv_status sv_shard_pack(sv_handle h, int32_t bit, int32_t value, void *dev_out) {
    SV_API_BEGIN
    if (!h || !dev_out) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    if (bit < 0) {
        check_cuda(cudaMemcpyAsync(dev_out, h->amp, bytes, cudaMemcpyDeviceToDevice, h->stream), "cudaMemcpyAsync(pack)");
    } else {
        if (bit >= h->n || (value != 0 && value != 1)) fail(SV_ERR_ARG, "sv_shard_pack: bit or value out of range");
        launch_shard_half(true, h->dtype, h->amp, h->n, bit, value, dev_out, h->stream);
    }
    SV_API_END
}

sv_status sv_shard_unpack(sv_handle h, int32_t bit, int32_t value, const void *dev_in) {
    SV_API_BEGIN
    if (!h || !dev_in) fail(SV_ERR_ARG, "null argument");
    const size_t bytes = (size_t(1) << h->n) * amp_bytes(h->dtype);
    if (bit < 0) {
        check_cuda(cudaMemcpyAsync(h->amp, dev_in, bytes, cudaMemcpyDeviceToDevice, h->stream), "cudaMemcpyAsync(unpack)");
    } else {
        if (bit >= h->n || (value != 0 && value != 1)) fail(SV_ERR_ARG, "sv_shard_unpack: bit or value out of range");
        launch_shard_half(false, h->dtype, h->amp, h->n, bit, value, const_cast<void *>(dev_in), h->stream);
    }
    SV_API_END
}

sv_status sv_get_apply_stats(sv_handle h, sv_apply_stats *out) {
    SV_API_BEGIN
    if (!h || !out) fail(SV_ERR_ARG, "null argument");
    if (h->profiling && !h->ev_marks.empty() && !h->stats_timed) {
        check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
        double ms[3] = {0, 0, 0};
        for (const auto &km : h->ev_marks) {
            float t = 0;
            check_cuda(cudaEventElapsedTime(&t, h->ev_pool[km.ev], h->ev_pool[km.ev + 1]), "cudaEventElapsedTime");
            ms[km.kind] += t;
        }
        h->stats.ms_gate = ms[0];
        h->stats.ms_block = ms[1];
        h->stats.ms_permute = ms[2];
        h->stats_timed = true;
    }
    *out = h->stats;
    SV_API_END
}

sv_status sv_get_launch_times(sv_handle h, int32_t *kind, int32_t *op_index, float *ms, int64_t max, int64_t *count) {
    SV_API_BEGIN
    if (!h || !count) fail(SV_ERR_ARG, "null argument");
    if (!h->profiling) fail(SV_ERR_ARG, "profiling is off");
    check_cuda(cudaStreamSynchronize(h->stream), "cudaStreamSynchronize");
    *count = (int64_t)h->ev_marks.size();
    for (int64_t k = 0; k < *count && k < max; ++k) {
        const auto &km = h->ev_marks[(size_t)k];
        float t = 0;
        check_cuda(cudaEventElapsedTime(&t, h->ev_pool[km.ev], h->ev_pool[km.ev + 1]), "cudaEventElapsedTime");
        if (kind) kind[k] = km.kind;
        if (op_index) op_index[k] = km.op;
        if (ms) ms[k] = t;
    }
    SV_API_END
}

sv_status sv_probabilities(sv_handle h, double *out, int32_t on_device) {
    SV_API_BEGIN
    if (!h || !out) fail(SV_ERR_ARG, "null argument");
    const int64_t len = int64_t(1) << h->n;
    if (on_device) {
        launch_probs(h->dtype, h->amp, h->n, out, 0, len, h->stream);
        check_dev_error(h);
    } else {
        const int64_t piece = std::min<int64_t>(len, int64_t(1) << 24);
        ensure_scratch(h, (size_t)piece * sizeof(double));
        for (int64_t first = 0; first < len; first += piece) {
            launch_probs(h->dtype, h->amp, h->n, h->scratch, first, piece, h->stream);
            check_cuda(cudaMemcpyAsync(out + first, h->scratch, (size_t)piece * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->stream), "cudaMemcpyAsync(probabilities)");
        }
        check_dev_error(h);
    }
    SV_API_END
}


sv_status sv_norm2(sv_handle h, double *out) {
    SV_API_BEGIN
    if (!h || !out) fail(SV_ERR_ARG, "null argument");
    const int nb = reduce_blocks(h->n);
    ensure_scratch(h, (size_t)nb * sizeof(double));
    launch_partial_norm(h->dtype, h->amp, h->n, h->scratch, nb, h->stream);
    std::vector<double> part((size_t)nb);
    check_cuda(cudaMemcpyAsync(part.data(), h->scratch, nb * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
               "cudaMemcpyAsync(partials)");
    check_dev_error(h);
    double s = 0;
    for (double v : part) s += v;
    *out = s;
    SV_API_END
}

sv_status sv_expval_pauli(sv_handle h, uint64_t x, uint64_t z, double *out) {
    SV_API_BEGIN
    if (!h || !out) fail(SV_ERR_ARG, "null argument");
    if ((x >> h->n) || (z >> h->n)) fail(SV_ERR_ARG, "Pauli mask outside the register");
    const int nb = reduce_blocks(h->n);
    ensure_scratch(h, (size_t)nb * 2 * sizeof(double));
    launch_partial_expval(h->dtype, h->amp, h->n, x, z, h->scratch, nb, h->stream);
    std::vector<double> part((size_t)nb * 2);
    check_cuda(cudaMemcpyAsync(part.data(), h->scratch, nb * 2 * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
               "cudaMemcpyAsync(partials)");
    check_dev_error(h);
    double sr = 0, si = 0;
    for (int b = 0; b < nb; ++b) {
        sr += part[2 * b];
        si += part[2 * b + 1];
    }
    // multiply by i^{popc(x & z)}
    switch (__builtin_popcountll(x & z) & 3) {
        case 1: { double t = sr; sr = -si; si = t; break; }
        case 2: sr = -sr; si = -si; break;
        case 3: { double t = sr; sr = si; si = -t; break; }
        default: break;
    }
    out[0] = sr;
    out[1] = si;
    SV_API_END
}

sv_status sv_sample(sv_handle h, int64_t shots, uint64_t seed, uint64_t *out) {
    SV_API_BEGIN
    if (!h || (shots > 0 && !out)) fail(SV_ERR_ARG, "null argument");
    if (shots < 0) fail(SV_ERR_ARG, "negative shot count");
    if (shots == 0) return SV_OK;
    const int sb = std::min(h->n, 10);
    const int64_t nb = int64_t(1) << (h->n - sb);
    // scratch: range sums, then per-shot (prefix, range, target) and results
    const size_t need = (size_t)nb * sizeof(double) + (size_t)shots * (sizeof(double) * 2 + sizeof(int64_t) + sizeof(uint64_t)) + 1024;
    ensure_scratch(h, need);
    double *sums = h->scratch;
    launch_block_sums(h->dtype, h->amp, h->n, sb, sums, h->stream);
    std::vector<double> incl((size_t)nb);
    check_cuda(cudaMemcpyAsync(incl.data(), sums, nb * sizeof(double), cudaMemcpyDeviceToHost, h->stream),
               "cudaMemcpyAsync(range sums)");
    check_dev_error(h);
    double acc = 0;
    for (int64_t b = 0; b < nb; ++b) {
        acc += incl[(size_t)b];
        incl[(size_t)b] = acc;
    }
    const double total = acc;
    if (!(total > 0)) fail(SV_ERR_ARG, "state has zero norm");
    std::vector<double> prefix((size_t)shots), target((size_t)shots);
    std::vector<int64_t> blk((size_t)shots);
    for (int64_t s = 0; s < shots; ++s) {
        const double t = splitmix_uniform(seed, (uint64_t)s) * total;
        // smallest range whose inclusive prefix exceeds t
        int64_t lo = 0, hi = nb - 1;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (incl[(size_t)mid] > t) hi = mid; else lo = mid + 1;
        }
        blk[(size_t)s] = lo;
        prefix[(size_t)s] = lo > 0 ? incl[(size_t)lo - 1] : 0.0;
        target[(size_t)s] = t;
    }
    unsigned char *p = reinterpret_cast<unsigned char *>(h->scratch) + (((size_t)nb * sizeof(double) + 255) / 256) * 256;
    double *d_prefix = reinterpret_cast<double *>(p);
    double *d_target = d_prefix + shots;
    int64_t *d_blk = reinterpret_cast<int64_t *>(d_target + shots);
    uint64_t *d_out = reinterpret_cast<uint64_t *>(d_blk + shots);
    check_cuda(cudaMemcpyAsync(d_prefix, prefix.data(), shots * sizeof(double), cudaMemcpyHostToDevice, h->stream), "H2D");
    check_cuda(cudaMemcpyAsync(d_target, target.data(), shots * sizeof(double), cudaMemcpyHostToDevice, h->stream), "H2D");
    check_cuda(cudaMemcpyAsync(d_blk, blk.data(), shots * sizeof(int64_t), cudaMemcpyHostToDevice, h->stream), "H2D");
    launch_sample_within(h->dtype, h->amp, h->n, sb, d_prefix, d_blk, d_target, shots, d_out, h->stream);
    check_cuda(cudaMemcpyAsync(out, d_out, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->stream), "D2H");
    check_dev_error(h);
    SV_API_END
}

}  // extern "C"
