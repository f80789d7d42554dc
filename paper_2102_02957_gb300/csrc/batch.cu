// Batched execution (host side) and the autotuner.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>

#include "sv_internal.h"

struct sv_batch {
    int count = 0;
    cudaStream_t stream = nullptr;  // the states' stream
    cudaStream_t work = nullptr;    // the batch's own stream (capturable; joined to `stream`)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int device = 0;
    unsigned char *dev = nullptr;  // one allocation: ops, programs, state pointers, counters
    size_t off_ops = 0, off_progs = 0, off_amps = 0, off_counters = 0, counters_bytes = 0;
    int nops = 0;
    int64_t total = 0;
    double bytes = 0;
    int use_tc = 0;  // 1: tensor-core sections, two pools a CTA; 2: three pools (chunks of <= 12 bits)
    uint64_t wait_ns = sv::kDefaultWaitNs;          // bound of the kernel's waits
    cudaGraph_t graph[2] = {nullptr, nullptr};     // per SV_BATCH_FROM_ZERO value
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    std::vector<std::pair<void *, int>> idle;       // states without gates: (amplitudes, n)
    ~sv_batch() {
        if (work) cudaStreamSynchronize(work);
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
        }
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (work) cudaStreamDestroy(work);
        if (dev) cudaFree(dev);
    }
};

namespace sv {
namespace {

void launch_once(sv_batch *b, int from_zero, int stall = 0) {
    if (from_zero)
        for (const auto &z : b->idle) launch_init_basis(SV_C64, z.first, z.second, 0, b->work);
    unsigned char *c = b->dev + b->off_counters;
    check_cuda(cudaMemsetAsync(c, 0, b->counters_bytes, b->work), "cudaMemsetAsync(batch counters)");
    int *ops_done = reinterpret_cast<int *>(c);
    int *chunks_done = ops_done + b->count;
    unsigned long long *next = reinterpret_cast<unsigned long long *>(c + (((size_t)(b->count + b->nops) * 4 + 15) & ~size_t(15)));
    int *err = reinterpret_cast<int *>(next + 1);
    launch_batch(b->dev + b->off_ops, b->nops, b->dev + b->off_progs,
                 reinterpret_cast<void *const *>(b->dev + b->off_amps), ops_done, chunks_done, next, b->total,
                 from_zero, b->use_tc, err, b->work, b->wait_ns, stall ? 0 : -1);
}

int *batch_err(sv_batch *b) {
    unsigned char *c = b->dev + b->off_counters;
    unsigned long long *next = reinterpret_cast<unsigned long long *>(c + (((size_t)(b->count + b->nops) * 4 + 15) & ~size_t(15)));
    return reinterpret_cast<int *>(next + 1);
}

}  // namespace
}  // namespace sv

using namespace sv;

#define SV_API_BEGIN try {
#define SV_API_END                 \
    return SV_OK;                  \
    }                              \
    catch (const sv::Error &e) {   \
        sv::set_error(e.msg);      \
        return e.code;             \
    }                              \
    catch (const std::bad_alloc &) { \
        sv::set_error("host allocation failed"); \
        return SV_ERR_OOM;         \
    }                              \
    catch (...) {                  \
        sv::set_error("unexpected exception"); \
        return SV_ERR_CUDA;        \
    }

extern "C" {

sv_status sv_batch_create(int32_t count, const sv_handle *states, const sv_gate *const *gates, const int64_t *n_gates,
                          const sv_options *opts, sv_batch_h *out) {
    SV_API_BEGIN
    if (!out || count <= 0 || !states || !gates || !n_gates) fail(SV_ERR_ARG, "sv_batch_create: bad arguments");
    *out = nullptr;
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    std::unique_ptr<sv_batch> b(new sv_batch());
    b->count = count;
    b->stream = states[0]->stream;
    b->device = dev;

    sv_options base;
    if (opts) base = *opts; else sv_options_default(&base);
    if (base.wait_limit_ms < 0) fail(SV_ERR_ARG, "wait_limit_ms must be >= 0");
    if (base.wait_limit_ms > 0) b->wait_ns = (uint64_t)base.wait_limit_ms * 1000000ull;
    std::vector<std::vector<BatchOp>> per_state((size_t)count);
    std::vector<unsigned char> progs;
    // tensor-core sections (complex64 chunks of >= 11 bits): groups fused in FP64 on the GPU
    const bool want_tc = base.use_tc != 0;
    const bool tc3 = want_tc && std::min(std::max(base.chunk_bits, 6), kBatchMaxChunkBits) <= kBatchTc3ChunkBits;
    std::vector<ComposeSeg> compose;
    std::vector<DevGate<double>> compose_gates;
    // per-state planning and program building, spread over host threads (each state into its own
    // buffers, merged in state order below, so the result does not depend on the threading)
    struct StateOut {
        std::vector<BatchOp> ops;
        std::vector<unsigned char> progs;
        std::vector<ComposeSeg> cs;
        std::vector<DevGate<double>> cg;
        bool idle = false;
        double bytes = 0;
        bool failed = false;
        sv_status code = SV_OK;
        std::string msg;
    };
    std::vector<StateOut> outs((size_t)count);
    for (int s = 0; s < count; ++s) {
        const sv_state *h = states[s];
        if (!h) fail(SV_ERR_ARG, "sv_batch_create: null state");
        if (h->dtype != SV_C64) fail(SV_ERR_UNSUPPORTED, "sv_batch_create: batched states are complex64");
        if (h->device != dev) fail(SV_ERR_ARG, "sv_batch_create: state on another device");
        if (h->n < 6) fail(SV_ERR_UNSUPPORTED, "sv_batch_create: states need at least 6 qubits");
        if (h->stream != b->stream) fail(SV_ERR_ARG, "sv_batch_create: all states must use one stream");
    }
    auto build_state = [&](int s, StateOut &out) {
        auto align_out = [&](size_t al) {
            while (out.progs.size() % al) out.progs.push_back(0);
        };
        const sv_state *h = states[s];
        sv_options o = base;
        o.chunk_bits = std::min(std::max(o.chunk_bits, 6), kBatchMaxChunkBits);
        o.gather_pinned = std::min(4, std::min(o.chunk_bits, h->n) - 2);
        o.reserve = 0;
        o.restore_layout = 1;
        o.diag_outside = 0;
        for (int64_t i = 0; i < n_gates[s]; ++i)
            if (gates[s][i].flags & SV_GATE_SWAP)
                fail(SV_ERR_UNSUPPORTED, "sv_batch_create: SWAP relabels are not batched");
        o.seg_bits = 4;
        o.use_tc = 0;  // the planner's own tensor-core rules do not apply to batch sections
        std::unique_ptr<sv_plan> plan(plan_blocking(h->n, gates[s], n_gates[s], o));
        if (plan->ops.empty()) out.idle = true;
        int opno = 0;
        for (const PlanOp &op : plan->ops) {
            if (op.gates.empty()) continue;
            if (op.kind == 1 || op.kind == 3) fail(SV_ERR_UNSUPPORTED, "sv_batch_create: SWAP relabels are not batched");
            // chunk-local order: contiguous low run, then the other chunk bits ascending
            const int n = h->n;
            const uint64_t mask = op.kind == 4 ? op.mask : ((uint64_t(1) << std::min(plan->c, n)) - 1);
            int low = 0;
            while (low < n && ((mask >> low) & 1)) ++low;
            std::vector<int> local_of(n, -1);
            BatchOp bo{};
            bo.state = s;
            bo.low = low;
            int k = 0;
            for (int q = 0; q < n; ++q) {
                if ((mask >> q) & 1) {
                    if (q >= low) bo.high[bo.nhigh++] = (int8_t)q;
                    local_of[q] = k++;
                } else {
                    bo.outer[bo.nouter++] = (int8_t)q;
                }
            }
            bo.ce = k;
            if (low < 4 || k - low > kBatchMaxChunkBits - 4)
                fail(SV_ERR_PLAN, "sv_batch_create: batched chunk without a 4-bit contiguous low run");
            bo.nchunks = int64_t(1) << (n - k);
            std::vector<BlockGate> loc = op.gates;
            for (BlockGate &g : loc)
                for (int j = 0; j < g.nq; ++j) g.phys[j] = local_of[g.phys[j]];
            // a register group with many gates continues in further groups on the same bits
            std::vector<HostSeg> segs;
            for (HostSeg &sg : segment_block(loc, k, 4, 8)) {
                constexpr size_t kMaxGatesPerGroup = 96;
                for (size_t g0 = 0; g0 < std::max<size_t>(sg.gates.size(), 1); g0 += kMaxGatesPerGroup) {
                    HostSeg part = sg;
                    const size_t g1 = std::min(sg.gates.size(), g0 + kMaxGatesPerGroup);
                    part.gates.assign(sg.gates.begin() + (ptrdiff_t)g0, sg.gates.begin() + (ptrdiff_t)g1);
                    segs.push_back(std::move(part));
                }
            }
            // the section's program in pieces of at most kBatchMaxProgBytes, each a 16-byte header
            // {nseg, ngate, bytes, 0} + register groups + gate records (SIMT) or the groups' B
            // operands and unitarity flags (tensor cores); the kernel runs the pieces one after
            // another on the resident chunk
            const bool tc = want_tc && k >= 11;
            align_out(256);
            BatchOp sec = bo;
            sec.op = opno++;
            sec.prog_off = (uint32_t)out.progs.size();
            sec.npiece = 0;
            sec.tc = tc ? 1 : 0;
            size_t p0 = 0;
            while (p0 < segs.size()) {
                size_t p1 = p0, gates_in = 0;
                while (p1 < segs.size()) {
                    const size_t g_next = gates_in + segs[p1].gates.size();
                    const size_t body = tc ? (p1 + 1 - p0) * (size_t)kBatchTcGroupBytes : g_next * sizeof(DevGate<float>);
                    const size_t bytes = 16 + ((p1 + 1 - p0) * sizeof(DevSeg) + 15) / 16 * 16 + body;
                    // SIMT pieces fit every kernel's buffer (a batch whose sections all stay on
                    // SIMT groups runs the SIMT kernel, whose buffer is the smallest)
                    const size_t limit = !tc ? (size_t)kBatchMaxProgBytes
                                         : tc3 ? (size_t)kBatchMaxProgBytesTc3
                                               : (size_t)kBatchMaxProgBytesTc;
                    if (bytes > limit && p1 > p0) break;
                    if (bytes > limit) fail(SV_ERR_UNSUPPORTED, "register group too large");
                    gates_in = g_next;
                    ++p1;
                }
                std::vector<DevSeg> ds;
                std::vector<DevGate<float>> dg;
                for (size_t q = p0; q < p1; ++q) {
                    const HostSeg &hs = segs[q];
                    DevSeg d;
                    std::memset(&d, 0, sizeof(d));
                    d.r = (int8_t)hs.r;
                    for (int t = 0; t < hs.r; ++t) d.pos[t] = (int8_t)hs.pos[t];
                    for (int t = 0; t < 5; ++t) d.lane[t] = (int8_t)hs.lane[t];
                    d.nrest = (int8_t)hs.nrest;
                    for (int t = 0; t < hs.nrest; ++t) d.rest[t] = (int8_t)hs.rest[t];
                    // the chunk arrives and leaves in the natural layout
                    d.flags = (int8_t)((q == 0 ? 1 : 0) | (q + 1 == segs.size() ? 2 : 0));
                    d.g0 = (int16_t)dg.size();
                    if (!tc) {
                        for (int32_t gi : hs.gates) {
                            DevGate<float> g;
                            encode_gate<float>(gates[s][loc[gi].gi], loc[gi], hs, g);
                            dg.push_back(g);
                        }
                    }
                    d.g1 = (int16_t)dg.size();
                    ds.push_back(d);
                }
                const size_t at = out.progs.size();
                out.progs.resize(at + 16, 0);
                const unsigned char *p = reinterpret_cast<const unsigned char *>(ds.data());
                out.progs.insert(out.progs.end(), p, p + ds.size() * sizeof(DevSeg));
                align_out(16);
                if (tc) {
                    for (size_t q = p0; q < p1; ++q) {  // B operands, written by the compose kernel
                        ComposeSeg cs{};
                        cs.b_off = (uint32_t)out.progs.size();
                        cs.flag_off = cs.b_off + TC_B_BYTES;
                        cs.g0 = (int32_t)out.cg.size();
                        for (int32_t gi : segs[q].gates) {
                            DevGate<double> g;
                            encode_gate<double>(gates[s][loc[gi].gi], loc[gi], segs[q], g);
                            out.cg.push_back(g);
                        }
                        cs.g1 = (int32_t)out.cg.size();
                        out.cs.push_back(cs);
                        out.progs.resize(out.progs.size() + kBatchTcGroupBytes, 0);
                    }
                } else {
                    p = reinterpret_cast<const unsigned char *>(dg.data());
                    out.progs.insert(out.progs.end(), p, p + dg.size() * sizeof(DevGate<float>));
                }
                align_out(16);
                const int32_t hd[4] = {(int32_t)ds.size(), (int32_t)dg.size(), (int32_t)(out.progs.size() - at), 0};
                std::memcpy(out.progs.data() + at, hd, sizeof(hd));
                ++sec.npiece;
                p0 = p1;
            }
            sec.prog_bytes = (uint32_t)(out.progs.size() - sec.prog_off);
            if (sec.npiece == 0) continue;
            out.bytes += 2.0 * 8.0 * std::ldexp(1.0, n);
            out.ops.push_back(sec);
        }
    
    };
    {
        const unsigned hw = std::thread::hardware_concurrency();
        const int nth = (int)std::max(1u, std::min(16u, std::min(hw ? hw : 1u, (unsigned)count)));
        auto work = [&](int t) {
            for (int s = t; s < count; s += nth) {
                try {
                    build_state(s, outs[(size_t)s]);
                } catch (const Error &e) {
                    outs[(size_t)s].failed = true;
                    outs[(size_t)s].code = e.code;
                    outs[(size_t)s].msg = e.msg;
                } catch (const std::bad_alloc &) {
                    outs[(size_t)s].failed = true;
                    outs[(size_t)s].code = SV_ERR_OOM;
                    outs[(size_t)s].msg = "host allocation failed";
                }
            }
        };
        std::vector<std::thread> pool;
        for (int t = 1; t < nth; ++t) pool.emplace_back(work, t);
        work(0);
        for (std::thread &th : pool) th.join();
    }
    // merge in state order
    auto align = [&](size_t al) {
        while (progs.size() % al) progs.push_back(0);
    };
    for (int s = 0; s < count; ++s) {
        StateOut &out = outs[(size_t)s];
        if (out.failed) fail(out.code, out.msg);
        if (out.idle) b->idle.emplace_back(states[s]->amp, states[s]->n);
        b->bytes += out.bytes;
        align(256);
        const uint32_t base_off = (uint32_t)progs.size();
        const int32_t gate_base = (int32_t)compose_gates.size();
        progs.insert(progs.end(), out.progs.begin(), out.progs.end());
        for (BatchOp &o : out.ops) {
            o.prog_off += base_off;
            per_state[(size_t)s].push_back(o);
        }
        for (ComposeSeg cs : out.cs) {
            cs.b_off += base_off;
            cs.flag_off += base_off;
            cs.g0 += gate_base;
            cs.g1 += gate_base;
            compose.push_back(cs);
        }
        compose_gates.insert(compose_gates.end(), out.cg.begin(), out.cg.end());
    }
    // queue order: section level by section level, round-robin over the states
    std::vector<BatchOp> ops;
    size_t level = 0;
    bool any = true;
    int64_t total = 0;
    while (any) {
        any = false;
        for (int s = 0; s < count; ++s) {
            if (level < per_state[(size_t)s].size()) {
                BatchOp o = per_state[(size_t)s][level];
                o.first = total;
                total += o.nchunks;
                ops.push_back(o);
                any = true;
            }
        }
        ++level;
    }
    b->nops = (int)ops.size();
    b->total = total;
    // device layout
    size_t off = 0;
    auto place = [&](size_t bytes) {
        off = (off + 255) & ~size_t(255);
        const size_t at = off;
        off += bytes;
        return at;
    };
    b->off_ops = place(ops.size() * sizeof(BatchOp));
    b->off_progs = place(progs.size());
    b->off_amps = place((size_t)count * sizeof(void *));
    b->counters_bytes = (((size_t)(count + b->nops) * 4 + 15) & ~size_t(15)) + 16;
    b->off_counters = place(b->counters_bytes);
    check_cuda(cudaMalloc(&b->dev, off), "cudaMalloc(batch)");
    check_cuda(cudaStreamCreateWithFlags(&b->work, cudaStreamNonBlocking), "cudaStreamCreate(batch)");
    check_cuda(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming), "cudaEventCreate(batch)");
    check_cuda(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming), "cudaEventCreate(batch)");
    std::vector<void *> amps((size_t)count);
    for (int s = 0; s < count; ++s) amps[(size_t)s] = states[s]->amp;
    check_cuda(cudaMemcpy(b->dev + b->off_ops, ops.data(), ops.size() * sizeof(BatchOp), cudaMemcpyHostToDevice), "H2D");
    if (!progs.empty())
        check_cuda(cudaMemcpy(b->dev + b->off_progs, progs.data(), progs.size(), cudaMemcpyHostToDevice), "H2D");
    check_cuda(cudaMemcpy(b->dev + b->off_amps, amps.data(), amps.size() * sizeof(void *), cudaMemcpyHostToDevice), "H2D");
    if (!compose.empty()) {  // fuse every tensor-core group into its B operand, once per batch
        unsigned char *tmp = nullptr;
        const size_t cs_bytes = compose.size() * sizeof(ComposeSeg);
        const size_t g_bytes = compose_gates.size() * sizeof(DevGate<double>);
        check_cuda(cudaMalloc(&tmp, cs_bytes + g_bytes + 256), "cudaMalloc(compose)");
        check_cuda(cudaMemcpy(tmp, compose.data(), cs_bytes, cudaMemcpyHostToDevice), "H2D");
        unsigned char *gdev = tmp + ((cs_bytes + 255) & ~size_t(255));
        if (g_bytes) check_cuda(cudaMemcpy(gdev, compose_gates.data(), g_bytes, cudaMemcpyHostToDevice), "H2D");
        try {
            launch_compose(tmp, (int)compose.size(), gdev, b->dev + b->off_progs, nullptr, 4, b->work);
            check_cuda(cudaStreamSynchronize(b->work), "cudaStreamSynchronize");
        } catch (...) {
            cudaFree(tmp);
            throw;
        }
        cudaFree(tmp);
        b->use_tc = tc3 ? 2 : 1;
    }
    *out = b.release();
    SV_API_END
}

sv_status sv_batch_run(sv_batch_h b, int32_t flags) {
    SV_API_BEGIN
    if (!b) fail(SV_ERR_ARG, "null batch");
    if (flags & ~(SV_BATCH_GRAPH | SV_BATCH_FROM_ZERO | SV_BATCH_TEST_STALL))
        fail(SV_ERR_ARG, "sv_batch_run: unknown flag");
    const int use_graph = flags & SV_BATCH_GRAPH, fz = (flags & SV_BATCH_FROM_ZERO) ? 1 : 0;
    const int stall = (flags & SV_BATCH_TEST_STALL) ? 1 : 0;
    if (stall && use_graph) fail(SV_ERR_ARG, "sv_batch_run: SV_BATCH_TEST_STALL is not combinable with SV_BATCH_GRAPH");
    // the batch's stream follows the states' stream, and the states' stream follows the batch
    check_cuda(cudaEventRecord(b->ev_in, b->stream), "cudaEventRecord");
    check_cuda(cudaStreamWaitEvent(b->work, b->ev_in, 0), "cudaStreamWaitEvent");
    if (!use_graph) {
        launch_once(b, fz, stall);
    } else {
        if (!b->exec[fz]) {
            check_cuda(cudaStreamBeginCapture(b->work, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
            try {
                launch_once(b, fz);
            } catch (...) {
                cudaGraph_t g = nullptr;
                cudaStreamEndCapture(b->work, &g);
                if (g) cudaGraphDestroy(g);
                throw;
            }
            check_cuda(cudaStreamEndCapture(b->work, &b->graph[fz]), "cudaStreamEndCapture");
            check_cuda(cudaGraphInstantiate(&b->exec[fz], b->graph[fz], 0), "cudaGraphInstantiate");
        }
        check_cuda(cudaGraphLaunch(b->exec[fz], b->work), "cudaGraphLaunch");
    }
    check_cuda(cudaEventRecord(b->ev_out, b->work), "cudaEventRecord");
    check_cuda(cudaStreamWaitEvent(b->stream, b->ev_out, 0), "cudaStreamWaitEvent");
    SV_API_END
}

sv_status sv_batch_sync(sv_batch_h b) {
    SV_API_BEGIN
    if (!b) fail(SV_ERR_ARG, "null batch");
    int e = 0;
    check_cuda(cudaMemcpyAsync(&e, batch_err(b), sizeof(int), cudaMemcpyDeviceToHost, b->work), "read error word");
    check_cuda(cudaStreamSynchronize(b->work), "cudaStreamSynchronize");
    if (e == DEV_ERR_TIMEOUT) fail(SV_ERR_TIMEOUT, "a bounded device wait in the batch expired");
    if (e != DEV_OK) fail(SV_ERR_CUDA, "batch error word set");
    SV_API_END
}

sv_status sv_batch_info(sv_batch_h b, int64_t *items, int32_t *sections, double *bytes_per_run) {
    SV_API_BEGIN
    if (!b) fail(SV_ERR_ARG, "null batch");
    if (items) *items = b->total;
    if (sections) *sections = b->nops;
    if (bytes_per_run) *bytes_per_run = b->bytes;
    SV_API_END
}

sv_status sv_batch_tune(int32_t count, const sv_handle *states, const sv_gate *const *gates, const int64_t *n_gates,
                        const sv_options *base, sv_options *best, double *best_ms) {
    SV_API_BEGIN
    if (!best || !states || count <= 0) fail(SV_ERR_ARG, "sv_batch_tune: bad arguments");
    sv_options b0;
    if (base) b0 = *base; else sv_options_default(&b0);
    cudaStream_t st = states[0]->stream;
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    double best_t = 1e300;
    sv_options best_o = b0;
    sv_status last = SV_OK;
    for (int c = 10; c <= kBatchMaxChunkBits; ++c) {
        sv_options o = b0;
        o.chunk_bits = c;
        sv_batch_h bt = nullptr;
        last = sv_batch_create(count, states, gates, n_gates, &o, &bt);
        if (last != SV_OK) continue;
        float ms = -1.f;
        if ((last = sv_batch_run(bt, SV_BATCH_FROM_ZERO)) == SV_OK && (last = sv_batch_sync(bt)) == SV_OK) {
            cudaEventRecord(e0, st);
            last = sv_batch_run(bt, SV_BATCH_FROM_ZERO);
            cudaEventRecord(e1, st);
            if (last == SV_OK && (last = sv_batch_sync(bt)) == SV_OK && cudaEventSynchronize(e1) == cudaSuccess)
                cudaEventElapsedTime(&ms, e0, e1);
        }
        sv_batch_free(bt);
        if (ms >= 0.f && ms < best_t) {
            best_t = ms;
            best_o = o;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_t >= 1e300) return last != SV_OK ? last : SV_ERR_UNSUPPORTED;
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    SV_API_END
}

sv_status sv_batch_free(sv_batch_h b) {
    SV_API_BEGIN
    delete b;
    SV_API_END
}

sv_status sv_autotune(int32_t n, int32_t dtype, const sv_gate *gates, int64_t n_gates, const sv_options *base,
                      sv_options *best, double *best_ms) {
    SV_API_BEGIN
    if (!best || (!gates && n_gates)) fail(SV_ERR_ARG, "sv_autotune: null argument");
    sv_options b0;
    if (base) b0 = *base; else sv_options_default(&b0);
    sv_handle h = nullptr;
    sv_status st = sv_create(n, dtype, nullptr, 0, nullptr, &h);
    if (st != SV_OK) return st;
    cudaEvent_t e0, e1;
    check_cuda(cudaEventCreate(&e0), "cudaEventCreate");
    check_cuda(cudaEventCreate(&e1), "cudaEventCreate");
    double best_t = 1e300;
    sv_options best_o = b0;
    const int cmax = std::min(n, 13);
    try {
        for (int c = std::max(std::min(n, 11), std::min(cmax, 6)); c <= cmax; ++c)
            for (int seg : {4, 5})
                for (int pin : {0, 4})
                    for (int tc : {0, 1})
                        for (int la : {0, 1}) {
                        if (dtype != SV_C64 && (seg == 5 || tc)) continue;
                        if (tc && seg != 4) continue;
                        if (pin && c - pin < 2) continue;
                        if (la && !pin) continue;  // look-ahead chunk choice: gathered chunks only
                        sv_options o = b0;
                        o.chunk_bits = c;
                        o.seg_bits = seg;
                        o.gather_pinned = pin;
                        o.use_tc = tc;
                        o.lookahead = la;
                        sv_plan_h p = nullptr;
                        if (sv_plan_blocking(n, gates, n_gates, &o, &p) != SV_OK) continue;
                        double ms = 1e300;
                        if (sv_init_basis(h, 0) == SV_OK && sv_apply_circuit(h, gates, n_gates, p) == SV_OK &&
                            sv_synchronize(h) == SV_OK) {
                            check_cuda(cudaEventRecord(e0, h->stream), "cudaEventRecord");
                            const sv_status a = sv_apply_circuit(h, gates, n_gates, p);
                            check_cuda(cudaEventRecord(e1, h->stream), "cudaEventRecord");
                            if (a == SV_OK && sv_synchronize(h) == SV_OK) {
                                float t = 0;
                                check_cuda(cudaEventElapsedTime(&t, e0, e1), "cudaEventElapsedTime");
                                ms = t;
                            }
                        }
                        sv_plan_free(p);
                        if (ms < best_t) {
                            best_t = ms;
                            best_o = o;
                        }
                    }
    } catch (...) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        sv_destroy(h);
        throw;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    sv_destroy(h);
    if (best_t >= 1e300) fail(SV_ERR_UNSUPPORTED, "sv_autotune: no candidate ran");
    *best = best_o;
    if (best_ms) *best_ms = best_t;
    SV_API_END
}

}  // extern "C"
