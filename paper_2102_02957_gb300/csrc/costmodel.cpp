// Learned cost model of blocking sections: sample collection (per-launch CUDA-event timings of
// the library's own sections), training and inference on the GPU (k_mlp.cu), and the steered
// planner entry point.  The paper has no counterpart: its transpiler rule (Sec. IV.A) stays
// the first candidate of every section and the default planner.
#include <cmath>
#include <cstring>
#include <numeric>

#include "sv_internal.h"

struct sv_costmodel {
    int device = 0;
    cudaStream_t stream = nullptr;
    float *params = nullptr, *mom1 = nullptr, *mom2 = nullptr;  // device, NPARAM each
    int64_t step = 0;
    std::vector<float> xs, us;  // samples: features (rows x 16) and measured microseconds
    double t_mean = 0.0, t_std = 1.0;
    bool trained = false;
    // device scratch, grown on demand
    unsigned char *scratch = nullptr;
    size_t scratch_bytes = 0;
    ~sv_costmodel() {
        if (stream) cudaStreamSynchronize(stream);
        if (params) cudaFree(params);
        if (mom1) cudaFree(mom1);
        if (mom2) cudaFree(mom2);
        if (scratch) cudaFree(scratch);
        if (stream) cudaStreamDestroy(stream);
    }
};

namespace sv {
namespace {

constexpr int NF = kNumFeatures;

uint64_t splitmix_next(uint64_t &state) {
    uint64_t z = (state += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
double splitmix_unit(uint64_t &state) { return (double)(splitmix_next(state) >> 11) * 0x1.0p-53; }

// Device scratch of the model: x (rows x 16), t (rows), idx (rows), y (rows), partial gradients,
// loss partials, loss.
struct Scratch {
    float *x, *t, *y, *part, *grad;
    int32_t *idx;
    double *lpart, *loss;
};

Scratch scratch_for(sv_costmodel *m, int64_t rows) {
    const int P = mlp_param_count();
    const int nblk = 128;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t need = al(rows * NF * 4) + 3 * al(rows * 4) + al(rows * 4) + al((size_t)nblk * P * 4) + al(P * 4) +
                        al(nblk * 8) + al(8);
    if (need > m->scratch_bytes) {
        if (m->scratch) check_cuda(cudaFree(m->scratch), "cudaFree");
        m->scratch = nullptr;
        m->scratch_bytes = 0;
        check_cuda(cudaMalloc(&m->scratch, need), "cudaMalloc(cost model scratch)");
        m->scratch_bytes = need;
    }
    unsigned char *p = m->scratch;
    Scratch s;
    s.x = reinterpret_cast<float *>(p); p += al(rows * NF * 4);
    s.t = reinterpret_cast<float *>(p); p += al(rows * 4);
    s.y = reinterpret_cast<float *>(p); p += al(rows * 4);
    s.idx = reinterpret_cast<int32_t *>(p); p += al(rows * 4);
    p += al(rows * 4);
    s.part = reinterpret_cast<float *>(p); p += al((size_t)nblk * P * 4);
    s.grad = reinterpret_cast<float *>(p); p += al(P * 4);
    s.lpart = reinterpret_cast<double *>(p); p += al(nblk * 8);
    s.loss = reinterpret_cast<double *>(p);
    return s;
}

void check_model(sv_costmodel *m) {
    if (!m) fail(SV_ERR_ARG, "null cost model");
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev != m->device) fail(SV_ERR_ARG, "cost model belongs to another device");
}

void forward_raw(sv_costmodel *m, const float *x, int64_t count, float *y) {
    if (count <= 0) return;
    Scratch s = scratch_for(m, count);
    check_cuda(cudaMemcpyAsync(s.x, x, count * NF * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
    launch_mlp_fwd(m->params, s.x, count, s.y, m->stream);
    check_cuda(cudaMemcpyAsync(y, s.y, count * 4, cudaMemcpyDeviceToHost, m->stream), "D2H");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
}

// One gradient (mode 0) or Adam step (mode 1) over rows [start, start + B) of the uploaded
// batch, in the order of idx (or natural when idx is null).
void grad_or_step(sv_costmodel *m, const Scratch &s, const int32_t *idx, int64_t start, int64_t B, int mode, float lr) {
    launch_mlp_grad(m->params, s.x, s.t, idx, start, B, s.part, s.lpart, m->stream);
    float c1 = 1.f, c2 = 1.f;
    if (mode == 1) {
        ++m->step;
        c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)m->step)));
        c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)m->step)));
    }
    launch_mlp_reduce(s.part, mlp_grad_blocks(B), s.lpart, s.loss, mode, s.grad, m->params, m->mom1, m->mom2, lr, c1,
                      c2, m->stream);
}

std::vector<float> predict_us(sv_costmodel *m, const float *x, int64_t count) {
    std::vector<float> y((size_t)count);
    forward_raw(m, x, count, y.data());
    for (float &v : y) v = (float)std::exp((double)v * m->t_std + m->t_mean);
    return y;
}

struct RandomChooser : SectionChooser {
    uint64_t state;
    explicit RandomChooser(uint64_t seed) : state(seed) {}
    int choose(const std::vector<SectionCandidate> &c) override {
        return (int)(splitmix_unit(state) * (double)c.size());
    }
};

// Most gates per predicted microsecond; the paper's rule (candidate 0) wins ties.  The planner
// asks once or twice per section, so the network is evaluated on the host from a copy of its
// parameters taken when the chooser is made (16 -> 64 -> 64 -> 1, the layout of k_mlp.cu), not
// by a kernel launch and a synchronisation per question.
struct ModelChooser : SectionChooser {
    sv_costmodel *m;
    std::vector<float> P;
    explicit ModelChooser(sv_costmodel *mm) : m(mm), P((size_t)mlp_param_count()) {
        check_cuda(cudaMemcpyAsync(P.data(), m->params, P.size() * sizeof(float), cudaMemcpyDeviceToHost, m->stream),
                   "D2H(cost model)");
        check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    }
    double predict_us_host(const float *x) const {
        constexpr int NIN = NF, NH = 64;
        const float *W1 = P.data(), *b1 = W1 + NH * NIN, *W2 = b1 + NH, *b2 = W2 + NH * NH, *w3 = b2 + NH;
        const float b3 = w3[NH];
        float h1[NH], h2[NH];
        for (int u = 0; u < NH; ++u) {
            float a = b1[u];
            for (int f = 0; f < NIN; ++f) a += W1[u * NIN + f] * x[f];
            h1[u] = a > 0.f ? a : 0.f;
        }
        float y = b3;
        for (int u = 0; u < NH; ++u) {
            float a = b2[u];
            for (int f = 0; f < NH; ++f) a += W2[u * NH + f] * h1[f];
            h2[u] = a > 0.f ? a : 0.f;
            y += w3[u] * h2[u];
        }
        return std::exp((double)y * m->t_std + m->t_mean);
    }
    int choose(const std::vector<SectionCandidate> &c) override {
        if (c.size() <= 1) return 0;
        std::vector<double> us(c.size());
        for (size_t k = 0; k < c.size(); ++k) us[k] = predict_us_host(c[k].f);
        int best = 0;
        double best_rate = (double)c[0].absorbed / std::max(1e-3, (double)us[0]);
        for (size_t k = 1; k < c.size(); ++k) {
            const double rate = (double)c[k].absorbed / std::max(1e-3, (double)us[k]);
            if (rate > best_rate * (1.0 + 1e-6)) {
                best_rate = rate;
                best = (int)k;
            }
        }
        return best;
    }
};

}  // namespace
}  // namespace sv

using namespace sv;

#define SV_API_BEGIN try {
#define SV_API_END                               \
    return SV_OK;                                \
    }                                            \
    catch (const sv::Error &e) {                 \
        sv::set_error(e.msg);                    \
        return e.code;                           \
    }                                            \
    catch (const std::bad_alloc &) {             \
        sv::set_error("host allocation failed"); \
        return SV_ERR_OOM;                       \
    }                                            \
    catch (...) {                                \
        sv::set_error("unexpected exception");   \
        return SV_ERR_CUDA;                      \
    }

extern "C" {

sv_status sv_costmodel_create(uint64_t seed, sv_costmodel_h *out) {
    SV_API_BEGIN
    if (!out) fail(SV_ERR_ARG, "null output");
    *out = nullptr;
    std::unique_ptr<sv_costmodel> m(new sv_costmodel());
    check_cuda(cudaGetDevice(&m->device), "cudaGetDevice");
    check_cuda(cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking), "cudaStreamCreate");
    const int P = mlp_param_count();
    check_cuda(cudaMalloc(&m->params, P * 4), "cudaMalloc");
    check_cuda(cudaMalloc(&m->mom1, P * 4), "cudaMalloc");
    check_cuda(cudaMalloc(&m->mom2, P * 4), "cudaMalloc");
    std::vector<float> h((size_t)P, 0.f);
    uint64_t st = seed;
    auto fill = [&](int off, int count, int fan_in) {
        const double a = std::sqrt(6.0 / fan_in);
        for (int k = 0; k < count; ++k) h[(size_t)(off + k)] = (float)((2.0 * splitmix_unit(st) - 1.0) * a);
    };
    fill(0, 64 * 16, 16);                 // W1
    fill(64 * 16 + 64, 64 * 64, 64);      // W2
    fill(64 * 16 + 64 + 64 * 64 + 64, 64, 64);  // w3
    check_cuda(cudaMemcpy(m->params, h.data(), P * 4, cudaMemcpyHostToDevice), "H2D");
    check_cuda(cudaMemset(m->mom1, 0, P * 4), "cudaMemset");
    check_cuda(cudaMemset(m->mom2, 0, P * 4), "cudaMemset");
    *out = m.release();
    SV_API_END
}

sv_status sv_costmodel_free(sv_costmodel_h m) {
    SV_API_BEGIN
    delete m;
    SV_API_END
}

sv_status sv_costmodel_get_params(sv_costmodel_h m, float *out, int64_t count) {
    SV_API_BEGIN
    check_model(m);
    if (!out || count != mlp_param_count()) fail(SV_ERR_ARG, "parameter count mismatch");
    check_cuda(cudaMemcpyAsync(out, m->params, count * 4, cudaMemcpyDeviceToHost, m->stream), "D2H");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    SV_API_END
}

sv_status sv_costmodel_set_params(sv_costmodel_h m, const float *in, int64_t count) {
    SV_API_BEGIN
    check_model(m);
    if (!in || count != mlp_param_count()) fail(SV_ERR_ARG, "parameter count mismatch");
    check_cuda(cudaMemcpyAsync(m->params, in, count * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
    check_cuda(cudaMemsetAsync(m->mom1, 0, count * 4, m->stream), "cudaMemset");
    check_cuda(cudaMemsetAsync(m->mom2, 0, count * 4, m->stream), "cudaMemset");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    m->step = 0;
    SV_API_END
}

sv_status sv_costmodel_forward(sv_costmodel_h m, const float *x, int64_t count, float *y) {
    SV_API_BEGIN
    check_model(m);
    if (count < 0 || (count && (!x || !y))) fail(SV_ERR_ARG, "bad arguments");
    forward_raw(m, x, count, y);
    SV_API_END
}

static void upload_batch(sv_costmodel *m, const Scratch &s, const float *x, const float *t, int64_t count) {
    check_cuda(cudaMemcpyAsync(s.x, x, count * NF * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
    check_cuda(cudaMemcpyAsync(s.t, t, count * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
}

sv_status sv_costmodel_gradient(sv_costmodel_h m, const float *x, const float *t, int64_t count, float *grad,
                                double *loss) {
    SV_API_BEGIN
    check_model(m);
    if (count <= 0 || !x || !t || !grad) fail(SV_ERR_ARG, "bad arguments");
    Scratch s = scratch_for(m, count);
    upload_batch(m, s, x, t, count);
    grad_or_step(m, s, nullptr, 0, count, 0, 0.f);
    check_cuda(cudaMemcpyAsync(grad, s.grad, mlp_param_count() * 4, cudaMemcpyDeviceToHost, m->stream), "D2H");
    double l = 0;
    check_cuda(cudaMemcpyAsync(&l, s.loss, 8, cudaMemcpyDeviceToHost, m->stream), "D2H");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    if (loss) *loss = l;
    SV_API_END
}

sv_status sv_costmodel_adam_step(sv_costmodel_h m, const float *x, const float *t, int64_t count, float lr,
                                 double *loss) {
    SV_API_BEGIN
    check_model(m);
    if (count <= 0 || !x || !t) fail(SV_ERR_ARG, "bad arguments");
    Scratch s = scratch_for(m, count);
    upload_batch(m, s, x, t, count);
    grad_or_step(m, s, nullptr, 0, count, 1, lr);
    double l = 0;
    check_cuda(cudaMemcpyAsync(&l, s.loss, 8, cudaMemcpyDeviceToHost, m->stream), "D2H");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    if (loss) *loss = l;
    SV_API_END
}

sv_status sv_costmodel_add_samples(sv_costmodel_h m, const float *x, const float *us, int64_t count) {
    SV_API_BEGIN
    if (!m || count < 0 || (count && (!x || !us))) fail(SV_ERR_ARG, "bad arguments");
    for (int64_t k = 0; k < count; ++k)
        if (!(us[k] > 0.f)) fail(SV_ERR_ARG, "sample times must be positive");
    m->xs.insert(m->xs.end(), x, x + count * NF);
    m->us.insert(m->us.end(), us, us + count);
    SV_API_END
}

sv_status sv_costmodel_num_samples(sv_costmodel_h m, int64_t *count) {
    SV_API_BEGIN
    if (!m || !count) fail(SV_ERR_ARG, "null argument");
    *count = (int64_t)m->us.size();
    SV_API_END
}

sv_status sv_costmodel_collect(sv_costmodel_h m, sv_handle h, const sv_gate *gates, int64_t n_gates,
                               const sv_options *opts, int32_t n_opts, uint64_t policy_seed, int64_t *added) {
    SV_API_BEGIN
    check_model(m);
    if (!h || !opts || n_opts <= 0) fail(SV_ERR_ARG, "bad arguments");
    int64_t count = 0;
    int32_t was_profiling = h->profiling ? 1 : 0;
    sv_set_profiling(h, 1);
    try {
        for (int k = 0; k < n_opts; ++k) {
            std::unique_ptr<RandomChooser> rc;
            if (policy_seed) rc.reset(new RandomChooser(policy_seed + (uint64_t)k));
            std::unique_ptr<sv_plan> plan(plan_blocking(h->n, gates, n_gates, opts[k], rc.get(), h->dtype));
            for (int rep = 0; rep < 2; ++rep) {
                sv_status st = sv_init_basis(h, 0);
                if (st == SV_OK) st = sv_apply_circuit(h, gates, n_gates, plan.get());
                if (st != SV_OK) fail(st, std::string("collect: ") + sv_last_error());
            }
            int64_t nl = 0;
            if (sv_get_launch_times(h, nullptr, nullptr, nullptr, 0, &nl) != SV_OK) fail(SV_ERR_CUDA, sv_last_error());
            std::vector<int32_t> kind((size_t)nl), opi((size_t)nl);
            std::vector<float> ms((size_t)nl);
            if (sv_get_launch_times(h, kind.data(), opi.data(), ms.data(), nl, &nl) != SV_OK)
                fail(SV_ERR_CUDA, sv_last_error());
            std::vector<double> op_ms(plan->ops.size(), 0.0);
            for (int64_t l = 0; l < nl; ++l)
                if (kind[(size_t)l] == 1 && opi[(size_t)l] >= 0) op_ms[(size_t)opi[(size_t)l]] += ms[(size_t)l];
            for (size_t oi = 0; oi < plan->ops.size(); ++oi) {
                const PlanOp &op = plan->ops[oi];
                if ((op.kind != 2 && op.kind != 4) || op.gates.empty() || op_ms[oi] <= 0.0) continue;
                float f[NF];
                section_features(*plan, op, gates, h->dtype, f);
                m->xs.insert(m->xs.end(), f, f + NF);
                m->us.push_back((float)(op_ms[oi] * 1000.0));
                ++count;
            }
        }
    } catch (...) {
        sv_set_profiling(h, was_profiling);
        throw;
    }
    sv_set_profiling(h, was_profiling);
    if (added) *added = count;
    SV_API_END
}

sv_status sv_costmodel_train(sv_costmodel_h m, int32_t epochs, int32_t batch, float lr, uint64_t seed, double *mse) {
    SV_API_BEGIN
    check_model(m);
    const int64_t N = (int64_t)m->us.size();
    if (N < 2) fail(SV_ERR_ARG, "sv_costmodel_train: fewer than two samples");
    if (epochs < 0 || batch < 1 || !(lr > 0.f)) fail(SV_ERR_ARG, "bad training arguments");
    // standardised log-microseconds
    std::vector<float> t((size_t)N);
    double mean = 0.0, var = 0.0;
    for (int64_t k = 0; k < N; ++k) mean += std::log((double)m->us[(size_t)k]);
    mean /= (double)N;
    for (int64_t k = 0; k < N; ++k) {
        const double d = std::log((double)m->us[(size_t)k]) - mean;
        var += d * d;
    }
    const double sd = std::max(1e-6, std::sqrt(var / (double)N));
    for (int64_t k = 0; k < N; ++k) t[(size_t)k] = (float)((std::log((double)m->us[(size_t)k]) - mean) / sd);
    m->t_mean = mean;
    m->t_std = sd;
    Scratch s = scratch_for(m, N);
    upload_batch(m, s, m->xs.data(), t.data(), N);
    std::vector<int32_t> perm((size_t)N);
    std::iota(perm.begin(), perm.end(), 0);
    uint64_t st = seed;
    for (int e = 0; e < epochs; ++e) {
        for (int64_t k = N - 1; k > 0; --k) {  // Fisher-Yates
            const int64_t j = (int64_t)(splitmix_unit(st) * (double)(k + 1));
            std::swap(perm[(size_t)k], perm[(size_t)j]);
        }
        check_cuda(cudaMemcpyAsync(s.idx, perm.data(), N * 4, cudaMemcpyHostToDevice, m->stream), "H2D");
        for (int64_t b0 = 0; b0 < N; b0 += batch)
            grad_or_step(m, s, s.idx, b0, std::min<int64_t>(batch, N - b0), 1, lr);
        // the index buffer is rewritten next epoch: keep the host copy alive until used
        check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    }
    grad_or_step(m, s, nullptr, 0, N, 0, 0.f);  // loss over all samples at the final parameters
    double l = 0;
    check_cuda(cudaMemcpyAsync(&l, s.loss, 8, cudaMemcpyDeviceToHost, m->stream), "D2H");
    check_cuda(cudaStreamSynchronize(m->stream), "cudaStreamSynchronize");
    m->trained = true;
    if (mse) *mse = l * sd * sd;
    SV_API_END
}

sv_status sv_costmodel_predict_us(sv_costmodel_h m, const float *x, int64_t count, float *us) {
    SV_API_BEGIN
    check_model(m);
    if (count < 0 || (count && (!x || !us))) fail(SV_ERR_ARG, "bad arguments");
    const std::vector<float> y = predict_us(m, x, count);
    std::memcpy(us, y.data(), y.size() * 4);
    SV_API_END
}

sv_status sv_costmodel_features(sv_plan_h plan, const sv_gate *gates, int32_t dtype, float *out, int64_t max_rows,
                                int64_t *rows) {
    SV_API_BEGIN
    if (!plan || !rows || (dtype != SV_C64 && dtype != SV_C128)) fail(SV_ERR_ARG, "bad arguments");
    if ((int64_t)plan->keys.size() > 0 && !gates) fail(SV_ERR_ARG, "null gate list");
    int64_t r = 0;
    for (const PlanOp &op : plan->ops) {
        if (op.kind != 2 && op.kind != 4) continue;
        if (out && r < max_rows) section_features(*plan, op, gates, dtype, out + r * NF);
        ++r;
    }
    *rows = r;
    SV_API_END
}

sv_status sv_plan_blocking_steered(int32_t n, const sv_gate *gates, int64_t n_gates, const sv_options *opts,
                                   int32_t dtype, sv_costmodel_h model, sv_plan_h *out) {
    SV_API_BEGIN
    if (!out || !opts) fail(SV_ERR_ARG, "null argument");
    *out = nullptr;
    check_model(model);
    if (!model->trained) fail(SV_ERR_ARG, "sv_plan_blocking_steered: the cost model is not trained");
    if (opts->gather_pinned <= 0) fail(SV_ERR_ARG, "sv_plan_blocking_steered: needs gathered chunks (gather_pinned > 0)");
    if (dtype != SV_C64 && dtype != SV_C128) fail(SV_ERR_ARG, "bad dtype");
    ModelChooser ch(model);
    sv_plan *p = plan_blocking(n, gates, n_gates, *opts, &ch, dtype);
    *out = p;
    SV_API_END
}

}  // extern "C"
