// Gate records (host, FP64): the u3 rotation of Sec. II.A Eq. 1, the CNOT of Eq. 2 and the
// standard gates used by the workloads.  Matrices are row-major in the local basis
// b = bit(q[0]) + 2*bit(q[1]).
#include <cmath>
#include <cstring>

#include "sv_internal.h"

namespace {

void put(sv_gate *g, int r, int c, double re, double im) {
    const int dim = 1 << g->nq;
    g->m[2 * (r * dim + c)] = re;
    g->m[2 * (r * dim + c) + 1] = im;
}

}  // namespace

extern "C" sv_status sv_gate_make(int32_t kind, const int32_t *qubits, const double *params, sv_gate *out) {
    try {
        if (!out || !qubits) sv::fail(SV_ERR_ARG, "sv_gate_make: null pointer");
        sv_gate g;
        std::memset(&g, 0, sizeof(g));
        auto need_params = [&]() {
            if (!params) sv::fail(SV_ERR_ARG, "sv_gate_make: this kind needs params");
        };
        auto one = [&](int q) { g.nq = 1; g.q[0] = q; g.q[1] = -1; };
        auto two = [&](int q0, int q1) {
            if (q0 == q1) sv::fail(SV_ERR_ARG, "sv_gate_make: repeated qubit");
            g.nq = 2; g.q[0] = q0; g.q[1] = q1;
        };
        switch (kind) {
            case SV_K_UNITARY1:
                need_params();
                one(qubits[0]);
                std::memcpy(g.m, params, 8 * sizeof(double));
                break;
            case SV_K_UNITARY2:
                need_params();
                two(qubits[0], qubits[1]);
                std::memcpy(g.m, params, 32 * sizeof(double));
                break;
            case SV_K_U3: {  // Eq. 1
                need_params();
                one(qubits[0]);
                const double th = params[0], ph = params[1], la = params[2];
                const double c = std::cos(th / 2), s = std::sin(th / 2);
                put(&g, 0, 0, c, 0);
                put(&g, 0, 1, -std::cos(la) * s, -std::sin(la) * s);
                put(&g, 1, 0, std::cos(ph) * s, std::sin(ph) * s);
                put(&g, 1, 1, std::cos(ph + la) * c, std::sin(ph + la) * c);
                break;
            }
            case SV_K_CX:  // Eq. 2: control is the higher local bit -> q[0] = target, q[1] = control
                two(qubits[1], qubits[0]);
                put(&g, 0, 0, 1, 0);
                put(&g, 1, 1, 1, 0);
                put(&g, 2, 3, 1, 0);
                put(&g, 3, 2, 1, 0);
                break;
            case SV_K_H: {
                one(qubits[0]);
                const double r = 1.0 / std::sqrt(2.0);
                put(&g, 0, 0, r, 0); put(&g, 0, 1, r, 0);
                put(&g, 1, 0, r, 0); put(&g, 1, 1, -r, 0);
                break;
            }
            case SV_K_X:
                one(qubits[0]);
                put(&g, 0, 1, 1, 0); put(&g, 1, 0, 1, 0);
                break;
            case SV_K_Y:
                one(qubits[0]);
                put(&g, 0, 1, 0, -1); put(&g, 1, 0, 0, 1);
                break;
            case SV_K_Z:
                one(qubits[0]);
                put(&g, 0, 0, 1, 0); put(&g, 1, 1, -1, 0);
                g.flags |= SV_GATE_DIAG;
                break;
            case SV_K_RY: {
                need_params();
                one(qubits[0]);
                const double c = std::cos(params[0] / 2), s = std::sin(params[0] / 2);
                put(&g, 0, 0, c, 0); put(&g, 0, 1, -s, 0);
                put(&g, 1, 0, s, 0); put(&g, 1, 1, c, 0);
                break;
            }
            case SV_K_RZ: {
                need_params();
                one(qubits[0]);
                const double h = params[0] / 2;
                put(&g, 0, 0, std::cos(h), -std::sin(h));
                put(&g, 1, 1, std::cos(h), std::sin(h));
                g.flags |= SV_GATE_DIAG;
                break;
            }
            case SV_K_CP:
                need_params();
                two(qubits[0], qubits[1]);
                put(&g, 0, 0, 1, 0); put(&g, 1, 1, 1, 0); put(&g, 2, 2, 1, 0);
                put(&g, 3, 3, std::cos(params[0]), std::sin(params[0]));
                g.flags |= SV_GATE_DIAG;
                break;
            case SV_K_CZ:
                two(qubits[0], qubits[1]);
                put(&g, 0, 0, 1, 0); put(&g, 1, 1, 1, 0); put(&g, 2, 2, 1, 0); put(&g, 3, 3, -1, 0);
                g.flags |= SV_GATE_DIAG;
                break;
            case SV_K_SWAP:
                two(qubits[0], qubits[1]);
                put(&g, 0, 0, 1, 0); put(&g, 1, 2, 1, 0); put(&g, 2, 1, 1, 0); put(&g, 3, 3, 1, 0);
                g.flags |= SV_GATE_SWAP;
                break;
            default:
                sv::fail(SV_ERR_ARG, "sv_gate_make: unknown kind");
        }
        for (int j = 0; j < g.nq; ++j)
            if (g.q[j] < 0 || g.q[j] > 63) sv::fail(SV_ERR_ARG, "sv_gate_make: qubit out of range");
        *out = g;
        return SV_OK;
    } catch (const sv::Error &e) {
        sv::set_error(e.msg);
        return e.code;
    }
}

// Many gate records in one call: entry i is sv_gate_make(kinds[i], qubits + 2 i,
// params + i * param_stride, out + i), with NULL params for kinds that take none.
extern "C" sv_status sv_gates_make(int64_t count, const int32_t *kinds, const int32_t *qubits, const double *params,
                                   int32_t param_stride, sv_gate *out) {
    if (count < 0 || param_stride < 0 || (count > 0 && (!kinds || !qubits || !out))) {
        sv::set_error("sv_gates_make: negative count or stride, or null pointer");
        return SV_ERR_ARG;
    }
    for (int64_t i = 0; i < count; ++i) {
        const int32_t k = kinds[i];
        const int need = k == SV_K_UNITARY1 ? 8
                         : k == SV_K_UNITARY2 ? 32
                         : k == SV_K_U3       ? 3
                         : (k == SV_K_RY || k == SV_K_RZ || k == SV_K_CP) ? 1
                                                                          : 0;
        if (need > param_stride || (need && !params)) {
            sv::set_error("sv_gates_make: gate " + std::to_string(i) + ": its kind needs " + std::to_string(need) +
                          " parameters per gate");
            return SV_ERR_ARG;
        }
        const sv_status s = sv_gate_make(k, qubits + 2 * i, need ? params + i * (int64_t)param_stride : nullptr, out + i);
        if (s != SV_OK) {
            sv::set_error("sv_gates_make: gate " + std::to_string(i) + ": " + sv_last_error());
            return s;
        }
    }
    return SV_OK;
}
