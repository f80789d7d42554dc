// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <memory>
#include <string>
#include <vector>

#include "../../include/sv.h"

namespace sv {

// ------------------------------------------------------------------ errors
struct Error {
    sv_status code;
    std::string msg;
};
void set_error(const std::string &msg);
[[noreturn]] void fail(sv_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);

// Device-side error codes written to the handle's error word.
enum : int { DEV_OK = 0, DEV_ERR_TIMEOUT = 1, DEV_ERR_BOUNDS = 2 };

// ------------------------------------------------------------------ plan (host)
struct BlockGate {
    int64_t gi;      // index into the caller's gate list
    int32_t nq;
    int32_t phys[2]; // physical bit of the gate's q[0], q[1] (gate's own order)
    int32_t label[2];
};

struct PlanOp {
    int32_t kind;  // 1 = chunk_swap round, 2 = block, 3 = output-reordering round
    std::vector<std::pair<int32_t, int32_t>> pairs;
    std::vector<BlockGate> gates;
};

struct GateKey {
    int32_t nq, q0, q1, flags;
    bool operator==(const GateKey &o) const {
        return nq == o.nq && q0 == o.q0 && q1 == o.q1 && (flags & SV_GATE_SWAP) == (o.flags & SV_GATE_SWAP);
    }
};

}  // namespace sv

struct sv_plan {
    int32_t n = 0, c = 0, reserve = 0, restore = 1, seg_bits = 4, use_tc = 0;
    std::vector<sv::PlanOp> ops;
    std::vector<int32_t> final_map;
    std::vector<sv::GateKey> keys;  // structure of the gate list it was made from
    int32_t n_segments = 0;
};

namespace sv {

sv_plan *plan_blocking(int n, const sv_gate *gates, int64_t n_gates, const sv_options &o);

// ------------------------------------------------------------------ block programs
constexpr int SEG_BITS = 4;            // amplitudes per register group = 2^SEG_BITS
constexpr int MAX_SEGS_PER_BLOCK = 512;
constexpr int MAX_GATES_PER_BLOCK = 1024;

// Gate op-codes inside a segment.
enum : int32_t { OP_DENSE1 = 0, OP_DENSE2 = 1, OP_DIAG1 = 2, OP_DIAG2 = 3, OP_PERM2 = 4 };

struct DevSeg {
    int32_t pos[SEG_BITS];  // physical bits (ascending) held in registers
    int32_t g0, g1;         // gate range [g0, g1) in the block's gate array
};

template <typename T>
struct DevGate {
    int32_t op;     // OP_*
    int32_t a, b;   // local register bits (a < b for 2-qubit ops)
    int32_t code;   // pair index of (a, b) / bit index a, for kernel dispatch
    T m[32];        // row-major complex matrix in local basis bit a + 2*bit b (diag: 4 entries)
};

struct HostSeg {
    int32_t pos[SEG_BITS];
    std::vector<int32_t> gates;  // indices into block gate list
};

// Split a block's gates (physical bits < c) into register groups of at most SEG_BITS bits.
std::vector<HostSeg> segment_block(const std::vector<BlockGate> &gates, int c);

template <typename T>
void encode_gate(const sv_gate &g, const BlockGate &bg, const HostSeg &seg, DevGate<T> &out);

// ------------------------------------------------------------------ kernels (launchers)
struct Mat1 { float m[8]; };
struct Mat2 { float m[32]; };
struct Mat1d { double m[8]; };
struct Mat2d { double m[32]; };

void launch_gate(int dtype, void *state, int n, const sv_gate &g, cudaStream_t st);
void launch_init_basis(int dtype, void *state, int n, uint64_t basis, cudaStream_t st);

struct PermPlan;  // defined in k_permute.cu
void launch_permute(int dtype, void *state, int n, const std::vector<std::pair<int32_t, int32_t>> &pairs,
                    cudaStream_t st);

void launch_block(int dtype, void *state, int n, int c, const void *dev_segs, int nseg,
                  const void *dev_gates, int ngates, int *dev_err, int threads, cudaStream_t st);
size_t devgate_bytes(int dtype);

// readouts
void launch_probs(int dtype, const void *state, int n, double *out, int64_t first, int64_t count,
                  cudaStream_t st);
void launch_partial_norm(int dtype, const void *state, int n, double *partials, int nblocks,
                         cudaStream_t st);
void launch_partial_expval(int dtype, const void *state, int n, uint64_t x, uint64_t z,
                           double *partials, int nblocks, cudaStream_t st);
void launch_block_sums(int dtype, const void *state, int n, int sum_bits, double *sums, cudaStream_t st);
void launch_sample_within(int dtype, const void *state, int n, int sum_bits, const double *prefix,
                          const int64_t *shot_block, const double *shot_target, int64_t shots,
                          uint64_t *out, cudaStream_t st);
double splitmix_uniform(uint64_t seed, uint64_t s);

int num_sms();

}  // namespace sv

// ------------------------------------------------------------------ state handle
struct sv_state {
    int32_t n = 0;
    int32_t dtype = SV_C64;
    void *amp = nullptr;      // device amplitudes
    bool owns_amp = false;
    cudaStream_t stream = nullptr;
    int *dev_err = nullptr;   // device error word
    double *scratch = nullptr;  // device scratch for reductions
    size_t scratch_bytes = 0;
    void *prog = nullptr;     // device block programs
    size_t prog_bytes = 0;
    void *prog_host = nullptr;  // pinned staging for programs
    size_t prog_host_bytes = 0;
    cudaEvent_t prog_event = nullptr;
    sv_apply_stats stats{};
    int device = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;                 // reusable timing events
    std::vector<std::pair<int, int>> ev_marks;        // (kind, index of start event) per launch
    bool stats_timed = false;
};
