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
    int32_t phys[2]; // physical bit of the gate's q[0], q[1] (gate's own order); after
                     // localize_gates: the chunk-local bit, or -1 for a qubit outside the chunk
    int32_t label[2];
    int32_t ext[2] = {-1, -1};  // after localize_gates: state bit of a qubit outside the chunk
};

struct PlanOp {
    int32_t kind;  // 1 = chunk_swap round, 2 = block, 3 = output-reordering round, 4 = gathered block
    std::vector<std::pair<int32_t, int32_t>> pairs;
    std::vector<BlockGate> gates;
    uint64_t mask = 0;  // chunk bits of a gathered block
    int32_t seg_bits = 0;  // tensor-core register-group width of this block (0: the plan's)
};

struct GateKey {
    int32_t nq, q0, q1, flags;
    bool operator==(const GateKey &o) const {
        return nq == o.nq && q0 == o.q0 && q1 == o.q1 && (flags & SV_GATE_SWAP) == (o.flags & SV_GATE_SWAP);
    }
};

}  // namespace sv

struct sv_plan {
    int32_t n = 0, c = 0, reserve = 0, restore = 1, seg_bits = 4, use_tc = 0, pinned = 0;
    int32_t tc_no_renorm = 0, wait_limit_ms = 0;  // executor options carried by the plan
    std::vector<sv::PlanOp> ops;
    std::vector<int32_t> final_map;
    std::vector<sv::GateKey> keys;  // structure of the gate list it was made from
};

namespace sv {

// Cost-model steering of the transpiler's QB_CHUNK choice (gathered chunks only): for every
// section the planner lists candidate chunk sets -- candidates[0] is always the paper's rule --
// with the gates each would take and its features, and a chooser picks one.
constexpr int kNumFeatures = 16;
struct SectionCandidate {
    uint64_t chosen = 0;  // qubits of the chunk
    int absorbed = 0;     // gates the section takes
    int ce = 0;           // chunk bits
    int seg_bits = 0;     // register-group width the features assume (0: the plan's)
    float f[kNumFeatures] = {0};
};
struct SectionChooser {
    virtual ~SectionChooser() = default;
    virtual int choose(const std::vector<SectionCandidate> &cands) = 0;
};

sv_plan *plan_blocking(int n, const sv_gate *gates, int64_t n_gates, const sv_options &o,
                       SectionChooser *chooser = nullptr, int dtype = SV_C64);
// The 16 features of a blocking section (kind 2 or 4) as the cost model sees it.
void section_features(const sv_plan &plan, const PlanOp &op, const sv_gate *gates, int dtype, float *out);

// ------------------------------------------------------------------ block programs
constexpr int SEG_BITS = 4;      // default register-group width (amplitudes per group = 2^SEG_BITS)
constexpr int MAX_SEG_BITS = 5;

// Shared-memory swizzle of a chunk: amplitude i lives in slot i ^ F(i), F(i) = XOR of V[k] over
// the set bits k >= SB of i (SB = 4 for complex64, 3 for complex128).  The V are distinct
// non-powers-of-two below 2^SB where possible, so that any SB of the chunk bits outside a
// register group, plus the low bits, enumerate distinct banks.
#define SV_SWZ64_LIST 0, 0, 0, 0, 3, 5, 6, 7, 9, 10, 11, 12, 13, 14, 15, 3, 5, 6, 7, 9, 10, 11, 12, 13
#define SV_SWZ128_LIST 0, 0, 0, 3, 5, 6, 7, 3, 5, 6, 7, 3, 5, 6, 7, 3, 5, 6, 7, 3, 5, 6, 7, 3
constexpr int kSwz64[24] = {SV_SWZ64_LIST};
constexpr int kSwz128[24] = {SV_SWZ128_LIST};

// Gate op-codes inside a segment.  The exchange codes (bit flip, the two CNOT orientations,
// SWAP) also carry their general form in m[] (dense 2x2 for OP_X1, the permutation of OP_PERM2
// for the others) for consumers that do not special-case them.
enum : int32_t {
    OP_DENSE1 = 0, OP_DENSE2 = 1, OP_DIAG1 = 2, OP_DIAG2 = 3, OP_PERM2 = 4,
    OP_CXA = 5,    // exchange local states 1 <-> 3: control = lower bit a, target = b
    OP_CXB = 6,    // exchange 2 <-> 3: control = b, target = a
    OP_SWAP2 = 7,  // exchange 1 <-> 2
    OP_X1 = 8,     // 1-qubit bit flip
    OP_DIAGX = 9   // diagonal gate with qubits outside the chunk: b = e0 | e1 << 8 (state bits,
                   // 0xFF = none); variant v = bit e0 + 2 bit e1 of the chunk's origin selects
                   // m[4v..4v+3], a diagonal (d0, d1) on register bit a (a phase: d0 = d1, a = 0)
};

// Register group as the kernel reads it.  A thread's group index g enumerates the chunk bits
// outside the group: g bits 0..4 land on lane[0..4], the higher bits on rest[0..nrest).
struct DevSeg {
    int8_t pos[8];    // group bits (ascending); r of them used
    int8_t lane[5];
    int8_t nrest;
    int8_t flags;     // 1: read the natural (unswizzled) layout, 2: write the natural layout
    int8_t r;
    int8_t rest[16];
    int16_t g0, g1;   // gate range [g0, g1) in the section's gate array
};
static_assert(sizeof(DevSeg) == 36, "DevSeg layout");

template <typename T>
struct DevGate {
    int32_t op;     // OP_*
    int32_t a, b;   // local register bits (a < b for 2-qubit ops)
    int32_t code;   // a for 1-qubit ops, a * 8 + b for 2-qubit ops
    T m[32];        // row-major complex matrix in local basis bit a + 2*bit b (diag: the diagonal)
};

struct HostSeg {
    int r = SEG_BITS;
    int32_t pos[8] = {0};
    int32_t lane[5] = {0};
    int32_t rest[16] = {0};
    int nrest = 0;
    int flags = 0;
    std::vector<int32_t> gates;  // indices into the section's gate list
};

// Split a section's gates (physical bits < width) into register groups of at most r bits,
// and choose each group's lane layout for elements of elem_bytes bytes.
// search = false: the greedy groups only (the cost model's cheap feature).
std::vector<HostSeg> segment_block(const std::vector<BlockGate> &gates, int width, int r, int elem_bytes,
                                   bool search = true);
int plan_segment_count(const sv_plan &plan);

template <typename T>
void encode_gate(const sv_gate &g, const BlockGate &bg, const HostSeg &seg, DevGate<T> &out);

// Gathered chunk: the state is viewed as a tensor of rank <= 5 whose dimension d covers the
// index bits [s[d], s[d+1]); each dimension starts with a run of chunk bits (its box, at most
// 8 bits), the bits above it up to the next dimension are addressed by coordinates.  Chunk bits
// outside the boxes are "loop" bits: one tensor copy per value.  Chunk-local bit order: the
// box bits of dimension 0, 1, ..., then the loop bits.
struct GatherArgs {
    int32_t rank;
    int32_t s[6];          // dimension start bits; s[rank] = n
    int32_t nouter, nloop;
    int32_t box_amps;      // amplitudes per tensor copy (2^(box bits))
    int8_t outer[64];      // chunk-index bit -> state bit
    int8_t loop[16];       // copy-index bit -> state bit
};

struct GatherLayout {
    GatherArgs args{};
    int box_len[5] = {0};
    int local_of[64];      // state bit -> chunk-local bit (-1 outside the chunk)
    int ce = 0;            // chunk bits
};

GatherLayout gather_layout(uint64_t mask, int n, int elem_bytes);

// A section's gates on chunk-local bits: bits < min(c, n) for a contiguous chunk (kind 2), the
// gathered layout's local order for kind 4 (`lay` non-null).  A qubit outside the chunk (only
// diagonal gates, diag_outside) gets phys = -1 and its state bit in ext.
std::vector<BlockGate> localize_gates(const PlanOp &op, int n, int c, const GatherLayout *lay);

// Tensor-core path: per register group, the gates to fuse and where its B operand goes.
struct ComposeSeg {
    int32_t g0, g1;     // gate range in the FP64 gate array
    uint32_t b_off;     // byte offset of the group's B_hi (B_lo follows at + tc_b_bytes(r) / 2) in the program
    uint32_t flag_off;  // where to write an int: 1 if the fused matrix is unitary (kNoFlag: none)
};
constexpr uint32_t kNoFlag = 0xFFFFFFFFu;
constexpr int TC_B_BYTES = 8192;  // B_hi + B_lo of one 4-bit register group (2 x 32 x 32 TF32)
// B_hi + B_lo of an r-bit group: two K x K TF32 matrices, K = 2^(r+1) reals per row.
constexpr int tc_b_bytes(int r) { return 8 << (2 * (r + 1)); }
static_assert(tc_b_bytes(4) == TC_B_BYTES, "B operand size");

// Batched execution: one blocking section of one state.  Chunk-local bit k is state bit k for
// k < low (the contiguous low run of the chunk) and high[k - low] above it; the chunk index
// enumerates the state bits outside the chunk, outer[] ascending.  The section's program is
// npiece consecutive pieces at prog_off, each {nseg, ngate, bytes, 0} + DevSeg[] + DevGate[].
struct BatchOp {
    int32_t state, op, ce, low;
    int64_t nchunks, first;  // chunks of this section; first global work-item index
    uint32_t prog_off, prog_bytes;
    int32_t npiece, tc;  // tc: tensor-core groups (pieces hold B operands instead of gate records)
    int32_t nhigh, nouter;
    int8_t high[24];
    int8_t outer[40];
};
constexpr int kBatchMaxChunkBits = 13;
constexpr int kBatchMaxProgBytes = 24 * 1024;    // program piece of a SIMT batch
constexpr int kBatchMaxProgBytesTc = 32 * 1024;  // ... of a batch with tensor-core sections (per pool)
// Tensor-core batches whose chunks have at most kBatchTc3ChunkBits bits run three pools per CTA
// (one tile buffer each) with program pieces of at most kBatchMaxProgBytesTc3 bytes.
constexpr int kBatchTc3ChunkBits = 12;
constexpr int kBatchMaxProgBytesTc3 = 38 * 1024;
constexpr int kBatchTcGroupBytes = TC_B_BYTES + 16;  // B operand + unitarity flag per group
// wait_ns bounds every device wait; stall_state >= 0 (a failure-path test) keeps that state's first
// section from releasing the later ones.
void launch_batch(const void *dev_ops, int nops, const void *dev_progs, void *const *dev_amps, int *dev_ops_done,
                  int *dev_chunks_done, unsigned long long *dev_next, int64_t total, int from_zero, int use_tc,
                  int *dev_err, cudaStream_t st, uint64_t wait_ns, int stall_state);
// Fuse register groups of r bits in FP64; *all_unitary (1 on entry; may be null) is cleared when
// a fused matrix is not unitary to 1e-10 (max |U^H U - I|).
void launch_compose(const void *dev_segs, int nseg, const void *dev_gates, void *dev_prog, int *all_unitary, int r,
                    cudaStream_t st);

// cost-model network kernels (k_mlp.cu)
int mlp_param_count();
int mlp_grad_blocks(int64_t B);
void launch_mlp_fwd(const float *P, const float *X, int64_t B, float *Y, cudaStream_t st);
void launch_mlp_grad(const float *P, const float *X, const float *T, const int32_t *idx, int64_t start, int64_t B,
                     float *part, double *lpart, cudaStream_t st);
void launch_mlp_reduce(const float *part, int nblk, const double *lpart, double *loss, int mode, float *grad, float *P,
                       float *M, float *V, float lr, float c1, float c2, cudaStream_t st);

// ------------------------------------------------------------------ kernels (launchers)
struct Mat1 { float m[8]; };
struct Mat2 { float m[32]; };
struct Mat1d { double m[8]; };
struct Mat2d { double m[32]; };

void launch_gate(int dtype, void *state, int n, const sv_gate &g, cudaStream_t st);
void launch_init_basis(int dtype, void *state, int n, uint64_t basis, cudaStream_t st);
// SIMT section programs of a contiguous-chunk plan, laid out as one device upload (api.cu).
struct SimtPrograms {
    struct Prog {
        size_t off;
        int nseg, ngate, op_index;
    };
    std::vector<unsigned char> host;
    std::vector<Prog> progs;
    int seg_bits = 4;
};
void build_simt_programs(const sv_plan *plan, const sv_gate *gates, int dtype, SimtPrograms &out);
// Amplitudes with bit `bit` == value, in index order, to / from a buffer of 2^(n-1) (k_shard.cu).
void launch_shard_half(bool pack, int dtype, void *state, int n, int bit, int value, void *buf, cudaStream_t st);

struct PermPlan;  // defined in k_permute.cu
void launch_permute(int dtype, void *state, int n, const std::vector<std::pair<int32_t, int32_t>> &pairs,
                    cudaStream_t st);

// Bounded device waits: wait_ns (kDefaultWaitNs unless the plan sets wait_limit_ms).
constexpr uint64_t kDefaultWaitNs = 4000000000ull;
void launch_block(int dtype, void *state, int n, int c, const void *dev_prog, int nseg, int ngates, int *dev_err,
                  int seg_bits, cudaStream_t st, uint64_t wait_ns = kDefaultWaitNs);
// Blocking section over a gathered chunk (bits in `mask`), fetched and written back with
// tensor copies.
void launch_block_gather(int dtype, void *state, int n, const GatherLayout &lay, const void *dev_prog, int nseg,
                         int ngates, int *dev_err, int seg_bits, cudaStream_t st, uint64_t wait_ns = kDefaultWaitNs);
// Tensor-core blocking section (complex64, register groups of seg_bits = 3, 4 or 5 bits, B
// operands in the program, tc_b_bytes(seg_bits) each); `lay` null for a contiguous chunk of c bits.
void launch_block_tc(void *state, int n, int c, const GatherLayout *lay, const void *dev_prog, int nseg, int *dev_err,
                     int seg_bits, cudaStream_t st, uint64_t wait_ns = kDefaultWaitNs);
size_t devgate_bytes(int dtype);

// readouts
void launch_probs(int dtype, const void *state, int n, double *out, int64_t first, int64_t count,
                  cudaStream_t st);
void launch_partial_norm(int dtype, const void *state, int n, double *partials, int nblocks,
                         cudaStream_t st);
// state <- state * sqrt(n_in / n_out) (complex64) when *flag != 0; partials: n_in's nblocks
// partial sums, then n_out's; d: one float of device scratch.
void launch_renorm(int dtype, void *state, int n, const double *partials, int nblocks, const int *flag, float *d,
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
struct sv_state;
namespace sv {
// Synchronise the handle's stream and turn its device error word into a status (clearing it).
void check_dev_error(sv_state *h);

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
    struct Mark {
        int kind, ev, op;  // launch kind, index of its start event, plan op (-1: per-gate)
    };
    std::vector<Mark> ev_marks;
    bool stats_timed = false;
};
