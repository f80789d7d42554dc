/* sv.h -- C ABI of the GB300 cache-blocked state-vector simulator.
 *
 * Method: Doi & Horii, "Cache Blocking Technique to Large Scale Quantum Computing Simulation
 * on Supercomputers" (arXiv 2102.02957).  An n-qubit state is 2^n complex amplitudes, index
 * bit k = qubit k (Sec. II.A, Fig. 1-2).  A transpiler (Sec. IV.A, Listing 3) inserts
 * chunk_swap gates so that runs of gates touch only the low c "chunk" bits; each run is then
 * applied chunk by chunk (Sec. IV.C, Listing 4).  On one GPU the chunk is staged once from
 * HBM into shared memory per run, and every chunk_swap round is one in-place HBM permutation
 * pass.
 *
 * Conventions for every entry point:
 *  - Every function returns an sv_status; nothing throws across the ABI.  On failure
 *    sv_last_error() returns a message for the calling thread (valid until its next call).
 *  - Pointers are plain host pointers unless a parameter says "device".  The library never
 *    takes ownership of caller memory; objects it creates (sv_handle, sv_plan_h) are freed
 *    by the matching destroy/free call.
 *  - Qubit numbering is little-endian (Sec. II.A: |2> = |10>).
 *  - Calls that launch GPU work are asynchronous on the handle's stream unless they return
 *    host data (readouts, sv_get_state), which synchronise that stream before returning.
 *  - Sizes: 1 <= n <= 34.  A gate acts on 1 or 2 distinct qubits < n.
 */
#ifndef SV_H
#define SV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum sv_status {
    SV_OK = 0,
    SV_ERR_ARG = 1,         /* invalid argument (null pointer, size or qubit out of range)   */
    SV_ERR_OOM = 2,         /* device or host allocation failed                               */
    SV_ERR_CUDA = 3,        /* a CUDA runtime call or kernel launch failed                    */
    SV_ERR_PLAN = 4,        /* plan does not match the state / gate list, or planning failed   */
    SV_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired; the state is undefined      */
    SV_ERR_UNSUPPORTED = 6  /* valid request that the library does not implement              */
} sv_status;

typedef enum sv_dtype {
    SV_C64 = 1,  /* complex64: interleaved (float re, float im), 8 bytes per amplitude    */
    SV_C128 = 2  /* complex128: interleaved (double re, double im), 16 bytes per amplitude */
} sv_dtype;

/* One gate.  nq = 1 or 2 qubits q[0] (, q[1]).  m is the row-major 2^nq x 2^nq complex
 * matrix, interleaved (re, im) doubles, in the local basis b = bit(q[0]) + 2*bit(q[1]);
 * entries past 2^nq x 2^nq are ignored.  flags: SV_GATE_SWAP marks a SWAP that the planner
 * applies as a relabel (no data movement; m must still hold the SWAP matrix for the
 * per-gate path).  SV_GATE_DIAG marks a diagonal matrix (a hint; m is authoritative). */
enum { SV_GATE_SWAP = 1, SV_GATE_DIAG = 2 };
typedef struct sv_gate {
    int32_t nq;
    int32_t q[2];
    int32_t flags;
    double m[32];
} sv_gate;

/* Gate kinds for sv_gate_make. params: U3 (theta, phi, lambda) per Sec. II.A Eq. 1 (the
 * paper's psi is phi); RY/RZ (theta); CP (phi); UNITARY1/UNITARY2 take 8/32 doubles of a
 * row-major interleaved matrix.  qubits: CX and CP and CZ take (control, target); the CX
 * matrix is Eq. 2 with the control as the higher local bit. */
typedef enum sv_gate_kind {
    SV_K_UNITARY1 = 0, SV_K_UNITARY2 = 1, SV_K_U3 = 2, SV_K_CX = 3, SV_K_H = 4, SV_K_X = 5,
    SV_K_Y = 6, SV_K_Z = 7, SV_K_RY = 8, SV_K_RZ = 9, SV_K_CP = 10, SV_K_CZ = 11, SV_K_SWAP = 12
} sv_gate_kind;

/* Build one gate record (gate matrices of Sec. II.A, Eq. 1 and Eq. 2; host FP64).
 * qubits: 1 or 2 entries by kind.  params: as listed above (NULL allowed for kinds without
 * parameters).  out: filled on success.  SV_ERR_ARG for an unknown kind or repeated qubit. */
sv_status sv_gate_make(int32_t kind, const int32_t *qubits, const double *params, sv_gate *out);

/* Build `count` gate records in one call (the same matrices as sv_gate_make, Sec. II.A).
 * kinds[count]; qubits[count][2] (the second entry of a 1-qubit kind is ignored);
 * params[count][param_stride] doubles, read only for kinds that take parameters, so
 * param_stride must be at least the largest such count among `kinds` (32 covers every kind;
 * params may be NULL when none takes any).  out[count]: all caller-owned host memory.
 * On an error no later entry is written; SV_ERR_ARG names the failing index. */
sv_status sv_gates_make(int64_t count, const int32_t *kinds, const int32_t *qubits, const double *params,
                        int32_t param_stride, sv_gate *out);

/* Planner / executor options.  Defaults from sv_options_default(). */
typedef struct sv_options {
    int32_t chunk_bits;     /* c: physical bits 0..c-1 form a chunk (Sec. II.B, IV.A); default 13 */
    int32_t reserve;        /* 0: chunk holds c chosen qubits; 1: c-1 (the listing's "nc-1"). default 0 */
    int32_t restore_layout; /* 1: end with the output reordering of Sec. IV.C (Fig. 10 (b)). default 1 */
    int32_t seg_bits;       /* register-group width used inside a chunk (4); fusion width on TC path */
    int32_t use_tc;         /* 1: apply fused groups as 3xTF32 tensor-core contractions (complex64) */
    int32_t use_model;      /* informational: 1 in plans made by sv_plan_blocking_steered; ignored as input */
    int32_t threads;        /* consumer threads per chunk CTA; 0 = auto                             */
    int32_t gather_pinned;  /* 0: the paper's chunk_swap rounds make every chunk bits 0..c-1.  p > 0:
                               gathered chunks -- a chunk is the low p bits plus c-p chosen bits,
                               fetched in place (no chunk_swap passes, no data reordering); the
                               transpiler's choice rule starts from the p pinned bits.  default 0 */
    int32_t diag_outside;   /* 1: diagonal gates (SV_GATE_DIAG with an exactly diagonal matrix) may
                               join a section while some of their qubits lie outside its chunk: those
                               qubits are constant over a chunk, so the gate acts there as a diagonal
                               on its chunk qubits (or a phase).  Ignored with use_tc.  default 0 */
    int32_t lookahead;      /* 1 (gathered chunks): choose each section's chunk by look-ahead -- grow it
                               from the pinned bits and the first gate by the pending gate whose qubits
                               let the section take the most gates -- instead of the paper's priority
                               rule.  A heuristic of this library, not the paper's.  default 0 */
    int32_t tc_no_renorm;   /* 1: leave out the norm restoration of tensor-core circuits (the state is
                               rescaled to its input norm after the last section when every fused
                               group is unitary), so the result shows the raw 3xTF32 error.  default 0 */
    int32_t wait_limit_ms;  /* bound of every device-side wait of the blocking kernels in milliseconds;
                               on expiry the kernel stops and the next synchronising call returns
                               SV_ERR_TIMEOUT.  0: the default (4000 ms).  Taken by sv_apply_circuit
                               from the plan's options. */
    int32_t reserved[4];
} sv_options;

void sv_options_default(sv_options *opts);

/* ------------------------------------------------------------------ state handles */
typedef struct sv_state *sv_handle;

/* Create an n-qubit state of `dtype`.  dev_buf: caller-owned DEVICE buffer of at least
 * 2^n * bytes-per-amplitude bytes, 256-byte aligned (e.g. a torch tensor); NULL lets the
 * library allocate (freed by sv_destroy).  cuda_stream: a cudaStream_t, or NULL for the
 * legacy default stream.  The amplitudes are undefined until sv_init_basis/sv_set_state. */
sv_status sv_create(int32_t n, int32_t dtype, void *dev_buf, size_t bytes, void *cuda_stream,
                    sv_handle *out);
sv_status sv_destroy(sv_handle h);

/* Set the state to the basis state |basis_index> (Sec. IV.C: zero every chunk, one
 * amplitude = 1).  basis_index < 2^n. */
sv_status sv_init_basis(sv_handle h, uint64_t basis_index);

/* Copy the 2^n amplitudes to / from HOST memory (pinned memory gives full bandwidth).
 * Layout as sv_dtype.  Synchronous with respect to the host. */
sv_status sv_get_state(sv_handle h, void *host_out);
sv_status sv_set_state(sv_handle h, const void *host_in);
/* The same copies, asynchronous on the handle's stream: host_out / host_in must be pinned host
 * memory that stays valid (and, for host_in, unchanged) until the stream has passed the copy
 * (sv_synchronize).  Copies on one handle's stream overlap kernels on another handle's stream. */
sv_status sv_get_state_async(sv_handle h, void *host_out);
sv_status sv_set_state_async(sv_handle h, const void *host_in);

/* Device pointer of the amplitude array (borrowed; valid until sv_destroy). */
sv_status sv_device_ptr(sv_handle h, void **dev_ptr);
sv_status sv_synchronize(sv_handle h);

/* ------------------------------------------------------------------ planning */
typedef struct sv_plan *sv_plan_h;

/* Cache-blocking transpiler of Sec. IV.A (Listing 3) on the host.  Deterministic: the same
 * input gives the same schedule.  Uses opts->chunk_bits, reserve, restore_layout, seg_bits,
 * use_tc and gather_pinned.  SV_ERR_ARG when a gate is wider than the chunk. */
sv_status sv_plan_blocking(int32_t n, const sv_gate *gates, int64_t n_gates,
                           const sv_options *opts, sv_plan_h *out);
sv_status sv_plan_free(sv_plan_h plan);

typedef struct sv_plan_info {
    int32_t n, chunk_bits, reserve, restore_layout;
    int32_t n_blocks;            /* blocking sections (one HBM sweep each)           */
    int32_t n_swap_rounds;       /* chunk_swap rounds (one in-place pass each)       */
    int32_t n_unpermute_rounds;  /* output-reordering rounds (0..2)                  */
    int32_t n_segments;          /* register groups over all blocks                  */
    int64_t n_gates_emitted;     /* gates inside blocks (SWAP relabels excluded)     */
    int32_t final_map[64];       /* physical bit of logical qubit q after the plan   */
} sv_plan_info;
sv_status sv_plan_get_info(sv_plan_h plan, sv_plan_info *info);
/* Register-group width (bits) of every blocking section's tensor-core groups, in plan order: the
 * plan's seg_bits, or the section's own width where a steered plan chose one (4 or 5 bits on a
 * chunk of at least 2^(width+7) amplitudes).  out (may be NULL) receives at most cap entries;
 * count receives the number of sections. */
sv_status sv_plan_get_widths(sv_plan_h plan, int32_t *out, int64_t cap, int64_t *count);

/* Integer serialisation of the schedule (used to compare schedules bit for bit):
 * [n, c, reserve, restore, n_ops, ops..., final_map[n]] with ops
 *   [1, r, (p, q) x r]                 chunk_swap round (p < c <= q)
 *   [2, G, (gate_index, nq, p0, p1) x G]  block; p0/p1 = physical bits of the gate's qubits in
 *                                         ascending logical order, p1 = -1 for 1 qubit
 *   [3, r, (p, q) x r]                 output-reordering round
 *   [4, mask, G, (gate_index, nq, p0, p1) x G]  gathered block over the chunk bits in `mask`.
 * Writes at most `cap` values to buf; *len receives the full length (call with cap 0 to
 * size the buffer). */
sv_status sv_plan_serialize(sv_plan_h plan, int64_t *buf, int64_t cap, int64_t *len);

/* ------------------------------------------------------------------ execution */
/* Apply the circuit.  plan == NULL: the plain per-gate path (one HBM sweep per gate, the
 * paper's baseline of Sec. V.A).  Otherwise the cache-blocked path (Listing 4): each chunk_swap
 * round is one in-place permutation pass and each blocking section one pass in which every
 * chunk is staged in shared memory, all its gates applied, and written back.  The plan must
 * have been made from the same n and gate list (SV_ERR_PLAN otherwise). */
sv_status sv_apply_circuit(sv_handle h, const sv_gate *gates, int64_t n_gates, sv_plan_h plan);

/* ------------------------------------------------------------------ partitioned states */
/* A state partitioned on its top qubits (Sec. II.B: the state vector is divided into pieces, one
 * per process, on the highest qubits; Sec. IV.C: blocks run on each piece alone, and a
 * chunk_swap of a chunk qubit with a partition qubit moves half of each piece to a partner,
 * Fig. 10 case (a); the output reordering can also swap two partition qubits, Fig. 10 case (b)).
 * One handle holds one piece: h->n = plan n - (partition qubits); its amplitude k is the state's
 * amplitude (piece index << h->n) | k.
 *
 * Run plan ops [op_begin, op_end) of a plan made with gather_pinned = 0 (contiguous chunks) on
 * the piece: blocking sections with SIMT register groups (the chunk must fit the piece: c <= h->n),
 * and the chunk_swap / reordering pairs whose two bits are both below h->n.  Pairs with a bit at
 * or above h->n are left to the caller, who exchanges data between pieces with sv_shard_pack /
 * sv_shard_unpack.  With h->n == plan n this is a part of sv_apply_circuit (without its
 * tensor-core sections).  Asynchronous on the handle's stream.  SV_ERR_PLAN for a plan of other
 * gates or a chunk wider than the piece; SV_ERR_UNSUPPORTED for gathered-chunk plans. */
sv_status sv_apply_plan_ops(sv_handle h, const sv_gate *gates, int64_t n_gates, sv_plan_h plan,
                            int32_t op_begin, int32_t op_end);
/* Copy the piece's amplitudes whose local bit `bit` equals `value` (0 or 1), in index order, to
 * the DEVICE buffer dev_out (2^(h->n - 1) amplitudes), or back from dev_in into the same places.
 * bit < 0 copies the whole piece (2^h->n amplitudes).  Asynchronous on the handle's stream; the
 * buffers are the caller's. */
sv_status sv_shard_pack(sv_handle h, int32_t bit, int32_t value, void *dev_out);
sv_status sv_shard_unpack(sv_handle h, int32_t bit, int32_t value, const void *dev_in);

/* ------------------------------------------------------------------ host-resident states */
/* Apply a plan (made with gather_pinned = 0) to a state kept in HOST memory, with the GPU as a
 * cache for its chunks (Sec. IV.C: chunks that do not fit in GPU memory stay in host memory and
 * are staged through the GPU; Sec. V.B: 33 to 35 qubits that way).  host_amps: the caller's 2^n
 * amplitudes (layout as sv_dtype; pinned memory lets the copies run at the link's rate).  The
 * plan runs in passes, each streaming the state through the device work buffer once: consecutive
 * sections and chunk_swap / reordering rounds share a pass when their sub-states fit half the
 * buffer (two are in flight, so copies overlap kernels).  dev_work: a DEVICE buffer of work_bytes
 * (the caller's), or NULL to let the library allocate work_bytes for the call; it must hold two
 * sub-states of 2^(c+2) amplitudes unless it holds the whole state twice.  Sections run on SIMT
 * register groups.  Synchronous: returns when the state in host memory is final.  passes (may be
 * NULL): the number of passes over the state.  SV_ERR_PLAN / SV_ERR_UNSUPPORTED as for
 * sv_apply_circuit and for gathered plans; SV_ERR_ARG for a work buffer that is too small. */
sv_status sv_apply_circuit_host(int32_t n, int32_t dtype, void *host_amps, const sv_gate *gates,
                                int64_t n_gates, sv_plan_h plan, void *dev_work, size_t work_bytes,
                                void *cuda_stream, int32_t *passes);

/* Statistics of the last sv_apply_circuit on this handle (host-side counts). */
typedef struct sv_apply_stats {
    int64_t kernel_launches;
    int64_t sweeps_block;       /* blocked-section passes                */
    int64_t sweeps_permute;     /* chunk_swap + reordering passes        */
    int64_t sweeps_gate;        /* per-gate passes                       */
    double algorithmic_bytes;   /* (passes) x 2 x 2^n x bytes/amplitude  */
    double ms_block;            /* device time of the blocked-section kernels (profiling on) */
    double ms_permute;          /* device time of the permutation kernels (profiling on)     */
    double ms_gate;             /* device time of the per-gate kernels (profiling on)        */
} sv_apply_stats;
/* Counts of the last sv_apply_circuit; with profiling on, also the summed device time of its
 * kernels by kind, taken from CUDA events recorded on the handle's stream around each launch
 * (this call then synchronises the stream). */
sv_status sv_get_apply_stats(sv_handle h, sv_apply_stats *out);

/* on != 0: record CUDA events around every kernel that sv_apply_circuit launches. */
sv_status sv_set_profiling(sv_handle h, int32_t on);

/* ------------------------------------------------------------------ batched execution */
/* Many independent complex64 states (noisy trajectories, parameter sets -- the paper's "shots",
 * Sec. IV.B) advanced by ONE persistent kernel launch.  Each state gets a gathered-chunk plan
 * (sv_options.chunk_bits capped at 13, gather_pinned = 4); a state that fits one chunk runs its
 * whole circuit in one shared-memory residency.  The launch drains a work queue of (state,
 * section, chunk) items; a chunk waits (bounded) for the earlier sections of its own state.
 * Constraints: every handle complex64, on the current device, n >= 6; gate lists without SWAP
 * relabels.  The batch object owns the device-side plans and queue; the states stay owned by
 * their handles.  All handles must share one CUDA stream, on which the work runs (SV_ERR_ARG
 * otherwise); SV_ERR_UNSUPPORTED for complex128, n < 6 or a SWAP gate. */
typedef struct sv_batch *sv_batch_h;
sv_status sv_batch_create(int32_t count, const sv_handle *states, const sv_gate *const *gates,
                          const int64_t *n_gates, const sv_options *opts, sv_batch_h *out);
/* Launch the batch once (asynchronous).  flags: SV_BATCH_GRAPH -- the launch (counter reset +
 * kernel) is captured once into a CUDA graph and replayed on later runs with the same flags;
 * SV_BATCH_FROM_ZERO -- every state starts from |0..0> (Sec. IV.C initial state): the first
 * section writes its chunks from the basis state instead of reading them, so the amplitudes
 * need no prior sv_init_basis.  SV_BATCH_TEST_STALL -- a test of the failure path: the first
 * section of the batch's first state never releases that state's later sections, so their
 * bounded waits (opts->wait_limit_ms of sv_batch_create, default 4000 ms) expire; the launch ends
 * and sv_batch_sync returns SV_ERR_TIMEOUT.  Not combinable with SV_BATCH_GRAPH. */
enum { SV_BATCH_GRAPH = 1, SV_BATCH_FROM_ZERO = 2, SV_BATCH_TEST_STALL = 4 };
sv_status sv_batch_run(sv_batch_h batch, int32_t flags);
/* Wait for the last run; SV_ERR_TIMEOUT if a bounded wait in the launch expired. */
sv_status sv_batch_sync(sv_batch_h batch);
/* Number of chunk work items and of (state, section) sweeps in the batch, and the amplitude
 * bytes one run reads and writes (2 x 8 B x 2^n per sweep of an n-qubit state).  NULL outputs
 * are skipped. */
sv_status sv_batch_info(sv_batch_h batch, int64_t *work_items, int32_t *sections, double *bytes_per_run);
sv_status sv_batch_free(sv_batch_h batch);
/* Autotune a batch: build it with chunk bits 10..13 (other fields from *base), time one run of
 * each after a warm-up run, and write the fastest options to *best and its time to *best_ms.
 * The circuits RUN on the given states: their amplitudes are overwritten (initialise them
 * afterwards).  Same constraints as sv_batch_create. */
sv_status sv_batch_tune(int32_t count, const sv_handle *states, const sv_gate *const *gates,
                        const int64_t *n_gates, const sv_options *base, sv_options *best, double *best_ms);

/* ------------------------------------------------------------------ autotuning */
/* Time candidate executions of this circuit on a scratch n-qubit state of `dtype` (chunk bits
 * 11..13, register-group width 4/5, gathered or chunk_swap layout, the paper's or the look-ahead
 * chunk choice, tensor cores on/off for complex64) and write the fastest options to *best (its
 * other fields are copied from *base).
 * best_ms receives the measured milliseconds of one application with those options.  Allocates
 * and frees its own scratch state; synchronises the device. */
sv_status sv_autotune(int32_t n, int32_t dtype, const sv_gate *gates, int64_t n_gates, const sv_options *base,
                      sv_options *best, double *best_ms);

/* ------------------------------------------------------------------ learned cost model */
/* The paper's QB_CHUNK rule (Sec. IV.A) is a fixed heuristic; the paper notes that better
 * schedules exist but gives no method (it has no counterpart of this section).  The library adds
 * a small regression network that predicts the kernel time of a blocking section from 16
 * features of it, trained on timings the library measures itself, and a planner variant in
 * which the prediction picks each section's chunk among candidates: the paper's rule (always
 * candidate 0), the rule with one or two fewer chunk qubits, and a look-ahead set that takes the
 * most gates.  Gathered chunks (gather_pinned > 0) only.  Every candidate is a valid section,
 * so no amplitude depends on the model.
 *
 * Network: x (16) -> relu(W1 x + b1) (64) -> relu(W2 h1 + b2) (64) -> y = w3 . h2 + b3, FP32;
 * y estimates the standardised log of the section's kernel microseconds.  Parameters, flat
 * (5313 floats): W1 (64 x 16, row-major), b1 (64), W2 (64 x 64, row-major), b2 (64), w3 (64),
 * b3.  Training: mean squared error, Adam (b1 0.9, b2 0.999, eps 1e-8) on the GPU by the
 * library's own forward / backward / update kernels.  A model lives on the device that was
 * current at creation; its calls synchronise. */
typedef struct sv_costmodel *sv_costmodel_h;
enum { SV_COSTMODEL_FEATURES = 16, SV_COSTMODEL_PARAMS = 5313 };
/* He-uniform weights (bound sqrt(6 / fan_in)) from a SplitMix64 stream seeded with `seed`,
 * zero biases, empty sample set. */
sv_status sv_costmodel_create(uint64_t seed, sv_costmodel_h *out);
sv_status sv_costmodel_free(sv_costmodel_h m);
/* Copy the flat parameters out / in (count must be SV_COSTMODEL_PARAMS); setting them clears
 * the Adam moments and step count. */
sv_status sv_costmodel_get_params(sv_costmodel_h m, float *out, int64_t count);
sv_status sv_costmodel_set_params(sv_costmodel_h m, const float *in, int64_t count);
/* Raw network outputs y for `count` host feature rows (count x 16, row-major) -> host out. */
sv_status sv_costmodel_forward(sv_costmodel_h m, const float *x, int64_t count, float *y);
/* Gradient of L = (1/count) sum (y_i - t_i)^2 at the current parameters (host in, host out:
 * grad has SV_COSTMODEL_PARAMS entries) and L itself. */
sv_status sv_costmodel_gradient(sv_costmodel_h m, const float *x, const float *t, int64_t count, float *grad,
                                double *loss);
/* One Adam step on this batch (raw targets t); loss receives L before the step. */
sv_status sv_costmodel_adam_step(sv_costmodel_h m, const float *x, const float *t, int64_t count, float lr,
                                 double *loss);
/* Training samples: feature rows and measured section times in microseconds. */
sv_status sv_costmodel_add_samples(sv_costmodel_h m, const float *x, const float *us, int64_t count);
sv_status sv_costmodel_num_samples(sv_costmodel_h m, int64_t *count);
/* Timing collector: for each of the n_opts option sets, plan the circuit (candidate sections
 * picked at random from a SplitMix64 stream seeded with policy_seed + k when policy_seed != 0,
 * else the paper's rule), apply it to h twice (the second timed per launch with CUDA events)
 * and add one sample per blocking section.  Overwrites h's amplitudes. */
sv_status sv_costmodel_collect(sv_costmodel_h m, sv_handle h, const sv_gate *gates, int64_t n_gates,
                               const sv_options *opts, int32_t n_opts, uint64_t policy_seed, int64_t *added);
/* Train on all samples: targets standardised log(us); `epochs` passes of shuffled minibatches
 * of `batch` samples (SplitMix64 shuffle seeded with `seed`), Adam with rate lr.  mse receives
 * the final mean squared error of log(us) over the samples. */
sv_status sv_costmodel_train(sv_costmodel_h m, int32_t epochs, int32_t batch, float lr, uint64_t seed, double *mse);
/* Predicted section kernel time in microseconds for `count` feature rows. */
sv_status sv_costmodel_predict_us(sv_costmodel_h m, const float *x, int64_t count, float *us);
/* Features of every blocking section of a plan, in plan order (rows x 16); rows receives the
 * number of sections (at most max_rows are written). */
sv_status sv_costmodel_features(sv_plan_h plan, const sv_gate *gates, int32_t dtype, float *out, int64_t max_rows,
                                int64_t *rows);
/* Planner with the model's steering (see above): per section, the candidate with the most gates
 * per predicted microsecond.  Same constraints and output as sv_plan_blocking; requires
 * opts->gather_pinned > 0 and a trained model. */
sv_status sv_plan_blocking_steered(int32_t n, const sv_gate *gates, int64_t n_gates, const sv_options *opts,
                                   int32_t dtype, sv_costmodel_h model, sv_plan_h *out);
/* Per-launch device times of the last sv_apply_circuit with profiling on: kind (0 per-gate,
 * 1 blocking section, 2 permutation), plan op index (-1 per-gate), milliseconds.  count
 * receives the number of launches (at most max entries are written).  Synchronises. */
sv_status sv_get_launch_times(sv_handle h, int32_t *kind, int32_t *op_index, float *ms, int64_t max, int64_t *count);

/* ------------------------------------------------------------------ readouts (FP64 accumulate) */
/* Measurement probabilities |a_i|^2 (Sec. II.A) for all 2^n indices.  out: 2^n doubles,
 * on the device when out_on_device != 0, else on the host. */
sv_status sv_probabilities(sv_handle h, double *out, int32_t out_on_device);

/* Sum of |a_i|^2. */
sv_status sv_norm2(sv_handle h, double *out);

/* Draw `shots` basis indices by inverse CDF: shot s is the smallest i with
 * sum_{k<=i} |a_k|^2 > u_s * sum_k |a_k|^2, u_s the s-th uniform of the SplitMix64 stream
 * seeded with `seed` (top 53 bits * 2^-53).  out: `shots` uint64 on the host. */
sv_status sv_sample(sv_handle h, int64_t shots, uint64_t seed, uint64_t *out);

/* <psi| P |psi> for the Pauli word P = i^{popcount(x&z)} X^x Z^z (Y where both bits are set).
 * out[0] = real part, out[1] = imaginary part (host). */
sv_status sv_expval_pauli(sv_handle h, uint64_t x_mask, uint64_t z_mask, double *out);

/* The same value as sv_expval_pauli, for callers that must not allocate memory at the time of
 * the call (a memory budget or pool they do not own, or loops where a cudaMalloc/cudaFree would
 * stall the device).  The paper has no counterpart; this is a service of this library.
 * It calls no cudaMalloc, cudaFree or other allocating routine: its partial sums go to a fixed
 * 64 KiB array compiled into the library (4096 (re, im) pairs plus the result), which every GPU
 * that loads the library holds until the process exits.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current, so make that
 * first call before any stream capture.  The handle's device must be the current device
 * (SV_ERR_ARG otherwise).  A state that would need more than 4096 partial sums (more than 512
 * SMs) is rejected with SV_ERR_UNSUPPORTED.  All calls share the array and it keeps the last
 * call's contents: calls whose kernels overlap on the GPU (different streams, threads) race
 * and must be serialised by the caller.  Synchronises the handle's stream; out[0] = real part,
 * out[1] = imaginary part (host). */
sv_status sv_expval_pauli_noalloc(sv_handle h, uint64_t x_mask, uint64_t z_mask, double *out);

/* Thread-local message for the last failed call on this thread ("" if none). */
const char *sv_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SV_H */
