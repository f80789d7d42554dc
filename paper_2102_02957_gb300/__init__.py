"""GB300 cache-blocked state-vector simulator (Doi & Horii, arXiv 2102.02957) -- Python binding.

Every step runs in the CUDA library libsv.so through its C ABI (include/sv.h); this module only
marshals arguments.  PyTorch is used for device memory and streams when the caller passes a
tensor buffer; it is not needed otherwise."""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import (GATE_DTYPE, SV_C64, SV_C128, SV_GATE_DIAG, SV_GATE_SWAP, SVError, check, lib,  # noqa: F401
                   sv_apply_stats, sv_options, sv_plan_info)

_KIND = {"u3": _lib.SV_K_U3, "cx": _lib.SV_K_CX, "h": _lib.SV_K_H, "x": _lib.SV_K_X, "y": _lib.SV_K_Y,
         "z": _lib.SV_K_Z, "ry": _lib.SV_K_RY, "rz": _lib.SV_K_RZ, "cp": _lib.SV_K_CP, "cz": _lib.SV_K_CZ,
         "swap": _lib.SV_K_SWAP}

DTYPES = {"c64": SV_C64, "c128": SV_C128, SV_C64: SV_C64, SV_C128: SV_C128}


def make_gates(descriptions) -> np.ndarray:
    """Gate records (sv_gate array) from (kind, qubits, params) descriptions, built by the
    library in one sv_gates_make call."""
    G = len(descriptions)
    out = np.zeros(G, dtype=GATE_DTYPE)
    kinds = np.empty(G, dtype=np.int32)
    qubits = np.zeros((G, 2), dtype=np.int32)
    params = np.zeros((G, 32), dtype=np.float64)
    as_complex = params.view(np.complex128)  # (G, 16): a unitary's row-major entries
    for i, (kind, qs, ps) in enumerate(descriptions):
        qubits[i, :len(qs)] = qs
        if kind == "unitary":
            m = np.asarray(ps[0], dtype=np.complex128)
            kinds[i] = _lib.SV_K_UNITARY1 if m.shape == (2, 2) else _lib.SV_K_UNITARY2
            as_complex[i, :m.size] = m.reshape(-1)
        else:
            kinds[i] = _KIND[kind]
            if ps:
                params[i, :len(ps)] = ps
    check(lib().sv_gates_make(G, kinds.ctypes.data, qubits.ctypes.data, params.ctypes.data, 32, out.ctypes.data))
    return out


def options(**kw) -> sv_options:
    o = sv_options()
    lib().sv_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "restore_layout":
            v = int(bool(v))
        setattr(o, k, int(v))
    return o


class Plan:
    """A cache-blocking schedule made by the library's planner (sv_plan_blocking), or, with a
    trained CostModel, by the steered planner (sv_plan_blocking_steered)."""

    def __init__(self, n: int, gates: np.ndarray, model: "CostModel | None" = None, dtype="c64", **opts):
        self._h = ctypes.c_void_p()
        o = options(**opts)
        if model is None:
            check(lib().sv_plan_blocking(n, gates.ctypes.data, len(gates), ctypes.byref(o), ctypes.byref(self._h)))
        else:
            check(lib().sv_plan_blocking_steered(n, gates.ctypes.data, len(gates), ctypes.byref(o), DTYPES[dtype],
                                                 model._h, ctypes.byref(self._h)))

    def features(self, gates: np.ndarray, dtype="c64") -> np.ndarray:
        """Cost-model features of every blocking section (sv_costmodel_features)."""
        rows = ctypes.c_int64()
        check(lib().sv_costmodel_features(self._h, gates.ctypes.data, DTYPES[dtype], None, 0, ctypes.byref(rows)))
        out = np.zeros((rows.value, _lib.SV_COSTMODEL_FEATURES), dtype=np.float32)
        check(lib().sv_costmodel_features(self._h, gates.ctypes.data, DTYPES[dtype], out.ctypes.data, rows.value,
                                          ctypes.byref(rows)))
        return out

    @property
    def handle(self):
        return self._h

    def info(self) -> sv_plan_info:
        inf = sv_plan_info()
        check(lib().sv_plan_get_info(self._h, ctypes.byref(inf)))
        return inf

    def widths(self):
        """Register-group width of every blocking section (sv_plan_get_widths)."""
        cnt = ctypes.c_int64()
        check(lib().sv_plan_get_widths(self._h, None, 0, ctypes.byref(cnt)))
        out = np.zeros(cnt.value, dtype=np.int32)
        check(lib().sv_plan_get_widths(self._h, out.ctypes.data, cnt.value, ctypes.byref(cnt)))
        return out

    def serialize(self):
        ln = ctypes.c_int64()
        check(lib().sv_plan_serialize(self._h, None, 0, ctypes.byref(ln)))
        buf = (ctypes.c_int64 * ln.value)()
        check(lib().sv_plan_serialize(self._h, buf, ln.value, ctypes.byref(ln)))
        return list(buf)

    def close(self):
        if self._h:
            lib().sv_plan_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def apply_host(n: int, host, gates: np.ndarray, plan: Plan, work_bytes: int, dtype="c64", dev_work=None,
               stream=None) -> int:
    """sv_apply_circuit_host: run `plan` on a state in host memory (`host`: a numpy array or a
    pinned CPU torch tensor of 2^n amplitudes, updated in place) through a device work buffer of
    work_bytes (dev_work: its address, or None to let the library allocate it).  Returns the
    number of passes over the state."""
    ptr = host.ctypes.data if isinstance(host, np.ndarray) else host.data_ptr()
    s = getattr(stream, "cuda_stream", stream)
    passes = ctypes.c_int32()
    check(lib().sv_apply_circuit_host(n, DTYPES[dtype], ptr, gates.ctypes.data, len(gates), plan.handle, dev_work,
                                      work_bytes, s, ctypes.byref(passes)))
    return passes.value


class StateVector:
    """n-qubit state on the GPU.  `buffer`: optional CUDA torch tensor that holds the amplitudes
    (caller-owned); `stream`: optional torch.cuda.Stream (or raw cudaStream_t int)."""

    def __init__(self, n: int, dtype="c64", buffer=None, stream=None):
        self.n = n
        self.dtype = DTYPES[dtype]
        self.amp_bytes = 8 if self.dtype == SV_C64 else 16
        self._buffer = buffer
        ptr = buffer.data_ptr() if buffer is not None else None
        nbytes = buffer.numel() * buffer.element_size() if buffer is not None else 0
        s = getattr(stream, "cuda_stream", stream)
        self._h = ctypes.c_void_p()
        check(lib().sv_create(n, self.dtype, ptr, nbytes, s, ctypes.byref(self._h)))

    # -- state
    def init_basis(self, index: int = 0):
        check(lib().sv_init_basis(self._h, index))

    def get_state(self, out: np.ndarray | None = None) -> np.ndarray:
        dt = np.complex64 if self.dtype == SV_C64 else np.complex128
        if out is None:
            out = np.empty(1 << self.n, dtype=dt)
        check(lib().sv_get_state(self._h, out.ctypes.data if isinstance(out, np.ndarray) else out))
        return out

    def set_state(self, host) -> None:
        ptr = host.ctypes.data if isinstance(host, np.ndarray) else host
        check(lib().sv_set_state(self._h, ptr))

    def set_state_async(self, host_ptr: int) -> None:
        """sv_set_state_async from pinned host memory at host_ptr (an integer address)."""
        check(lib().sv_set_state_async(self._h, host_ptr))

    def get_state_async(self, host_ptr: int) -> None:
        """sv_get_state_async into pinned host memory at host_ptr."""
        check(lib().sv_get_state_async(self._h, host_ptr))

    def device_ptr(self) -> int:
        p = ctypes.c_void_p()
        check(lib().sv_device_ptr(self._h, ctypes.byref(p)))
        return p.value

    def synchronize(self):
        check(lib().sv_synchronize(self._h))

    # -- execution
    def apply(self, gates: np.ndarray, plan: Plan | None = None):
        check(lib().sv_apply_circuit(self._h, gates.ctypes.data, len(gates), plan.handle if plan else None))

    def apply_ops(self, gates: np.ndarray, plan: Plan, op_begin: int, op_end: int):
        """sv_apply_plan_ops: plan ops [op_begin, op_end) on this state, which may be one piece of
        a larger partitioned state (pairs that reach above this piece are skipped)."""
        check(lib().sv_apply_plan_ops(self._h, gates.ctypes.data, len(gates), plan.handle, op_begin, op_end))

    def pack(self, bit: int, value: int, dev_out: int) -> None:
        """sv_shard_pack into the device buffer at dev_out (an integer address)."""
        check(lib().sv_shard_pack(self._h, bit, value, dev_out))

    def unpack(self, bit: int, value: int, dev_in: int) -> None:
        check(lib().sv_shard_unpack(self._h, bit, value, dev_in))

    def set_profiling(self, on: bool = True):
        check(lib().sv_set_profiling(self._h, int(bool(on))))

    def launch_times(self):
        """(kind, plan op index, milliseconds) per launch of the last profiled apply."""
        cnt = ctypes.c_int64()
        check(lib().sv_get_launch_times(self._h, None, None, None, 0, ctypes.byref(cnt)))
        k = np.zeros(cnt.value, dtype=np.int32)
        o = np.zeros(cnt.value, dtype=np.int32)
        ms = np.zeros(cnt.value, dtype=np.float32)
        check(lib().sv_get_launch_times(self._h, k.ctypes.data, o.ctypes.data, ms.ctypes.data, cnt.value,
                                        ctypes.byref(cnt)))
        return k, o, ms

    def stats(self) -> sv_apply_stats:
        s = sv_apply_stats()
        check(lib().sv_get_apply_stats(self._h, ctypes.byref(s)))
        return s

    # -- readouts
    def probabilities(self, out=None) -> np.ndarray:
        if out is None:
            out = np.empty(1 << self.n, dtype=np.float64)
        if isinstance(out, np.ndarray):
            check(lib().sv_probabilities(self._h, out.ctypes.data, 0))
        else:  # a CUDA torch tensor of float64
            check(lib().sv_probabilities(self._h, out.data_ptr(), 1))
        return out

    def norm2(self) -> float:
        v = ctypes.c_double()
        check(lib().sv_norm2(self._h, ctypes.byref(v)))
        return v.value

    def sample(self, shots: int, seed: int) -> np.ndarray:
        out = np.empty(shots, dtype=np.uint64)
        check(lib().sv_sample(self._h, shots, seed, out.ctypes.data))
        return out

    def expval_pauli(self, x_mask: int, z_mask: int) -> complex:
        v = (ctypes.c_double * 2)()
        check(lib().sv_expval_pauli(self._h, x_mask, z_mask, v))
        return complex(v[0], v[1])

    def expval_pauli_noalloc(self, x_mask: int, z_mask: int) -> complex:
        """sv_expval_pauli_noalloc: same value, partial sums in the library's fixed scratch."""
        v = (ctypes.c_double * 2)()
        check(lib().sv_expval_pauli_noalloc(self._h, x_mask, z_mask, v))
        return complex(v[0], v[1])

    def close(self):
        if self._h:
            lib().sv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """Many complex64 states advanced by one persistent launch (sv_batch_*).  `states` are
    StateVector objects, `gate_lists` one gate array per state; both must outlive the batch."""

    def __init__(self, states, gate_lists, **opts):
        if len(states) != len(gate_lists):
            raise ValueError("one gate list per state")
        self._h = ctypes.c_void_p()
        self._states = list(states)
        self._gates = [np.ascontiguousarray(g) for g in gate_lists]
        cnt = len(self._states)
        hs = (ctypes.c_void_p * cnt)(*[s._h.value for s in self._states])
        gp = (ctypes.c_void_p * cnt)(*[g.ctypes.data for g in self._gates])
        ng = (ctypes.c_int64 * cnt)(*[len(g) for g in self._gates])
        o = options(**opts)
        check(lib().sv_batch_create(cnt, hs, gp, ng, ctypes.byref(o), ctypes.byref(self._h)))

    def run(self, use_graph: bool = False, from_zero: bool = False, test_stall: bool = False):
        """One launch; from_zero: every state starts from |0..0> (no sv_init_basis needed);
        test_stall: SV_BATCH_TEST_STALL (a failure-path test: the launch times out)."""
        flags = ((_lib.SV_BATCH_GRAPH if use_graph else 0) | (_lib.SV_BATCH_FROM_ZERO if from_zero else 0)
                 | (_lib.SV_BATCH_TEST_STALL if test_stall else 0))
        check(lib().sv_batch_run(self._h, flags))

    def synchronize(self):
        check(lib().sv_batch_sync(self._h))

    def info(self):
        """(chunk work items, state sections, amplitude bytes read + written per run)."""
        items, sections, nbytes = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_double()
        check(lib().sv_batch_info(self._h, ctypes.byref(items), ctypes.byref(sections), ctypes.byref(nbytes)))
        return items.value, sections.value, nbytes.value

    def close(self):
        if self._h:
            lib().sv_batch_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_OPT_KEYS = ("chunk_bits", "reserve", "restore_layout", "seg_bits", "use_tc", "use_model", "threads", "gather_pinned",
             "diag_outside", "lookahead", "tc_no_renorm", "wait_limit_ms")


def batch_tune(states, gate_lists, **base):
    """sv_batch_tune: pick the batch's chunk bits by timing runs ON these states (their amplitudes
    are overwritten).  Returns (options dict, milliseconds of one run)."""
    gl = [np.ascontiguousarray(g) for g in gate_lists]
    cnt = len(states)
    hs = (ctypes.c_void_p * cnt)(*[s._h.value for s in states])
    gp = (ctypes.c_void_p * cnt)(*[g.ctypes.data for g in gl])
    ng = (ctypes.c_int64 * cnt)(*[len(g) for g in gl])
    b = options(**base)
    best = sv_options()
    ms = ctypes.c_double()
    check(lib().sv_batch_tune(cnt, hs, gp, ng, ctypes.byref(b), ctypes.byref(best), ctypes.byref(ms)))
    return {k: getattr(best, k) for k in _OPT_KEYS}, ms.value


def autotune(n: int, gates: np.ndarray, dtype="c64", **base):
    """sv_autotune: time candidate options for this circuit on a scratch state; returns
    (options dict, milliseconds of one application)."""
    b = options(**base)
    best = sv_options()
    ms = ctypes.c_double()
    check(lib().sv_autotune(n, DTYPES[dtype], gates.ctypes.data, len(gates), ctypes.byref(b), ctypes.byref(best),
                            ctypes.byref(ms)))
    return {k: getattr(best, k) for k in _OPT_KEYS}, ms.value


class CostModel:
    """The learned section-time model (sv_costmodel_*): GPU training and inference kernels."""

    NF = _lib.SV_COSTMODEL_FEATURES
    NP = _lib.SV_COSTMODEL_PARAMS

    def __init__(self, seed: int = 0):
        self._h = ctypes.c_void_p()
        check(lib().sv_costmodel_create(seed, ctypes.byref(self._h)))

    def params(self) -> np.ndarray:
        out = np.zeros(self.NP, dtype=np.float32)
        check(lib().sv_costmodel_get_params(self._h, out.ctypes.data, self.NP))
        return out

    def set_params(self, p) -> None:
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(lib().sv_costmodel_set_params(self._h, p.ctypes.data, p.size))

    def forward(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.NF)
        y = np.zeros(len(x), dtype=np.float32)
        check(lib().sv_costmodel_forward(self._h, x.ctypes.data, len(x), y.ctypes.data))
        return y

    def gradient(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.NF)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.NP, dtype=np.float32)
        loss = ctypes.c_double()
        check(lib().sv_costmodel_gradient(self._h, x.ctypes.data, t.ctypes.data, len(x), g.ctypes.data,
                                          ctypes.byref(loss)))
        return g, loss.value

    def adam_step(self, x, t, lr: float) -> float:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.NF)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = ctypes.c_double()
        check(lib().sv_costmodel_adam_step(self._h, x.ctypes.data, t.ctypes.data, len(x), lr, ctypes.byref(loss)))
        return loss.value

    def add_samples(self, x, us) -> None:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.NF)
        us = np.ascontiguousarray(us, dtype=np.float32)
        check(lib().sv_costmodel_add_samples(self._h, x.ctypes.data, us.ctypes.data, len(x)))

    def num_samples(self) -> int:
        c = ctypes.c_int64()
        check(lib().sv_costmodel_num_samples(self._h, ctypes.byref(c)))
        return c.value

    def collect(self, state: StateVector, gates: np.ndarray, option_sets, policy_seed: int = 0) -> int:
        arr = (sv_options * len(option_sets))(*[options(**o) for o in option_sets])
        added = ctypes.c_int64()
        check(lib().sv_costmodel_collect(self._h, state._h, gates.ctypes.data, len(gates), arr, len(option_sets),
                                         policy_seed, ctypes.byref(added)))
        return added.value

    def train(self, epochs: int = 200, batch: int = 256, lr: float = 1e-3, seed: int = 1) -> float:
        mse = ctypes.c_double()
        check(lib().sv_costmodel_train(self._h, epochs, batch, lr, seed, ctypes.byref(mse)))
        return mse.value

    def predict_us(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float32).reshape(-1, self.NF)
        us = np.zeros(len(x), dtype=np.float32)
        check(lib().sv_costmodel_predict_us(self._h, x.ctypes.data, len(x), us.ctypes.data))
        return us

    def close(self):
        if self._h:
            lib().sv_costmodel_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
