"""Thin Python binding of the C ABI in ``include/tanq.h`` (ctypes).

Argument marshalling only: op names become the header's enum values, numpy
arrays become pointers, vec(rho) is reshaped to and from the matrix rho[r, c]
(vec index r + c 2^n). Every step of the simulation runs in the CUDA
library; there is no CPU fallback, and loading fails loudly when
``libtanq.so`` has not been built.

PyTorch supplies the plumbing when it is importable: the state's CUDA stream
is the current torch stream and vec(rho) is a tensor from torch's caching
allocator (``tq_create_on``).
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_double, c_int, c_int32, c_size_t, c_uint64, c_void_p

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtanq.so")

# enum values of include/tanq.h (a CPU test checks them against the header)
PRECISION = {"fp64": 0, "split": 1}
STATUS = {0: "TQ_OK", 1: "TQ_ERR_ARG", 2: "TQ_ERR_QUBIT", 3: "TQ_ERR_OOM", 4: "TQ_ERR_CUDA",
          5: "TQ_ERR_TIMEOUT", 6: "TQ_ERR_STATE", 7: "TQ_ERR_UNSUPPORTED"}
GATES = {"id": 0, "h": 1, "x": 2, "y": 3, "z": 4, "s": 5, "sdg": 6, "t": 7, "tdg": 8, "sx": 9,
         "rx": 10, "ry": 11, "rz": 12, "su2": 13, "cx": 32, "cz": 33, "swap": 34, "rzz": 35}
CHANNELS = {"depol": 0, "ad": 1, "pd": 2, "thermal": 3, "reset": 4}
OP_UNITARY, OP_KRAUS, OP_GATE, OP_CHANNEL = 0, 1, 2, 3


class TqOp(ctypes.Structure):
    _fields_ = [("kind", c_int32), ("k", c_int32), ("qubits", c_int32 * 4), ("m", c_int32),
                ("name", c_int32), ("params", c_double * 4), ("mats", POINTER(c_double))]


class TqKernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", c_uint64), ("total_ms", c_double),
                ("flops", c_double), ("bytes", c_double)]


class TqError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)} ({_lib.tq_status_string(status).decode() if _lib else ''})")


_lib = None

# (name, restype, argtypes) of every exported function
_SIGNATURES = [
    ("tq_create", c_int, [c_int, c_int, c_void_p, POINTER(c_void_p)]),
    ("tq_create_on", c_int, [c_int, c_int, c_void_p, c_void_p, c_size_t, POINTER(c_void_p)]),
    ("tq_free", None, [c_void_p]),
    ("tq_info", c_int, [c_void_p, POINTER(c_int), POINTER(c_int)]),
    ("tq_reset", c_int, [c_void_p]),
    ("tq_rho_device_ptr", c_int, [c_void_p, POINTER(c_void_p)]),
    ("tq_set_hermitian", c_int, [c_void_p, c_int]),
    ("tq_is_hermitian_mode", c_int, [c_void_p, POINTER(c_int)]),
    ("tq_set_fp64_engine", c_int, [c_void_p, c_int]),
    ("tq_fp64_on_tensor", c_int, [c_void_p, POINTER(c_int)]),
    ("tq_get_rho", c_int, [c_void_p, POINTER(c_double)]),
    ("tq_set_rho", c_int, [c_void_p, POINTER(c_double)]),
    ("tq_apply_gate", c_int, [c_void_p, POINTER(c_int), c_int, POINTER(c_double)]),
    ("tq_apply_kraus", c_int, [c_void_p, POINTER(c_int), c_int, c_int, POINTER(c_double)]),
    ("tq_run_circuit", c_int, [c_void_p, POINTER(TqOp), c_size_t, c_int, POINTER(c_size_t)]),
    ("tq_trace", c_int, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    ("tq_expect_z", c_int, [c_void_p, POINTER(c_uint64), c_int, POINTER(c_double)]),
    ("tq_probs", c_int, [c_void_p, POINTER(c_double)]),
    ("tq_measure", c_int, [c_void_p, c_int, c_double, POINTER(c_int), POINTER(c_double)]),
    ("tq_probs_readout", c_int, [c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_double)]),
    ("tq_sample", c_int, [c_void_p, POINTER(c_double), c_int, POINTER(c_double), POINTER(c_double),
                          POINTER(c_uint64)]),
    ("tq_program_create", c_int, [c_int, c_int, POINTER(TqOp), c_size_t, c_int, POINTER(c_void_p)]),
    ("tq_program_run", c_int, [c_void_p, c_void_p]),
    ("tq_program_info", c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_int), POINTER(c_size_t)]),
    ("tq_program_free", None, [c_void_p]),
    ("tq_expect_z_device", c_int, [c_void_p, c_void_p, c_int, c_void_p]),
    ("tq_batch_create", c_int, [c_int, c_void_p, POINTER(c_void_p)]),
    ("tq_batch_add", c_int, [c_void_p, c_int, POINTER(TqOp), c_size_t, c_int, POINTER(c_uint64), c_int,
                             POINTER(c_int)]),
    ("tq_batch_set_tile", c_int, [c_void_p, c_int, c_int]),
    ("tq_batch_run", c_int, [c_void_p]),
    ("tq_batch_test_wait_limit", c_int, [c_void_p, ctypes.c_longlong, c_int]),
    ("tq_batch_set_fp64_engine", c_int, [c_void_p, c_int]),
    ("tq_batch_tensor_jobs", c_int, [c_void_p, POINTER(c_size_t)]),
    ("tq_test_tc_wait_limit", c_int, [ctypes.c_longlong, c_int]),
    ("tq_batch_wait", c_int, [c_void_p]),
    ("tq_batch_result", c_int, [c_void_p, c_int, POINTER(c_double)]),
    ("tq_batch_get_rho", c_int, [c_void_p, c_int, POINTER(c_double)]),
    ("tq_batch_info", c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t), POINTER(c_size_t)]),
    ("tq_batch_work", c_int, [c_void_p, POINTER(c_double), POINTER(c_double)]),
    ("tq_batch_free", None, [c_void_p]),
    ("tq_autotune", c_int, [c_int, c_int, ctypes.c_char_p, POINTER(c_int), POINTER(c_int), POINTER(c_double)]),
    ("tq_autotune_engine", c_int, [c_int, c_int, c_int, ctypes.c_char_p, POINTER(c_int), POINTER(c_int),
                                   POINTER(c_double)]),
    ("tq_server_create", c_int, [c_int, c_void_p, c_size_t, c_size_t, c_int, POINTER(c_void_p)]),
    ("tq_server_submit", c_int, [c_void_p, c_int, POINTER(TqOp), c_size_t, c_int, POINTER(c_uint64), c_int,
                                 POINTER(c_int)]),
    ("tq_server_step", c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    ("tq_server_step_async", c_int, [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int)]),
    ("tq_server_gpu_ms", c_int, [c_void_p, POINTER(c_double)]),
    ("tq_server_set_fp64_engine", c_int, [c_void_p, c_int]),
    ("tq_server_poll", c_int, [c_void_p, c_int, POINTER(c_int), POINTER(c_double)]),
    ("tq_server_info", c_int, [c_void_p, POINTER(c_size_t), POINTER(ctypes.c_ulonglong),
                               POINTER(ctypes.c_ulonglong)]),
    ("tq_server_free", None, [c_void_p]),
    ("tq_expect_z_noalloc", c_int, [c_void_p, c_int, c_int, c_void_p, c_int, c_void_p, c_void_p]),
    ("tq_pipe_rate", c_int, [c_int, c_int, POINTER(c_double), POINTER(c_double)]),
    ("tq_profile_enable", c_int, [c_void_p, c_int]),
    ("tq_profile_read", c_int, [c_void_p, POINTER(TqKernelStat), c_int, POINTER(c_int)]),
    ("tq_launch_count", c_int, [c_void_p, POINTER(c_uint64)]),
    ("tq_gate_matrix", c_int, [c_int, POINTER(c_double), POINTER(c_int), POINTER(c_double)]),
    ("tq_channel_kraus", c_int, [c_int, c_int, POINTER(c_double), c_int, POINTER(c_int), POINTER(c_double)]),
    ("tq_plan_fusion", c_int, [c_int, POINTER(TqOp), c_size_t, c_int, c_int, POINTER(c_int), POINTER(c_int),
                               POINTER(c_size_t)]),
    ("tq_group_base", c_uint64, [c_uint64, POINTER(c_int), c_int]),
    ("tq_op_pattern", c_int, [POINTER(TqOp), POINTER(c_int), POINTER(c_int), POINTER(ctypes.c_uint16)]),
    ("tq_status_string", ctypes.c_char_p, [c_int]),
    ("tq_version", ctypes.c_char_p, []),
]


def load(path: str = LIB_PATH):
    """Load libtanq.so (raises if it is missing: build it first)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2404_13184_gb300.build.build() (or "
                           "__graft_entry__.build()) first; there is no fallback path")
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, what: str):
    if st != 0:
        raise TqError(st, what)


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(POINTER(c_double))


def _mats_array(mats) -> np.ndarray:
    arr = np.ascontiguousarray(np.stack([np.asarray(m, dtype=np.complex128) for m in mats]))
    return arr.view(np.float64).reshape(-1)


class Program:
    """Ops marshalled into a tq_op array (kept alive with their matrices)."""

    def __init__(self, ops):
        self.n_ops = len(ops)
        self.arr = (TqOp * max(1, len(ops)))()
        self._keep = []
        for i, (name, qubits, params) in enumerate(ops):
            o = self.arr[i]
            o.k = len(qubits)
            for j, q in enumerate(qubits):
                o.qubits[j] = int(q)
            if name in GATES:
                o.kind, o.name = OP_GATE, GATES[name]
                for j, v in enumerate(params):
                    o.params[j] = float(v)
            elif name in CHANNELS:
                o.kind, o.name = OP_CHANNEL, CHANNELS[name]
                for j, v in enumerate(params):
                    o.params[j] = float(v)
            elif name in ("unitary", "kraus"):
                m = _mats_array(params)
                self._keep.append(m)
                o.kind = OP_UNITARY if name == "unitary" else OP_KRAUS
                o.m = len(params)
                o.mats = _dptr(m)
            else:
                raise ValueError(f"unknown op {name!r}")


class DeviceProgram:
    """A circuit planned and uploaded to device memory once (tq_program)."""

    def __init__(self, n: int, ops, width: int = -1, precision: str = "fp64"):
        lib = load()
        prog = ops if isinstance(ops, Program) else Program(ops)
        self.n, self.precision = n, precision
        self._h = c_void_p()
        _check(lib.tq_program_create(n, PRECISION[precision], prog.arr, prog.n_ops, width, ctypes.byref(self._h)),
               "tq_program_create")
        no, nb, mw, tb = c_size_t(0), c_size_t(0), c_int(0), c_size_t(0)
        _check(lib.tq_program_info(self._h, ctypes.byref(no), ctypes.byref(nb), ctypes.byref(mw), ctypes.byref(tb)),
               "tq_program_info")
        self.n_ops, self.n_blocks, self.max_width, self.table_bytes = no.value, nb.value, mw.value, tb.value

    def free(self):
        if self._h:
            _lib.tq_program_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """Many independent circuits run in one persistent launch (tq_batch)."""

    def __init__(self, precision: str = "fp64", stream=None, engine: str = "auto"):
        lib = load()
        self.precision = precision
        torch = _torch_plumbing()
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        self._h = c_void_p()
        self._nmasks = []
        self._n = []
        _check(lib.tq_batch_create(PRECISION[precision], c_void_p(stream), ctypes.byref(self._h)), "tq_batch_create")
        if engine != "auto":
            self.set_fp64_engine(engine)

    def set_fp64_engine(self, engine: str):
        """Engine of the tile jobs: "auto" / "tensor" (tensor cores) or "dfma" (the persistent kernel)."""
        _check(_lib.tq_batch_set_fp64_engine(self._h, ENGINES[engine]), "tq_batch_set_fp64_engine")

    def tensor_jobs(self) -> int:
        """Jobs of the last planned run on a batched tensor-core pass."""
        v = c_size_t(0)
        _check(_lib.tq_batch_tensor_jobs(self._h, ctypes.byref(v)), "tq_batch_tensor_jobs")
        return v.value

    def add(self, n: int, ops, width: int = -1, masks=()) -> int:
        prog = ops if isinstance(ops, Program) else Program(ops)
        m = (c_uint64 * max(1, len(masks)))(*[int(v) for v in masks])
        j = c_int(0)
        _check(_lib.tq_batch_add(self._h, n, prog.arr, prog.n_ops, width, m, len(masks), ctypes.byref(j)),
               "tq_batch_add")
        self._nmasks.append(len(masks))
        self._n.append(n)
        return j.value

    def set_tile(self, n: int, tile_log2: int):
        _check(_lib.tq_batch_set_tile(self._h, n, tile_log2), "tq_batch_set_tile")

    def run(self):
        _check(_lib.tq_batch_run(self._h), "tq_batch_run")

    def test_wait_limit(self, max_spin: int, never_ready_job: int = -1):
        _check(_lib.tq_batch_test_wait_limit(self._h, max_spin, never_ready_job), "tq_batch_test_wait_limit")

    def wait(self):
        _check(_lib.tq_batch_wait(self._h), "tq_batch_wait")

    def result(self, job: int) -> np.ndarray:
        out = np.zeros(2 + self._nmasks[job])
        _check(_lib.tq_batch_result(self._h, job, _dptr(out)), "tq_batch_result")
        return out

    def rho(self, job: int) -> np.ndarray:
        n = self._n[job]
        N = 1 << n
        out = np.zeros(2 << (2 * n))
        _check(_lib.tq_batch_get_rho(self._h, job, _dptr(out)), "tq_batch_get_rho")
        return out.view(np.complex128).reshape(N, N).T.copy()

    def info(self):
        a, b, c = c_size_t(0), c_size_t(0), c_size_t(0)
        _check(_lib.tq_batch_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "tq_batch_info")
        return {"jobs": a.value, "items": b.value, "rho_bytes": c.value}

    def work(self) -> dict:
        """Algorithmic flops and HBM bytes of one run (after a run)."""
        f, by = c_double(), c_double()
        _check(_lib.tq_batch_work(self._h, ctypes.byref(f), ctypes.byref(by)), "tq_batch_work")
        return {"flops": f.value, "bytes": by.value}

    def free(self):
        if self._h:
            _lib.tq_batch_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def autotune(precision: str, n: int, cache_path: str | None = None, engine: str = "auto"):
    """(tile_log2, fusion width, ms per run) for the batch engine at n qubits
    (FP64: on the given engine)."""
    lib = load()
    t, w, ms = c_int(0), c_int(0), c_double(0)
    path = cache_path.encode() if cache_path else None
    if engine == "auto":
        _check(lib.tq_autotune(PRECISION[precision], n, path, ctypes.byref(t), ctypes.byref(w), ctypes.byref(ms)),
               "tq_autotune")
    else:
        _check(lib.tq_autotune_engine(PRECISION[precision], ENGINES[engine], n, path, ctypes.byref(t),
                                      ctypes.byref(w), ctypes.byref(ms)), "tq_autotune_engine")
    return t.value, w.value, ms.value


class Server:
    """Continuous-batching serving loop (tq_server)."""

    def __init__(self, precision: str = "fp64", rho_budget: int = 1 << 30, table_budget: int = 1 << 28,
                 max_live: int = 64, stream=None, engine: str | None = None):
        lib = load()
        self.precision = precision
        torch = _torch_plumbing()
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        self._h = c_void_p()
        self._nmasks = {}
        _check(lib.tq_server_create(PRECISION[precision], c_void_p(stream), rho_budget, table_budget, max_live,
                                    ctypes.byref(self._h)), "tq_server_create")
        if engine is not None:
            self.set_fp64_engine(engine)

    def submit(self, n: int, ops, width: int = -1, masks=()) -> int:
        prog = ops if isinstance(ops, Program) else Program(ops)
        m = (c_uint64 * max(1, len(masks)))(*[int(v) for v in masks])
        rid = c_int(0)
        _check(_lib.tq_server_submit(self._h, n, prog.arr, prog.n_ops, width, m, len(masks), ctypes.byref(rid)),
               "tq_server_submit")
        self._nmasks[rid.value] = len(masks)
        return rid.value

    def step(self):
        a, b, c = c_int(0), c_int(0), c_int(0)
        _check(_lib.tq_server_step(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "tq_server_step")
        return a.value, b.value, c.value

    def set_fp64_engine(self, engine: str):
        """'auto', 'dfma' or 'tensor' (tq_server_set_fp64_engine)."""
        _check(_lib.tq_server_set_fp64_engine(self._h, ENGINES[engine]), "tq_server_set_fp64_engine")

    def step_async(self):
        """Collect the previous tick, launch the next one, return at once:
        (live after the launched tick, queued, finished by the collected tick)."""
        a, b, c = c_int(0), c_int(0), c_int(0)
        _check(_lib.tq_server_step_async(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "tq_server_step_async")
        return a.value, b.value, c.value

    def gpu_ms(self) -> float:
        v = c_double(0.0)
        _check(_lib.tq_server_gpu_ms(self._h, ctypes.byref(v)), "tq_server_gpu_ms")
        return v.value

    def poll(self, rid: int):
        st = c_int(0)
        out = np.zeros(2 + self._nmasks[rid])
        _check(_lib.tq_server_poll(self._h, rid, ctypes.byref(st), _dptr(out)), "tq_server_poll")
        return st.value, (out if st.value == 2 else None)

    def info(self):
        a, b, c = c_size_t(0), ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
        _check(_lib.tq_server_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "tq_server_info")
        return {"rho_live_bytes": a.value, "ticks": b.value, "blocks_applied": c.value}

    def free(self):
        if self._h:
            _lib.tq_server_free(self._h)
            self._h = c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def test_tc_wait_limit(max_tries: int, skip_mma: bool = False):
    """Failure-path test hook of the split tensor-core pass (see
    tq_test_tc_wait_limit): max_tries 0 restores the default."""
    _check(load().tq_test_tc_wait_limit(max_tries, 1 if skip_mma else 0), "tq_test_tc_wait_limit")


def plan_fusion(n: int, ops, width: int, precision: str = "fp64"):
    """(block index of every op, width of every block) from the library's planner."""
    lib = load()
    prog = ops if isinstance(ops, Program) else Program(ops)
    boo = (c_int * max(1, prog.n_ops))()
    bw = (c_int * max(1, prog.n_ops))()
    nb = c_size_t(0)
    _check(lib.tq_plan_fusion(n, prog.arr, prog.n_ops, width, PRECISION[precision], boo, bw, ctypes.byref(nb)),
           "tq_plan_fusion")
    return list(boo[:prog.n_ops]), list(bw[:nb.value])


def gate_matrix(name: str, params=()) -> np.ndarray:
    lib = load()
    p = np.zeros(4)
    p[:len(params)] = params
    out = np.zeros(32)
    k = c_int(0)
    _check(lib.tq_gate_matrix(GATES[name], _dptr(p), ctypes.byref(k), _dptr(out)), "tq_gate_matrix")
    d = 1 << k.value
    return out[:2 * d * d].view(np.complex128).reshape(d, d)


def channel_kraus(name: str, k: int, params) -> list[np.ndarray]:
    lib = load()
    p = np.zeros(4)
    p[:len(params)] = params
    m = c_int(0)
    _check(lib.tq_channel_kraus(CHANNELS[name], k, _dptr(p), 0, ctypes.byref(m), None), "tq_channel_kraus")
    d = 1 << k
    out = np.zeros(m.value * 2 * d * d)
    _check(lib.tq_channel_kraus(CHANNELS[name], k, _dptr(p), m.value, ctypes.byref(m), _dptr(out)), "tq_channel_kraus")
    arr = out.view(np.complex128).reshape(m.value, d, d)
    return [arr[i] for i in range(m.value)]


ENGINES = {"auto": 0, "dfma": 1, "tensor": 2}
PIPES = {"dfma": 0, "dmma": 1, "ffma": 2, "cvt_f64_s64": 3, "cvt_f64_f32": 4}


def pipe_rate(pipe: str, iters: int = 2048):
    """Measured issue rate of an arithmetic pipe on the current device (see
    tq_pipe_rate in include/tanq.h): (ops or flops per second, ms of the best
    launch)."""
    lib = load()
    r, ms = c_double(0.0), c_double(0.0)
    _check(lib.tq_pipe_rate(PIPES[pipe], iters, ctypes.byref(r), ctypes.byref(ms)), "tq_pipe_rate")
    return r.value, ms.value


def expect_z_noalloc(rho_dev_ptr: int, n: int, precision: str, masks_dev_ptr: int, n_masks: int,
                     out_dev_ptr: int, stream=None):
    """Allocation-free <Z> readout on caller-owned device buffers (see
    tq_expect_z_noalloc in include/tanq.h)."""
    lib = load()
    _check(lib.tq_expect_z_noalloc(c_void_p(rho_dev_ptr), n, PRECISION[precision], c_void_p(masks_dev_ptr), n_masks,
                                   c_void_p(out_dev_ptr), c_void_p(stream)), "tq_expect_z_noalloc")


def op_pattern(op) -> np.ndarray:
    """Boolean 4^k x 4^k structural pattern of an op's superoperator."""
    lib = load()
    prog = Program([op])
    w, nnz = c_int(0), c_int(0)
    rows = (ctypes.c_uint16 * 16)()
    _check(lib.tq_op_pattern(prog.arr, ctypes.byref(w), ctypes.byref(nnz), rows), "tq_op_pattern")
    D = 1 << (2 * w.value)
    return np.array([[(rows[i] >> j) & 1 for j in range(D)] for i in range(D)], dtype=bool)


def group_base(g: int, positions) -> int:
    lib = load()
    pos = (c_int * len(positions))(*positions)
    return int(lib.tq_group_base(g, pos, len(positions)))


def _torch_plumbing():
    try:
        import torch
        if torch.cuda.is_available():
            return torch
    except Exception:
        pass
    return None


class State:
    """A density matrix on the GPU (tq_state)."""

    def __init__(self, n: int, precision: str = "fp64", stream=None, torch_memory: bool = True,
                 hermitian: bool = True, engine: str | None = None):
        lib = load()
        self.n = n
        self.precision = precision
        self._buf = None
        self._h = c_void_p()
        torch = _torch_plumbing()
        if stream is None and torch is not None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = stream
        prec = PRECISION[precision]
        if torch_memory and torch is not None:
            nbytes = (16 if precision == "fp64" else 8) << (2 * n)
            self._buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
            _check(lib.tq_create_on(n, prec, c_void_p(stream), c_void_p(self._buf.data_ptr()), nbytes,
                                    ctypes.byref(self._h)), "tq_create_on")
        else:
            _check(lib.tq_create(n, prec, c_void_p(stream), ctypes.byref(self._h)), "tq_create")
        if not hermitian:
            _check(lib.tq_set_hermitian(self._h, 0), "tq_set_hermitian")
        if engine is not None:
            self.set_fp64_engine(engine)

    def set_hermitian(self, on: bool):
        _check(_lib.tq_set_hermitian(self._h, 1 if on else 0), "tq_set_hermitian")

    def set_fp64_engine(self, engine: str):
        """'auto', 'dfma' or 'tensor' (tq_set_fp64_engine)."""
        _check(_lib.tq_set_fp64_engine(self._h, ENGINES[engine]), "tq_set_fp64_engine")

    def fp64_on_tensor(self) -> bool:
        v = c_int(0)
        _check(_lib.tq_fp64_on_tensor(self._h, ctypes.byref(v)), "tq_fp64_on_tensor")
        return bool(v.value)

    def hermitian_mode(self) -> bool:
        v = c_int(0)
        _check(_lib.tq_is_hermitian_mode(self._h, ctypes.byref(v)), "tq_is_hermitian_mode")
        return bool(v.value)

    # -- lifetime
    def free(self):
        if self._h:
            _lib.tq_free(self._h)
            self._h = c_void_p()
        self._buf = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.free()

    # -- evolution
    def run(self, ops, width: int = -1) -> int:
        prog = ops if isinstance(ops, Program) else Program(ops)
        nb = c_size_t(0)
        _check(_lib.tq_run_circuit(self._h, prog.arr, prog.n_ops, width, ctypes.byref(nb)), "tq_run_circuit")
        return nb.value

    def run_program(self, prog: "DeviceProgram"):
        _check(_lib.tq_program_run(self._h, prog._h), "tq_program_run")

    def expect_z_device(self, masks_dev_ptr: int, n_masks: int, out_dev_ptr: int):
        _check(_lib.tq_expect_z_device(self._h, c_void_p(masks_dev_ptr), n_masks, c_void_p(out_dev_ptr)),
               "tq_expect_z_device")

    def profile(self, on: bool = True):
        _check(_lib.tq_profile_enable(self._h, 1 if on else 0), "tq_profile_enable")

    def profile_stats(self) -> dict:
        arr = (TqKernelStat * 32)()
        cnt = c_int(0)
        _check(_lib.tq_profile_read(self._h, arr, 32, ctypes.byref(cnt)), "tq_profile_read")
        return {arr[i].name.decode(): {"launches": int(arr[i].launches), "total_ms": float(arr[i].total_ms),
                                       "flops": float(arr[i].flops), "bytes": float(arr[i].bytes)}
                for i in range(min(cnt.value, 32))}

    def launch_count(self) -> int:
        v = c_uint64(0)
        _check(_lib.tq_launch_count(self._h, ctypes.byref(v)), "tq_launch_count")
        return int(v.value)

    def apply_gate(self, qubits, U):
        q = (c_int * len(qubits))(*qubits)
        m = _mats_array([U])
        _check(_lib.tq_apply_gate(self._h, q, len(qubits), _dptr(m)), "tq_apply_gate")

    def apply_kraus(self, qubits, kraus):
        q = (c_int * len(qubits))(*qubits)
        m = _mats_array(kraus)
        _check(_lib.tq_apply_kraus(self._h, q, len(qubits), len(kraus), _dptr(m)), "tq_apply_kraus")

    def reset(self):
        _check(_lib.tq_reset(self._h), "tq_reset")

    # -- readouts
    def trace(self) -> complex:
        re, im = c_double(), c_double()
        _check(_lib.tq_trace(self._h, ctypes.byref(re), ctypes.byref(im)), "tq_trace")
        return complex(re.value, im.value)

    def expect_z(self, masks) -> np.ndarray:
        masks = [int(m) for m in masks]
        arr = (c_uint64 * max(1, len(masks)))(*masks)
        out = np.zeros(max(1, len(masks)))
        _check(_lib.tq_expect_z(self._h, arr, len(masks), _dptr(out)), "tq_expect_z")
        return out[:len(masks)]

    def probs(self) -> np.ndarray:
        out = np.zeros(1 << self.n)
        _check(_lib.tq_probs(self._h, _dptr(out)), "tq_probs")
        return out

    def measure(self, qubit: int, u: float):
        """(outcome, probability) of a selective measurement; rho collapses."""
        m, p = c_int(0), c_double(0)
        _check(_lib.tq_measure(self._h, qubit, float(u), ctypes.byref(m), ctypes.byref(p)), "tq_measure")
        return m.value, p.value

    def probs_readout(self, e10, e01) -> np.ndarray:
        a = np.ascontiguousarray(e10, dtype=np.float64)
        b = np.ascontiguousarray(e01, dtype=np.float64)
        out = np.zeros(1 << self.n)
        _check(_lib.tq_probs_readout(self._h, _dptr(a), _dptr(b), _dptr(out)), "tq_probs_readout")
        return out

    def sample(self, uniforms, e10=None, e01=None) -> np.ndarray:
        u = np.ascontiguousarray(uniforms, dtype=np.float64)
        out = np.zeros(len(u), dtype=np.uint64)
        a = None if e10 is None else np.ascontiguousarray(e10, dtype=np.float64)
        b = None if e01 is None else np.ascontiguousarray(e01, dtype=np.float64)
        _check(_lib.tq_sample(self._h, _dptr(u), len(u), None if a is None else _dptr(a),
                              None if b is None else _dptr(b), out.ctypes.data_as(POINTER(c_uint64))), "tq_sample")
        return out

    def vec(self) -> np.ndarray:
        out = np.zeros(2 << (2 * self.n))
        _check(_lib.tq_get_rho(self._h, _dptr(out)), "tq_get_rho")
        return out.view(np.complex128)

    def rho(self) -> np.ndarray:
        """rho[r, c] from vec(rho) (column-stacked: vec index r + c 2^n)."""
        N = 1 << self.n
        return self.vec().reshape(N, N).T.copy()

    def set_rho(self, rho: np.ndarray):
        N = 1 << self.n
        v = np.ascontiguousarray(np.asarray(rho, dtype=np.complex128).T).reshape(N * N)
        flat = v.view(np.float64)
        _check(_lib.tq_set_rho(self._h, _dptr(flat)), "tq_set_rho")

    def device_ptr(self) -> int:
        p = c_void_p()
        _check(_lib.tq_rho_device_ptr(self._h, ctypes.byref(p)), "tq_rho_device_ptr")
        return p.value
