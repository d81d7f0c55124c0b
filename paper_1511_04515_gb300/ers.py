"""Python binding of libers (include/ers.h): argument marshalling only.

Every step of the transient runs in the library's CUDA kernels; this module converts
numpy / scipy.sparse inputs into the C structures, passes PyTorch's CUDA stream through when
asked, and raises ErsError on any non-OK status.  There is no CPU fallback: if libers.so is
missing or no GPU is present, the calls fail loudly.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libers.so")

STATUS = {0: "OK", 1: "INVALID", 2: "SINGULAR", 3: "NONFINITE", 4: "STEP_UNDERFLOW",
          5: "KRYLOV", 6: "TIMEOUT", 7: "CUDA", 8: "OOM"}


class ErsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"ers status {STATUS.get(status, status)}: {msg}")
        self.status = status


class Csr(C.Structure):
    _fields_ = [("n_rows", C.c_int32), ("n_cols", C.c_int32), ("nnz", C.c_int32),
                ("rowptr", C.POINTER(C.c_int32)), ("colidx", C.POINTER(C.c_int32)),
                ("val", C.POINTER(C.c_double))]


class Mosfet(C.Structure):
    _fields_ = [("type", C.c_int32), ("d", C.c_int32), ("g", C.c_int32), ("s", C.c_int32),
                ("vt", C.c_double), ("k", C.c_double), ("lam", C.c_double)]


class Pwl(C.Structure):
    _fields_ = [("npts", C.c_int32), ("t", C.POINTER(C.c_double)), ("v", C.POINTER(C.c_double))]


class Opts(C.Structure):
    _fields_ = [("eps_krylov", C.c_double), ("E_rr", C.c_double), ("alpha", C.c_double),
                ("beta", C.c_double), ("gamma", C.c_double), ("h_min", C.c_double),
                ("h_max", C.c_double), ("h_init", C.c_double), ("vdd", C.c_double),
                ("gmin", C.c_double),
                ("i_grow", C.c_int32), ("m_min", C.c_int32), ("m_max", C.c_int32),
                ("combined_vector", C.c_int32), ("correction", C.c_int32),
                ("ordering", C.c_int32)]


class Instance(C.Structure):
    _fields_ = [("G", C.POINTER(Csr)), ("C", C.POINTER(Csr)), ("B", C.POINTER(Csr)),
                ("dev", C.POINTER(Mosfet)), ("ndev", C.c_int32), ("u", C.POINTER(Pwl)),
                ("p", C.c_int32)]


class StepRecord(C.Structure):
    _fields_ = [("h", C.c_double), ("h_max", C.c_double), ("err", C.c_double), ("E", C.c_double),
                ("dF", C.c_double), ("m", C.c_int32), ("m_max", C.c_int32),
                ("landed", C.c_int32), ("retries", C.c_int32)]


CTRL_HISTORY = 8
CTRL_FEATURES = 32


class Stats(C.Structure):
    _fields_ = [("steps", C.c_int64), ("rejects", C.c_int64), ("refactors", C.c_int64),
                ("krylov_vectors", C.c_int64), ("solves", C.c_int64),
                ("n", C.c_int32), ("nsn", C.c_int32), ("nlevels", C.c_int32),
                ("etree_height", C.c_int32), ("max_front", C.c_int32),
                ("nnz_L", C.c_int64), ("factor_doubles", C.c_int64),
                ("arena_doubles", C.c_int64), ("refactor_flops", C.c_double),
                ("kernel_launches", C.c_int64), ("solve_passes", C.c_int64),
                ("solve_rhs", C.c_int64), ("solve_ms", C.c_double),
                ("solve_bytes_per_pass", C.c_double), ("solve_fma_per_rhs", C.c_double),
                ("graph_launches", C.c_int64), ("merged_blocks", C.c_int64),
                ("merged_columns", C.c_int64), ("merged_inverse_doubles", C.c_int64),
                ("merged_inverse_flops", C.c_double), ("host_syncs", C.c_int64),
                ("host_polls", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


EXPORTS = ["ers_default_opts", "ers_create", "ers_set_stream", "ers_dc", "ers_refactor",
           "ers_step", "ers_run", "ers_get_state", "ers_set_state", "ers_get_state_dev",
           "ers_set_state_dev", "ers_solve", "ers_spmv_C", "ers_mevp", "ers_phi_small",
           "ers_stats", "ers_profile", "ers_analyze", "ers_last_error", "ers_destroy",
           "ers_solve_dev_noalloc", "ers_create_batch", "ers_run_batch", "ers_get_state_inst",
           "ers_ctrl_features", "ers_ctrl_target", "ers_mlp_nparam", "ers_mlp_create",
           "ers_mlp_set_params", "ers_mlp_get_params", "ers_mlp_forward", "ers_mlp_forward_dev",
           "ers_mlp_grad", "ers_mlp_adam_step", "ers_mlp_train", "ers_mlp_last_error",
           "ers_mlp_destroy", "ers_batch_set_controller", "ers_batch_trace", "ers_batch_records",
           "ers_batch_samples", "ers_batch_ctrl_stats", "ers_ctrl_propose",
           "ers_batch_set_graphs", "ers_autotune", "ers_solve_plan_check",
           "ers_wait_selftest", "ers_plan_array", "ers_partition_lpt", "ers_fp64_fma_peak",
           "ers_pwl_ramp"]

_lib = None


def lib():
    """Load libers.so (built by paper_1511_04515_gb300.build.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise OSError(f"{LIB_PATH} is missing: run paper_1511_04515_gb300.build.build() first")
    L = C.CDLL(LIB_PATH)
    P, D, I32 = C.c_void_p, C.c_double, C.c_int32
    pd = C.POINTER(C.c_double)
    pi = C.POINTER(C.c_int32)
    pf = C.POINTER(C.c_float)
    sig = {
        "ers_default_opts": ([C.POINTER(Opts)], C.c_int),
        "ers_create": ([C.POINTER(P), C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr),
                        C.POINTER(Mosfet), I32, C.POINTER(Pwl), I32, pi, I32, C.POINTER(Opts)],
                       C.c_int),
        "ers_set_stream": ([P, P], C.c_int),
        "ers_dc": ([P, pd], C.c_int),
        "ers_refactor": ([P], C.c_int),
        "ers_step": ([P, D, I32, pi, pd], C.c_int),
        "ers_run": ([P, D, D, I32, pi, pi], C.c_int),
        "ers_get_state": ([P, pd, pd, pd], C.c_int),
        "ers_set_state": ([P, D, pd, D], C.c_int),
        "ers_get_state_dev": ([P, P], C.c_int),
        "ers_set_state_dev": ([P, D, P, D], C.c_int),
        "ers_solve": ([P, pd, pd], C.c_int),
        "ers_spmv_C": ([P, pd, pd], C.c_int),
        "ers_mevp": ([P, pd, D, I32, pd, pi], C.c_int),
        "ers_phi_small": ([P, pd, I32, I32, D, pd, pd], C.c_int),
        "ers_stats": ([P, C.POINTER(Stats)], C.c_int),
        "ers_autotune": ([P, I32, I32, pd, pi], C.c_int),
        "ers_wait_selftest": ([P], C.c_int),
        "ers_profile": ([P, I32], C.c_int),
        "ers_solve_dev_noalloc": ([P, P, P], C.c_int),
        "ers_create_batch": ([C.POINTER(P), C.POINTER(Instance), I32, pi, I32, C.POINTER(Opts)],
                             C.c_int),
        "ers_partition_lpt": ([pd, I32, I32, pi], C.c_int),
        "ers_pwl_ramp": ([C.POINTER(Pwl), I32, D, D, pi], C.c_int),
        "ers_fp64_fma_peak": ([I32, pd], C.c_int),
        "ers_run_batch": ([P, D, D, I32, pi, pi], C.c_int),
        "ers_get_state_inst": ([P, I32, pd, pd, pd], C.c_int),
        "ers_analyze": ([C.POINTER(Csr), C.POINTER(Opts), C.POINTER(Stats), pi], C.c_int),
        "ers_plan_array": ([C.POINTER(Csr), C.POINTER(Opts), C.c_int32, C.c_void_p,
                            C.POINTER(C.c_int64)], C.c_int),
        "ers_solve_plan_check": ([C.POINTER(Csr), C.POINTER(Opts), C.POINTER(C.c_int64)],
                                 C.c_int),
        "ers_ctrl_features": ([C.POINTER(StepRecord), I32, pf], C.c_int),
        "ers_ctrl_target": ([C.POINTER(StepRecord), I32, C.POINTER(StepRecord), pf], C.c_int),
        "ers_ctrl_propose": ([pf, C.POINTER(StepRecord), D, I32, pd, pi], C.c_int),
        "ers_mlp_nparam": ([], I32),
        "ers_mlp_create": ([C.POINTER(P), C.c_uint64], C.c_int),
        "ers_mlp_set_params": ([P, pf], C.c_int),
        "ers_mlp_get_params": ([P, pf], C.c_int),
        "ers_mlp_forward": ([P, pf, I32, pf], C.c_int),
        "ers_mlp_forward_dev": ([P, P, I32, P, P], C.c_int),
        "ers_mlp_grad": ([P, pf, pf, I32, pf, pf], C.c_int),
        "ers_mlp_adam_step": ([P, pf, pf, I32, C.c_float, pf], C.c_int),
        "ers_mlp_train": ([P, pf, pf, I32, I32, I32, C.c_float, C.c_uint64, pf], C.c_int),
        "ers_mlp_last_error": ([P], C.c_char_p),
        "ers_mlp_destroy": ([P], None),
        "ers_batch_set_controller": ([P, P, I32, D], C.c_int),
        "ers_batch_trace": ([P, I32], C.c_int),
        "ers_batch_set_graphs": ([P, I32], C.c_int),
        "ers_batch_records": ([P, I32, C.POINTER(StepRecord), I32, pi], C.c_int),
        "ers_batch_samples": ([P, pf, pf, I32, pi], C.c_int),
        "ers_batch_ctrl_stats": ([P, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                  C.POINTER(C.c_int64)], C.c_int),
        "ers_last_error": ([P], C.c_char_p),
        "ers_destroy": ([P], None),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def _device_list(devices):
    """(int32 pointer or None, count) for a device list argument; keeps the array alive on
    the returned pointer's _keep attribute."""
    if not devices:
        return None, 0
    arr = np.ascontiguousarray(np.asarray(devices, np.int32))
    ptr = arr.ctypes.data_as(C.POINTER(C.c_int32))
    ptr._keep = arr
    return ptr, int(arr.size)


def fp64_fma_peak(device: int = 0) -> float:
    """Measured FP64 FMA rate of a device in TFLOP/s (see ers.h)."""
    v = C.c_double(0.0)
    rc = lib().ers_fp64_fma_peak(int(device), C.byref(v))
    if rc != 0:
        raise ErsError(rc, "FP64 peak probe failed")
    return v.value


def partition_lpt(costs, nparts: int) -> np.ndarray:
    """Part of each job under longest-processing-time-first over nparts parts (host-only;
    the device split of ers_create_batch, see ers.h)."""
    c = np.ascontiguousarray(np.asarray(costs, np.float64))
    out = np.zeros(c.size, np.int32)
    rc = lib().ers_partition_lpt(_dptr(c), int(c.size), int(nparts), _iptr(out))
    if rc != 0:
        raise ErsError(rc, "partition: costs must be finite and >= 0, nparts >= 1")
    return out


def pwl_ramp(pwl: Sequence, t: float, h: float) -> bool:
    """The set-up step's ramp test on the host (see ers.h): True when some of the PWL inputs
    (a sequence of (times, values)) has pwl(t + h) != pwl(t)."""
    hold = [(np.ascontiguousarray(tt, np.float64), np.ascontiguousarray(vv, np.float64))
            for tt, vv in pwl]
    pw = (Pwl * max(1, len(hold)))()
    for q, (tt, vv) in enumerate(hold):
        pw[q] = Pwl(int(tt.size), _dptr(tt), _dptr(vv))
    out = np.zeros(1, np.int32)
    rc = lib().ers_pwl_ramp(pw, len(hold), float(t), float(h), _iptr(out))
    if rc != 0:
        raise ErsError(rc, "pwl_ramp: corner times must increase")
    return bool(out[0])


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _iptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _fptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def _records(recs) -> C.Array:
    """Sequence of dicts / tuples (h, h_max, err, E, dF, m, m_max, landed, retries) -> array."""
    arr = (StepRecord * max(len(recs), 1))()
    for q, r in enumerate(recs):
        if isinstance(r, dict):
            arr[q] = StepRecord(**r)
        else:
            arr[q] = StepRecord(*r)
    return arr


def ctrl_features(recs) -> np.ndarray:
    """Network input of the learned controller from a step history (host-only, see ers.h)."""
    arr = _records(recs)
    out = np.zeros(CTRL_FEATURES, np.float32)
    rc = lib().ers_ctrl_features(arr, len(recs), _fptr(out))
    if rc != 0:
        raise ErsError(rc, "ers_ctrl_features")
    return out


def ctrl_target(recs, nxt):
    """Training target (2 floats) of the step after recs[-1], or None if unusable."""
    arr = _records(recs)
    nx = _records([nxt])
    out = np.zeros(2, np.float32)
    rc = lib().ers_ctrl_target(arr, len(recs), nx, _fptr(out))
    return out if rc == 0 else None


def ctrl_propose(y, last, margin=0.0, m_min=3):
    """(h_next, m_start) from a network output and the last accepted step (see ers.h)."""
    yy = np.ascontiguousarray(y, np.float32)
    lr = _records([last])
    h = C.c_double(0.0)
    m = C.c_int32(0)
    rc = lib().ers_ctrl_propose(_fptr(yy), lr, float(margin), int(m_min), C.byref(h), C.byref(m))
    if rc != 0:
        raise ErsError(rc, "ers_ctrl_propose")
    return h.value, m.value


class Mlp:
    """The learned controller's network (ers_mlp_*): BF16 tensor-core forward/backward and Adam."""

    def __init__(self, seed: int = 0):
        L = lib()
        self.nparam = int(L.ers_mlp_nparam())
        self._h = C.c_void_p()
        rc = L.ers_mlp_create(C.byref(self._h), int(seed))
        if rc != 0:
            msg = L.ers_mlp_last_error(self._h).decode() if self._h else ""
            if self._h:
                L.ers_mlp_destroy(self._h)
            self._h = None
            raise ErsError(rc, msg)

    @property
    def handle(self):
        return self._h

    def _check(self, rc):
        if rc != 0:
            raise ErsError(rc, lib().ers_mlp_last_error(self._h).decode())

    def close(self):
        if self._h:
            lib().ers_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        p = np.zeros(self.nparam, np.float32)
        self._check(lib().ers_mlp_get_params(self._h, _fptr(p)))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.nparam
        self._check(lib().ers_mlp_set_params(self._h, _fptr(p)))

    def forward(self, X) -> np.ndarray:
        X = np.ascontiguousarray(X, np.float32).reshape(-1, CTRL_FEATURES)
        Y = np.zeros((X.shape[0], 2), np.float32)
        self._check(lib().ers_mlp_forward(self._h, _fptr(X), X.shape[0], _fptr(Y)))
        return Y

    def forward_dev(self, x_ptr: int, n: int, y_ptr: int, stream=None):
        handle = getattr(stream, "cuda_stream", stream)
        self._check(lib().ers_mlp_forward_dev(self._h, C.c_void_p(x_ptr), int(n),
                                              C.c_void_p(y_ptr),
                                              C.c_void_p(handle) if handle else None))

    def grad(self, X, T):
        X = np.ascontiguousarray(X, np.float32).reshape(-1, CTRL_FEATURES)
        T = np.ascontiguousarray(T, np.float32).reshape(-1, 2)
        g = np.zeros(self.nparam, np.float32)
        loss = C.c_float(0.0)
        self._check(lib().ers_mlp_grad(self._h, _fptr(X), _fptr(T), X.shape[0], _fptr(g),
                                       C.byref(loss)))
        return g, loss.value

    def adam_step(self, X, T, lr: float = 1e-3) -> float:
        X = np.ascontiguousarray(X, np.float32).reshape(-1, CTRL_FEATURES)
        T = np.ascontiguousarray(T, np.float32).reshape(-1, 2)
        loss = C.c_float(0.0)
        self._check(lib().ers_mlp_adam_step(self._h, _fptr(X), _fptr(T), X.shape[0], float(lr),
                                            C.byref(loss)))
        return loss.value

    def train(self, X, T, epochs: int = 50, batch: int = 256, lr: float = 1e-3,
              seed: int = 0) -> float:
        X = np.ascontiguousarray(X, np.float32).reshape(-1, CTRL_FEATURES)
        T = np.ascontiguousarray(T, np.float32).reshape(-1, 2)
        loss = C.c_float(0.0)
        self._check(lib().ers_mlp_train(self._h, _fptr(X), _fptr(T), X.shape[0], int(epochs),
                                        int(batch), float(lr), int(seed), C.byref(loss)))
        return loss.value


class _CsrHold:
    """Keeps the numpy arrays of a CSR alive while the C structure points at them."""

    def __init__(self, mat, shape=None):
        indptr = np.ascontiguousarray(mat.indptr, dtype=np.int32)
        indices = np.ascontiguousarray(mat.indices, dtype=np.int32)
        data = np.ascontiguousarray(mat.data, dtype=np.float64)
        rows, cols = shape if shape is not None else mat.shape
        self.arrays = (indptr, indices, data)
        self.c = Csr(int(rows), int(cols), int(indices.size), _iptr(indptr), _iptr(indices),
                     _dptr(data))


def default_opts() -> Opts:
    o = Opts()
    lib().ers_default_opts(C.byref(o))
    return o


def make_opts(**kw) -> Opts:
    o = default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def analyze(pattern, ordering: Optional[int] = None) -> dict:
    """Host-only symbolic analysis of a square CSR pattern (no GPU needed); ordering as the
    field of ers_opts."""
    h = _CsrHold(pattern)
    st = Stats()
    n = pattern.shape[0]
    perm = np.zeros(n, np.int32)
    o = make_opts() if ordering is None else make_opts(ordering=ordering)
    rc = lib().ers_analyze(C.byref(h.c), C.byref(o), C.byref(st), _iptr(perm))
    if rc != 0:
        raise ErsError(rc, "symbolic analysis failed")
    d = st.as_dict()
    d["perm"] = perm
    return d


def solve_plan_check(pattern, ordering: Optional[int] = None) -> dict:
    """Host-only check of the solve work lists of a square CSR pattern (see ers.h); raises
    ErsError when a property is violated."""
    h = _CsrHold(pattern)
    counts = np.zeros(8, np.int64)
    o = make_opts() if ordering is None else make_opts(ordering=ordering)
    rc = lib().ers_solve_plan_check(C.byref(h.c), C.byref(o),
                                    counts.ctypes.data_as(C.POINTER(C.c_int64)))
    if rc != 0:
        raise ErsError(rc, "solve plan check failed")
    keys = ["fwd_entries", "bwd_entries", "fwd_lane_items", "bwd_lane_items",
            "fwd_warp_supernodes", "bwd_warp_supernodes", "fwd_diag", "bwd_diag"]
    return dict(zip(keys, counts.tolist()))


PLAN_ARRAYS = [("perm", np.int32), ("sn_start", np.int32), ("sn_parent", np.int32),
               ("level", np.int32), ("rows", np.int32), ("rel", np.int32), ("a_ptr", np.int32),
               ("a_idx", np.int32), ("a_src", np.int32), ("ch_ptr", np.int32),
               ("ch_list", np.int32), ("lvl_slot_ptr", np.int32), ("lvl_slot", np.int32),
               ("rptr", np.int64), ("front_off", np.int64), ("asm_dst", np.int64),
               ("arena", np.int64)]


def plan_arrays(pattern, ordering: Optional[int] = None) -> dict:
    """Host-only export of the symbolic plan of a square CSR pattern (see ers_plan_array in
    ers.h): every array by name, in the plan's (new) node order."""
    h = _CsrHold(pattern)
    o = make_opts() if ordering is None else make_opts(ordering=ordering)
    out = {}
    for which, (name, dt) in enumerate(PLAN_ARRAYS):
        ln = C.c_int64(0)
        rc = lib().ers_plan_array(C.byref(h.c), C.byref(o), which, None, C.byref(ln))
        if rc != 0:
            raise ErsError(rc, "plan export failed")
        a = np.zeros(ln.value, dt)
        if ln.value:
            rc = lib().ers_plan_array(C.byref(h.c), C.byref(o), which,
                                      a.ctypes.data_as(C.c_void_p), C.byref(ln))
            if rc != 0:
                raise ErsError(rc, "plan export failed")
        out[name] = a
    return out


class Simulator:
    """One circuit on one GPU: C x' + G_lin x + i_dev(x) = B u(t) (see include/ers.h)."""

    def __init__(self, G, Cmat, B, dev=None, pwl: Sequence = (), opts: Optional[Opts] = None,
                 stream=None, device: Optional[int] = None):
        L = lib()
        n = G.shape[0]
        self.n = n
        self._G = _CsrHold(G)
        self._C = _CsrHold(Cmat)
        self._B = _CsrHold(B, (n, B.shape[1]))
        p = B.shape[1]
        ndev = 0 if dev is None else len(dev)
        devs = (Mosfet * max(ndev, 1))()
        for i in range(ndev):
            d = dev[i]
            devs[i] = Mosfet(int(d["type"]), int(d["d"]), int(d["g"]), int(d["s"]),
                             float(d["vt"]), float(d["k"]), float(d["lam"]))
        self._pwl_arrays = []
        pw = (Pwl * max(p, 1))()
        for q, (tt, vv) in enumerate(pwl):
            tt = np.ascontiguousarray(tt, np.float64)
            vv = np.ascontiguousarray(vv, np.float64)
            self._pwl_arrays.append((tt, vv))
            pw[q] = Pwl(int(tt.size), _dptr(tt), _dptr(vv))
        self.opts = opts if opts is not None else default_opts()
        self._ctx = C.c_void_p()
        dl, nd = _device_list(None if device is None else [device])
        rc = L.ers_create(C.byref(self._ctx), C.byref(self._G.c), C.byref(self._C.c),
                          C.byref(self._B.c), devs if ndev else None, ndev,
                          pw if p else None, p, dl, nd, C.byref(self.opts))
        if rc != 0:
            msg = L.ers_last_error(self._ctx).decode() if self._ctx else ""
            if self._ctx:
                L.ers_destroy(self._ctx)
            self._ctx = None
            raise ErsError(rc, msg)
        if stream is not None:
            self.set_stream(stream)

    @classmethod
    def from_circuit(cls, circ, opts: Optional[Opts] = None, stream=None,
                     device: Optional[int] = None):
        return cls(circ.G, circ.C, circ.B, circ.dev, circ.pwl, opts=opts, stream=stream,
                   device=device)

    def _check(self, rc):
        if rc != 0:
            raise ErsError(rc, lib().ers_last_error(self._ctx).decode())

    def close(self):
        if self._ctx:
            lib().ers_destroy(self._ctx)
            self._ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        """stream: torch.cuda.Stream, an int handle, or None (private stream)."""
        handle = getattr(stream, "cuda_stream", stream)
        self._check(lib().ers_set_stream(self._ctx, C.c_void_p(handle) if handle else None))

    def dc(self, x0=None):
        arr = None if x0 is None else np.ascontiguousarray(x0, np.float64)
        self._check(lib().ers_dc(self._ctx, _dptr(arr) if arr is not None else None))

    def refactor(self):
        self._check(lib().ers_refactor(self._ctx))

    def step(self, h: float, m: int = 0):
        mu = C.c_int32(0)
        err = C.c_double(0.0)
        self._check(lib().ers_step(self._ctx, float(h), int(m), C.byref(mu), C.byref(err)))
        return mu.value, err.value

    def run(self, t_end: float, tol: float = 1e-6, max_steps: int = 0):
        ns = C.c_int32(0)
        nr = C.c_int32(0)
        self._check(lib().ers_run(self._ctx, float(t_end), float(tol), int(max_steps),
                                  C.byref(ns), C.byref(nr)))
        return ns.value, nr.value

    def profile(self, enable: bool = True):
        self._check(lib().ers_profile(self._ctx, int(bool(enable))))

    def state(self):
        x = np.zeros(self.n)
        t = C.c_double(0.0)
        h = C.c_double(0.0)
        self._check(lib().ers_get_state(self._ctx, C.byref(t), _dptr(x), C.byref(h)))
        return t.value, x, h.value

    def set_state(self, t: float, x, h: float = 0.0):
        x = np.ascontiguousarray(x, np.float64)
        self._check(lib().ers_set_state(self._ctx, float(t), _dptr(x), float(h)))

    def get_state_dev(self, ptr: int):
        self._check(lib().ers_get_state_dev(self._ctx, C.c_void_p(ptr)))

    def set_state_dev(self, t: float, ptr: int, h: float = 0.0):
        self._check(lib().ers_set_state_dev(self._ctx, float(t), C.c_void_p(ptr), float(h)))

    def solve(self, b):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros(self.n)
        self._check(lib().ers_solve(self._ctx, _dptr(b), _dptr(x)))
        return x

    def solve_dev_noalloc(self, b_ptr: int, x_ptr: int):
        """x = G_k^-1 b on device buffers without any device allocation (see ers.h)."""
        self._check(lib().ers_solve_dev_noalloc(self._ctx, C.c_void_p(b_ptr), C.c_void_p(x_ptr)))

    def spmv_C(self, v):
        v = np.ascontiguousarray(v, np.float64)
        y = np.zeros(self.n)
        self._check(lib().ers_spmv_C(self._ctx, _dptr(v), _dptr(y)))
        return y

    def mevp(self, v, h: float, m: int = 0):
        v = np.ascontiguousarray(v, np.float64)
        out = np.zeros(self.n)
        mu = C.c_int32(0)
        self._check(lib().ers_mevp(self._ctx, _dptr(v), float(h), int(m), _dptr(out), C.byref(mu)))
        return out, mu.value

    def phi_small(self, H, h: float):
        H = np.asfortranarray(H, np.float64)
        m = H.shape[1]
        y = np.zeros(m)
        last = C.c_double(0.0)
        self._check(lib().ers_phi_small(self._ctx, _dptr(H.ravel(order="F")), int(H.shape[0]), m,
                                        float(h), _dptr(y), C.byref(last)))
        return y, last.value

    def wait_selftest(self) -> int:
        """Status of the bounded-wait self-test (ERS_ERR_TIMEOUT = 6 expected; see ers.h)."""
        return int(lib().ers_wait_selftest(self._ctx))

    def autotune(self, nrhs: int = 2, passes: int = 5):
        """Pick the resident CTAs per SM of the solve kernels by timing (see ers.h); returns
        (chosen, [ms at 1, 2, 3 CTAs per SM])."""
        ms = np.zeros(3)
        ch = C.c_int32(0)
        self._check(lib().ers_autotune(self._ctx, int(nrhs), int(passes), _dptr(ms), C.byref(ch)))
        return ch.value, ms.tolist()

    def stats(self) -> dict:
        st = Stats()
        self._check(lib().ers_stats(self._ctx, C.byref(st)))
        return st.as_dict()


def _circuit_parts(circ):
    G = _CsrHold(circ.G)
    Cm = _CsrHold(circ.C)
    n = circ.G.shape[0]
    B = _CsrHold(circ.B, (n, circ.B.shape[1]))
    dev = circ.dev
    ndev = 0 if dev is None else len(dev)
    devs = (Mosfet * max(ndev, 1))()
    for i in range(ndev):
        d = dev[i]
        devs[i] = Mosfet(int(d["type"]), int(d["d"]), int(d["g"]), int(d["s"]),
                         float(d["vt"]), float(d["k"]), float(d["lam"]))
    p = circ.B.shape[1]
    arrays = []
    pw = (Pwl * max(p, 1))()
    for q, (tt, vv) in enumerate(circ.pwl):
        tt = np.ascontiguousarray(tt, np.float64)
        vv = np.ascontiguousarray(vv, np.float64)
        arrays.append((tt, vv))
        pw[q] = Pwl(int(tt.size), _dptr(tt), _dptr(vv))
    return dict(G=G, C=Cm, B=B, devs=devs, ndev=ndev, pw=pw, p=p, arrays=arrays, n=n)


class BatchSimulator(Simulator):
    """Many independent circuits in one context (ers_create_batch): one refactor and one
    solve pass per step cover all of them; each keeps its own Algorithm-2 controller."""

    def __init__(self, circuits, opts: Optional[Opts] = None, stream=None,
                 devices: Optional[Sequence[int]] = None):
        """devices: the CUDA device list (None: the current device); with several entries
        the instances are split over them by ers_partition_lpt (see ers.h)."""
        L = lib()
        self._parts = [_circuit_parts(c) for c in circuits]
        self.sizes = [pt["n"] for pt in self._parts]
        self.n = int(sum(self.sizes))
        self.ninst = len(circuits)
        inst = (Instance * self.ninst)()
        for k, pt in enumerate(self._parts):
            inst[k] = Instance(C.pointer(pt["G"].c), C.pointer(pt["C"].c), C.pointer(pt["B"].c),
                               pt["devs"] if pt["ndev"] else None, pt["ndev"],
                               pt["pw"] if pt["p"] else None, pt["p"])
        self.opts = opts if opts is not None else default_opts()
        self._ctx = C.c_void_p()
        dl, nd = _device_list(devices)
        rc = L.ers_create_batch(C.byref(self._ctx), inst, self.ninst, dl, nd, C.byref(self.opts))
        if rc != 0:
            msg = L.ers_last_error(self._ctx).decode() if self._ctx else ""
            if self._ctx:
                L.ers_destroy(self._ctx)
            self._ctx = None
            raise ErsError(rc, msg)
        if stream is not None:
            self.set_stream(stream)

    def run_batch(self, t_end: float, tol: float = 1e-6, max_steps: int = 0):
        ns = np.zeros(self.ninst, np.int32)
        nr = np.zeros(self.ninst, np.int32)
        self._check(lib().ers_run_batch(self._ctx, float(t_end), float(tol), int(max_steps),
                                        _iptr(ns), _iptr(nr)))
        return ns, nr

    def set_controller(self, mlp: Optional["Mlp"], parts: int = 3, margin: float = 0.0):
        """Learned (h, m) proposer (None = the plain controller of Alg. 2); parts: 1 = use the
        proposed step size, 2 = the proposed first residual-test dimension, 3 = both; margin
        (log2) is subtracted from the proposed step ratios."""
        self._mlp = mlp
        self._check(lib().ers_batch_set_controller(self._ctx, mlp.handle if mlp else None,
                                                   int(parts), float(margin)))

    def set_graphs(self, enable: bool = True):
        """Batched Arnoldi iterations as CUDA graph replays (default) or separate launches."""
        self._check(lib().ers_batch_set_graphs(self._ctx, int(bool(enable))))

    def trace(self, enable: bool = True):
        self._check(lib().ers_batch_trace(self._ctx, int(bool(enable))))

    def records(self, k: int) -> list:
        cnt = C.c_int32(0)
        self._check(lib().ers_batch_records(self._ctx, int(k), None, 0, C.byref(cnt)))
        arr = (StepRecord * max(cnt.value, 1))()
        self._check(lib().ers_batch_records(self._ctx, int(k), arr, cnt.value, C.byref(cnt)))
        return [{f: getattr(arr[q], f) for f, _ in StepRecord._fields_} for q in range(cnt.value)]

    def samples(self):
        cnt = C.c_int32(0)
        self._check(lib().ers_batch_samples(self._ctx, None, None, 0, C.byref(cnt)))
        X = np.zeros((max(cnt.value, 1), CTRL_FEATURES), np.float32)
        T = np.zeros((max(cnt.value, 1), 2), np.float32)
        self._check(lib().ers_batch_samples(self._ctx, _fptr(X), _fptr(T), cnt.value,
                                            C.byref(cnt)))
        return X[:cnt.value], T[:cnt.value]

    def ctrl_stats(self) -> dict:
        a, b, k = C.c_int64(0), C.c_int64(0), C.c_int64(0)
        self._check(lib().ers_batch_ctrl_stats(self._ctx, C.byref(a), C.byref(b), C.byref(k)))
        return {"proposals": a.value, "rejected": b.value, "krylov_vectors": k.value}

    def state_inst(self, k: int):
        x = np.zeros(self.sizes[k])
        t = C.c_double(0.0)
        h = C.c_double(0.0)
        self._check(lib().ers_get_state_inst(self._ctx, int(k), C.byref(t), _dptr(x), C.byref(h)))
        return t.value, x, h.value
