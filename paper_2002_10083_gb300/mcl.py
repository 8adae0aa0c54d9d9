"""Python binding of the C ABI in include/mcl.h (argument marshalling only).

Every step of the MCL iteration runs in the CUDA library libmcl.so; this
module only moves pointers and sizes across the ABI.  PyTorch provides
device memory (its caching allocator is handed to the library as the
allocator callback) and streams.  There is no CPU fallback: if the library
or a GPU is missing, every entry point raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np
import torch

from . import build as _build

MCL_OK = 0
STATUS = {0: "MCL_OK", 1: "MCL_ERR_INVALID", 2: "MCL_ERR_OOM", 3: "MCL_ERR_CUDA",
          4: "MCL_ERR_TIMEOUT", 5: "MCL_ERR_NOT_CONVERGED", 6: "MCL_ERR_INTERNAL"}
OPT_SIZING, OPT_CONF_MASK, OPT_VALIDATE, OPT_EST_SCALE, OPT_ITERATION, OPT_PHASE_BUDGET = 1, 2, 3, 4, 5, 6
OPT_COHEN_KEYS, OPT_COHEN_SEED = 7, 8
OPT_GRAPH, OPT_GRAPH_CAP = 9, 10
OPT_SMALL_MAX, OPT_TABLE, OPT_PLAN, OPT_GROUP_BUDGET, OPT_BUCKET_BUDGET = 11, 12, 13, 14, 15
SIZING_COHEN = 3
SIZING_PARAMS, SIZING_EXACT, SIZING_FLOPS = -1, 0, 1
MAX_SELECT_K = 4096


class MclError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _Csc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("nnz", ctypes.c_int64), ("colptr", ctypes.c_void_p),
                ("rowidx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class _Params(ctypes.Structure):
    _fields_ = [("threshold", ctypes.c_float), ("select_k", ctypes.c_int32),
                ("recover_pct", ctypes.c_float), ("recover_k", ctypes.c_int32),
                ("inflation", ctypes.c_float), ("chaos_eps", ctypes.c_double),
                ("max_iters", ctypes.c_int32), ("use_estimator", ctypes.c_int32),
                ("batched", ctypes.c_int32)]


class _Stats(ctypes.Structure):
    _fields_ = [("flops", ctypes.c_int64), ("nnz_in", ctypes.c_int64), ("nnz_b", ctypes.c_int64),
                ("nnz_out", ctypes.c_int64), ("estimator_misses", ctypes.c_int64),
                ("range_splits", ctypes.c_int64), ("chaos", ctypes.c_double),
                ("ms_colstats", ctypes.c_float), ("ms_estimate", ctypes.c_float),
                ("ms_bin", ctypes.c_float), ("ms_numeric", ctypes.c_float),
                ("ms_compact", ctypes.c_float), ("ms_chaos", ctypes.c_float),
                ("ms_total", ctypes.c_float), ("bins_used", ctypes.c_int32),
                ("iterations", ctypes.c_int32), ("phases", ctypes.c_int32),
                ("graph_replays", ctypes.c_int32), ("exact_from", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("flops_run", ctypes.c_int64),
                ("alg_bytes_run", ctypes.c_int64)]


class _MergeStats(ctypes.Structure):
    _fields_ = [("stages", ctypes.c_int32), ("merges", ctypes.c_int32),
                ("partial_entries", ctypes.c_int64), ("binary_peak_entries", ctypes.c_int64),
                ("live_peak_entries", ctypes.c_int64), ("merged_entries", ctypes.c_int64)]


_ALLOC = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)

# symbol name -> (restype, argtypes); every entry point declared in include/mcl.h
P = ctypes.c_void_p
SIGNATURES = {
    "mcl_version": (ctypes.c_char_p, []),
    "mcl_launch_count": (ctypes.c_int64, []),
    "mcl_create": (ctypes.c_int, [ctypes.POINTER(P), ctypes.c_int, _ALLOC, _FREE, P]),
    "mcl_destroy": (None, [P]),
    "mcl_last_error": (ctypes.c_char_p, [P]),
    "mcl_expand": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.POINTER(_Params),
                                  ctypes.POINTER(_Csc), ctypes.POINTER(ctypes.c_double), P]),
    "mcl_expand_split": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.POINTER(_Params),
                                        ctypes.c_int32, ctypes.POINTER(_Csc),
                                        ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(_MergeStats), P]),
    "mcl_prune_select_recover": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.POINTER(_Params),
                                                ctypes.POINTER(_Csc), P]),
    "mcl_inflate_normalize": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.c_float, P]),
    "mcl_chaos": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.POINTER(ctypes.c_double), P, P]),
    "mcl_components": (ctypes.c_int, [P, ctypes.POINTER(_Csc), P, P]),
    "mcl_run": (ctypes.c_int, [P, ctypes.POINTER(_Csc), P, ctypes.c_int32, ctypes.POINTER(_Params),
                               P, ctypes.POINTER(ctypes.c_int32), P, ctypes.POINTER(_Csc), P]),
    "mcl_symbolic": (ctypes.c_int, [P, ctypes.POINTER(_Csc), P, P, P]),
    "mcl_get_stats": (ctypes.c_int, [P, ctypes.POINTER(_Stats)]),
    "mcl_set_option": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int64]),
    "mcl_estimator_load": (ctypes.c_int, [P, P, P, ctypes.c_float]),
    "mcl_features": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.c_int32, P, P, P]),
    "mcl_mlp_forward": (ctypes.c_int, [P, P, ctypes.c_int64, P, P, P, P]),
    "mcl_mlp_backward": (ctypes.c_int, [P, P, P, ctypes.c_int64, P, P, ctypes.c_float, P, P, P]),
    "mcl_adam_step": (ctypes.c_int, [P, P, P, P, P, ctypes.c_int64, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, P, P]),
    "mcl_estimate": (ctypes.c_int, [P, ctypes.POINTER(_Csc), P, P]),
    "mcl_symbolic_noalloc": (ctypes.c_int, [ctypes.POINTER(_Csc), P, P, ctypes.c_char_p,
                                            ctypes.c_size_t, P]),
    "mcl_cohen_estimate": (ctypes.c_int, [P, ctypes.POINTER(_Csc), ctypes.c_int32, ctypes.c_uint64,
                                          P, P]),
}
MLP_NPARAM = 5378
NFEATURES = 16

_lib = None
_lib_lock = threading.Lock()


def launch_count() -> int:
    """Kernels launched by libmcl.so in this process so far."""
    return int(load().mcl_launch_count())


def symbolic_noalloc(A: "DeviceCSC", flops=None, nnz_out=None, stream=None):
    """mcl_symbolic_noalloc: flops_j and nnz((AA)_*j) into caller-allocated
    int64 device tensors, with no context and no allocation in the library."""
    lib = load()
    a = A.c()
    err = ctypes.create_string_buffer(512)
    st = lib.mcl_symbolic_noalloc(ctypes.byref(a),
                                  P(flops.data_ptr()) if flops is not None else None,
                                  P(nnz_out.data_ptr()) if nnz_out is not None else None,
                                  err, len(err), _stream_ptr(stream))
    if st != MCL_OK:
        raise MclError(st, err.value.decode())


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libmcl.so (building it first if stale); raise if unavailable."""
    global _lib
    with _lib_lock:
        if _lib is None:
            path = _build.build() if build_if_missing else _build.LIB
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library missing: {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


@dataclasses.dataclass
class Params:
    threshold: float = 1e-4
    select_k: int = 1100
    recover_pct: float = 0.9
    recover_k: int = 0
    inflation: float = 2.0
    chaos_eps: float = 1e-3
    max_iters: int = 30
    use_estimator: int = 0
    batched: int = 0

    def c(self) -> _Params:
        return _Params(self.threshold, self.select_k, self.recover_pct, self.recover_k,
                       self.inflation, self.chaos_eps, self.max_iters, self.use_estimator,
                       self.batched)


@dataclasses.dataclass
class DeviceCSC:
    """CSC matrix in device memory: int64 colptr, int32 rowidx, float32 val."""
    n: int
    colptr: torch.Tensor
    rowidx: torch.Tensor
    val: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    @staticmethod
    def from_host(A, device="cuda") -> "DeviceCSC":
        colptr = torch.from_numpy(np.ascontiguousarray(A.colptr, np.int64)).to(device)
        rowidx = torch.from_numpy(np.ascontiguousarray(A.rowidx, np.int32)).to(device)
        val = torch.from_numpy(np.ascontiguousarray(A.val, np.float32)).to(device)
        return DeviceCSC(int(A.n), colptr, rowidx, val)

    def to_host(self):
        from .synth import CSC
        return CSC(n=self.n, colptr=self.colptr.cpu().numpy(), rowidx=self.rowidx.cpu().numpy(),
                   val=self.val.cpu().numpy().astype(np.float64))

    def c(self) -> _Csc:
        return _Csc(self.n, self.nnz, self.colptr.data_ptr(),
                    self.rowidx.data_ptr() if self.nnz else None,
                    self.val.data_ptr() if self.nnz else None)


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """An mcl_ctx bound to one CUDA device; torch's caching allocator
    provides every device buffer the library allocates."""

    def __init__(self, device: int = 0):
        if not torch.cuda.is_available():
            raise RuntimeError("MCL requires a CUDA GPU; none is available")
        self.lib = load()
        self.device = device
        self._owned = {}  # data_ptr -> tensor (memory handed to the library)
        self._alloc_cb = _ALLOC(self._alloc)
        self._free_cb = _FREE(self._free)
        h = ctypes.c_void_p()
        st = self.lib.mcl_create(ctypes.byref(h), device, self._alloc_cb, self._free_cb, None)
        if st != MCL_OK:
            raise MclError(st, "mcl_create failed")
        self.h = h

    # allocator callbacks -------------------------------------------------
    def _alloc(self, nbytes, user, stream):
        try:
            with torch.cuda.device(self.device):
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
            p = t.data_ptr()
            self._owned[p] = t
            return p
        except Exception:  # OOM -> NULL, the library returns MCL_ERR_OOM
            return None

    def _free(self, ptr, user, stream):
        self._owned.pop(ptr, None)

    def _adopt(self, ptr, count, dtype) -> torch.Tensor:
        t = self._owned.pop(ptr)
        nbytes = count * torch.empty(0, dtype=dtype).element_size()
        return t[:nbytes].view(dtype)

    def _adopt_csc(self, out: _Csc) -> DeviceCSC:
        colptr = self._adopt(out.colptr, out.n + 1, torch.int64)
        rowidx = self._adopt(out.rowidx, out.nnz, torch.int32)
        val = self._adopt(out.val, out.nnz, torch.float32)
        return DeviceCSC(int(out.n), colptr, rowidx, val)

    def close(self):
        if getattr(self, "h", None):
            self.lib.mcl_destroy(self.h)
            self.h = None
        self._owned.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != MCL_OK:
            msg = self.lib.mcl_last_error(self.h)
            raise MclError(st, msg.decode() if msg else "")

    # entry points ----------------------------------------------------------
    def set_option(self, option: int, value: int):
        self._check(self.lib.mcl_set_option(self.h, option, int(value)))

    def expand(self, A: DeviceCSC, prm: Params, stream=None):
        """One fused MCL iteration -> (A_next, chaos)."""
        a = A.c()
        p = prm.c()
        out = _Csc()
        ch = ctypes.c_double(0.0)
        self._check(self.lib.mcl_expand(self.h, ctypes.byref(a), ctypes.byref(p),
                                        ctypes.byref(out), ctypes.byref(ch), _stream_ptr(stream)))
        return self._adopt_csc(out), ch.value

    def expand_split(self, A: DeviceCSC, prm: Params, nstages: int, stream=None):
        """One MCL iteration with the inner dimension split into `nstages`
        blocks and the partial products binary-merged -> (A_next, chaos, stats)."""
        a = A.c()
        p = prm.c()
        out = _Csc()
        ch = ctypes.c_double(0.0)
        ms = _MergeStats()
        self._check(self.lib.mcl_expand_split(self.h, ctypes.byref(a), ctypes.byref(p),
                                              int(nstages), ctypes.byref(out), ctypes.byref(ch),
                                              ctypes.byref(ms), _stream_ptr(stream)))
        stats = {name: getattr(ms, name) for name, _ in _MergeStats._fields_}
        return self._adopt_csc(out), ch.value, stats

    def prune_select_recover(self, B: DeviceCSC, prm: Params, stream=None) -> DeviceCSC:
        b = B.c()
        p = prm.c()
        out = _Csc()
        self._check(self.lib.mcl_prune_select_recover(self.h, ctypes.byref(b), ctypes.byref(p),
                                                      ctypes.byref(out), _stream_ptr(stream)))
        return self._adopt_csc(out)

    def inflate_normalize(self, A: DeviceCSC, r: float, stream=None) -> DeviceCSC:
        """In place on A.val; returns A."""
        a = A.c()
        self._check(self.lib.mcl_inflate_normalize(self.h, ctypes.byref(a), float(r),
                                                   _stream_ptr(stream)))
        return A

    def chaos(self, A: DeviceCSC, per_column=False, stream=None):
        a = A.c()
        ch = ctypes.c_double(0.0)
        cols = torch.empty(max(A.n, 1), dtype=torch.float64, device=A.colptr.device) if per_column else None
        self._check(self.lib.mcl_chaos(self.h, ctypes.byref(a), ctypes.byref(ch),
                                       ctypes.c_void_p(cols.data_ptr()) if cols is not None else None,
                                       _stream_ptr(stream)))
        return (ch.value, cols[:A.n]) if per_column else ch.value

    def components(self, A: DeviceCSC, stream=None) -> torch.Tensor:
        a = A.c()
        lab = torch.empty(max(A.n, 1), dtype=torch.int32, device=A.colptr.device)
        self._check(self.lib.mcl_components(self.h, ctypes.byref(a), ctypes.c_void_p(lab.data_ptr()),
                                            _stream_ptr(stream)))
        return lab[:A.n]

    def symbolic(self, A: DeviceCSC, stream=None):
        """(flops_j, nnz((AA)_*j)) as device int64 tensors."""
        a = A.c()
        dev = A.colptr.device
        fl = torch.empty(max(A.n, 1), dtype=torch.int64, device=dev)
        nz = torch.empty(max(A.n, 1), dtype=torch.int64, device=dev)
        self._check(self.lib.mcl_symbolic(self.h, ctypes.byref(a), ctypes.c_void_p(fl.data_ptr()),
                                          ctypes.c_void_p(nz.data_ptr()), _stream_ptr(stream)))
        return fl[:A.n], nz[:A.n]

    def run(self, A0: DeviceCSC, prm: Params, comp_offsets=None, keep_final=True, stream=None):
        """Algorithm 1 to convergence -> (labels, iterations, chaos history, final A or None)."""
        a = A0.c()
        p = prm.c()
        lab = torch.empty(max(A0.n, 1), dtype=torch.int32, device=A0.colptr.device)
        it = ctypes.c_int32(0)
        hist = (ctypes.c_double * max(prm.max_iters, 1))()
        out = _Csc()
        offs = None
        ncomp = 0
        if comp_offsets is not None:
            offs = np.ascontiguousarray(comp_offsets, dtype=np.int32)
            ncomp = len(offs) - 1
        st = self.lib.mcl_run(self.h, ctypes.byref(a),
                              offs.ctypes.data_as(ctypes.c_void_p) if offs is not None else None,
                              ncomp, ctypes.byref(p), ctypes.c_void_p(lab.data_ptr()),
                              ctypes.byref(it), hist,
                              ctypes.byref(out) if keep_final else None, _stream_ptr(stream))
        if st not in (MCL_OK, 5):
            self._check(st)
        final = self._adopt_csc(out) if keep_final and out.colptr else None
        return lab[:A0.n], it.value, list(hist[:it.value]), final, st == 5

    # learned estimator ------------------------------------------------------
    def estimator_load(self, w_bf16: np.ndarray, norm: np.ndarray, safety: float):
        w = np.ascontiguousarray(w_bf16, dtype=np.uint16)
        nm = np.ascontiguousarray(norm, dtype=np.float32)
        assert w.size == MLP_NPARAM and nm.size == 2 * NFEATURES
        self._check(self.lib.mcl_estimator_load(self.h, w.ctypes.data_as(P), nm.ctypes.data_as(P),
                                                float(safety)))

    def features(self, A: DeviceCSC, iteration: int = 1, prev_logcf=None, stream=None):
        a = A.c()
        f = torch.empty((max(A.n, 1), NFEATURES), dtype=torch.float32, device=A.colptr.device)
        self._check(self.lib.mcl_features(self.h, ctypes.byref(a), int(iteration),
                                          P(prev_logcf.data_ptr()) if prev_logcf is not None else None,
                                          P(f.data_ptr()), _stream_ptr(stream)))
        return f[:A.n]

    def mlp_forward(self, feats, w_bf16_dev, norm_dev, stream=None):
        n = feats.shape[0]
        out = torch.empty((max(n, 1), 2), dtype=torch.float32, device=feats.device)
        self._check(self.lib.mcl_mlp_forward(self.h, P(feats.data_ptr()), n, P(w_bf16_dev.data_ptr()),
                                             P(norm_dev.data_ptr()), P(out.data_ptr()),
                                             _stream_ptr(stream)))
        return out[:n]

    def mlp_backward(self, feats, targets, w_bf16_dev, norm_dev, scale, grad, loss, stream=None):
        n = feats.shape[0]
        self._check(self.lib.mcl_mlp_backward(self.h, P(feats.data_ptr()), P(targets.data_ptr()), n,
                                              P(w_bf16_dev.data_ptr()), P(norm_dev.data_ptr()),
                                              float(scale), P(grad.data_ptr()), P(loss.data_ptr()),
                                              _stream_ptr(stream)))

    def adam_step(self, master, m, v, grad, step, lr, w_bf16_dev, beta1=0.9, beta2=0.999,
                  eps=1e-8, stream=None):
        self._check(self.lib.mcl_adam_step(self.h, P(master.data_ptr()), P(m.data_ptr()),
                                           P(v.data_ptr()), P(grad.data_ptr()), int(step), float(lr),
                                           float(beta1), float(beta2), float(eps),
                                           P(w_bf16_dev.data_ptr()), _stream_ptr(stream)))

    def estimate(self, A: DeviceCSC, stream=None):
        a = A.c()
        est = torch.empty(max(A.n, 1), dtype=torch.int64, device=A.colptr.device)
        self._check(self.lib.mcl_estimate(self.h, ctypes.byref(a), P(est.data_ptr()),
                                          _stream_ptr(stream)))
        return est[:A.n]

    def cohen_estimate(self, A: DeviceCSC, keys: int = 8, seed: int = 2002, stream=None):
        """Cohen's estimate of nnz((AA)_*j) per column (device float32)."""
        a = A.c()
        est = torch.empty(max(A.n, 1), dtype=torch.float32, device=A.colptr.device)
        self._check(self.lib.mcl_cohen_estimate(self.h, ctypes.byref(a), int(keys), int(seed),
                                                P(est.data_ptr()), _stream_ptr(stream)))
        return est[:A.n]

    def stats(self) -> dict:
        s = _Stats()
        self._check(self.lib.mcl_get_stats(self.h, ctypes.byref(s)))
        return {name: getattr(s, name) for name, _ in _Stats._fields_}
