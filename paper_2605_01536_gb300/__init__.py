"""Python binding of the GB300 generalized-winding-number library.

Thin ctypes marshalling over the C ABI in ``include/gwn.h``: every computation
runs in the CUDA library ``_lib/libgwn.so`` (built by :func:`build`).  There is
no CPU fallback: if the library is missing or no GPU is present the calls raise.
PyTorch is used only for device memory and streams; numpy arrays (host memory)
are accepted too, in which case the library stages them through the device and
the call returns numpy arrays.

The method (arXiv 2605.01536): w(q) = chi + (1/4pi) sum_{(a,b) in dM}
Area(A, B, -x0) with x0 = +z (Eq. 9, Algorithm 1, Supp. S2.1).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

__all__ = ["build", "load", "Mesh", "Batch", "ParamSurface", "GwnError", "lib_path", "Config", "Counters", "MeshInfo",
           "BatchConfig", "MlpConfig", "profile_enable", "profile_read", "measure_pipe_peaks"]

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "_lib", "libgwn.so")
_lock = threading.Lock()
_lib = None

GWN_OK = 0
_ERRORS = {1: "GWN_ERR_INVALID_ARG", 2: "GWN_ERR_INVALID_MESH", 3: "GWN_ERR_NOT_BUILT",
           4: "GWN_ERR_CUDA", 5: "GWN_ERR_OOM", 6: "GWN_ERR_TRAVERSAL_LIMIT"}


class GwnError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERRORS.get(code, code)}: {msg}")
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [("queries_per_thread", ctypes.c_int32), ("boundary_tile", ctypes.c_int32),
                ("chain_boundary", ctypes.c_int32), ("classify_margin", ctypes.c_float),
                ("quantize_bits", ctypes.c_int32), ("fp64_cancel", ctypes.c_int32),
                ("group_test", ctypes.c_int32), ("reserved", ctypes.c_int32 * 9)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int64), ("nt", ctypes.c_int64), ("n_boundary_edges", ctypes.c_int64),
                ("n_boundary_points", ctypes.c_int64), ("n_boundary_loops", ctypes.c_int64),
                ("n_bvh_nodes", ctypes.c_int64), ("built", ctypes.c_int32), ("device", ctypes.c_int32)]


class Counters(ctypes.Structure):
    _fields_ = [("error_flags", ctypes.c_uint64), ("exact_edge", ctypes.c_uint64),
                ("exact_plane", ctypes.c_uint64), ("exact_branch", ctypes.c_uint64),
                ("apex_terms", ctypes.c_uint64), ("degenerate_terms", ctypes.c_uint64),
                ("fp64_reevaluations", ctypes.c_uint64), ("surrogate_queries", ctypes.c_uint64),
                ("surrogate_fallbacks", ctypes.c_uint64), ("gradient_skipped", ctypes.c_uint64),
                ("cancel_terms", ctypes.c_uint64), ("cancel_overflow", ctypes.c_uint64),
                ("reserved", ctypes.c_uint64 * 4)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class MlpConfig(ctypes.Structure):
    """Training settings of the learned surrogate (zero fields take the library defaults)."""
    _fields_ = [("steps", ctypes.c_int32), ("batch", ctypes.c_int32), ("lr", ctypes.c_float),
                ("margin", ctypes.c_float), ("seed", ctypes.c_uint64), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("band_res", ctypes.c_int32),
                ("band_dilate", ctypes.c_int32), ("chi_tol", ctypes.c_float), ("reserved", ctypes.c_int32 * 6)]


class ParamConfig(ctypes.Structure):
    """Settings of a parametric surface (gwn_param_config)."""
    _fields_ = [("quad_tol", ctypes.c_double), ("flat_tol", ctypes.c_double), ("fp64", ctypes.c_int32),
                ("max_panels", ctypes.c_int32), ("max_nodes", ctypes.c_int32)]


# name -> (restype, argtypes) of every function declared in include/gwn.h
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_S = ctypes.c_int
SIGNATURES = {
    "gwn_version": (ctypes.c_char_p, []),
    "gwn_last_error": (ctypes.c_char_p, []),
    "gwn_mesh_create": (_S, [_P, _I64, _P, _I64, _P, _P, ctypes.POINTER(_P)]),
    "gwn_mesh_destroy": (_S, [_P]),
    "gwn_build_accel": (_S, [_P, _P]),
    "gwn_mesh_get_info": (_S, [_P, ctypes.POINTER(MeshInfo)]),
    "gwn_mesh_get_boundary": (_S, [_P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "gwn_mesh_get_boundary_points": (_S, [_P, _P, _I64, ctypes.POINTER(_I64), _P]),
    "gwn_query_batch": (_S, [_P, _P, _I64, _P, _P, _P]),
    "gwn_query_chi": (_S, [_P, _P, _I64, _P, _P]),
    "gwn_query_chi_visits": (_S, [_P, _P, _I64, _P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                  _P]),
    "gwn_query_direct": (_S, [_P, _P, _I64, _P, _P]),
    "gwn_query_gradient": (_S, [_P, _P, _I64, _P, _P]),
    "gwn_query_grid_chi": (_S, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P]),
    "gwn_classify_grid": (_S, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P]),
    "gwn_classify": (_S, [_P, _P, _I64, _P, _P, _P]),
    "gwn_classify_static": (_S, [_P, _P, _I64, _P, _P, _P]),
    "gwn_get_counters": (_S, [_P, ctypes.POINTER(Counters), _S, _P]),
    "gwn_batch_create": (_S, [ctypes.POINTER(_P), ctypes.c_int32, _P, _P, ctypes.POINTER(_P)]),
    "gwn_batch_destroy": (_S, [_P]),
    "gwn_batch_run": (_S, [_P, _P, _P, _P, _P]),
    "gwn_batch_autotune": (_S, [_P, _P, _P, _P, ctypes.c_char_p, _P]),
    "gwn_batch_get_config": (_S, [_P, _P, ctypes.POINTER(_I64)]),
    "gwn_debug_tc_gemm": (_S, [_P, _P, ctypes.c_int32, _P, _P]),
    "gwn_param_config_default": (None, [ctypes.POINTER(ParamConfig)]),
    "gwn_param_create": (_S, [_P, ctypes.c_int32, ctypes.POINTER(ParamConfig), ctypes.POINTER(_P)]),
    "gwn_param_destroy": (_S, [_P]),
    "gwn_param_get_boundary": (_S, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "gwn_param_query": (_S, [_P, _P, _I64, _P, _P, _P]),
    "gwn_param_query_grid": (_S, [_P, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, ctypes.c_int32, _P, _P, _P]),
    "gwn_param_status": (_S, [_P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                              ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64), ctypes.c_int]),
    "gwn_surrogate_num_params": (ctypes.c_int32, []),
    "gwn_surrogate_train": (_S, [_P, _P, _P, _I64, ctypes.POINTER(MlpConfig), ctypes.POINTER(ctypes.c_float), _P]),
    "gwn_surrogate_predict": (_S, [_P, _P, _I64, _P, _P]),
    "gwn_surrogate_params": (_S, [_P, _P, _P, ctypes.c_int32]),
    "gwn_surrogate_grad": (_S, [_P, _P, _P, _I64, _P, ctypes.POINTER(ctypes.c_float), _P]),
    "gwn_surrogate_calibrate": (_S, [_P, _P, _I64, ctypes.c_double, ctypes.c_float, ctypes.POINTER(ctypes.c_float),
                                     ctypes.POINTER(_I64), _P]),
    "gwn_surrogate_save": (_S, [_P, ctypes.c_char_p]),
    "gwn_surrogate_load": (_S, [_P, ctypes.c_char_p]),
    "gwn_surrogate_detach": (_S, [_P]),
    "gwn_profile_enable": (_S, [_S]),
    "gwn_profile_read": (_S, [_P, _S, ctypes.POINTER(_S)]),
    "gwn_measure_pipe_peaks": (_S, [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32), _P]),
}


def lib_path() -> str:
    return _LIB_PATH


def build(force: bool = False) -> str:
    """Compile the CUDA library in-tree (nvcc, sm_103a)."""
    from . import _build
    return _build.build(force=force)


def load():
    """Load ``libgwn.so`` and bind every C entry point.  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_LIB_PATH):
                raise ImportError(f"{_LIB_PATH} is missing: build the CUDA library first "
                                  "(python -c 'import __graft_entry__ as g; g.build()')")
            lib = ctypes.CDLL(_LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(code: int):
    if code != GWN_OK:
        raise GwnError(code, load().gwn_last_error().decode(errors="replace"))


def _torch():
    import torch
    return torch


def _is_torch(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor)


def _stream_ptr(stream=None):
    torch = _torch()
    if stream is None:
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _points(x, name):
    """Validate an [n,3] float32 array; return (pointer, n, is_device, keepalive)."""
    if _is_torch(x):
        if x.dtype != _torch().float32 or x.dim() != 2 or x.shape[1] != 3:
            raise ValueError(f"{name} must be a float32 tensor of shape [n, 3]")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return ctypes.c_void_p(x.data_ptr() if x.numel() else 0), int(x.shape[0]), x.is_cuda, x
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError(f"{name} must have shape [n, 3]")
    return a.ctypes.data_as(ctypes.c_void_p), int(a.shape[0]), False, a


def _alloc_like(q, is_dev, n, dtype_np, dtype_name):
    """Output buffer matching the query's memory: CUDA tensor, pinned host tensor
    (for a pinned host query tensor) or numpy array."""
    if _is_torch(q) and (is_dev or q.is_pinned()):
        torch = _torch()
        if is_dev:
            t = torch.empty(n, dtype=getattr(torch, dtype_name), device=q.device)
        else:
            t = torch.empty(n, dtype=getattr(torch, dtype_name), pin_memory=True)
        return t, ctypes.c_void_p(t.data_ptr() if n else 0)
    a = np.empty(n, dtype=dtype_np)
    return a, a.ctypes.data_as(ctypes.c_void_p)


class BatchConfig(ctypes.Structure):
    _fields_ = [("queries_per_thread", ctypes.c_int32), ("points_per_item", ctypes.c_int32),
                ("tile", ctypes.c_int32), ("grid_blocks", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("tune_queries_per_mesh", ctypes.c_int32), ("reserved", ctypes.c_int32 * 10)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_ if k != "reserved"}


class KernelStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("kernels", ctypes.c_int64)]


def profile_enable(on: bool = True):
    """Start (or stop) per-kernel CUDA-event timing inside the library."""
    _check(load().gwn_profile_enable(1 if on else 0))


def measure_pipe_peaks(stream=None) -> dict:
    """Measured FFMA, FFMA2 and SFU throughputs of the current device (gwn_measure_pipe_peaks)."""
    f1, f, m, n = ctypes.c_double(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    _check(load().gwn_measure_pipe_peaks(ctypes.byref(f1), ctypes.byref(f), ctypes.byref(m), ctypes.byref(n),
                                         _stream_ptr(stream)))
    return {"ffma_per_s": f1.value, "ffma2_per_s": f.value, "mufu_per_s": m.value, "sm_count": n.value}


def profile_read(with_kernels: bool = False) -> dict:
    """{step name: (runs, total ms)} since the last enable/read; with_kernels
    adds the number of CUDA kernels those runs launched: (runs, ms, kernels)."""
    cap = 64
    arr = (KernelStat * cap)()
    n = ctypes.c_int()
    _check(load().gwn_profile_read(arr, cap, ctypes.byref(n)))
    out = {}
    for i in range(min(n.value, cap)):
        v = (int(arr[i].launches), float(arr[i].total_ms))
        out[arr[i].name.decode()] = v + (int(arr[i].kernels),) if with_kernels else v
    return out


class Mesh:
    """An oriented triangle mesh on the GPU.

    ``V``: float32 [nv, 3], ``F``: int32 [nt, 3] (numpy or torch, host or CUDA).
    ``config``: optional dict of :class:`Config` fields.
    """

    def __init__(self, V, F, config: dict | None = None, build: bool = True, stream=None):
        lib = load()
        if _is_torch(V):
            V = V.detach().to("cpu").numpy()
        if _is_torch(F):
            F = F.detach().to("cpu").numpy()
        V = np.ascontiguousarray(V, dtype=np.float32).reshape(-1, 3)
        F = np.ascontiguousarray(F, dtype=np.int32).reshape(-1, 3)
        cfg = Config()
        for k, v in (config or {}).items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        sp = _stream_ptr(stream)
        _check(lib.gwn_mesh_create(V.ctypes.data_as(_P), V.shape[0], F.ctypes.data_as(_P), F.shape[0],
                                   ctypes.byref(cfg), sp, ctypes.byref(h)))
        self._h = h
        self.nv, self.nt = V.shape[0], F.shape[0]
        if build:
            self.build(stream)

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(load().gwn_mesh_destroy(self._h))
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

    @property
    def handle(self):
        return self._h

    # -- build / info
    def build(self, stream=None):
        _check(load().gwn_build_accel(self._h, _stream_ptr(stream)))

    def info(self) -> dict:
        inf = MeshInfo()
        _check(load().gwn_mesh_get_info(self._h, ctypes.byref(inf)))
        return {k: int(getattr(inf, k)) for k, _ in MeshInfo._fields_}

    def boundary_edges(self, stream=None) -> np.ndarray:
        nb = self.info()["n_boundary_edges"]
        out = np.empty((max(nb, 1), 2), dtype=np.int32)
        n = ctypes.c_int64()
        _check(load().gwn_mesh_get_boundary(self._h, out.ctypes.data_as(_P), out.shape[0], ctypes.byref(n),
                                            _stream_ptr(stream)))
        return out[: n.value].copy()

    def boundary_points(self, stream=None) -> np.ndarray:
        """Chained boundary points (float32 [npts, 4]: x, y, z, edge-to-next flag)."""
        npts = self.info()["n_boundary_points"]
        out = np.empty((max(npts, 1), 4), dtype=np.float32)
        n = ctypes.c_int64()
        _check(load().gwn_mesh_get_boundary_points(self._h, out.ctypes.data_as(_P), out.shape[0], ctypes.byref(n),
                                                   _stream_ptr(stream)))
        return out[: n.value].copy()

    def counters(self, reset: bool = False, stream=None) -> dict:
        c = Counters()
        _check(load().gwn_get_counters(self._h, ctypes.byref(c), 1 if reset else 0, _stream_ptr(stream)))
        return c.as_dict()

    # -- queries
    def query(self, q, want_chi: bool = True, stream=None):
        """Antipodal w (float32 [n]) and chi (int32 [n], or None)."""
        qp, n, dev, keep = _points(q, "q")
        w, wp = _alloc_like(q, dev, n, np.float32, "float32")
        chi, cp = _alloc_like(q, dev, n, np.int32, "int32") if want_chi else (None, None)
        _check(load().gwn_query_batch(self._h, qp, n, wp, cp, _stream_ptr(stream)))
        return w, chi

    def chi(self, q, stream=None):
        qp, n, dev, keep = _points(q, "q")
        chi, cp = _alloc_like(q, dev, n, np.int32, "int32")
        _check(load().gwn_query_chi(self._h, qp, n, cp, _stream_ptr(stream)))
        return chi

    def chi_visits(self, q, stream=None):
        """(chi, nodes read, triangles tested): the crossing counts from the
        instrumented walk, with the traversal's visit totals over the queries."""
        qp, n, dev, keep = _points(q, "q")
        chi, cp = _alloc_like(q, dev, n, np.int32, "int32")
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().gwn_query_chi_visits(self._h, qp, n, cp, ctypes.byref(a), ctypes.byref(b), _stream_ptr(stream)))
        return chi, int(a.value), int(b.value)

    def direct(self, q, stream=None):
        """Direct solid-angle sum (baseline), float32 [n]."""
        qp, n, dev, keep = _points(q, "q")
        w, wp = _alloc_like(q, dev, n, np.float32, "float32")
        _check(load().gwn_query_direct(self._h, qp, n, wp, _stream_ptr(stream)))
        return w

    def gradient(self, q, stream=None):
        """grad w (float32 [n, 3]) by Supp. S4, Algorithm 3."""
        qp, n, dev, keep = _points(q, "q")
        if _is_torch(q) and (dev or q.is_pinned()):
            torch = _torch()
            g = torch.empty((n, 3), dtype=torch.float32, device=q.device if dev else "cpu", pin_memory=not dev)
            gp = ctypes.c_void_p(g.data_ptr() if n else 0)
        else:
            g = np.empty((n, 3), dtype=np.float32)
            gp = g.ctypes.data_as(ctypes.c_void_p)
        _check(load().gwn_query_gradient(self._h, qp, n, gp, _stream_ptr(stream)))
        return g

    # -- rectilinear grids with ray reuse (outputs [nz, ny, nx], x fastest)
    @staticmethod
    def _axes(x, y, z):
        axes = [np.ascontiguousarray(np.asarray(a.detach().cpu() if _is_torch(a) else a, dtype=np.float32).reshape(-1))
                for a in (x, y, z)]
        return axes, [a.ctypes.data_as(_P) for a in axes]

    def _grid_out(self, shape, np_dtype, torch_dtype, device):
        if device:
            torch = _torch()
            t = torch.empty(shape, dtype=getattr(torch, torch_dtype), device="cuda")
            return t, ctypes.c_void_p(t.data_ptr() if t.numel() else 0)
        a = np.empty(shape, dtype=np_dtype)
        return a, a.ctypes.data_as(_P)

    def grid_chi(self, x, y, z, device: bool = True, stream=None):
        """Crossing numbers of the grid cells (x[i], y[j], z[k]), int32 [nz, ny, nx]."""
        (ax, ay, az), (px, py, pz) = self._axes(x, y, z)
        chi, cp = self._grid_out((len(az), len(ay), len(ax)), np.int32, "int32", device)
        _check(load().gwn_query_grid_chi(self._h, px, len(ax), py, len(ay), pz, len(az), cp, _stream_ptr(stream)))
        return chi

    def classify_grid(self, x, y, z, want_w: bool = False, device: bool = True, stream=None):
        """Labels (uint8 [nz, ny, nx]) and optionally w of the grid cells."""
        (ax, ay, az), (px, py, pz) = self._axes(x, y, z)
        shape = (len(az), len(ay), len(ax))
        lab, lp = self._grid_out(shape, np.uint8, "uint8", device)
        w, wp = self._grid_out(shape, np.float32, "float32", device) if want_w else (None, None)
        _check(load().gwn_classify_grid(self._h, px, len(ax), py, len(ay), pz, len(az), lp, wp, _stream_ptr(stream)))
        return (lab, w) if want_w else lab

    def classify(self, q, want_w: bool = False, stream=None):
        """Labels (uint8 [n], 1 iff w > 1/2) and optionally w."""
        qp, n, dev, keep = _points(q, "q")
        lab, lp = _alloc_like(q, dev, n, np.uint8, "uint8")
        w, wp = _alloc_like(q, dev, n, np.float32, "float32") if want_w else (None, None)
        _check(load().gwn_classify(self._h, qp, n, lp, wp, _stream_ptr(stream)))
        return (lab, w) if want_w else lab


    # -- learned surrogate (a per-mesh MLP of w on the tensor cores; gated, exact fallback)
    def train_surrogate(self, samples, targets=None, config: dict | None = None, stream=None) -> float:
        """Train the surrogate on CUDA float32 samples [n, 3] (targets: CUDA float32 [n],
        default: w from the antipodal path).  Returns the last batch's mean squared error."""
        qp, n, dev, keep = _points(samples, "samples")
        if not dev:
            raise ValueError("samples must be a CUDA tensor")
        tp = None
        if targets is not None:
            if not (_is_torch(targets) and targets.is_cuda and targets.dtype.is_floating_point):
                raise ValueError("targets must be a CUDA float32 tensor")
            targets = targets.contiguous().float()
            tp = ctypes.c_void_p(targets.data_ptr())
        cfg = MlpConfig()
        for k, v in (config or {}).items():
            setattr(cfg, k, v)
        loss = ctypes.c_float()
        _check(load().gwn_surrogate_train(self._h, qp, tp, n, ctypes.byref(cfg), ctypes.byref(loss),
                                          _stream_ptr(stream)))
        return float(loss.value)

    def surrogate_predict(self, q, stream=None):
        """Raw network output w_hat (CUDA float32 [n]) for CUDA queries."""
        torch = _torch()
        qp, n, dev, keep = _points(q, "q")
        if not dev:
            raise ValueError("q must be a CUDA tensor")
        w = torch.empty(n, dtype=torch.float32, device=q.device)
        _check(load().gwn_surrogate_predict(self._h, qp, n, ctypes.c_void_p(w.data_ptr()), _stream_ptr(stream)))
        return w

    def surrogate_params(self):
        """(FP32 parameter vector, input box [lo xyz, hi xyz]) as numpy arrays."""
        lib = load()
        p = np.empty(lib.gwn_surrogate_num_params(), np.float32)
        box = np.empty(6, np.float32)
        _check(lib.gwn_surrogate_params(self._h, p.ctypes.data_as(_P), box.ctypes.data_as(_P), 0))
        return p, box

    def set_surrogate_params(self, params, box):
        lib = load()
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.size != lib.gwn_surrogate_num_params():
            raise ValueError(f"expected {lib.gwn_surrogate_num_params()} parameters")
        b = np.ascontiguousarray(box, dtype=np.float32).reshape(6)
        _check(lib.gwn_surrogate_params(self._h, p.ctypes.data_as(_P), b.ctypes.data_as(_P), 1))

    def surrogate_grad(self, q, targets, stream=None):
        """(gradient of the mean squared error wrt the parameters, loss) on CUDA q, targets."""
        lib = load()
        qp, n, dev, keep = _points(q, "q")
        if not dev or not (_is_torch(targets) and targets.is_cuda):
            raise ValueError("q and targets must be CUDA tensors")
        targets = targets.contiguous().float()
        g = np.empty(lib.gwn_surrogate_num_params(), np.float32)
        loss = ctypes.c_float()
        _check(lib.gwn_surrogate_grad(self._h, qp, ctypes.c_void_p(targets.data_ptr()), n, g.ctypes.data_as(_P),
                                      ctypes.byref(loss), _stream_ptr(stream)))
        return g, float(loss.value)

    def calibrate_surrogate(self, samples, max_error_rate: float = 0.0, min_margin: float = 0.1, stream=None):
        """Raise the gate margin until at most ``max_error_rate`` of the held-out CUDA
        ``samples`` are answered by the network with a wrong label.  Returns
        (margin, confidently wrong samples at that margin)."""
        qp, n, dev, keep = _points(samples, "samples")
        if not dev:
            raise ValueError("samples must be a CUDA tensor")
        mg = ctypes.c_float()
        errs = ctypes.c_int64()
        _check(load().gwn_surrogate_calibrate(self._h, qp, n, float(max_error_rate), float(min_margin),
                                              ctypes.byref(mg), ctypes.byref(errs), _stream_ptr(stream)))
        return float(mg.value), int(errs.value)

    def save_surrogate(self, path: str):
        _check(load().gwn_surrogate_save(self._h, os.fsencode(path)))

    def load_surrogate(self, path: str):
        _check(load().gwn_surrogate_load(self._h, os.fsencode(path)))

    def detach_surrogate(self):
        _check(load().gwn_surrogate_detach(self._h))


class ParamSurface:
    """Untrimmed bicubic Bezier patches (float32 [np, 4, 4, 3]) on the GPU (Sec. 4.4).

    Keyword settings (library defaults when omitted): ``quad_tol``, ``flat_tol``,
    ``fp64`` (every quadrature panel in FP64), ``max_panels``, ``max_nodes``."""

    def __init__(self, patches, **settings):
        lib = load()
        if _is_torch(patches):
            patches = patches.detach().to("cpu").numpy()
        P = np.ascontiguousarray(patches, dtype=np.float32).reshape(-1, 4, 4, 3)
        cfg = ParamConfig()
        lib.gwn_param_config_default(ctypes.byref(cfg))
        for k, v in settings.items():
            if k not in dict(ParamConfig._fields_):
                raise TypeError(f"unknown setting {k!r}")
            setattr(cfg, k, int(v) if k in ("fp64", "max_panels", "max_nodes") else float(v))
        h = ctypes.c_void_p()
        _check(lib.gwn_param_create(P.ctypes.data_as(_P), P.shape[0], ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self.n_patches = P.shape[0]
        self.config = {k: getattr(cfg, k) for k, _ in ParamConfig._fields_}

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(load().gwn_param_destroy(self._h))
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

    def boundary_curves(self) -> np.ndarray:
        lib = load()
        n = ctypes.c_int32()
        _check(lib.gwn_param_get_boundary(self._h, None, 0, ctypes.byref(n)))
        out = np.empty((max(n.value, 1), 4, 3), np.float32)
        _check(lib.gwn_param_get_boundary(self._h, out.ctypes.data_as(_P), n.value, ctypes.byref(n)))
        return out[: n.value].copy()

    def query(self, q, stream=None):
        """(w float32 [n], chi int32 [n]) for CUDA queries [n, 3]."""
        torch = _torch()
        qp, n, dev, keep = _points(q, "q")
        if not dev:
            raise ValueError("q must be a CUDA tensor")
        w = torch.empty(n, dtype=torch.float32, device=q.device)
        chi = torch.empty(n, dtype=torch.int32, device=q.device)
        _check(load().gwn_param_query(self._h, qp, n, ctypes.c_void_p(w.data_ptr() if n else 0),
                                      ctypes.c_void_p(chi.data_ptr() if n else 0), _stream_ptr(stream)))
        return w, chi

    def query_grid(self, x, y, z, stream=None):
        """(w float32 [nz, ny, nx], chi int32 [nz, ny, nx]) of the cells (x[i], y[j], z[k]), on the GPU."""
        torch = _torch()
        axes = [np.ascontiguousarray(np.asarray(a.detach().cpu() if _is_torch(a) else a, dtype=np.float32).reshape(-1))
                for a in (x, y, z)]
        shape = (len(axes[2]), len(axes[1]), len(axes[0]))
        w = torch.empty(shape, dtype=torch.float32, device="cuda")
        chi = torch.empty(shape, dtype=torch.int32, device="cuda")
        n = w.numel()
        _check(load().gwn_param_query_grid(self._h, axes[0].ctypes.data_as(_P), len(axes[0]), axes[1].ctypes.data_as(_P),
                                           len(axes[1]), axes[2].ctypes.data_as(_P), len(axes[2]),
                                           ctypes.c_void_p(w.data_ptr() if n else 0),
                                           ctypes.c_void_p(chi.data_ptr() if n else 0), _stream_ptr(stream)))
        return w, chi

    def status(self, reset: bool = False):
        a, b, c, d = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().gwn_param_status(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d),
                                       1 if reset else 0))
        return {"budget_hits": int(a.value), "unconverged": int(b.value), "panels": int(c.value),
                "panels_fp64": int(d.value)}


class Batch:
    """Many built meshes evaluated in one persistent, graph-captured launch.

    ``meshes``: list of :class:`Mesh` (kept alive by the batch); ``counts``: the
    number of queries of each mesh, in order (the query rows are concatenated).
    """

    def __init__(self, meshes, counts, config: dict | None = None):
        lib = load()
        self._meshes = list(meshes)
        counts = np.asarray(counts, dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
        self.total = int(self.offsets[-1])
        arr = (_P * max(len(self._meshes), 1))(*[m.handle for m in self._meshes])
        cfg = BatchConfig()
        for k, v in (config or {}).items():
            setattr(cfg, k, v)
        h = ctypes.c_void_p()
        _check(lib.gwn_batch_create(arr, len(self._meshes), self.offsets.ctypes.data_as(_P), ctypes.byref(cfg),
                                    ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(load().gwn_batch_destroy(self._h))
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

    def run(self, q, w=None, chi=None, stream=None):
        """w (float32 [total]) and chi (int32 [total]) for the concatenated queries (CUDA tensors)."""
        torch = _torch()
        qp, n, dev, keep = _points(q, "q")
        if n != self.total or not dev:
            raise ValueError(f"q must be a CUDA tensor with {self.total} rows")
        if w is None:
            w = torch.empty(n, dtype=torch.float32, device=q.device)
        if chi is None:
            chi = torch.empty(n, dtype=torch.int32, device=q.device)
        _check(load().gwn_batch_run(self._h, qp, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(chi.data_ptr()),
                                    _stream_ptr(stream)))
        return w, chi

    def autotune(self, q, cache_path: str | None = None, stream=None) -> dict:
        torch = _torch()
        qp, n, dev, keep = _points(q, "q")
        w = torch.empty(n, dtype=torch.float32, device=q.device)
        cfg = BatchConfig()
        _check(load().gwn_batch_autotune(self._h, qp, ctypes.c_void_p(w.data_ptr()), _stream_ptr(stream),
                                         cache_path.encode() if cache_path else None, ctypes.byref(cfg)))
        return cfg.as_dict()

    def config(self) -> dict:
        cfg = BatchConfig()
        n = ctypes.c_int64()
        _check(load().gwn_batch_get_config(self._h, ctypes.byref(cfg), ctypes.byref(n)))
        d = cfg.as_dict()
        d["n_items"] = int(n.value)
        return d
