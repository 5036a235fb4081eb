"""Python binding of the C ABI in include/mf.h (argument marshalling only).

Every step of the solver runs in libmf.so (hand-written CUDA for sm_103a).
This module only converts numpy arrays / torch tensors into pointers and
sizes, calls the C functions of the same names and raises on a nonzero
status.  If the library has not been built it raises: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIBPATH = os.path.join(_HERE, "_lib", "libmf.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_EOVERFLOW, MF_ESWEEPLIMIT, MF_EROUNDLIMIT, MF_ESTATE = range(8)
MF_STATE_HOST = 1


def paper_stencil(c: int) -> int:
    """Connectivity code of the Sec. 7.1 synthetic stencil of connectivity c
    (c = 8, 12, ..., 28; MF_PAPER_STENCIL in mf.h); c = 4 is the plain 4."""
    return 4 if c == 4 else 100 + c


def arcs_of(connectivity: int) -> int:
    """Arcs per vertex of a connectivity code (2H)."""
    return connectivity - 100 if connectivity > 100 else connectivity
STATUS_NAMES = ["MF_OK", "MF_EINVAL", "MF_ENOMEM", "MF_ECUDA", "MF_EOVERFLOW", "MF_ESWEEPLIMIT",
                "MF_EROUNDLIMIT", "MF_ESTATE"]

# every symbol include/mf.h declares
EXPORTS = ["mf_default_opts", "mf_create_grid", "mf_create_grid_ex", "mf_set_caps", "mf_set_caps_batch", "mf_solve", "mf_begin", "mf_sweep",
           "mf_finish", "mf_boundary_relabel", "mf_region_reduction", "mf_get_cut", "mf_get_cuts_batch", "mf_flow_value", "mf_get_residual", "mf_get_labels", "mf_destroy",
           "mf_last_error", "mf_min_cut_2d_noalloc", "mf_solve_batch", "mf_warm_features", "mf_warm_targets",
           "mf_warm_start", "mf_warm_start_batch", "mf_certify", "mf_get_flow", "mf_load_model", "mf_cnn_create", "mf_cnn_destroy", "mf_cnn_last_error", "mf_cnn_num_params",
           "mf_cnn_get_params", "mf_cnn_set_params", "mf_cnn_get_grads", "mf_cnn_forward", "mf_cnn_infer",
           "mf_cnn_zero_grad",
           "mf_cnn_backward", "mf_cnn_mse", "mf_cnn_adam_step"]


class mf_opts(ctypes.Structure):
    _fields_ = [("max_sweeps", ctypes.c_int32), ("partial_discharge", ctypes.c_int32),
                ("global_gap", ctypes.c_int32), ("global_relabel_period", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("kernel_variant", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("graph_loop", ctypes.c_int32),
                ("boundary_relabel_period", ctypes.c_int32), ("global_relabel_first", ctypes.c_int32),
                ("region_reduction", ctypes.c_int32), ("reserved", ctypes.c_int32 * 5)]


class mf_stats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int32), ("boundary_size", ctypes.c_int32),
                ("discharges", ctypes.c_int64), ("discharged_vertices", ctypes.c_int64),
                ("stages", ctypes.c_int64), ("rounds", ctypes.c_int64), ("flow_value", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("gaps", ctypes.c_int32), ("cut_passes", ctypes.c_int32),
                ("ms_init", ctypes.c_double), ("ms_sweeps", ctypes.c_double), ("ms_cut", ctypes.c_double),
                ("ms_total", ctypes.c_double), ("ms_discharge", ctypes.c_double), ("ms_fuse", ctypes.c_double),
                ("global_relabels", ctypes.c_int32), ("relabel_levels", ctypes.c_int32),
                ("projection_rounds", ctypes.c_int32), ("boundary_relabels", ctypes.c_int32),
                ("boundary_relabel_levels", ctypes.c_int32), ("discharge_launches", ctypes.c_int32),
                ("reduced_vertices", ctypes.c_int32), ("reserved", ctypes.c_int32 * 1),
                ("ms_relabel", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class MFError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


_P, _I, _I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
# every exported call with its ctypes (restype, argtypes): a call without
# argtypes would pass 64-bit pointers as C int
SIGNATURES = {
    "mf_default_opts": (None, [ctypes.POINTER(mf_opts)]),
    "mf_create_grid": (_I, [ctypes.POINTER(_P), _I, _P, _I, _P, _P]),
    "mf_create_grid_ex": (_I, [ctypes.POINTER(_P), _I, _P, _I, _P, _P, _I]),
    "mf_set_caps": (_I, [_P, _P, _P, _P, _I]),
    "mf_set_caps_batch": (_I, [_P, _I, _P, _P, _P, _I]),
    "mf_get_cuts_batch": (_I, [_P, _I, _I, _P, _I, _P]),
    "mf_solve": (_I, [_P, ctypes.POINTER(mf_opts), ctypes.POINTER(mf_stats)]),
    "mf_begin": (_I, [_P, ctypes.POINTER(mf_opts)]),
    "mf_sweep": (_I, [_P, ctypes.POINTER(ctypes.c_int32)]),
    "mf_finish": (_I, [_P]),
    "mf_boundary_relabel": (_I, [_P, _P]),
    "mf_region_reduction": (_I, [_P, _P, _P, _I, _P]),
    "mf_get_cut": (_I, [_P, _P, _I, _I]),
    "mf_flow_value": (_I, [_P, ctypes.POINTER(_I64)]),
    "mf_get_residual": (_I, [_P, _P, _P, _P, _I]),
    "mf_get_labels": (_I, [_P, _P, ctypes.POINTER(ctypes.c_int32), _I]),
    "mf_destroy": (_I, [_P]),
    "mf_last_error": (ctypes.c_char_p, [_P]),
    "mf_min_cut_2d_noalloc": (_I, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "mf_solve_batch": (_I, [_P, _I, ctypes.POINTER(mf_opts), ctypes.POINTER(mf_stats)]),
    "mf_warm_features": (_I, [_P, _P]),
    "mf_warm_targets": (_I, [_P, _P]),
    "mf_warm_start": (_I, [_P, _P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "mf_warm_start_batch": (_I, [_P, _I, _P, ctypes.c_int32, _P]),
    "mf_get_flow": (_I, [_P, _P]),
    "mf_load_model": (_I, [_P, ctypes.c_char_p]),
    "mf_certify": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int32)]),
    "mf_cnn_create": (_I, [ctypes.POINTER(_P), _I, _I, ctypes.c_uint64, _P]),
    "mf_cnn_destroy": (_I, [_P]),
    "mf_cnn_last_error": (ctypes.c_char_p, [_P]),
    "mf_cnn_num_params": (_I64, [_P]),
    "mf_cnn_get_params": (_I, [_P, _P, _I]),
    "mf_cnn_set_params": (_I, [_P, _P, _I]),
    "mf_cnn_get_grads": (_I, [_P, _P, _I]),
    "mf_cnn_forward": (_I, [_P, _P, _I, _I, _I, _P]),
    "mf_cnn_infer": (_I, [_P, _P, _I, _I, _I, _P]),
    "mf_cnn_zero_grad": (_I, [_P]),
    "mf_cnn_backward": (_I, [_P, _P, _P]),
    "mf_cnn_mse": (_I, [_P, _P, _P, _P, _I64, ctypes.POINTER(ctypes.c_double)]),
    "mf_cnn_adam_step": (_I, [_P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]),
}

_lib = None


def load(path: str = LIBPATH):
    """Load libmf.so (raises if it is missing: build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libmf.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    if set(SIGNATURES) != set(EXPORTS):
        raise ImportError("binding signatures and exported names differ")
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


_OPT_FIELDS = {name for name, _ in mf_opts._fields_ if name != "reserved"}


def default_opts(**kw) -> mf_opts:
    """mf_opts with the library's defaults, then the given fields (an unknown
    name raises instead of becoming a Python attribute the library never sees)."""
    unknown = set(kw) - _OPT_FIELDS
    if unknown:
        raise TypeError(f"unknown mf_opts fields: {sorted(unknown)}")
    o = mf_opts()
    load().mf_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, int(v))
    return o


_CUDA_STREAM_LEGACY = 1  # the cudaStream_t value of the legacy default stream


def _stream_arg(stream):
    """cudaStream_t for the library.  An explicit stream (torch stream or raw
    handle) is used as given; with none, torch's current stream when torch's
    CUDA is in use, so that library calls and torch kernels on the caller's
    stream stay ordered; otherwise NULL (the library's own stream).  torch's
    default stream has handle 0, which the library would read as NULL, so it
    is passed as the legacy-stream handle instead."""
    if stream is None:
        torch = sys.modules.get("torch")
        if torch is None or not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    h = stream if isinstance(stream, int) else stream.cuda_stream
    return h if h else _CUDA_STREAM_LEGACY


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor (contiguous int32/uint8)."""
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), int(a.is_cuda)
    raise TypeError(f"unsupported buffer type {type(a)}")


def min_cut_2d_noalloc(dims, connectivity, res, tres, exc, smin, smax, stream=None):
    """Allocation-free cut extraction (see include/mf.h): all buffers are
    device tensors; raises MFError on a nonzero status."""
    lib = load()
    d = (ctypes.c_int64 * 2)(int(dims[0]), int(dims[1]))
    ptrs = []
    for a in (res, tres, exc, smin, smax):
        p, dev = _ptr(a)
        if not dev:
            raise ValueError("mf_min_cut_2d_noalloc takes device buffers")
        ptrs.append(p)
    s = _stream_arg(stream)
    st = lib.mf_min_cut_2d_noalloc(d, int(connectivity), *ptrs, s)
    if st != MF_OK:
        raise MFError(st, lib.mf_last_error(None).decode())


def warm_start_batch(grids, preds, max_rounds=0):
    """mf_warm_start_batch: preds[i] a device float tensor [N+2, n] or None;
    returns the phases of each grid (-1: no preflow, cold)."""
    lib = load()
    n = len(grids)
    arr = (ctypes.c_void_p * n)(*[g._h.value for g in grids])
    ps = (ctypes.c_void_p * n)(*[None if p is None else _ptr(p)[0] for p in preds])
    rounds = (ctypes.c_int32 * n)()
    st = lib.mf_warm_start_batch(arr, n, ps, int(max_rounds), rounds)
    if st != MF_OK:
        raise MFError(st, lib.mf_last_error(grids[0]._h).decode())
    return list(rounds)


def set_caps_batch(grids, caps):
    """mf_set_caps_batch: caps[i] = (cs, ct, nlink) for grids[i] (all host or
    all device buffers); one wait for all grids."""
    lib = load()
    n = len(grids)
    arr = (ctypes.c_void_p * n)(*[g._h.value for g in grids])
    pcs, pct, pnl, devs = [], [], [], set()
    for cs, ct, nl in caps:
        for buf, out in ((cs, pcs), (ct, pct), (nl, pnl)):
            p, dev = _ptr(buf)
            out.append(p)
            devs.add(dev)
    if len(devs) != 1:
        raise ValueError("the capacities must all be host or all be device buffers")
    st = lib.mf_set_caps_batch(arr, n, (ctypes.c_void_p * n)(*pcs), (ctypes.c_void_p * n)(*pct),
                               (ctypes.c_void_p * n)(*pnl), devs.pop())
    if st != MF_OK:
        raise MFError(st, lib.mf_last_error(grids[0]._h).decode())


def get_cuts_batch(grids, which=0, outs=None):
    """mf_get_cuts_batch: the cut `which` of every grid into outs (uint8
    buffers, all host or all device; allocated on the host if None) and every
    flow value; one wait for all grids.  Returns (outs, flows)."""
    lib = load()
    n = len(grids)
    if outs is None:
        outs = [np.empty(g.n, dtype=np.uint8) for g in grids]
    arr = (ctypes.c_void_p * n)(*[g._h.value for g in grids])
    ptrs, devs = [], set()
    for o in outs:
        p, dev = _ptr(o)
        ptrs.append(p)
        devs.add(dev)
    if len(devs) != 1:
        raise ValueError("the outputs must all be host or all be device buffers")
    flows = (ctypes.c_int64 * n)()
    st = lib.mf_get_cuts_batch(arr, n, int(which), (ctypes.c_void_p * n)(*ptrs), devs.pop(), flows)
    if st != MF_OK:
        raise MFError(st, lib.mf_last_error(grids[0]._h).decode())
    return outs, list(flows)


def solve_batch(grids, opts: mf_opts | None = None):
    """mf_solve_batch over a list of Grid objects; returns their mf_stats."""
    lib = load()
    n = len(grids)
    arr = (ctypes.c_void_p * n)(*[g._h.value for g in grids])
    stats = (mf_stats * n)()
    st = lib.mf_solve_batch(arr, n, None if opts is None else ctypes.byref(opts), stats)
    if st != MF_OK:
        raise MFError(st, lib.mf_last_error(grids[0]._h).decode())
    return list(stats)


class Grid:
    """One grid instance (owns a mf_grid handle)."""

    def __init__(self, dims, connectivity, tile=None, stream=None, host_state=False):
        """host_state: the planes live in pinned host memory (MF_STATE_HOST)."""
        lib = load()
        dims = tuple(int(d) for d in dims) + (1,) * (3 - len(dims))
        self.ndim = 3 if connectivity == 6 else 2
        self.dims = dims
        self.conn = connectivity
        self.n = dims[0] * dims[1] * dims[2]
        self.H = arcs_of(connectivity) // 2
        d = (ctypes.c_int64 * 3)(*dims)
        t = None if tile is None else (ctypes.c_int32 * 3)(*(tuple(tile) + (1,) * (3 - len(tile))))
        s = _stream_arg(stream)
        h = ctypes.c_void_p()
        st = lib.mf_create_grid_ex(ctypes.byref(h), self.ndim, d, connectivity, t, s, MF_STATE_HOST if host_state else 0)
        if st != MF_OK:
            raise MFError(st, lib.mf_last_error(None).decode())
        self._h = h
        self._lib = lib

    def _check(self, st):
        if st != MF_OK:
            raise MFError(st, self._lib.mf_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_caps(self, cs, ct, nlink):
        pc, dc = _ptr(cs)
        pt, dt = _ptr(ct)
        pn, dn = _ptr(nlink)
        if not (dc == dt == dn):
            raise ValueError("cs, ct and nlink must all be host or all be device buffers")
        self._check(self._lib.mf_set_caps(self._h, pc, pt, pn, dc))

    def solve(self, opts: mf_opts | None = None, check=True):
        stats = mf_stats()
        st = self._lib.mf_solve(self._h, None if opts is None else ctypes.byref(opts), ctypes.byref(stats))
        if check:
            self._check(st)
        return stats

    def begin(self, opts: mf_opts | None = None):
        self._check(self._lib.mf_begin(self._h, None if opts is None else ctypes.byref(opts)))

    def sweep(self) -> int:
        a = ctypes.c_int32()
        self._check(self._lib.mf_sweep(self._h, ctypes.byref(a)))
        return a.value

    def finish(self):
        self._check(self._lib.mf_finish(self._h))

    def boundary_relabel(self) -> dict:
        """One boundary relabel (Sec. 6.1) on the current state (after begin or
        a sweep): dict(active, levels, merged, applied)."""
        info = (ctypes.c_int32 * 4)()
        self._check(self._lib.mf_boundary_relabel(self._h, ctypes.addressof(info)))
        return {"active": info[0], "levels": info[1], "merged": info[2], "applied": bool(info[3])}

    def region_reduction(self, tile=None, out=None):
        """Region reduction of Sec. 8 (mf_region_reduction): (codes uint8[n],
        counts [strong sources, strong sinks, weak sources, weak sinks])."""
        if out is None:
            out = np.empty(self.n, dtype=np.uint8)
        p, dev = _ptr(out)
        t = None if tile is None else (ctypes.c_int32 * 3)(*(tuple(tile) + (1,) * (3 - len(tile))))
        cnt = (ctypes.c_int64 * 4)()
        self._check(self._lib.mf_region_reduction(self._h, t, p, dev, ctypes.addressof(cnt)))
        return out, list(cnt)

    def get_cut(self, which=0, out=None):
        if out is None:
            out = np.empty(self.n, dtype=np.uint8)
        p, dev = _ptr(out)
        self._check(self._lib.mf_get_cut(self._h, p, int(which), dev))
        return out

    def flow_value(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.mf_flow_value(self._h, ctypes.byref(v)))
        return v.value

    def get_residual(self):
        res = np.empty((2 * self.H, self.n), dtype=np.int32)
        tres = np.empty(self.n, dtype=np.int32)
        exc = np.empty(self.n, dtype=np.int32)
        self._check(self._lib.mf_get_residual(self._h, res.ctypes.data, tres.ctypes.data, exc.ctypes.data, 0))
        return res, tres, exc

    def warm_features(self, x):
        """x: device float tensor [2+N, n]."""
        p, dev = _ptr(x)
        assert dev
        self._check(self._lib.mf_warm_features(self._h, p))

    def warm_targets(self, t):
        """t: device float tensor [N+2, n] (after a solve)."""
        p, dev = _ptr(t)
        assert dev
        self._check(self._lib.mf_warm_targets(self._h, p))

    def warm_start(self, pred, max_rounds=0, check=True):
        """Project a prediction (device float [N+2, n]) to the initial preflow of
        the next solve with warm_start=1; returns (status, rounds)."""
        p, dev = _ptr(pred)
        assert dev
        r = ctypes.c_int32()
        st = self._lib.mf_warm_start(self._h, p, int(max_rounds), ctypes.byref(r))
        if check:
            self._check(st)
        return st, r.value

    def certify(self):
        """(certified, cut capacity of S_min, violations) of the last solve."""
        cut, bad, ok = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int32()
        self._check(self._lib.mf_certify(self._h, ctypes.byref(cut), ctypes.byref(bad), ctypes.byref(ok)))
        return bool(ok.value), cut.value, bad.value

    def get_flow(self):
        """Residual capacities int32[2H, n] (mf_get_flow)."""
        res = np.empty((self.H * 2, self.n), dtype=np.int32)
        self._check(self._lib.mf_get_flow(self._h, res.ctypes.data))
        return res

    def get_labels(self):
        lab = np.empty(self.n, dtype=np.int32)
        dinf = ctypes.c_int32()
        self._check(self._lib.mf_get_labels(self._h, lab.ctypes.data, ctypes.byref(dinf), 0))
        return lab, dinf.value


class CNN:
    """The warm-start network (see include/mf.h); buffers are torch CUDA tensors."""

    def __init__(self, channels=6, seed=0, stream=None):
        lib = load()
        h = ctypes.c_void_p()
        s = _stream_arg(stream)
        st = lib.mf_cnn_create(ctypes.byref(h), channels, channels, ctypes.c_uint64(seed), s)
        if st != MF_OK:
            raise MFError(st, lib.mf_last_error(None).decode())
        self._h, self._lib, self.channels = h, lib, channels

    def _check(self, st):
        if st != MF_OK:
            raise MFError(st, self._lib.mf_cnn_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mf_cnn_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_params(self):
        return int(self._lib.mf_cnn_num_params(self._h))

    def get_params(self):
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(self._lib.mf_cnn_get_params(self._h, out.ctypes.data, 0))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self._lib.mf_cnn_set_params(self._h, p.ctypes.data, 0))

    def get_grads(self):
        out = np.empty(self.num_params, dtype=np.float32)
        self._check(self._lib.mf_cnn_get_grads(self._h, out.ctypes.data, 0))
        return out

    def forward(self, x, y):
        N, C, H, W = x.shape
        self._check(self._lib.mf_cnn_forward(self._h, x.data_ptr(), N, H, W, y.data_ptr()))

    def infer(self, x, y):
        N, C, H, W = x.shape
        self._check(self._lib.mf_cnn_infer(self._h, x.data_ptr(), N, H, W, y.data_ptr()))

    def load(self, path):
        """Parameters from a .npy file (mf_load_model)."""
        self._check(self._lib.mf_load_model(self._h, os.fsencode(path)))

    def zero_grad(self):
        self._check(self._lib.mf_cnn_zero_grad(self._h))

    def backward(self, x, dy):
        self._check(self._lib.mf_cnn_backward(self._h, x.data_ptr(), dy.data_ptr()))

    def mse(self, y, t, dy):
        loss = ctypes.c_double()
        self._check(self._lib.mf_cnn_mse(self._h, y.data_ptr(), t.data_ptr(), dy.data_ptr(), y.numel(),
                                         ctypes.byref(loss)))
        return loss.value

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self._lib.mf_cnn_adam_step(self._h, lr, beta1, beta2, eps))
