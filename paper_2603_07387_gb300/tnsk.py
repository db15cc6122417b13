"""ctypes binding of libtnsk (include/tnsk.h). Argument marshalling only.

Every step of the estimators runs in the CUDA kernels of libtnsk.so; this module
turns Python lists and torch CUDA tensors into the C structs and raises on a
non-OK status. It fails loudly when libtnsk.so has not been built: there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field
from typing import Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtnsk.so")

TNSK_OK = 0
ERR_UNREACHABLE = -7
STATUS = {
    0: "TNSK_OK",
    -1: "TNSK_ERR_INVALID",
    -2: "TNSK_ERR_CYCLIC",
    -3: "TNSK_ERR_UNSUPPORTED",
    -4: "TNSK_ERR_CUDA",
    -5: "TNSK_ERR_OOM",
    -6: "TNSK_ERR_TIMEOUT",
    -7: "TNSK_ERR_UNREACHABLE",
}
F64, F32, BF16 = 0, 1, 2
GENERAL, ACYCLIC, CROSSCORR = 1, 2, 3  # tnsk_method (CROSSCORR: the earlier cross-correlation estimator)
KERNEL_KINDS = ("tables", "m1_scatter", "m1_spectrum", "m2_leaf", "m2_compose", "m2_vbuild", "m2_gemm",
                "m2_root", "combine", "m2_scatter", "pairs", "normalize", "m2_prep")
PREC_FP32, PREC_BF16, PREC_FP64, PREC_AUTO = 0, 1, 2, 3

# exported symbols declared in include/tnsk.h
SYMBOLS = (
    "tnsk_create",
    "tnsk_destroy",
    "tnsk_set_stream",
    "tnsk_count_sketch",
    "tnsk_m1_sketch",
    "tnsk_estimate",
    "tnsk_estimate_batch",
    "tnsk_estimate_static",
    "tnsk_rewrite",
    "tnsk_plan_create",
    "tnsk_plan_create_scheduled",
    "tnsk_autotune",
    "tnsk_plan_run",
    "tnsk_plan_destroy",
    "tnsk_plan_set_prelude",
    "tnsk_profile",
    "tnsk_profile_read",
    "tnsk_debug_inject",
    "tnsk_sync",
    "tnsk_probe_shared_atomics",
    "tnsk_probe_shared_int_adds",
    "tnsk_auto_report",
    "tnsk_combine",
    "tnsk_stream_create",
    "tnsk_stream_update",
    "tnsk_stream_estimate",
    "tnsk_stream_sketches",
    "tnsk_stream_destroy",
    "tnsk_mlp_num_params",
    "tnsk_mlp_create",
    "tnsk_mlp_destroy",
    "tnsk_mlp_get",
    "tnsk_mlp_set",
    "tnsk_mlp_loss_grad",
    "tnsk_mlp_train",
    "tnsk_mlp_predict",
    "tnsk_mlp_save",
    "tnsk_mlp_load",
    "tnsk_features",
    "tnsk_pairs_create",
    "tnsk_pairs_run",
    "tnsk_pairs_destroy",
    "tnsk_contract_pairs",
    "tnsk_choose_params",
    "tnsk_choose_params_batch",
    "tnsk_choose_params_rate",
    "tnsk_status_string",
    "tnsk_last_error",
)


class TnskError(RuntimeError):
    def __init__(self, status: int, message: str = ""):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class _Rung(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("a", ctypes.c_int64),
        ("s", ctypes.c_int64),
        ("c", ctypes.c_int64),
        ("b", ctypes.c_int64),
        ("d", ctypes.c_int64),
    ]


class _Tensor(ctypes.Structure):
    _fields_ = [
        ("order", ctypes.c_int32),
        ("dims", ctypes.POINTER(ctypes.c_int64)),
        ("data", ctypes.c_void_p),
        ("dtype", ctypes.c_int32),
        ("rung", ctypes.POINTER(_Rung)),
    ]


class _Network(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int32),
        ("X", ctypes.POINTER(_Tensor)),
        ("t", ctypes.c_int32),
        ("edges", ctypes.POINTER(ctypes.c_int32)),
        ("n_open", ctypes.c_int32),
        ("open", ctypes.POINTER(ctypes.c_int32)),
    ]


SCATTER_LISTS = 16


class Schedule(ctypes.Structure):
    """tnsk_schedule: per scatter list (order class c + 4 x kernel kind) the most reps
    per work item and the chunk multiple; zeros are the defaults."""
    _fields_ = [("rep_cap", ctypes.c_int32 * SCATTER_LISTS), ("chunk_scale", ctypes.c_int32 * SCATTER_LISTS)]

    def as_dict(self):
        return {"rep_cap": list(self.rep_cap), "chunk_scale": list(self.chunk_scale)}

    @classmethod
    def from_dict(cls, d) -> "Schedule":
        """The schedule of a table {"rep_cap": [...], "chunk_scale": [...]} (one non-negative
        integer per scatter list; 0 keeps the default), e.g. one tnsk_autotune found."""
        s = cls()
        for key in ("rep_cap", "chunk_scale"):
            vals = [int(v) for v in d[key]]
            if len(vals) != SCATTER_LISTS or min(vals) < 0:
                raise ValueError(f"{key}: {SCATTER_LISTS} non-negative integers expected")
            getattr(s, key)[:] = vals
        return s

    def save(self, path: str):
        """Writes the schedule as a JSON table (as_dict) for later plans."""
        import json

        with open(path, "w") as f:
            json.dump(self.as_dict(), f)

    @classmethod
    def load(cls, path: str) -> "Schedule":
        """A schedule saved by save(): ctx.plan(..., schedule=Schedule.load(path))."""
        import json

        with open(path) as f:
            return cls.from_dict(json.load(f))


class _Params(ctypes.Structure):
    _fields_ = [
        ("m", ctypes.c_int64),
        ("reps", ctypes.c_int32),
        ("groups", ctypes.c_int32),
        ("seed", ctypes.c_uint64),
        ("method", ctypes.c_int32),
        ("root", ctypes.c_int32),
        ("prec", ctypes.c_int32),
        ("rep0", ctypes.c_int32),
    ]


_lib = None


def load_library(path: str = LIB_PATH):
    """Loads libtnsk.so; raises if it is missing (build it with __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtnsk.so not found at {path}: build it with __graft_entry__.build()")
    L = ctypes.CDLL(path)
    vp, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64
    L.tnsk_create.restype = i32
    L.tnsk_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp]
    pi32, pi64 = ctypes.POINTER(i32), ctypes.POINTER(i64)
    L.tnsk_rewrite.restype = i32
    L.tnsk_rewrite.argtypes = [vp, vp, i32, pi32, pi32, pi32, i64, pi64, i32, pi32, pi32]
    L.tnsk_destroy.restype = i32
    L.tnsk_destroy.argtypes = [vp]
    L.tnsk_set_stream.restype = i32
    L.tnsk_set_stream.argtypes = [vp, vp]
    L.tnsk_count_sketch.restype = i32
    L.tnsk_count_sketch.argtypes = [vp, u64, u64, u64, i64, i64, vp, vp]
    L.tnsk_m1_sketch.restype = i32
    L.tnsk_m1_sketch.argtypes = [vp, ctypes.POINTER(_Network), ctypes.POINTER(_Params), vp]
    L.tnsk_estimate.restype = i32
    L.tnsk_estimate.argtypes = [vp, ctypes.POINTER(_Network), ctypes.POINTER(_Params), vp, vp]
    L.tnsk_estimate_batch.restype = i32
    L.tnsk_estimate_batch.argtypes = [vp, i32, ctypes.POINTER(_Network), ctypes.POINTER(_Params),
                                      ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.tnsk_estimate_static.restype = i32
    L.tnsk_estimate_static.argtypes = [ctypes.POINTER(_Network), ctypes.POINTER(_Params), vp, vp, vp]
    L.tnsk_plan_create.restype = i32
    L.tnsk_plan_create.argtypes = [vp, i32, ctypes.POINTER(_Network), ctypes.POINTER(_Params), ctypes.POINTER(vp),
                                   ctypes.POINTER(vp), ctypes.POINTER(vp)]
    L.tnsk_plan_create_scheduled.restype = i32
    L.tnsk_plan_create_scheduled.argtypes = [vp, i32, ctypes.POINTER(_Network), ctypes.POINTER(_Params),
                                             ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(Schedule),
                                             ctypes.POINTER(vp)]
    L.tnsk_autotune.restype = i32
    L.tnsk_autotune.argtypes = [vp, i32, ctypes.POINTER(_Network), ctypes.POINTER(_Params), i32,
                                ctypes.POINTER(Schedule), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    L.tnsk_plan_run.restype = i32
    L.tnsk_plan_run.argtypes = [vp, vp]
    L.tnsk_plan_destroy.restype = i32
    L.tnsk_plan_destroy.argtypes = [vp]
    L.tnsk_plan_set_prelude.restype = i32
    L.tnsk_plan_set_prelude.argtypes = [vp, vp, vp]
    L.tnsk_profile.restype = i32
    L.tnsk_profile.argtypes = [vp, i32]
    L.tnsk_profile_read.restype = i32
    L.tnsk_profile_read.argtypes = [vp, vp, vp]
    L.tnsk_debug_inject.restype = i32
    L.tnsk_debug_inject.argtypes = [vp, i32]
    L.tnsk_sync.restype = i32
    L.tnsk_sync.argtypes = [vp]
    f32p, dp = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double)
    for name, args in [
        ("tnsk_mlp_num_params", [ctypes.POINTER(i64)]),
        ("tnsk_mlp_create", [vp, u64, ctypes.POINTER(vp)]),
        ("tnsk_mlp_destroy", [vp]),
        ("tnsk_mlp_get", [vp, f32p, f32p]),
        ("tnsk_mlp_set", [vp, vp, f32p, f32p]),
        ("tnsk_mlp_loss_grad", [vp, vp, vp, vp, i64, vp, dp]),
        ("tnsk_mlp_train", [vp, vp, vp, vp, i64, i32, i32, ctypes.c_float, u64, dp]),
        ("tnsk_mlp_predict", [vp, vp, vp, i64, vp, i32]),
        ("tnsk_mlp_save", [vp, ctypes.c_char_p]),
        ("tnsk_mlp_load", [vp, vp, ctypes.c_char_p]),
        ("tnsk_features", [vp, ctypes.POINTER(_Network), ctypes.POINTER(_Params), f32p]),
        ("tnsk_pairs_create", [vp, i32, vp, ctypes.POINTER(vp)]),
        ("tnsk_pairs_run", [vp, vp]),
        ("tnsk_pairs_destroy", [vp]),
        ("tnsk_contract_pairs", [vp, i32, vp]),
        ("tnsk_choose_params", [vp, ctypes.POINTER(_Network), ctypes.c_double, vp, ctypes.POINTER(_Params), dp]),
        ("tnsk_choose_params_batch", [vp, i32, vp, ctypes.c_double, vp, i32, vp, vp, vp]),
        ("tnsk_choose_params_rate", [vp, i32, vp, ctypes.c_double, vp, i32, vp, vp, vp]),
    ]:
        getattr(L, name).restype = i32
        getattr(L, name).argtypes = args
    L.tnsk_combine.restype = i32
    L.tnsk_combine.argtypes = [vp, i32, i64, vp, i32, vp]
    L.tnsk_stream_create.restype = i32
    L.tnsk_stream_create.argtypes = [vp, ctypes.POINTER(_Network), ctypes.POINTER(_Params), vp, vp, ctypes.POINTER(vp)]
    L.tnsk_stream_update.restype = i32
    L.tnsk_stream_update.argtypes = [vp, vp, i64, vp, vp, vp]
    L.tnsk_stream_estimate.restype = i32
    L.tnsk_stream_estimate.argtypes = [vp, vp]
    L.tnsk_stream_sketches.restype = i32
    L.tnsk_stream_sketches.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(ctypes.c_int64)]
    L.tnsk_stream_destroy.restype = i32
    L.tnsk_stream_destroy.argtypes = [vp]
    L.tnsk_probe_shared_atomics.restype = i32
    L.tnsk_probe_shared_atomics.argtypes = [vp, ctypes.POINTER(ctypes.c_double)]
    L.tnsk_probe_shared_int_adds.restype = i32
    L.tnsk_probe_shared_int_adds.argtypes = [vp, vp]
    L.tnsk_auto_report.restype = i32
    L.tnsk_auto_report.argtypes = [vp, vp, vp]
    L.tnsk_status_string.restype = ctypes.c_char_p
    L.tnsk_status_string.argtypes = [i32]
    L.tnsk_last_error.restype = ctypes.c_char_p
    L.tnsk_last_error.argtypes = [vp]
    _lib = L
    return L


@dataclass
class Network:
    """Tensors (torch CUDA tensors, row-major/contiguous), contractions E as pairs of
    global 0-based mode ids, and the output order of the open modes."""

    tensors: Sequence
    edges: Sequence[tuple[int, int]]
    open: Sequence[int] = ()

    def __getstate__(self):  # the cached marshalled form (ctypes) stays behind
        d = dict(self.__dict__)
        d.pop("_holder", None)
        return d


@dataclass
class Params:
    m: int
    reps: int
    groups: int = 1
    seed: int = 0
    method: int = GENERAL
    root: int = -1
    prec: int = PREC_FP32
    rep0: int = 0  # first repetition index (shards of one estimate)


def _dtype_code(t):
    import torch

    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.float64:
        return F64
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported tensor dtype {t.dtype}")


class Rung:
    """A grouped tensor (tnsk_rung): R[(i, j), (k, l)] = sum_s A[i, s, k] B[j, s, l] for
    contiguous FP32 CUDA tensors A [a, s, c] and B [b, s, d]; an order-2 tensor of
    shape (a*b, c*d) whose entries the method-2 sketch product forms from A and B."""

    def __init__(self, A, B):
        if A.dim() != 3 or B.dim() != 3 or A.shape[1] != B.shape[1]:
            raise ValueError("rung factors are [a, s, c] and [b, s, d] with equal s")
        self.A, self.B = A, B
        a, s, c = A.shape
        b, _, d = B.shape
        self.shape = (a * b, c * d)

    def dim(self):
        return 2

    def numel(self):
        return self.shape[0] * self.shape[1]


class Zeros:
    """An all-zero tensor of the given shape that is never stored (data NULL): a
    turnstile stream's sparse input, whose nonzeros arrive as updates."""

    def __init__(self, *shape, dtype=None):
        self.shape = tuple(int(d) for d in shape)
        self.dtype = dtype

    def dim(self):
        return len(self.shape)

    def numel(self):
        n = 1
        for d in self.shape:
            n *= d
        return n


class _NetHolder:
    """Owns the ctypes arrays behind one tnsk_network."""

    def __init__(self, net: Network):
        self.dims = []
        self.rungs = []
        tens = (_Tensor * max(1, len(net.tensors)))()
        for k, x in enumerate(net.tensors):
            if isinstance(x, Rung):
                for f in (x.A, x.B):
                    if not f.is_contiguous() or _dtype_code(f) != F32:
                        raise ValueError(f"tensor {k}: rung factors must be contiguous FP32")
                a, s, c = x.A.shape
                b, _, dd = x.B.shape
                g = _Rung(x.A.data_ptr(), x.B.data_ptr(), a, s, c, b, dd)
                self.rungs.append(g)
                d = (ctypes.c_int64 * 2)(*x.shape)
                self.dims.append(d)
                tens[k].order = 2
                tens[k].dims = ctypes.cast(d, ctypes.POINTER(ctypes.c_int64))
                tens[k].data = None
                tens[k].dtype = F32
                tens[k].rung = ctypes.pointer(g)
                continue
            if isinstance(x, Zeros):  # all zeros, data NULL (turnstile streams only)
                d = (ctypes.c_int64 * max(1, len(x.shape)))(*x.shape)
                self.dims.append(d)
                tens[k].order = len(x.shape)
                tens[k].dims = ctypes.cast(d, ctypes.POINTER(ctypes.c_int64))
                tens[k].data = None
                tens[k].dtype = F32 if x.dtype is None else _dtype_code(x)
                continue
            if x.numel() > 0 and not x.is_contiguous():
                raise ValueError(f"tensor {k} must be contiguous (row-major)")
            d = (ctypes.c_int64 * max(1, x.dim()))(*x.shape)
            self.dims.append(d)
            tens[k].order = x.dim()
            tens[k].dims = ctypes.cast(d, ctypes.POINTER(ctypes.c_int64))
            tens[k].data = x.data_ptr() if x.numel() > 0 else None
            tens[k].dtype = _dtype_code(x)
        self.tens = tens
        flat = [int(m) for e in net.edges for m in e]
        self.edges = (ctypes.c_int32 * max(1, len(flat)))(*flat)
        self.open = (ctypes.c_int32 * max(1, len(net.open)))(*[int(g) for g in net.open])
        self.c = _Network(
            len(net.tensors),
            ctypes.cast(tens, ctypes.POINTER(_Tensor)),
            len(net.edges),
            ctypes.cast(self.edges, ctypes.POINTER(ctypes.c_int32)),
            len(net.open),
            ctypes.cast(self.open, ctypes.POINTER(ctypes.c_int32)),
        )
        self.keep = list(net.tensors)


def _storage_key(x):
    if isinstance(x, Rung):
        return (x.A.data_ptr(), x.B.data_ptr())
    if isinstance(x, Zeros):
        return None
    return x.data_ptr()


def _holder(net: Network) -> _NetHolder:
    """The network's marshalled form (_NetHolder), built on first use and kept on the
    Network while it holds the same tensor objects over the same storage, the same
    edges and the same open modes; a batch of many networks then costs one check per
    network instead of a rebuild."""
    h = net.__dict__.get("_holder")
    ts = net.tensors
    if (h is not None and len(h.keep) == len(ts) and all(a is b for a, b in zip(h.keep, ts))
            and h.storage == [_storage_key(x) for x in ts] and h.edge_list == list(net.edges)
            and h.open_ == list(net.open)):
        return h
    h = _NetHolder(net)
    h.storage = [_storage_key(x) for x in ts]
    h.edge_list = list(net.edges)
    h.open_ = list(net.open)
    net.__dict__["_holder"] = h
    return h


def _params(p: Params) -> _Params:
    return _Params(int(p.m), int(p.reps), int(p.groups), int(p.seed) & ((1 << 64) - 1), int(p.method),
                   int(p.root), int(p.prec), int(p.rep0))


def estimate_static(net: Network, params: Params, out, per_rep=None, stream=None):
    """tnsk_estimate_static: method-1 estimate with no device allocation (all scratch
    in the library's fixed 16 MiB device array). Needs no Context."""
    L = load_library()
    nh = _holder(net)
    pr = _params(params)
    st = L.tnsk_estimate_static(ctypes.byref(nh.c), ctypes.byref(pr), out.data_ptr(),
                                per_rep.data_ptr() if per_rep is not None else None,
                                ctypes.c_void_p(int(stream)) if stream else None)
    if st != TNSK_OK:
        raise TnskError(st, "tnsk_estimate_static")


def rewrite(net: Network, params: Params):
    """tnsk_rewrite: the network the library plans after the WLOG rewrites of Sec. 4.1,
    computed on the host (no device work; tensors may be CPU tensors): (shapes, edges,
    copy) with copy[k] True for a WLOG 1 copy tensor."""
    L = load_library()
    nh = _holder(net)
    pr = _params(params)
    q = sum(len(x.shape) for x in net.tensors)
    cap_t, cap_e = len(net.tensors) + max(1, len(net.edges)), max(1, 2 * len(net.edges))
    cap_d = q + 2 * len(net.edges) + 1
    p_out, t_out = ctypes.c_int32(), ctypes.c_int32()
    order = (ctypes.c_int32 * cap_t)()
    copy = (ctypes.c_int32 * cap_t)()
    dims = (ctypes.c_int64 * cap_d)()
    edges = (ctypes.c_int32 * (2 * cap_e))()
    st = L.tnsk_rewrite(ctypes.byref(nh.c), ctypes.byref(pr), cap_t, ctypes.byref(p_out), order, copy, cap_d, dims,
                        cap_e, ctypes.byref(t_out), edges)
    if st != TNSK_OK:
        raise TnskError(st, "tnsk_rewrite")
    shapes, o = [], 0
    for k in range(p_out.value):
        shapes.append(tuple(int(dims[o + j]) for j in range(order[k])))
        o += order[k]
    E = [(int(edges[2 * e]), int(edges[2 * e + 1])) for e in range(t_out.value)]
    return shapes, E, [bool(copy[k]) for k in range(p_out.value)]


class Plan:
    """A planned batch (tnsk_plan): run() enqueues the whole batch on the ctx stream.
    Keeps references to the tensors and outputs whose addresses it holds."""

    def __init__(self, ctx, handle, tensors, outs, per_reps):
        self.ctx, self.h = ctx, handle
        self._keep = (tensors, outs, per_reps)

    def run(self):
        self.ctx._check(self.ctx.lib.tnsk_plan_run(self.ctx.h, self.h))

    def set_prelude(self, pairs: "Pairs | None"):
        """Run `pairs` ahead of the plan's method-2 work in every run(), beside its
        method-1 work (tnsk_plan_set_prelude); None detaches."""
        self.ctx._check(self.ctx.lib.tnsk_plan_set_prelude(self.ctx.h, self.h, pairs.h if pairs else None))
        self._prelude = pairs  # kept alive while attached

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnsk_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Stream:
    """A turnstile stream (tnsk_stream): method-1 sketches of one network kept on the
    device; update() adds deltas to tensor entries, estimate() recomputes the outputs."""

    def __init__(self, ctx, handle, tensors, out, per_rep, prec=0):
        self.ctx, self.h = ctx, handle
        self.prec = prec
        self._keep = (tensors, out, per_rep)  # the tensors until the first sketching has run

    def update(self, tensor, index, delta):
        """Device arrays [n]: tensor (int32, 0-based tensor of the network), index (int64,
        row-major flat entry index), delta (float64)."""
        import torch

        assert tensor.dtype == torch.int32 and index.dtype == torch.int64 and delta.dtype == torch.float64
        assert tensor.is_cuda and index.is_cuda and delta.is_cuda
        assert tensor.is_contiguous() and index.is_contiguous() and delta.is_contiguous()
        n = tensor.numel()
        assert index.numel() == n and delta.numel() == n
        self._upd = (tensor, index, delta)  # alive until the next update (stream order)
        self.ctx._check(self.ctx.lib.tnsk_stream_update(self.ctx.h, self.h, n, tensor.data_ptr(), index.data_ptr(),
                                                        delta.data_ptr()))

    def estimate(self):
        self.ctx._check(self.ctx.lib.tnsk_stream_estimate(self.ctx.h, self.h))

    def sketches(self):
        """tnsk_stream_sketches: a torch view (no copy) of the stored sketches, FP32 or
        FP64 by the stream's precision, to be summed across processes that stream parts
        of the same tensors before estimate(). Valid while the stream is open."""
        import torch

        x = ctypes.c_void_p()
        n = ctypes.c_int64()
        self.ctx._check(self.ctx.lib.tnsk_stream_sketches(self.h, ctypes.byref(x), ctypes.byref(n)))
        typestr = "<f8" if self.prec == PREC_FP64 else "<f4"

        class _View:  # CUDA array interface over the stream's buffer
            __cuda_array_interface__ = {"shape": (int(n.value),), "typestr": typestr,
                                        "data": (int(x.value or 0), False), "version": 3}

        return torch.as_tensor(_View(), device="cuda")

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.tnsk_stream_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


MLP_FEATURES = 9


class _PairJob(ctypes.Structure):
    _fields_ = [
        ("A", ctypes.c_void_p),
        ("B", ctypes.c_void_p),
        ("n_shared", ctypes.c_int32),
        ("a_modes", ctypes.POINTER(ctypes.c_int32)),
        ("b_modes", ctypes.POINTER(ctypes.c_int32)),
        ("out_perm", ctypes.POINTER(ctypes.c_int32)),
        ("out", ctypes.c_void_p),
    ]


def _tensor(t):
    """A one-element tnsk_tensor array for a torch device tensor (keeps its dims alive)."""
    dims = (ctypes.c_int64 * max(1, t.dim()))(*t.shape)
    arr = (_Tensor * 1)()
    arr[0].order = t.dim()
    arr[0].dims = ctypes.cast(dims, ctypes.POINTER(ctypes.c_int64))
    arr[0].data = t.data_ptr()
    arr[0].dtype = _dtype_code(t)
    arr._dims = dims
    return arr


class _PairJobs:
    """Owns the ctypes structures behind an array of tnsk_pair_job. A job is
    (A, B, a_modes, b_modes, out_perm or None, out) with torch device tensors."""

    def __init__(self, jobs):
        self.keep = []
        arr = (_PairJob * max(1, len(jobs)))()
        for i, (A, B, am, bm, perm, out) in enumerate(jobs):
            ta, tb = _tensor(A), _tensor(B)
            am_c = (ctypes.c_int32 * max(1, len(am)))(*am)
            bm_c = (ctypes.c_int32 * max(1, len(bm)))(*bm)
            pm_c = (ctypes.c_int32 * max(1, len(perm)))(*perm) if perm is not None else None
            self.keep += [ta, tb, am_c, bm_c, pm_c]
            arr[i].A = ctypes.addressof(ta[0])
            arr[i].B = ctypes.addressof(tb[0])
            arr[i].n_shared = len(am)
            arr[i].a_modes = ctypes.cast(am_c, ctypes.POINTER(ctypes.c_int32))
            arr[i].b_modes = ctypes.cast(bm_c, ctypes.POINTER(ctypes.c_int32))
            arr[i].out_perm = ctypes.cast(pm_c, ctypes.POINTER(ctypes.c_int32)) if pm_c is not None else None
            arr[i].out = out.data_ptr()
        self.arr, self.n = arr, len(jobs)


class Pairs:
    """tnsk_pairs: exact pair contractions validated once, one launch per run()."""

    def __init__(self, ctx: "Context", jobs):
        self.ctx, self.lib = ctx, ctx.lib
        self._jobs = _PairJobs(jobs)
        h = ctypes.c_void_p()
        ctx._check(self.lib.tnsk_pairs_create(ctx.h, self._jobs.n, ctypes.addressof(self._jobs.arr),
                                              ctypes.byref(h)))
        self.h = h

    def run(self):
        self.ctx._check(self.lib.tnsk_pairs_run(self.ctx.h, self.h))

    def close(self):
        if self.h is not None:
            self.lib.tnsk_pairs_destroy(self.h)
            self.h = None


class Mlp:
    """The learned sketch-size predictor (tnsk_mlp_*); device tensors are FP32 torch
    tensors, X of shape [n, MLP_FEATURES], y of shape [n]."""

    def __init__(self, ctx: "Context", seed: int = 0):
        self.ctx, self.lib = ctx, ctx.lib
        h = ctypes.c_void_p()
        ctx._check(self.lib.tnsk_mlp_create(ctx.h, int(seed) & ((1 << 64) - 1), ctypes.byref(h)))
        self.h = h
        n = ctypes.c_int64(0)
        self.lib.tnsk_mlp_num_params(ctypes.byref(n))
        self.n_params = n.value

    def close(self):
        if self.h is not None:
            self.lib.tnsk_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get(self):
        import numpy as np

        th = np.zeros(self.n_params, dtype=np.float32)
        nm = np.zeros(2 * MLP_FEATURES, dtype=np.float32)
        st = self.lib.tnsk_mlp_get(self.h, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                   nm.ctypes.data_as(ctypes.POINTER(ctypes.c_float)))
        if st != 0:
            raise TnskError(st, "tnsk_mlp_get")
        return th, nm

    def set(self, theta, norm):
        import numpy as np

        th = np.ascontiguousarray(theta, dtype=np.float32)
        nm = np.ascontiguousarray(norm, dtype=np.float32)
        assert th.size == self.n_params and nm.size == 2 * MLP_FEATURES
        self.ctx._check(self.lib.tnsk_mlp_set(self.ctx.h, self.h, th.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                              nm.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def loss_grad(self, X, y, grad=None) -> float:
        loss = ctypes.c_double(0.0)
        self.ctx._check(self.lib.tnsk_mlp_loss_grad(self.ctx.h, self.h, X.data_ptr(), y.data_ptr(), X.shape[0],
                                                    grad.data_ptr() if grad is not None else None,
                                                    ctypes.byref(loss)))
        return loss.value

    def train(self, X, y, epochs: int, batch: int = 256, lr: float = 1e-3, seed: int = 0) -> float:
        loss = ctypes.c_double(0.0)
        self.ctx._check(self.lib.tnsk_mlp_train(self.ctx.h, self.h, X.data_ptr(), y.data_ptr(), X.shape[0],
                                                int(epochs), int(batch), float(lr), int(seed) & ((1 << 64) - 1),
                                                ctypes.byref(loss)))
        return loss.value

    def predict(self, X, y, bf16: bool = True):
        self.ctx._check(self.lib.tnsk_mlp_predict(self.ctx.h, self.h, X.data_ptr(), X.shape[0], y.data_ptr(),
                                                  1 if bf16 else 0))

    def save(self, path: str):
        st = self.lib.tnsk_mlp_save(self.h, path.encode())
        if st != 0:
            raise TnskError(st, f"tnsk_mlp_save {path}")

    def load(self, path: str):
        self.ctx._check(self.lib.tnsk_mlp_load(self.ctx.h, self.h, path.encode()))


class Context:
    """A libtnsk context bound to one device and one CUDA stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        h = ctypes.c_void_p()
        sp = None if stream is None else ctypes.c_void_p(int(stream))
        st = self.lib.tnsk_create(ctypes.byref(h), int(device), sp)
        if st != TNSK_OK:
            raise TnskError(st, "tnsk_create failed")
        self.h = h

    def _check(self, st):
        if st != TNSK_OK:
            raise TnskError(st, self.lib.tnsk_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.tnsk_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream):
        self._check(self.lib.tnsk_set_stream(self.h, ctypes.c_void_p(int(stream)) if stream else None))

    def count_sketch(self, seed: int, rep: int, tid: int, n: int, m: int, bins, signs):
        self._check(self.lib.tnsk_count_sketch(self.h, seed & ((1 << 64) - 1), rep, tid, n, m,
                                               bins.data_ptr() if n else None, signs.data_ptr() if n else None))

    def m1_sketch(self, net: Network, params: Params, x):
        """tnsk_m1_sketch: method-1 sketches of every tensor into x (device, [reps][sum_k
        O_k m]); for a network with hyperedges the WLOG 1 copy tensors' sketches follow
        the caller's tensors (``rewrite`` gives the planned network)."""
        nh = _holder(net)
        pr = _params(params)
        self._check(self.lib.tnsk_m1_sketch(self.h, ctypes.byref(nh.c), ctypes.byref(pr), x.data_ptr()))

    def estimate(self, net: Network, params: Params, out, per_rep=None):
        nh = _holder(net)
        pr = _params(params)
        self._check(self.lib.tnsk_estimate(self.h, ctypes.byref(nh.c), ctypes.byref(pr), out.data_ptr(),
                                           per_rep.data_ptr() if per_rep is not None else None))

    def estimate_batch(self, nets: Sequence[Network], params: Sequence[Params], outs, per_reps=None):
        B = len(nets)
        holders = [_holder(n) for n in nets]
        carr = (_Network * max(1, B))(*[h.c for h in holders])
        parr = (_Params * max(1, B))(*[_params(p) for p in params])
        oarr = (ctypes.c_void_p * max(1, B))(*[o.data_ptr() for o in outs])
        rarr = None
        if per_reps is not None:
            rarr = (ctypes.c_void_p * max(1, B))(*[(r.data_ptr() if r is not None else None) for r in per_reps])
        self._check(self.lib.tnsk_estimate_batch(self.h, B, carr, parr, oarr, rarr))
        return holders  # callers may keep them alive until the stream completes

    def pairs(self, jobs) -> "Pairs":
        """tnsk_pairs_create: jobs of (A, B, a_modes, b_modes, out_perm or None, out)."""
        return Pairs(self, jobs)

    def contract_pairs(self, jobs):
        """tnsk_contract_pairs: the jobs once (waits for them)."""
        j = _PairJobs(jobs)
        self._check(self.lib.tnsk_contract_pairs(self.h, j.n, ctypes.addressof(j.arr)))

    def stream(self, net: Network, params: Params, out, per_rep=None) -> "Stream":
        """tnsk_stream_create: sketch the network's tensors now (method 1), write the
        estimate to out (and per_rep), keep the sketches for turnstile updates."""
        nh = _holder(net)
        pr = _params(params)
        h = ctypes.c_void_p()
        self._check(self.lib.tnsk_stream_create(self.h, ctypes.byref(nh.c), ctypes.byref(pr), out.data_ptr(),
                                                per_rep.data_ptr() if per_rep is not None else None,
                                                ctypes.byref(h)))
        return Stream(self, h, list(net.tensors), out, per_rep, params.prec)

    def autotune(self, nets: Sequence[Network], params: Sequence[Params], trials: int = 3):
        """tnsk_autotune: (Schedule, default scatter ms, tuned scatter ms) for the batch."""
        B = len(nets)
        holders = [_holder(n) for n in nets]
        carr = (_Network * max(1, B))(*[h.c for h in holders])
        parr = (_Params * max(1, B))(*[_params(p) for p in params])
        sched = Schedule()
        d, t = ctypes.c_double(0.0), ctypes.c_double(0.0)
        self._check(self.lib.tnsk_autotune(self.h, B, carr, parr, trials, ctypes.byref(sched), ctypes.byref(d),
                                           ctypes.byref(t)))
        return sched, d.value, t.value

    def plan(self, nets: Sequence[Network], params: Sequence[Params], outs, per_reps=None,
             schedule: "Schedule | None" = None) -> "Plan":
        """tnsk_plan_create (tnsk_plan_create_scheduled with a schedule): plan a batch
        once; run it with Plan.run()."""
        B = len(nets)
        holders = [_holder(n) for n in nets]
        carr = (_Network * max(1, B))(*[h.c for h in holders])
        parr = (_Params * max(1, B))(*[_params(p) for p in params])
        oarr = (ctypes.c_void_p * max(1, B))(*[o.data_ptr() for o in outs])
        rarr = None
        if per_reps is not None:
            rarr = (ctypes.c_void_p * max(1, B))(*[(r.data_ptr() if r is not None else None) for r in per_reps])
        h = ctypes.c_void_p()
        if schedule is None:
            self._check(self.lib.tnsk_plan_create(self.h, B, carr, parr, oarr, rarr, ctypes.byref(h)))
        else:
            self._check(self.lib.tnsk_plan_create_scheduled(self.h, B, carr, parr, oarr, rarr, ctypes.byref(schedule),
                                                            ctypes.byref(h)))
        return Plan(self, h, [n.tensors for n in nets], list(outs), per_reps)

    def profile(self, enable: bool = True):
        self._check(self.lib.tnsk_profile(self.h, 1 if enable else 0))

    def debug_inject(self, what: int = 1):
        """Tests only: the next launch sequence's TMA-fed tensor-core products issue no
        loads, so their bounded waits run out (tnsk_sync then reports TNSK_ERR_TIMEOUT)."""
        self._check(self.lib.tnsk_debug_inject(self.h, int(what)))

    def profile_read(self):
        """{kernel kind: (total ms, launches)} since the last read (waits for the stream)."""
        ms = (ctypes.c_double * len(KERNEL_KINDS))()
        n = (ctypes.c_int64 * len(KERNEL_KINDS))()
        self._check(self.lib.tnsk_profile_read(self.h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KERNEL_KINDS)}

    def combine(self, per_rep, groups: int, out):
        """tnsk_combine: out[o] = median of `groups` group means of per_rep[:, o] (FP64,
        device tensors; per_rep is [R][O] contiguous, out holds O entries)."""
        assert per_rep.is_cuda and out.is_cuda and per_rep.is_contiguous() and out.is_contiguous()
        R = per_rep.shape[0]
        O = per_rep.numel() // max(R, 1)
        self._check(self.lib.tnsk_combine(self.h, R, O, per_rep.data_ptr(), groups, out.data_ptr()))

    def features(self, net: Network, params: Params):
        """tnsk_features: the predictor's inputs for a network at params.m, params.reps."""
        import numpy as np

        nh = _holder(net)
        pr = _params(params)
        f = (ctypes.c_float * MLP_FEATURES)()
        self._check(self.lib.tnsk_features(self.h, ctypes.byref(nh.c), ctypes.byref(pr), f))
        return np.array(f[:], dtype=np.float32)

    def choose_params(self, net: Network, target_err: float, params: Params, mlp=None):
        """tnsk_choose_params: (params with the chosen m, predicted error), or (None,
        the best candidate's predicted error) when no m <= 2^16 meets the target
        (TNSK_ERR_UNREACHABLE); other errors raise."""
        import dataclasses

        nh = _holder(net)
        pr = _params(params)
        err = ctypes.c_double(0.0)
        st = self.lib.tnsk_choose_params(self.h, ctypes.byref(nh.c), float(target_err),
                                         mlp.h if mlp is not None else None, ctypes.byref(pr), ctypes.byref(err))
        if st == ERR_UNREACHABLE:
            return None, err.value
        self._check(st)
        return dataclasses.replace(params, m=int(pr.m)), err.value

    def choose_params_batch(self, nets: Sequence[Network], target_err: float, params: Sequence[Params], mlp=None,
                            pilot_reps: int = 16, rate: bool = False):
        """tnsk_choose_params_batch (tnsk_choose_params_rate with rate=True): ([params with
        m and reps chosen], [predicted error], [how: 0 predictor, 1 pilot, 2 flagged: not
        sized to the target])."""
        import dataclasses

        fn = self.lib.tnsk_choose_params_rate if rate else self.lib.tnsk_choose_params_batch
        B = len(nets)
        holders = [_holder(n) for n in nets]
        carr = (_Network * max(1, B))(*[h.c for h in holders])
        parr = (_Params * max(1, B))(*[_params(p) for p in params])
        err = (ctypes.c_double * max(1, B))()
        how = (ctypes.c_int32 * max(1, B))()
        self._check(fn(self.h, B, carr, float(target_err), mlp.h if mlp is not None else None, int(pilot_reps), parr,
                       err, how))
        out = [dataclasses.replace(p, m=int(parr[i].m), reps=int(parr[i].reps), groups=int(parr[i].groups))
               for i, p in enumerate(params)]
        return out, [err[i] for i in range(B)], [how[i] for i in range(B)]

    def probe_shared_atomics(self) -> float:
        """Random-bin FP32 shared-memory atomic adds per second (a measurement aid)."""
        r = ctypes.c_double(0.0)
        self._check(self.lib.tnsk_probe_shared_atomics(self.h, ctypes.byref(r)))
        return r.value

    def probe_shared_int_adds(self) -> float:
        """Random-bin 32-bit integer shared-memory adds per second (measurement aid)."""
        v = ctypes.c_double(0.0)
        self._check(self.lib.tnsk_probe_shared_int_adds(self.h, ctypes.byref(v)))
        return v.value

    def auto_report(self):
        """(reps recomputed in FP64, largest relative rounding bound of a per-rep value)
        of the last TNSK_PREC_AUTO estimate on this context."""
        n, b = ctypes.c_int32(0), ctypes.c_double(0.0)
        self._check(self.lib.tnsk_auto_report(self.h, ctypes.byref(n), ctypes.byref(b)))
        return int(n.value), float(b.value)

    def sync(self):
        self._check(self.lib.tnsk_sync(self.h))
