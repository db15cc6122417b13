"""FP64 CPU oracle for "Approximating Tensor Network Contraction with Sketches".

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers. It shares no code with the
CUDA library (``paper_2603_07387_gb300``) and does not import it.

A network is passed as plain data: ``tensors`` (list of arrays, row-major),
``edges`` (list of (u, v) global 0-based mode ids, numbered across X_1..X_p in
order) and ``open_modes`` (the output order of the uncontracted modes).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

from .exact import frobenius_product, tc_definition, tc_einsum, tc_reduced, tc_sequential  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "tnsk_oracle.c")

ORC_OK, ORC_INVALID, ORC_CYCLIC, ORC_UNSUPPORTED = 0, -1, -2, -3


class OracleError(RuntimeError):
    def __init__(self, status):
        super().__init__(f"oracle status {status}")
        self.status = status


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, -O2, FP64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "tnsk_oracle.h"))
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


class _Net(ctypes.Structure):
    _fields_ = [
        ("p", ctypes.c_int32),
        ("order", ctypes.POINTER(ctypes.c_int32)),
        ("dims", ctypes.POINTER(ctypes.c_int64)),
        ("data", ctypes.POINTER(ctypes.POINTER(ctypes.c_double))),
        ("t", ctypes.c_int32),
        ("edges", ctypes.POINTER(ctypes.c_int32)),
        ("n_open", ctypes.c_int32),
        ("open", ctypes.POINTER(ctypes.c_int32)),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        u64, i64, i32, vp = ctypes.c_uint64, ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p
        L.orc_splitmix64.restype = u64
        L.orc_splitmix64.argtypes = [u64]
        L.orc_tid.restype = u64
        L.orc_tid.argtypes = [i32, i64, i64, i64, i64]
        L.orc_count_sketch.restype = None
        L.orc_count_sketch.argtypes = [u64, u64, u64, i64, i64, vp, vp]
        L.orc_dft.restype = None
        L.orc_dft.argtypes = [i64, vp, vp, vp, vp]
        L.orc_fft.restype = None
        L.orc_fft.argtypes = [i64, vp, vp, vp, vp]
        L.orc_m1_tables.restype = ctypes.c_int
        L.orc_m1_tables.argtypes = [ctypes.POINTER(_Net), u64, i32, i64, vp, vp]
        L.orc_m1_sketch.restype = ctypes.c_int
        L.orc_m1_sketch.argtypes = [ctypes.POINTER(_Net), i64, i32, vp, vp, i32, vp]
        L.orc_m1_estimate.restype = ctypes.c_int
        L.orc_m1_estimate.argtypes = [ctypes.POINTER(_Net), i64, i32, vp, vp, vp, vp]
        L.orc_m2_estimate.restype = ctypes.c_int
        L.orc_m2_estimate.argtypes = [ctypes.POINTER(_Net), i32, i64, i32, u64, vp, vp, vp, vp]
        L.orc_combine.restype = ctypes.c_int
        L.orc_combine.argtypes = [i32, i64, vp, i32, vp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


class _NetHolder:
    """Keeps the numpy buffers behind an _Net alive."""

    def __init__(self, tensors, edges, open_modes):
        # np.array(order="C") keeps 0-d scalars 0-d (ascontiguousarray would make them 1-d)
        self.tensors = [np.array(x, dtype=np.float64, order="C", copy=True) for x in tensors]
        self.order = np.array([x.ndim for x in self.tensors], dtype=np.int32)
        self.dims = np.array([d for x in self.tensors for d in x.shape] or [0], dtype=np.int64)
        self.edges = np.array([m for e in edges for m in e] or [0], dtype=np.int32)
        self.open = np.array(list(open_modes) or [0], dtype=np.int32)
        P = ctypes.POINTER(ctypes.c_double)
        self.ptrs = (P * max(1, len(self.tensors)))(
            *[x.ctypes.data_as(P) if x.size else ctypes.cast(ctypes.c_void_p(8), P) for x in self.tensors]
        )
        self.net = _Net(
            len(self.tensors),
            self.order.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            self.dims.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
            self.ptrs,
            len(edges),
            self.edges.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
            len(open_modes),
            self.open.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
        )
        self.t = len(edges)
        self.edge_dims = [int(self.dims[u]) for u, _ in edges]
        self.L = int(sum(self.edge_dims))
        self.O = int(np.prod([int(self.dims[g]) for g in open_modes])) if len(open_modes) else 1
        off = np.concatenate([[0], np.cumsum(self.order)]).astype(int)
        self.mode_off = off
        contracted = set(m for e in edges for m in e)
        self.open_tot = []
        for k, x in enumerate(self.tensors):
            o = 1
            for g in range(off[k], off[k + 1]):
                if g not in contracted:
                    o *= int(self.dims[g])
            self.open_tot.append(o)


def _check(st):
    if st != ORC_OK:
        raise OracleError(st)


def splitmix64(state: int) -> int:
    return int(lib().orc_splitmix64(state & ((1 << 64) - 1)))


def tid(kind: int, a: int = 0, b: int = 0, c: int = 0, d: int = 0) -> int:
    return int(lib().orc_tid(kind, a, b, c, d))


def count_sketch(seed: int, rep: int, table_id: int, n: int, m: int):
    """(bins, signs) of the count sketch h, s on [n] -> [m] of the hash contract."""
    bins = np.zeros(max(n, 1), dtype=np.int64)
    signs = np.zeros(max(n, 1), dtype=np.int8)
    lib().orc_count_sketch(seed, rep, table_id, n, m, _ptr(bins), _ptr(signs))
    return bins[:n], signs[:n]


def dft(x):
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(re)
    lib().orc_dft(len(x), _ptr(re), _ptr(im), _ptr(ore), _ptr(oim))
    return ore + 1j * oim


def fft(x):
    x = np.asarray(x, dtype=np.complex128)
    re, im = np.ascontiguousarray(x.real), np.ascontiguousarray(x.imag)
    ore, oim = np.zeros_like(re), np.zeros_like(re)
    lib().orc_fft(len(x), _ptr(re), _ptr(im), _ptr(ore), _ptr(oim))
    return ore + 1j * oim


def m1_tables(tensors, edges, open_modes, seed: int, reps: int, m: int):
    h = _NetHolder(tensors, edges, open_modes)
    bins = np.zeros((reps, max(h.L, 1)), dtype=np.int64)
    signs = np.zeros((reps, max(h.L, 1)), dtype=np.int8)
    _check(lib().orc_m1_tables(ctypes.byref(h.net), seed, reps, m, _ptr(bins), _ptr(signs)))
    return bins[:, : h.L].copy(), signs[:, : h.L].copy()


def m1_sketch(tensors, edges, open_modes, m: int, bins, signs, abs_mode: bool = False):
    """Per-tensor method-1 sketches x_k (Eq. 1 hash form), shape [R, sum_k O_k*m]."""
    h = _NetHolder(tensors, edges, open_modes)
    bins = np.ascontiguousarray(bins, dtype=np.int64).reshape(-1, h.L) if h.L else np.zeros((len(bins), 1), np.int64)
    signs = np.ascontiguousarray(signs, dtype=np.int8).reshape(-1, h.L) if h.L else np.zeros((len(bins), 1), np.int8)
    R = bins.shape[0]
    X = m * sum(h.open_tot)
    x = np.zeros((R, max(X, 1)), dtype=np.float64)
    _check(lib().orc_m1_sketch(ctypes.byref(h.net), m, R, _ptr(bins), _ptr(signs), int(abs_mode), _ptr(x)))
    return x[:, :X]


def m1_estimate(tensors, edges, open_modes, m: int, reps: int | None = None, seed: int | None = None,
                bins=None, signs=None):
    """Per-rep method-1 estimates y[R, O] and scales s[R, O] (Alg. 1 / Eq. 1).

    Tables come from the hash contract (``seed``) unless ``bins``/``signs`` are
    given ([R, L] arrays, L = sum of edge dims)."""
    h = _NetHolder(tensors, edges, open_modes)
    if bins is None:
        bins, signs = m1_tables(tensors, edges, open_modes, seed, reps, m)
    bins = np.ascontiguousarray(bins, dtype=np.int64)
    signs = np.ascontiguousarray(signs, dtype=np.int8)
    R = bins.shape[0]
    if h.L == 0:
        bins = np.zeros((R, 1), np.int64)
        signs = np.zeros((R, 1), np.int8)
    y = np.zeros((R, max(h.O, 1)), dtype=np.float64)
    s = np.zeros((R, max(h.O, 1)), dtype=np.float64)
    _check(lib().orc_m1_estimate(ctypes.byref(h.net), m, R, _ptr(bins), _ptr(signs), _ptr(y), _ptr(s)))
    return y[:, : h.O], s[:, : h.O]


def m2_estimate(tensors, edges, m: int, reps: int, seed: int, root: int = 0, edge_bins=None, edge_signs=None):
    """Per-rep method-2 estimates y[R] and scales s[R] (Alg. 2, 4, 5)."""
    h = _NetHolder(tensors, edges, [])
    y = np.zeros(max(reps, 1), dtype=np.float64)
    s = np.zeros(max(reps, 1), dtype=np.float64)
    eb = es = None
    if edge_bins is not None:
        eb = np.ascontiguousarray(edge_bins, dtype=np.int64).reshape(reps, h.L)
        es = np.ascontiguousarray(edge_signs, dtype=np.int8).reshape(reps, h.L)
    _check(lib().orc_m2_estimate(ctypes.byref(h.net), root, m, reps, seed, _ptr(eb), _ptr(es), _ptr(y), _ptr(s)))
    return y[:reps], s[:reps]


def combine(per_rep, groups: int = 1):
    """Median of ``groups`` contiguous group means (groups = 1: the mean)."""
    a = np.ascontiguousarray(np.asarray(per_rep, dtype=np.float64))
    if a.ndim == 1:
        a = a[:, None]
    R, O = a.shape
    out = np.zeros(max(O, 1), dtype=np.float64)
    _check(lib().orc_combine(R, O, _ptr(a), groups, _ptr(out)))
    return out[:O]
