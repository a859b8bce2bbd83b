"""TEST INFRASTRUCTURE ONLY: Python access to the FP64 CPU oracle (``stl_oracle.c``).

The oracle computes STL robustness traces and their analytic (sub)gradients from the
plain definitions of the paper (Sec. III-B Eq. "quantitative", Sec. IV-B/IV-C, Sec. VI
Eq. "smooth mask").  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline /
reference legs of ``bench.py`` may import this package.  It shares no code with the CUDA
library: it parses the formula tuples of ``workloads`` with its own code below and
compiles its own C file with gcc.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# node encoding private to the oracle (mirrors the enum in stl_oracle.c)
_OPS = {"pred>": 0, "pred<": 1, "true": 2, "not": 3, "and": 4, "or": 5, "eventually": 6,
        "always": 7, "until": 8, "eventually_sm": 9, "always_sm": 10, "norm>": 11, "norm<": 12,
        "until_sm": 13}
HARD, SMOOTH, SOFTMAX = 0, 1, 2


class _ONode(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("c0", ctypes.c_int32), ("c1", ctypes.c_int32),
                ("slot", ctypes.c_int32), ("a", ctypes.c_double), ("b", ctypes.c_double),
                ("pad_mode", ctypes.c_int32), ("w_off", ctypes.c_int32),
                ("pad_value", ctypes.c_double), ("c", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile ``stl_oracle.c`` into ``liboracle.so`` (plain C, -O2, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                                   "-fno-fast-math", "-o", tmp, _SRC, "-lm", "-lpthread"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        common = [ctypes.POINTER(_ONode), ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int]
        lib.oracle_forward.argtypes = common + [ctypes.c_void_p, ctypes.c_int]
        lib.oracle_forward.restype = ctypes.c_int
        lib.oracle_backward.argtypes = common + [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]
        lib.oracle_backward.restype = ctypes.c_int
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def num_threads() -> int:
    return int(_load().oracle_num_threads())


class _Flat:
    """Post-order (children before parents) flattening of a formula tuple tree."""

    def __init__(self, tree, D):
        self.D = D
        self.nodes = []
        self.weights = []
        self.n_slots = 0
        self.root = self._add(tree)
        arr = (_ONode * len(self.nodes))()
        for i, n in enumerate(self.nodes):
            arr[i] = n
        self.arr = arr
        self.w = np.asarray(self.weights if self.weights else [0.0], dtype=np.float64)

    def _add(self, f):
        op = f[0]
        nd = _ONode()
        nd.c0 = nd.c1 = nd.slot = -1
        nd.pad_mode, nd.pad_value = 0, 0.0
        if op == "pred":
            _, rel, w, c = f
            if len(w) != self.D:
                raise ValueError("predicate weight length != D")
            nd.op = _OPS["pred>" if rel == ">" else "pred<"]
            nd.w_off = len(self.weights)
            self.weights.extend(float(np.float32(v)) for v in w)
            nd.c = float(np.float32(c))
        elif op == "norm":
            _, rel, scale, centre, r = f
            if len(scale) != self.D or len(centre) != self.D:
                raise ValueError("norm predicate scale/centre length != D")
            nd.op = _OPS["norm>" if rel == ">" else "norm<"]
            nd.w_off = len(self.weights)
            self.weights.extend(float(np.float32(v)) for v in scale)
            self.weights.extend(float(np.float32(v)) for v in centre)
            nd.c = float(np.float32(r))
        elif op == "true":
            nd.op = _OPS["true"]
        elif op == "not":
            nd.c0 = self._add(f[1])
            nd.op = _OPS["not"]
        elif op in ("and", "or"):
            nd.c0 = self._add(f[1])
            nd.c1 = self._add(f[2])
            nd.op = _OPS[op]
        elif op in ("eventually", "always", "until", "eventually_sm", "always_sm", "until_sm"):
            a, b, slot, pad = f[1]
            nd.c0 = self._add(f[2])
            if op in ("until", "until_sm"):
                nd.c1 = self._add(f[3])
            nd.op = _OPS[op]
            nd.a, nd.b = float(a), float(b)
            if slot is not None:
                nd.slot = int(slot)
                self.n_slots = max(self.n_slots, slot + 1)
            if pad is not None:
                nd.pad_mode, nd.pad_value = 1, float(pad)
        else:
            raise ValueError(f"unknown operator {op!r}")
        self.nodes.append(nd)
        return len(self.nodes) - 1


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _prep(tree, sig, offsets, bounds):
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    if offsets is None:
        if sig.ndim != 3:
            raise ValueError("dense signal must be [B,T,D]")
        B, T, D = sig.shape
        offsets = np.arange(B + 1, dtype=np.int64) * T
        flat = sig.reshape(B * T, D)
    else:
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        flat = sig
        B, D = len(offsets) - 1, sig.shape[1]
    fl = _Flat(tree, D)
    n_slots = fl.n_slots
    if bounds is not None:
        bounds = np.ascontiguousarray(bounds, dtype=np.float64)
        n_slots = bounds.shape[1]
    elif n_slots:
        raise ValueError("formula uses per-trace bounds but none were given")
    return fl, flat, offsets, B, D, bounds, n_slots


def robustness(tree, sig, bounds=None, mode=HARD, tau=1.0, mask_c=5.0, mask_eps=1e-3,
               exact=False, offsets=None, n_threads=0):
    """Robustness trace of ``tree``: float64 ``[B,T]`` (dense) or ``[sum T]`` (ragged).

    ``sig`` is widened to float64; with ``exact=False`` predicates round every operation to
    float32 (bit-compatible with float32 arithmetic on float32 inputs), with ``exact=True``
    they run in float64 (for finite differences)."""
    fl, flat, offsets, B, D, bounds, n_slots = _prep(tree, sig, offsets, bounds)
    out = np.zeros(int(offsets[-1]), dtype=np.float64)
    rc = _load().oracle_forward(fl.arr, len(fl.nodes), fl.root, _ptr(fl.w), D, _ptr(flat), _ptr(offsets),
                                B, _ptr(bounds), n_slots, int(mode), float(tau), float(mask_c),
                                float(mask_eps), int(exact), _ptr(out), int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_forward failed")
    return out.reshape(sig.shape[0], sig.shape[1]) if sig.ndim == 3 else out


def robustness_grad(tree, sig, grad_out, bounds=None, mode=HARD, tau=1.0, mask_c=5.0, mask_eps=1e-3,
                    exact=False, offsets=None, n_threads=0):
    """Gradient of sum(grad_out * rho) w.r.t. the signal (float64, shaped like ``sig``) and
    the per-trace bounds (float64 ``[B, n_slots, 2]`` or None)."""
    fl, flat, offsets, B, D, bounds, n_slots = _prep(tree, sig, offsets, bounds)
    gout = np.ascontiguousarray(np.asarray(grad_out, dtype=np.float64).reshape(-1))
    gsig = np.zeros((int(offsets[-1]), D), dtype=np.float64)
    gb = np.zeros((B, n_slots, 2), dtype=np.float64) if n_slots else None
    rc = _load().oracle_backward(fl.arr, len(fl.nodes), fl.root, _ptr(fl.w), D, _ptr(flat), _ptr(offsets),
                                 B, _ptr(bounds), n_slots, int(mode), float(tau), float(mask_c),
                                 float(mask_eps), int(exact), _ptr(gout), _ptr(gsig), _ptr(gb),
                                 int(n_threads))
    if rc != 0:
        raise RuntimeError("oracle_backward failed")
    if sig.ndim == 3:
        gsig = gsig.reshape(sig.shape)
    return gsig, gb


def robustness_ragged_multi(formulas, formula_id, sig, offsets, bounds=None, **kw):
    """Ragged batch where trace i follows ``formulas[formula_id[i]]``; packed float64 output."""
    offsets = np.asarray(offsets, dtype=np.int64)
    out = np.zeros(int(offsets[-1]), dtype=np.float64)
    formula_id = np.asarray(formula_id)
    for k, f in enumerate(formulas):
        idx = np.nonzero(formula_id == k)[0]
        if len(idx) == 0:
            continue
        sub_off = np.zeros(len(idx) + 1, dtype=np.int64)
        sub_off[1:] = np.cumsum(offsets[idx + 1] - offsets[idx])
        sub_sig = np.concatenate([sig[offsets[i]:offsets[i + 1]] for i in idx])
        sub_b = None if bounds is None else bounds[idx]
        r = robustness(f, sub_sig, bounds=sub_b, offsets=sub_off, **kw)
        for j, i in enumerate(idx):
            out[offsets[i]:offsets[i + 1]] = r[sub_off[j]:sub_off[j + 1]]
    return out


def robustness_grad_ragged_multi(formulas, formula_id, sig, offsets, grad_out, bounds=None, **kw):
    """Ragged gradient where trace i follows ``formulas[formula_id[i]]``: packed float64 signal
    gradient [sum T, D] and bounds gradient [n, n_slots, 2] (or None)."""
    offsets = np.asarray(offsets, dtype=np.int64)
    formula_id = np.asarray(formula_id)
    gout = np.asarray(grad_out, dtype=np.float64)
    gsig = np.zeros((int(offsets[-1]), sig.shape[1]), dtype=np.float64)
    gb = None if bounds is None else np.zeros((len(formula_id), bounds.shape[1], 2), dtype=np.float64)
    for k, f in enumerate(formulas):
        idx = np.nonzero(formula_id == k)[0]
        if len(idx) == 0:
            continue
        sub_off = np.zeros(len(idx) + 1, dtype=np.int64)
        sub_off[1:] = np.cumsum(offsets[idx + 1] - offsets[idx])
        sub_sig = np.concatenate([sig[offsets[i]:offsets[i + 1]] for i in idx])
        sub_g = np.concatenate([gout[offsets[i]:offsets[i + 1]] for i in idx])
        sub_b = None if bounds is None else bounds[idx]
        g, b = robustness_grad(f, sub_sig, sub_g, bounds=sub_b, offsets=sub_off, **kw)
        for j, i in enumerate(idx):
            gsig[offsets[i]:offsets[i + 1]] = g[sub_off[j]:sub_off[j + 1]]
            if gb is not None and b is not None:
                gb[i] = b[j]
    return gsig, gb


__all__ = ["robustness_grad_ragged_multi", "build", "robustness", "robustness_grad", "robustness_ragged_multi", "num_threads",
           "HARD", "SMOOTH", "SOFTMAX", "math"]
