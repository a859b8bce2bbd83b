"""ctypes binding of libstl (include/stl.h): argument marshalling only.

Every step of the robustness path runs in the CUDA library; this module converts a formula
given as nested tuples (the format documented in ``Formula``) into the C ABI's node array,
passes device pointers and the current CUDA stream, and raises on any non-zero status.  There
is no CPU fallback: if ``libstl.so`` is missing or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import math
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libstl.so")

STL_HARD, STL_SMOOTH, STL_SOFTMAX = 0, 1, 2
OPS = {"pred>": 0, "pred<": 1, "true": 2, "not": 3, "and": 4, "or": 5, "eventually": 6, "always": 7,
       "until": 8, "eventually_sm": 9, "always_sm": 10, "norm>": 11, "norm<": 12, "until_sm": 13}
STATUS = {0: "ok", -1: "invalid argument", -2: "unsupported", -3: "CUDA error", -4: "workspace too small",
          -5: "device wait timed out", -6: "device-side data check failed"}

EXPORTED = ["stl_compile", "stl_destroy", "stl_set_launch", "stl_get_launch", "stl_workspace_size",
            "stl_robustness", "stl_robustness_backward", "stl_get_device_status", "stl_status_string",
            "stl_last_error", "stl_version"]


class StlNode(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int32), ("child0", ctypes.c_int32), ("child1", ctypes.c_int32),
                ("bound_slot", ctypes.c_int32), ("a", ctypes.c_float), ("b", ctypes.c_float),
                ("pad_mode", ctypes.c_int32), ("pad_value", ctypes.c_float),
                ("pred_offset", ctypes.c_int32), ("pred_c", ctypes.c_float)]


KERNEL_AUTO, KERNEL_INTERPRETER, KERNEL_COMPILED = 0, 1, 2
KERNELS = {"auto": KERNEL_AUTO, "interpreter": KERNEL_INTERPRETER, "compiled": KERNEL_COMPILED}
KERNEL_NAMES = {v: k for k, v in KERNELS.items()}


class StlParams(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tau", ctypes.c_float), ("mask_c", ctypes.c_float),
                ("mask_eps", ctypes.c_float)]


class StlLaunch(ctypes.Structure):
    _fields_ = [("tile", ctypes.c_int32), ("threads", ctypes.c_int32), ("segment", ctypes.c_int32),
                ("kernel", ctypes.c_int32)]


class StlError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"libstl: {STATUS.get(status, status)}: {message}")
        self.status = status


_lib = None


def load(path: str = LIB_PATH):
    """Load libstl.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} not found: build it with `python -m paper_2501_04194_gb300.build` "
                          "(or __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.stl_compile.argtypes = [ctypes.POINTER(StlNode), i32, vp, i32, i32, i32, ctypes.POINTER(vp)]
    lib.stl_destroy.argtypes = [vp]
    lib.stl_destroy.restype = None
    lib.stl_set_launch.argtypes = [vp, ctypes.POINTER(StlLaunch)]
    lib.stl_get_launch.argtypes = [vp, i64, i64, ctypes.POINTER(StlParams), i32, ctypes.POINTER(StlLaunch)]
    lib.stl_workspace_size.argtypes = [vp, i64, i64, ctypes.POINTER(StlParams), i32, ctypes.POINTER(sz)]
    lib.stl_robustness.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), vp, vp, sz, vp]
    lib.stl_robustness_backward.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), vp, vp, vp, vp,
                                            sz, vp]
    lib.stl_robustness_and_backward.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), vp, vp, vp,
                                                vp, vp, sz, vp]
    lib.stl_get_device_status.argtypes = [vp, ctypes.POINTER(i32)]
    lib.stl_status_string.argtypes = [i32]
    lib.stl_status_string.restype = ctypes.c_char_p
    lib.stl_last_error.restype = ctypes.c_char_p
    lib.stl_version.restype = ctypes.c_char_p
    for name in ("stl_compile", "stl_set_launch", "stl_get_launch", "stl_workspace_size", "stl_robustness",
                 "stl_robustness_backward", "stl_robustness_and_backward", "stl_get_device_status"):
        getattr(lib, name).restype = ctypes.c_int32
    _lib = lib
    return lib


def check(status: int):
    if status != 0:
        raise StlError(status, load().stl_last_error().decode())


def flatten(tree, D):
    """Nested-tuple formula -> (list of StlNode children-first with the root last, weights, n_slots).

    Tuple format (Sec. III-B grammar plus the derived and smoothed operators):
      ("pred", ">" | "<", weights[D], c), ("norm", ">" | "<", scales[D], centre[D], r),
      ("true",), ("not", f), ("and", f, g), ("or", f, g),
      ("eventually" | "always" | "eventually_sm" | "always_sm", I, f), ("until", I, f, g)
    with I = (a, b, slot, pad): b may be inf; slot None or a bounds column; pad None (repeat the
    last sample) or a constant."""
    nodes, weights = [], []
    n_slots = 0

    def add(f):
        nonlocal n_slots
        op = f[0]
        nd = StlNode(op=0, child0=-1, child1=-1, bound_slot=-1, a=0.0, b=0.0, pad_mode=0, pad_value=0.0,
                     pred_offset=0, pred_c=0.0)
        if op == "pred":
            _, rel, w, c = f
            if len(w) != D:
                raise ValueError(f"predicate has {len(w)} weights, signal has D={D}")
            nd.op = OPS["pred>" if rel == ">" else "pred<"]
            nd.pred_offset = len(weights)
            weights.extend(float(v) for v in w)
            nd.pred_c = float(c)
        elif op == "norm":
            _, rel, scale, centre, r = f
            if len(scale) != D or len(centre) != D:
                raise ValueError(f"norm predicate needs {D} scales and {D} centre coordinates")
            nd.op = OPS["norm>" if rel == ">" else "norm<"]
            nd.pred_offset = len(weights)
            weights.extend(float(v) for v in scale)
            weights.extend(float(v) for v in centre)
            nd.pred_c = float(r)
        elif op == "true":
            nd.op = OPS["true"]
        elif op == "not":
            nd.child0 = add(f[1])
            nd.op = OPS["not"]
        elif op in ("and", "or"):
            nd.child0 = add(f[1])
            nd.child1 = add(f[2])
            nd.op = OPS[op]
        elif op in ("eventually", "always", "until", "eventually_sm", "always_sm", "until_sm"):
            a, b, slot, pad = f[1]
            nd.child0 = add(f[2])
            if op in ("until", "until_sm"):
                nd.child1 = add(f[3])
            nd.op = OPS[op]
            nd.a = float(a)
            nd.b = math.inf if math.isinf(b) else float(b)
            if slot is not None:
                nd.bound_slot = int(slot)
                n_slots = max(n_slots, int(slot) + 1)
            if pad is not None:
                nd.pad_mode, nd.pad_value = 1, float(pad)
        else:
            raise ValueError(f"unknown operator {op!r}")
        nodes.append(nd)
        return len(nodes) - 1

    add(tree)
    return nodes, weights, n_slots


def params(mode=STL_HARD, tau=1.0, mask_c=5.0, mask_eps=1e-3) -> StlParams:
    if isinstance(mode, str):
        mode = {"hard": STL_HARD, "smooth": STL_SMOOTH, "softmax": STL_SOFTMAX}[mode]
    return StlParams(int(mode), float(tau), float(mask_c), float(mask_eps))


class Formula:
    """A compiled formula (host handle of the C library)."""

    def __init__(self, tree, D: int, n_slots: int | None = None):
        lib = load()
        nodes, weights, ns = flatten(tree, D)
        self.tree, self.D = tree, D
        self.n_slots = ns if n_slots is None else int(n_slots)
        arr = (StlNode * len(nodes))(*nodes)
        w = (ctypes.c_float * max(1, len(weights)))(*weights)
        h = ctypes.c_void_p()
        check(lib.stl_compile(arr, len(nodes), ctypes.cast(w, ctypes.c_void_p), len(weights), D, self.n_slots,
                              ctypes.byref(h)))
        self._h = h
        self.n_nodes = len(nodes)

    @property
    def handle(self):
        return self._h

    def set_launch(self, tile=0, threads=0, segment=0, kernel=KERNEL_AUTO):
        """stl_set_launch; kernel: "auto", "interpreter" or "compiled" (or the stl_kernel value)."""
        k = KERNELS[kernel] if isinstance(kernel, str) else int(kernel)
        check(load().stl_set_launch(self._h, ctypes.byref(StlLaunch(tile, threads, segment, k))))

    def get_launch(self, B, T, p: StlParams, backward=False):
        out = StlLaunch()
        check(load().stl_get_launch(self._h, B, T, ctypes.byref(p), int(backward), ctypes.byref(out)))
        return dict(tile=out.tile, threads=out.threads, segment=out.segment, kernel=KERNEL_NAMES.get(out.kernel))

    def compile_kernel(self, backward=False, T=1 << 20, threads=0, tile=0):
        """stl_compile_kernel: generate and compile this formula's kernel for one direction
        (NVRTC; no GPU needed).  Returns (tile, dynamic shared memory bytes)."""
        lib = load()
        fn = lib.stl_compile_kernel
        if fn.argtypes is None:
            fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.POINTER(StlLaunch),
                           ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
            fn.restype = ctypes.c_int32
        t, sm = ctypes.c_int32(), ctypes.c_int32()
        check(fn(self._h, int(backward), int(T), ctypes.byref(StlLaunch(tile, threads, 0, KERNEL_COMPILED)),
                 ctypes.byref(t), ctypes.byref(sm)))
        return int(t.value), int(sm.value)

    def autotune(self, sig_ptr, B, T, bounds_ptr, p: StlParams, backward, grad_out_ptr, out_ptr, gb_ptr, ws_ptr,
                 ws_bytes, stream):
        """stl_autotune: time candidate launch shapes, keep the best for this direction.
        Returns (launch dict, mean ms of the winner or -1 if it came from STL_TUNE_CACHE)."""
        lib = load()
        fn = lib.stl_autotune
        if fn.argtypes is None:
            vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
            fn.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), i32, vp, vp, vp, vp, sz, vp,
                           ctypes.POINTER(StlLaunch), ctypes.POINTER(ctypes.c_float)]
            fn.restype = i32
        best, ms = StlLaunch(), ctypes.c_float()
        check(fn(self._h, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), int(backward), grad_out_ptr, out_ptr, gb_ptr,
                 ws_ptr, ws_bytes, stream, ctypes.byref(best), ctypes.byref(ms)))
        return (dict(tile=best.tile, threads=best.threads, segment=best.segment,
                     kernel=KERNEL_NAMES.get(best.kernel)), float(ms.value))

    def workspace_size(self, B, T, p: StlParams, backward=False) -> int:
        n = ctypes.c_size_t()
        check(load().stl_workspace_size(self._h, B, T, ctypes.byref(p), int(backward), ctypes.byref(n)))
        return int(n.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.stl_destroy(h)
            self._h = None


def _pipeline_setup(lib):
    if getattr(lib, "_pipe_ready", False):
        return
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    lib.stl_pipeline_staging_size.argtypes = [vp, i64, i64, ctypes.POINTER(StlParams), i32, ctypes.POINTER(sz)]
    lib.stl_pipeline_staging_size.restype = i32
    lib.stl_robustness_host_pipelined.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), vp, vp, vp, vp,
                                                  i64, vp, sz, vp]
    lib.stl_robustness_host_pipelined.restype = i32
    lib._pipe_ready = True


def pipeline_staging_size(f: Formula, chunk, T, p: StlParams, backward) -> int:
    lib = load()
    _pipeline_setup(lib)
    n = ctypes.c_size_t()
    check(lib.stl_pipeline_staging_size(f.handle, chunk, T, ctypes.byref(p), int(backward), ctypes.byref(n)))
    return int(n.value)


def robustness_host_pipelined_raw(f: Formula, sig_ptr, B, T, bounds_ptr, p: StlParams, gout_ptr, out_ptr, gsig_ptr,
                                  gb_ptr, chunk, staging_ptr, staging_bytes, stream):
    lib = load()
    _pipeline_setup(lib)
    check(lib.stl_robustness_host_pipelined(f.handle, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), gout_ptr, out_ptr,
                                            gsig_ptr, gb_ptr, chunk, staging_ptr, staging_bytes, stream))


def robustness_raw(f: Formula, sig_ptr, B, T, bounds_ptr, p: StlParams, out_ptr, ws_ptr, ws_bytes, stream):
    check(load().stl_robustness(f.handle, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), out_ptr, ws_ptr, ws_bytes,
                                stream))


def robustness_backward_raw(f: Formula, sig_ptr, B, T, bounds_ptr, p: StlParams, gout_ptr, gsig_ptr, gb_ptr,
                            ws_ptr, ws_bytes, stream):
    check(load().stl_robustness_backward(f.handle, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), gout_ptr,
                                         gsig_ptr, gb_ptr, ws_ptr, ws_bytes, stream))


def robustness_and_backward_raw(f: Formula, sig_ptr, B, T, bounds_ptr, p: StlParams, gout_ptr, out_ptr, gsig_ptr,
                                gb_ptr, ws_ptr, ws_bytes, stream):
    check(load().stl_robustness_and_backward(f.handle, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), gout_ptr,
                                             out_ptr, gsig_ptr, gb_ptr, ws_ptr, ws_bytes, stream))


def robustness_backward_noalloc_raw(f: Formula, sig_ptr, B, T, bounds_ptr, p: StlParams, gout_ptr, gsig_ptr,
                                    gb_ptr, stream):
    """stl_robustness_backward_noalloc: the backward without a caller-provided workspace (its
    scratch is the library's static device array; see include/stl.h)."""
    lib = load()
    fn = lib.stl_robustness_backward_noalloc
    if fn.argtypes is None:
        vp, i64 = ctypes.c_void_p, ctypes.c_int64
        fn.argtypes = [vp, vp, i64, i64, vp, ctypes.POINTER(StlParams), vp, vp, vp, vp]
        fn.restype = ctypes.c_int32
    check(fn(f.handle, sig_ptr, B, T, bounds_ptr, ctypes.byref(p), gout_ptr, gsig_ptr, gb_ptr, stream))


class FormulaSet:
    """Formulas of the same D evaluated together by the ragged launch (stl_set_* in stl.h)."""

    def __init__(self, formulas):
        lib = load()
        self._setup(lib)
        self.formulas = list(formulas)   # keep the handles alive
        arr = (ctypes.c_void_p * len(self.formulas))(*[f.handle.value for f in self.formulas])
        h = ctypes.c_void_p()
        check(lib.stl_set_create(arr, len(self.formulas), ctypes.byref(h)))
        self._h = h
        self.D = self.formulas[0].D
        self.n_slots = max(f.n_slots for f in self.formulas)

    @staticmethod
    def _setup(lib):
        if getattr(lib, "_set_ready", False):
            return
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
        lib.stl_set_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)]
        lib.stl_set_create.restype = i32
        lib.stl_set_destroy.argtypes = [vp]
        lib.stl_set_destroy.restype = None
        lib.stl_set_prepare.argtypes = [vp, i64, i64, ctypes.POINTER(StlParams), i32, ctypes.POINTER(sz)]
        lib.stl_set_prepare.restype = i32
        lib.stl_robustness_ragged.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, ctypes.POINTER(StlParams), vp, vp,
                                              sz, vp]
        lib.stl_robustness_ragged.restype = i32
        lib.stl_robustness_ragged_backward.argtypes = [vp, vp, vp, vp, vp, i64, vp, i32, ctypes.POINTER(StlParams),
                                                       vp, vp, vp, vp, sz, vp]
        lib.stl_robustness_ragged_backward.restype = i32
        lib.stl_set_autotune.argtypes = [vp, i64, i64, ctypes.POINTER(StlParams), i32, vp, vp, vp, vp, vp, i32, vp, vp,
                                         vp, vp, ctypes.POINTER(StlLaunch), ctypes.POINTER(ctypes.c_float),
                                         ctypes.POINTER(sz)]
        lib.stl_set_autotune.restype = i32
        lib.stl_set_set_launch.argtypes = [vp, i32, ctypes.POINTER(StlLaunch)]
        lib.stl_set_set_launch.restype = i32
        lib._set_ready = True

    @property
    def handle(self):
        return self._h

    def prepare(self, n_traces, T_max, p: StlParams, backward=False) -> int:
        n = ctypes.c_size_t()
        check(load().stl_set_prepare(self._h, n_traces, T_max, ctypes.byref(p), int(backward), ctypes.byref(n)))
        return int(n.value)

    def set_launch(self, backward, tile=0, threads=0):
        """stl_set_set_launch: fix the launch shape of one direction (zeros: the planner's)."""
        check(load().stl_set_set_launch(self._h, int(backward), ctypes.byref(StlLaunch(tile, threads, 0, 0))))

    def autotune(self, n_traces, T_max, p: StlParams, backward, sig_ptr, off_ptr, fid_ptr, order_ptr, bounds_ptr,
                 gout_ptr, out_ptr, gb_ptr, stream):
        """stl_set_autotune: time the candidate launch shapes on this batch, keep the fastest and
        leave the set prepared with it.  Returns (workspace bytes, (threads, tile), best ms)."""
        best = StlLaunch()
        ms = ctypes.c_float()
        n = ctypes.c_size_t()
        check(load().stl_set_autotune(self._h, n_traces, T_max, ctypes.byref(p), int(backward), sig_ptr, off_ptr,
                                      fid_ptr, order_ptr, bounds_ptr, self.n_slots, gout_ptr, out_ptr, gb_ptr, stream,
                                      ctypes.byref(best), ctypes.byref(ms), ctypes.byref(n)))
        return int(n.value), (int(best.threads), int(best.tile)), float(ms.value)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.stl_set_destroy(h)
            self._h = None


def robustness_ragged_raw(s: FormulaSet, sig_ptr, off_ptr, fid_ptr, order_ptr, n, bounds_ptr, p, out_ptr, ws_ptr,
                          ws_bytes, stream):
    check(load().stl_robustness_ragged(s.handle, sig_ptr, off_ptr, fid_ptr, order_ptr, n, bounds_ptr, s.n_slots,
                                       ctypes.byref(p), out_ptr, ws_ptr, ws_bytes, stream))


def robustness_ragged_backward_raw(s: FormulaSet, sig_ptr, off_ptr, fid_ptr, order_ptr, n, bounds_ptr, p, gout_ptr,
                                   gsig_ptr, gb_ptr, ws_ptr, ws_bytes, stream):
    check(load().stl_robustness_ragged_backward(s.handle, sig_ptr, off_ptr, fid_ptr, order_ptr, n, bounds_ptr,
                                                s.n_slots, ctypes.byref(p), gout_ptr, gsig_ptr, gb_ptr, ws_ptr,
                                                ws_bytes, stream))


def device_status(stream=None) -> int:
    st = ctypes.c_int32()
    check(load().stl_get_device_status(stream, ctypes.byref(st)))
    return int(st.value)


# ---------------------------------------------------------------- planning helpers (stl_plan.h)
def plan_lib():
    """libstl with the argument types of the stl_plan.h entry points set."""
    lib = load()
    if getattr(lib, "_plan_ready", False):
        return lib
    vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
    sigs = {
        "stl_rollout": [vp, i64, i32, f32, vp, vp],
        "stl_plan_adam_step": [vp, vp, vp, vp, vp, i64, i32, f32, f32, f32, f32, f32, i32, vp, vp],
        "stl_plan_check": [vp, vp, vp, i32, vp, i64, i32, vp, vp],
        "stl_gemm_bf16": [vp, i32, i32, vp, i32, i32, i32, i32, i32, vp, i32, vp, vp, i32, vp],
        "stl_mse_grad": [vp, vp, i64, f32, vp, vp, vp],
        "stl_relu_backward": [vp, vp, i64, vp, vp],
        "stl_colsum_bf16": [vp, i32, i32, vp, vp],
        "stl_adam": [vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp, vp],
        "stl_to_bf16": [vp, i64, vp, vp],
        "stl_gather_rows": [vp, i64, vp, i64, i32, vp, vp],
        "stl_trajopt_seed": [vp, vp, i64, i32, vp, vp],
        "stl_trajopt_step": [vp, vp, vp, vp, vp, vp, vp, vp, vp, i64, i32, i32, i32, f32, f32, f32, f32, f32, f32,
                             f32, i32, vp, vp, vp],
    }
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = i32
    lib._plan_ready = True
    return lib


def plan_call(name, *args):
    """Call one stl_plan.h entry point (pointers as ints or None) and raise on a bad status."""
    check(getattr(plan_lib(), name)(*args))
