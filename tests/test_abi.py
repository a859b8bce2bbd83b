"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every entry point
declared in include/*.h, and rejects malformed formulas and arguments with the documented
status before anything is launched."""
import ctypes
import math
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lib():
    from paper_2501_04194_gb300 import build as b
    b.build()
    from paper_2501_04194_gb300 import binding
    return binding, binding.load()


def declared_functions():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"^\s*(?:STL_API\s+)?(?:stl_status|void|const char \*)\s*\*?\s*(stl_\w+)\s*\(",
                                text, flags=re.M))
    return sorted(names)


def test_header_declares_the_abi():
    names = declared_functions()
    for required in ("stl_compile", "stl_robustness", "stl_robustness_backward", "stl_destroy",
                     "stl_workspace_size", "stl_status_string", "stl_rollout", "stl_plan_adam_step",
                     "stl_gemm_bf16"):
        assert required in names


def test_library_exports_every_declared_symbol():
    binding, lib = _lib()
    out = subprocess.run(["nm", "-D", "--defined-only", binding.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    for name in declared_functions():
        assert name in exported, name
        assert getattr(lib, name) is not None
    # nothing else of the C ABI namespace leaks
    assert not any(e.startswith("_Z") and "stl" in e and "KProgram" in e for e in exported)


def test_status_strings_and_version():
    _, lib = _lib()
    assert lib.stl_status_string(0) == b"ok"
    assert lib.stl_status_string(-1) == b"invalid argument"
    assert b"sm_103a" in lib.stl_version()


def _compile(binding, nodes, weights, D=1, n_slots=0):
    arr = (binding.StlNode * len(nodes))(*nodes)
    w = (ctypes.c_float * max(1, len(weights)))(*weights)
    h = ctypes.c_void_p()
    rc = binding.load().stl_compile(arr, len(nodes), ctypes.cast(w, ctypes.c_void_p), len(weights), D, n_slots,
                                    ctypes.byref(h))
    if rc == 0:
        binding.load().stl_destroy(h)
    return rc, binding.load().stl_last_error().decode()


def N(binding, op, c0=-1, c1=-1, slot=-1, a=0.0, b=0.0, pad=0, padv=0.0, off=0, c=0.0):
    return binding.StlNode(op, c0, c1, slot, a, b, pad, padv, off, c)


def test_compile_accepts_and_rejects():
    binding, _ = _lib()
    ok = [N(binding, 0), N(binding, 6, c0=0, a=1, b=3)]
    assert _compile(binding, ok, [1.0])[0] == 0
    cases = {
        "bad op": [N(binding, 0), N(binding, 42, c0=0)],
        "child after parent": [N(binding, 6, c0=1, a=0, b=1), N(binding, 0)],
        "two parents": [N(binding, 0), N(binding, 3, c0=0), N(binding, 4, c0=0, c1=1)],
        "a > b": [N(binding, 0), N(binding, 6, c0=0, a=5, b=2)],
        "non-integer window": [N(binding, 0), N(binding, 6, c0=0, a=0.5, b=2)],
        "weights out of range": [N(binding, 0, off=3)],
        "unused child set": [N(binding, 0), N(binding, 3, c0=0, c1=0)],
        "slot out of range": [N(binding, 0), N(binding, 6, c0=0, a=0, b=4, slot=2)],
        "infinite smooth mask": [N(binding, 0), N(binding, 9, c0=0, a=0, b=math.inf)],
        "bad pad mode": [N(binding, 0), N(binding, 6, c0=0, a=0, b=1, pad=7)],
        "orphan": [N(binding, 0), N(binding, 0, off=0), N(binding, 3, c0=1)],
    }
    for name, nodes in cases.items():
        rc, msg = _compile(binding, nodes, [1.0])
        assert rc == -1, name
        assert msg, name


def test_flatten_orders_children_first():
    from paper_2501_04194_gb300 import binding
    import workloads as W
    nodes, w, ns = binding.flatten(W.config1_formula(), 3)
    assert len(nodes) == 7 and ns == 0 and len(w) == 9
    for i, nd in enumerate(nodes):
        assert nd.child0 < i and nd.child1 < i
    assert nodes[-1].op == binding.OPS["or"]


def test_null_arguments_are_rejected_before_any_launch():
    binding, lib = _lib()
    from paper_2501_04194_gb300.binding import Formula
    import workloads as W
    f = Formula(W.config0_formula(), D=2)
    p = binding.params("hard")
    rc = lib.stl_robustness(f.handle, None, 4, 10, None, ctypes.byref(p), None, None, 0, None)
    assert rc == -1
    rc = lib.stl_robustness(f.handle, ctypes.c_void_p(16), 4, 0, None, ctypes.byref(p), ctypes.c_void_p(16), None, 0,
                            None)
    assert rc == -1
    bad = binding.params("smooth", tau=-1.0)
    rc = lib.stl_robustness(f.handle, ctypes.c_void_p(16), 4, 10, None, ctypes.byref(bad), ctypes.c_void_p(16), None,
                            0, None)
    assert rc == -1 and b"tau" in lib.stl_last_error()
    # B == 0 is a no-op
    assert lib.stl_robustness(f.handle, None, 0, 10, None, ctypes.byref(p), None, None, 0, None) == 0
    # the one-launch robustness and gradient needs rho, grad_out and grad_sig
    v = ctypes.c_void_p(16)
    rc = lib.stl_robustness_and_backward(f.handle, v, 4, 10, None, ctypes.byref(p), v, None, v, None, None, 0, None)
    assert rc == -1 and b"out" in lib.stl_last_error()
    rc = lib.stl_robustness_and_backward(f.handle, v, 4, 10, None, ctypes.byref(p), None, v, v, None, None, 0, None)
    assert rc == -1 and b"grad_out" in lib.stl_last_error()
    assert lib.stl_robustness_and_backward(f.handle, None, 0, 10, None, ctypes.byref(p), None, None, None, None, None,
                                           0, None) == 0
