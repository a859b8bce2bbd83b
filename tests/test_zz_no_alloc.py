"""The allocation-free backward (stl_robustness_backward_noalloc) against the regular one.

It exists for callers that may not allocate device memory while running; it takes no
workspace and keeps its scratch in the library's static device array.  Called through the C
ABI twice in a row (the array keeps the previous call's contents), on cases whose backward
needs scratch (smooth Until), one large enough that fewer CTAs are launched, a hard case that
needs none, and one whose single-CTA scratch exceeds the array (a clear error, no launch).
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


def rel_err(a, b):
    a = a.double().cpu().numpy().reshape(a.shape[0], -1)
    b = b.double().cpu().numpy().reshape(b.shape[0], -1)
    scale = np.maximum(np.abs(b).max(axis=1, keepdims=True), 1e-30)
    return float((np.abs(a - b) / scale).max())


def noalloc_backward(stl, f, x, g, p, bounds=None):
    from paper_2501_04194_gb300.binding import robustness_backward_noalloc_raw
    B, T, D = x.shape
    gs = torch.full((B, T, D), float("nan"), device=x.device)
    gb = None
    if bounds is not None:
        gb = torch.full_like(bounds, float("nan"))
    stream = torch.cuda.current_stream().cuda_stream
    robustness_backward_noalloc_raw(f, x.data_ptr(), B, T, None if bounds is None else bounds.data_ptr(), p,
                                    g.data_ptr(), gs.data_ptr(), None if gb is None else gb.data_ptr(), stream)
    return gs, gb


@pytest.mark.parametrize("mode,B,T", [("smooth", 8, 2000), ("smooth", 2048, 3000), ("hard", 64, 5000)])
def test_noalloc_matches_workspace_backward(stl, mode, B, T):
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params(mode, tau=10.0)
    x = torch.from_numpy(W.random_walk(B, T, 3, seed=7)).cuda()
    for call in range(2):
        g = torch.from_numpy(np.random.default_rng(call).normal(size=(B, T)).astype(np.float32)).cuda()
        ref, _ = stl.robustness_backward(f, x, g, p=p)
        got, _ = noalloc_backward(stl, f, x, g, p)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all()
        assert rel_err(got, ref) <= GRAD_TOL


def test_noalloc_bound_gradients_on_a_reduced_grid(stl):
    # a per-trace sigmoid-masked window (config-2 shape) beside a smooth Until whose per-thread
    # arrays make the scratch of all resident CTAs exceed the array: fewer CTAs walk the
    # traces, and grad_bounds (cleared by the call) must still match the workspace backward
    f = stl.Formula(W.Or(W.config2_formula(), W.Until(0, 600, W.gt([1.0], 0.0), W.lt([1.0], 0.5))), D=1)
    p = stl.params("smooth", tau=10.0, mask_c=5.0, mask_eps=1e-3)
    sig, bounds = W.config2_inputs(B=2048, T=3000, seed=3)
    x = torch.from_numpy(sig).cuda()
    bd = torch.from_numpy(bounds).cuda()
    for call in range(2):
        g = torch.from_numpy(np.random.default_rng(10 + call).normal(size=(2048, 3000)).astype(np.float32)).cuda()
        ref, ref_gb = stl.robustness_backward(f, x, g, bounds=bd, p=p)
        got, got_gb = noalloc_backward(stl, f, x, g, p, bounds=bd)
        torch.cuda.synchronize()
        assert torch.isfinite(got).all() and torch.isfinite(got_gb).all()
        assert rel_err(got, ref) <= GRAD_TOL
        assert rel_err(got_gb, ref_gb) <= GRAD_TOL


def test_noalloc_empty_batch(stl):
    # B = 0 is checked and launches nothing, whatever the formula would need for long traces
    f = stl.Formula(W.Until(0, 70000, W.gt([1.0], 0.0), W.lt([1.0], 0.5)), D=1)
    p = stl.params("smooth", tau=5.0)
    x = torch.zeros((0, 71000, 1), device="cuda")
    g = torch.zeros((0, 71000), device="cuda")
    got, _ = noalloc_backward(stl, f, x, g, p)
    assert got.shape == (0, 71000, 1)


def test_noalloc_rejects_scratch_beyond_its_array(stl):
    # twelve nested Always_[0,60000] over traces of 800,000 samples: the node buffers that spill
    # out of shared memory (value and adjoint, spans 60,000 .. 720,000 samples) need about 37 MB
    # for one CTA of any size, more than the 32 MiB array; the call is rejected before any launch
    from paper_2501_04194_gb300.binding import StlError
    f = W.gt([1.0], 0.0)
    for _ in range(12):
        f = W.Always(0, 60000, f)
    f = stl.Formula(f, D=1)
    p = stl.params("smooth", tau=5.0)
    x = torch.zeros((2, 800000, 1), device="cuda")
    g = torch.zeros((2, 800000), device="cuda")
    with pytest.raises(StlError) as ei:
        noalloc_backward(stl, f, x, g, p)
    assert ei.value.status == -4 and "static scratch" in str(ei.value)
