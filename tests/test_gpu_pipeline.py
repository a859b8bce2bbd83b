"""The host-buffer pipeline (stl_robustness_host_pipelined) against the device-buffer calls:
chunks on two streams, a batch that is not a multiple of the chunk, per-trace bounds with
their gradients, hard and smooth modes."""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("mode", ["hard", "smooth", "softmax"])
def test_host_pipeline_matches_device_calls(stl, mode):
    B, T = 37, 1500
    tree, D = W.config1_formula(), 3
    f = stl.Formula(tree, D=D)
    p = stl.params(mode, tau=10.0)
    x = W.random_walk(B, T, D, seed=3)
    g = np.random.default_rng(4).normal(size=(B, T)).astype(np.float32)
    xd, gd = torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()
    rho_ref = stl.robustness(f, xd, p=p).cpu()
    gs_ref, _ = stl.robustness_backward(f, xd, gd, p=p)
    pipe = stl.HostPipeline(f, T, p, chunk=8, backward=True)
    hx, hg = torch.from_numpy(x).pin_memory(), torch.from_numpy(g).pin_memory()
    out = torch.full((B, T), float("nan")).pin_memory()
    gs = torch.full((B, T, D), float("nan")).pin_memory()
    pipe(hx, grad_out=hg, out=out, grad_sig=gs)
    torch.cuda.synchronize()
    if mode == "hard":
        assert torch.equal(out, rho_ref)
    else:
        assert float((out - rho_ref).abs().max() / rho_ref.abs().max()) < 1e-6
    gs_ref = gs_ref.cpu()
    if mode == "hard":
        assert torch.equal(gs, gs_ref)   # chunks change the launch shape, not the hard gradient
    else:
        assert float((gs - gs_ref).abs().max() / gs_ref.abs().max()) < 1e-5


def test_host_pipeline_bounds_and_forward_only(stl):
    sig, bounds = W.config2_inputs(B=21, T=700, seed=5)
    f = stl.Formula(W.config2_formula(), D=1, n_slots=1)
    p = stl.params("smooth", tau=10.0)
    xd, bd = torch.from_numpy(sig).cuda(), torch.from_numpy(bounds).cuda()
    g = torch.from_numpy(np.random.default_rng(6).normal(size=(21, 700)).astype(np.float32))
    rho_ref = stl.robustness(f, xd, bd, p).cpu()
    gs_ref, gb_ref = stl.robustness_backward(f, xd, g.cuda(), bd, p)
    pipe = stl.HostPipeline(f, 700, p, chunk=4, backward=True)
    hx, hb, hg = (torch.from_numpy(sig).pin_memory(), torch.from_numpy(bounds).pin_memory(), g.pin_memory())
    out = torch.zeros((21, 700)).pin_memory()
    gs = torch.zeros((21, 700, 1)).pin_memory()
    gb = torch.zeros((21, 1, 2)).pin_memory()
    pipe(hx, grad_out=hg, bounds=hb, out=out, grad_sig=gs, grad_bounds=gb)
    torch.cuda.synchronize()
    assert float((out - rho_ref).abs().max()) < 1e-5
    assert float((gs - gs_ref.cpu()).abs().max() / gs_ref.abs().max()) < 1e-5
    assert float((gb - gb_ref.cpu()).abs().max() / gb_ref.abs().max()) < 1e-5
    fwd_only = stl.HostPipeline(f, 700, p, chunk=16, backward=False)
    out2 = torch.zeros((21, 700)).pin_memory()
    fwd_only(hx, bounds=hb, out=out2)
    torch.cuda.synchronize()
    assert torch.equal(out2, out)
