"""GPU parity of the one-launch robustness and gradient (stl_robustness_and_backward): rho
against the forward launch and the FP64 oracle, the gradients against the oracle, including
traces split into segments (the backward's warm-up samples must not write rho) and
per-trace masked bounds."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

VAL_TOL = 1e-5
GRAD_TOL = 1e-4


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


def per_trace_err(got, ref):
    B = ref.shape[0]
    g = np.asarray(got, dtype=np.float64).reshape(B, -1)
    r = np.asarray(ref, dtype=np.float64).reshape(B, -1)
    scale = np.maximum(np.abs(r).max(axis=1, keepdims=True), 1e-30)
    return (np.abs(g - r) / scale).max()


@pytest.mark.parametrize("launch", [None, dict(tile=256, segment=700), dict(tile=512, threads=256, segment=1100),
                                    dict(tile=448, threads=64)])
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 10.0), ("softmax", 10.0)])
def test_fused_matches_separate_calls_and_oracle(stl, launch, mode, tau):
    sig = W.config1_inputs(B=5, T=3001, seed=4)
    tree = W.config1_formula()
    gout = np.random.default_rng(2).normal(size=(5, 3001)).astype(np.float32)
    f = stl.Formula(tree, D=3)
    if launch:
        f.set_launch(**launch)
    p = stl.params(mode, tau=tau)
    x = torch.from_numpy(sig).cuda()
    g = torch.from_numpy(gout).cuda()
    rho_sep = stl.robustness(f, x, p=p).cpu().numpy()
    gs_sep, _ = stl.robustness_backward(f, x, g, p=p)
    rho, gs, gb = stl.robustness_and_grad(f, x, g, p=p)
    torch.cuda.synchronize()
    rho, gs, gs_sep = rho.cpu().numpy(), gs.cpu().numpy(), gs_sep.cpu().numpy()
    assert gb is None
    om = {"hard": oracle.HARD, "smooth": oracle.SMOOTH, "softmax": oracle.SOFTMAX}[mode]
    ref = oracle.robustness(tree, sig, mode=om, tau=tau)
    gref, _ = oracle.robustness_grad(tree, sig, gout.astype(np.float64), mode=om, tau=tau)
    if mode == "hard":
        np.testing.assert_array_equal(rho, rho_sep)
        np.testing.assert_array_equal(rho, ref.astype(np.float32))
    else:
        assert per_trace_err(rho, ref) <= VAL_TOL
        assert per_trace_err(rho, rho_sep) <= VAL_TOL
    assert per_trace_err(gs, gref) <= GRAD_TOL
    assert per_trace_err(gs, gs_sep) <= GRAD_TOL


@pytest.mark.parametrize("mode", ["hard", "smooth"])
def test_fused_masked_bounds(stl, mode):
    sig, bounds = W.config2_inputs(B=16, T=2000, seed=0)
    tree = W.config2_formula()
    gout = np.random.default_rng(3).normal(size=(16, 2000)).astype(np.float32)
    f = stl.Formula(tree, D=1, n_slots=1)
    p = stl.params(mode, tau=10.0, mask_c=5.0, mask_eps=1e-3)
    x = torch.from_numpy(sig).cuda()
    bt = torch.from_numpy(bounds).cuda()
    g = torch.from_numpy(gout).cuda()
    rho, gs, gb = stl.robustness_and_grad(f, x, g, bounds=bt, p=p)
    torch.cuda.synchronize()
    om = oracle.HARD if mode == "hard" else oracle.SMOOTH
    ref = oracle.robustness(tree, sig, bounds=bounds, mode=om, tau=10.0, mask_c=5.0, mask_eps=1e-3)
    gref, gbref = oracle.robustness_grad(tree, sig, gout.astype(np.float64), bounds=bounds, mode=om, tau=10.0,
                                         mask_c=5.0, mask_eps=1e-3)
    if mode == "hard":
        np.testing.assert_array_equal(rho.cpu().numpy(), ref.astype(np.float32))
        assert np.all(gb.cpu().numpy() == 0)
    else:
        assert per_trace_err(rho.cpu().numpy(), ref) <= VAL_TOL
        assert per_trace_err(gb.cpu().numpy(), gbref) <= GRAD_TOL
    assert per_trace_err(gs.cpu().numpy(), gref) <= GRAD_TOL
