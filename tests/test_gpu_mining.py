"""GPU checks of the interval-mining helpers (include/stl_mining.h, mining.py).

- the loss seed and the parameter update against numpy written from their definitions;
- the vectorised interval sweep against the FP64 oracle (smooth-mask Always, Sec. VI);
- gradient descent recovering the interval of a synthetic mining dataset (Sec. VII-C example).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mining():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2501_04194_gb300 import mining as M
    assert torch.cuda.is_available()
    return M


def test_seed_and_update(mining):
    from paper_2501_04194_gb300.binding import check
    lib = mining._lib()
    st = torch.cuda.current_stream().cuda_stream
    rng = np.random.default_rng(0)
    N, T = 1000, 20
    rho = rng.normal(size=(N, T)).astype(np.float32)
    rd = torch.from_numpy(rho).cuda()
    gout = torch.full((N, T), 5.0, device="cuda")
    loss = torch.zeros(1, device="cuda")
    check(lib.stl_mining_seed(rd.data_ptr(), N, T, gout.data_ptr(), loss.data_ptr(), st))
    g = gout.cpu().numpy()
    r0 = rho[:, 0].astype(np.float64)
    assert np.array_equal(g[:, 0], np.where(r0 < 0, np.float32(-1.0 / N), 0).astype(np.float32))
    assert np.all(g[:, 1:] == 5.0)
    assert abs(float(loss.item()) - np.maximum(-r0, 0).mean()) < 1e-5
    gb = rng.normal(size=(N, 2, 2)).astype(np.float32)
    theta = torch.tensor([-0.5, 0.7], device="cuda")
    bounds = torch.zeros((N, 2, 2), device="cuda")
    lr, gamma = 0.01, 0.1
    check(lib.stl_mining_update(theta.data_ptr(), torch.from_numpy(gb).cuda().data_ptr(), N, 2, 1, T, lr, gamma,
                                bounds.data_ptr(), st))
    a, b = 1 / (1 + math.exp(0.5)), 1 / (1 + math.exp(-0.7))
    al = -0.5 - lr * (T * gb[:, 1, 0].astype(np.float64).sum() + gamma) * a * (1 - a)
    be = 0.7 - lr * (T * gb[:, 1, 1].astype(np.float64).sum() - gamma) * b * (1 - b)
    np.testing.assert_allclose(theta.cpu().numpy(), [al, be], rtol=1e-5, atol=1e-6)
    bd = bounds.cpu().numpy()
    np.testing.assert_allclose(bd[:, 1, 0], T / (1 + math.exp(-al)), rtol=1e-5)
    np.testing.assert_allclose(bd[:, 1, 1], T / (1 + math.exp(-be)), rtol=1e-5)
    assert np.all(bd[:, 0, :] == 0)


def test_interval_sweep_matches_oracle(mining):
    T = 20
    sig = W.mining_dataset(1, T=T, seed=3)[0, :, 0]
    g = np.linspace(0.02, 0.98, 17)
    a, b = np.meshgrid(g, g, indexing="ij")
    keep = a < b
    a, b = a[keep], b[keep]
    rho0, ms = mining.interval_sweep(sig, a, b, c=5.0, eps=1e-3, tau=10.0)
    K = len(a)
    bounds = np.stack([a * T, b * T], axis=1).astype(np.float32).reshape(K, 1, 2)
    x = np.broadcast_to(sig.reshape(1, T, 1), (K, T, 1)).astype(np.float32)
    ref = oracle.robustness(mining.always_interval_formula(T), x, bounds=bounds, mode=oracle.SMOOTH, tau=10.0,
                            mask_c=5.0, mask_eps=1e-3)[:, 0]
    scale = np.maximum(np.abs(ref), 1.0)
    assert np.max(np.abs(rho0 - ref) / scale) < 1e-5


def test_mine_interval_recovers_the_interval(mining):
    """5000 steps of size 1e-2 from (0.1, 0.9), c and tau annealed 1 -> 20 (the example's
    setting): the interval of the data, (0.23, 0.59) up to the edge noise, is recovered."""
    sig = W.mining_dataset(1000, T=20, seed=4)
    res = mining.mine_interval(sig, steps=5000, lr=1e-2, gamma=0.1, record_every=500)
    assert 0.2 <= res["a"] <= 0.32 and 0.52 <= res["b"] <= 0.62, res
    assert res["history"][-1][3] < res["history"][0][3]


def test_per_trace_descent_step_follows_the_oracle_gradient(mining):
    # config-2 shape at a size the oracle finishes quickly: one step of the per-trace descent moves
    # each (a_n, b_n) by -lr (N dL/dbounds + (gamma, -gamma)), with the bound gradient of the
    # loss seed -1/N [rho_n(0) < 0] taken from the FP64 oracle, then the clamps
    N, T = 64, 600
    sig, bounds = W.config2_inputs(B=N, T=T, seed=4)
    tree = W.config2_formula()
    kw = dict(mode=oracle.SMOOTH, tau=10.0, mask_c=5.0, mask_eps=1e-3)
    rho = oracle.robustness(tree, sig, bounds=bounds, **kw)
    g = np.zeros((N, T))
    g[:, 0] = np.where(rho[:, 0].astype(np.float32) < 0, -1.0 / N, 0.0)
    _, gb = oracle.robustness_grad(tree, sig, g, bounds=bounds, **kw)
    lr, gamma = 2.0, 0.01
    a = np.clip(bounds[:, 0, 0] - lr * (N * gb[:, 0, 0] + gamma), 0.0, 100.0)
    b = np.clip(bounds[:, 0, 1] - lr * (N * gb[:, 0, 1] - gamma), a + 1.0, 400.0)
    r = mining.per_trace_descent(sig, bounds, steps=1, lr=lr, gamma=gamma)
    got = r["bounds"][:, 0, :]
    sure = np.abs(rho[:, 0]) > 1e-3   # traces whose seed sign cannot differ by rounding
    assert sure.sum() > N // 2
    np.testing.assert_allclose(got[sure, 0], a[sure], rtol=1e-4, atol=1e-3)
    np.testing.assert_allclose(got[sure, 1], b[sure], rtol=1e-4, atol=1e-3)


def test_per_trace_descent_lowers_the_loss(mining):
    sig, bounds = W.config2_inputs(B=512, T=2000, seed=6)
    r = mining.per_trace_descent(sig, bounds, steps=200)
    assert r["loss"] < r["loss0"]
    bd = r["bounds"][:, 0, :]
    assert np.all(bd[:, 0] >= 0) and np.all(bd[:, 1] <= 400.0) and np.all(bd[:, 1] - bd[:, 0] >= 1.0 - 1e-4)
