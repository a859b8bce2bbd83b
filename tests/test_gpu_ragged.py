"""Ragged batches in one persistent launch: uneven trace lengths, 16 seed-generated formulas
of depth <= 4 with per-trace bounds (the config-3 shape at a size the oracle finishes in
seconds), checked trace by trace against the FP64 oracle; the processing order does not change
the result; a CUDA-graph replay reproduces the eager result; bad per-trace data is rejected on
the device without a fault."""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

VAL_TOL, GRAD_TOL = 1e-5, 1e-4


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    return m


def per_trace_err(got, ref, offsets):
    worst = 0.0
    for i in range(len(offsets) - 1):
        g = np.asarray(got[offsets[i]:offsets[i + 1]], dtype=np.float64)
        r = np.asarray(ref[offsets[i]:offsets[i + 1]], dtype=np.float64)
        fin = np.isfinite(r)
        assert np.array_equal(fin, np.isfinite(g))
        scale = max(np.abs(r[fin]).max() if fin.any() else 0.0, 1e-30)
        worst = max(worst, float((np.abs(g[fin] - r[fin]) / scale).max()) if fin.any() else 0.0)
    return worst


def make_batch(stl, wl, mode, order=None):
    fs = [stl.Formula(f, D=4, n_slots=wl["n_slots"]) for f in wl["formulas"]]
    fset = stl.FormulaSet(fs)
    p = stl.params(mode, tau=3.0)
    rb = stl.RaggedBatch(fset, torch.from_numpy(wl["signal"]), torch.from_numpy(wl["offsets"]),
                         torch.from_numpy(wl["formula_id"]), bounds=torch.from_numpy(wl["bounds"]), p=p,
                         order=None if order is None else torch.from_numpy(order))
    return rb, fs, fset


@pytest.mark.parametrize("mode", ["hard", "smooth"])
def test_ragged_matches_oracle(stl, mode):
    wl = W.config3_workload(n_traces=40, t_lo=50, t_hi=2000, seed=3)
    rb, _, _ = make_batch(stl, wl, mode)
    rng = np.random.default_rng(0)
    gout = rng.normal(size=int(wl["offsets"][-1])).astype(np.float32)
    rho = rb.forward().cpu().numpy()
    gs, gb = rb.backward(torch.from_numpy(gout).cuda())
    gs = gs.cpu().numpy()
    torch.cuda.synchronize()
    from paper_2501_04194_gb300.binding import device_status
    assert device_status() == 0
    om = oracle.HARD if mode == "hard" else oracle.SMOOTH
    kw = dict(mode=om, tau=3.0)
    ref = oracle.robustness_ragged_multi(wl["formulas"], wl["formula_id"], wl["signal"], wl["offsets"],
                                         bounds=wl["bounds"], **kw)
    if mode == "hard":
        np.testing.assert_array_equal(rho, ref.astype(np.float32))
    else:
        assert per_trace_err(rho, ref, wl["offsets"]) <= VAL_TOL
    gref, _ = oracle.robustness_grad_ragged_multi(wl["formulas"], wl["formula_id"], wl["signal"], wl["offsets"],
                                                  gout.astype(np.float64), bounds=wl["bounds"], **kw)
    assert per_trace_err(gs.reshape(-1, 4), gref, wl["offsets"]) <= GRAD_TOL


def test_ragged_order_and_graph_replay(stl):
    wl = W.config3_workload(n_traces=64, t_lo=50, t_hi=3000, seed=5)
    lengths = np.diff(wl["offsets"])
    order = np.argsort(-lengths, kind="stable").astype(np.int32)
    rb0, _, _ = make_batch(stl, wl, "hard")
    rb1, _, _ = make_batch(stl, wl, "hard", order=order)
    g = torch.randn(int(wl["offsets"][-1]), device="cuda")
    a = rb0.forward().clone()
    ga, _ = rb0.backward(g)
    ga = ga.clone()
    b = rb1.forward().clone()
    gb, _ = rb1.backward(g)
    assert torch.equal(a, b)
    assert torch.equal(ga, gb)   # hard-mode gradients are fixed-point sums: order-independent
    graph = rb1.capture(g)
    rb1.out.zero_()
    rb1.gsig.zero_()
    for _ in range(2):
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(rb1.out, a)
        assert torch.equal(rb1.gsig, ga)


def test_ragged_bad_formula_id_is_rejected_on_device(stl):
    from paper_2501_04194_gb300.binding import device_status
    wl = W.config3_workload(n_traces=8, t_lo=50, t_hi=400, seed=7)
    wl["formula_id"] = wl["formula_id"].copy()
    wl["formula_id"][3] = 99
    rb, _, _ = make_batch(stl, wl, "hard")
    device_status()
    rb.forward()
    torch.cuda.synchronize()
    assert device_status() == -6
    assert device_status() == 0


def test_autotune_keeps_parity_and_uses_the_cache(stl, tmp_path, monkeypatch):
    """The autotuner picks a launch shape that still matches the oracle, and a second tuning
    with STL_TUNE_CACHE set is served from the cache file."""
    monkeypatch.setenv("STL_TUNE_CACHE", str(tmp_path / "tune.txt"))
    tree = W.config1_formula()
    sig = W.config1_inputs(B=12, T=4000, seed=11)
    x = torch.from_numpy(sig).cuda()
    for bwd in (False, True):
        f = stl.Formula(tree, D=3)
        p = stl.params("hard")
        launch, ms = stl.autotune(f, x, p=p, backward=bwd)
        assert launch["threads"] in (256, 512) and launch["tile"] >= 256 and ms > 0
        rho = stl.robustness(f, x, p=p).cpu().numpy()
        np.testing.assert_array_equal(rho, oracle.robustness(tree, sig).astype(np.float32))
        g = np.random.default_rng(1).normal(size=(12, 4000)).astype(np.float32)
        gs, _ = stl.robustness_backward(f, x, torch.from_numpy(g).cuda(), p=p)
        gref, _ = oracle.robustness_grad(tree, sig, g.astype(np.float64))
        err = np.abs(gs.cpu().numpy() - gref).max() / np.abs(gref).max()
        assert err <= GRAD_TOL
        f2 = stl.Formula(tree, D=3)
        launch2, ms2 = stl.autotune(f2, x, p=p, backward=bwd)
        assert launch2 == launch and ms2 == -1.0


@pytest.mark.parametrize("mode", ["hard", "smooth"])
def test_ragged_autotuned_set_matches_the_default_plan(stl, mode):
    # stl_set_autotune picks a launch shape per direction; the results are those of the default
    # plan (hard: bit for bit, values and fixed-point gradients; smooth: within tolerance)
    # (smooth: shorter traces, the FP64 oracle's literal smooth-Until adjoint is O(b^2) per sample)
    wl = W.config3_workload(n_traces=48, t_lo=50, t_hi=6000 if mode == "hard" else 1500, seed=9)
    lengths = np.diff(wl["offsets"])
    order = np.argsort(-lengths, kind="stable").astype(np.int32)
    rb0, fs, _ = make_batch(stl, wl, mode, order=order)
    p = stl.params(mode, tau=3.0)
    rb1 = stl.RaggedBatch(stl.FormulaSet(fs), torch.from_numpy(wl["signal"]), torch.from_numpy(wl["offsets"]),
                          torch.from_numpy(wl["formula_id"]), bounds=torch.from_numpy(wl["bounds"]), p=p,
                          order=torch.from_numpy(order), tune=True)
    assert rb1.shapes["forward"]["threads"] in (64, 256, 512) and rb1.shapes["backward"]["tile"] >= 256
    g = torch.from_numpy(np.random.default_rng(2).normal(size=int(wl["offsets"][-1])).astype(np.float32)).cuda()
    a = rb0.forward().clone()
    ga = rb0.backward(g)[0].clone()
    b = rb1.forward().clone()
    gb = rb1.backward(g)[0].clone()
    if mode == "hard":
        assert torch.equal(a, b) and torch.equal(ga, gb)
    else:
        # float sums in another order: both launch shapes against the FP64 oracle
        offs = wl["offsets"]
        kw = dict(mode=oracle.SMOOTH, tau=3.0, bounds=wl["bounds"])
        ref = oracle.robustness_ragged_multi(wl["formulas"], wl["formula_id"], wl["signal"], offs, **kw)
        gref, _ = oracle.robustness_grad_ragged_multi(wl["formulas"], wl["formula_id"], wl["signal"], offs,
                                                      g.cpu().numpy().astype(np.float64), **kw)
        for rho, gs in ((a, ga), (b, gb)):
            assert per_trace_err(rho.cpu().numpy(), ref, offs) <= VAL_TOL
            assert per_trace_err(gs.cpu().numpy().reshape(-1, 4), gref, offs) <= GRAD_TOL
