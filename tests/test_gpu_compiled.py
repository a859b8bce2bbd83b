"""GPU parity of the formula-compiled kernels (STL_KERNEL_COMPILED) through the C ABI.

Each case runs the compiled kernel and checks it against the FP64 oracle with the bars of the
other parity tests (hard robustness bit-exact, gradients within 1e-4 of the per-trace scale)
and against the interpreter: robustness and gradient must be bit-identical (both paths use the
same float32 predicate arithmetic, combines, tie rules and 64-bit fixed-point deposits).
Shapes span several tiles with ragged tails, both CTA sizes, segments (backward warm-up),
windows past the end of the trace with both pads, ties, and the full-size headline launch.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W
from test_gpu_parity import per_trace_err, GRAD_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


def both(stl, tree, sig, launch, seed=0, fused=False):
    """rho and gradient from the compiled kernel (with `launch`) and from the interpreter."""
    B, T, D = sig.shape
    x = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    g = torch.from_numpy(np.random.default_rng(seed).normal(size=(B, T)).astype(np.float32)).cuda()
    p = stl.params("hard")
    out = {}
    for kind in ("compiled", "interpreter"):
        f = stl.Formula(tree, D=D)
        if kind == "compiled":
            f.set_launch(kernel="compiled", **launch)
            assert f.get_launch(B, T, p, False)["kernel"] == "compiled"
        else:
            f.set_launch(kernel="interpreter")
        rho = stl.robustness(f, x, p=p)
        gs, _ = stl.robustness_backward(f, x, g, p=p)
        res = [rho.cpu().numpy(), gs.cpu().numpy()]
        if fused:
            r2, g2, _ = stl.robustness_and_grad(f, x, g, p=p)
            res += [r2.cpu().numpy(), g2.cpu().numpy()]
        out[kind] = res
    torch.cuda.synchronize()
    return out, g.cpu().numpy().astype(np.float64)


def check(stl, tree, sig, launch=None, seed=0, fused=False, oracle_traces=None):
    out, gout = both(stl, tree, sig, launch or {}, seed, fused)
    rc, gc = out["compiled"][:2]
    ri, gi = out["interpreter"][:2]
    np.testing.assert_array_equal(rc, ri)
    np.testing.assert_array_equal(gc, gi)
    if fused:
        np.testing.assert_array_equal(out["compiled"][2], rc)
        np.testing.assert_array_equal(out["compiled"][3], gc)
    idx = list(range(sig.shape[0])) if oracle_traces is None else oracle_traces
    sub = sig[idx]
    ref = oracle.robustness(tree, sub)
    np.testing.assert_array_equal(rc[idx], ref.astype(np.float32))
    gref, _ = oracle.robustness_grad(tree, sub, gout[idx])
    assert per_trace_err(gc[idx], gref) <= GRAD_TOL


# ------------------------------------------------------------------ configs
def test_config0(stl):
    check(stl, W.config0_formula(), W.config0_inputs(), fused=True)


@pytest.mark.parametrize("launch", [{}, dict(tile=1024), dict(threads=256, tile=2048), dict(tile=512, segment=900),
                                    dict(threads=256, tile=768, segment=1700)])
@pytest.mark.parametrize("T", [1000, 3001])
def test_config1_tiles_and_segments(stl, launch, T):
    check(stl, W.config1_formula(), W.config1_inputs(B=5, T=T, seed=4), launch=launch, seed=1, fused=True)


def test_config1_long_traces(stl):
    check(stl, W.config1_formula(), W.config1_inputs(B=3, T=20000, seed=6), seed=2)


TABLE3 = W.table3_formulas(D=2, I=(2, 37))


@pytest.mark.parametrize("k", range(3, 6))
def test_table3_formulas(stl, k):
    check(stl, TABLE3[k], W.random_walk(3, 1100, 2, seed=10 + k), launch=dict(tile=512))


@pytest.mark.parametrize("k", range(3))
def test_table3_unbounded_intervals_stay_with_the_interpreter(stl, k):
    """phi_1..phi_3 use [0, inf) (b = T - 1): outside the compiled kernels; the automatic choice
    runs them in the interpreter, a forced compiled launch is refused."""
    x = torch.from_numpy(W.random_walk(2, 600, 2, seed=k)).cuda().repeat(1024, 1, 1)
    p = stl.params("hard")
    f = stl.Formula(TABLE3[k], D=2)
    assert f.get_launch(x.shape[0], 600, p, False)["kernel"] == "interpreter"
    f.set_launch(kernel="compiled")
    with pytest.raises(stl.StlError):
        stl.robustness(f, x, p=p)


# ------------------------------------------------------------------ ends of traces, pads, degenerate shapes
EDGE = [
    ("T2", W.Until(0, 3, W.gt([1, 0], 0.0), W.lt([0, 1], 0.2)), 2, 2),
    ("window_longer_than_trace", W.Always(3, 90, W.gt([1], 0.1)), 1, 17),
    ("const_pad", W.Eventually(2, 40, W.gt([1, 0], 0.0), pad=-0.25), 2, 33),
    ("const_pad_until", W.Until(1, 30, W.gt([1, 0], 0.0), W.lt([0, 1], 0.3), pad=0.1), 2, 45),
    ("true_until", W.Until(2, 9, W.true(), W.gt([1], 0.0)), 1, 50),
    ("a_eq_b", W.And(W.Eventually(4, 4, W.gt([1, 0], 0.0)), W.Until(3, 3, W.gt([1, 0], 0.1), W.gt([0, 1], 0.0))), 2, 64),
    ("not_chain", W.Not(W.Or(W.Not(W.gt([1], 0.0)), W.Always(1, 5, W.Not(W.lt([1], 0.2))))), 1, 77),
    ("predicate_root", W.gt([1, -1], 0.1), 2, 600),
    ("nested_pads", W.Always(0, 50, W.Or(W.Eventually(10, 30, W.gt([1, 0], 0.2), pad=0.0),
                                         W.Not(W.Until(0, 20, W.gt([0, 1], -0.1), W.lt([1, 0], 0.0))))), 2, 700),
    ("pad_chain_const_under_last", W.Eventually(0, 40, W.Always(0, 25, W.And(W.gt([1, 0], 0.0), W.lt([0, 1], 0.4)),
                                                                pad=0.3)), 2, 260),
    ("windows_past_end", W.And(W.Eventually(500, 900, W.gt([1, 0], 0.0), pad=-0.5),
                               W.Always(3, 12, W.lt([0, 1], 1.0))), 2, 700),
    ("T1", W.Or(W.Always(0, 40, W.gt([1, 0], 0.0)), W.Until(0, 9, W.gt([0, 1], 0.1), W.lt([1, 1], 0.0))), 2, 1),
    ("true_root", W.true(), 1, 90),
    ("not_true_or", W.Or(W.Not(W.true()), W.Eventually(0, 30, W.gt([1], 0.2))), 1, 120),
    ("D7", W.Until(2, 50, W.gt([1, -1, 0, 0.5, 0, 0, 2], 0.1), W.lt([0, 0, 1, 1, 1, -1, 0], 0.3)), 7, 400),
]


@pytest.mark.parametrize("name,tree,D,T", EDGE, ids=[e[0] for e in EDGE])
@pytest.mark.parametrize("launch", [dict(tile=512), dict(threads=256, tile=512, segment=300)])
def test_degenerate(stl, name, tree, D, T, launch):
    check(stl, tree, W.random_walk(3, T, D, seed=5), launch=launch, fused=True)


def test_long_interval_shrinks_the_tile(stl):
    """Spans of 12,000 samples: the tile shrinks until the buffers fit in shared memory."""
    tree = W.And(W.Eventually(0, 12000, W.gt([1, 0], 0.3)), W.Always(100, 4000, W.lt([0, 1], 0.5)))
    check(stl, tree, W.random_walk(2, 30000, 2, seed=8), oracle_traces=[1])


def test_automatic_choice_falls_back_when_buffers_do_not_fit(stl):
    """Nested windows whose spans add to 45,000 samples fit no compiled tile: the automatic
    choice runs the interpreter (and the call succeeds)."""
    tree = W.Eventually(0, 15000, W.Always(0, 15000, W.Eventually(0, 15000, W.gt([1], 0.0))))
    p = stl.params("hard")
    f = stl.Formula(tree, D=1)
    assert f.get_launch(64, 60000, p, False)["kernel"] == "interpreter"
    x = torch.from_numpy(W.random_walk(2, 1000, 1, seed=3)).cuda().repeat(32, 40, 1)
    rho = stl.robustness(f, x, p=p)
    assert rho.shape == (64, 40000)


def test_ties_follow_the_oracle(stl):
    """Integer-valued signals: exact ties everywhere; the selections must be the oracle's."""
    rng = np.random.default_rng(9)
    sig = rng.integers(-3, 4, size=(8, 4000, 3)).astype(np.float32)
    for tree in (W.config1_formula(), W.Until(2, 25, W.gt([1, 0, 0], 0), W.gt([0, 1, 0], 0)),
                 W.Always(0, 40, W.Eventually(3, 19, W.lt([0, 0, 1], 0.0)))):
        check(stl, tree, sig, launch=dict(tile=1024))


@pytest.mark.parametrize("K", [5, 6, 7, 13, 14, 30, 31, 200, 401])
def test_window_lengths_with_ties(stl, K):
    """Direct loops (K < 6), runs of 3 .. 15, the direct middle and both level-2 middles
    (sliding blocks for max / min, aligned blocks for the Until's clamps) on integer signals."""
    rng = np.random.default_rng(K)
    sig = rng.integers(-2, 3, size=(4, 5000, 2)).astype(np.float32)
    for tree in (W.Eventually(1, K, W.gt([1, 0], 0.0)), W.Always(0, K - 1, W.lt([0, 1], 0.5)),
                 W.Until(K - 1, 2 * K + 20, W.gt([1, 0], -1.0), W.gt([0, 1], 0.0))):
        check(stl, tree, sig, launch=dict(tile=2048))


# ------------------------------------------------------------------ the headline launch
def test_config1_full_size_default_launch(stl):
    """B=1024, T=50000 with the automatic kernel choice (the compiled kernel at this size):
    sampled traces against the oracle, every value and gradient against the interpreter."""
    B, T = 1024, 50000
    sig = W.config1_inputs(B=B, T=T, seed=0)
    tree = W.config1_formula()
    p = stl.params("hard")
    f = stl.Formula(tree, D=3)
    assert f.get_launch(B, T, p, False)["kernel"] == "compiled"
    assert f.get_launch(B, T, p, True)["kernel"] == "compiled"
    x = torch.from_numpy(sig).cuda()
    g = torch.from_numpy(np.random.default_rng(2).normal(size=(B, T)).astype(np.float32)).cuda()
    rho = stl.robustness(f, x, p=p)
    gs, _ = stl.robustness_backward(f, x, g, p=p)
    fi = stl.Formula(tree, D=3)
    fi.set_launch(kernel="interpreter")
    assert torch.equal(rho, stl.robustness(fi, x, p=p))
    assert torch.equal(gs, stl.robustness_backward(fi, x, g, p=p)[0])
    idx = [0, 700]
    ref = oracle.robustness(tree, sig[idx])
    np.testing.assert_array_equal(rho[idx].cpu().numpy(), ref.astype(np.float32))
    gref, _ = oracle.robustness_grad(tree, sig[idx], g[idx].cpu().numpy().astype(np.float64))
    assert per_trace_err(gs[idx].cpu().numpy(), gref) <= GRAD_TOL


def test_autotune_over_both_kernels(stl):
    """The autotuner times interpreter and compiled shapes; whichever wins, results match."""
    sig = W.config1_inputs(B=64, T=20000, seed=1)
    x = torch.from_numpy(sig).cuda()
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("hard")
    ref = stl.robustness(f, x, p=p).clone()
    for bwd in (False, True):
        launch, _ = stl.autotune(f, x, p=p, backward=bwd)
        assert launch["kernel"] in ("compiled", "interpreter")
    assert torch.equal(stl.robustness(f, x, p=p), ref)


def test_not_applicable_is_an_error(stl):
    """Forcing the compiled kernel where it does not apply fails on the host, before a launch."""
    f = stl.Formula(W.Eventually(0, math.inf, W.gt([1], 0.0)), D=1)
    f.set_launch(kernel="compiled")
    with pytest.raises(stl.StlError):
        stl.robustness(f, torch.zeros((2, 50, 1), device="cuda"))
    f = stl.Formula(W.Eventually(10, 20, W.gt([1], 0.0)), D=1)
    f.set_launch(kernel="compiled")
    with pytest.raises(stl.StlError):   # every read of the predicate lies past the end (T <= a)
        stl.robustness(f, torch.zeros((2, 10, 1), device="cuda"), p=stl.params("hard"))
    check(stl, W.Eventually(10, 20, W.gt([1], 0.0)), W.random_walk(2, 11, 1, seed=1))   # T = a + 1
    with pytest.raises(stl.StlError):   # smooth semantics run in the interpreter only
        stl.robustness(f, torch.zeros((2, 500, 1), device="cuda"), p=stl.params("smooth", tau=2.0))


def test_bounds_checked_build(stl, monkeypatch):
    """STL_FK_CHECK=1 generates the kernels with every shared-memory index compared against the
    length of its buffer (an index outside is not performed and sets the device status word to
    STL_ERR_DEVICE_CHECK): a stand-in for compute-sanitizer, which is closed on this machine.  The
    shapes of the parity tests, both adjoint-ring placements and both pad kinds run clean and
    give the same results as the unchecked kernels."""
    from paper_2501_04194_gb300.binding import device_status
    monkeypatch.setenv("STL_FK_CHECK", "1")
    device_status()
    sig1 = W.config1_inputs(B=3, T=3001, seed=4)
    for launch in ({}, dict(tile=512, segment=900), dict(threads=256, tile=768), dict(threads=256, tile=1024)):
        check(stl, W.config1_formula(), sig1, launch=launch, fused=True)
    for name, tree, D, T in EDGE:
        check(stl, tree, W.random_walk(3, T, D, seed=5), launch=dict(tile=512, segment=300), fused=True)
    rng = np.random.default_rng(3)
    ties = rng.integers(-2, 3, size=(3, 3000, 2)).astype(np.float32)
    for K in (6, 30, 401):
        check(stl, W.Until(K - 1, 2 * K + 20, W.gt([1, 0], -1.0), W.gt([0, 1], 0.0)), ties, launch=dict(tile=2048))
        check(stl, W.Eventually(1, K, W.gt([1, 0], 0.0)), ties, launch=dict(tile=1024))
    check(stl, W.config1_formula(), W.config1_inputs(B=4, T=50000, seed=2), oracle_traces=[0])
    torch.cuda.synchronize()
    assert device_status() == 0


@pytest.mark.parametrize("seed", range(10))
def test_random_formulas(stl, seed):
    """Seed-generated formulas of depth <= 4 (static intervals up to 300, Not nodes, constant
    pads), several tiles and a ragged tail: compiled == interpreter bit for bit, and the oracle."""
    rng = np.random.default_rng(200 + seed)
    tree = W.static_random_formula(rng, 3, 3 + seed % 2, 300)
    T = int(rng.integers(1500, 4000))
    launch = dict(tile=512) if seed % 3 == 0 else dict(threads=256, tile=1024, segment=T // 2) if seed % 3 == 1 else {}
    check(stl, tree, W.random_walk(3, T, 3, seed=seed), launch=launch, fused=seed % 2 == 0)
