"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle.

Bars (per trace, relative to the trace's largest |reference| value):
  hard-mode robustness   bit-exact float32 (selections; predicates without FMA)
  smooth robustness      1e-5
  gradients              1e-4
Sizes span several streaming steps (tile forced to 256) and ragged tails, traces split into
segments (backward warm-up), and the degenerate cases: T = 1, windows longer than the trace,
constant pads, True, a = b, b = inf.
"""
import math

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
    fin = np.isfinite(r)
    assert np.array_equal(fin, np.isfinite(g)) and np.array_equal(g[~fin], r[~fin])
    scale = np.where(fin, np.abs(r), 0).max(axis=1, keepdims=True)
    scale = np.maximum(scale, 1e-30)
    with np.errstate(invalid="ignore"):   # inf - inf where both are the same infinity
        d = np.where(fin, np.abs(g - r), 0) / scale
    return d.max()


def run(stl, tree, sig, bounds=None, mode="hard", tau=1.0, mask_c=5.0, mask_eps=1e-3, launch=None, gout=None,
        expect_clean_status=True):
    D = sig.shape[2]
    f = stl.Formula(tree, D=D, n_slots=None if bounds is None else bounds.shape[1])
    if launch:
        f.set_launch(**launch)
    p = stl.params(mode, tau=tau, mask_c=mask_c, mask_eps=mask_eps)
    x = torch.from_numpy(np.ascontiguousarray(sig)).cuda()
    bt = None if bounds is None else torch.from_numpy(bounds).cuda()
    rho = stl.robustness(f, x, bt, p).cpu().numpy()
    gs = gb = None
    if gout is not None:
        g = torch.from_numpy(gout.astype(np.float32)).cuda()
        gs, gb = stl.robustness_backward(f, x, g, bt, p)
        gs = gs.cpu().numpy()
        gb = None if gb is None else gb.cpu().numpy()
    torch.cuda.synchronize()
    if expect_clean_status:
        from paper_2501_04194_gb300.binding import device_status
        assert device_status() == 0, "per-trace bounds outside the compiled caps"
    return rho, gs, gb


def check(stl, tree, sig, bounds=None, mode="hard", tau=1.0, mask_c=5.0, mask_eps=1e-3, launch=None, seed=0,
          grad=True):
    rng = np.random.default_rng(seed)
    B, T, _ = sig.shape
    gout = rng.normal(size=(B, T)).astype(np.float32) if grad else None
    rho, gs, gb = run(stl, tree, sig, bounds, mode, tau, mask_c, mask_eps, launch, gout)
    om = {"hard": oracle.HARD, "smooth": oracle.SMOOTH, "softmax": oracle.SOFTMAX}[mode]
    ref = oracle.robustness(tree, sig, bounds=bounds, mode=om, tau=tau, mask_c=mask_c, mask_eps=mask_eps)
    if mode == "hard":
        np.testing.assert_array_equal(rho, ref.astype(np.float32))
    else:
        assert per_trace_err(rho, ref) <= VAL_TOL
    if grad:
        gref, gbref = oracle.robustness_grad(tree, sig, gout.astype(np.float64), bounds=bounds, mode=om, tau=tau,
                                             mask_c=mask_c, mask_eps=mask_eps)
        assert per_trace_err(gs, gref) <= GRAD_TOL
        if gbref is not None and mode != "hard":
            assert per_trace_err(gb, gbref) <= GRAD_TOL
        elif gb is not None:
            assert np.all(gb == 0)


# ------------------------------------------------------------------ configs
def test_config0(stl):
    sig = W.config0_inputs()
    check(stl, W.config0_formula(), sig)
    check(stl, W.config0_formula(), sig, mode="smooth", tau=5.0)


@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 10.0)])
@pytest.mark.parametrize("T", [1000, 2345])
def test_config1_small_batch(stl, mode, tau, T):
    sig = W.config1_inputs(B=6, T=T, seed=3)
    check(stl, W.config1_formula(), sig, mode=mode, tau=tau)


@pytest.mark.parametrize("launch", [dict(tile=256), dict(tile=256, segment=700), dict(tile=512, threads=256),
                                    dict(tile=1024, threads=256, segment=1500), dict(tile=448, threads=64),
                                    dict(tile=256, threads=64, segment=900)])
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 10.0)])
def test_config1_streaming_and_segments(stl, launch, mode, tau):
    sig = W.config1_inputs(B=5, T=3001, seed=4)
    check(stl, W.config1_formula(), sig, mode=mode, tau=tau, launch=launch, seed=1)


def test_config2_smooth_mask(stl):
    sig, bounds = W.config2_inputs(B=32, T=2000, seed=0)
    check(stl, W.config2_formula(), sig, bounds=bounds, mode="smooth", tau=10.0, mask_c=5.0, mask_eps=1e-3)
    check(stl, W.config2_formula(), sig, bounds=bounds, mode="hard", mask_c=5.0, mask_eps=1e-3)


@pytest.mark.parametrize("c,eps", [(0.7, 1e-3), (1.5, 1e-2), (5.0, 1e-3)])
@pytest.mark.parametrize("op", ["eventually", "always"])
def test_smooth_mask_plateau_and_edge_bands(stl, c, eps, op):
    # logsumexp mode: offsets whose float weight is exactly 1 - eps go through a sliding window,
    # the two edge bands tap by tap; per-trace widths b - a in [20, 300] give plateaus from none
    # (short windows at c = 0.7) to most of the support, one and several steps per trace
    sig, bounds = W.config2_inputs(B=24, T=1500, seed=11)
    ctor = W.EventuallySm if op == "eventually" else W.AlwaysSm
    tree = ctor(100, 400, W.gt([1.0], 0.8), slot=0)
    for launch in (None, dict(tile=256)):
        check(stl, tree, sig, bounds=bounds, mode="smooth", tau=10.0, mask_c=c, mask_eps=eps, launch=launch)


@pytest.mark.parametrize("mode", ["hard", "smooth"])
def test_always_sm_small_sharpness(stl, mode):
    rng = np.random.default_rng(7)
    sig = rng.normal(size=(6, 700, 1)).astype(np.float32)
    a = rng.uniform(0, 30, size=6)
    bounds = np.stack([a, a + rng.uniform(5, 60, size=6)], 1).astype(np.float32)[:, None, :]
    tree = W.AlwaysSm(40, 100, W.lt([1.0], 0.3), slot=0)
    check(stl, tree, sig, bounds=bounds, mode=mode, tau=3.0, mask_c=0.7, mask_eps=1e-2, launch=dict(tile=256))


# ------------------------------------------------------------------ formula families
TABLE3 = W.table3_formulas(D=2, I=(2, 37))


@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 4.0)])
def test_table3_formulas(stl, k, mode, tau):
    T = 300 if k < 3 else 1100
    sig = W.random_walk(3, T, 2, seed=10 + k)
    check(stl, TABLE3[k], sig, mode=mode, tau=tau, launch=dict(tile=256))


def _random_ragged_bounds(rng, B, n_slots, cap):
    a = rng.integers(0, cap // 2 + 1, size=(B, n_slots))
    b = a + rng.integers(0, cap // 2 + 1, size=(B, n_slots))
    return np.stack([a, b], axis=2).astype(np.float32)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 3.0)])
def test_random_formulas_per_trace_bounds(stl, seed, mode, tau):
    rng = np.random.default_rng(100 + seed)
    ctr = [0]
    tree = W.random_formula(rng, 3, 3 if seed % 2 else 4, ctr, b_cap=60.0)
    n_slots = max(1, ctr[0])
    B, T = 4, int(rng.integers(150, 1300))
    sig = W.random_walk(B, T, 3, seed=seed)
    bounds = _random_ragged_bounds(rng, B, n_slots, 60)
    check(stl, tree, sig, bounds=bounds, mode=mode, tau=tau, launch=dict(tile=256, segment=400 if seed % 3 == 0 else 0))


# ------------------------------------------------------------------ softmax-weighted mode
SOFT_CASES = [
    ("config0", W.config0_formula(), 2, 100, None),
    ("config1", W.config1_formula(), 3, 1500, dict(tile=256)),
    ("config1_segments", W.config1_formula(), 3, 2100, dict(tile=256, segment=700)),
    ("until_pad", W.Until(2, 40, W.gt([1, 0], 0.0), W.lt([0, 1], 0.3), pad=0.2), 2, 333, dict(tile=64)),
    ("until_unbounded", W.Until(0, math.inf, W.gt([1, 0], -0.3), W.gt([0, 1], 0.4)), 2, 150, None),
    ("windows_const_pad", W.And(W.Eventually(3, 60, W.gt([1, 0], 0.0), pad=-0.5), W.Always(0, 7, W.lt([0, 1], 1.0))), 2,
     700, dict(tile=128)),
    ("or_not", W.Or(W.Not(W.gt([1], 0.2)), W.Always(1, 30, W.gt([1], -0.5))), 1, 400, None),
    ("table3_phi4", W.table3_formulas(D=2, I=(2, 37))[3], 2, 600, dict(tile=256)),
]


@pytest.mark.parametrize("name,tree,D,T,launch", SOFT_CASES, ids=[c[0] for c in SOFT_CASES])
@pytest.mark.parametrize("tau", [1.0, 8.0])
def test_softmax_mode(stl, name, tree, D, T, launch, tau):
    sig = W.random_walk(4, T, D, seed=len(name))
    check(stl, tree, sig, mode="softmax", tau=tau, launch=launch)


@pytest.mark.parametrize("op", ["eventually_sm", "always_sm"])
def test_softmax_smooth_mask(stl, op):
    sig, bounds = W.config2_inputs(B=16, T=700, seed=3)
    tree = (op, (120.0, 450.0, 0, None), W.gt([1.0], 0.8))
    check(stl, tree, sig, bounds=bounds, mode="softmax", tau=10.0, mask_c=5.0, launch=dict(tile=256))


# ------------------------------------------------------------------ Until over a masked interval
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 4.0), ("softmax", 4.0)])
@pytest.mark.parametrize("nested", [False, True])
def test_until_sm(stl, mode, tau, nested):
    rng = np.random.default_rng(50)
    B, T = 6, 900
    sig = W.random_walk(B, T, 2, seed=51)
    u = W.UntilSm(60.0, 120.0, W.gt([1, 0], 0.0), W.lt([0, 1], 0.3), slot=0)
    tree = W.Always(0, 30, u) if nested else u
    a = rng.uniform(0.0, 50.0, size=B)
    b = a + rng.uniform(5.0, 60.0, size=B)
    bounds = np.stack([a, np.minimum(b, 119.0)], axis=1).astype(np.float32)[:, None, :]
    bounds[0, 0] = [0.0, 0.6]   # a support of one or two offsets
    check(stl, tree, sig, bounds=bounds, mode=mode, tau=tau, mask_c=2.0, launch=dict(tile=256))


# ------------------------------------------------------------------ region (norm) predicates
@pytest.mark.parametrize("D", [1, 2, 3, 5])
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 3.0)])
def test_norm_predicates(stl, D, mode, tau):
    """Inside/outside-ball predicates in a reach/avoid tree, several tiles and a ragged tail,
    one sample exactly at a centre (mu = 0: zero subgradient on both sides), a zero scale."""
    rng = np.random.default_rng(40 + D)
    sig = W.random_walk(5, 1337, D, seed=D)
    g1 = [float(v) for v in sig[1, 600]]
    g2 = [float(v) for v in rng.normal(size=D)]
    s2 = [0.0 if (d == D - 1 and D > 1) else float(rng.uniform(0.5, 2.0)) for d in range(D)]
    tree = W.And(W.Eventually(5, 60, W.norm_lt([1.0] * D, g1, 0.4)),
                 W.Or(W.Always(0, 25, W.norm_gt(s2, g2, 0.7)), W.Until(0, 30, W.norm_gt([1.0] * D, g1, 0.2),
                                                                       W.gt([1.0] + [0.0] * (D - 1), 0.3))))
    check(stl, tree, sig, mode=mode, tau=tau, launch=dict(tile=256))


@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 20.0)])
def test_reach_avoid_rollouts(stl, mode, tau):
    """The control-synthesis specification (reach a goal disc within [50, 150], avoid three
    obstacle discs throughout) on rollouts of the saturated single integrator, T = 200."""
    for k, (g, o, r) in enumerate(W.config4_problems(3, seed=7)):
        u = W.random_controls(64, seed=k, scale=2.0)
        sig = W.rollout(u) + np.float32(0.3) * np.asarray(g, dtype=np.float32) * np.float32(k)
        check(stl, W.reach_avoid_formula(g, o, r), sig.astype(np.float32), mode=mode, tau=tau, seed=k)


# ------------------------------------------------------------------ degenerate cases
EDGE = [
    ("T1", W.config1_formula(), 3, 1),
    ("T2", W.Until(0, 3, W.gt([1, 0], 0.0), W.lt([0, 1], 0.2)), 2, 2),
    ("window_longer_than_trace", W.Always(3, 90, W.gt([1], 0.1)), 1, 17),
    ("const_pad", W.Eventually(2, 40, W.gt([1, 0], 0.0), pad=-0.25), 2, 33),
    ("const_pad_until", W.Until(1, 30, W.gt([1, 0], 0.0), W.lt([0, 1], 0.3), pad=0.1), 2, 45),
    ("true_until", W.Until(2, 9, W.true(), W.gt([1], 0.0)), 1, 50),
    ("a_eq_b", W.And(W.Eventually(4, 4, W.gt([1, 0], 0.0)), W.Until(3, 3, W.gt([1, 0], 0.1), W.gt([0, 1], 0.0))), 2, 64),
    ("unbounded", W.Eventually(0, math.inf, W.Always(0, math.inf, W.gt([1], 0.0))), 1, 300),
    ("unbounded_until", W.Until(0, math.inf, W.gt([1, 0], -0.5), W.gt([0, 1], 0.5)), 2, 260),
    ("not_chain", W.Not(W.Or(W.Not(W.gt([1], 0.0)), W.Always(1, 5, W.Not(W.lt([1], 0.2))))), 1, 77),
]


@pytest.mark.parametrize("name,tree,D,T", EDGE, ids=[e[0] for e in EDGE])
@pytest.mark.parametrize("mode,tau", [("hard", 1.0), ("smooth", 2.0)])
def test_degenerate(stl, name, tree, D, T, mode, tau):
    sig = W.random_walk(3, T, D, seed=5)
    if name == "true_until" and mode == "smooth":
        tau = 6.0
    check(stl, tree, sig, mode=mode, tau=tau, launch=dict(tile=32) if T > 40 else None)


def test_ties_follow_the_oracle(stl):
    """Integer-valued signals make exact ties everywhere; hard gradients must still land on
    the same samples as the oracle's tie rule."""
    rng = np.random.default_rng(9)
    sig = rng.integers(-3, 4, size=(8, 400, 3)).astype(np.float32)
    for tree in (W.config1_formula(), W.Until(2, 25, W.gt([1, 0, 0], 0), W.gt([0, 1, 0], 0)),
                 W.Always(0, 40, W.Eventually(3, 19, W.lt([0, 0, 1], 0.0)))):
        check(stl, tree, sig, launch=dict(tile=64))


@pytest.mark.parametrize("K", [6, 7, 9, 13, 14])
def test_short_windows_with_ties(stl, K):
    """Windows of 6..14 samples (runs of 3 below 14) and an Until whose first window has K
    samples, on integer signals full of ties: values bit-exact, gradients on the oracle's
    tie-broken samples."""
    rng = np.random.default_rng(K)
    sig = rng.integers(-2, 3, size=(5, 700, 2)).astype(np.float32)
    for tree in (W.Eventually(1, K, W.gt([1, 0], 0.0)), W.Always(0, K - 1, W.lt([0, 1], 0.5)),
                 W.Until(K - 1, K + 20, W.gt([1, 0], -1.0), W.gt([0, 1], 0.0))):
        check(stl, tree, sig, launch=dict(tile=256))
        check(stl, tree, sig, launch=dict(tile=448, threads=64))


def test_empty_batch(stl):
    f = stl.Formula(W.config0_formula(), D=2)
    x = torch.zeros((0, 10, 2), device="cuda")
    out = stl.robustness(f, x)
    assert out.shape == (0, 10)


def test_bounds_outside_caps_set_the_device_status(stl):
    from paper_2501_04194_gb300.binding import device_status
    device_status()
    tree = W.Eventually(0, 10, W.gt([1], 0.0), slot=0)
    sig = W.random_walk(2, 50, 1, seed=0)
    bounds = np.array([[[0, 5]], [[2, 30]]], dtype=np.float32)   # 30 > cap 10
    run(stl, tree, sig, bounds=bounds, expect_clean_status=False)
    assert device_status() == -6
    assert device_status() == 0




@pytest.mark.parametrize("mode", ["hard", "smooth", "softmax"])
def test_masked_window_with_empty_support(stl, mode):
    """Per-trace bounds with a = b give a mask that is positive nowhere (Eq. smooth mask with
    eps > 0): Eventually is -inf and Always +inf at every sample, with zero gradient; the other
    traces of the batch are ordinary."""
    rng = np.random.default_rng(11)
    sig = rng.normal(size=(4, 600, 1)).astype(np.float32)
    bounds = np.array([[[10.0, 10.0]], [[5.0, 60.0]], [[0.0, 0.0]], [[20.0, 90.0]]], dtype=np.float32)
    trees = [W.EventuallySm(40, 100, W.gt([1.0], 0.1), slot=0)]
    if mode == "hard":
        trees.append(W.Or(W.AlwaysSm(40, 100, W.lt([1.0], 0.5), slot=0), W.gt([1.0], 2.5)))
    for tree in trees:
        check(stl, tree, sig, bounds=bounds, mode=mode, tau=5.0, mask_c=5.0, mask_eps=1e-3)

# ------------------------------------------------------------------ long steps: direct-read forward
# Hard forward steps of at least 4096 new samples per node take the direct-read passes (pads
# filled past the end of the trace, runs of 15 for long windows); these launches force them,
# with the last step of each trace short and long, pads of both kinds, windows past the end,
# b = inf, per-trace and masked bounds, and traces split into segments.
LONG_CASES = [
    ("config1_512", W.config1_formula(), 3, 20000, dict(tile=7168, threads=512), None),
    ("config1_256_segments", W.config1_formula(), 3, 12001, dict(tile=4096, threads=256, segment=6000), None),
    ("until_const_pad", W.Until(2, 40, W.gt([1, 0], 0.0), W.lt([0, 1], 0.3), pad=0.2), 2, 9001,
     dict(tile=4096, threads=512), None),
    ("until_a0_ev", W.Eventually(0, 3000, W.Until(0, 17, W.gt([1, 0], -0.2), W.gt([0, 1], 0.1))), 2, 8192,
     dict(tile=4096, threads=512), None),
    ("always_to_end", W.Or(W.Always(0, math.inf, W.gt([1, 0], -2.0)), W.Not(W.lt([0, 1], 0.5))), 2, 6000,
     dict(tile=4096, threads=512), None),
    ("windows_past_end", W.And(W.Eventually(5000, 9000, W.gt([1, 0], 0.0), pad=-0.5),
                               W.Always(3, 12, W.lt([0, 1], 1.0))), 2, 7000, dict(tile=7168, threads=512), None),
    ("slots", W.Eventually(300, 900, W.Always(100, 400, W.gt([1], 0.1), slot=1), slot=0), 1, 9000,
     dict(tile=4096, threads=512), "slots"),
    ("masked", W.EventuallySm(100.0, 400.0, W.gt([1], 0.8), slot=0), 1, 8000, dict(tile=4096, threads=512), "masked"),
    ("table3_phi4", W.table3_formulas(D=2, I=(2, 37))[3], 2, 10000, dict(tile=4096, threads=512), None),
]


@pytest.mark.parametrize("name,tree,D,T,launch,kind", LONG_CASES, ids=[c[0] for c in LONG_CASES])
def test_long_steps_hard(stl, name, tree, D, T, launch, kind):
    sig = W.random_walk(4, T, D, seed=len(name))
    bounds = None
    rng = np.random.default_rng(len(name))
    if kind == "slots":
        outer = np.stack([rng.uniform(0, 300, 4), rng.uniform(600, 900, 4)], 1)
        inner = np.stack([rng.uniform(0, 100, 4), rng.uniform(200, 400, 4)], 1)
        bounds = np.floor(np.stack([outer, inner], 1)).astype(np.float32)
    elif kind == "masked":
        a = rng.uniform(0, 100, 4)
        bounds = np.stack([a, a + rng.uniform(20, 300, 4)], 1).astype(np.float32)[:, None, :]
    check(stl, tree, sig, bounds=bounds, mode="hard", launch=launch)

# ------------------------------------------------------------------ full-size spot checks
def test_config1_full_size_sampled(stl):
    """B=1024, T=50000 (the benchmark launch): sampled traces checked against the oracle."""
    B, T = 1024, 50000
    sig = W.config1_inputs(B=B, T=T, seed=0)
    tree = W.config1_formula()
    f = stl.Formula(tree, D=3)
    p = stl.params("hard")
    x = torch.from_numpy(sig).cuda()
    rho = stl.robustness(f, x, p=p)
    gout = torch.from_numpy(np.random.default_rng(2).normal(size=(B, T)).astype(np.float32)).cuda()
    gs, _ = stl.robustness_backward(f, x, gout, p=p)
    torch.cuda.synchronize()
    idx = [0, 511, 1023]
    sub = sig[idx]
    ref = oracle.robustness(tree, sub)
    np.testing.assert_array_equal(rho[idx].cpu().numpy(), ref.astype(np.float32))
    gref, _ = oracle.robustness_grad(tree, sub, gout[idx].cpu().numpy().astype(np.float64))
    assert per_trace_err(gs[idx].cpu().numpy(), gref) <= GRAD_TOL
