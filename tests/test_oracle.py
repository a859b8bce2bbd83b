"""Pins for the FP64 oracle: it is checked against things other than itself.

- the worked Example 1 (Sec. IV-B) from tests/golden/example1.txt;
- the paper's masking construction (Sec. IV-B / IV-C) evaluated by brute force on every
  window of tiny traces with many ties, in hard and smooth mode;
- the derived-operator identities of Sec. III-B (Or, Eventually, Always);
- the textbook backward recurrence of the unbounded Until;
- the Boolean semantics (Eq. "boolean") against the sign of the robustness;
- the temperature limit and error bound of the logsumexp (Sec. III-C);
- logsumexp flattening (Sec. IV-D) and the closed flat form of the smooth Until;
- float32 predicate arithmetic against numpy float32;
- FP64 central finite differences and torch autograd of the masked construction for
  every gradient, including those of the smooth-mask bounds (Sec. VI).
"""
import math
import os

import numpy as np
import pytest
import torch
from scipy.special import logsumexp

import masked_reference as mr
import oracle
import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
HARD, SMOOTH = oracle.HARD, oracle.SMOOTH


def one(sig1d):
    return np.asarray(sig1d, dtype=np.float32).reshape(1, -1, 1)


def x_pred():
    return W.gt([1.0], 0.0)


# ------------------------------------------------------------------ Example 1
def test_example1_golden():
    lines = [l for l in open(os.path.join(HERE, "golden", "example1.txt")) if l.strip() and not l.startswith("#")]
    assert len(lines) == 2
    for line in lines:
        lhs, rhs = line.split("|")
        toks = lhs.split()
        pad = None if toks[0] == "last" else float(toks[0])
        a, b = float(toks[1]), float(toks[2])
        s = [float(v) for v in toks[3:]]
        want = np.array([float(v) for v in rhs.split()])
        got = oracle.robustness(W.Eventually(a, b, x_pred(), pad=pad), one(s))[0]
        np.testing.assert_array_equal(got, want)


# ------------------------------------------------------------------ brute-force masking
def _tiny_signals(rng, T, n=4):
    out = [rng.integers(-2, 3, size=T).astype(np.float32) for _ in range(n)]
    out.append(np.zeros(T, dtype=np.float32))
    return out


@pytest.mark.parametrize("op", ["eventually", "always"])
@pytest.mark.parametrize("pad", [None, -3.0])
def test_windows_match_masking(op, pad):
    rng = np.random.default_rng(1)
    for T in range(1, 9):
        for s in _tiny_signals(rng, T):
            xt = torch.tensor(s, dtype=torch.float64)
            for a in range(0, T + 2):
                for b in list(range(a, T + 2)) + [math.inf]:
                    f = (op, (float(a), float(b), None, pad), x_pred())
                    got = oracle.robustness(f, one(s))[0]
                    want = mr.eventually_always(xt, a, b, pad, op, True, 1.0).numpy()
                    np.testing.assert_array_equal(got, want, err_msg=f"{op} [{a},{b}] T={T}")
                    for tau in (0.7, 3.0):
                        got = oracle.robustness(f, one(s), mode=SMOOTH, tau=tau)[0]
                        want = mr.eventually_always(xt, a, b, pad, op, False, tau).numpy()
                        np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pad", [None, 1.0])
def test_until_matches_masking(pad):
    rng = np.random.default_rng(2)
    for T in range(1, 8):
        for _ in range(3):
            s = rng.integers(-2, 3, size=(T, 2)).astype(np.float32)
            xt = torch.tensor(s, dtype=torch.float64)
            for a in range(0, T + 1):
                for b in list(range(a, T + 2)) + [math.inf]:
                    f = W.Until(a, b, W.gt([1, 0], 0.0), W.gt([0, 1], 0.0), pad=pad)
                    got = oracle.robustness(f, s[None])[0]
                    want = mr.until(xt[:, 0], xt[:, 1], a, b, pad, True, 1.0).numpy()
                    np.testing.assert_array_equal(got, want, err_msg=f"U[{a},{b}] T={T}")
                    got = oracle.robustness(f, s[None], mode=SMOOTH, tau=2.0)[0]
                    want = mr.until(xt[:, 0], xt[:, 1], a, b, pad, False, 2.0).numpy()
                    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11)


def test_nested_formulas_match_masking():
    rng = np.random.default_rng(3)
    forms = [W.config0_formula(), W.config1_formula()] + W.table3_formulas(D=2, I=(1, 4))
    for f in forms:
        D = 3 if f is forms[1] else 2
        for T in (5, 13, 29):
            s = rng.normal(size=(T, D)).astype(np.float32)
            xt = torch.tensor(s, dtype=torch.float64)
            got = oracle.robustness(f, s[None], exact=True)[0]
            want = mr.evaluate(f, xt, hard=True).numpy()
            np.testing.assert_array_equal(got, want)
            got = oracle.robustness(f, s[None], mode=SMOOTH, tau=1.5, exact=True)[0]
            want = mr.evaluate(f, xt, hard=False, tau=1.5).numpy()
            np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10)


# ------------------------------------------------------------------ identities
def test_until_unbounded_textbook_recurrence():
    """phi U_[0,inf) psi satisfies U_t = max(min(phi_t, psi_t), min(phi_t, U_{t+1}))."""
    rng = np.random.default_rng(4)
    for T in (1, 2, 7, 40):
        s = rng.integers(-3, 4, size=(T, 2)).astype(np.float32)
        got = oracle.robustness(W.Until(0, math.inf, W.gt([1, 0], 0.0), W.gt([0, 1], 0.0)), s[None])[0]
        p, q = s[:, 0].astype(np.float64), s[:, 1].astype(np.float64)
        U = np.empty(T)
        U[T - 1] = min(p[T - 1], q[T - 1])
        for t in range(T - 2, -1, -1):
            U[t] = max(min(p[t], q[t]), min(p[t], U[t + 1]))
        np.testing.assert_array_equal(got, U)


@pytest.mark.parametrize("mode,tau", [(HARD, 1.0), (SMOOTH, 2.5)])
def test_derived_operator_identities(mode, tau):
    rng = np.random.default_rng(5)
    s = rng.normal(size=(3, 60, 2)).astype(np.float32)
    p, q = W.gt([1, 0], 0.1), W.lt([0, 1], 0.3)
    exact = (lambda a, b: np.testing.assert_array_equal(a, b)) if mode == HARD else \
        (lambda a, b: np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-12))
    R = lambda f: oracle.robustness(f, s, mode=mode, tau=tau)  # noqa: E731
    for (a, b) in ((0, 0), (2, 9), (5, 80)):
        exact(R(W.Always(a, b, p)), -R(W.Eventually(a, b, W.Not(p))))
        exact(R(W.Eventually(a, b, q)), R(W.Until(a, b, W.true(), q)))
    exact(R(W.Or(p, q)), -R(W.And(W.Not(p), W.Not(q))))
    if mode == HARD:
        exact(R(W.Until(0, 0, p, q)), R(W.And(p, q)))


def test_boolean_semantics_sign():
    rng = np.random.default_rng(6)
    forms = [W.config0_formula(), W.Until(1, 3, W.gt([1, 0], 0.0), W.lt([0, 1], 0.2)),
             W.Or(W.Always(0, 2, W.gt([1, 0], 0.3)), W.Not(W.Eventually(1, 4, W.lt([1, 1], 0.0)))),
             W.Until(0, 2, W.Eventually(0, 1, W.gt([0, 1], -0.2)), W.Always(1, 2, W.gt([1, 0], 0.1)), pad=0.5),
             W.And(W.Eventually(0, 4, W.norm_lt([1, 1], [0.3, -0.2], 0.9)),
                   W.Always(0, 3, W.norm_gt([1, 0.5], [-0.4, 0.6], 0.4)))]
    for f in forms:
        for _ in range(20):
            T = int(rng.integers(1, 10))
            s = rng.normal(size=(T, 2)).astype(np.float32)
            rho = oracle.robustness(f, s[None])[0]
            for t in range(T):
                if rho[t] > 0:
                    assert mr.boolean(f, s, t)
                elif rho[t] < 0:
                    assert not mr.boolean(f, s, t)


# ------------------------------------------------------------------ smooth semantics
def test_tau_limit_and_bound():
    """hard <= smooth-max <= hard + ln(K)/tau over a window of K entries (Sec. III-C)."""
    rng = np.random.default_rng(7)
    s = rng.normal(size=(2, 50, 1)).astype(np.float32)
    f = W.Eventually(3, 12, x_pred())
    hard = oracle.robustness(f, s)
    for tau in (1.0, 10.0, 100.0, 1e4):
        sm = oracle.robustness(f, s, mode=SMOOTH, tau=tau)
        assert np.all(sm >= hard - 1e-12)
        assert np.all(sm <= hard + math.log(10) / tau + 1e-12)
    g = W.config1_formula()
    s3 = rng.normal(size=(2, 80, 3)).astype(np.float32)
    h3 = oracle.robustness(g, s3)
    errs = [np.abs(oracle.robustness(g, s3, mode=SMOOTH, tau=tau) - h3).max() for tau in (10.0, 100.0, 1000.0)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 0.02


def test_lse_flattening():
    """Nested logsumexp And equals one flat logsumexp (Sec. IV-D)."""
    rng = np.random.default_rng(8)
    s = rng.normal(size=(2, 30, 3)).astype(np.float32)
    ps = [W.gt(W.onehot(3, d), 0.0) for d in range(3)]
    tau = 3.0
    got = oracle.robustness(W.And(W.And(ps[0], ps[1]), ps[2]), s, mode=SMOOTH, tau=tau)
    want = -logsumexp(-tau * s.astype(np.float64), axis=2) / tau
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_smooth_until_flat_form():
    """Smooth Until equals (1/tau) log sum_i 1/(S_t(i) + Q_{t+i}) with S_t(i) = sum_{k<=i} e^{-tau phi},
    Q = e^{-tau psi}: the nested logsumexps of Sec. IV-C flattened (Sec. IV-D)."""
    rng = np.random.default_rng(9)
    T, a, b, tau = 25, 2, 7, 1.7
    s = rng.normal(size=(T, 2)).astype(np.float32)
    got = oracle.robustness(W.Until(a, b, W.gt([1, 0], 0.0), W.gt([0, 1], 0.0)), s[None], mode=SMOOTH, tau=tau)[0]
    p, q = s[:, 0].astype(np.float64), s[:, 1].astype(np.float64)
    rd = lambda x, j: x[min(j, T - 1)]  # noqa: E731
    want = np.empty(T)
    for t in range(T):
        acc = 0.0
        for i in range(a, b + 1):
            S = sum(math.exp(-tau * rd(p, t + k)) for k in range(i + 1))
            acc += 1.0 / (S + math.exp(-tau * rd(q, t + i)))
        want[t] = math.log(acc) / tau
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)


def test_smooth_mask_limits():
    """Eq. "smooth mask": with c large and eps small the mask is 1 inside [a,b], 1/2 at the
    integer endpoints and 0 outside, so hard mode equals the hard window and smooth mode the
    closed form (1/tau) log(sum_{a<i<b} e^{tau x} + (e^{tau x_a} + e^{tau x_b})/2)."""
    rng = np.random.default_rng(10)
    T = 40
    s = rng.normal(size=(1, T, 1)).astype(np.float32)
    a, b = 4, 11
    bounds = np.array([[[a, b]]], dtype=np.float32)
    f = W.EventuallySm(20, 30, x_pred(), slot=0)
    hard = oracle.robustness(f, s, bounds=bounds, mask_c=200.0, mask_eps=1e-9)
    np.testing.assert_array_equal(hard, oracle.robustness(W.Eventually(a, b, x_pred()), s))
    tau = 2.0
    sm = oracle.robustness(f, s, bounds=bounds, mode=SMOOTH, tau=tau, mask_c=200.0, mask_eps=1e-12)[0]
    x = s[0, :, 0].astype(np.float64)
    rd = lambda j: x[min(j, T - 1)]  # noqa: E731
    want = [math.log(sum(math.exp(tau * rd(t + i)) for i in range(a + 1, b)) +
                     0.5 * (math.exp(tau * rd(t + a)) + math.exp(tau * rd(t + b)))) / tau for t in range(T)]
    np.testing.assert_allclose(sm, want, rtol=1e-9, atol=1e-9)


def test_smooth_mask_empty_support():
    """Eq. "smooth mask" with a = b: sigma(c(i-a)) - sigma(c(i-b)) = 0 for every offset, so with
    eps > 0 no mask weight is positive and the window is empty: Eventually is the max over an
    empty set, -inf, Always +inf, in every mode (the log of an empty sum), and nothing selects
    a sample, so the signal and bound gradients are zero."""
    rng = np.random.default_rng(12)
    s = rng.normal(size=(2, 50, 1)).astype(np.float32)
    bounds = np.array([[[7.0, 7.0]], [[3.0, 20.0]]], dtype=np.float32)
    for mode in (HARD, SMOOTH, oracle.SOFTMAX):
        for op, sgn in ((W.EventuallySm, 1.0), (W.AlwaysSm, -1.0)):
            f = op(10, 30, x_pred(), slot=0)
            r = oracle.robustness(f, s, bounds=bounds, mode=mode, tau=3.0, mask_c=5.0, mask_eps=1e-3)
            assert np.all(r[0] == -sgn * np.inf)
            assert np.all(np.isfinite(r[1]))
            g, gb = oracle.robustness_grad(f, s, np.ones((2, 50)), bounds=bounds, mode=mode, tau=3.0,
                                           mask_c=5.0, mask_eps=1e-3)
            assert np.all(g[0] == 0) and np.all(gb[0] == 0)


@pytest.mark.parametrize("c", [1.5, 5.0])
@pytest.mark.parametrize("mode", ["hard", "smooth", "softmax"])
@pytest.mark.parametrize("op", ["eventually", "always"])
def test_smooth_mask_support_has_no_cutoff(c, mode, op):
    """The smooth-mask window of Sec. VI against the unroll over EVERY offset (no support
    cutoff; tests/masked_reference.py): at c = 1.5 the mask stays above eps = 1e-3 for about
    4.6 steps past b and at c = 5 for about 1.4, so a support that stopped short of the last
    positive weight would drop terms.  Values, the signal gradient and d/da, d/db (torch
    autograd of the unroll) must agree.  Trace 1 ends inside the support (pad reads)."""
    rng = np.random.default_rng(21)
    T = 40
    s = rng.normal(size=(3, T, 1))
    s[:, :, 0] += np.linspace(0.0, 2.0, T)       # rising: the far edge of the window dominates
    gout = rng.normal(size=(3, T))
    bounds = np.array([[[2.3, 9.6]], [[0.4, 31.7]], [[5.0, 5.8]]])
    hard = {"hard": True, "smooth": False, "softmax": None}[mode]
    omode = {"hard": HARD, "smooth": SMOOTH, "softmax": oracle.SOFTMAX}[mode]
    ctor = W.EventuallySm if op == "eventually" else W.AlwaysSm
    f = ctor(40, 45, x_pred(), slot=0)
    kw = dict(mode=omode, tau=2.0, mask_c=c, mask_eps=1e-3, exact=True)
    got = oracle.robustness(f, s, bounds=bounds, **kw)
    g, gb = oracle.robustness_grad(f, s, gout, bounds=bounds, **kw)
    for b in range(3):
        x = torch.tensor(s[b, :, 0], requires_grad=True)
        a_t = torch.tensor(bounds[b, 0, 0], requires_grad=True)
        b_t = torch.tensor(bounds[b, 0, 1], requires_grad=True)
        y = mr.smooth_mask_window(x, a_t, b_t, c, 1e-3, None, op, hard, 2.0)
        np.testing.assert_allclose(got[b], y.detach().numpy(), rtol=1e-12, atol=1e-12)
        (y * torch.tensor(gout[b])).sum().backward()
        np.testing.assert_allclose(g[b, :, 0], x.grad.numpy(), rtol=1e-9, atol=1e-12)
        if mode == "hard":
            assert gb[b, 0, 0] == 0 and gb[b, 0, 1] == 0
        else:
            np.testing.assert_allclose(gb[b, 0], [a_t.grad.item(), b_t.grad.item()], rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("D", [1, 2, 3, 5])
def test_norm_predicate_float32_order(D):
    """Region predicates (Sec. VII-A) at random points whose distances are not exact: the
    oracle's rounded mode must equal numpy float32 arithmetic in the stated order (difference,
    scale, square, squares summed left to right, correctly rounded square root, then the
    radius), bit for bit.  A double-precision sum, another summation order or a fused
    multiply-add would differ on some of these 2000 points."""
    rng = np.random.default_rng(100 + D)
    s = (rng.normal(size=(4, 500, D)) * rng.uniform(0.1, 30.0, size=(4, 1, D))).astype(np.float32)
    sc = rng.uniform(0.2, 3.0, size=D).astype(np.float32)
    g = rng.normal(size=D).astype(np.float32) * np.float32(5)
    r = np.float32(rng.uniform(0.5, 4.0))
    u = (s[..., 0] - g[0]) * sc[0]
    q = u * u
    for d in range(1, D):
        u = (s[..., d] - g[d]) * sc[d]
        q = q + u * u
    mu = np.sqrt(q)
    assert mu.dtype == np.float32
    inside = oracle.robustness(W.norm_lt(sc.tolist(), g.tolist(), float(r)), s)
    np.testing.assert_array_equal(inside, (r - mu).astype(np.float64))
    outside = oracle.robustness(W.norm_gt(sc.tolist(), g.tolist(), float(r)), s)
    np.testing.assert_array_equal(outside, (mu - r).astype(np.float64))
    # the same points through a double-precision distance differ somewhere (the pin has teeth)
    mu64 = np.sqrt((((s.astype(np.float64) - g) * sc) ** 2).sum(axis=-1)).astype(np.float32)
    assert D == 1 or np.any(mu64 != mu)


def test_predicate_float32_rounding():
    rng = np.random.default_rng(11)
    s = (rng.normal(size=(2, 64, 3)) * 1e3).astype(np.float32)
    w = np.array([0.3, -1.7, 2.9], dtype=np.float32)
    c = np.float32(0.1234)
    got = oracle.robustness(W.gt(w.tolist(), float(c)), s)
    acc = s[..., 0] * w[0]
    acc = acc + s[..., 1] * w[1]
    acc = acc + s[..., 2] * w[2]
    want = (acc - c).astype(np.float32)
    np.testing.assert_array_equal(got, want.astype(np.float64))
    got = oracle.robustness(W.lt(w.tolist(), float(c)), s)
    np.testing.assert_array_equal(got, (c - acc).astype(np.float64))


def test_norm_predicate_pythagorean_points():
    """Region predicates of Sec. VII-A at points whose distances are exact integers
    (3-4-5 and 5-12-13 triangles), so every float32 step is exact: inside = r - dist,
    outside = dist - r.  A zero scale drops its dimension."""
    g = (1.0, 2.0, 0.0)
    pts = np.array([[[4.0, 6.0, 7.0], [1.0, 2.0, -3.0], [6.0, 14.0, 0.5], [-2.0, -2.0, 9.0]]], dtype=np.float32)
    dist = np.array([5.0, 0.0, 13.0, 5.0])
    inside = oracle.robustness(W.norm_lt([1, 1, 0], g, 2.5), pts)[0]
    np.testing.assert_array_equal(inside, (np.float32(2.5) - dist.astype(np.float32)).astype(np.float64))
    outside = oracle.robustness(W.norm_gt([1, 1, 0], g, 2.5), pts)[0]
    np.testing.assert_array_equal(outside, -inside)
    # scales: s = (2, 2, 0) doubles every distance
    np.testing.assert_array_equal(oracle.robustness(W.norm_gt([2, 2, 0], g, 0.0), pts)[0], 2 * dist)


def test_norm_predicate_gradient_closed_form():
    """d(r - ||x - g||)/dx = -(x - g)/||x - g|| (the unit vector, here (3/5, 4/5)), and the
    subgradient 0 at the centre; the scale enters squared: s_d^2 (x_d - g_d) / ||.||."""
    pts = np.array([[[4.0, 6.0], [1.0, 2.0]]], dtype=np.float32)
    g, _ = oracle.robustness_grad(W.norm_lt([1, 1], [1.0, 2.0], 0.3), pts, np.ones((1, 2)))
    np.testing.assert_allclose(g[0], [[-0.6, -0.8], [0.0, 0.0]], rtol=0, atol=1e-15)
    g, _ = oracle.robustness_grad(W.norm_gt([2, 1], [1.0, 2.0], 0.3), pts, np.ones((1, 2)))
    n = math.sqrt(36 + 16)
    np.testing.assert_allclose(g[0], [[4 * 3 / n, 4 / n], [0.0, 0.0]], rtol=1e-6)


def test_reach_avoid_straight_line():
    """Eventually inside a goal disc and always outside an obstacle disc along x_t = (t/10, 0):
    the closest approach to the goal (1, 0) is at t = 10 (margin r_g), to the obstacle
    (0.5, 0.5) at t = 5 (distance 0.5), so rho_0 = min(r_g, 0.5 - r_o)."""
    T = 21
    xs = np.zeros((1, T, 2), dtype=np.float32)
    xs[0, :, 0] = np.arange(T, dtype=np.float32) / np.float32(10)
    reach = W.Eventually(0, T - 1, W.norm_lt([1, 1], [1.0, 0.0], 0.3))
    avoid = W.Always(0, T - 1, W.norm_gt([1, 1], [0.5, 0.5], 0.3))
    np.testing.assert_allclose(oracle.robustness(reach, xs)[0, 0], 0.3, atol=1e-6)
    np.testing.assert_allclose(oracle.robustness(avoid, xs)[0, 0], 0.2, atol=1e-6)
    np.testing.assert_allclose(oracle.robustness(W.And(reach, avoid), xs)[0, 0], 0.2, atol=1e-6)
    # the hard gradient of rho_0 lands on the obstacle's closest sample: (x_5 - o)/|x_5 - o| = (0, -1)
    gout = np.zeros((1, T)); gout[0, 0] = 1.0
    g, _ = oracle.robustness_grad(W.And(reach, avoid), xs, gout)
    want = np.zeros((T, 2)); want[5] = [0.0, -1.0]
    np.testing.assert_allclose(g[0], want, atol=1e-6)


def test_ragged_equals_dense():
    rng = np.random.default_rng(12)
    s = rng.normal(size=(3, 50, 3)).astype(np.float32)
    f = W.config1_formula()
    dense = oracle.robustness(f, s)
    off = np.arange(4, dtype=np.int64) * 50
    np.testing.assert_array_equal(oracle.robustness(f, s.reshape(150, 3), offsets=off), dense.reshape(-1))


# ------------------------------------------------------------------ gradients
def _fd(fun, x, h=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp = x.copy(); xp[i] += h
        xm = x.copy(); xm[i] -= h
        g[i] = (fun(xp) - fun(xm)) / (2 * h)
    return g


GRAD_FORMULAS = [
    ("c0", W.config0_formula(), 2),
    ("c1", W.Or(W.Always(0, 5, W.Until(1, 4, W.gt([1, 0, 0], 0.0), W.lt([0, 1, 1], 0.2))),
                W.Eventually(0, 7, W.gt([0, 0, 1], 0.3))), 3),
    ("untilpad", W.Until(0, 3, W.Eventually(1, 2, W.gt([1, 0], 0.0)), W.lt([0, 1], 0.1), pad=0.4), 2),
    ("alw_or", W.Always(2, 6, W.Or(W.gt([1, -1], 0.0), W.Not(W.lt([0.5, 1], 0.2)))), 2),
    ("reach_avoid", W.And(W.Eventually(0, 6, W.norm_lt([1, 1], [0.5, -0.2], 0.8)),
                          W.Always(0, 9, W.norm_gt([1, 0.5], [-0.3, 0.4], 0.5))), 2),
]


@pytest.mark.parametrize("name,f,D", GRAD_FORMULAS, ids=[g[0] for g in GRAD_FORMULAS])
@pytest.mark.parametrize("mode,tau", [(HARD, 1.0), (SMOOTH, 2.0)])
def test_gradient_finite_differences(name, f, D, mode, tau):
    """FP64 central differences (h = 1e-6) at tie-free random points."""
    rng = np.random.default_rng(13)
    T = 14
    s = rng.normal(size=(1, T, D))
    gout = rng.normal(size=(1, T))
    g, _ = oracle.robustness_grad(f, s, gout, mode=mode, tau=tau, exact=True)
    loss = lambda x: float((oracle.robustness(f, x, mode=mode, tau=tau, exact=True) * gout).sum())  # noqa: E731
    fd = _fd(loss, s)
    np.testing.assert_allclose(g, fd, rtol=1e-6, atol=1e-6 * max(1.0, np.abs(g).max()))


@pytest.mark.parametrize("name,f,D", GRAD_FORMULAS, ids=[g[0] for g in GRAD_FORMULAS])
@pytest.mark.parametrize("hard", [True, False])
def test_gradient_matches_autograd_of_masking(name, f, D, hard):
    rng = np.random.default_rng(14)
    T = 17
    s = rng.normal(size=(T, D)).astype(np.float32)
    gout = rng.normal(size=(T,))
    tau = 1.3
    xt = torch.tensor(s, dtype=torch.float64, requires_grad=True)
    y = mr.evaluate(f, xt, hard=hard, tau=tau)
    (y * torch.tensor(gout)).sum().backward()
    g, _ = oracle.robustness_grad(f, s[None], gout[None], mode=HARD if hard else SMOOTH, tau=tau, exact=True)
    np.testing.assert_allclose(g[0], xt.grad.numpy(), rtol=1e-9, atol=1e-9)


def test_hard_tie_rules():
    """Reading R5 on hand-worked cases."""
    # window max: the earliest of the tied maxima takes the gradient
    s = one([1, 3, 3, 0])
    g, _ = oracle.robustness_grad(W.Eventually(0, 2, x_pred()), s, np.array([[1.0, 0, 0, 0]]))
    np.testing.assert_array_equal(g[0, :, 0], [0, 1, 0, 0])
    # And: the left operand wins a tie
    s2 = np.array([[[2.0, 2.0]]], dtype=np.float32)
    g, _ = oracle.robustness_grad(W.And(W.gt([1, 0], 0), W.gt([0, 1], 0)), s2, np.array([[1.0]]))
    np.testing.assert_array_equal(g[0, 0], [1, 0])
    # Until, phi=[5,1,4], psi=[0,1,9] over [0,2]: z = [0, 1, 1] -> earliest i* = 1;
    # min(P=1, psi=1) tie -> P wins -> earliest argmin of phi over [0,1] = index 1 (phi)
    s3 = np.array([[[5, 0], [1, 1], [4, 9]]], dtype=np.float32)
    g, _ = oracle.robustness_grad(W.Until(0, 2, W.gt([1, 0], 0), W.gt([0, 1], 0)), s3, np.array([[1.0, 0, 0]]))
    np.testing.assert_array_equal(g[0], [[0, 0], [1, 0], [0, 0]])
    # Until, phi=[1,1,4], psi=[0,0,9] over [0,2]: z = [0, 0, 1] -> i* = 2; P = 1 < 9 wins;
    # the running minimum P is reached first at index 0 (tied with index 1) -> phi[0]
    s4 = np.array([[[1, 0], [1, 0], [4, 9]]], dtype=np.float32)
    g, _ = oracle.robustness_grad(W.Until(0, 2, W.gt([1, 0], 0), W.gt([0, 1], 0)), s4, np.array([[1.0, 0, 0]]))
    np.testing.assert_array_equal(g[0], [[1, 0], [0, 0], [0, 0]])
    # Until, phi=[9,9,9], psi=[2,5,5] over [0,2]: z = [2,5,5] -> earliest maximiser i* = 1 (psi)
    s5 = np.array([[[9, 2], [9, 5], [9, 5]]], dtype=np.float32)
    g, _ = oracle.robustness_grad(W.Until(0, 2, W.gt([1, 0], 0), W.gt([0, 1], 0)), s5, np.array([[1.0, 0, 0]]))
    np.testing.assert_array_equal(g[0], [[0, 0], [0, 1], [0, 0]])
    # pad reads map to the last sample
    g, _ = oracle.robustness_grad(W.Eventually(2, 5, x_pred()), one([0, 1, 2]), np.array([[0.0, 1.0, 1.0]]))
    np.testing.assert_array_equal(g[0, :, 0], [0, 0, 2])


def test_smooth_mask_gradients_fd():
    """Gradients of the sigmoid-masked windows (Sec. VI) w.r.t. the signal and both bounds."""
    rng = np.random.default_rng(15)
    T = 30
    s = rng.normal(size=(2, T, 1))
    gout = rng.normal(size=(2, T))
    bounds = np.array([[[3.3, 9.6]], [[0.4, 17.2]]])
    for op in (W.EventuallySm, W.AlwaysSm):
        f = op(30, 40, x_pred(), slot=0)
        kw = dict(mode=SMOOTH, tau=2.0, mask_c=1.5, mask_eps=1e-3, exact=True)
        g, gb = oracle.robustness_grad(f, s, gout, bounds=bounds, **kw)
        loss_b = lambda bb: float((oracle.robustness(f, s, bounds=bb, **kw) * gout).sum())  # noqa: E731
        loss_s = lambda x: float((oracle.robustness(f, x, bounds=bounds, **kw) * gout).sum())  # noqa: E731
        np.testing.assert_allclose(gb, _fd(loss_b, bounds), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(g, _fd(loss_s, s), rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------------ softmax-weighted mode (R17)
SOFTMAX = oracle.SOFTMAX


def test_softmax_worked_values():
    """Hand-computed: at tau = ln 2 the weights of {0, 1} are {1, 2} for the max (value 2/3)
    and {1, 1/2} for the min (value 1/3); a window that reads past the end counts the last
    sample once per read (the multiset {1, 1, 1})."""
    s = one([0.0, 1.0])
    tau = math.log(2.0)
    ev = oracle.robustness(W.Eventually(0, 1, x_pred()), s, mode=SOFTMAX, tau=tau)[0]
    np.testing.assert_allclose(ev, [2 / 3, 1.0], rtol=1e-14)
    al = oracle.robustness(W.Always(0, 1, x_pred()), s, mode=SOFTMAX, tau=tau)[0]
    np.testing.assert_allclose(al, [1 / 3, 1.0], rtol=1e-14)
    s3 = one([0.0, 1.0, -1.0])
    ev3 = oracle.robustness(W.Eventually(0, 2, x_pred()), s3, mode=SOFTMAX, tau=tau)[0]
    # t = 0: {0, 1, -1} -> weights {1, 2, 1/2}; t = 2: {-1, -1, -1}
    np.testing.assert_allclose(ev3[[0, 2]], [(0 + 2 - 0.5) / 3.5, -1.0], rtol=1e-14)


def test_softmax_limits():
    """tau -> 0: the arithmetic mean of the window's multiset (pads included); tau -> inf:
    the hard value (well-separated samples)."""
    rng = np.random.default_rng(30)
    T = 12
    x = rng.permutation(T).astype(np.float32)      # distinct integers
    f = W.Eventually(2, 5, x_pred())
    lo = oracle.robustness(f, one(x), mode=SOFTMAX, tau=1e-7)[0]
    ext = np.concatenate([x, np.full(5, x[-1])]).astype(np.float64)
    mean = np.array([ext[t + 2:t + 6].mean() for t in range(T)])
    np.testing.assert_allclose(lo, mean, rtol=0, atol=1e-5)
    hi = oracle.robustness(f, one(x), mode=SOFTMAX, tau=60.0)[0]
    hard = oracle.robustness(f, one(x))[0]
    np.testing.assert_allclose(hi, hard, rtol=0, atol=1e-20 + 4 * 2 * math.exp(-60.0))


@pytest.mark.parametrize("op", ["eventually", "always"])
@pytest.mark.parametrize("pad", [None, -3.0])
def test_softmax_windows_match_masking(op, pad):
    rng = np.random.default_rng(31)
    for T in range(1, 8):
        for s in _tiny_signals(rng, T, n=2):
            xt = torch.tensor(s, dtype=torch.float64)
            for a in range(0, T + 1):
                for b in list(range(a, T + 2)) + [math.inf]:
                    f = (op, (float(a), float(b), None, pad), x_pred())
                    got = oracle.robustness(f, one(s), mode=SOFTMAX, tau=1.3)[0]
                    want = mr.eventually_always(xt, a, b, pad, op, None, 1.3).numpy()
                    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("pad", [None, 1.0])
def test_softmax_until_matches_masking(pad):
    rng = np.random.default_rng(32)
    for T in range(1, 7):
        for _ in range(2):
            s = rng.normal(size=(T, 2)).astype(np.float32)
            xt = torch.tensor(s, dtype=torch.float64)
            for a in range(0, T + 1):
                for b in list(range(a, T + 2)) + [math.inf]:
                    f = W.Until(a, b, W.gt([1, 0], 0.0), W.gt([0, 1], 0.0), pad=pad)
                    got = oracle.robustness(f, s[None], mode=SOFTMAX, tau=1.7)[0]
                    want = mr.until(xt[:, 0], xt[:, 1], a, b, pad, None, 1.7).numpy()
                    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-11)


def test_softmax_nested_and_duality():
    """Nested formulas against the masking construction; Always phi = -Eventually(not phi);
    unlike logsumexp, the softmax-weighted window is not the nesting of two-term operators
    (Sec. IV-D): Eventually_[0,2] p differs from p or (p one step later) or (two steps later)."""
    rng = np.random.default_rng(33)
    for f in [W.config0_formula(), W.config1_formula()] + W.table3_formulas(D=2, I=(1, 4))[:5]:
        D = 3 if f == W.config1_formula() else 2
        s = rng.normal(size=(17, D)).astype(np.float32)
        got = oracle.robustness(f, s[None], mode=SOFTMAX, tau=1.5, exact=True)[0]
        want = mr.evaluate(f, torch.tensor(s, dtype=torch.float64), hard=None, tau=1.5).numpy()
        np.testing.assert_allclose(got, want, rtol=1e-10, atol=1e-10)
    s = rng.normal(size=(1, 20, 1)).astype(np.float32)
    al = oracle.robustness(W.Always(2, 6, x_pred()), s, mode=SOFTMAX, tau=2.0)
    ev = oracle.robustness(W.Not(W.Eventually(2, 6, W.Not(x_pred()))), s, mode=SOFTMAX, tau=2.0)
    np.testing.assert_allclose(al, ev, rtol=1e-13, atol=1e-13)
    flat = oracle.robustness(W.Eventually(0, 2, x_pred()), s, mode=SOFTMAX, tau=2.0)[0, :10]
    nest = oracle.robustness(W.Or(x_pred(), W.Eventually(1, 2, x_pred())), s, mode=SOFTMAX, tau=2.0)[0, :10]
    assert np.abs(flat - nest).max() > 1e-3
    flat_l = oracle.robustness(W.Eventually(0, 2, x_pred()), s, mode=SMOOTH, tau=2.0)[0, :10]
    nest_l = oracle.robustness(W.Or(x_pred(), W.Eventually(1, 2, x_pred())), s, mode=SMOOTH, tau=2.0)[0, :10]
    np.testing.assert_allclose(flat_l, nest_l, rtol=1e-12)


@pytest.mark.parametrize("name,f,D", GRAD_FORMULAS, ids=[g[0] for g in GRAD_FORMULAS])
def test_softmax_gradients(name, f, D):
    """FP64 central differences, and torch autograd of the masking construction."""
    rng = np.random.default_rng(34)
    T = 13
    s = rng.normal(size=(1, T, D))
    gout = rng.normal(size=(1, T))
    g, _ = oracle.robustness_grad(f, s, gout, mode=SOFTMAX, tau=1.2, exact=True)
    loss = lambda x: float((oracle.robustness(f, x, mode=SOFTMAX, tau=1.2, exact=True) * gout).sum())  # noqa: E731
    np.testing.assert_allclose(g, _fd(loss, s), rtol=1e-6, atol=1e-6 * max(1.0, np.abs(g).max()))
    xt = torch.tensor(s[0], dtype=torch.float64, requires_grad=True)
    (mr.evaluate(f, xt, hard=None, tau=1.2) * torch.tensor(gout[0])).sum().backward()
    np.testing.assert_allclose(g[0], xt.grad.numpy(), rtol=1e-9, atol=1e-9)


def test_softmax_smooth_mask_gradients_fd():
    rng = np.random.default_rng(35)
    T = 30
    s = rng.normal(size=(2, T, 1))
    gout = rng.normal(size=(2, T))
    bounds = np.array([[[3.3, 9.6]], [[0.4, 17.2]]])
    for op in (W.EventuallySm, W.AlwaysSm):
        f = op(30, 40, x_pred(), slot=0)
        kw = dict(mode=SOFTMAX, tau=2.0, mask_c=1.5, mask_eps=1e-3, exact=True)
        g, gb = oracle.robustness_grad(f, s, gout, bounds=bounds, **kw)
        loss_b = lambda bb: float((oracle.robustness(f, s, bounds=bb, **kw) * gout).sum())  # noqa: E731
        loss_s = lambda x: float((oracle.robustness(f, x, bounds=bounds, **kw) * gout).sum())  # noqa: E731
        np.testing.assert_allclose(gb, _fd(loss_b, bounds), rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(g, _fd(loss_s, s), rtol=1e-6, atol=1e-7)


# ------------------------------------------------------------------ Until over a masked interval (R20)
def test_until_sm_sharp_mask_reduces_to_until():
    """With a sharp mask (c = 50) and bounds (3.3, 9.6) the support is {4, ..., 9} with weights
    1 - eps up to e^-15: hard mode equals the Until over [4, 9] exactly, logsumexp mode equals it
    plus log(1 - eps) / tau, and the softmax-weighted mode (equal weights cancel) equals it."""
    rng = np.random.default_rng(40)
    s = rng.normal(size=(3, 30, 2)).astype(np.float32)
    phi, psi = W.gt([1, 0], 0.0), W.gt([0, 1], 0.2)
    fsm = W.UntilSm(20, 20, phi, psi, slot=0)
    bounds = np.tile(np.array([[[3.3, 9.6]]], dtype=np.float32), (3, 1, 1))
    fu = W.Until(4, 9, phi, psi)
    kw = dict(mask_c=50.0, mask_eps=1e-3)
    np.testing.assert_array_equal(oracle.robustness(fsm, s, bounds=bounds, **kw), oracle.robustness(fu, s))
    tau = 2.0
    got = oracle.robustness(fsm, s, bounds=bounds, mode=SMOOTH, tau=tau, **kw)
    want = oracle.robustness(fu, s, mode=SMOOTH, tau=tau) + math.log(1 - 1e-3) / tau
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-6)
    got = oracle.robustness(fsm, s, bounds=bounds, mode=SOFTMAX, tau=tau, **kw)
    np.testing.assert_allclose(got, oracle.robustness(fu, s, mode=SOFTMAX, tau=tau), rtol=0, atol=1e-6)


@pytest.mark.parametrize("mode", [SMOOTH, SOFTMAX])
def test_until_sm_gradients_fd(mode):
    rng = np.random.default_rng(41)
    T = 24
    s = rng.normal(size=(2, T, 2))
    gout = rng.normal(size=(2, T))
    bounds = np.array([[[2.3, 7.6]], [[0.4, 11.2]]])
    f = W.UntilSm(20, 20, W.gt([1, 0], 0.0), W.gt([0, 1], 0.1), slot=0)
    kw = dict(mode=mode, tau=1.5, mask_c=1.5, mask_eps=1e-3, exact=True)
    g, gb = oracle.robustness_grad(f, s, gout, bounds=bounds, **kw)
    loss_b = lambda bb: float((oracle.robustness(f, s, bounds=bb, **kw) * gout).sum())  # noqa: E731
    loss_s = lambda x: float((oracle.robustness(f, x, bounds=bounds, **kw) * gout).sum())  # noqa: E731
    np.testing.assert_allclose(gb, _fd(loss_b, bounds), rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(g, _fd(loss_s, s), rtol=1e-6, atol=1e-7)


def test_until_sm_hard_gradient_is_one_hot():
    rng = np.random.default_rng(42)
    s = rng.normal(size=(1, 25, 2))
    f = W.UntilSm(20, 20, W.gt([1, 0], 0.0), W.gt([0, 1], 0.1), slot=0)
    bounds = np.array([[[2.3, 7.6]]])
    for t in (0, 5, 24):
        gout = np.zeros((1, 25)); gout[0, t] = 1.0
        g, gb = oracle.robustness_grad(f, s, gout, bounds=bounds, mask_c=50.0)
        assert np.count_nonzero(g) == 1 and np.abs(g).sum() == 1.0 and np.all(gb == 0)
