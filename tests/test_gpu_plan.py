"""GPU checks of the planning helpers (include/stl_plan.h) and of the batched reach/avoid solver.

- rollout and the fused rollout-adjoint + Adam step against float64 numpy written from the
  dynamics x_{t+1} = x_t + dt tanh(u_t) (the numpy adjoint is itself checked against central
  differences);
- the solved/active bookkeeping;
- the BF16 tensor-core GEMM in all four transpose combinations, with bias / ReLU / bf16
  output, against float32 torch matmuls of the same bf16 values;
- the MLP forward against a torch evaluation with the same bf16 roundings, and its training
  reducing the loss;
- the solver: every problem it reports solved has oracle hard robustness >= 0 at t = 0 on the
  final trajectory, and the rest are < 0.
"""
import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

DT = 0.1


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


def call(name, *args):
    from paper_2501_04194_gb300.binding import plan_call
    plan_call(name, *args)


def stream():
    return torch.cuda.current_stream().cuda_stream


def np_rollout(u):
    return np.cumsum(DT * np.tanh(u.astype(np.float64)), axis=1)


def np_rollout_adjoint(u, xbar):
    """dL/du for L = sum xbar * x(u): dt (1 - tanh^2 u_t) sum_{s >= t} xbar_s."""
    suf = np.cumsum(xbar[:, ::-1].astype(np.float64), axis=1)[:, ::-1]
    return DT * (1 - np.tanh(u.astype(np.float64)) ** 2) * suf


def test_numpy_adjoint_matches_finite_differences():
    rng = np.random.default_rng(0)
    u = rng.normal(size=(2, 9, 2))
    xbar = rng.normal(size=(2, 9, 2))
    g = np_rollout_adjoint(u, xbar)
    h = 1e-6
    for idx in np.ndindex(u.shape):
        up, um = u.copy(), u.copy()
        up[idx] += h
        um[idx] -= h
        fd = ((np_rollout(up) - np_rollout(um)) * xbar).sum() / (2 * h)
        assert abs(fd - g[idx]) < 1e-7


@pytest.mark.parametrize("T", [1, 31, 200, 1000])
def test_rollout(stl, T):
    rng = np.random.default_rng(T)
    u = (2 * rng.normal(size=(37, T, 2))).astype(np.float32)
    ud = torch.from_numpy(u).cuda()
    x = torch.full_like(ud, float("nan"))
    call("stl_rollout", ud.data_ptr(), 37, T, DT, x.data_ptr(), stream())
    np.testing.assert_allclose(x.cpu().numpy(), np_rollout(u), rtol=1e-5, atol=1e-5)


def test_plan_adam_step(stl):
    rng = np.random.default_rng(3)
    B, T, lr, b1, b2, eps = 9, 200, 0.05, 0.9, 0.999, 1e-8
    u = rng.normal(size=(B, T, 2)).astype(np.float32)
    m = (0.01 * rng.normal(size=(B, T, 2))).astype(np.float32)
    v = (0.01 * rng.random(size=(B, T, 2))).astype(np.float32)
    xbar = rng.normal(size=(B, T, 2)).astype(np.float32)
    active = np.array([1, 0, 1, 1, 0, 1, 1, 1, 0], dtype=np.int32)
    step = 3
    d = {k: torch.from_numpy(a.copy()).cuda() for k, a in dict(u=u, m=m, v=v, xbar=xbar).items()}
    x = torch.from_numpy(np_rollout(u).astype(np.float32)).cuda()
    act = torch.from_numpy(active).cuda()
    call("stl_plan_adam_step", d["u"].data_ptr(), d["m"].data_ptr(), d["v"].data_ptr(), d["xbar"].data_ptr(),
         act.data_ptr(), B, T, DT, lr, b1, b2, eps, step, x.data_ptr(), stream())
    g = np_rollout_adjoint(u, xbar)
    m2 = b1 * m + (1 - b1) * g
    v2 = b2 * v + (1 - b2) * g * g
    u2 = u - lr * (m2 / (1 - b1 ** step)) / (np.sqrt(v2 / (1 - b2 ** step)) + eps)
    keep = active[:, None, None] == 0
    u2 = np.where(keep, u, u2)
    np.testing.assert_allclose(d["u"].cpu().numpy(), u2, rtol=1e-5, atol=2e-6)
    np.testing.assert_allclose(d["m"].cpu().numpy(), np.where(keep, m, m2), rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(d["v"].cpu().numpy(), np.where(keep, v, v2), rtol=1e-4, atol=1e-7)
    np.testing.assert_allclose(x.cpu().numpy(), np_rollout(np.where(keep, u, d["u"].cpu().numpy())), rtol=1e-5,
                               atol=1e-5)


def test_plan_check(stl):
    B, T = 70, 5
    rho = torch.full((B * T,), -1.0, device="cuda")
    rho[0::T][::3] = 0.5
    rho[T * 7] = 0.0
    active = torch.ones(B, dtype=torch.int32, device="cuda")
    active[1] = 0
    solved = torch.full((B,), -1, dtype=torch.int32, device="cuda")
    gout = torch.full((B * T,), 7.0, device="cuda")
    n_active = torch.zeros(1, dtype=torch.int32, device="cuda")
    call("stl_plan_check", rho.data_ptr(), active.data_ptr(), solved.data_ptr(), 12, gout.data_ptr(), B, T,
         n_active.data_ptr(), stream())
    r0 = rho[0::T].cpu().numpy()
    was = np.ones(B, dtype=bool)
    was[1] = False
    now_solved = was & (r0 >= 0)
    a = active.cpu().numpy()
    assert np.array_equal(a, (was & ~now_solved).astype(np.int32))
    s = solved.cpu().numpy()
    assert np.all(s[now_solved] == 12) and np.all(s[~now_solved] == -1)
    go = gout.cpu().numpy().reshape(B, T)
    assert np.array_equal(go[:, 0], np.where(a == 1, -1.0, 0.0)) and np.all(go[:, 1:] == 7.0)
    assert int(n_active.item()) == int(a.sum())


def bf16(x):
    return torch.from_numpy(np.asarray(x, dtype=np.float32)).to(torch.bfloat16)


@pytest.mark.parametrize("ta,tb", [(0, 0), (1, 0), (0, 1), (1, 1)])
@pytest.mark.parametrize("M,N,K", [(70, 45, 33), (128, 256, 16), (5, 400, 256), (200, 136, 72), (4096, 256, 256)])
def test_gemm_bf16(stl, ta, tb, M, N, K):
    rng = np.random.default_rng(M + N + K + 2 * ta + tb)
    A = bf16(rng.normal(size=(K, M) if ta else (M, K)))
    Bm = bf16(rng.normal(size=(N, K) if tb else (K, N)))
    bias = torch.from_numpy(rng.normal(size=N).astype(np.float32)).cuda()
    Ad, Bd = A.cuda().view(torch.int16), Bm.cuda().view(torch.int16)
    ref = (A.float().T if ta else A.float()) @ (Bm.float().T if tb else Bm.float())
    for use_bias, relu in ((False, False), (True, True)):
        cf = torch.full((M, N), float("nan"), device="cuda")
        cb = torch.zeros((M, N), dtype=torch.int16, device="cuda")
        call("stl_gemm_bf16", Ad.data_ptr(), M if ta else K, ta, Bd.data_ptr(), K if tb else N, tb, M, N, K,
             bias.data_ptr() if use_bias else None, int(relu), cf.data_ptr(), cb.data_ptr(), N, stream())
        want = ref + (bias.cpu() if use_bias else 0)
        if relu:
            want = want.clamp_min(0)
        got = cf.cpu()
        tol = 1e-5 * K * float(A.float().abs().max() * Bm.float().abs().max())
        assert float((got - want).abs().max()) <= tol
        gb = cb.cpu().view(torch.bfloat16).float()
        assert torch.equal(gb, got.to(torch.bfloat16).float())


def test_mlp_forward_matches_torch(stl):
    from paper_2501_04194_gb300.planning import WarmStartMLP
    net = WarmStartMLP(T=200, seed=1)
    rng = np.random.default_rng(5)
    X = torch.from_numpy(rng.normal(size=(37, 16)).astype(np.float32)).cuda()
    got = net.forward(X).cpu()
    a = X.cpu().to(torch.bfloat16).float()
    for l, (w, b) in enumerate(zip(net.W, net.b)):
        z = a @ w.cpu().to(torch.bfloat16).float() + b.cpu()
        a = z.clamp_min(0).to(torch.bfloat16).float() if l < len(net.W) - 1 else z
    err = float((got - a).abs().max() / a.abs().max())
    assert err < 2e-2   # bf16 activations rounded at slightly different points of equal sums


def test_mlp_training_reduces_loss(stl):
    from paper_2501_04194_gb300.planning import WarmStartMLP
    rng = np.random.default_rng(6)
    n = 2048
    X = rng.normal(size=(n, 16)).astype(np.float32)
    P = rng.normal(size=(16, 400)).astype(np.float32) / 4
    Y = np.tanh(X @ P).astype(np.float32)
    net = WarmStartMLP(T=200, seed=2)
    hist = net.fit(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), epochs=8, batch=256, lr=1e-3)
    assert hist[-1] < 0.5 * hist[0], hist


def test_solver_decisions_match_the_oracle(stl):
    from paper_2501_04194_gb300.planning import ReachAvoidSolver
    probs = W.config4_problems(48, seed=11)
    forms = [W.reach_avoid_formula(g, o, r) for g, o, r in probs]
    solver = ReachAvoidSolver(forms, T=200, tau=20.0)
    u0 = torch.from_numpy(W.random_controls(48, seed=3, scale=0.1)).cuda()
    solved, iters, ms = solver.solve(u0, max_iters=300, lr=0.05, check_every=10)
    assert (solved >= 0).mean() > 0.5
    x = solver.x.cpu().numpy().reshape(48, 200, 2)
    for b in range(48):
        rho0 = oracle.robustness(forms[b], x[b:b + 1])[0, 0]
        assert (rho0 >= 0) == (solved[b] >= 0), (b, rho0, solved[b])


def test_warm_start_pipeline_small(stl):
    """Train on 8192 solved problems, evaluate on 1024 held-out ones: the warm start keeps the
    success rate and needs no more Adam steps (median) than the cold start; warm-start
    solutions are confirmed by the oracle's hard robustness on a sample."""
    from paper_2501_04194_gb300 import planning as PL
    probs = W.config4_problems(8192 + 1024, seed=21)
    forms = [W.reach_avoid_formula(g, o, r) for g, o, r in probs]
    mlp, frac, hist = PL.train_warm_start(probs[:8192], forms[:8192], max_iters=200, epochs=10)
    assert frac > 0.9 and hist[-1] < hist[0]
    res = PL.warm_vs_cold(mlp, probs[8192:], forms[8192:], max_iters=200)
    assert res["warm"]["success"] >= res["cold"]["success"] - 0.02
    assert res["warm"]["median_steps"] <= res["cold"]["median_steps"]
    # oracle check of warm-start trajectories that were solved at step 0
    feats = torch.from_numpy(PL.problem_features(probs[8192:8192 + 64])).cuda()
    u0 = mlp.forward(feats).reshape(64, 200, 2)
    solver = PL.ReachAvoidSolver(forms[8192:8192 + 64])
    solver.rollout(u0.reshape(64 * 200, 2).contiguous(), solver.x)
    rho = solver.hard_robustness().cpu().numpy().reshape(64, 200)
    x = solver.x.cpu().numpy().reshape(64, 200, 2)
    for b in range(0, 64, 4):
        ref = oracle.robustness(forms[8192 + b], x[b:b + 1])[0]
        np.testing.assert_array_equal(rho[b], ref.astype(np.float32))


def np_trajopt_step(u, mu, vu, th, mth, vth, xbar, gb, gam, T, dt, start, umax, inom, lr_u, lr_th, step):
    """The update of stl_trajopt_step written from its definition, in float64."""
    b1, b2, eps = 0.9, 0.999, 1e-8
    c1, c2 = 1 / (1 - b1 ** step), 1 / (1 - b2 ** step)
    suf = np.cumsum(xbar[:, ::-1].astype(np.float64), axis=1)[:, ::-1]
    nrm = np.linalg.norm(u.astype(np.float64), axis=2, keepdims=True)
    g3, g4 = gam[:, 2, None, None] / T, gam[:, 3, None, None] / T
    gu = dt * suf + np.where(nrm > umax, g3 / np.maximum(nrm, 1e-30), 0) * u + 2 * g4 * u
    mu2 = b1 * mu + (1 - b1) * gu
    vu2 = b2 * vu + (1 - b2) * gu * gu
    u2 = u - lr_u * mu2 * c1 / (np.sqrt(vu2 * c2) + eps)
    x2 = np.asarray(start)[None, None, :] + dt * np.cumsum(u2, axis=1)
    a, bb = 1 / (1 + np.exp(-th[:, 0])), 1 / (1 + np.exp(-th[:, 1]))
    e = np.exp(2 * (inom - bb + a))
    gth = np.stack([(T * gb[:, 0, 0] + 2 * gam[:, 1] * e) * a * (1 - a),
                    (T * gb[:, 0, 1] - 2 * gam[:, 1] * e) * bb * (1 - bb)], axis=1)
    mth2 = b1 * mth + (1 - b1) * gth
    vth2 = b2 * vth + (1 - b2) * gth * gth
    th2 = th - lr_th * mth2 * c1 / (np.sqrt(vth2 * c2) + eps)
    return u2, mu2, vu2, x2, th2


def test_trajopt_step(stl):
    rng = np.random.default_rng(8)
    B, T, dt, umax, inom, lr_u, lr_th, step = 6, 51, 0.1, 2.0, 0.2, 0.05, 0.02, 4
    u = (1.5 * rng.normal(size=(B, T, 2))).astype(np.float32)
    mu = (0.01 * rng.normal(size=(B, T, 2))).astype(np.float32)
    vu = (0.01 * rng.random(size=(B, T, 2))).astype(np.float32)
    xbar = rng.normal(size=(B, T, 2)).astype(np.float32)
    gb = (0.1 * rng.normal(size=(B, 1, 2))).astype(np.float32)
    gam = rng.uniform(0.1, 2.0, size=(B, 4)).astype(np.float32)
    th = np.stack([np.full(B, -1.5), np.full(B, 1.2)], axis=1).astype(np.float32)
    mth = (0.01 * rng.normal(size=(B, 2))).astype(np.float32)
    vth = (0.01 * rng.random(size=(B, 2))).astype(np.float32)
    d = {k: torch.from_numpy(np.ascontiguousarray(v)).cuda() for k, v in
         dict(u=u, mu=mu, vu=vu, xbar=xbar, gb=gb, gam=gam, th=th, mth=mth, vth=vth).items()}
    x = torch.zeros((B, T, 2), device="cuda")
    bounds = torch.zeros((B, 1, 2), device="cuda")
    call("stl_trajopt_step", d["u"].data_ptr(), d["mu"].data_ptr(), d["vu"].data_ptr(), d["th"].data_ptr(),
         d["mth"].data_ptr(), d["vth"].data_ptr(), d["xbar"].data_ptr(), d["gb"].data_ptr(), d["gam"].data_ptr(),
         B, T, 1, 0, dt, 0.5, -0.25, umax, inom, lr_u, lr_th, step, x.data_ptr(), bounds.data_ptr(), stream())
    u2, mu2, vu2, x2, th2 = np_trajopt_step(u, mu, vu, th, mth, vth, xbar, gb, gam, T, dt, (0.5, -0.25), umax, inom,
                                           lr_u, lr_th, step)
    np.testing.assert_allclose(d["u"].cpu().numpy(), u2, rtol=1e-5, atol=2e-6)
    np.testing.assert_allclose(d["mu"].cpu().numpy(), mu2, rtol=1e-4, atol=1e-6)
    np.testing.assert_allclose(x.cpu().numpy(), x2, rtol=1e-5, atol=2e-5)
    np.testing.assert_allclose(d["th"].cpu().numpy(), th2, rtol=1e-5, atol=1e-6)
    ab = 1 / (1 + np.exp(-th2.astype(np.float64)))
    np.testing.assert_allclose(bounds.cpu().numpy()[:, 0, :], T * ab, rtol=1e-5)


def test_interval_trajopt_example(stl):
    """The trajectory-planning example with a learnable interval (T = 51, coefficients
    (1.1, 0.05, 2, 0.5), (a, b) from (0.14, 0.82)) over a few coefficient settings at once: the
    interval grows past the nominal 0.2, the paper's setting ends within a small margin of
    satisfaction (the loss only sees the smooth robustness) and one of the settings satisfies
    the specification; the hard robustness of the final trajectories and bounds matches the
    oracle bit for bit."""
    from paper_2501_04194_gb300 import planning as PL
    T = 51
    form = PL.interval_trajopt_formula(T, (1.5, 1.0), 0.6, (3.0, 2.5), 0.3)
    gam = np.array([[1.1, 0.05, 2.0, 0.5], [1.1, 0.2, 2.0, 0.5], [2.0, 0.05, 2.0, 0.1]], dtype=np.float32)
    res = PL.interval_trajopt(form, gam, T=T, steps=1500)
    assert np.all(res["b"] - res["a"] > 0.2)
    assert res["rho_hard"][0] > -0.05 and np.any(res["rho_hard"] >= 0), res["rho_hard"]
    ref = oracle.robustness(form, res["x"], bounds=res["bounds"])[:, 0]
    np.testing.assert_array_equal(res["rho_hard"], ref.astype(np.float32))
