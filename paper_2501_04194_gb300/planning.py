"""Gradient-through-robustness trajectory optimisation and its learned warm start.

A batch of control-synthesis problems (one reach/avoid formula per problem, Sec. VII-A use of
the smooth robustness) is solved together: every iteration evaluates the hard robustness of
the current trajectories (one ragged launch), marks the problems whose robustness at t = 0 is
>= 0 as solved, back-propagates the smooth robustness at t = 0 of the others (one ragged
backward launch) and takes one Adam step on their controls through the rollout adjoint (one
fused kernel).  A small MLP with BF16 weights maps the problem parameters to a control
sequence that the same solver starts from.  Every step runs in libstl's kernels
(include/stl.h, include/stl_plan.h); torch only allocates device memory and names the stream.
"""
from __future__ import annotations

import numpy as np
import torch

from .binding import (Formula, FormulaSet, params, plan_call, robustness_ragged_backward_raw,
                      robustness_ragged_raw)

DT = 0.1
N_FEATURES = 16   # 11 problem parameters, zero-padded to one MMA k-step


def _p(t):
    return None if t is None else t.data_ptr()


def problem_features(problems) -> np.ndarray:
    """[n, 16] float32: goal / 3, obstacle centres / 3, radii, zero padding."""
    out = np.zeros((len(problems), N_FEATURES), dtype=np.float32)
    for i, (g, o, r) in enumerate(problems):
        o = np.asarray(o, dtype=np.float32).reshape(-1, 2)
        vals = np.concatenate([np.asarray(g, dtype=np.float32) / 3.0, o.reshape(-1) / 3.0,
                               np.asarray(r, dtype=np.float32)])
        out[i, :vals.size] = vals
    return out


class ReachAvoidSolver:
    """Batched Adam on the controls u [B, T, 2] of B problems, one formula per problem."""

    def __init__(self, formulas, T: int = 200, tau: float = 20.0, device="cuda"):
        self.B, self.T, self.dev = len(formulas), T, torch.device(device)
        self.fset = FormulaSet([Formula(f, D=2) for f in formulas])
        self.p_hard = params("hard")
        self.p_smooth = params("smooth", tau=tau)
        B, dev = self.B, self.dev
        nf = self.fset.prepare(B, T, self.p_hard, False)
        nb = self.fset.prepare(B, T, self.p_smooth, True)
        self.ws_f = torch.empty(nf // 4 + 1, dtype=torch.float32, device=dev)
        self.ws_b = torch.empty(nb // 4 + 1, dtype=torch.float32, device=dev)
        self.nf, self.nb = nf, nb
        self.offsets = torch.arange(B + 1, dtype=torch.int64, device=dev) * T
        self.fid = torch.arange(B, dtype=torch.int32, device=dev)
        z = lambda *s: torch.zeros(s, dtype=torch.float32, device=dev)  # noqa: E731
        self.u, self.m, self.v, self.x, self.xbar = (z(B * T, 2) for _ in range(5))
        self.rho = z(B * T)
        self.gout = z(B * T)
        self.active = torch.zeros(B, dtype=torch.int32, device=dev)
        self.solved = torch.zeros(B, dtype=torch.int32, device=dev)
        self.n_active = torch.zeros(1, dtype=torch.int32, device=dev)

    def _stream(self):
        return torch.cuda.current_stream(self.dev).cuda_stream

    def rollout(self, u, x):
        plan_call("stl_rollout", _p(u), self.B, self.T, DT, _p(x), self._stream())

    def hard_robustness(self):
        """Hard robustness traces [B*T] of the current trajectories."""
        robustness_ragged_raw(self.fset, _p(self.x), _p(self.offsets), _p(self.fid), None, self.B, None,
                              self.p_hard, _p(self.rho), _p(self.ws_f), self.nf, self._stream())
        return self.rho

    def solve(self, u0: torch.Tensor, max_iters: int = 600, lr: float = 0.05, check_every: int = 20,
              stop_frac: float = 1.0):
        """Run Adam from u0 [B, T, 2] until a fraction stop_frac of the problems (default: every
        problem) has hard robustness >= 0 at t = 0 or max_iters steps were taken.  Returns
        solved_iter (numpy [B]: Adam steps taken when the problem was first seen solved, -1 if
        never), the number of iterations run and the device time per iteration (ms)."""
        stop_active = int(np.floor((1.0 - stop_frac) * self.B + 1e-9))
        st = self._stream()
        self.u.copy_(u0.reshape(self.B * self.T, 2))
        self.m.zero_()
        self.v.zero_()
        self.gout.zero_()
        self.active.fill_(1)
        self.solved.fill_(-1)
        self.rollout(self.u, self.x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        it = 0
        while True:
            self.hard_robustness()
            check = it % check_every == 0 or it == max_iters
            if check:
                self.n_active.zero_()
            plan_call("stl_plan_check", _p(self.rho), _p(self.active), _p(self.solved), it, _p(self.gout), self.B,
                      self.T, _p(self.n_active) if check else None, st)
            if it == max_iters or (check and int(self.n_active.item()) <= stop_active):
                break
            robustness_ragged_backward_raw(self.fset, _p(self.x), _p(self.offsets), _p(self.fid), None, self.B, None,
                                           self.p_smooth, _p(self.gout), _p(self.xbar), None, _p(self.ws_b), self.nb,
                                           st)
            it += 1
            plan_call("stl_plan_adam_step", _p(self.u), _p(self.m), _p(self.v), _p(self.xbar), _p(self.active),
                      self.B, self.T, DT, lr, 0.9, 0.999, 1e-8, it, _p(self.x), st)
        e1.record()
        torch.cuda.synchronize(self.dev)
        ms = e0.elapsed_time(e1)
        return self.solved.cpu().numpy(), it, ms / max(it, 1)


class WarmStartMLP:
    """MLP 16 -> 256 -> 256 -> 256 -> 2T with ReLU, BF16 weights and activations, FP32
    accumulation and FP32 master weights (Adam).  Maps problem features to controls."""

    def __init__(self, T: int = 200, hidden: int = 256, seed: int = 0, device="cuda"):
        self.dev = torch.device(device)
        self.dims = [N_FEATURES, hidden, hidden, hidden, 2 * T]
        rng = np.random.default_rng(seed)
        self.W, self.b, self.Wb = [], [], []
        self.mW, self.vW, self.mb, self.vb = [], [], [], []
        for k, n in zip(self.dims[:-1], self.dims[1:]):
            w = (rng.normal(size=(k, n)) * np.sqrt(2.0 / k)).astype(np.float32)
            self.W.append(torch.from_numpy(w).to(self.dev))
            self.b.append(torch.zeros(n, dtype=torch.float32, device=self.dev))
            self.Wb.append(torch.empty((k, n), dtype=torch.int16, device=self.dev))
            for lst, shape in ((self.mW, (k, n)), (self.vW, (k, n)), (self.mb, (n,)), (self.vb, (n,))):
                lst.append(torch.zeros(shape, dtype=torch.float32, device=self.dev))
        for w, wb in zip(self.W, self.Wb):
            plan_call("stl_to_bf16", _p(w), w.numel(), _p(wb), self._stream())
        self.step = 0

    def _stream(self):
        return torch.cuda.current_stream(self.dev).cuda_stream

    def _gemm(self, a, lda, ta, b, ldb, tb, M, N, K, bias=None, relu=False, out_f32=None, out_bf16=None):
        plan_call("stl_gemm_bf16", _p(a), lda, int(ta), _p(b), ldb, int(tb), M, N, K, _p(bias), int(relu),
                  _p(out_f32), _p(out_bf16), N, self._stream())

    def forward(self, x_f32: torch.Tensor, keep: bool = False):
        """x [M, 16] float32 -> output [M, 2T] float32 (activations kept for backward if keep)."""
        M = x_f32.shape[0]
        a = torch.empty((M, N_FEATURES), dtype=torch.int16, device=self.dev)
        plan_call("stl_to_bf16", _p(x_f32), x_f32.numel(), _p(a), self._stream())
        acts = [a]
        out = None
        L = len(self.W)
        for l in range(L):
            K, N = self.dims[l], self.dims[l + 1]
            if l < L - 1:
                nxt = torch.empty((M, N), dtype=torch.int16, device=self.dev)
                self._gemm(acts[-1], K, False, self.Wb[l], N, False, M, N, K, bias=self.b[l], relu=True, out_bf16=nxt)
                acts.append(nxt)
            else:
                out = torch.empty((M, N), dtype=torch.float32, device=self.dev)
                self._gemm(acts[-1], K, False, self.Wb[l], N, False, M, N, K, bias=self.b[l], out_f32=out)
        if keep:
            self._acts = acts
        return out

    def train_step(self, x_f32: torch.Tensor, y: torch.Tensor, lr: float = 1e-3, loss_acc=None):
        """One Adam step on the mean squared error of forward(x) against y; the summed squared
        error is added to loss_acc (device float32 [1]) when given."""
        M = x_f32.shape[0]
        z = self.forward(x_f32, keep=True)
        L = len(self.W)
        st = self._stream()
        dz = torch.empty((M, self.dims[-1]), dtype=torch.int16, device=self.dev)
        plan_call("stl_mse_grad", _p(z), _p(y), z.numel(), 2.0 / z.numel(), _p(dz), _p(loss_acc), st)
        self.step += 1
        for l in range(L - 1, -1, -1):
            K, N = self.dims[l], self.dims[l + 1]
            a_prev = self._acts[l]
            gW = torch.empty((K, N), dtype=torch.float32, device=self.dev)
            gb = torch.empty(N, dtype=torch.float32, device=self.dev)
            self._gemm(a_prev, K, True, dz, N, False, K, N, M, out_f32=gW)      # a_prev^T dz
            plan_call("stl_colsum_bf16", _p(dz), M, N, _p(gb), st)
            if l > 0:
                da = torch.empty((M, K), dtype=torch.float32, device=self.dev)
                self._gemm(dz, N, False, self.Wb[l], N, True, M, K, N, out_f32=da)   # dz W^T
                dz = torch.empty((M, K), dtype=torch.int16, device=self.dev)
                plan_call("stl_relu_backward", _p(da), _p(a_prev), da.numel(), _p(dz), st)
            plan_call("stl_adam", _p(self.W[l]), _p(gW), _p(self.mW[l]), _p(self.vW[l]), gW.numel(), lr, 0.9, 0.999,
                      1e-8, self.step, _p(self.Wb[l]), st)
            plan_call("stl_adam", _p(self.b[l]), _p(gb), _p(self.mb[l]), _p(self.vb[l]), gb.numel(), lr, 0.9, 0.999,
                      1e-8, self.step, None, st)

    def fit(self, X: torch.Tensor, Y: torch.Tensor, epochs: int = 30, batch: int = 256, lr: float = 1e-3,
            seed: int = 0):
        """Minibatch Adam over (X [n, 16], Y [n, 2T]) float32 device tensors; returns the mean
        squared error of each epoch."""
        n = X.shape[0]
        rng = np.random.default_rng(seed)
        st = self._stream()
        hist = []
        xb = torch.empty((batch, X.shape[1]), dtype=torch.float32, device=self.dev)
        yb = torch.empty((batch, Y.shape[1]), dtype=torch.float32, device=self.dev)
        for _ in range(epochs):
            perm = torch.from_numpy(rng.permutation(n).astype(np.int64)).to(self.dev)
            tot = torch.zeros(1, dtype=torch.float32, device=self.dev)
            for s in range(0, n - batch + 1, batch):
                idx = perm[s:s + batch]
                plan_call("stl_gather_rows", _p(X), n, _p(idx), batch, X.shape[1], _p(xb), st)
                plan_call("stl_gather_rows", _p(Y), n, _p(idx), batch, Y.shape[1], _p(yb), st)
                self.train_step(xb, yb, lr, loss_acc=tot)
            hist.append(float(tot.item()) / (max(1, n // batch) * batch * Y.shape[1]))
        return hist


# ---------------------------------------------------------------- the warm-start pipeline
U_CLIP = 3.0   # controls are learned inside [-3, 3] (tanh(3) = 0.995 of the speed limit)


def solve_batches(formulas, u0_fn, batch: int = 4096, T: int = 200, tau: float = 20.0, max_iters: int = 300,
                  lr: float = 0.05, check_every: int = 10, device="cuda"):
    """Solve many problems in batches.  u0_fn(lo, hi) gives the starting controls [hi-lo, T, 2]
    (device float32) of problems lo..hi-1.  Returns (solved_iter [n], final controls [n, T, 2]
    on the host, ms per iteration of each batch)."""
    n = len(formulas)
    solved = np.full(n, -1, dtype=np.int64)
    u_out = np.zeros((n, T, 2), dtype=np.float32)
    ms_iter = []
    for lo in range(0, n, batch):
        hi = min(n, lo + batch)
        solver = ReachAvoidSolver(formulas[lo:hi], T=T, tau=tau, device=device)
        s, _, ms = solver.solve(u0_fn(lo, hi), max_iters=max_iters, lr=lr, check_every=check_every)
        solved[lo:hi] = s
        u_out[lo:hi] = solver.u.reshape(hi - lo, T, 2).cpu().numpy()
        ms_iter.append(ms)
    return solved, u_out, ms_iter


def train_warm_start(problems, formulas, T: int = 200, batch: int = 4096, max_iters: int = 300, lr: float = 0.05,
                     epochs: int = 30, seed: int = 0, device="cuda"):
    """Solve the training problems from a cold start, then fit the MLP to the solved controls.
    Returns (mlp, fraction solved, training-loss history)."""
    rng_u = np.random.default_rng(seed)
    dev = torch.device(device)

    def cold(lo, hi):
        return torch.from_numpy((0.1 * rng_u.normal(size=(hi - lo, T, 2))).astype(np.float32)).to(dev)

    solved, u, _ = solve_batches(formulas, cold, batch=batch, T=T, max_iters=max_iters, lr=lr, device=device)
    ok = solved >= 0
    X = torch.from_numpy(problem_features([p for p, k in zip(problems, ok) if k])).to(dev)
    Y = torch.from_numpy(np.clip(u[ok], -U_CLIP, U_CLIP).reshape(int(ok.sum()), 2 * T)).to(dev)
    mlp = WarmStartMLP(T=T, seed=seed, device=device)
    hist = mlp.fit(X, Y, epochs=epochs, batch=256, lr=1e-3, seed=seed)
    return mlp, float(ok.mean()), hist


def warm_vs_cold(mlp, problems, formulas, T: int = 200, batch: int = 4096, max_iters: int = 300, lr: float = 0.05,
                 seed: int = 1, device="cuda"):
    """Solve held-out problems from a cold start and from the MLP's warm start with the same
    solver; time to hard robustness >= 0 of a problem = its Adam steps x the batch's time per
    step (+ the MLP inference time per batch, warm start only)."""
    dev = torch.device(device)
    rng_u = np.random.default_rng(seed)
    feats = torch.from_numpy(problem_features(problems)).to(dev)
    inf_ms = []

    def cold(lo, hi):
        return torch.from_numpy((0.1 * rng_u.normal(size=(hi - lo, T, 2))).astype(np.float32)).to(dev)

    def warm(lo, hi):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = mlp.forward(feats[lo:hi].contiguous())
        e1.record()
        torch.cuda.synchronize(dev)
        inf_ms.append(e0.elapsed_time(e1))
        return out.reshape(hi - lo, T, 2)

    res = {}
    for name, fn in (("cold", cold), ("warm", warm)):
        solved, _, ms = solve_batches(formulas, fn, batch=batch, T=T, max_iters=max_iters, lr=lr, device=device)
        per_batch_ms = np.repeat(ms, [min(batch, len(formulas) - lo) for lo in range(0, len(formulas), batch)])
        t = solved * per_batch_ms
        if name == "warm":
            t = t + np.repeat(inf_ms, [min(batch, len(formulas) - lo) for lo in range(0, len(formulas), batch)])
        ok = solved >= 0
        res[name] = {"success": float(ok.mean()),
                     "median_steps": float(np.median(solved[ok])) if ok.any() else None,
                     "p90_steps": float(np.percentile(solved[ok], 90)) if ok.any() else None,
                     "median_ms": float(np.median(t[ok])) if ok.any() else None,
                     "p90_ms": float(np.percentile(t[ok], 90)) if ok.any() else None,
                     "ms_per_step": float(np.mean(ms)),
                     "solved_at_start": float((solved == 0).mean())}
    res["warm"]["mlp_inference_ms_per_batch"] = float(np.mean(inf_ms)) if inf_ms else None
    # measured, not modelled: host wall time from the start of each arm (the MLP inference
    # included for the warm start) until 99 % of a batch of problems is solved, with a check of
    # the solved count after every Adam step (one host synchronisation per step)
    import time as _time
    n0 = min(batch, len(formulas))
    solver = ReachAvoidSolver(formulas[:n0], T=T, device=device)
    for name in ("cold", "warm"):
        u_cold = cold(0, n0)
        solver.solve(u_cold, max_iters=2, lr=lr, check_every=1)   # warm-up of the launch path
        torch.cuda.synchronize(dev)
        t0 = _time.perf_counter()
        u0 = u_cold if name == "cold" else mlp.forward(feats[:n0].contiguous()).reshape(n0, T, 2)
        s99, it99, _ = solver.solve(u0, max_iters=max_iters, lr=lr, check_every=1, stop_frac=0.99)
        torch.cuda.synchronize(dev)
        wall = 1e3 * (_time.perf_counter() - t0)
        reached = float((s99 >= 0).mean())
        res[name]["measured_wall_ms_to_99pct_of_batch"] = wall if reached >= 0.99 else None
        res[name]["measured_steps_to_99pct"] = int(it99) if reached >= 0.99 else None
        res[name]["measured_batch"] = n0
    return res


# ---------------------------------------------------------------- learnable time interval
def interval_trajopt_formula(T: int, target, target_r: float, goal, goal_r: float):
    """Always over the learnable interval (bounds slot 0, caps: the whole trace) inside the target
    disc, and Eventually (over the rest of the trace) inside the goal disc."""
    inside_target = ("norm", "<", (1.0, 1.0), tuple(float(v) for v in target), float(target_r))
    inside_goal = ("norm", "<", (1.0, 1.0), tuple(float(v) for v in goal), float(goal_r))
    return ("and", ("always_sm", (float(T), float(T), 0, None), inside_target),
            ("eventually", (0.0, float("inf"), None, None), inside_goal))


def interval_trajopt(formula, gam: np.ndarray, T: int = 51, steps: int = 2000, dt: float = 0.1,
                     u_max: float = 2.0, i_nom: float = 0.2, ab0=(0.14, 0.82), lr_u: float = 0.05,
                     lr_theta: float = 0.02, tau: float = 10.0, mask_c: float = 5.0, start=(0.0, 0.0), seed: int = 0,
                     device="cuda"):
    """Optimise controls and the interval (a, b) of the trajectory-planning example for B
    coefficient settings gam [B, 4] = (g1, g2, g3, g4) at once.  Returns dict(a, b [B], hard
    robustness at t = 0 [B], x [B, T, 2], us_per_step)."""
    B = int(gam.shape[0])
    dev = torch.device(device)
    st = torch.cuda.current_stream(dev).cuda_stream
    f = Formula(formula, D=2, n_slots=1)
    ps = params("smooth", tau=tau, mask_c=mask_c)
    ph = params("hard", mask_c=mask_c)
    rng = np.random.default_rng(seed)
    u = torch.from_numpy(rng.normal(size=(B, T, 2)).astype(np.float32)).to(dev)
    x = torch.empty_like(u)
    z = lambda *s: torch.zeros(s, dtype=torch.float32, device=dev)  # noqa: E731
    mu, vu, xbar = z(B, T, 2), z(B, T, 2), z(B, T, 2)
    a0, b0 = ab0
    theta = torch.tensor([[np.log(a0 / (1 - a0)), np.log(b0 / (1 - b0))]] * B, dtype=torch.float32, device=dev)
    mth, vth = z(B, 2), z(B, 2)
    bounds = torch.tensor([[[a0 * T, b0 * T]]] * B, dtype=torch.float32, device=dev)
    gb = z(B, 1, 2)
    rho, gout = z(B, T), z(B, T)
    g = torch.from_numpy(np.ascontiguousarray(gam, dtype=np.float32)).to(dev)
    n_ws = max(f.workspace_size(B, T, ps, False), f.workspace_size(B, T, ps, True), f.workspace_size(B, T, ph, False))
    ws = torch.empty(n_ws // 4 + 1, dtype=torch.float32, device=dev)
    # x from the initial controls: one step with zero gradients and zero learning rates
    plan_call("stl_trajopt_step", _p(u), _p(mu), _p(vu), _p(theta), _p(mth), _p(vth), _p(xbar), _p(gb), _p(g), B, T, 1,
              0, dt, start[0], start[1], u_max, i_nom, 0.0, 0.0, 1, _p(x), _p(bounds), st)
    mu.zero_(); vu.zero_(); mth.zero_(); vth.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(1, steps + 1):
        robustness_raw_dense(f, x, B, T, bounds, ps, rho, ws, n_ws, st)
        plan_call("stl_trajopt_seed", _p(rho), _p(g), B, T, _p(gout), st)
        robustness_backward_raw_dense(f, x, B, T, bounds, ps, gout, xbar, gb, ws, n_ws, st)
        plan_call("stl_trajopt_step", _p(u), _p(mu), _p(vu), _p(theta), _p(mth), _p(vth), _p(xbar), _p(gb), _p(g), B,
                  T, 1, 0, dt, start[0], start[1], u_max, i_nom, lr_u, lr_theta, k, _p(x), _p(bounds), st)
    e1.record()
    robustness_raw_dense(f, x, B, T, bounds, ph, rho, ws, n_ws, st)
    torch.cuda.synchronize(dev)
    th = theta.cpu().numpy()
    ab = 1.0 / (1.0 + np.exp(-th))
    return {"a": ab[:, 0], "b": ab[:, 1], "rho_hard": rho[:, 0].cpu().numpy(), "x": x.cpu().numpy(),
            "bounds": bounds.cpu().numpy(), "us_per_step": 1e3 * e0.elapsed_time(e1) / steps}


def robustness_raw_dense(f, x, B, T, bounds, p, out, ws, n_ws, stream):
    from .binding import robustness_raw
    robustness_raw(f, _p(x), B, T, _p(bounds), p, _p(out), _p(ws), n_ws, stream)


def robustness_backward_raw_dense(f, x, B, T, bounds, p, gout, gsig, gb, ws, n_ws, stream):
    from .binding import robustness_backward_raw
    robustness_backward_raw(f, _p(x), B, T, _p(bounds), p, _p(gout), _p(gsig), _p(gb), _p(ws), n_ws, stream)
