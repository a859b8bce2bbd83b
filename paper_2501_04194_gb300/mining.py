"""Time-interval search and specification mining with the smooth interval mask (Sec. VI).

- ``interval_sweep``: robustness at t = 0 of Always_[aT, bT](s > c0) for many (a, b) at once,
  one trace per interval in a single launch (the vectorised sweep of Sec. VI);
- ``mine_interval``: gradient descent on the largest interval [a, b] that a dataset satisfies,
  loss (1/N) sum max(-rho, 0) + gamma (a - b) with a, b = sigmoid(alpha), sigmoid(beta), the mask
  sharpness c and the temperature tau annealed on a sigmoid schedule (the mining example of
  Sec. VII-C).  Each step is four launches: forward, loss seed, backward with the bound gradients,
  and the parameter update (include/stl_mining.h).
"""
from __future__ import annotations

import ctypes
import math

import numpy as np
import torch

from .binding import Formula, check, load, params, robustness_backward_raw, robustness_raw


def _p(t):
    return None if t is None else t.data_ptr()


def _lib():
    lib = load()
    if not getattr(lib, "_mining_ready", False):
        vp, i32, i64, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float
        lib.stl_mining_seed.argtypes = [vp, i64, i32, vp, vp, vp]
        lib.stl_mining_seed.restype = i32
        lib.stl_mining_update.argtypes = [vp, vp, i64, i32, i32, i32, f32, f32, vp, vp]
        lib.stl_mining_update.restype = i32
        lib.stl_mining_update_traces.argtypes = [vp, vp, i64, i32, i32, f32, f32, f32, f32, f32, f32, vp]
        lib.stl_mining_update_traces.restype = i32
        lib._mining_ready = True
    return lib


def always_interval_formula(T: int, c0: float = 0.0):
    """Always over the per-trace interval in bounds slot 0 (caps: the whole trace) of s > c0."""
    return ("always_sm", (float(T), float(T), 0, None), ("pred", ">", (1.0,), float(c0)))


def interval_sweep(signal: np.ndarray, a: np.ndarray, b: np.ndarray, c: float = 5.0, eps: float = 1e-3,
                   tau: float = 10.0, device="cuda"):
    """rho_0 of Always_[aT, bT](s > 0) for the one signal [T] and every (a[k], b[k]); returns
    (rho0 [K] numpy, device milliseconds of the launch)."""
    T = int(signal.shape[0])
    K = int(len(a))
    dev = torch.device(device)
    f = Formula(always_interval_formula(T), D=1, n_slots=1)
    p = params("smooth", tau=tau, mask_c=c, mask_eps=eps)
    x = torch.from_numpy(np.ascontiguousarray(np.broadcast_to(signal.astype(np.float32).reshape(1, T, 1),
                                                              (K, T, 1)))).to(dev)
    bd = torch.from_numpy(np.stack([a * T, b * T], axis=1).astype(np.float32).reshape(K, 1, 2)).to(dev)
    out = torch.empty((K, T), dtype=torch.float32, device=dev)
    n = f.workspace_size(K, T, p, False)
    ws = torch.empty(n // 4 + 1, dtype=torch.float32, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    robustness_raw(f, x.data_ptr(), K, T, bd.data_ptr(), p, out.data_ptr(), ws.data_ptr(), n, st)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    robustness_raw(f, x.data_ptr(), K, T, bd.data_ptr(), p, out.data_ptr(), ws.data_ptr(), n, st)
    e1.record()
    torch.cuda.synchronize(dev)
    return out[:, 0].cpu().numpy(), e0.elapsed_time(e1)


def sigmoid_schedule(k: int, K: int, lo: float, hi: float, sharp: float = 10.0) -> float:
    return lo + (hi - lo) / (1.0 + math.exp(-sharp * (k / max(K - 1, 1) - 0.5)))


def mine_interval(signals: np.ndarray, steps: int = 5000, lr: float = 1e-2, gamma: float = 0.1,
                  ab0=(0.1, 0.9), c_range=(1.0, 20.0), tau_range=(1.0, 20.0), eps: float = 1e-3,
                  record_every: int = 500, device="cuda"):
    """Gradient descent on (a, b) for signals [N, T, 1]; returns dict(a, b, history [(step, a, b,
    loss)], us_per_step)."""
    N, T = int(signals.shape[0]), int(signals.shape[1])
    dev = torch.device(device)
    lib = _lib()
    st = torch.cuda.current_stream(dev).cuda_stream
    f = Formula(always_interval_formula(T), D=1, n_slots=1)
    x = torch.from_numpy(np.ascontiguousarray(signals, dtype=np.float32)).to(dev)
    a0, b0 = ab0
    theta = torch.tensor([math.log(a0 / (1 - a0)), math.log(b0 / (1 - b0))], dtype=torch.float32, device=dev)
    bounds = torch.tensor([[a0 * T, b0 * T]], dtype=torch.float32).repeat(N, 1).reshape(N, 1, 2).to(dev)
    rho = torch.empty((N, T), dtype=torch.float32, device=dev)
    gout = torch.zeros((N, T), dtype=torch.float32, device=dev)
    gsig = torch.empty((N, T, 1), dtype=torch.float32, device=dev)
    gb = torch.empty((N, 1, 2), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    p_worst = params("smooth", tau=tau_range[0], mask_c=min(c_range), mask_eps=eps)
    n_ws = max(f.workspace_size(N, T, p_worst, False), f.workspace_size(N, T, p_worst, True))
    ws = torch.empty(n_ws // 4 + 1, dtype=torch.float32, device=dev)
    hist = []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for k in range(steps):
        p = params("smooth", tau=sigmoid_schedule(k, steps, *tau_range), mask_c=sigmoid_schedule(k, steps, *c_range),
                   mask_eps=eps)
        robustness_raw(f, x.data_ptr(), N, T, bounds.data_ptr(), p, rho.data_ptr(), ws.data_ptr(), n_ws, st)
        rec = record_every and (k % record_every == 0 or k == steps - 1)
        if rec:
            loss.zero_()
        check(lib.stl_mining_seed(rho.data_ptr(), N, T, gout.data_ptr(), loss.data_ptr() if rec else None, st))
        robustness_backward_raw(f, x.data_ptr(), N, T, bounds.data_ptr(), p, gout.data_ptr(), gsig.data_ptr(),
                                gb.data_ptr(), ws.data_ptr(), n_ws, st)
        if rec:
            th = theta.cpu().numpy()
            a, b = 1 / (1 + np.exp(-th))
            hist.append((k, float(a), float(b), float(loss.item()) + gamma * float(a - b)))
        check(lib.stl_mining_update(theta.data_ptr(), gb.data_ptr(), N, 1, 0, T, lr, gamma, bounds.data_ptr(), st))
    e1.record()
    torch.cuda.synchronize(dev)
    th = theta.cpu().numpy()
    a, b = 1 / (1 + np.exp(-th))
    return {"a": float(a), "b": float(b), "history": hist, "us_per_step": 1e3 * e0.elapsed_time(e1) / steps}


def per_trace_descent(signals: np.ndarray, bounds: np.ndarray, steps: int = 200, lr: float = 2.0,
                      gamma: float = 0.01, c: float = 5.0, eps: float = 1e-3, tau: float = 10.0,
                      a_cap: float = 100.0, b_cap: float = 400.0, formula=None, tune: bool = False,
                      device="cuda"):
    """The parameter-mining descent of config 2: each trace n has its own learnable interval
    (a_n, b_n) (in steps) of Eventually over the sigmoid-masked window of s > 0.8, and takes
    ``steps`` gradient steps on max(-rho_n(0), 0) - gamma (b_n - a_n).  One step is four
    launches: robustness, loss seed, backward with the bound gradients, per-trace update.
    tune: pick both launch shapes with stl_autotune first.
    Returns dict(bounds [N, 1, 2] numpy, loss0, loss, ms_per_step, steps, launch)."""
    N, T = int(signals.shape[0]), int(signals.shape[1])
    dev = torch.device(device)
    lib = _lib()
    st = torch.cuda.current_stream(dev).cuda_stream
    tree = formula or ("eventually_sm", (a_cap, b_cap, 0, None), ("pred", ">", (1.0,), 0.8))
    f = Formula(tree, D=1, n_slots=1)
    p = params("smooth", tau=tau, mask_c=c, mask_eps=eps)
    x = torch.from_numpy(np.ascontiguousarray(signals, dtype=np.float32)).to(dev)
    bd = torch.from_numpy(np.ascontiguousarray(bounds, dtype=np.float32)).to(dev)
    rho = torch.empty((N, T), dtype=torch.float32, device=dev)
    gout = torch.zeros((N, T), dtype=torch.float32, device=dev)
    gsig = torch.empty((N, T, 1), dtype=torch.float32, device=dev)
    gb = torch.empty((N, 1, 2), dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    if tune:   # launch shapes of both directions from stl_autotune, before any timing
        from .torch_api import autotune
        autotune(f, x, bounds=bd, p=p, backward=False)
        autotune(f, x, bounds=bd, p=p, backward=True)
    n_ws = max(f.workspace_size(N, T, p, False), f.workspace_size(N, T, p, True))
    ws = torch.empty(n_ws // 4 + 1, dtype=torch.float32, device=dev)

    def step(rec=False):
        robustness_raw(f, x.data_ptr(), N, T, bd.data_ptr(), p, rho.data_ptr(), ws.data_ptr(), n_ws, st)
        check(lib.stl_mining_seed(rho.data_ptr(), N, T, gout.data_ptr(), loss.data_ptr() if rec else None, st))
        robustness_backward_raw(f, x.data_ptr(), N, T, bd.data_ptr(), p, gout.data_ptr(), gsig.data_ptr(),
                                gb.data_ptr(), ws.data_ptr(), n_ws, st)
        check(lib.stl_mining_update_traces(bd.data_ptr(), gb.data_ptr(), N, 1, 0, lr, gamma, float(N), a_cap, b_cap,
                                           1.0, st))

    def total_loss():
        loss.zero_()
        robustness_raw(f, x.data_ptr(), N, T, bd.data_ptr(), p, rho.data_ptr(), ws.data_ptr(), n_ws, st)
        check(lib.stl_mining_seed(rho.data_ptr(), N, T, gout.data_ptr(), loss.data_ptr(), st))
        w = (bd[:, 0, 1] - bd[:, 0, 0]).mean()
        return float(loss.item()) - gamma * float(w.item())

    loss0 = total_loss()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    return {"bounds": bd.cpu().numpy(), "loss0": loss0, "loss": total_loss(), "ms_per_step": ms / steps,
            "steps": steps, "launch": {"forward": f.get_launch(N, T, p, False), "backward": f.get_launch(N, T, p, True)}}
