"""The paper's own masking construction, in PyTorch FP64 on the CPU, for small traces.

Used only to pin the oracle (``oracle/``): it reaches the robustness trace by a different
route -- unroll the padded child trace into a (T+P) x T array (Sec. IV-B, Steps 1-3) or a
(T+P) x T x K array for Until (Sec. IV-C), fill the masked-out entries with +-inf and
reduce -- and torch autograd differentiates it, independently of the oracle's hand-written
adjoints.  P = b pad rows, so every read at j >= T sees the pad (reading R2).
"""
from __future__ import annotations

import math

import numpy as np
import torch

BIG = math.inf


def _pad(x, P, pad):
    if P <= 0:
        return x
    if pad is None:
        tail = x[-1:].expand(P)
    else:
        tail = torch.full((P,), float(pad), dtype=x.dtype)
    return torch.cat([x, tail])


def _window(a, b, T):
    ia = int(a)
    ib = T - 1 if math.isinf(b) else int(b)
    return ia, max(ib, ia)


def _softw(v, dim, tau, sgn):
    """Softmax-weighted max (sgn = 1) / min (sgn = -1) along dim; masked-out entries are
    -sgn*inf and carry no weight."""
    p = torch.softmax(sgn * tau * v, dim=dim)
    return (p * torch.where(torch.isfinite(v), v, torch.zeros_like(v))).sum(dim=dim)


def _smin(v, dim, tau, hard):
    if hard:
        return v.amin(dim=dim)
    if hard is None:
        return _softw(v, dim, tau, -1.0)
    return -torch.logsumexp(-tau * v, dim=dim) / tau


def _smax(v, dim, tau, hard):
    if hard:
        return v.amax(dim=dim)
    if hard is None:
        return _softw(v, dim, tau, 1.0)
    return torch.logsumexp(tau * v, dim=dim) / tau


def eventually_always(x, a, b, pad, op, hard, tau):
    """Sec. IV-B: unroll to S[j, t] = s_pad[j], keep t+a <= j <= t+b, reduce columns."""
    T = x.shape[0]
    ia, ib = _window(a, b, T)
    xp = _pad(x, ib, pad)
    R = xp.shape[0]
    S = xp[:, None].expand(R, T)
    j = torch.arange(R)[:, None]
    t = torch.arange(T)[None, :]
    keep = (j >= t) & (j >= t + ia) & (j <= t + ib)     # M_subsig + M_time
    if op == "eventually":
        return _smax(S.masked_fill(~keep, -BIG), 0, tau, hard)
    return _smin(S.masked_fill(~keep, BIG), 0, tau, hard)


def until(p, q, a, b, pad, hard, tau):
    """Sec. IV-C: 3-D unroll, S1 = stack of masked mins, S2 = min, S3 = max over i."""
    T = p.shape[0]
    ia, ib = _window(a, b, T)
    pp, qp = _pad(p, ib, pad), _pad(q, ib, pad)
    R = pp.shape[0]
    K = ib - ia + 1
    j = torch.arange(R)[:, None, None]
    t = torch.arange(T)[None, :, None]
    i = ia + torch.arange(K)[None, None, :]
    keep_p = (j >= t) & (j <= t + i)          # Always_[0,i] phi
    keep_q = j == t + i                       # Always_[i,i] psi
    Sp = pp[:, None, None].expand(R, T, K).masked_fill(~keep_p, BIG)
    Sq = qp[:, None, None].expand(R, T, K).masked_fill(~keep_q, BIG)
    S1 = torch.stack([_smin(Sp, 0, tau, hard), _smin(Sq, 0, tau, hard)], dim=0)
    S2 = _smin(S1, 0, tau, hard)
    return _smax(S2, 1, tau, hard)


def smooth_mask_window(x, a, b, c, eps, pad, op, hard, tau):
    """Sec. VI, Eq. "smooth mask", by the unroll of Sec. IV-B with NO support cutoff: every
    offset i = 0 .. T + b + 64 of the padded child trace gets the mask weight
    m_i = max(sigma(c(i - a)) - sigma(c(i - b)) - eps, 0), which enters the reduction as the
    log-weight log m_i (-inf where m_i = 0; reading R6).  ``a`` and ``b`` are torch scalars
    (in steps), so autograd gives d/da and d/db.  hard=True: max / min over {i : m_i > 0};
    False: logsumexp; None: softmax-weighted."""
    T = x.shape[0]
    N = T + int(math.ceil(float(torch.as_tensor(b).detach()))) + 64
    xp = _pad(x, N, pad)
    i = torch.arange(N, dtype=x.dtype)
    m = torch.sigmoid(c * (i - a)) - torch.sigmoid(c * (i - b)) - eps
    pos = m > 0
    m = torch.where(pos, m, torch.ones_like(m))          # no log(0) on the autograd path
    logm = torch.where(pos, torch.log(m), torch.full_like(m, -math.inf))
    t = torch.arange(T)[None, :]
    S = xp[i.long()[:, None] + t]                         # S[i, t] = padded x[t + i]
    sgn = 1.0 if op == "eventually" else -1.0
    if hard:
        fill = -sgn * math.inf
        v = S.masked_fill(~pos[:, None], fill)
        return v.amax(dim=0) if sgn > 0 else v.amin(dim=0)
    z = sgn * tau * S + logm[:, None]
    if hard is None:
        w = torch.softmax(z, dim=0)
        return (w * torch.where(pos[:, None], S, torch.zeros_like(S))).sum(dim=0)
    return sgn * torch.logsumexp(z, dim=0) / tau


def evaluate(f, x, hard=True, tau=1.0):
    """Robustness trace of formula tuple ``f`` on one trace ``x`` [T, D] (torch fp64).
    hard=True: min/max; False: logsumexp; None: softmax-weighted min/max."""
    op = f[0]
    if op == "pred":
        # predicate parameters are float32 numbers (the libraries store them as float)
        _, rel, w, c = f
        w = [float(np.float32(v)) for v in w]
        c = float(np.float32(c))
        mu = x @ torch.tensor(w, dtype=x.dtype)
        return mu - c if rel == ">" else c - mu
    if op == "norm":
        # distance of the scaled offset from the centre (Sec. VII-A region predicates)
        _, rel, sc, g, r = f
        sc = torch.tensor([float(np.float32(v)) for v in sc], dtype=x.dtype)
        g = torch.tensor([float(np.float32(v)) for v in g], dtype=x.dtype)
        mu = torch.sqrt((((x - g) * sc) ** 2).sum(dim=1))
        r = float(np.float32(r))
        return mu - r if rel == ">" else r - mu
    if op == "true":
        return torch.full((x.shape[0],), BIG, dtype=x.dtype)
    if op == "not":
        return -evaluate(f[1], x, hard, tau)
    if op in ("and", "or"):
        u = torch.stack([evaluate(f[1], x, hard, tau), evaluate(f[2], x, hard, tau)])
        return _smin(u, 0, tau, hard) if op == "and" else _smax(u, 0, tau, hard)
    a, b, slot, pad = f[1]
    if op in ("eventually", "always"):
        return eventually_always(evaluate(f[2], x, hard, tau), a, b, pad, op, hard, tau)
    if op == "until":
        return until(evaluate(f[2], x, hard, tau), evaluate(f[3], x, hard, tau), a, b, pad, hard, tau)
    raise ValueError(op)


def boolean(f, x, t, T=None):
    """Boolean semantics (Sec. III-B, Eq. "boolean") of ``f`` at sub-trajectory start ``t``
    on a numpy trace ``x`` [T, D]; reads past the end follow the pad reading R2."""
    T = x.shape[0] if T is None else T
    op = f[0]
    if op == "pred":
        _, rel, w, c = f
        w = [float(np.float32(v)) for v in w]
        c = float(np.float32(c))
        mu = float(sum(wd * float(xd) for wd, xd in zip(w, x[min(t, T - 1)])))
        return mu > c if rel == ">" else mu < c
    if op == "norm":
        _, rel, sc, g, r = f
        row = x[min(t, T - 1)]
        mu = math.sqrt(sum((float(np.float32(s_)) * (float(xd) - float(np.float32(gd)))) ** 2
                           for s_, gd, xd in zip(sc, g, row)))
        r = float(np.float32(r))
        return mu > r if rel == ">" else mu < r
    if op == "true":
        return True
    if op == "not":
        return not boolean(f[1], x, t, T)
    if op == "and":
        return boolean(f[1], x, t, T) and boolean(f[2], x, t, T)
    if op == "or":
        return boolean(f[1], x, t, T) or boolean(f[2], x, t, T)
    a, b, slot, pad = f[1]
    ia, ib = _window(a, b, T)

    def child(g, j):
        if j < T:
            return boolean(g, x, j, T)
        if pad is None:
            return boolean(g, x, T - 1, T)
        return pad > 0

    if op == "eventually":
        return any(child(f[2], t + i) for i in range(ia, ib + 1))
    if op == "always":
        return all(child(f[2], t + i) for i in range(ia, ib + 1))
    if op == "until":
        return any(child(f[3], t + i) and all(child(f[2], t + k) for k in range(0, i + 1))
                   for i in range(ia, ib + 1))
    raise ValueError(op)
