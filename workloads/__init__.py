"""Seeded synthetic inputs and formula syntax trees for the STL robustness workloads.

This module is shared by the tests, ``bench.py`` and the smoke check.  It produces
plain data only -- float32 signal arrays, bounds arrays and formula syntax trees made
of nested tuples -- and holds none of the robustness arithmetic: both the CUDA
library's binding and the CPU oracle parse the same tuple format with their own code.

Formula syntax tree (the STL grammar of Sec. III-B, Eq. "STL grammar", plus the derived
Or / Eventually / Always and the smoothed-interval operators of Sec. VI):

    ("pred", ">", w, c)        mu(x) - c  with mu(x) = sum_d w[d] * x[d]   (Eq. quantitative)
    ("pred", "<", w, c)        c - mu(x)
    ("norm", ">", s, g, r)     ||diag(s)(x - g)||_2 - r   (outside a ball; Sec. VII-A regions)
    ("norm", "<", s, g, r)     r - ||diag(s)(x - g)||_2   (inside it)
    ("true",)                  the constant formula T (rho_max = +inf)
    ("not", f)
    ("and", f, g)              ("or", f, g)
    ("eventually", I, f)       ("always", I, f)
    ("until", I, f, g)         f U_I g
    ("eventually_sm", I, f)    ("always_sm", I, f)     sigmoid-masked interval (Eq. smooth mask)
    ("until_sm", I, f, g)      f U g with the sigmoid-masked interval on the outer offsets

An interval ``I`` is the tuple ``(a, b, slot, pad)``:
    a, b  -- bounds in time steps (b may be ``inf`` = the whole signal);
             when ``slot`` is not None they are the largest values the per-trace bounds
             ``bounds[:, slot, :]`` may take, and the per-trace values are used instead;
    slot  -- None, or the column of the per-trace ``bounds[B, n_slots, 2]`` array;
    pad   -- None (reads past the end repeat the last sample) or a float constant.
"""
from __future__ import annotations

import math

import numpy as np

INF = math.inf


# ----------------------------------------------------------------------------- formulas
def interval(a, b, slot=None, pad=None):
    return (float(a), float(b), None if slot is None else int(slot), None if pad is None else float(pad))


def gt(w, c):
    return ("pred", ">", tuple(float(v) for v in w), float(c))


def lt(w, c):
    return ("pred", "<", tuple(float(v) for v in w), float(c))


def norm_gt(scale, centre, r):
    return ("norm", ">", tuple(float(v) for v in scale), tuple(float(v) for v in centre), float(r))


def norm_lt(scale, centre, r):
    return ("norm", "<", tuple(float(v) for v in scale), tuple(float(v) for v in centre), float(r))


def true():
    return ("true",)


def Not(f):
    return ("not", f)


def And(f, g):
    return ("and", f, g)


def Or(f, g):
    return ("or", f, g)


def Eventually(a, b, f, slot=None, pad=None):
    return ("eventually", interval(a, b, slot, pad), f)


def Always(a, b, f, slot=None, pad=None):
    return ("always", interval(a, b, slot, pad), f)


def Until(a, b, f, g, slot=None, pad=None):
    return ("until", interval(a, b, slot, pad), f, g)


def EventuallySm(a, b, f, slot=None, pad=None):
    return ("eventually_sm", interval(a, b, slot, pad), f)


def UntilSm(a, b, f, g, slot=None, pad=None):
    return ("until_sm", interval(a, b, slot, pad), f, g)


def AlwaysSm(a, b, f, slot=None, pad=None):
    return ("always_sm", interval(a, b, slot, pad), f)


def onehot(D, d, scale=1.0):
    w = [0.0] * D
    w[d] = float(scale)
    return w


def formula_depth(f) -> int:
    """Operator depth above the predicates (a predicate or True has depth 0)."""
    op = f[0]
    if op in ("pred", "true"):
        return 0
    kids = [k for k in f[1:] if isinstance(k, tuple) and k and isinstance(k[0], str)]
    return 1 + max(formula_depth(k) for k in kids)


def count_slots(f) -> int:
    """1 + the largest bounds slot used anywhere in the tree (0 if none)."""
    n = 0
    op = f[0]
    if op in ("eventually", "always", "until", "eventually_sm", "always_sm"):
        slot = f[1][2]
        if slot is not None:
            n = slot + 1
    for k in f[1:]:
        if isinstance(k, tuple) and k and isinstance(k[0], str):
            n = max(n, count_slots(k))
    return n


# ----------------------------------------------------------------------------- signals
def random_walk(B, T, D, sigma=0.1, seed=0, chunk=64):
    """s[b,0,:] = 0, s[b,t,:] = s[b,t-1,:] + N(0, sigma^2); increments and cumsum in
    float64 (numpy PCG64 stream of ``seed``), cast to float32.  Generated ``chunk``
    traces at a time so that large batches do not need a float64 copy of the whole
    array."""
    rng = np.random.default_rng(seed)
    out = np.empty((B, T, D), dtype=np.float32)
    for b0 in range(0, B, chunk):
        nb = min(chunk, B - b0)
        inc = rng.normal(0.0, sigma, size=(nb, T, D))
        inc[:, 0, :] = 0.0
        out[b0:b0 + nb] = np.cumsum(inc, axis=1).astype(np.float32)
    return out


def noisy_sinusoid(B, T, f_lo=50.0, f_hi=400.0, noise=0.05, seed=0):
    """s[b,t,0] = sin(2 pi t / f_b) + N(0, noise^2), f_b ~ U[f_lo, f_hi] per trace."""
    rng = np.random.default_rng(seed)
    f = rng.uniform(f_lo, f_hi, size=(B, 1))
    t = np.arange(T, dtype=np.float64)[None, :]
    s = np.sin(2.0 * np.pi * t / f) + rng.normal(0.0, noise, size=(B, T))
    return s.astype(np.float32)[:, :, None]


# ----------------------------------------------------------------------------- configs
def config0_formula():
    """Always_[0,99](s_x > -1.0) AND Eventually_[10,40](s_y - 0.5 > 0)."""
    return And(Always(0, 99, gt([1, 0], -1.0)), Eventually(10, 40, gt([0, 1], 0.5)))


def config0_inputs():
    return random_walk(8, 100, 2, seed=0)


def config1_formula():
    """(Always_[0,500]((s_x > 0) Until_[5,200] (s_y + s_z < 0.2))) OR Eventually_[0,1000](s_z > 1)."""
    return Or(Always(0, 500, Until(5, 200, gt([1, 0, 0], 0.0), lt([0, 1, 1], 0.2))),
              Eventually(0, 1000, gt([0, 0, 1], 1.0)))


def config1_inputs(B=1024, T=10000, seed=0):
    return random_walk(B, T, 3, seed=seed)


CONFIG2_A_MAX = 100.0
CONFIG2_B_MAX = 400.0


def config2_formula(a_max=CONFIG2_A_MAX, b_max=CONFIG2_B_MAX):
    """Eventually over a sigmoid-masked per-trace interval [a_b, b_b] of (s > 0.8)."""
    return EventuallySm(a_max, b_max, gt([1.0], 0.8), slot=0)


def config2_inputs(B=4096, T=2000, seed=0):
    """Noisy sinusoids and per-trace learnable bounds a ~ U[0,100], b = a + U[20,300]."""
    sig = noisy_sinusoid(B, T, seed=seed)
    rng = np.random.default_rng(seed + 1000)
    a = rng.uniform(0.0, 100.0, size=B)
    b = a + rng.uniform(20.0, 300.0, size=B)
    bounds = np.stack([a, b], axis=1).astype(np.float32)[:, None, :]
    return sig, bounds


def random_formula(rng, D, depth, slot_counter, b_cap):
    """A seed-generated formula of operator depth <= ``depth`` over And/Or/Always/Eventually/Until
    with affine predicates (one-hot or +-1 weights, c ~ N(0,1)).  Every temporal node
    takes its interval from its own bounds slot, whose largest allowed value is ``b_cap``."""
    def pred():
        if rng.random() < 0.5:
            w = onehot(D, int(rng.integers(D)))
        else:
            w = [float(rng.choice([-1.0, 1.0])) if rng.random() < 0.6 else 0.0 for _ in range(D)]
            if all(v == 0.0 for v in w):
                w[int(rng.integers(D))] = 1.0
        c = float(np.float32(rng.normal()))
        return gt(w, c) if rng.random() < 0.5 else lt(w, c)

    def build(d):
        if d == 0:
            return pred()
        op = str(rng.choice(["and", "or", "always", "eventually", "until"], p=[0.15, 0.15, 0.25, 0.25, 0.2]))
        if op in ("and", "or"):
            return (op, build(d - 1), build(int(rng.integers(0, d))))
        slot = slot_counter[0]
        slot_counter[0] += 1
        iv = interval(b_cap, b_cap, slot, None)   # caps for the per-trace (a, b)
        if op == "until":
            return ("until", iv, build(d - 1), build(int(rng.integers(0, d))))
        return (op, iv, build(d - 1))

    return build(depth)


def static_random_formula(rng, D, depth, b_cap, not_prob=0.15, const_pad_prob=0.2):
    """A seed-generated formula of operator depth <= ``depth`` like ``random_formula``, but with
    static integer intervals 0 <= a <= b <= ``b_cap`` drawn per temporal node, occasional Not
    nodes and occasional constant pads (the shapes the formula-compiled kernels serve)."""
    def pred():
        w = onehot(D, int(rng.integers(D))) if rng.random() < 0.5 else \
            [float(rng.choice([-1.0, 1.0])) if rng.random() < 0.6 else 0.0 for _ in range(D)]
        if all(v == 0.0 for v in w):
            w[int(rng.integers(D))] = 1.0
        c = float(np.float32(rng.normal()))
        return gt(w, c) if rng.random() < 0.5 else lt(w, c)

    def build(d):
        if d == 0:
            f = pred()
        else:
            op = str(rng.choice(["and", "or", "always", "eventually", "until"], p=[0.15, 0.15, 0.25, 0.25, 0.2]))
            if op in ("and", "or"):
                f = (op, build(d - 1), build(int(rng.integers(0, d))))
            else:
                a = int(rng.integers(0, b_cap // 3 + 1))
                b = a + int(rng.integers(0, b_cap - a + 1))
                pad = float(np.float32(rng.normal())) if rng.random() < const_pad_prob else None
                iv = interval(a, b, None, pad)
                f = ("until", iv, build(d - 1), build(int(rng.integers(0, d)))) if op == "until" else (op, iv, build(d - 1))
        return Not(f) if rng.random() < not_prob else f

    return build(depth)


def config3_workload(n_traces=10000, t_lo=50, t_hi=20000, D=4, n_formulas=16, max_depth=4, seed=0):
    """Ragged batch: lengths ~ U[t_lo, t_hi], random-walk signals packed as [sum T, D],
    16 seed-generated formulas (seed+1) and per-trace integer bounds a < b ~ U[0, 0.2 T_b]."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(t_lo, t_hi + 1, size=n_traces).astype(np.int64)
    offsets = np.zeros(n_traces + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(lengths)
    frng = np.random.default_rng(seed + 1)
    formulas, n_slots = [], []
    for _ in range(n_formulas):
        ctr = [0]
        f = random_formula(frng, D, int(frng.integers(1, max_depth + 1)), ctr, float(int(0.2 * t_hi)))
        formulas.append(f)
        n_slots.append(ctr[0])
    formula_id = rng.integers(0, n_formulas, size=n_traces).astype(np.int32)
    S = max(1, max(n_slots))
    bounds = np.zeros((n_traces, S, 2), dtype=np.float32)
    for i in range(n_traces):
        cap = max(1, int(0.2 * lengths[i]))
        for s in range(S):
            a, b = sorted(rng.integers(0, cap + 1, size=2).tolist())
            if a == b:
                b = a + 1
            bounds[i, s, 0], bounds[i, s, 1] = a, b
    sig = np.empty((int(offsets[-1]), D), dtype=np.float32)
    srng = np.random.default_rng(seed + 2)
    for i in range(n_traces):
        T = int(lengths[i])
        inc = srng.normal(0.0, 0.1, size=(T, D))
        inc[0, :] = 0.0
        sig[offsets[i]:offsets[i + 1]] = np.cumsum(inc, axis=0).astype(np.float32)
    return dict(signal=sig, offsets=offsets, lengths=lengths, formula_id=formula_id,
                formulas=formulas, n_slots=S, bounds=bounds, t_cap=int(t_hi))


# Table III formula templates (structures only; the predicates are synthetic).
def table3_formulas(D=2, I=(0, 20)):
    a, b = I
    pv = lambda k: gt(onehot(D, 0), 0.1 * k)          # noqa: E731  varphi_k
    ps = lambda k: lt(onehot(D, 1), 1.0 + 0.1 * k)    # noqa: E731  psi_k
    phi1 = Always(0, INF, And(pv(0), ps(0)))
    phi2 = Eventually(0, INF, Always(0, INF, And(pv(0), ps(0))))
    phi3 = Until(0, INF, pv(0), ps(0))
    inner = And(pv(0), ps(0))
    for k in (1, 2, 3):
        inner = And(And(pv(k), ps(k)), Eventually(a, b, inner))
    phi4 = Eventually(a, b, inner)
    phi5 = Eventually(a, b, And(And(pv(2), ps(2)), Eventually(a, b, Always(a, b, And(pv(0), ps(0))))))
    phi6 = Eventually(a, b, And(pv(9), ps(9)))
    for k in range(8, -1, -1):
        phi6 = And(phi6, Eventually(a, b, And(pv(k), ps(k))))
    return [phi1, phi2, phi3, phi4, phi5, phi6]


# Reach/avoid planning problems (the control-synthesis workload): 2-D single integrator with
# saturated controls, x_{t+1} = x_t + dt * tanh(u_t) from x_0 = 0, evaluated on x_1..x_T.
CONFIG4_T = 200
CONFIG4_OBSTACLES = 3


def reach_avoid_formula(goal, obstacles, radii, reach=(50, 150), goal_r=0.3):
    """Eventually_[reach] inside the goal disc (radius goal_r), and, for every obstacle k,
    Always outside the disc of radius r_k around o_k."""
    f = Eventually(reach[0], reach[1], norm_lt([1.0, 1.0], goal, goal_r))
    for o, r in zip(obstacles, radii):
        f = And(f, Always(0, INF, norm_gt([1.0, 1.0], o, r)))
    return f


def config4_problems(n, seed=0, n_obstacles=CONFIG4_OBSTACLES):
    """n problems: goal g and obstacle centres o_k ~ U[-3, 3]^2, radii r_k ~ U[0.3, 0.8];
    problems with the origin or the goal inside an obstacle are redrawn."""
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < n:
        g = rng.uniform(-3.0, 3.0, size=2).astype(np.float32)
        o = rng.uniform(-3.0, 3.0, size=(n_obstacles, 2)).astype(np.float32)
        r = rng.uniform(0.3, 0.8, size=n_obstacles).astype(np.float32)
        if np.any(np.linalg.norm(o, axis=1) <= r) or np.any(np.linalg.norm(o - g, axis=1) <= r):
            continue
        out.append((g, o, r))
    return out


def rollout(u, dt=0.1):
    """Trajectories [B, T, 2] (float32) of x_{t+1} = x_t + dt tanh(u_t), x_0 = 0, for controls
    u [B, T, 2]; sample t of the result is x_{t+1}."""
    u = np.asarray(u, dtype=np.float64)
    return np.cumsum(dt * np.tanh(u), axis=1).astype(np.float32)


def random_controls(B, T=CONFIG4_T, seed=0, scale=1.0):
    rng = np.random.default_rng(seed)
    return (scale * rng.normal(size=(B, T, 2))).astype(np.float32)


# Specification-mining data: signals of T samples equal to 1 inside a noisy interval around
# (a, b) (fractions of the trace) and 0 elsewhere, plus Gaussian noise on every sample.
def mining_dataset(N=1000, T=20, a=0.23, b=0.59, edge_sigma=0.02, noise=0.05, seed=0):
    rng = np.random.default_rng(seed)
    an = a + edge_sigma * rng.normal(size=(N, 1))
    bn = b + edge_sigma * rng.normal(size=(N, 1))
    t = np.arange(T)[None, :] / T
    s = ((t >= an) & (t <= bn)).astype(np.float64) + noise * rng.normal(size=(N, T))
    return s.astype(np.float32)[:, :, None]
