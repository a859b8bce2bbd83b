"""Parity at the benchmarked sizes, on sampled traces.

- Config 3 at its real shape: 10,000 ragged traces of 50..20,000 samples (1.0e8 samples),
  D = 4, 16 formulas of depth <= 4, per-trace intervals up to 0.2 T_b on every slot, one
  persistent launch per direction in the bench's launch configuration (longest trace first).
  Hard, logsumexp and softmax-weighted.  The oracle checks about a dozen traces: in hard mode
  the longest trace, the longest trace of the deepest formula and ten random ones; in the
  smooth modes the oracle's literal Until loops cost O(T b^2) per node, so the sample is drawn
  from the traces whose oracle cost is bounded (the longest and the deepest-formula trace among
  them included).
- Config 1 in the smooth modes at T = 10000, B = 1024 (the bench's smooth launch): three traces.
Values: hard bit-exact, smooth within 1e-5 of each trace's largest |rho|; gradients within
1e-4 of each trace's largest |grad|.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

VAL_TOL, GRAD_TOL = 1e-5, 1e-4
TAU = 10.0
OMODE = {"hard": oracle.HARD, "smooth": oracle.SMOOTH, "softmax": oracle.SOFTMAX}


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def wl3():
    return W.config3_workload()


def rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(got))
    if not fin.any():
        return 0.0
    scale = max(np.abs(ref[fin]).max(), 1e-30)
    return float((np.abs(got[fin] - ref[fin]) / scale).max())


def smooth_oracle_cost(f, T, bounds_row):
    """Rough operation count of the oracle's smooth evaluation of one trace (forward + backward):
    its Until is O(T b^2), its windows O(T (b - a + 1))."""
    op = f[0]
    if op in ("pred", "norm", "true"):
        return 0.0
    if op == "not":
        return smooth_oracle_cost(f[1], T, bounds_row)
    if op in ("and", "or"):
        return smooth_oracle_cost(f[1], T, bounds_row) + smooth_oracle_cost(f[2], T, bounds_row)
    a, b, slot, _ = f[1]
    if slot is not None:
        a, b = float(bounds_row[slot, 0]), float(bounds_row[slot, 1])
    kids = sum(smooth_oracle_cost(c, T, bounds_row) for c in f[2:])
    if op == "until":
        return kids + 2.0 * T * (b + 1) ** 2
    return kids + 2.0 * T * (b - a + 1)


def run_ragged(stl, wl, mode):
    lengths = np.diff(wl["offsets"])
    order = np.argsort(-lengths, kind="stable").astype(np.int32)
    fs = [stl.Formula(t, D=4, n_slots=wl["n_slots"]) for t in wl["formulas"]]
    p = stl.params(mode, tau=TAU)
    rb = stl.RaggedBatch(stl.FormulaSet(fs), torch.from_numpy(wl["signal"]), torch.from_numpy(wl["offsets"]),
                         torch.from_numpy(wl["formula_id"]), bounds=torch.from_numpy(wl["bounds"]), p=p,
                         order=torch.from_numpy(order))
    gout = np.random.default_rng(3).normal(size=int(wl["offsets"][-1])).astype(np.float32)
    rho = rb.forward().cpu().numpy()
    gs, _ = rb.backward(torch.from_numpy(gout).cuda())
    gs = gs.cpu().numpy()
    torch.cuda.synchronize()
    from paper_2501_04194_gb300.binding import device_status
    assert device_status() == 0
    return rho, gs, gout


def sample_traces(wl, mode, n_random=10, budget=2.5e9):
    lengths = np.diff(wl["offsets"])
    fid = wl["formula_id"]
    depth = np.array([W.formula_depth(f) for f in wl["formulas"]])
    if mode == "hard":
        eligible = np.arange(len(lengths))
    else:
        cost = np.array([smooth_oracle_cost(wl["formulas"][fid[i]], int(lengths[i]), wl["bounds"][i])
                         for i in range(len(lengths))])
        eligible = np.nonzero(cost <= budget)[0]
    assert len(eligible) >= n_random + 2
    pick = [int(eligible[np.argmax(lengths[eligible])])]
    deep = eligible[depth[fid[eligible]] == depth[fid[eligible]].max()]
    pick.append(int(deep[np.argmax(lengths[deep])]))
    rng = np.random.default_rng(11)
    rest = np.setdiff1d(eligible, pick)
    pick += [int(i) for i in rng.choice(rest, size=n_random, replace=False)]
    return pick


@pytest.mark.parametrize("mode", ["hard", "smooth", "softmax"])
def test_config3_full_size_sampled(stl, wl3, mode):
    wl = wl3
    rho, gs, gout = run_ragged(stl, wl, mode)
    pick = sample_traces(wl, mode)
    offs = wl["offsets"]
    lens = np.diff(offs)[pick]
    sub_off = np.zeros(len(pick) + 1, dtype=np.int64)
    sub_off[1:] = np.cumsum(lens)
    sl = [slice(int(offs[i]), int(offs[i + 1])) for i in pick]
    sub_sig = np.concatenate([wl["signal"][s] for s in sl])
    sub_g = np.concatenate([gout[s] for s in sl]).astype(np.float64)
    kw = dict(mode=OMODE[mode], tau=TAU, bounds=wl["bounds"][pick])
    ref = oracle.robustness_ragged_multi(wl["formulas"], wl["formula_id"][pick], sub_sig, sub_off, **kw)
    gref, _ = oracle.robustness_grad_ragged_multi(wl["formulas"], wl["formula_id"][pick], sub_sig, sub_off, sub_g,
                                                  **kw)
    assert max(lens) >= (19000 if mode == "hard" else 1000)
    for k, s in enumerate(sl):
        r = ref[sub_off[k]:sub_off[k + 1]]
        if mode == "hard":
            np.testing.assert_array_equal(rho[s], r.astype(np.float32), err_msg=f"trace {pick[k]}")
        else:
            assert rel_err(rho[s], r) <= VAL_TOL, f"trace {pick[k]}"
        assert rel_err(gs[s], gref[sub_off[k]:sub_off[k + 1]]) <= GRAD_TOL, f"trace {pick[k]}"


@pytest.mark.parametrize("mode", ["smooth", "softmax"])
def test_config1_smooth_T10000_sampled(stl, mode):
    B, T = 1024, 10000
    tree = W.config1_formula()
    f = stl.Formula(tree, D=3)
    p = stl.params(mode, tau=TAU)
    sig = W.random_walk(B, T, 3, seed=0)
    x = torch.from_numpy(sig).cuda()
    g = np.random.default_rng(4).normal(size=(B, T)).astype(np.float32)
    rho = stl.robustness(f, x, p=p).cpu().numpy()
    gs, _ = stl.robustness_backward(f, x, torch.from_numpy(g).cuda(), p=p)
    gs = gs.cpu().numpy()
    pick = [0, 511, 1023]
    ref = oracle.robustness(tree, sig[pick], mode=OMODE[mode], tau=TAU)
    gref, _ = oracle.robustness_grad(tree, sig[pick], g[pick].astype(np.float64), mode=OMODE[mode], tau=TAU)
    for k, b in enumerate(pick):
        assert rel_err(rho[b], ref[k]) <= VAL_TOL
        assert rel_err(gs[b], gref[k]) <= GRAD_TOL
