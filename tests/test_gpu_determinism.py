"""Run-to-run and launch-shape determinism of the gradients.

Hard mode: every root gradient is rounded to a 64-bit fixed-point integer (scale from the
trace's largest root gradient) before any addition, so the signal gradient is bit-identical
across repeated launches, CTA sizes, tiles, segmentations, the one-launch robustness-and-
gradient call and the ragged path.  Logsumexp mode: adjoints are fixed-point sums as well, so
repeated launches of one shape agree bit for bit.  The softmax-weighted mode adds floats in an
order set by the scheduling of warps; there two launches may differ, within float32
summation error.
"""
import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stl():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2501_04194_gb300 as m
    assert torch.cuda.is_available()
    return m


def _inputs(B, T, D, seed):
    x = torch.from_numpy(W.random_walk(B, T, D, seed=seed)).cuda()
    g = torch.from_numpy(np.random.default_rng(seed + 1).normal(size=(B, T)).astype(np.float32)).cuda()
    return x, g


def test_hard_gradient_is_bitwise_repeatable(stl):
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("hard")
    x, g = _inputs(64, 12000, 3, 31)
    ref, _ = stl.robustness_backward(f, x, g, p=p)
    for _ in range(3):
        got, _ = stl.robustness_backward(f, x, g, p=p)
        assert torch.equal(got, ref)


@pytest.mark.parametrize("tile,threads,segment", [(448, 64, 0), (1792, 256, 0), (7168, 512, 0),
                                                  (3584, 512, 2500), (2048, 256, 4096)])
def test_hard_gradient_is_independent_of_the_launch_shape(stl, tile, threads, segment):
    f0 = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("hard")
    x, g = _inputs(16, 9000, 3, 32)
    ref, _ = stl.robustness_backward(f0, x, g, p=p)
    f = stl.Formula(W.config1_formula(), D=3)
    f.set_launch(tile=tile, threads=threads, segment=segment)
    got, _ = stl.robustness_backward(f, x, g, p=p)
    assert torch.equal(got, ref)
    rho, got2, _ = stl.robustness_and_grad(f, x, g, p=p)
    assert torch.equal(got2, ref)


def test_hard_gradient_with_large_and_tiny_upstream_gradients(stl):
    # the fixed-point scale follows each trace's largest |g|: a trace whose upstream gradient
    # is scaled by a power of two (far from 1 either way, still normal floats) gets the same
    # integers, hence the unscaled gradient times that power, bit for bit
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("hard")
    x, g = _inputs(4, 5000, 3, 33)
    x4 = x[:1].expand(4, -1, -1).contiguous()
    g4 = g[:1].expand(4, -1).contiguous()
    base, _ = stl.robustness_backward(f, x4[:1], g4[:1], p=p)
    scale = torch.tensor([2.0 ** 60, 1.0, 2.0 ** -60, 2.0 ** -100], device="cuda")[:, None]
    got, _ = stl.robustness_backward(f, x4, g4 * scale, p=p)
    for b in range(4):
        assert torch.equal(got[b], base[0] * scale[b, 0])


def test_logsumexp_gradient_is_bitwise_repeatable(stl):
    # the logsumexp adjoints are fixed-point sums too: the same launch shape gives the same bits
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("smooth", tau=10.0)
    x, g = _inputs(16, 3000, 3, 34)
    ref, _ = stl.robustness_backward(f, x, g, p=p)
    for _ in range(3):
        got, _ = stl.robustness_backward(f, x, g, p=p)
        assert torch.equal(got, ref)


def test_softmax_gradient_differs_at_most_by_summation_error(stl):
    f = stl.Formula(W.config1_formula(), D=3)
    p = stl.params("softmax", tau=10.0)
    x, g = _inputs(16, 3000, 3, 34)
    ref, _ = stl.robustness_backward(f, x, g, p=p)
    scale = ref.abs().amax(dim=(1, 2), keepdim=True).clamp_min(1e-30)
    for _ in range(3):
        got, _ = stl.robustness_backward(f, x, g, p=p)
        assert float(((got - ref).abs() / scale).max()) < 1e-5
