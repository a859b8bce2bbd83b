"""CPU checks of the formula-compiled kernels' code generation: NVRTC compiles the generated
source for sm_103a without a GPU (stl_compile_kernel), the tile shrinks until the buffers fit
in shared memory, and formulas outside the compiled set are refused on the host."""
import math

import pytest

import workloads as W


@pytest.fixture(scope="module")
def stl():
    import paper_2501_04194_gb300 as m
    try:
        m.load()
    except ImportError as e:   # the library is built by __graft_entry__.build()
        pytest.skip(str(e))
    return m


CASES = [
    ("config1", W.config1_formula(), 3),
    ("config0", W.config0_formula(), 2),
    ("table3_phi6", W.table3_formulas(D=2, I=(2, 37))[5], 2),
    ("pads", W.Always(0, 50, W.Or(W.Eventually(10, 30, W.gt([1, 0], 0.2), pad=0.0),
                                  W.Not(W.Until(0, 20, W.gt([0, 1], -0.1), W.lt([1, 0], 0.0))))), 2),
    ("long_until", W.Until(300, 4000, W.gt([1], -0.5), W.lt([1], 0.5)), 1),
]


@pytest.mark.parametrize("name,tree,D", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("backward", [False, True])
def test_generated_kernels_compile(stl, name, tree, D, backward):
    f = stl.Formula(tree, D=D)
    tile, smem = f.compile_kernel(backward=backward, T=50000)
    assert tile % 32 == 0 and 512 <= tile <= (7680 if not backward else 4608)
    assert 0 < smem <= 227 * 1024


def test_tile_and_ring_placement(stl):
    """The forward takes 512 x 15 samples per step; the backward's 64-bit adjoint rings would
    limit its tile to 3072 in shared memory, so they move to the workspace (L2) and the tile
    is the requested 512 x 9; a small tile keeps them in shared memory."""
    f = stl.Formula(W.config1_formula(), D=3)
    t_fwd, s_fwd = f.compile_kernel(backward=False, T=50000)
    t_bwd, s_bwd = f.compile_kernel(backward=True, T=50000)
    assert t_fwd == 7680
    assert t_bwd == 4608 and s_bwd <= 227 * 1024
    p = stl.params("hard")
    f.set_launch(kernel="compiled")
    assert f.workspace_size(1024, 50000, p, backward=True) > 0     # rings in the workspace
    assert f.workspace_size(1024, 50000, p, backward=False) == 0
    t_small, s_small = f.compile_kernel(backward=True, T=50000, threads=256, tile=1024)
    assert t_small == 1024 and s_small < s_bwd
    f.set_launch(kernel="compiled", threads=256, tile=1024)
    assert f.workspace_size(1024, 50000, p, backward=True) == 0    # rings in shared memory


@pytest.mark.parametrize("tree,D", [
    (W.Eventually(0, math.inf, W.gt([1], 0.0)), 1),                       # unbounded interval
    (W.Eventually(0, 10, W.gt([1], 0.0), slot=0), 1),                     # per-trace bounds
    (W.And(W.norm_lt([1.0, 1.0], [0.0, 0.0], 1.0), W.gt([1, 0], 0.0)), 2),   # norm predicate
    (W.Always(0, 20000, W.gt([1], 0.0)), 1),                              # interval past 16000
])
def test_outside_the_compiled_set_is_refused(stl, tree, D):
    f = stl.Formula(tree, D=D, n_slots=1)
    with pytest.raises(stl.StlError):
        f.compile_kernel(backward=False)


@pytest.mark.parametrize("seed", range(6))
def test_random_formulas_compile(stl, seed):
    """Seed-generated formulas of depth 4 (static intervals, Not nodes, constant pads)."""
    import numpy as np
    tree = W.static_random_formula(np.random.default_rng(200 + seed), 3, 4, 300)
    f = stl.Formula(tree, D=3)
    for backward in (False, True):
        tile, smem = f.compile_kernel(backward=backward, T=20000)
        assert tile >= 512 and smem <= 227 * 1024


def test_kernel_choice_and_launch_validation(stl):
    """Host logic of the kernel selector: the automatic choice takes the compiled kernel for a
    large hard call with static intervals and no explicit shape; launch shapes are validated
    before anything runs (768 / 1024 threads only for the compiled kernels, 64 never)."""
    p = stl.params("hard")
    f = stl.Formula(W.config1_formula(), D=3)
    assert f.get_launch(1024, 50000, p, False)["kernel"] == "compiled"
    assert f.get_launch(1024, 50000, p, True)["kernel"] == "compiled"
    for kernel, threads in (("compiled", 64), ("interpreter", 768), ("auto", 1024)):
        with pytest.raises(stl.StlError):
            f.set_launch(kernel=kernel, threads=threads)
    f.set_launch(kernel="compiled", threads=768, tile=768 * 7)
    assert f.get_launch(1024, 50000, p, False) == dict(tile=768 * 7, threads=768, segment=0, kernel="compiled")
    with pytest.raises(stl.StlError):
        f.set_launch(kernel=5)
    # a forced compiled launch of a formula outside the compiled set fails on the host
    g = stl.Formula(W.Eventually(0, 10, W.gt([1], 0.0), slot=0), D=1, n_slots=1)
    g.set_launch(kernel="compiled")
    with pytest.raises(stl.StlError):
        g.get_launch(1024, 50000, p, False)
