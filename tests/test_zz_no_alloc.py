"""cd_column_density_noalloc against cd_column_density.

The no-allocation entry point keeps its scratch in a fixed device array inside
the library, for simulation codes that reserve all device memory at start-up
and must not allocate inside their time-step loop.  Its output must match the
regular entry point within the FP32 tolerance of the other GPU tests, on two
calls in a row (the second call reuses the array the first one left behind).
This file is named so that pytest collects it last.
"""
import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import colden, synth

pytestmark = pytest.mark.gpu
RTOL = 1e-5          # same FP32 tolerance as the parity tests
SHIELD_ATOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _outputs(tree, nd):
    return (torch.full((tree.n_leaf * nd,), -1.0, device="cuda"),
            torch.full((tree.n_leaf * nd,), -1.0, device="cuda"),
            torch.full((tree.n_leaf,), -1.0, device="cuda"))


@pytest.mark.parametrize("L,nside", [(2, 1), (5, 2), (6, 2)])
def test_noalloc_matches_regular_entry_point_twice(L, nside):
    box = 10 * synth.PC_CM
    geom = colden.precompute_geometry("healpix", nside)
    nd = geom.n_dir
    rho_a = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=40 + L)
    rho_b = synth.lognormal_iid(1 << L, 10.0, 1.5, seed=50 + L)
    tree = colden.build_tree_uniform(torch.from_numpy(rho_a).cuda(), box)
    for rho in (rho_a, rho_b):      # two calls in a row, different inputs
        colden.tree_update(tree, torch.from_numpy(rho).cuda().reshape(-1))
        ref = _outputs(tree, nd)
        colden.column_density(tree, geom, n_h=ref[0], a_v=ref[1], shield=ref[2])
        got = _outputs(tree, nd)
        colden.column_density_noalloc(tree, geom, n_h=got[0], a_v=got[1], shield=got[2])
        torch.cuda.synchronize()
        r = [t.double().cpu().numpy() for t in ref]
        g = [t.double().cpu().numpy() for t in got]
        assert np.all(g[0] > 0) and np.all(g[2] > 0)
        assert np.max(np.abs(g[0] - r[0]) / r[0]) <= RTOL
        assert np.max(np.abs(g[1] - r[1]) / r[1]) <= RTOL
        assert np.max(np.abs(g[2] - r[2])) <= SHIELD_ATOL


def test_noalloc_allocates_nothing_per_call():
    """The property the entry point exists for: once its set-up call (all
    outputs NULL) has loaded the fixed array, calls on a fresh tree that never
    went through cd_column_density leave the device's free memory unchanged
    (the regular entry point would allocate the tree's scratch on its first
    call: about 10 MB here), and their output matches the oracle."""
    import oracle
    L, box = 6, 10 * synth.PC_CM
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=77)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    out = _outputs(tree, nd)
    colden.column_density_noalloc(tree, geom)          # set-up call: no outputs
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        colden.column_density_noalloc(tree, geom, n_h=out[0], a_v=out[1], shield=out[2])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    lv, ijk = tree.leaves()
    rows = np.random.default_rng(9).choice(tree.n_leaf, size=200, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density(oracle.dirs_healpix(2), lv[rows], ijk[rows])
    got = out[0].reshape(-1, nd)[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) <= RTOL
    # the regular entry point on the same kind of fresh tree does allocate
    tree2 = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    colden.column_density(tree2, geom, n_h=out[0])
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] < free1


def test_noalloc_rejects_trees_beyond_the_fixed_scratch():
    geom = colden.precompute_geometry("healpix", 2)
    rho = np.ones((128, 128, 128), np.float32)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), synth.PC_CM)
    sh = torch.empty(tree.n_leaf, device="cuda")
    with pytest.raises(colden.ColdenError) as e:
        colden.column_density_noalloc(tree, geom, shield=sh)
    assert e.value.code == colden.CD_EINVAL and "16 MiB" in str(e.value)
    assert colden.load().cd_column_density_noalloc(None, None, None, None, None, None,
                                                    None) == colden.CD_EINVAL
