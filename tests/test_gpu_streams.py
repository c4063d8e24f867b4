"""Concurrent evaluation on the tree's side streams.

An evaluation runs its independent steps (the far-shell prefix chain, the oct
shells, the leaves of each AMR level) on two side streams joined back into
the caller's stream; with per-launch timing on it runs them in order on the
caller's stream.  The kernels and their inputs are the same either way, so
the results must be bitwise identical, and work the caller enqueues on its
stream afterwards must see the finished outputs.
"""
import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)
    yield
    colden.stats_reset(timing=False)


def _amr_tree(nfine=64, base=4, seed=17):
    fine = synth.lognormal_grf(nfine, 30.0, 2.0, seed=seed)
    lv = synth.amr_leaves(fine, base, [40.0, 60.0])
    return colden.build_tree_amr(lv["base"], lv["lmax"], 10 * PC, lv["level"], lv["ijk"], lv["rho"]), lv


def _eval(tree, geom, precision, timing):
    colden.stats_reset(timing=timing)
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=precision)
    colden.device_status()
    colden.stats_reset(timing=False)
    return n_h.cpu().numpy(), sh.cpu().numpy()


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
@pytest.mark.parametrize("kind", ["uniform", "amr", "amr_insitu"])
def test_concurrent_matches_in_order(kind, precision):
    if kind == "uniform":
        rho = synth.lognormal_grf(64, 30.0, 2.0, seed=5)
        tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), 10 * PC)
    else:
        tree, _ = _amr_tree()
    mode = colden.MODE_INSITU if kind == "amr_insitu" else colden.MODE_PREC
    geom = colden.precompute_geometry("healpix", 2, mode=mode)
    a = _eval(tree, geom, precision, timing=False)
    b = _eval(tree, geom, precision, timing=True)
    assert np.all(a[0] > 0) and np.all(a[1] > 0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_callers_stream_sees_the_joined_outputs():
    """Outputs prefilled with -1 are copied on the caller's (non-default)
    stream right after the call, with no synchronisation in between: the copy
    must see the leaves written on the side streams."""
    tree, _ = _amr_tree(nfine=128, base=5)
    geom = colden.precompute_geometry("healpix", 2)
    ref = _eval(tree, geom, colden.BF16, timing=True)
    nd = geom.n_dir
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
        sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
        colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16, stream=st)
        n_copy = n_h.clone()
        s_copy = sh.clone()
    st.synchronize()
    colden.device_status()
    assert np.array_equal(n_copy.cpu().numpy(), ref[0])
    assert np.array_equal(s_copy.cpu().numpy(), ref[1])


def test_back_to_back_updates_on_one_stream():
    """Three density updates and evaluations enqueued on one stream without a
    synchronisation: each evaluation matches a fresh tree of its densities."""
    tree, lv = _amr_tree(seed=23)
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    rng = np.random.default_rng(4)
    rhos = [(lv["rho"] * rng.uniform(0.5, 2.0, size=len(lv["rho"]))).astype(np.float32) for _ in range(3)]
    st = torch.cuda.Stream()
    outs = []
    with torch.cuda.stream(st):
        for r in rhos:
            colden.tree_update(tree, torch.from_numpy(r).cuda(), stream=st)
            n_h = torch.empty(tree.n_leaf * nd, device="cuda")
            colden.column_density(tree, geom, n_h=n_h, precision=colden.BF16, stream=st)
            outs.append(n_h)
    st.synchronize()
    colden.device_status()
    for i, (r, got) in enumerate(zip(rhos, outs)):
        fresh = colden.build_tree_amr(lv["base"], lv["lmax"], 10 * PC, lv["level"], lv["ijk"], r)
        want, _ = _eval(fresh, geom, colden.BF16, timing=False)
        g = got.cpu().numpy()
        bad = np.nonzero(g != want)[0]
        assert len(bad) == 0, (i, len(bad), bad[:8], g[bad[:4]], want[bad[:4]])


def test_new_geometry_serves_another_stream_at_once():
    """cd_precompute_geometry returns with its tables complete: an evaluation
    enqueued right away on a non-blocking stream (not ordered after the
    stream the tables were built on) sees all of them."""
    tree, _ = _amr_tree(seed=29)
    ref_geom = colden.precompute_geometry("healpix", 2)
    ref = _eval(tree, ref_geom, colden.BF16, timing=True)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        geom = colden.precompute_geometry("healpix", 2, stream=torch.cuda.default_stream())
        n_h = torch.full((tree.n_leaf * geom.n_dir,), -1.0, device="cuda")
        colden.column_density(tree, geom, n_h=n_h, precision=colden.BF16, stream=st)
    st.synchronize()
    colden.device_status()
    assert np.array_equal(n_h.cpu().numpy(), ref[0])
