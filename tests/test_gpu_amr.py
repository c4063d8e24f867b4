"""AMR octrees through the C ABI against the FP64 oracle.

Tolerance as for the uniform FP32 path: 1e-5 relative on N_H and A_V, 1e-5
absolute on the screening factor (the same positive-sum rounding argument).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
RTOL = 1e-5
SHIELD_ATOL = 1e-5
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _mesh(nfine=32, base=3, thr=(40.0, 60.0), seed=7):
    fine = synth.lognormal_grf(nfine, 30.0, 2.0, seed=seed)
    return synth.amr_leaves(fine, base, list(thr))


def _run(tree, geom, precision=colden.FP32):
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    a_v = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    colden.device_status()
    return [t.double().cpu().numpy() for t in (n_h, a_v, sh)]


@pytest.mark.parametrize("dset", [("healpix", 1, 0), ("healpix", 2, 0), ("mxn", 5, 8), ("axes", 0, 0)])
def test_amr_parity_all_leaves(dset):
    lv = _mesh()
    box = 10 * PC
    assert len(np.unique(lv["level"])) == 3
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry(dset[0], dset[1], dset[2])
    nd = geom.n_dir
    n_h, a_v, sh = _run(tree, geom)
    olv, oijk = tree.leaves()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density(geom.dirs, olv, oijk)
    rel = np.abs(n_h.reshape(-1, nd) - ref) / ref
    assert rel.max() <= RTOL, rel.max()
    assert np.max(np.abs(a_v.reshape(-1, nd) - oracle.a_v(ref)) / oracle.a_v(ref)) <= RTOL
    assert np.max(np.abs(sh - oracle.shield(ref))) <= SHIELD_ATOL


def test_amr_output_order_is_depth_first_and_complete():
    lv = _mesh()
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"], lv["ijk"], lv["rho"])
    olv, oijk = tree.leaves()
    assert tree.n_leaf == len(lv["level"])
    fine = np.zeros(len(olv), dtype=np.int64)
    for b in range(lv["lmax"]):
        for a in range(3):
            fine |= ((oijk[:, a].astype(np.int64) >> b) & 1) << (3 * b + a)
    fine <<= 3 * (lv["lmax"] - olv.astype(np.int64))
    assert np.all(np.diff(fine) > 0)
    got = set(zip(olv.tolist(), map(tuple, oijk.tolist())))
    want = set(zip(lv["level"].tolist(), map(tuple, lv["ijk"].tolist())))
    assert got == want


def test_amr_leaf_order_of_the_caller_does_not_matter():
    lv = _mesh(seed=8)
    perm = np.random.default_rng(1).permutation(len(lv["level"]))
    geom = colden.precompute_geometry("healpix", 1)
    a = colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"], lv["ijk"], lv["rho"])
    b = colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"][perm], lv["ijk"][perm], lv["rho"][perm])
    assert np.array_equal(a.leaves()[1], b.leaves()[1])
    for x, y in zip(_run(a, geom), _run(b, geom)):
        assert np.array_equal(x, y)


def test_amr_uniform_leaf_set_matches_uniform_tree():
    rho = synth.lognormal_iid(16, 10.0, 1.5, seed=3)
    ijk = oracle.morton_ijk(4)
    r = rho[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    geom = colden.precompute_geometry("healpix", 2)
    amr = colden.build_tree_amr(4, 4, PC, np.full(len(r), 4), ijk, r)
    uni = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), PC)
    assert np.array_equal(amr.leaves()[1], uni.leaves()[1])
    a, b = _run(amr, geom), _run(uni, geom)
    assert np.max(np.abs(a[0] - b[0]) / b[0]) <= 1e-6
    assert np.max(np.abs(a[2] - b[2])) <= 1e-6


def test_amr_update_matches_rebuild():
    lv = _mesh(seed=9)
    geom = colden.precompute_geometry("healpix", 2)
    r2 = (lv["rho"] * np.random.default_rng(2).uniform(0.5, 2.0, size=len(lv["rho"]))).astype(np.float32)
    t = colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"], lv["ijk"], lv["rho"])
    _run(t, geom)
    colden.tree_update(t, torch.from_numpy(r2).cuda())
    a = _run(t, geom)
    b = _run(colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"], lv["ijk"], r2), geom)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_amr_rejects_bad_leaf_sets():
    lv = _mesh()
    with pytest.raises(colden.ColdenError):          # gap
        colden.build_tree_amr(lv["base"], lv["lmax"], PC, lv["level"][1:], lv["ijk"][1:], lv["rho"][1:])
    dl = np.concatenate([lv["level"], lv["level"][:1]])
    di = np.concatenate([lv["ijk"], lv["ijk"][:1]])
    dr = np.concatenate([lv["rho"], lv["rho"][:1]])
    with pytest.raises(colden.ColdenError):          # overlap
        colden.build_tree_amr(lv["base"], lv["lmax"], PC, dl, di, dr)
    with pytest.raises(colden.ColdenError):          # level outside [base, lmax]
        colden.build_tree_amr(lv["base"] + 1, lv["lmax"], PC, lv["level"], lv["ijk"], lv["rho"])


def test_amr_1024_effective_sampled():
    """AMR config: base 128^3 in a 20 pc box, 3 extra levels refined where the
    block mean exceeds 10^(2+l) cm^-3 on a seeded k^-11/3 log-normal field
    (mean 30, sigma_ln 2, seed 2) at 1024^3 resolution, 48 HEALPix directions;
    sampled leaves of every level vs the oracle."""
    lv = synth.amr_leaves_grf_torch(10, 7, [1e2, 1e3, 1e4], 30.0, 2.0, seed=2)
    torch.cuda.empty_cache()
    box = 20 * PC
    counts = np.bincount(lv["level"], minlength=11)[7:]
    assert np.all(counts > 0), counts
    tree = colden.build_tree_amr(7, 10, box, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    n_h = torch.empty(tree.n_leaf * nd, device="cuda")
    sh = torch.empty(tree.n_leaf, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, shield=sh)
    colden.device_status()
    olv, oijk = tree.leaves()
    rng = np.random.default_rng(3)
    sel = np.concatenate([rng.choice(np.nonzero(olv == l)[0], 40) for l in range(7, 11)])
    T = oracle.Tree.amr(7, 10, box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density(geom.dirs, olv[sel], oijk[sel])
    got = n_h.reshape(-1, nd)[torch.from_numpy(sel).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) <= RTOL
    assert np.max(np.abs(sh[torch.from_numpy(sel).cuda()].double().cpu().numpy() - oracle.shield(ref))) <= SHIELD_ATOL


# BF16 tensor-core contraction over the AMR receiver lists (levels >= 4); the
# tolerance of the uniform BF16 path: 1e-2 relative on N_H (BF16 densities and
# weights, FP32 accumulation of positive terms), 5e-3 on the screening factor.
BF16_RTOL = 1e-2
BF16_SHIELD_ATOL = 5e-3


@pytest.mark.parametrize("dset", [("healpix", 1, 0), ("healpix", 2, 0), ("mxn", 4, 4)])
def test_amr_bf16_parity_all_leaves(dset):
    fine = synth.lognormal_grf(64, 30.0, 2.0, seed=17)
    lv = synth.amr_leaves(fine, 4, [40.0, 60.0])
    box = 10 * PC
    assert len(np.unique(lv["level"])) == 3
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry(dset[0], dset[1], dset[2])
    nd = geom.n_dir
    n_h, a_v, sh = _run(tree, geom, precision=colden.BF16)
    n32, _, _ = _run(tree, geom, precision=colden.FP32)
    olv, oijk = tree.leaves()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density(geom.dirs, olv, oijk)
    rel = np.abs(n_h.reshape(-1, nd) - ref) / ref
    assert rel.max() <= BF16_RTOL, rel.max()
    assert np.max(np.abs(sh - oracle.shield(ref))) <= BF16_SHIELD_ATOL
    # the tensor cores did run (BF16 rounding differs from the FP32 path)
    assert np.max(np.abs(n_h - n32) / n32) > 1e-5


def test_amr_bf16_1024_effective_sampled():
    lv = synth.amr_leaves_grf_torch(10, 7, [1e2, 1e3, 1e4], 30.0, 2.0, seed=2)
    torch.cuda.empty_cache()
    box = 20 * PC
    tree = colden.build_tree_amr(7, 10, box, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry("healpix", 2)
    nd = geom.n_dir
    n_h = torch.empty(tree.n_leaf * nd, device="cuda")
    sh = torch.empty(tree.n_leaf, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16)
    colden.device_status()
    olv, oijk = tree.leaves()
    rng = np.random.default_rng(4)
    sel = np.concatenate([rng.choice(np.nonzero(olv == l)[0], 40) for l in range(7, 11)])
    T = oracle.Tree.amr(7, 10, box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density(geom.dirs, olv[sel], oijk[sel])
    got = n_h.reshape(-1, nd)[torch.from_numpy(sel).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) <= BF16_RTOL
    assert np.max(np.abs(sh[torch.from_numpy(sel).cuda()].double().cpu().numpy() - oracle.shield(ref))) <= BF16_SHIELD_ATOL


def _mesh3():
    """Three refined levels above a 16^3 base (128^3 effective): the two
    finest dense levels are filled only where read (the rest of the level
    below the finest holds NaN), so any read outside the painted part would
    show as a non-finite column."""
    fine = synth.lognormal_grf(128, 30.0, 2.0, seed=23)
    lv = synth.amr_leaves(fine, 4, [35.0, 55.0, 80.0])
    assert len(np.unique(lv["level"])) == 4
    return lv


@pytest.mark.parametrize("precision,mode", [(colden.FP32, "prec"), (colden.BF16, "prec"), (colden.FP32, "insitu"),
                                            (colden.FP32, "cone")])
def test_amr_three_refined_levels_all_leaves(precision, mode):
    lv = _mesh3()
    box = 10 * PC
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    gmode = {"prec": colden.MODE_PREC, "insitu": colden.MODE_INSITU, "cone": colden.MODE_CONE}[mode]
    geom = colden.precompute_geometry("healpix", 1, mode=gmode)
    nd = geom.n_dir
    n_h, a_v, sh = _run(tree, geom, precision=precision)
    assert np.all(np.isfinite(n_h)) and np.all(np.isfinite(sh))
    olv, oijk = tree.leaves()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    if mode == "cone":
        sel = np.sort(np.random.default_rng(5).choice(tree.n_leaf, 400, replace=False))
        ref = T.column_density_cone(geom.dirs, olv[sel], oijk[sel])
        got = n_h.reshape(-1, nd)[sel]
    else:
        ref = T.column_density(geom.dirs, olv, oijk, mode=oracle.MODE_INSITU if mode == "insitu" else oracle.MODE_PREC)
        got = n_h.reshape(-1, nd)
    tol = RTOL if precision == colden.FP32 or mode == "insitu" else BF16_RTOL
    assert np.max(np.abs(got - ref) / ref) <= tol
    # an update to new densities gives the rebuilt tree's columns bit for bit
    r2 = (lv["rho"] * np.random.default_rng(6).uniform(0.5, 2.0, size=len(lv["rho"]))).astype(np.float32)
    colden.tree_update(tree, torch.from_numpy(r2).cuda())
    a = _run(tree, geom, precision=precision)
    b = _run(colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], r2), geom,
             precision=precision)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_amr_bf16_parent_rows_staged_per_oct_give_the_same_columns():
    """The BF16 leaf kernel stages the parents' prefix rows of a list tile as
    one span (the common case) or one row per oct (spans wider than 16 rows);
    forcing the per-oct form everywhere changes no bit."""
    lv = _mesh3()
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], 10 * PC, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry("healpix", 2)
    a = _run(tree, geom, precision=colden.BF16)
    colden.debug_leaf_span(0)
    try:
        b = _run(tree, geom, precision=colden.BF16)
    finally:
        colden.debug_leaf_span(-1)
    c = _run(tree, geom, precision=colden.BF16)
    for x, y, z in zip(a, b, c):
        assert np.array_equal(x, y) and np.array_equal(x, z)
