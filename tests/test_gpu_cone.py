"""Cone-averaged geometric factors (CD_MODE_CONE) against the oracle.

The oracle averages its single-ray column over the sub-rays of each
direction's cone; the library averages the geometric factors K over the same
sub-rays once, in FP64, and then runs the unchanged hot path.  The column is
linear in K, so both compute the same quantity; the tolerances are those of the
single-ray paths (FP32 1e-5, BF16 1e-2 relative on N_H).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
RTOL, SHIELD_ATOL = 1e-5, 1e-5
BF16_RTOL, BF16_SHIELD_ATOL = 1e-2, 1e-2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


CUSTOM3 = np.array([[1.0, 2.0, 3.0], [-0.3, 0.1, -1.0], [0.0, 0.7, -0.2]])
DIRSETS = {
    "healpix1": ("healpix", 1, 0, None),
    "healpix2": ("healpix", 2, 0, None),
    "mxn43": ("mxn", 4, 3, None),
    "axes": ("axes", 0, 0, None),
    "custom3": ("custom", 0, 0, CUSTOM3),
    "custom1": ("custom", 0, 0, CUSTOM3[:1]),     # one direction: its cone is the whole sphere
}


def _geom(name, mode=colden.MODE_CONE):
    scheme, p0, p1, d = DIRSETS[name]
    return colden.precompute_geometry(scheme, p0, p1, dirs=d, mode=mode)


def _run(tree, geom, precision=colden.FP32):
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    a_v = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    colden.device_status()
    return [t.double().cpu().numpy() for t in (n_h, a_v, sh)]


def _check(n_h, a_v, sh, ref, sel, nd, rtol, sh_atol):
    g = n_h.reshape(-1, nd)[sel]
    rel = np.abs(g - ref) / ref
    assert rel.max() <= rtol, "max rel N_H err %.3g" % rel.max()
    assert np.max(np.abs(a_v.reshape(-1, nd)[sel] - oracle.a_v(ref)) / oracle.a_v(ref)) <= rtol
    assert np.max(np.abs(sh[sel] - oracle.shield(ref))) <= sh_atol
    assert np.all(np.isfinite(n_h)) and np.all(n_h > 0) and np.all((sh > 0) & (sh <= 1))


@pytest.mark.parametrize("name", list(DIRSETS))
def test_sub_rays_match_oracle(name):
    g = _geom(name)
    assert g.n_sub == oracle.CONE_RINGS * oracle.CONE_AZIMUTHS == 32
    want = oracle.cone_rays(g.dirs)
    assert g.rays.shape == want.shape
    assert np.max(np.abs(g.rays - want)) <= 1e-14
    p = _geom(name, colden.MODE_PREC)
    assert p.n_sub == 1 and np.array_equal(p.rays[:, 0], p.dirs)


@pytest.mark.parametrize("name", list(DIRSETS))
def test_cone_fp32_parity_uniform(name):
    L, box = 4, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=41)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = _geom(name)
    nd = geom.n_dir
    n_h, a_v, sh = _run(tree, geom)
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(1).choice(len(lv), 400 if nd > 12 else len(lv), replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density_cone(geom.dirs, lv[sel], ijk[sel])
    _check(n_h, a_v, sh, ref, sel, nd, RTOL, SHIELD_ATOL)


@pytest.mark.parametrize("nside", [1, 2])
def test_cone_parity_with_the_oracles_own_directions(nside):
    """The oracle builds its HEALPix set independently (last bits may differ);
    the cone frame must not depend on them."""
    L, box = 5, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=47)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = colden.precompute_geometry("healpix", nside, mode=colden.MODE_CONE)
    dirs = oracle.dirs_healpix(nside)
    assert np.max(np.abs(geom.rays - oracle.cone_rays(dirs))) <= 1e-13
    n_h, a_v, sh = _run(tree, geom)
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(6).choice(len(lv), 600, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density_cone(dirs, lv[sel], ijk[sel])
    _check(n_h, a_v, sh, ref, sel, geom.n_dir, RTOL, SHIELD_ATOL)


def test_cone_differs_from_single_ray():
    L, box = 5, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=42)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    cone = _run(tree, _geom("healpix1"))[0]
    ray = _run(tree, _geom("healpix1", colden.MODE_PREC))[0]
    rel = np.abs(cone - ray) / ray
    assert rel.max() > 0.05          # the cone smooths a log-normal field
    assert np.median(rel) < 0.5


@pytest.mark.parametrize("name", ["healpix1", "healpix2", "mxn43", "axes"])
def test_cone_fp32_parity_sampled_6(name):
    """64^3 leaves: several tensor-core-size levels and a deeper prefix chain."""
    L, box = 6, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=43)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = _geom(name)
    n_h, a_v, sh = _run(tree, geom)
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(2).choice(len(lv), 250, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density_cone(geom.dirs, lv[sel], ijk[sel])
    _check(n_h, a_v, sh, ref, sel, geom.n_dir, RTOL, SHIELD_ATOL)


@pytest.mark.parametrize("name", ["healpix1", "healpix2", "mxn43"])
def test_cone_bf16_parity(name):
    L, box = 6, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=44)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = _geom(name)
    n_h, a_v, sh = _run(tree, geom, colden.BF16)
    n32 = _run(tree, geom, colden.FP32)[0]
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(3).choice(len(lv), 250, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density_cone(geom.dirs, lv[sel], ijk[sel])
    _check(n_h, a_v, sh, ref, sel, geom.n_dir, BF16_RTOL, BF16_SHIELD_ATOL)
    assert np.max(np.abs(n_h - n32) / n32) > 1e-5      # the tensor-core path ran


def test_cone_bf16_256cube_sampled():
    """The 256^3, 48-direction workload with cone factors: sampled leaves."""
    L, box = 8, 10 * PC
    rho = synth.lognormal_grf(256, 30.0, 2.0, seed=2)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = _geom("healpix2")
    n_h, _, sh = _run(tree, geom, colden.BF16)
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(4).choice(len(lv), 60, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density_cone(geom.dirs, lv[sel], ijk[sel])
    rel = np.abs(n_h.reshape(-1, 48)[sel] - ref) / ref
    assert rel.max() <= BF16_RTOL, rel.max()
    assert np.max(np.abs(sh[sel] - oracle.shield(ref))) <= BF16_SHIELD_ATOL


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
def test_cone_amr_parity(precision):
    fine = synth.lognormal_grf(64, 30.0, 2.0, seed=17)
    lv = synth.amr_leaves(fine, 4, [40.0, 60.0])
    box = 10 * PC
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    geom = _geom("healpix1")
    n_h, a_v, sh = _run(tree, geom, precision)
    olv, oijk = tree.leaves()
    sel = np.random.default_rng(5).choice(len(olv), min(len(olv), 800), replace=False)
    T = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density_cone(geom.dirs, olv[sel], oijk[sel])
    if precision == colden.FP32:
        _check(n_h, a_v, sh, ref, sel, 12, RTOL, SHIELD_ATOL)
    else:
        _check(n_h, a_v, sh, ref, sel, 12, BF16_RTOL, BF16_SHIELD_ATOL)


def test_cone_noalloc_and_batch_match():
    L, box = 5, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=45)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = _geom("healpix2")
    want = _run(tree, geom)[0]
    n_h = torch.full((tree.n_leaf * 48,), -1.0, device="cuda")
    colden.column_density_noalloc(tree, geom, n_h=n_h)
    torch.cuda.synchronize()
    assert np.array_equal(n_h.double().cpu().numpy(), want)
    n_b = torch.full((tree.n_leaf * 48,), -1.0, device="cuda")
    colden.column_density_batch([tree], [geom], n_h=[n_b])
    torch.cuda.synchronize()
    assert np.array_equal(n_b.double().cpu().numpy(), want)


def test_cone_rejected_by_learned_inputs():
    rho = synth.lognormal_grf(16, 30.0, 2.0, seed=46)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), PC)
    geom = _geom("healpix1")
    x = torch.zeros((tree.n_leaf, 8 * 12 + 1), device="cuda")
    with pytest.raises(colden.ColdenError) as e:
        colden.learned_features(tree, geom, x)
    assert e.value.code == colden.CD_EUNSUPPORTED
