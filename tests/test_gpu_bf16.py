"""Parity of the BF16 tensor-core path (tcgen05 shell contraction) with the
FP64 oracle.

Tolerance: densities and weights are rounded to BF16 (relative 2^-9 each) and
products accumulate in FP32 on the tensor cores; every term of N_H is
positive, so the relative error of N_H is bounded by about 2 x 2^-9 ~ 0.4 %
plus FP32 rounding.  The path is held to 1e-2 relative on N_H and A_V.  The
screening factor changes by at most max_x (x e^-x) x 1e-2 < 3.7e-3 for a 1e-2
relative change of every A_V, so it is held to 5e-3 absolute.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
RTOL = 1e-2
SHIELD_ATOL = 5e-3
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


DIRS = {
    "healpix1": (("healpix", 1, 0, None), lambda: oracle.dirs_healpix(1)),
    "healpix2": (("healpix", 2, 0, None), lambda: oracle.dirs_healpix(2)),
    "mxn58": (("mxn", 5, 8, None), lambda: oracle.dirs_mxn(5, 8)),
    "custom8": (("custom", 0, 0, np.random.default_rng(4).normal(size=(8, 3))),
                lambda: oracle.dirs_custom(np.random.default_rng(4).normal(size=(8, 3)))),
    "axes": (("axes", 0, 0, None), lambda: oracle.dirs_axes()),
}


def _geom(name):
    (scheme, p0, p1, d), ref = DIRS[name]
    return colden.precompute_geometry(scheme, p0, p1, dirs=d), ref()


def _morton(ijk):
    m = np.zeros(len(ijk), dtype=np.int64)
    for b in range(21):
        for a in range(3):
            m |= ((ijk[:, a] >> b) & 1) << (3 * b + a)
    return m


def _run(tree, geom, precision):
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    a_v = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    colden.device_status()
    return [t.double().cpu().numpy() for t in (n_h, a_v, sh)]


@pytest.mark.parametrize("L", [4, 5, 6])
@pytest.mark.parametrize("dset", ["healpix1", "healpix2", "mxn58", "custom8", "axes"])
def test_bf16_parity_full(L, dset):
    box = 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=200 + L)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom(dset)
    nd = geom.n_dir
    n_h, a_v, sh = _run(tree, geom, colden.BF16)
    lv, ijk = tree.leaves()
    if L == 6:   # 262144 leaves: compare a seeded sample, properties everywhere
        sel = np.random.default_rng(L).choice(len(lv), 3000, replace=False)
    else:
        sel = np.arange(len(lv))
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, lv[sel], ijk[sel])
    g = n_h.reshape(-1, nd)[sel]
    rel = np.abs(g - ref) / ref
    assert rel.max() <= RTOL, rel.max()
    assert np.max(np.abs(a_v.reshape(-1, nd)[sel] - oracle.a_v(ref)) / oracle.a_v(ref)) <= RTOL
    assert np.max(np.abs(sh[sel] - oracle.shield(ref))) <= SHIELD_ATOL
    assert np.all(n_h > 0) and np.all(np.isfinite(n_h)) and np.all((sh > 0) & (sh <= 1))


def test_bf16_differs_from_fp32_but_within_tolerance():
    """The BF16 form really is a different arithmetic (not the FP32 kernel)."""
    L, box = 6, 10 * PC
    rho = synth.lognormal_grf(64, 30.0, 2.0, seed=9)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, _ = _geom("healpix2")
    a = _run(tree, geom, colden.FP32)[0]
    b = _run(tree, geom, colden.BF16)[0]
    rel = np.abs(a - b) / a
    assert rel.max() > 1e-5          # rounded to BF16 somewhere
    assert rel.max() <= RTOL


@pytest.mark.parametrize("dset", ["healpix1", "healpix2", "mxn58", "custom8"])
def test_bf16_parity_128cube(dset):
    """128^3 leaves: the oct level (k = 6) and the level above take the
    TMA-fed tensor-core shell kernel; every leaf against the FP32 path,
    sampled leaves against the oracle."""
    L, box = 7, 10 * PC
    rho = synth.lognormal_grf(128, 30.0, 2.0, seed=300)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom(dset)
    nd = geom.n_dir
    n_h, _, sh = _run(tree, geom, colden.BF16)
    n32, _, sh32 = _run(tree, geom, colden.FP32)
    rel = np.abs(n_h - n32) / n32
    assert rel.max() <= RTOL, rel.max()
    assert np.max(np.abs(sh - sh32)) <= SHIELD_ATOL
    lv, ijk = tree.leaves()
    sel = np.random.default_rng(7).choice(len(lv), 400, replace=False)
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, lv[sel], ijk[sel])
    assert np.max(np.abs(n_h.reshape(-1, nd)[sel] - ref) / ref) <= RTOL


def test_bf16_parity_256cube_sampled():
    """256^3 leaves, 10 pc, k^-11/3 log-normal (mean 30, sigma_ln 2, seed 2),
    48 HEALPix directions: the full-size launch, sampled leaves vs the oracle."""
    L, box = 8, 10 * PC
    rho = synth.lognormal_grf(256, 30.0, 2.0, seed=2)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom("healpix2")
    n_h, _, sh = _run(tree, geom, colden.BF16)
    rng = np.random.default_rng(5)
    ijk = np.concatenate([rng.integers(0, 256, size=(150, 3)),
                          np.array([[x, y, z] for x in (0, 255) for y in (0, 255) for z in (0, 255)])])
    rows = _morton(ijk)
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, np.full(len(ijk), L), ijk)
    nd = geom.n_dir
    rel = np.abs(n_h.reshape(-1, nd)[rows] - ref) / ref
    assert rel.max() <= RTOL, rel.max()
    assert np.max(np.abs(sh[rows] - oracle.shield(ref))) <= SHIELD_ATOL
