"""Parity of the FP32 CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (FP32 path): every N_H is a sum of 30..200 positive terms, each a
product of an FP32 density (itself a mean of FP32 values) and an FP32-rounded
FP64 path length, accumulated in FP32.  The relative rounding error of such a
sum is below n * 2^-24 ~ 1.2e-5 in the worst case and ~1e-6 in practice, so
N_H and A_V are held to 1e-5 relative.  shield is a mean of exp(-2.5 A_V);
its error is at most max_x (x e^-x) * 1e-5 < 4e-6 plus the exp rounding, so
it is held to 1e-5 absolute.
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


DIRSETS = {
    "healpix1": (("healpix", 1, 0, None), lambda: oracle.dirs_healpix(1)),
    "healpix2": (("healpix", 2, 0, None), lambda: oracle.dirs_healpix(2)),
    "mxn58": (("mxn", 5, 8, None), lambda: oracle.dirs_mxn(5, 8)),
    "mxn712": (("mxn", 7, 12, None), lambda: oracle.dirs_mxn(7, 12)),
    "axes": (("axes", 0, 0, None), lambda: oracle.dirs_axes()),
    "custom7": (("custom", 0, 0, np.random.default_rng(3).normal(size=(7, 3))),
                lambda: oracle.dirs_custom(np.random.default_rng(3).normal(size=(7, 3)))),
}


def _geom(name):
    (scheme, p0, p1, d), ref = DIRSETS[name]
    return colden.precompute_geometry(scheme, p0, p1, dirs=d), ref()


def _run(tree, geom, precision=colden.FP32, want=("n_h", "a_v", "shield")):
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda") if "n_h" in want else None
    a_v = torch.full((tree.n_leaf * nd,), -1.0, device="cuda") if "a_v" in want else None
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda") if "shield" in want else None
    colden.column_density(tree, geom, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    torch.cuda.synchronize()
    f = lambda t: None if t is None else t.cpu().numpy().astype(np.float64)
    return f(n_h), f(a_v), f(sh)


def _compare(got_nh, got_av, got_sh, ref, nd, rtol=RTOL, sh_atol=SHIELD_ATOL):
    g = got_nh.reshape(-1, nd)
    rel = np.abs(g - ref) / ref
    assert np.all(np.isfinite(g))
    assert rel.max() <= rtol, "max rel N_H err %.3g at %s" % (rel.max(), np.unravel_index(rel.argmax(), rel.shape))
    if got_av is not None:
        av_ref = oracle.a_v(ref)
        assert np.max(np.abs(got_av.reshape(-1, nd) - av_ref) / av_ref) <= rtol
    if got_sh is not None:
        assert np.max(np.abs(got_sh - oracle.shield(ref))) <= sh_atol


def test_leaf_order_is_morton():
    for L in (1, 3, 5):
        rho = np.ones((1 << L,) * 3, np.float32)
        t = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), 1.0)
        lv, ijk = t.leaves()
        assert np.all(lv == L)
        assert np.array_equal(ijk, oracle.morton_ijk(L))
        assert t.n_leaf == 8 ** L and t.n_oct == 8 ** (L - 1)


@pytest.mark.parametrize("name", list(DIRSETS))
def test_directions_match_oracle(name):
    g, ref = _geom(name)
    assert g.n_dir == ref.shape[0]
    assert np.allclose(g.dirs, ref, rtol=0, atol=1e-15)


@pytest.mark.parametrize("L", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dset", ["healpix1", "axes", "mxn58", "custom7"])
def test_fp32_parity_small_trees(L, dset):
    box = 10 * PC
    rho = synth.lognormal_iid(1 << L, 10.0, 1.5, seed=100 + L)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom(dset)
    n_h, a_v, sh = _run(tree, geom)
    lv, ijk = tree.leaves()
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, lv, ijk)
    _compare(n_h, a_v, sh, ref, geom.n_dir)


def test_fp32_parity_32cube_full():
    """32^3 uniform leaves in a 10 pc box, i.i.d. log-normal (mean 10, sigma_ln
    1.5, seed 1), 12 HEALPix directions: every leaf and direction."""
    L, box = 5, 10 * PC
    rho = synth.lognormal_iid(32, 10.0, 1.5, seed=1)
    tree = colden.build_tree_uniform(rho, box)        # host path
    geom, dirs = _geom("healpix1")
    n_h, a_v, sh = _run(tree, geom)
    lv, ijk = tree.leaves()
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, lv, ijk)
    _compare(n_h, a_v, sh, ref, geom.n_dir)


def _sample_leaves(L, n, seed):
    """Random leaves plus the eight box corners and a few face/edge cells."""
    rng = np.random.default_rng(seed)
    m = (1 << L) - 1
    ijk = rng.integers(0, m + 1, size=(n, 3))
    corners = np.array([[x, y, z] for x in (0, m) for y in (0, m) for z in (0, m)])
    faces = np.array([[0, m // 2, m // 3], [m, 1, m // 2], [m // 2, 0, m], [1, m, 0]])
    return np.concatenate([ijk, corners, faces]).astype(np.int64)


def _morton(ijk):
    m = np.zeros(len(ijk), dtype=np.int64)
    for b in range(21):
        for a in range(3):
            m |= ((ijk[:, a] >> b) & 1) << (3 * b + a)
    return m


def test_fp32_parity_256cube_sampled():
    """256^3 leaves (levels 0..8), 10 pc, k^-11/3 log-normal field (mean 30,
    sigma_ln 2, seed 2), 48 HEALPix directions: the full-size launch, checked
    on sampled leaves (corners, faces, random) one by one against the oracle."""
    L, box = 8, 10 * PC
    rho = synth.lognormal_grf(256, 30.0, 2.0, seed=2)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom("healpix2")
    n_h, a_v, sh = _run(tree, geom, want=("n_h", "shield"))
    ijk = _sample_leaves(L, 120, seed=5)
    rows = _morton(ijk)
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, np.full(len(ijk), L), ijk)
    nd = geom.n_dir
    _compare(n_h.reshape(-1, nd)[rows].ravel(), None, sh[rows], ref, nd)
    # properties at every leaf: positive, finite, shield in (0, 1]
    assert np.all(n_h > 0) and np.all(np.isfinite(n_h))
    assert np.all((sh > 0) & (sh <= 1))


def test_tree_update_matches_rebuild():
    L, box = 5, 3 * PC
    r1 = synth.lognormal_iid(32, 10.0, 1.5, seed=7)
    r2 = synth.lognormal_grf(32, 30.0, 2.0, seed=8)
    geom, _ = _geom("healpix2")
    t = colden.build_tree_uniform(torch.from_numpy(r1).cuda(), box)
    _run(t, geom)
    colden.tree_update(t, torch.from_numpy(r2).cuda().reshape(-1))
    a = _run(t, geom)
    b = _run(colden.build_tree_uniform(r2, box), geom)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("offset", [1, 2])
def test_unaligned_density_input_matches_aligned(offset):
    """A device density array that starts 4 or 8 bytes past an allocation
    (the restriction reads pairs of leaves when the array is 8-byte aligned)."""
    L, box = 5, 3 * PC
    rho = synth.lognormal_grf(32, 30.0, 2.0, seed=13)
    geom, _ = _geom("healpix1")
    want = _run(colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box), geom)
    buf = torch.zeros(rho.size + offset, device="cuda")
    buf[offset:] = torch.from_numpy(rho).cuda().reshape(-1)
    t = colden.build_tree_uniform(buf[offset:].reshape(rho.shape), box)
    got = _run(t, geom)
    for x, y in zip(got, want):
        assert np.array_equal(x, y)
    colden.tree_update(t, buf[offset:])
    for x, y in zip(_run(t, geom), want):
        assert np.array_equal(x, y)


def test_only_requested_outputs_written_and_launches_counted():
    L = 4
    rho = synth.lognormal_iid(16, 10.0, 1.5, seed=9)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), PC)
    geom, _ = _geom("healpix1")
    colden.stats_reset(timing=True)
    n_h, a_v, sh = _run(tree, geom, want=("shield",))
    assert n_h is None and a_v is None and np.all(sh > 0)
    n_shell, ms_shell = colden.stats_get(colden.K_SHELL)
    n_leaf, ms_leaf = colden.stats_get(colden.K_LEAF)
    assert n_shell == 1 and n_leaf == 1 and ms_leaf > 0
    colden.stats_reset(timing=False)


@pytest.mark.parametrize("offset", [0, 1])
def test_unaligned_outputs_take_the_generic_kernel(offset):
    L, box = 4, 2 * PC
    rho = synth.lognormal_grf(16, 30.0, 2.0, seed=12)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom, dirs = _geom("healpix1")
    nd = geom.n_dir
    buf = torch.full((tree.n_leaf * nd + 4,), -1.0, device="cuda")
    sbuf = torch.full((tree.n_leaf + 4,), -1.0, device="cuda")
    n_h, sh = buf[offset:offset + tree.n_leaf * nd], sbuf[offset:offset + tree.n_leaf]
    colden.column_density(tree, geom, n_h=n_h, shield=sh)
    colden.device_status()
    lv, ijk = tree.leaves()
    ref = oracle.Tree.uniform(rho, box).column_density(dirs, lv, ijk)
    _compare(n_h.double().cpu().numpy(), None, sh.double().cpu().numpy(), ref, nd)
    assert buf[:offset].eq(-1).all() and buf[offset + tree.n_leaf * nd:].eq(-1).all()


def test_invalid_arguments_rejected():
    with pytest.raises(colden.ColdenError):
        colden.precompute_geometry("mxn", 0, 4)
    with pytest.raises(colden.ColdenError):
        colden.precompute_geometry("custom", dirs=np.zeros((2, 3)))
    bad = np.ones((8, 8, 8), np.float32)
    bad[1, 2, 3] = -1.0
    with pytest.raises(colden.ColdenError):
        colden.build_tree_uniform(bad, PC)
    bad[1, 2, 3] = np.nan
    with pytest.raises(colden.ColdenError):
        colden.build_tree_uniform(bad, PC)
