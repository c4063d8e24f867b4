"""Edge cases of the path: the degenerate all-zero field, the largest uniform
tree and the deepest AMR tree the API accepts.

A box with no gas has no column in any direction (Eq. N_discret sums
densities times path lengths): N_H and A_V are exactly zero and the screening
factor exactly one, in both precisions.  The largest uniform tree
(leaf level 10, 1024^3 leaves, 12 HEALPix directions) runs the whole path at
full size, every index at its widest (30-bit Morton keys, 2^30 leaves x 12
directions = 1.3e10 outputs), checked against the FP64 oracle on sampled leaves
including the eight box corners, at the FP32 (1e-5) and BF16 (1e-2) tolerances."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

pytestmark = pytest.mark.gpu
PC = synth.PC_CM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _morton(ijk):
    m = np.zeros(len(ijk), dtype=np.int64)
    for b in range(21):
        for a in range(3):
            m |= ((ijk[:, a].astype(np.int64) >> b) & 1) << (3 * b + a)
    return m


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
@pytest.mark.parametrize("L", [2, 5])
def test_empty_box_has_no_column(precision, L):
    g = colden.precompute_geometry("healpix", 2)
    t = colden.build_tree_uniform(torch.zeros((1 << L,) * 3, device="cuda"), 10 * PC)
    nd = g.n_dir
    n_h = torch.full((t.n_leaf * nd,), -1.0, device="cuda")
    a_v = torch.full_like(n_h, -1.0)
    sh = torch.full((t.n_leaf,), -1.0, device="cuda")
    colden.column_density(t, g, n_h=n_h, a_v=a_v, shield=sh, precision=precision)
    torch.cuda.synchronize()
    colden.device_status()
    assert torch.all(n_h == 0) and torch.all(a_v == 0) and torch.all(sh == 1)
    t.free()
    g.free()


def test_largest_tree_1024cube_sampled():
    L, box = 10, 10 * PC
    rho_d = synth.lognormal_grf_torch(1 << L, 30.0, 2.0, 7, device="cuda").contiguous()
    t = colden.build_tree_uniform(rho_d, box)
    assert t.n_leaf == 1 << 30 and t.max_level == L
    rho = rho_d.cpu().numpy()
    del rho_d
    torch.cuda.empty_cache()
    g = colden.precompute_geometry("healpix", 1)
    nd = g.n_dir
    rng = np.random.default_rng(9)
    ijk = np.concatenate([rng.integers(0, 1 << L, size=(150, 3)),
                          np.array([[x, y, z] for x in (0, 1023) for y in (0, 1023) for z in (0, 1023)])])
    rows = torch.from_numpy(_morton(ijk)).cuda()
    ref = oracle.Tree.uniform(rho, box).column_density(oracle.dirs_healpix(1), np.full(len(ijk), L), ijk)
    del rho
    n_h = torch.empty(t.n_leaf * nd, device="cuda")
    sh = torch.empty(t.n_leaf, device="cuda")
    for precision, rtol, satol in ((colden.BF16, 1e-2, 5e-3), (colden.FP32, 1e-5, 1e-5)):
        n_h.fill_(-1.0)
        colden.column_density(t, g, n_h=n_h, shield=sh, precision=precision)
        torch.cuda.synchronize()
        colden.device_status()
        got = n_h.view(-1, nd)[rows].double().cpu().numpy()
        rel = np.abs(got - ref) / ref
        assert rel.max() <= rtol, (precision, rel.max())
        assert np.max(np.abs(sh[rows].double().cpu().numpy() - oracle.shield(ref))) <= satol
    t.free()
    g.free()


def _cascade(base, lmax, point, seed):
    """Leaves of a tree refined cell by cell around one point: at every level
    from base to lmax - 1 the cell containing `point` (fractions of the box)
    is split, every other cell of the level is a leaf; densities i.i.d.
    log-normal."""
    levels, ijks = [], []
    for l in range(base, lmax + 1):
        n = 1 << l
        here = [int(p * n) for p in point]
        if l == base:
            cells = [(i, j, k) for k in range(n) for j in range(n) for i in range(n)]
        else:
            up = [2 * c for c in prev]
            cells = [(up[0] + (o & 1), up[1] + ((o >> 1) & 1), up[2] + (o >> 2)) for o in range(8)]
        for c in cells:
            if l < lmax and list(c) == here:
                continue
            levels.append(l)
            ijks.append(c)
        prev = here
    rng = np.random.default_rng(seed)
    rho = np.exp(rng.normal(np.log(10.0), 1.5, size=len(levels))).astype(np.float32)
    return np.array(levels, np.int8), np.array(ijks, np.int32), rho


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
def test_deepest_amr_tree_all_leaves(precision):
    """The deepest AMR tree the API accepts (max_level 11, a 2048^3-effective
    finest cell) refined around one point from an 8^3 base: every leaf against
    the oracle."""
    base, lmax, box = 3, 11, 10 * PC
    lvl, ijk, rho = _cascade(base, lmax, (0.31, 0.62, 0.47), seed=21)
    t = colden.build_tree_amr(base, lmax, box, lvl, ijk, rho)
    assert t.max_level == lmax and t.n_leaf == len(lvl)
    g = colden.precompute_geometry("healpix", 2)
    nd = g.n_dir
    n_h = torch.full((t.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((t.n_leaf,), -1.0, device="cuda")
    colden.column_density(t, g, n_h=n_h, shield=sh, precision=precision)
    torch.cuda.synchronize()
    colden.device_status()
    olv, oijk = t.leaves()
    ref = oracle.Tree.amr(base, lmax, box, lvl, ijk, rho).column_density(oracle.dirs_healpix(2), olv, oijk)
    rtol, satol = (1e-5, 1e-5) if precision == colden.FP32 else (1e-2, 5e-3)
    rel = np.abs(n_h.view(-1, nd).double().cpu().numpy() - ref) / ref
    assert rel.max() <= rtol, rel.max()
    assert np.max(np.abs(sh.double().cpu().numpy() - oracle.shield(ref))) <= satol
    t.free()
    g.free()
