"""The spherical-cloud test of §4.1 (Table 2, spherical cloud columns) on the
GPU path: a uniform sphere (R = 12.5 pc, n = 1000 cm^-3) in a 50 pc box of
10 cm^-3, refined on density to 512^3 effective (base 128^3, two AMR levels).
The extinction maps chi = <exp(-sigma N)> (Eqs. eq_chi, eq_tau, chi_discret,
sigma = 2e-21 cm^2) of the cells of the three midplanes from the tree method
(FP32, AMR lists) are compared pixel by pixel (512^2 per plane) with the
exact ray-marcher from each pixel cell, Delta chi = |chi - chi_ref| (Eq. eq2).

The paper's reference traced 50 rays; here the reference uses the tree's own
directions (the only difference left is the tree approximation), so the means
come out below the printed ones (they also carry the angular sampling of the
reference), most of all for the six axis rays, which here are exact
one-dimensional sums up to the coarse-level averaging.  The largest
differences sit at the sphere's edge and are the tree's own: for 12, 40 and 84
directions they match the printed maxima to within a factor 1.5 (measured
0.086, 0.067, 0.067 against 0.094, 0.068, 0.090).  Required: every mean below
the printed mean and below 0.05, every maximum below 0.25 and below the printed
maximum for six rays, and the 12/40/84-direction maxima within a factor 1.5 of
the printed ones."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
SIGMA = 2e-21
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table2_sphere_dchi.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _table2():
    out = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            n, mean, mx = line.split()
            out[int(n)] = (float(mean), float(mx))
    return out


def _spread(v):
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b)
    return out


def _plane_maps(olv, oijk, lmax=9):
    """For each midplane (x, y, z = half the box): the index of the leaf that
    holds each level-lmax cell just above the plane, [512, 512]."""
    side = 1 << lmax
    half = side // 2
    maps = []
    for axis in range(3):
        a, b = [q for q in range(3) if q != axis]
        m = np.full((side, side), -1, dtype=np.int64)
        for l in np.unique(olv):
            s = 1 << (lmax - int(l))
            sel = np.flatnonzero((olv == l) & (oijk[:, axis] == half // s))
            if sel.size == 0:
                continue
            d = np.arange(s)
            zero = np.zeros((1, s, s), dtype=np.int64)
            A = (oijk[sel, a][:, None, None] * s + d[None, :, None] + zero).reshape(-1)
            B = (oijk[sel, b][:, None, None] * s + d[None, None, :] + zero).reshape(-1)
            m[A, B] = np.repeat(sel, s * s)
        assert np.all(m >= 0)
        maps.append(m)
    return maps


def _pixel_cells(lmax=9):
    side = 1 << lmax
    half = side // 2
    u, v = np.meshgrid(np.arange(side), np.arange(side), indexing="ij")
    u, v = u.reshape(-1), v.reshape(-1)
    h = np.full_like(u, half)
    cells = []
    for axis in range(3):
        ijk = [None, None, None]
        a, b = [q for q in range(3) if q != axis]
        ijk[axis], ijk[a], ijk[b] = h, u, v
        cells.append((_spread(ijk[0]) | (_spread(ijk[1]) << np.uint64(1)) | (_spread(ijk[2]) << np.uint64(2))).astype(np.int64))
    return cells


SETS = {6: ("axes", 0, 0), 12: ("mxn", 3, 4), 40: ("mxn", 5, 8), 84: ("mxn", 7, 12)}
BOX, RADIUS = 50 * PC, 12.5 * PC


def _oracle_dirs(scheme, p0, p1):
    return oracle.dirs_axes() if scheme == "axes" else oracle.dirs_mxn(p0, p1)


@pytest.fixture(scope="module")
def sphere_mesh():
    """The §4.1 cloud: the fine 512^3 field, its AMR leaves (base 128^3, two
    refined levels where the block mean exceeds 10.5 cm^-3, i.e. every block
    touching the sphere), the library's AMR tree and the uniform 512^3 tree the
    ray-marcher walks."""
    fine = synth.sphere(512, BOX, RADIUS, 1000.0, 10.0)
    lv = synth.amr_leaves(fine, 7, [10.5, 10.5])
    tree = colden.build_tree_amr(7, 9, BOX, lv["level"], lv["ijk"], lv["rho"])
    uni = colden.build_tree_uniform(torch.from_numpy(fine).cuda(), BOX)
    return lv, tree, uni


def test_sphere_mesh_columns_match_oracle(sphere_mesh):
    """The tree-method columns of the spherical-cloud mesh (FP32, AMR lists)
    and the exact ray-marcher's columns from the map's pixel cells, against the
    FP64 oracle on the same mesh and the same M x N / axis direction sets of
    Table 2: 1e-5 relative on N_H (the FP32 parity tolerance) and 2e-5 on the
    ray-marcher (FP32 sums over up to 1.5 x 512 cell crossings).  Sampled: 300
    pixel cells spread over the three midplanes, plus pixels at the sphere's
    edge, where the maxima of Table 2 sit."""
    lv, tree, uni = sphere_mesh
    T = oracle.Tree.amr(lv["base"], lv["lmax"], BOX, lv["level"], lv["ijk"], lv["rho"])
    olv, oijk = tree.leaves()
    maps = _plane_maps(olv, oijk)
    cells = _pixel_cells()
    rng = np.random.default_rng(21)
    half = 256
    u, v = np.meshgrid(np.arange(512), np.arange(512), indexing="ij")
    r_pix = np.hypot(u + 0.5 - half, v + 0.5 - half).reshape(-1)   # pixel distance (cells) from the sphere's axis
    edge = np.flatnonzero(np.abs(r_pix - RADIUS / BOX * 512) < 1.0)
    picks = []   # (plane, pixel)
    for axis in range(3):
        picks += [(axis, int(p)) for p in rng.choice(512 * 512, size=100, replace=False)]
        picks += [(axis, int(p)) for p in rng.choice(edge, size=8, replace=False)]
    leaf_rows = np.array([maps[a].reshape(-1)[p] for a, p in picks])
    pix_keys = np.array([cells[a][p] for a, p in picks], dtype=np.uint64)
    pix_ijk = np.stack([_compact(pix_keys >> np.uint64(q)) for q in range(3)], axis=1).astype(np.int32)
    pix_lv = np.full(len(picks), 9, dtype=np.int32)
    for ndir, (scheme, p0, p1) in SETS.items():
        geom = colden.precompute_geometry(scheme, p0, p1)
        dirs = _oracle_dirs(scheme, p0, p1)
        n_h = torch.empty(tree.n_leaf * ndir, device="cuda")
        colden.column_density(tree, geom, n_h=n_h, precision=colden.FP32)
        got = n_h.reshape(-1, ndir)[torch.from_numpy(leaf_rows).cuda()].double().cpu().numpy()
        ref = T.column_density(dirs, olv[leaf_rows], oijk[leaf_rows])
        rel = np.max(np.abs(got - ref) / ref)
        assert rel <= 1e-5, "%d directions: max rel N_H error %.3g vs the oracle" % (ndir, rel)
        ray = torch.empty((len(picks), ndir), device="cuda")
        colden.raymarch(uni, geom, ray, leaves=torch.from_numpy(pix_keys.astype(np.int64)).cuda())
        ref_ray = T.raymarch(dirs, pix_lv, pix_ijk)
        rel_ray = np.max(np.abs(ray.double().cpu().numpy() - ref_ray) / ref_ray)
        assert rel_ray <= 2e-5, "%d directions: max rel ray-marcher error %.3g vs the oracle" % (ndir, rel_ray)
        colden.device_status()


def _compact(v):
    v = np.asarray(v, dtype=np.uint64)
    out = np.zeros_like(v)
    for b in range(10):
        out |= ((v >> np.uint64(3 * b)) & np.uint64(1)) << np.uint64(b)
    return out


def test_sphere_extinction_maps_vs_ray_marcher_table2(sphere_mesh):
    lv, tree, uni = sphere_mesh
    counts = np.bincount(lv["level"], minlength=10)[7:]
    assert np.all(counts > 0)
    olv, oijk = tree.leaves()
    maps = [torch.from_numpy(m.reshape(-1)).cuda() for m in _plane_maps(olv, oijk)]
    cells = [torch.from_numpy(c).cuda() for c in _pixel_cells()]
    table = _table2()
    got = {}
    for ndir, (scheme, p0, p1) in SETS.items():
        geom = colden.precompute_geometry(scheme, p0, p1)
        n_h = torch.empty(tree.n_leaf * ndir, device="cuda")
        colden.column_density(tree, geom, n_h=n_h, precision=colden.FP32)
        chi_leaf = torch.exp(-SIGMA * n_h.reshape(-1, ndir).double()).mean(dim=1)
        dchi = []
        for m, c in zip(maps, cells):
            ray = torch.empty((c.numel(), ndir), device="cuda")
            colden.raymarch(uni, geom, ray, leaves=c)
            chi_ray = torch.exp(-SIGMA * ray.double()).mean(dim=1)
            dchi.append((chi_leaf[m] - chi_ray).abs())
        d = torch.cat(dchi)
        got[ndir] = (float(d.mean()), float(d.max()))
        colden.device_status()
    for ndir, (mean, mx) in got.items():
        print("directions %2d: mean dchi %.4f (paper %.3f), max %.4f (paper %.3f)"
              % (ndir, mean, table[ndir][0], mx, table[ndir][1]))
    for ndir, (mean, mx) in got.items():
        assert mean < table[ndir][0] and mean < 0.05
        assert mx < 0.25
    assert got[6][1] < table[6][1]
    for ndir in (12, 40, 84):
        assert table[ndir][1] / 1.5 < got[ndir][1] < 1.5 * table[ndir][1]
