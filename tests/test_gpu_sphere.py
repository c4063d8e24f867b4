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


def test_sphere_extinction_maps_vs_ray_marcher_table2():
    box, R = 50 * PC, 12.5 * PC
    fine = synth.sphere(512, box, R, 1000.0, 10.0)
    lv = synth.amr_leaves(fine, 7, [10.5, 10.5])
    counts = np.bincount(lv["level"], minlength=10)[7:]
    assert np.all(counts > 0)
    tree = colden.build_tree_amr(7, 9, box, lv["level"], lv["ijk"], lv["rho"])
    uni = colden.build_tree_uniform(torch.from_numpy(fine).cuda(), box)
    del fine
    olv, oijk = tree.leaves()
    maps = [torch.from_numpy(m.reshape(-1)).cuda() for m in _plane_maps(olv, oijk)]
    cells = [torch.from_numpy(c).cuda() for c in _pixel_cells()]
    table = _table2()
    got = {}
    for ndir, (scheme, p0, p1) in {6: ("axes", 0, 0), 12: ("mxn", 3, 4), 40: ("mxn", 5, 8),
                                   84: ("mxn", 7, 12)}.items():
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
