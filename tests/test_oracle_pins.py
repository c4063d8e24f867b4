"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: values the
paper prints (golden files with their citation), closed forms, special cases
that reduce to one-dimensional sums, invariants, and brute force on tiny
inputs.  All run on the CPU (no GPU marker).
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1410_0624_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
PC = 3.0857e18


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------------------
# Directions
# ---------------------------------------------------------------------------

def test_theta_values_printed_in_sec4_4():
    for M, m, theta in _golden("theta_fig_nnoprec_prec.txt"):
        M, m, theta = int(M), int(m), float(theta)
        d = oracle.dirs_mxn(M, 4)
        # index (m-1)*N + (n-1); n = 1 is phi = 0
        v = d[(m - 1) * 4 + 0]
        assert abs(v[1]) < 1e-15 and v[0] > 0  # phi = 0
        assert round(float(np.arccos(v[2])), 3) == theta


def test_mxn_equal_cos_theta_spacing():
    # delta cos(theta) = 2/M between consecutive rings, bin centres (§3.2)
    for M, N in [(3, 4), (5, 8), (7, 12)]:
        d = oracle.dirs_mxn(M, N).reshape(M, N, 3)
        z = d[:, 0, 2]
        assert np.allclose(np.diff(z), -2.0 / M, atol=1e-14)
        assert np.allclose(z[0], 1 - 1.0 / M, atol=1e-14)
        phi = np.arctan2(d[0, :, 1], d[0, :, 0]) % (2 * np.pi)
        assert np.allclose(phi, 2 * np.pi * np.arange(N) / N, atol=1e-12)


def test_healpix_rings_gorski2005():
    rows = _golden("healpix_rings_gorski2005.txt")
    for nside in (1, 2):
        d = oracle.dirs_healpix(nside)
        assert d.shape == (12 * nside * nside, 3)
        assert np.allclose(np.linalg.norm(d, axis=1), 1.0, atol=1e-14)
        want = [(int(a) / int(b), int(c)) for ns, a, b, c in rows if int(ns) == nside]
        got_z = np.round(d[:, 2], 12)
        start = 0
        for z, cnt in want:
            ring = got_z[start:start + cnt]
            assert np.allclose(ring, z, atol=1e-12), (nside, z)
            start += cnt
        assert start == d.shape[0]
        assert np.allclose(d.sum(axis=0), 0.0, atol=1e-12)


def test_healpix_nside1_shares_rings_with_paper_3x4():
    hp = oracle.dirs_healpix(1)
    mn = oracle.dirs_mxn(3, 4)
    assert np.allclose(np.sort(hp[:, 2]), np.sort(mn[:, 2]), atol=1e-12)


def test_direction_snapping():
    d = oracle.dirs_mxn(3, 4)
    # phi = pi/2 gives cos(phi) ~ 6e-17, which is set to exactly zero
    assert np.all((np.abs(d) == 0.0) | (np.abs(d) > 1e-14))


# ---------------------------------------------------------------------------
# Ray / cube lengths
# ---------------------------------------------------------------------------

def test_ray_cube_closed_forms():
    c = oracle.ray_cube
    assert c([0.5, 0.5, 0.5], [1, 0, 0], [0, 0, 0], 1.0) == pytest.approx(0.5, abs=1e-15)
    assert c([-3.0, 0.5, 0.5], [1, 0, 0], [0, 0, 0], 1.0) == pytest.approx(1.0, abs=1e-15)
    s3 = 1 / np.sqrt(3)
    assert c([-1.0, -1.0, -1.0], [s3, s3, s3], [0, 0, 0], 1.0) == pytest.approx(np.sqrt(3), rel=1e-14)
    assert c([2.0, 0.5, 0.5], [1, 0, 0], [0, 0, 0], 1.0) == 0.0       # behind
    assert c([-1.0, 1.5, 0.5], [1, 0, 0], [0, 0, 0], 1.0) == 0.0      # miss
    # scale covariance: length in a cube of side h scales with h
    p = np.array([0.3, 0.2, 0.1])
    d = np.array([0.48, 0.6, 0.64])
    assert c(p * 7, d, [0, 0, 0], 7.0) == pytest.approx(7 * c(p, d, [0, 0, 0], 1.0), rel=1e-14)


def test_ray_cube_row_additivity():
    rng = np.random.default_rng(5)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        p = rng.uniform(0.1, 0.9, size=3) + 2
        total = 0.0
        for ijk in itertools.product(range(6), repeat=3):
            total += oracle.ray_cube(p, d, np.array(ijk, float), 1.0)
        # exit distance of the 6^3 block [0, 6]^3
        t = np.inf
        for a in range(3):
            if d[a] > 0:
                t = min(t, (6 - p[a]) / d[a])
            elif d[a] < 0:
                t = min(t, (0 - p[a]) / d[a])
        assert total == pytest.approx(t, rel=1e-12)


# ---------------------------------------------------------------------------
# Tree: volume means (§3 intro, coarse density = mean)
# ---------------------------------------------------------------------------

def _block_mean(f, b):
    n = f.shape[0] // b
    return f.reshape(n, b, n, b, n, b).astype(np.float64).mean(axis=(1, 3, 5))


def test_uniform_levels_are_block_means():
    rho = synth.lognormal_iid(16, 10.0, 1.5, seed=3)
    T = oracle.Tree.uniform(rho, 1.0)
    for l in range(0, 5):
        bm = _block_mean(rho, 1 << (4 - l))
        n = 1 << l
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ijk = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
        got = T.rho(np.full(n ** 3, l), ijk)
        assert np.allclose(got, bm.ravel(), rtol=1e-13, atol=0)


def _amr_case(seed=7):
    fine = synth.lognormal_grf(32, 30.0, 2.0, seed=seed)
    return fine, synth.amr_leaves(fine, 3, [40.0, 60.0])


def _paint(leaves, lmax):
    n = 1 << lmax
    g = np.zeros((n, n, n))
    for l, (i, j, k), r in zip(leaves["level"], leaves["ijk"], leaves["rho"]):
        s = 1 << (lmax - l)
        g[k * s:(k + 1) * s, j * s:(j + 1) * s, i * s:(i + 1) * s] = r
    return g


def test_amr_levels_are_volume_means_of_leaf_field():
    fine, lv = _amr_case()
    assert len(np.unique(lv["level"])) == 3
    T = oracle.Tree.amr(lv["base"], lv["lmax"], 1.0, lv["level"], lv["ijk"], lv["rho"])
    painted = _paint(lv, lv["lmax"])
    for l in range(0, 6):
        bm = _block_mean(painted, 1 << (5 - l))
        n = 1 << l
        z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        ijk = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
        got = T.rho(np.full(n ** 3, l), ijk)
        assert np.allclose(got, bm.ravel(), rtol=1e-12, atol=0), l


def test_amr_rejects_bad_leaf_sets():
    _, lv = _amr_case()
    with pytest.raises(ValueError):
        oracle.Tree.amr(lv["base"], lv["lmax"], 1.0, lv["level"][1:], lv["ijk"][1:], lv["rho"][1:])
    dup_l = np.concatenate([lv["level"], lv["level"][:1]])
    dup_i = np.concatenate([lv["ijk"], lv["ijk"][:1]])
    dup_r = np.concatenate([lv["rho"], lv["rho"][:1]])
    with pytest.raises(ValueError):
        oracle.Tree.amr(lv["base"], lv["lmax"], 1.0, dup_l, dup_i, dup_r)


# ---------------------------------------------------------------------------
# The two-level approximation: 73 configurations (§3.3)
# ---------------------------------------------------------------------------

def test_seventy_three_reference_configurations():
    want = {r[0]: int(r[1]) for r in _golden("configurations_sec3_3.txt")}
    l0, box = 5, 1.0
    n = 1 << l0
    rng = np.random.default_rng(0)
    classes = {"1": set(), "2": set(), "3+": set()}
    for ijk in rng.integers(0, n, size=(3000, 3)):
        for l in range(l0 - 1, 0, -1):
            p = oracle.pref(box, l0, ijk, l, oracle.MODE_PREC)
            dxl = box / (1 << l)
            a_l = np.array(ijk) >> (l0 - l)
            rel = tuple(np.round((p - a_l * dxl) / dxl, 9))
            dl = l0 - l
            classes["1" if dl == 1 else "2" if dl == 2 else "3+"].add(rel)
            if dl <= 3:  # exact for these shells: the oct centre
                q = oracle.pref(box, l0, ijk, l, oracle.MODE_INSITU)
                assert np.allclose(p, q, rtol=0, atol=1e-15)
    for k in ("1", "2", "3+"):
        assert len(classes[k]) == want[k]
    assert sum(len(v) for v in classes.values()) == want["total"]


# ---------------------------------------------------------------------------
# Closed form for a uniform density (P1)
# ---------------------------------------------------------------------------

def _exit(lo, hi, p, d):
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (hi[a] - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, (lo[a] - p[a]) / d[a])
    return t


def _closed_form_uniform(n0, box, l0, ijk, d, mode):
    """Every region of the method is a box containing the ray origin, so each
    shell's path is exit(outer box) - exit(inner box)."""
    ijk = np.array(ijk)
    dx = lambda l: box / (1 << l)
    xt = (ijk + 0.5) * dx(l0)
    oct_lo = (ijk >> 1) * dx(l0 - 1)
    N = _exit(oct_lo, oct_lo + dx(l0 - 1), xt, d)
    for l in range(l0 - 1, 0, -1):
        r = (l0 - 1) if mode == oracle.MODE_INSITU else min(l + 2, l0 - 1)
        p = ((ijk >> (l0 - r)) + 0.5) * dx(r)
        a_lm1 = ijk >> (l0 - l + 1)
        a_l = ijk >> (l0 - l)
        out_lo = np.maximum((a_lm1 - 1) * dx(l - 1), 0.0)
        out_hi = np.minimum((a_lm1 + 2) * dx(l - 1), box)
        if l == l0 - 1:
            in_lo, in_hi = a_l * dx(l), (a_l + 1) * dx(l)
        else:
            in_lo = np.maximum((a_l - 1) * dx(l), 0.0)
            in_hi = np.minimum((a_l + 2) * dx(l), box)
        N += _exit(out_lo, out_hi, p, d) - _exit(in_lo, in_hi, p, d)
    return n0 * N


@pytest.mark.parametrize("L", [1, 2, 3, 5])
@pytest.mark.parametrize("mode", [oracle.MODE_PREC, oracle.MODE_INSITU])
def test_uniform_density_closed_form(mode, L):
    box, n0 = 10 * PC, 7.0
    rho = np.full((1 << L,) * 3, n0, dtype=np.float32)
    T = oracle.Tree.uniform(rho, box)
    rng = np.random.default_rng(1)
    ijk = rng.integers(0, 1 << L, size=(60, 3))
    for dirs in (oracle.dirs_healpix(1), oracle.dirs_healpix(2), oracle.dirs_mxn(5, 8),
                 oracle.dirs_axes()):
        got = T.column_density(dirs, np.full(len(ijk), L), ijk, mode=mode)
        for t in range(len(ijk)):
            for di in range(len(dirs)):
                want = _closed_form_uniform(n0, box, L, ijk[t], dirs[di], mode)
                assert got[t, di] == pytest.approx(want, rel=1e-12)


def test_insitu_uniform_is_distance_to_box_edge_telescoped():
    L, box, n0 = 4, 1.0, 3.0
    T = oracle.Tree.uniform(np.full((16, 16, 16), n0, np.float32), box)
    dirs = oracle.dirs_healpix(2)
    ijk = np.array([[0, 0, 0], [5, 9, 2], [15, 15, 15], [7, 8, 8]])
    got = T.column_density(dirs, np.full(4, L), ijk, mode=oracle.MODE_INSITU)
    for t in range(4):
        xt = (ijk[t] + 0.5) / 16
        lo = (ijk[t] >> 1) / 8
        xo = lo + 1 / 16
        for di, d in enumerate(dirs):
            want = n0 * (_exit(lo, lo + 1 / 8, xt, d) + _exit([0] * 3, [1] * 3, xo, d)
                         - _exit(lo, lo + 1 / 8, xo, d))
            assert got[t, di] == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------------------
# Six axis rays: one-dimensional sums, no geometric correction (§4.3) (P4)
# ---------------------------------------------------------------------------

def _axis_row_sum(levels, box, l0, ijk, axis, sign):
    """N along +-axis as sums of (level density x dx) along cell rows."""
    ijk = np.array(ijk)
    dx = lambda l: box / (1 << l)
    other = [a for a in range(3) if a != axis]

    def val(l, c):
        n = 1 << l
        if np.any(c < 0) or np.any(c >= n):
            return 0.0
        return levels[l][c[2], c[1], c[0]]

    N = 0.5 * dx(l0) * val(l0, ijk)
    if (ijk[axis] & 1) == (0 if sign > 0 else 1):
        c = ijk.copy()
        c[axis] += sign
        N += dx(l0) * val(l0, c)
    for l in range(l0 - 1, 0, -1):
        r = min(l + 2, l0 - 1)
        p = ((ijk >> (l0 - r)) + 0.5) * dx(r)
        row = np.floor(p / dx(l)).astype(int)
        a_lm1 = ijk >> (l0 - l + 1)
        a_l = ijk >> (l0 - l)
        for cx in range(2 * (a_lm1[axis] - 1), 2 * (a_lm1[axis] + 2)):
            c = row.copy()
            c[axis] = cx
            if l == l0 - 1:
                inner = np.all(c == a_l)
            else:
                inner = np.all(np.abs(c - a_l) <= 1)
            if inner or np.any(np.abs(c[other] - 2 * a_lm1[other] - 0.5) > 3):
                continue
            lo, hi = cx * dx(l), (cx + 1) * dx(l)
            if sign > 0:
                seg = max(0.0, hi - max(lo, p[axis]))
            else:
                seg = max(0.0, min(hi, p[axis]) - lo)
            N += val(l, c) * seg
    return N


def test_six_axis_rays_reduce_to_row_sums():
    L, box = 4, 2.0
    rho = synth.lognormal_iid(16, 10.0, 1.5, seed=11)
    T = oracle.Tree.uniform(rho, box)
    levels = {l: _block_mean(rho, 1 << (L - l)) for l in range(L + 1)}
    dirs = oracle.dirs_axes()
    rng = np.random.default_rng(2)
    ijk = rng.integers(0, 16, size=(40, 3))
    got = T.column_density(dirs, np.full(40, L), ijk)
    for t in range(40):
        for di, (axis, sign) in enumerate([(0, 1), (0, -1), (1, 1), (1, -1), (2, 1), (2, -1)]):
            want = _axis_row_sum(levels, box, L, ijk[t], axis, sign)
            assert got[t, di] == pytest.approx(want, rel=1e-12)


# ---------------------------------------------------------------------------
# Invariants (P5)
# ---------------------------------------------------------------------------

def test_linearity_and_nonnegativity():
    L, box = 4, 1.0
    r1 = synth.lognormal_iid(16, 10.0, 1.5, seed=1)
    r2 = synth.lognormal_grf(16, 30.0, 2.0, seed=2)
    a, b = 0.75, 2.5
    ijk = np.random.default_rng(3).integers(0, 16, size=(50, 3))
    dirs = oracle.dirs_healpix(1)
    lv = np.full(50, L)
    n1 = oracle.Tree.uniform(r1, box).column_density(dirs, lv, ijk)
    n2 = oracle.Tree.uniform(r2, box).column_density(dirs, lv, ijk)
    mix = (a * r1.astype(np.float64) + b * r2.astype(np.float64)).astype(np.float32)
    # float32 rounding of the mixed field is the only difference
    n12 = oracle.Tree.uniform(mix, box).column_density(dirs, lv, ijk)
    assert np.allclose(n12, a * n1 + b * n2, rtol=2e-7)
    assert np.all(n1 > 0) and np.all(n2 > 0)


def _symmetric_field(n):
    c = (n - 1) / 2
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    s = np.sort(np.stack([np.abs(x - c), np.abs(y - c), np.abs(z - c)]), axis=0)
    return (1.0 + s[0] + 3.0 * s[1] ** 1.5 + 0.3 * np.cos(s[2])).astype(np.float32)


def _apply(perm, flip, n, ijk, d):
    ijk2 = np.array([ijk[perm[a]] for a in range(3)])
    d2 = np.array([d[perm[a]] for a in range(3)])
    for a in range(3):
        if flip[a]:
            ijk2[a] = n - 1 - ijk2[a]
            d2[a] = -d2[a]
    return ijk2, d2


@pytest.mark.parametrize("full_group", [True, False])
def test_cube_symmetry_equivariance(full_group):
    L, box = 4, 1.0
    n = 1 << L
    T = oracle.Tree.uniform(_symmetric_field(n), box)
    dirs = oracle.dirs_axes() if full_group else oracle.dirs_healpix(2)
    ijk = np.random.default_rng(4).integers(0, n, size=(12, 3))
    base = T.column_density(dirs, np.full(12, L), ijk)
    perms = list(itertools.permutations(range(3))) if full_group else [(0, 1, 2), (1, 0, 2)]
    count = 0
    for perm in perms:
        for flip in itertools.product([0, 1], repeat=3):
            g_ijk, order = [], []
            ok = True
            for t in range(12):
                g_ijk.append(_apply(perm, flip, n, ijk[t], np.zeros(3))[0])
            for di in range(len(dirs)):
                _, gd = _apply(perm, flip, n, np.zeros(3, int), dirs[di])
                j = np.where(np.all(np.abs(dirs - gd) < 1e-12, axis=1))[0]
                if len(j) != 1:
                    ok = False
                    break
                order.append(j[0])
            assert ok, (perm, flip)
            got = T.column_density(dirs, np.full(12, L), np.array(g_ijk))
            assert np.allclose(got[:, order], base, rtol=1e-12)
            count += 1
    assert count == (48 if full_group else 16)


# ---------------------------------------------------------------------------
# Brute-force reference (§4): exactness of the ray-marcher (P6)
# ---------------------------------------------------------------------------

def test_raymarch_uniform_box_is_density_times_distance():
    box, n0 = 3.0, 4.0
    T = oracle.Tree.uniform(np.full((8, 8, 8), n0, np.float32), box)
    dirs = oracle.dirs_healpix(2)
    ijk = np.random.default_rng(6).integers(0, 8, size=(20, 3))
    got = T.raymarch(dirs, np.full(20, 3), ijk)
    for t in range(20):
        x = (ijk[t] + 0.5) * box / 8
        for di, d in enumerate(dirs):
            assert got[t, di] == pytest.approx(n0 * _exit([0] * 3, [box] * 3, x, d), rel=1e-12)


def test_raymarch_matches_all_cell_sum_on_tiny_grid():
    rho = synth.lognormal_iid(8, 10.0, 1.5, seed=9)
    T = oracle.Tree.uniform(rho, 1.0)
    dirs = oracle.dirs_mxn(5, 8)
    for ijk in ([0, 0, 0], [3, 4, 5], [7, 1, 6]):
        got = T.raymarch(dirs, [3], [ijk])[0]
        want = T.raysum_allcells(dirs, (np.array(ijk) + 0.5) / 8)
        assert np.allclose(got, want, rtol=1e-12)


def test_raymarch_matches_midpoint_sampling():
    rho = synth.lognormal_iid(8, 10.0, 1.0, seed=10)
    T = oracle.Tree.uniform(rho, 1.0)
    d = oracle.dirs_custom([[0.3, 0.5, 0.81]])
    x0 = (np.array([2, 3, 1]) + 0.5) / 8
    got = T.raymarch(d, [3], [[2, 3, 1]])[0, 0]
    tmax = _exit([0] * 3, [1] * 3, x0, d[0])
    ns = 400000
    s = (np.arange(ns) + 0.5) * tmax / ns
    pts = np.clip(np.floor((x0[None] + s[:, None] * d[0][None]) * 8).astype(int), 0, 7)
    want = rho[pts[:, 2], pts[:, 1], pts[:, 0]].astype(np.float64).sum() * tmax / ns
    assert got == pytest.approx(want, rel=1e-3)


def test_amr_raymarch_equals_painted_uniform():
    _, lv = _amr_case()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], 1.0, lv["level"], lv["ijk"], lv["rho"])
    U = oracle.Tree.uniform(_paint(lv, lv["lmax"]).astype(np.float32), 1.0)
    dirs = oracle.dirs_healpix(1)
    fine = lv["level"] == lv["lmax"]
    sel = np.nonzero(fine)[0][:30]
    a = T.raymarch(dirs, lv["level"][sel], lv["ijk"][sel])
    b = U.raymarch(dirs, lv["level"][sel], lv["ijk"][sel])
    assert np.allclose(a, b, rtol=1e-12)


# ---------------------------------------------------------------------------
# AMR tree method: finest targets see the same volume means as on the painted grid
# ---------------------------------------------------------------------------

def test_amr_tree_method_equals_painted_uniform_for_finest_leaves():
    _, lv = _amr_case()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], 1.0, lv["level"], lv["ijk"], lv["rho"])
    U = oracle.Tree.uniform(_paint(lv, lv["lmax"]).astype(np.float32), 1.0)
    dirs = oracle.dirs_healpix(2)
    sel = np.nonzero(lv["level"] == lv["lmax"])[0][:40]
    for mode in (oracle.MODE_PREC, oracle.MODE_INSITU):
        a = T.column_density(dirs, lv["level"][sel], lv["ijk"][sel], mode=mode)
        b = U.column_density(dirs, lv["level"][sel], lv["ijk"][sel], mode=mode)
        assert np.allclose(a, b, rtol=1e-12)


def test_amr_uniform_leaf_set_equals_uniform_tree():
    rho = synth.lognormal_iid(8, 10.0, 1.5, seed=12)
    ijk = oracle.morton_ijk(3)
    r = rho[ijk[:, 2], ijk[:, 1], ijk[:, 0]]
    T = oracle.Tree.amr(3, 3, 1.0, np.full(512, 3), ijk, r)
    U = oracle.Tree.uniform(rho, 1.0)
    dirs = oracle.dirs_healpix(1)
    assert np.allclose(T.column_density(dirs, np.full(512, 3), ijk),
                       U.column_density(dirs, np.full(512, 3), ijk), rtol=1e-14)


# ---------------------------------------------------------------------------
# Accuracy statements of the paper (statistical, P6/P7)
# ---------------------------------------------------------------------------

def test_extinction_error_within_ten_percent_vs_raymarch():
    """§4 / §6: the extinction error of the tree method stays below ~10 %."""
    L = 5
    box = 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 1.5, seed=21)
    T = oracle.Tree.uniform(rho, box)
    dirs = oracle.dirs_mxn(5, 8)
    ijk = np.random.default_rng(7).integers(0, 1 << L, size=(300, 3))
    lv = np.full(300, L)
    tree = T.column_density(dirs, lv, ijk)
    ray = T.raymarch(dirs, lv, ijk)
    dchi = np.abs(oracle.chi(tree) - oracle.chi(ray))
    assert dchi.mean() < 0.1
    assert np.all(tree > 0) and np.all(ray > 0)


def test_prec_vs_insitu_extinction_difference_small():
    """§4.3, Table 1: <|chi_prec - chi_insitu|> below ~0.004 on the paper's
    cloud; on a synthetic turbulent-like field we require < 0.01."""
    L = 6
    box = 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=22)
    T = oracle.Tree.uniform(rho, box)
    dirs = oracle.dirs_mxn(3, 4)
    ijk = np.random.default_rng(8).integers(0, 1 << L, size=(400, 3))
    lv = np.full(400, L)
    a = T.column_density(dirs, lv, ijk, mode=oracle.MODE_PREC)
    b = T.column_density(dirs, lv, ijk, mode=oracle.MODE_INSITU)
    assert np.mean(np.abs(oracle.chi(a) - oracle.chi(b))) < 0.01
    assert np.mean(np.abs(a - b) / b) < 0.15


def test_per_level_slots_sum_to_total():
    L = 5
    rho = synth.lognormal_iid(32, 10.0, 1.5, seed=1)
    T = oracle.Tree.uniform(rho, 1.0)
    dirs = oracle.dirs_healpix(1)
    ijk = np.random.default_rng(9).integers(0, 32, size=(20, 3))
    tot, pl = T.column_density(dirs, np.full(20, L), ijk, per_level=L)
    assert np.allclose(pl.sum(axis=1), tot, rtol=1e-13)
