"""Pins of the oracle's cone-averaged columns (CPU only).

A direction of an equal-solid-angle set stands for a bin of 4 pi / n_dir
steradians (§3.2); the cone option averages the geometric factors over a
circular cap of that solid angle.  The pins check the sub-ray pattern against
its definition (ring heights, equal azimuth steps, mean vector of the cap), the
averaged internal term against the exact cap integral of a cube's exit
distance, and the averaged uniform-density columns against the mean of the
per-ray closed form.
"""
import numpy as np
import pytest

import oracle
from test_oracle_pins import PC, _closed_form_uniform

R, P = oracle.CONE_RINGS, oracle.CONE_AZIMUTHS


def _sets():
    return {"healpix2": oracle.dirs_healpix(2), "mxn4x3": oracle.dirs_mxn(4, 3), "axes": oracle.dirs_axes(),
            "custom": oracle.dirs_custom([[1, 2, 3], [-0.3, 0.1, -1], [0, 0, 1]])}


@pytest.mark.parametrize("name", ["healpix2", "mxn4x3", "axes", "custom"])
def test_cone_ray_pattern(name):
    dirs = _sets()[name]
    nd = len(dirs)
    cos_a = 1.0 - 2.0 / nd
    rays = oracle.cone_rays(dirs)
    assert rays.shape == (nd, R * P, 3)
    assert np.allclose(np.linalg.norm(rays, axis=2), 1.0, atol=1e-15)
    for d in range(nd):
        u = dirs[d]
        v = rays[d].reshape(R, P, 3)
        cos_t = v @ u
        # ring r sits at the middle of the r-th equal step in cos theta
        for r in range(R):
            assert np.allclose(cos_t[r], 1.0 - (r + 0.5) * (1.0 - cos_a) / R, atol=1e-13)
        perp = v - cos_t[..., None] * u
        ang = np.zeros((R, P))
        ref = perp[0, 0] / np.linalg.norm(perp[0, 0])
        third = np.cross(u, ref)
        for r in range(R):
            for j in range(P):
                ang[r, j] = np.arctan2(perp[r, j] @ third, perp[r, j] @ ref)
        # equal azimuth steps of 2 pi / P, odd rings turned by half a step
        for r in range(R):
            step = np.angle(np.exp(1j * np.diff(ang[r])))
            assert np.allclose(step, 2 * np.pi / P, atol=1e-12)
            off = np.angle(np.exp(1j * (ang[r, 0] - ang[0, 0])))
            assert off == pytest.approx(np.pi / P if r & 1 else 0.0, abs=1e-12)
        # the mean of the sub-rays is <cos theta> u over the cap: (1 + cos alpha) / 2 u
        assert np.allclose(v.reshape(-1, 3).mean(axis=0), 0.5 * (1.0 + cos_a) * u, atol=1e-14)


@pytest.mark.parametrize("name", ["healpix2", "mxn4x3", "axes"])
def test_frame_is_stable_under_last_bit_changes(name):
    """Sets with exact ties (|u_x| = |u_y| at 45 degrees, zero components) give
    the same sub-rays when every component moves by a few ulps, as happens
    between two independent computations of the same direction set."""
    dirs = _sets()[name]
    rng = np.random.default_rng(0)
    base = oracle.cone_rays(dirs)
    for _ in range(20):
        d = dirs * (1.0 + rng.integers(-4, 5, size=dirs.shape) * 2.0 ** -52)
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        assert np.max(np.abs(oracle.cone_rays(d, n_bins=len(dirs)) - base)) < 1e-13


def test_zero_cone_is_the_ray():
    dirs = oracle.dirs_healpix(1)
    rays = oracle.cone_rays(dirs, cos_alpha=1.0)
    assert np.array_equal(rays, np.repeat(dirs[:, None, :], R * P, axis=1))


def _lone_leaf(L=3, ijk=(3, 4, 5), box=1.0):
    n = 1 << L
    rho = np.zeros((n, n, n), dtype=np.float32)
    rho[ijk[2], ijk[1], ijk[0]] = 1.0
    return oracle.Tree.uniform(rho, box), box / n


@pytest.mark.parametrize("n_bins", [48, 12])
def test_internal_term_is_cap_average_of_exit_distance(n_bins):
    """Only the target cell is dense, so the column is its internal term: the
    exit distance from the cell centre, 0.5 dx / max_a |v_a|, averaged over the
    sub-rays.  For the +z direction and a cap inside the +z face's pyramid
    (alpha <= 45 deg) the cap integral is 0.5 dx ln(1/cos a) / (1 - cos a); the
    equal-solid-angle rings reach it to the midpoint rule's O(h^2) error."""
    T, dx = _lone_leaf()
    dirs = oracle.dirs_custom([[0, 0, 1], [1, 0, 0], [0, -1, 0], [1, 1, 1], [-2, 1, 0.5]])
    got = T.column_density_cone(dirs, [3], [(3, 4, 5)], n_bins=n_bins)[0]
    rays = oracle.cone_rays(dirs, n_bins)
    exact_mean = (0.5 * dx / np.abs(rays).max(axis=2)).mean(axis=1)
    assert np.allclose(got, exact_mean, rtol=1e-13)
    cos_a = 1.0 - 2.0 / n_bins
    cap = 0.5 * dx * np.log(1.0 / cos_a) / (1.0 - cos_a)
    h = (1.0 - cos_a) / R
    bound = h * h / 24.0 * (2.0 * 0.5 * dx / cos_a ** 3)    # midpoint rule: h^2/24 max|f''|
    for d in range(3):                                       # the three axis directions
        assert abs(got[d] - cap) <= 1.05 * bound
    # rings evenly spaced in theta instead of cos theta would miss by ~alpha^2/12
    alpha = np.arccos(cos_a)
    assert cap * alpha ** 2 / 12 > 20 * bound


@pytest.mark.parametrize("mode", [oracle.MODE_PREC, oracle.MODE_INSITU])
def test_uniform_density_cone_is_mean_of_ray_closed_forms(mode):
    L, box, n0 = 4, 10 * PC, 3.0
    T = oracle.Tree.uniform(np.full((1 << L,) * 3, n0, dtype=np.float32), box)
    ijk = np.random.default_rng(5).integers(0, 1 << L, size=(12, 3))
    for dirs in (oracle.dirs_healpix(1), oracle.dirs_axes()):
        got = T.column_density_cone(dirs, np.full(len(ijk), L), ijk, mode=mode)
        rays = oracle.cone_rays(dirs)
        for t in range(len(ijk)):
            for d in range(len(dirs)):
                want = np.mean([_closed_form_uniform(n0, box, L, ijk[t], v, mode) for v in rays[d]])
                assert got[t, d] == pytest.approx(want, rel=1e-12)


def test_cone_column_lies_between_sub_ray_extremes():
    T = oracle.Tree.uniform(np.random.default_rng(2).lognormal(0, 1.5, (16, 16, 16)).astype(np.float32), 1.0)
    dirs = oracle.dirs_healpix(1)
    ijk = np.array([[1, 2, 3], [8, 8, 8], [15, 0, 7]])
    got = T.column_density_cone(dirs, [4] * 3, ijk)
    per = T.column_density(oracle.cone_rays(dirs).reshape(-1, 3), [4] * 3, ijk).reshape(3, 12, R * P)
    assert np.all(got >= per.min(axis=2) * (1 - 1e-14)) and np.all(got <= per.max(axis=2) * (1 + 1e-14))
    # and the cone smooths the field: it differs from the central ray
    ray = T.column_density(dirs, [4] * 3, ijk)
    assert np.max(np.abs(got / ray - 1.0)) > 1e-2
