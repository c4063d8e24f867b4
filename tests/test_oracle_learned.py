"""Pins of the learned-correction oracle (oracle/learned.py) against facts that
do not come from the oracle itself: identities of GELU, its distance from the
erf form (Python's math.erf), finite differences of the loss, the closed form
of Adam under a constant gradient, special weight settings where the network
reduces to plain matrix products or to its last bias, and the per-level slots
of a uniform density, which are differences of exit distances of nested boxes.
CPU only."""
import math

import numpy as np
import pytest

import oracle
from oracle import learned as ol
from paper_1410_0624_gb300 import synth

PC = 3.0857e18


# ---------------------------------------------------------------------------
# GELU
# ---------------------------------------------------------------------------

def test_gelu_odd_part_identity():
    """x Phi~(x) with Phi~ odd around 1/2 gives gelu(x) - gelu(-x) = x."""
    x = np.linspace(-9, 9, 1001)
    assert np.allclose(ol.gelu(x) - ol.gelu(-x), x, rtol=0, atol=1e-13)
    assert ol.gelu(np.array(0.0)) == 0.0


def test_gelu_tanh_form_close_to_erf_form():
    x = np.linspace(-8, 8, 3201)
    exact = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in x])
    assert np.max(np.abs(ol.gelu(x) - exact)) < 1e-3
    # far tails: identity and zero
    assert ol.gelu(np.array(30.0)) == pytest.approx(30.0, rel=1e-15)
    assert abs(ol.gelu(np.array(-30.0))) < 1e-300


def test_gelu_grad_matches_finite_differences():
    x = np.linspace(-6, 6, 241)
    h = 1e-6
    fd = (ol.gelu(x + h) - ol.gelu(x - h)) / (2 * h)
    assert np.allclose(ol.gelu_grad(x), fd, rtol=0, atol=1e-8)
    assert ol.gelu_grad(np.array(0.0)) == pytest.approx(0.5, abs=1e-15)


# ---------------------------------------------------------------------------
# Network: special cases
# ---------------------------------------------------------------------------

def _tiny(n_dir=2, hidden=5, seed=0):
    rng = np.random.default_rng(seed)
    n_in = ol.n_inputs(n_dir)
    p = {"W1": rng.uniform(0.01, 0.2, (hidden, n_in)), "b1": np.full(hidden, 20.0),
         "W2": rng.uniform(0.01, 0.2, (hidden, hidden)), "b2": np.full(hidden, 20.0),
         "W3": rng.uniform(-1, 1, (n_dir, hidden)), "b3": rng.uniform(-1, 1, n_dir)}
    return p, n_in


def test_forward_linear_regime_is_plain_matrix_products():
    """Every pre-activation >= 10: GELU is the identity to FP64 rounding, so the
    network is the affine map W3 (W2 (W1 u + b1) + b2) + b3, written here with
    explicit loops over the weight matrices' rows."""
    n_dir, hidden = 2, 5
    p, n_in = _tiny(n_dir, hidden)
    rng = np.random.default_rng(3)
    x = rng.uniform(0, 1, (4, n_in))
    mu, sinv = np.full(n_in, -0.5), np.full(n_in, 2.0)       # u = 2 x + 1 > 0
    got, (_, z1, _, z2, _) = ol.forward(p, mu, sinv, x)
    assert z1.min() >= 10 and z2.min() >= 10
    for r in range(len(x)):
        u = [2.0 * v + 1.0 for v in x[r]]
        h1 = [sum(p["W1"][j][i] * u[i] for i in range(n_in)) + p["b1"][j] for j in range(hidden)]
        h2 = [sum(p["W2"][j][i] * h1[i] for i in range(hidden)) + p["b2"][j] for j in range(hidden)]
        want = [sum(p["W3"][d][i] * h2[i] for i in range(hidden)) + p["b3"][d] for d in range(n_dir)]
        assert np.allclose(got[r], want, rtol=1e-13, atol=0)


def test_forward_off_regime_is_last_bias():
    p, n_in = _tiny()
    p["b2"] = np.full_like(p["b2"], -60.0)
    x = np.random.default_rng(4).uniform(0, 1, (3, n_in))
    got, _ = ol.forward(p, np.zeros(n_in), np.ones(n_in), x)
    assert np.allclose(got, p["b3"][None, :], rtol=0, atol=1e-250)


def test_loss_gradient_matches_finite_differences():
    n_dir, hidden = 3, 6
    n_in = ol.n_inputs(n_dir)
    flat = synth.mlp_init(n_dir, hidden, seed=5).astype(np.float64)
    rng = np.random.default_rng(6)
    x = rng.normal(40, 3, (7, n_in))
    y = rng.normal(0, 0.3, (7, n_dir))
    mu, sinv = ol.normaliser(x)
    p = ol.unpack(flat, n_dir, hidden)
    _, g = ol.loss_grad(p, mu, sinv, x, y)
    gflat = ol.pack(g)
    h = 1e-6
    for k in range(flat.size):
        a, b = flat.copy(), flat.copy()
        a[k] += h
        b[k] -= h
        fd = (ol.loss(ol.unpack(a, n_dir, hidden), mu, sinv, x, y) -
              ol.loss(ol.unpack(b, n_dir, hidden), mu, sinv, x, y)) / (2 * h)
        assert gflat[k] == pytest.approx(fd, rel=1e-5, abs=1e-9), k


def test_adam_constant_gradient_closed_form():
    """With a constant gradient g the bias-corrected moments are exactly g and
    g^2, so every step moves a parameter by lr g / (|g| + eps)."""
    rng = np.random.default_rng(7)
    p0 = rng.normal(size=50)
    g = rng.normal(size=50)
    g[0] = 0.0
    m = np.zeros(50)
    v = np.zeros(50)
    p = p0.copy()
    lr, eps = 1e-3, 1e-8
    for t in range(1, 6):
        p, m, v = ol.adam(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p, p0 - t * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-13)
    assert p[0] == p0[0]


def test_apply_falls_back_where_delta_is_not_finite():
    n = np.array([[1.0, 2.0, 3.0, 4.0]])
    d = np.array([[0.0, math.log(2.0), np.nan, np.inf]])
    assert np.allclose(ol.apply(n, d), [[1.0, 4.0, 3.0, 4.0]], rtol=1e-15)


def test_apply_range_limits():
    """Infinite range: the unguarded form; a closed range keeps its end
    points and falls back outside; an empty range (lo > hi) is the plain
    method everywhere."""
    n = np.array([[1.0, 2.0, 3.0, 4.0, 5.0]])
    d = np.array([[-1.0, -0.5, 0.25, 0.5, 2.0]])
    assert np.array_equal(ol.apply(n, d, -math.inf, math.inf), ol.apply(n, d))
    got = ol.apply(n, d, -0.5, 0.5)
    assert np.allclose(got, [[1.0, 2.0 * math.exp(-0.5), 3.0 * math.exp(0.25), 4.0 * math.exp(0.5), 5.0]],
                       rtol=1e-15)
    assert np.array_equal(ol.apply(n, d, 1.0, -1.0), n)
    assert np.array_equal(ol.apply(n, np.array([[np.nan, np.inf, -np.inf, 0.0, 0.0]]), -10, 10),
                          [[1.0, 2.0, 3.0, 4.0, 5.0]])


def test_delta_range_of_targets():
    y = np.array([0.3, -1.25, np.nan, 2.5, np.inf, -np.inf, 0.0])
    assert ol.delta_range(y, 0.5) == (-1.75, 3.0)
    assert ol.delta_range(y, 0.0) == (-1.25, 2.5)
    lo, hi = ol.delta_range(np.array([np.nan]), 1.0)
    assert lo > hi


def test_range_falls_back_to_the_plain_method():
    """Where delta leaves the trusted range the learned column is the plain
    tree method's column (the slot sum of the per-level oracle, checked here
    against the C oracle's own total); inside it, the corrected column.  A
    64^3 box of random densities and a seeded network whose biases put every
    even direction's delta near 3 and every odd one's near 0."""
    rng = np.random.default_rng(11)
    L, box = 6, 10 * PC
    rho = rng.lognormal(1.0, 1.5, size=(1 << L,) * 3)
    T = oracle.Tree.uniform(rho, box)
    dirs = oracle.dirs_healpix(1)
    ijk = rng.integers(0, 1 << L, size=(40, 3)).astype(np.int32)
    lv = np.full(40, L, dtype=np.int8)
    tot, pl = T.column_density(dirs, lv, ijk, per_level=L)
    slots = ol.slots_from_levels(pl)
    nd, H = dirs.shape[0], 16
    p = ol.unpack(rng.normal(scale=0.05, size=ol.n_params(nd, H)), nd, H)
    p["b3"][:] = np.where(np.arange(nd) % 2 == 0, 3.0, 0.0)
    x = ol.features(slots, rho[ijk[:, 2], ijk[:, 1], ijk[:, 0]])
    mu, sinv = ol.normaliser(x)
    delta, _ = ol.forward(p, mu, sinv, x)
    out_of_range = np.abs(delta) > 1.0
    assert np.array_equal(out_of_range, np.broadcast_to(np.arange(nd) % 2 == 0, delta.shape))
    assert np.allclose(ol.apply(ol.tree_total(slots), delta, 1.0, -1.0), tot, rtol=1e-13)
    out = ol.apply(ol.tree_total(slots), delta, -1.0, 1.0)
    assert np.allclose(out[out_of_range], tot[out_of_range], rtol=1e-13)
    assert np.allclose(out[~out_of_range], (tot * np.exp(delta))[~out_of_range], rtol=1e-13)


def test_normaliser_moments():
    x = np.array([[1.0, 5.0, 7.0], [2.0, 5.0, 7.0 + 1e-4], [3.0, 5.0, 7.0], [4.0, 5.0, 7.0 + 1e-4]])
    mu, sinv = ol.normaliser(x)
    assert np.allclose(mu, [2.5, 5.0, 7.00005])
    assert np.allclose(sinv, [1.0 / math.sqrt(1.25), 0.0, 0.0])


def test_standardise_clips_and_ignores_constant_columns():
    x = np.array([[0.0, 5.0], [1.0, 5.0], [100.0, 9.0]])
    mu, sinv = ol.normaliser(x[:2])
    u = ol.standardise(x, mu, sinv)
    assert np.allclose(u[:2, 0], [-1.0, 1.0])
    assert u[2, 0] == ol.U_MAX            # far outside the training range: clipped
    assert np.all(u[:, 1] == 0.0)          # no spread in training: ignored


# ---------------------------------------------------------------------------
# Features: per-level slots of a uniform density
# ---------------------------------------------------------------------------

def _exit(lo, hi, p, d):
    t = np.inf
    for a in range(3):
        if d[a] > 0:
            t = min(t, (hi[a] - p[a]) / d[a])
        elif d[a] < 0:
            t = min(t, (lo[a] - p[a]) / d[a])
    return t


def _uniform_slot_terms(n0, box, l0, ijk, d):
    """Per Delta_l: n0 x (exit of the outer box - exit of the inner box) from
    the shell's reference point; Delta_l = 0 is the exit of the oct from the
    leaf centre.  Reference point: centre of the ancestor at min(l+2, l0-1)."""
    ijk = np.array(ijk)
    dx = lambda l: box / (1 << l)
    xt = (ijk + 0.5) * dx(l0)
    oct_lo = (ijk >> 1) * dx(l0 - 1)
    terms = [n0 * _exit(oct_lo, oct_lo + dx(l0 - 1), xt, d)]
    for l in range(l0 - 1, 0, -1):
        r = min(l + 2, l0 - 1)
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
        terms.append(n0 * (_exit(out_lo, out_hi, p, d) - _exit(in_lo, in_hi, p, d)))
    return terms


def _path_leaves(base, lmax, cells):
    """Leaf set refining one cell per level from `base` to `lmax`: cells[l] is
    the index (i, j, k) at level l of the refined cell (l = base..lmax-1)."""
    lv, ijk = [], []
    for l in range(base, lmax + 1):
        n = 1 << l
        if l == base:
            cand = [(i, j, k) for k in range(n) for j in range(n) for i in range(n)]
        else:
            c = np.array(cells[l - 1])
            cand = [tuple(2 * c + np.array([o & 1, (o >> 1) & 1, o >> 2])) for o in range(8)]
        for q in cand:
            if l < lmax and tuple(q) == tuple(cells[l]):
                continue
            lv.append(l)
            ijk.append(q)
    return np.array(lv), np.array(ijk, dtype=np.int64)


def test_slots_of_uniform_density_are_box_exit_differences():
    """A leaf ten levels deep: slots 0..6 are the single levels Delta_l = 0..6
    and slot 7 sums Delta_l = 7, 8 and 9 (the shell of level 1 is empty: the
    3^3 block around a level-1 cell covers the box)."""
    base, lmax, n0, box = 3, 10, 5.0, 10 * PC
    deep = np.array([600, 154, 803])                 # the finest leaf's index at level 10
    cells = {l: tuple(deep >> (lmax - l)) for l in range(base, lmax)}
    lv, ijk = _path_leaves(base, lmax, cells)
    T = oracle.Tree.amr(base, lmax, box, lv.astype(np.int8), ijk.astype(np.int32),
                        np.full(len(lv), n0, dtype=np.float32))
    dirs = oracle.dirs_healpix(1)
    sel = np.flatnonzero(lv == lmax)
    tot, pl = T.column_density(dirs, lv[sel], ijk[sel], per_level=lmax)
    slots = ol.slots_from_levels(pl)
    assert np.allclose(ol.tree_total(slots), tot, rtol=1e-13)
    for r, t in enumerate(sel):
        for di, d in enumerate(dirs):
            terms = _uniform_slot_terms(n0, box, lmax, ijk[t], d)
            want = terms[:7] + [terms[7] + terms[8] + terms[9]]
            assert terms[9] == 0.0
            assert np.allclose(slots[r, :, di], want, rtol=1e-11, atol=1e-11 * max(terms))


def test_features_floor_and_density_column():
    slots = np.zeros((2, ol.SLOTS, 3))
    slots[0, 0] = [1e18, 5e15, 0.0]
    x = ol.features(slots, np.array([30.0, 0.0]))
    assert x.shape == (2, ol.SLOTS * 3 + 1)
    assert x[0, 0] == pytest.approx(math.log(1e18), rel=1e-15)
    assert x[0, 1] == x[0, 2] == math.log(1e16)
    assert x[0, -1] == pytest.approx(math.log(30.0), rel=1e-15)
    assert x[1, -1] == pytest.approx(math.log(1e-10), rel=1e-15)
    assert np.all(x[1, :-1] == math.log(1e16))
