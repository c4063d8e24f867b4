"""The in-situ variant (§4.3: every shell seen from the oct centre) through the
C ABI against the FP64 oracle's in-situ mode, and the accuracy statement of
Table 1 (precalculated vs in-situ extinction maps).

Tolerance: the GPU walks each shell's cells in FP32 with every crossing
recomputed from its face; the sum over a shell's few cells and over the levels
is a positive sum, held to 1e-5 relative like the FP32 path."""
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
SIGMA = 2e-21
RTOL = 1e-5
pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_prec_vs_insitu.txt")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _run(tree, geom, precision=colden.FP32):
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=precision)
    colden.device_status()
    return n_h.reshape(-1, nd).double().cpu().numpy(), sh.double().cpu().numpy()


@pytest.mark.parametrize("L", [2, 3, 5, 6])
@pytest.mark.parametrize("dset", [("healpix", 2, 0), ("mxn", 5, 8), ("axes", 0, 0)])
def test_insitu_uniform_matches_oracle(L, dset):
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=50 + L)
    box = 10 * PC
    tree = colden.build_tree_uniform(rho, box)
    geom = colden.precompute_geometry(dset[0], dset[1], dset[2], mode=colden.MODE_INSITU)
    got, sh = _run(tree, geom)
    _, ijk = tree.leaves()
    sel = np.random.default_rng(L).choice(tree.n_leaf, min(tree.n_leaf, 600), replace=False)
    T = oracle.Tree.uniform(rho, box)
    ref = T.column_density(geom.dirs, np.full(len(sel), L), ijk[sel], mode=oracle.MODE_INSITU)
    assert np.max(np.abs(got[sel] - ref) / ref) <= RTOL
    assert np.max(np.abs(sh[sel] - oracle.shield(ref))) <= 1e-5


def test_insitu_amr_matches_oracle():
    fine = synth.lognormal_grf(64, 30.0, 2.0, seed=61)
    lv = synth.amr_leaves(fine, 4, [40.0, 60.0])
    box = 10 * PC
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    geom = colden.precompute_geometry("healpix", 2, mode=colden.MODE_INSITU)
    got, _ = _run(tree, geom, precision=colden.BF16)       # in-situ runs FP32 whatever is asked
    olv, oijk = tree.leaves()
    T = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    ref = T.column_density(geom.dirs, olv, oijk, mode=oracle.MODE_INSITU)
    assert np.max(np.abs(got - ref) / ref) <= RTOL


def test_insitu_equals_prec_when_every_shell_is_exact():
    """With leaves at level 4 every shell is Delta_l <= 3, where the two-level
    approximation is exact (§3.3): two different GPU computations of the same
    numbers."""
    rho = synth.lognormal_grf(16, 30.0, 2.0, seed=62)
    tree = colden.build_tree_uniform(rho, 10 * PC)
    a, _ = _run(tree, colden.precompute_geometry("healpix", 2))
    b, _ = _run(tree, colden.precompute_geometry("healpix", 2, mode=colden.MODE_INSITU))
    assert np.max(np.abs(a - b) / a) <= RTOL


def test_prec_vs_insitu_extinction_table1():
    """Table 1: <|chi_prec - chi_in_situ|> of 0.0028 / 0.0037 / 0.0034 for
    12 / 40 / 84 directions on the paper's turbulent cloud.  On a seeded
    turbulent-like field (256^3, k^-11/3 log-normal, sigma_ln 2, 10 pc) the
    differences must be of that order (below 0.01) and the two forms must
    agree on the mean column to a few per cent (Table 1's ~7 % in N)."""
    want = {int(r.split()[0]): float(r.split()[1]) for r in open(GOLDEN) if r.strip() and not r.startswith("#")}
    rho = synth.lognormal_grf_torch(256, 30.0, 2.0, 2, device="cuda").contiguous()
    tree = colden.build_tree_uniform(rho, 10 * PC)
    for ndir, (M, N) in {12: (3, 4), 40: (5, 8), 84: (7, 12)}.items():
        out = {}
        for mode in (colden.MODE_PREC, colden.MODE_INSITU):
            geom = colden.precompute_geometry("mxn", M, N, mode=mode)
            n_h = torch.empty(tree.n_leaf * ndir, device="cuda")
            colden.column_density(tree, geom, n_h=n_h, precision=colden.FP32)
            out[mode] = n_h.reshape(-1, ndir)
        chi = {m: torch.exp(-SIGMA * v.double()).mean(dim=1) for m, v in out.items()}
        dchi = float((chi[colden.MODE_PREC] - chi[colden.MODE_INSITU]).abs().mean())
        dn = float(((out[colden.MODE_PREC] - out[colden.MODE_INSITU]).abs() / out[colden.MODE_INSITU]).mean())
        print("directions %d: <|chi_prec - chi_insitu|> = %.4f (Table 1: %.4f); <|dN|/N> = %.4f" % (ndir, dchi, want[ndir], dn))
        assert dchi < 0.01
        assert dn < 0.15
