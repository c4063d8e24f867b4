"""The heating epilogue (cd_heating, §5) against the FP64 oracle.

Tolerance: each output is a handful of FP32 operations on FP32 inputs (a
product, a square root, two divisions, two powf calls of at most a few ulps),
so 1e-5 relative holds with a wide margin; the oracle evaluates the same FP32
input values in FP64.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
RTOL = 1e-5

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _inputs(n, seed):
    rng = np.random.default_rng(seed)
    chi = rng.uniform(0.0, 1.0, n).astype(np.float32)
    chi[:7] = [0.0, 1.0, 1e-6, 0.5, 1e-3, 0.25, 0.999]
    T = (10.0 ** rng.uniform(1.0, 4.2, n)).astype(np.float32)
    T[7] = 0.0
    ne = (10.0 ** rng.uniform(-4.0, 0.5, n)).astype(np.float32)
    return chi, T, ne


def _leaf_rho(tree, T_or):
    lv, ijk = tree.leaves()
    return T_or.rho(lv, ijk)


def _cuda(a, offset=0):
    """a copy on the device; offset > 0 gives a view starting `offset` floats
    into a larger buffer (16-byte misaligned for offset 1)."""
    buf = torch.zeros(len(a) + offset, device="cuda")
    buf[offset:] = torch.from_numpy(a).cuda()
    return buf[offset:]


@pytest.mark.parametrize("offset", [0, 1])
def test_heating_parity_uniform(offset):
    L, box = 5, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=61)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    n = tree.n_leaf
    chi, T, ne = _inputs(n, 1)
    outs = [_cuda(np.full(n, -1.0, np.float32), offset) for _ in range(3)]
    colden.heating(tree, _cuda(chi, offset), _cuda(T, offset), _cuda(ne, offset), 1.7, *outs)
    colden.device_status()
    g, uv, cr = (o.double().cpu().numpy() for o in outs)
    nrho = _leaf_rho(tree, oracle.Tree.uniform(rho, box))
    wg, wuv, wcr = oracle.heating(chi, nrho, T, ne, 1.7)
    for got, want in ((g, wg), (uv, wuv), (cr, wcr)):
        nz = want != 0
        assert np.all(got[~nz] == 0)
        assert np.max(np.abs(got[nz] - want[nz]) / want[nz]) <= RTOL


def test_heating_amr_uses_output_order_densities():
    fine = synth.lognormal_grf(32, 30.0, 2.0, seed=7)
    lv = synth.amr_leaves(fine, 3, [40.0, 60.0])
    box = 10 * PC
    # leaves handed over in a shuffled order: the outputs still follow cd_tree_leaves
    perm = np.random.default_rng(3).permutation(len(lv["level"]))
    tree = colden.build_tree_amr(lv["base"], lv["lmax"], box, lv["level"][perm], lv["ijk"][perm], lv["rho"][perm])
    n = tree.n_leaf
    chi, T, ne = _inputs(n, 2)
    uv = torch.empty(n, device="cuda")
    cr = torch.empty(n, device="cuda")
    colden.heating(tree, _cuda(chi), _cuda(T), _cuda(ne), 1.7, gamma_uv=uv, gamma_cr=cr)
    colden.device_status()
    T_or = oracle.Tree.amr(lv["base"], lv["lmax"], box, lv["level"], lv["ijk"], lv["rho"])
    _, wuv, wcr = oracle.heating(chi, _leaf_rho(tree, T_or), T, ne, 1.7)
    got_uv, got_cr = uv.double().cpu().numpy(), cr.double().cpu().numpy()
    nz = wuv != 0
    assert np.max(np.abs(got_uv[nz] - wuv[nz]) / wuv[nz]) <= RTOL
    assert np.max(np.abs(got_cr - wcr) / wcr) <= RTOL


def test_heating_from_the_papers_chi():
    """chi = <exp(-2e-21 N)> from cd_column_density (av_per_nh = 1,
    shield_k = 2e-21), then the heating, against the oracle chain."""
    L, box = 5, 10 * PC
    rho = synth.lognormal_grf(1 << L, 30.0, 2.0, seed=62)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), box)
    geom = colden.precompute_geometry("mxn", 3, 4)          # the 12 directions of §5
    n = tree.n_leaf
    chi = torch.empty(n, device="cuda")
    colden.column_density(tree, geom, shield=chi, av_per_nh=1.0, shield_k=2e-21)
    _, T, ne = _inputs(n, 3)
    uv = torch.empty(n, device="cuda")
    g = torch.empty(n, device="cuda")
    colden.heating(tree, chi, _cuda(T), _cuda(ne), oracle.G0_DRAINE, g0_eff=g, gamma_uv=uv)
    colden.device_status()
    T_or = oracle.Tree.uniform(rho, box)
    lv, ijk = tree.leaves()
    N = T_or.column_density(oracle.dirs_mxn(3, 4), lv, ijk)
    wchi = oracle.chi(N)
    assert np.max(np.abs(chi.double().cpu().numpy() - wchi)) <= 1e-5
    wg, wuv, _ = oracle.heating(wchi, T_or.rho(lv, ijk), T, ne)
    # chi carries an absolute error <= 1e-5, i.e. a relative one of 1e-5 / chi;
    # G0_eff inherits it and Gamma_UV at most twice it (|d ln eps / d ln G0| < 1)
    rel_chi = 1e-5 / wchi
    assert np.all(np.abs(g.double().cpu().numpy() - wg) / wg <= rel_chi + RTOL)
    assert np.all(np.abs(uv.double().cpu().numpy() - wuv) / wuv <= 2 * rel_chi + RTOL)


def test_heating_arguments():
    rho = np.ones((4, 4, 4), np.float32) * 5.0
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), PC)
    chi = torch.ones(64, device="cuda")
    cr = torch.empty(64, device="cuda")
    colden.heating(tree, chi, gamma_cr=cr)                   # T and n_e not needed
    colden.device_status()
    assert torch.all(cr == torch.tensor(5e-27, dtype=torch.float32, device="cuda"))
    uv = torch.empty(64, device="cuda")
    with pytest.raises(colden.ColdenError) as e:
        colden.heating(tree, chi, gamma_uv=uv)
    assert e.value.code == colden.CD_EINVAL
    with pytest.raises(colden.ColdenError) as e:
        colden.heating(tree, chi, G0=-1.0, gamma_cr=cr)
    assert e.value.code == colden.CD_EINVAL
    colden.heating(tree, chi)                                # no outputs: nothing to do
