"""Failure detection on the GPU without a fault.

Every pipeline wait of the library's kernels is bounded: a wait that runs out
sets a device flag, the kernel lets the copies and tensor-core products it has
issued land (with the full limit), frees its tensor memory and returns, and
cd_device_status reports CD_ETIMEOUT.  The testing hook cd_debug_wait_polls(0)
makes the pipeline waits of the tensor-core leaf kernel (the BF16 leaf
epilogue; here with 24 M x N directions) give up without polling, so every
CTA takes that path; nothing
traps and the context stays usable: the flag is cleared by the report and the
next evaluation matches the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1410_0624_gb300 import colden, synth

pytestmark = pytest.mark.gpu
BOX = 10 * synth.PC_CM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _oracle_check(tree, rho, n_h, sh, nd, rows):
    lv, ijk = tree.leaves()
    ref = oracle.Tree.uniform(rho, BOX).column_density(oracle.dirs_mxn(4, 6), lv[rows], ijk[rows])
    got = n_h.reshape(-1, nd)[torch.from_numpy(rows).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - ref) / ref) <= 1e-2
    assert np.max(np.abs(sh.cpu().numpy()[rows] - oracle.shield(ref))) <= 5e-3


def test_bounded_wait_runs_out_and_the_context_recovers():
    rho = synth.lognormal_grf(32, 30.0, 2.0, seed=61)
    tree = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    geom = colden.precompute_geometry("mxn", 4, 6)     # 24 directions
    nd = geom.n_dir
    n_h = torch.full((tree.n_leaf * nd,), -1.0, device="cuda")
    sh = torch.full((tree.n_leaf,), -1.0, device="cuda")
    colden.device_status()                      # no flag left over from earlier work
    colden.debug_wait_polls(0)
    try:
        colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16)
        with pytest.raises(colden.ColdenError) as e:
            colden.device_status()
        assert e.value.code == colden.CD_ETIMEOUT and "bounded wait" in str(e.value)
    finally:
        colden.debug_wait_polls(-1)
    # every CTA gave up before its first tile: no row was written
    assert torch.all(sh == -1.0)
    colden.device_status()                      # the report cleared the flag
    colden.column_density(tree, geom, n_h=n_h, shield=sh, precision=colden.BF16)
    colden.device_status()
    rows = np.random.default_rng(3).choice(tree.n_leaf, size=300, replace=False)
    _oracle_check(tree, rho, n_h, sh, nd, rows)
