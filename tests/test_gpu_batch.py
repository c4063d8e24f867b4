"""Batched evaluation: per-box launches and the captured graph against
per-box cd_column_density calls (bitwise: the same kernels on the same data)."""
import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import colden, synth

PC = synth.PC_CM
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _boxes(seed=0):
    """Uneven boxes: uniform 8^3 .. 64^3 and AMR meshes, 12 or 48 directions."""
    rng = np.random.default_rng(seed)
    specs = [("u", 3, 48), ("u", 4, 12), ("a", 16, 12), ("u", 5, 48), ("a", 32, 48), ("u", 6, 12), ("u", 4, 48)]
    trees, geoms, rhos = [], [], []
    g12, g48 = colden.precompute_geometry("healpix", 1), colden.precompute_geometry("healpix", 2)
    for kind, size, nd in specs:
        sig = float(rng.uniform(1.0, 2.5))
        if kind == "u":
            rho = synth.lognormal_grf(1 << size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            trees.append(colden.build_tree_uniform(torch.from_numpy(rho).cuda(), 10 * PC))
            rhos.append(rho.reshape(-1))
        else:
            fine = synth.lognormal_grf(size, 30.0, sig, seed=int(rng.integers(1 << 30)))
            lv = synth.amr_leaves(fine, int(np.log2(size)) - 2, [60.0, 120.0])
            trees.append(colden.build_tree_amr(lv["base"], lv["lmax"], 10 * PC, lv["level"], lv["ijk"], lv["rho"]))
            rhos.append(lv["rho"])
        geoms.append(g12 if nd == 12 else g48)
    return trees, geoms, rhos


def _outs(trees, geoms):
    nh = [torch.full((t.n_leaf * g.n_dir,), -1.0, device="cuda") for t, g in zip(trees, geoms)]
    sh = [torch.full((t.n_leaf,), -1.0, device="cuda") for t in trees]
    return nh, sh


def _ref(trees, geoms, precision):
    nh, sh = _outs(trees, geoms)
    for t, g, a, b in zip(trees, geoms, nh, sh):
        colden.column_density(t, g, n_h=a, shield=b, precision=precision)
    torch.cuda.synchronize()
    return [x.cpu() for x in nh], [x.cpu() for x in sh]


@pytest.mark.parametrize("precision", [colden.FP32, colden.BF16])
def test_batch_eager_and_graph_equal_per_box(precision):
    trees, geoms, rhos = _boxes()
    rn, rs = _ref(trees, geoms, precision)
    nh, sh = _outs(trees, geoms)
    colden.column_density_batch(trees, geoms, n_h=nh, shield=sh, precision=precision)
    torch.cuda.synchronize()
    for a, b in zip(nh + sh, rn + rs):
        assert torch.equal(a.cpu(), b)
    nh2, sh2 = _outs(trees, geoms)
    batch = colden.Batch(trees, geoms, n_h=nh2, shield=sh2, precision=precision)
    info = batch.info()
    assert info["width"] in (1, 2, 4, 8) and info["kernel_nodes"] > len(trees)
    for x in nh2 + sh2:
        x.fill_(-1.0)
    batch.run()
    torch.cuda.synchronize()
    for a, b in zip(nh2 + sh2, rn + rs):
        assert torch.equal(a.cpu(), b)
    colden.device_status()
    batch.free()


def test_graph_replay_sees_updated_densities():
    trees, geoms, rhos = _boxes(seed=1)
    nh, sh = _outs(trees, geoms)
    batch = colden.Batch(trees, geoms, n_h=nh, shield=sh)
    rng = np.random.default_rng(5)
    new = [(r * rng.uniform(0.5, 2.0, size=r.shape)).astype(np.float32) for r in rhos]
    for t, r in zip(trees, new):
        colden.tree_update(t, torch.from_numpy(r).cuda())
    batch.run()
    torch.cuda.synchronize()
    got = [x.cpu() for x in nh + sh]
    rn, rs = _ref(trees, geoms, colden.FP32)
    for a, b in zip(got, rn + rs):
        assert torch.equal(a, b)
    batch.free()
