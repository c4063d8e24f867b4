"""cd_column_density_host: densities from and results to host memory.  The
host results equal the device entry point's bit for bit: uniform trees with
the chunked leaf stage (copies overlapped) and without it (small trees), AMR
trees, FP32 and BF16, pinned and pageable buffers, any subset of outputs,
with and without new densities."""
import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import colden, synth

pytestmark = pytest.mark.gpu
BOX = 10 * synth.PC_CM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _device(tree, geom, prec):
    nh = torch.empty(tree.n_leaf * geom.n_dir, device="cuda")
    av = torch.empty_like(nh)
    sh = torch.empty(tree.n_leaf, device="cuda")
    colden.column_density(tree, geom, n_h=nh, a_v=av, shield=sh, precision=prec)
    torch.cuda.synchronize()
    return nh.cpu(), av.cpu(), sh.cpu()


@pytest.mark.parametrize("L", [3, 5, 6])
@pytest.mark.parametrize("prec", [colden.FP32, colden.BF16])
def test_uniform_host_outputs_equal_device_outputs(L, prec):
    g = colden.precompute_geometry("healpix", 2)
    rho = synth.lognormal_grf(1 << L, 30.0, 1.8, seed=L)
    t = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    ref = _device(t, g, prec)
    n = t.n_leaf * g.n_dir
    h = [torch.full((n,), -1.0).pin_memory(), torch.full((n,), -1.0).pin_memory(),
         torch.full((t.n_leaf,), -1.0).pin_memory()]
    colden.column_density_host(t, g, n_h=h[0], a_v=h[1], shield=h[2], precision=prec)
    torch.cuda.synchronize()
    for a, b in zip(h, ref):
        assert torch.equal(a, b)
    # new densities from the host, pageable numpy outputs, a subset of the outputs
    rho2 = (rho * np.float32(1.7)).astype(np.float32)
    nh = np.full(n, -1.0, np.float32)
    sh = np.full(t.n_leaf, -1.0, np.float32)
    colden.column_density_host(t, g, rho=np.ascontiguousarray(rho2.reshape(-1)), n_h=nh, shield=sh, precision=prec)
    torch.cuda.synchronize()
    t2 = colden.build_tree_uniform(torch.from_numpy(rho2).cuda(), BOX)
    ref2 = _device(t2, g, prec)
    assert np.array_equal(nh, ref2[0].numpy()) and np.array_equal(sh, ref2[2].numpy())
    # the tree itself now holds the new densities
    ref3 = _device(t, g, prec)
    assert torch.equal(ref3[0], ref2[0])
    t.free()
    t2.free()
    g.free()


def test_amr_host_outputs_equal_device_outputs():
    g = colden.precompute_geometry("healpix", 1)
    lv = synth.amr_leaves(synth.lognormal_grf(64, 30.0, 2.0, seed=5), 4, [60.0, 120.0])
    t = colden.build_tree_amr(lv["base"], lv["lmax"], BOX, lv["level"], lv["ijk"], lv["rho"])
    for prec in (colden.FP32, colden.BF16):
        ref = _device(t, g, prec)
        n = t.n_leaf * g.n_dir
        h = [torch.empty(n).pin_memory(), torch.empty(n).pin_memory(), torch.empty(t.n_leaf).pin_memory()]
        colden.column_density_host(t, g, rho=np.asarray(lv["rho"], np.float32), n_h=h[0], a_v=h[1], shield=h[2],
                                   precision=prec)
        torch.cuda.synchronize()
        for a, b in zip(h, ref):
            assert torch.equal(a, b)
    t.free()
    g.free()
