"""Checkpoint round trips on the device: a tree or geometry loaded from its
image gives bit-identical columns to the one it was saved from (uniform and
AMR meshes; HEALPix, M x N, custom and cone geometries), a re-saved image is
byte-identical, a loaded AMR tree takes density updates in output order, and
an image whose tables or directions do not match what the library rebuilds
is refused."""
import struct

import numpy as np
import pytest
import torch

from paper_1410_0624_gb300 import colden, synth

pytestmark = pytest.mark.gpu
BOX = 10 * synth.PC_CM


@pytest.fixture(scope="module", autouse=True)
def _lib():
    colden.load(build_if_missing=True)


def _cols(tree, geom, precision):
    nh = torch.empty(tree.n_leaf * geom.n_dir, device="cuda")
    sh = torch.empty(tree.n_leaf, device="cuda")
    colden.column_density(tree, geom, n_h=nh, shield=sh, precision=precision)
    torch.cuda.synchronize()
    return nh.cpu(), sh.cpu()


def _amr(seed=4):
    fine = synth.lognormal_grf(64, 30.0, 2.0, seed=seed)
    return synth.amr_leaves(fine, 4, [60.0, 120.0])


@pytest.mark.parametrize("kind", ["uniform", "amr"])
def test_tree_image_round_trip(kind):
    g = colden.precompute_geometry("healpix", 2)
    if kind == "uniform":
        rho = synth.lognormal_grf(32, 30.0, 1.5, seed=3)
        t = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    else:
        lv = _amr()
        t = colden.build_tree_amr(lv["base"], lv["lmax"], BOX, lv["level"], lv["ijk"], lv["rho"])
    img = colden.tree_image(t)
    t2 = colden.tree_from_image(img)
    assert (t2.n_leaf, t2.max_level, t2.base_level, t2.n_oct) == (t.n_leaf, t.max_level, t.base_level, t.n_oct)
    for a, b in zip(t.leaves(), t2.leaves()):
        assert np.array_equal(a, b)
    assert colden.tree_image(t2) == img
    for prec in (colden.FP32, colden.BF16):
        for x, y in zip(_cols(t, g, prec), _cols(t2, g, prec)):
            assert torch.equal(x, y)
    if kind == "amr":
        # the loaded tree takes densities in output order (the order saved)
        n = t.n_leaf
        rho_out = np.frombuffer(img, dtype=np.float32, count=n, offset=8 + 12 + 16 + n * 13).copy()
        colden.tree_update(t, torch.from_numpy(np.asarray(lv["rho"], np.float32) * 2).cuda())
        colden.tree_update(t2, torch.from_numpy(rho_out * 2).cuda())
        for x, y in zip(_cols(t, g, colden.FP32), _cols(t2, g, colden.FP32)):
            assert torch.equal(x, y)
    t.free()
    t2.free()
    g.free()


GEOMS = [("healpix", 1, 0, None, colden.MODE_PREC), ("mxn", 4, 6, None, colden.MODE_PREC),
         ("custom", 0, 0, np.random.default_rng(5).normal(size=(20, 3)), colden.MODE_PREC),
         ("healpix", 1, 0, None, colden.MODE_CONE)]


@pytest.mark.parametrize("spec", GEOMS, ids=["healpix", "mxn", "custom", "cone"])
def test_geometry_image_round_trip(spec):
    scheme, p0, p1, dirs, mode = spec
    g = colden.precompute_geometry(scheme, p0, p1, dirs=dirs, mode=mode)
    img = colden.geometry_image(g)
    g2 = colden.geometry_from_image(img)
    assert np.array_equal(g.dirs, g2.dirs) and np.array_equal(g.rays, g2.rays)
    assert colden.geometry_hash(g) == colden.geometry_hash(g2)
    assert colden.geometry_image(g2) == img
    rho = synth.lognormal_grf(32, 30.0, 1.5, seed=8)
    t = colden.build_tree_uniform(torch.from_numpy(rho).cuda(), BOX)
    for prec in (colden.FP32, colden.BF16):
        for x, y in zip(_cols(t, g, prec), _cols(t, g2, prec)):
            assert torch.equal(x, y)
    t.free()
    g.free()
    g2.free()


def _reseal(body: bytes) -> bytes:
    return body + struct.pack("<Q", colden.fnv1a64(body))


def test_geometry_image_with_other_tables_or_directions_is_refused():
    g = colden.precompute_geometry("healpix", 1)
    img = colden.geometry_image(g)
    body = bytearray(img[:-8])
    # the table hash sits just before the image hash
    bad_tab = bytearray(body)
    bad_tab[-1] ^= 1
    # the first stored direction's last bit
    bad_dir = bytearray(body)
    bad_dir[8 + 24] ^= 1
    for b in (bad_tab, bad_dir):
        with pytest.raises(colden.ColdenError) as e:
            colden.geometry_from_image(_reseal(bytes(b)))
        assert e.value.code == colden.CD_EINVAL
    # a flipped byte without resealing fails the image hash
    with pytest.raises(colden.ColdenError):
        colden.geometry_from_image(img[:40] + bytes([img[40] ^ 1]) + img[41:])
    g.free()
