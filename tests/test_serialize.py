"""Checkpoint images (cd_tree_save/load, cd_geom_save/load): the checksum
against the published FNV-1a test vectors, and the host-side refusal of
damaged or foreign images (no GPU needed: the checks run before any device
work)."""
import struct

import pytest

from paper_1410_0624_gb300 import _build, colden


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return colden.load()


def test_fnv1a64_published_vectors(lib):
    # FNV-1a 64-bit test vectors of the algorithm's authors
    assert colden.fnv1a64(b"") == 0xCBF29CE484222325
    assert colden.fnv1a64(b"a") == 0xAF63DC4C8601EC8C
    assert colden.fnv1a64(b"foobar") == 0x85944171F73967E8


def _sealed(body: bytes) -> bytes:
    return body + struct.pack("<Q", colden.fnv1a64(body))


@pytest.mark.parametrize("loader", ["tree", "geom"])
def test_damaged_and_foreign_images_are_refused(lib, loader):
    load = colden.tree_from_image if loader == "tree" else colden.geometry_from_image
    cases = [
        b"",                                                   # empty
        b"\x00" * 7,                                           # shorter than a hash
        b"CDTREE01" + b"\x00" * 40,                            # hash does not match
        _sealed(b"XXXXXXXX" + b"\x00" * 40),                   # sealed, wrong magic
    ]
    if loader == "tree":
        # sealed, right magic, sizes that do not add up (n_leaf = 5, no arrays)
        cases.append(_sealed(b"CDTREE01" + struct.pack("<iiidq", 0, 1, 1, 1.0, 5)))
        # sealed, uniform, n_leaf not 8^L
        cases.append(_sealed(b"CDTREE01" + struct.pack("<iiidq", 0, 1, 1, 1.0, 1) + b"\x01" + b"\x00" * 16))
    else:
        # sealed, right magic, n_dir = 0
        cases.append(_sealed(b"CDGEOM01" + struct.pack("<iiiiii", 0, 1, 0, 0, 0, 0) + b"\x00" * 16))
        # sealed, sizes that do not add up (12 dirs declared, none stored)
        cases.append(_sealed(b"CDGEOM01" + struct.pack("<iiiiii", 0, 1, 0, 0, 12, 0) + b"\x00" * 16))
    for img in cases:
        with pytest.raises(colden.ColdenError) as e:
            load(img, stream=0)   # the legacy stream handle: nothing reaches the device
        assert e.value.code == colden.CD_EINVAL, (img[:16], e.value)
