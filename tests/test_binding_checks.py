"""The Python binding checks every buffer before anything reaches the
library: wrong type, too few elements or another device than the tree's
raise ValueError, and the library is never called (CPU test: the library is
replaced by a stub that fails on any call but cd_opts_default)."""
from unittest import mock

import pytest
import torch

from paper_1410_0624_gb300 import colden


class _Stub:
    def cd_opts_default(self, o):
        pass

    def __getattr__(self, name):
        raise AssertionError("the library was called (%s) although a buffer was invalid" % name)


class _Handle:
    def __init__(self, **kw):
        self.__dict__.update(kw)
        self.handle = colden.ctypes.c_void_p(1)


@pytest.fixture
def stub(monkeypatch):
    monkeypatch.setattr(colden, "_lib", _Stub())
    # CPU tensors stand in for CUDA ones; their device index is None, so the
    # fake tree lives on "device None" as well
    with mock.patch.object(torch.Tensor, "is_cuda", new_callable=mock.PropertyMock, return_value=True):
        yield


def _tree(n_leaf=64, device=None):
    return _Handle(n_leaf=n_leaf, device=device)


def _geom(n_dir=12):
    return _Handle(n_dir=n_dir)


def test_undersized_outputs_rejected(stub):
    t, g = _tree(), _geom()
    ok = torch.empty(64 * 12)
    with pytest.raises(ValueError, match="n_h holds 767"):
        colden.column_density(t, g, n_h=torch.empty(64 * 12 - 1))
    with pytest.raises(ValueError, match="a_v"):
        colden.column_density(t, g, n_h=ok, a_v=torch.empty(10))
    with pytest.raises(ValueError, match="shield holds 63"):
        colden.column_density(t, g, shield=torch.empty(63))
    with pytest.raises(ValueError, match="shield"):
        colden.column_density_noalloc(t, g, shield=torch.empty(1))
    with pytest.raises(ValueError, match="gamma_cr"):
        colden.heating(t, torch.empty(64), gamma_cr=torch.empty(63))


def test_wrong_type_and_device_rejected(stub):
    t, g = _tree(), _geom()
    with pytest.raises(ValueError, match="float32"):
        colden.column_density(t, g, n_h=torch.empty(64 * 12, dtype=torch.float64))
    with pytest.raises(ValueError, match="contiguous"):
        colden.column_density(t, g, n_h=torch.empty(2 * 64 * 12)[::2])
    with pytest.raises(ValueError, match="cuda:3"):
        colden.column_density(_tree(device=3), g, n_h=torch.empty(64 * 12))


def test_batch_outputs_rejected_per_box(stub):
    trees, geoms = [_tree(64), _tree(512)], [_geom(12), _geom(48)]
    good = [torch.empty(64 * 12), torch.empty(512 * 48)]
    bad = [torch.empty(64 * 12), torch.empty(512 * 48 - 4)]
    with pytest.raises(ValueError, match="n_h of box 1"):
        colden.column_density_batch(trees, geoms, n_h=bad)
    with pytest.raises(ValueError, match="shield of box 0"):
        colden.column_density_batch(trees, geoms, n_h=good, shield=[torch.empty(1), None])
    with pytest.raises(ValueError, match="lists 1 buffers"):
        colden.Batch(trees, geoms, n_h=good[:1])
    with pytest.raises(ValueError, match="geometries"):
        colden.Batch(trees, geoms[:1], n_h=good)


def test_eval_graph_buffers_checked_before_the_library(stub):
    """colden.EvalGraph checks rho (n_leaf floats) and the outputs as the
    evaluation does, before cd_eval_graph_create is reached."""
    t, g = _tree(), _geom()
    with pytest.raises(ValueError, match="rho holds 63"):
        colden.EvalGraph(t, g, rho=torch.empty(63), n_h=torch.empty(64 * 12))
    with pytest.raises(ValueError, match="n_h holds 767"):
        colden.EvalGraph(t, g, rho=torch.empty(64), n_h=torch.empty(64 * 12 - 1))
    with pytest.raises(ValueError, match="shield"):
        colden.EvalGraph(t, g, shield=torch.empty(10))
    with pytest.raises(ValueError):
        colden.EvalGraph(t, g, rho=torch.empty(64, dtype=torch.float64))


def test_fit_delta_range_passes_the_target_count(monkeypatch):
    """Net.fit_delta_range hands the library every target (numel) and the
    margin; the range it reports is the library's."""
    calls = {}

    class Lib:
        def cd_net_fit_delta_range(self, h, n, y, margin, stream):
            calls.update(n=n, margin=margin)
            return 0

        def cd_net_get_delta_range(self, h, lo, hi):
            lo._obj.value, hi._obj.value = -1.5, 2.5
            return 0

    monkeypatch.setattr(colden, "_lib", Lib())
    net = object.__new__(colden.Net)
    net._h = colden.ctypes.c_void_p(1)
    with mock.patch.object(torch.Tensor, "is_cuda", new_callable=mock.PropertyMock, return_value=True):
        got = net.fit_delta_range(torch.empty(7, 48), 0.25, stream=0)
    net._h = None
    assert calls == {"n": 7 * 48, "margin": 0.25}
    assert got == (-1.5, 2.5)
