"""Thin ctypes binding of libcolden.so (include/colden.h).

Argument marshalling only: every step of the column-density path runs in the
library's CUDA kernels.  PyTorch provides device memory and streams.  There is
no CPU fallback: if the library is missing or was not built, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

from . import _build

CD_OK, CD_EINVAL, CD_ENOMEM, CD_ECUDA, CD_ETIMEOUT, CD_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
DIRS_HEALPIX, DIRS_MXN, DIRS_AXES, DIRS_CUSTOM = 0, 1, 2, 3
MODE_PREC, MODE_INSITU, MODE_CONE = 0, 1, 2
FP32, BF16 = 0, 1

_STATUS = {CD_EINVAL: "EINVAL", CD_ENOMEM: "ENOMEM", CD_ECUDA: "ECUDA", CD_ETIMEOUT: "ETIMEOUT",
           CD_EUNSUPPORTED: "EUNSUPPORTED"}

# every symbol include/colden.h declares (checked by the ABI test)
EXPORTS = (
    "cd_opts_default", "cd_build_tree_uniform", "cd_build_tree_amr", "cd_tree_update", "cd_precompute_geometry",
    "cd_column_density", "cd_tree_info", "cd_tree_leaves", "cd_geom_info", "cd_geom_rays", "cd_stats_reset",
    "cd_stats_get", "cd_heating",
    "cd_tree_free", "cd_geom_free", "cd_last_error", "cd_column_density_noalloc", "cd_device_status",
    "cd_column_density_batch", "cd_batch_create", "cd_batch_run", "cd_batch_info", "cd_batch_plan", "cd_batch_free",
    "cd_debug_wait_polls", "cd_debug_batch_form", "cd_stats_flops", "cd_debug_leaf_span",
    "cd_tree_save", "cd_tree_load", "cd_geom_save", "cd_geom_load", "cd_geom_hash", "cd_fnv1a64",
    "cd_checked_status", "cd_debug_check_probe", "cd_column_density_host",
    "cd_eval_graph_create", "cd_eval_graph_launch", "cd_eval_graph_info", "cd_eval_graph_free",
    # include/colden_learned.h
    "cd_adam_default", "cd_net_num_params", "cd_raymarch", "cd_learned_features", "cd_learned_targets",
    "cd_net_create", "cd_net_fit_normaliser", "cd_net_forward", "cd_net_loss_grad", "cd_net_train_step",
    "cd_net_get_state", "cd_net_set_state", "cd_net_info", "cd_net_free", "cd_net_set_delta_range",
    "cd_net_get_delta_range", "cd_net_fit_delta_range",
)
_VOID = ("cd_opts_default", "cd_tree_free", "cd_geom_free", "cd_last_error", "cd_stats_reset", "cd_batch_free",
         "cd_eval_graph_free", "cd_debug_leaf_span",
         "cd_adam_default", "cd_net_free", "cd_net_num_params", "cd_debug_wait_polls", "cd_debug_batch_form")
K_RESTRICT, K_SHELL, K_LEAF, K_OTHER, K_NET, K_FEATURES, K_RAYMARCH, K_LEARNED, K_HEATING = range(9)
KERNEL_KINDS = ("restrict", "shell", "leaf", "other", "net", "features", "raymarch", "learned", "heating")


class ColdenError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_STATUS.get(code, code), msg))
        self.code = code


class Adam(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_double), ("beta1", ctypes.c_double), ("beta2", ctypes.c_double),
                ("eps", ctypes.c_double)]


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("reserved0", ctypes.c_int), ("av_per_nh", ctypes.c_double),
                ("shield_k", ctypes.c_double), ("net", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Loads libcolden.so (libcolden_checked.so, the bounds-checked test build,
    when the environment sets COLDEN_CHECKED=1); raises if it is absent (no
    fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    checked = os.environ.get("COLDEN_CHECKED") == "1"
    path = _build.LIB_CHECKED if checked else _build.LIB
    if not os.path.exists(path):
        if build_if_missing:
            _build.build(checked=checked)
        else:
            raise RuntimeError("%s is not built (run __graft_entry__.build())" % os.path.basename(path))
    L = ctypes.CDLL(path)
    P, I, D, I64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    L.cd_opts_default.argtypes = [ctypes.POINTER(Opts)]
    L.cd_opts_default.restype = None
    L.cd_build_tree_uniform.argtypes = [I, D, P, I, P, ctypes.POINTER(P)]
    L.cd_tree_update.argtypes = [P, P, I, P]
    L.cd_build_tree_amr.argtypes = [I, I, D, I64, P, P, P, I, P, ctypes.POINTER(P)]
    L.cd_stats_reset.argtypes = [I]
    L.cd_stats_reset.restype = None
    L.cd_stats_get.argtypes = [I, ctypes.POINTER(I64), ctypes.POINTER(D)]
    L.cd_stats_flops.argtypes = [I, ctypes.POINTER(D)]
    L.cd_precompute_geometry.argtypes = [I, I, I, P, I, I, P, ctypes.POINTER(P)]
    L.cd_column_density.argtypes = [P, P, ctypes.POINTER(Opts), P, P, P, P]
    L.cd_column_density_noalloc.argtypes = [P, P, ctypes.POINTER(Opts), P, P, P, P]
    L.cd_device_status.argtypes = [P]
    L.cd_debug_wait_polls.argtypes = [I64]
    L.cd_debug_wait_polls.restype = None
    L.cd_debug_batch_form.argtypes = [I]
    L.cd_debug_leaf_span.argtypes = [I]
    L.cd_debug_batch_form.restype = None
    SZ = ctypes.c_size_t
    L.cd_tree_save.argtypes = [P, P, SZ, ctypes.POINTER(SZ), P]
    L.cd_tree_load.argtypes = [P, SZ, P, ctypes.POINTER(P)]
    L.cd_geom_save.argtypes = [P, P, SZ, ctypes.POINTER(SZ)]
    L.cd_geom_load.argtypes = [P, SZ, P, ctypes.POINTER(P)]
    L.cd_geom_hash.argtypes = [P, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64)]
    L.cd_column_density_host.argtypes = [P, P, ctypes.POINTER(Opts), P, P, P, P, P]
    L.cd_checked_status.argtypes = [ctypes.POINTER(I), ctypes.POINTER(I64)]
    L.cd_debug_check_probe.argtypes = [I64, P]
    L.cd_fnv1a64.argtypes = [P, SZ]
    L.cd_fnv1a64.restype = ctypes.c_uint64
    L.cd_column_density_batch.argtypes = [I, P, P, ctypes.POINTER(Opts), P, P, P, P]
    L.cd_batch_create.argtypes = [I, P, P, ctypes.POINTER(Opts), P, P, P, P, ctypes.POINTER(P)]
    L.cd_batch_run.argtypes = [P, P]
    L.cd_batch_info.argtypes = [P, ctypes.POINTER(I), P, ctypes.POINTER(I64)]
    L.cd_batch_plan.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), P]
    L.cd_eval_graph_create.argtypes = [P, P, ctypes.POINTER(Opts), P, P, P, P, P, ctypes.POINTER(P)]
    L.cd_eval_graph_launch.argtypes = [P, P]
    L.cd_eval_graph_info.argtypes = [P, ctypes.POINTER(I64)]
    L.cd_eval_graph_free.argtypes = [P]
    L.cd_eval_graph_free.restype = None
    L.cd_batch_free.argtypes = [P]
    L.cd_batch_free.restype = None
    L.cd_tree_info.argtypes = [P, ctypes.POINTER(I64), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I64)]
    L.cd_tree_leaves.argtypes = [P, P, P]
    L.cd_geom_info.argtypes = [P, ctypes.POINTER(I), P]
    L.cd_geom_rays.argtypes = [P, ctypes.POINTER(I), P]
    L.cd_heating.argtypes = [P, P, P, P, ctypes.c_double, P, P, P, P]
    L.cd_tree_free.argtypes = [P]
    L.cd_tree_free.restype = None
    L.cd_geom_free.argtypes = [P]
    L.cd_geom_free.restype = None
    L.cd_last_error.argtypes = []
    L.cd_last_error.restype = ctypes.c_char_p
    L.cd_adam_default.argtypes = [ctypes.POINTER(Adam)]
    L.cd_adam_default.restype = None
    L.cd_net_num_params.argtypes = [I, I]
    L.cd_net_num_params.restype = I64
    L.cd_raymarch.argtypes = [P, P, I64, P, P, P]
    L.cd_learned_features.argtypes = [P, P, I64, P, P, P, P]
    L.cd_learned_targets.argtypes = [I64, P, P, P, P]
    L.cd_net_create.argtypes = [I, I, P, ctypes.POINTER(P)]
    L.cd_net_fit_normaliser.argtypes = [P, I64, P, P]
    L.cd_net_forward.argtypes = [P, I64, P, P, P]
    L.cd_net_loss_grad.argtypes = [P, I64, P, P, P, P, P, P]
    L.cd_net_train_step.argtypes = [P, I64, P, P, P, ctypes.POINTER(Adam), P, P]
    L.cd_net_get_state.argtypes = [P, P, P, P, P, P, ctypes.POINTER(I64)]
    L.cd_net_set_state.argtypes = [P, P, P, P, P, P, I64]
    L.cd_net_info.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I64)]
    L.cd_net_set_delta_range.argtypes = [P, ctypes.c_double, ctypes.c_double]
    L.cd_net_get_delta_range.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.cd_net_fit_delta_range.argtypes = [P, I64, P, ctypes.c_double, P]
    L.cd_net_free.argtypes = [P]
    L.cd_net_free.restype = None
    for name in EXPORTS:
        if name not in _VOID and name != "cd_fnv1a64":   # the rest return cd_status
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


def _check(code):
    if code != CD_OK:
        raise ColdenError(code, load().cd_last_error().decode(errors="replace"))


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dptr(t, numel=None, device=None, name="buffer"):
    """Device pointer of a contiguous float32 CUDA tensor (or None).  Raises
    ValueError, before anything is enqueued, when the tensor has the wrong
    type, holds fewer than `numel` elements or lives on another device than
    `device` (the tree's)."""
    return _checked_ptr(t, "float32", numel, device, name)


def _checked_ptr(t, dtype_name, numel, device, name):
    if t is None:
        return None
    import torch
    dtype = getattr(torch, dtype_name)
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous %s CUDA tensor" % (name, dtype_name))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s holds %d elements but %d are needed" % (name, t.numel(), numel))
    if device is not None and t.device.index != device:
        raise ValueError("%s is on cuda:%s but the tree is on cuda:%s" % (name, t.device.index, device))
    return t.data_ptr()


def _current_device():
    import torch
    return torch.cuda.current_device()


def opts_default() -> Opts:
    o = Opts()
    load().cd_opts_default(ctypes.byref(o))
    return o


class Tree:
    """Library-owned octree (cd_tree)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        n_leaf, n_oct = ctypes.c_int64(), ctypes.c_int64()
        lmax, base = ctypes.c_int(), ctypes.c_int()
        _check(load().cd_tree_info(self._h, ctypes.byref(n_leaf), ctypes.byref(lmax), ctypes.byref(base),
                                   ctypes.byref(n_oct)))
        self.n_leaf, self.max_level, self.base_level, self.n_oct = n_leaf.value, lmax.value, base.value, n_oct.value
        self.device = _current_device()   # trees live on the device current at build time

    @property
    def handle(self):
        return self._h

    def leaves(self):
        """(level int8 [n], ijk int32 [n, 3]) of every leaf in output order."""
        lv = np.zeros(self.n_leaf, dtype=np.int8)
        ijk = np.zeros((self.n_leaf, 3), dtype=np.int32)
        _check(load().cd_tree_leaves(self._h, lv.ctypes.data_as(ctypes.c_void_p),
                                     ijk.ctypes.data_as(ctypes.c_void_p)))
        return lv, ijk

    def free(self):
        if self._h is not None and self._h.value:
            load().cd_tree_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Geometry:
    """Library-owned geometry tables (cd_geom)."""

    def __init__(self, handle):
        self._h = ctypes.c_void_p(handle)
        nd = ctypes.c_int()
        _check(load().cd_geom_info(self._h, ctypes.byref(nd), None))
        self.n_dir = nd.value
        d = np.zeros((self.n_dir, 3))
        _check(load().cd_geom_info(self._h, ctypes.byref(nd), d.ctypes.data_as(ctypes.c_void_p)))
        self.dirs = d
        ns = ctypes.c_int()
        _check(load().cd_geom_rays(self._h, ctypes.byref(ns), None))
        self.n_sub = ns.value
        r = np.zeros((self.n_dir, self.n_sub, 3))
        _check(load().cd_geom_rays(self._h, ctypes.byref(ns), r.ctypes.data_as(ctypes.c_void_p)))
        self.rays = r

    @property
    def handle(self):
        return self._h

    def free(self):
        if self._h is not None and self._h.value:
            load().cd_geom_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_tree_uniform(rho, box_cm: float, stream=None) -> Tree:
    """cd_build_tree_uniform.  rho: [n, n, n] float32 indexed [z, y, x]; a CUDA
    tensor (device path) or a numpy array / CPU tensor (host path)."""
    import torch
    if isinstance(rho, torch.Tensor) and rho.is_cuda:
        ptr, on_dev, keep = _dptr(rho, name="rho"), 1, rho
    else:
        keep = np.ascontiguousarray(rho.cpu().numpy() if isinstance(rho, torch.Tensor) else rho, dtype=np.float32)
        ptr, on_dev = keep.ctypes.data, 0
    n = keep.shape[0]
    L = int(n).bit_length() - 1
    if keep.shape != (n, n, n) or (1 << L) != n:
        raise ValueError("rho must be a cube of side 2^L")
    h = ctypes.c_void_p()
    _check(load().cd_build_tree_uniform(L, float(box_cm), ctypes.c_void_p(ptr), on_dev,
                                        ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return Tree(h.value)


def build_tree_amr(base_level: int, max_level: int, box_cm: float, level, ijk, rho, stream=None) -> Tree:
    """cd_build_tree_amr.  level int8 [n], ijk int32 [n, 3] (host); rho float32
    [n] as a CUDA tensor (device path) or numpy / CPU tensor (host path)."""
    import torch
    lv = np.ascontiguousarray(level, dtype=np.int8).reshape(-1)
    ix = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
    if isinstance(rho, torch.Tensor) and rho.is_cuda:
        if rho.numel() != lv.shape[0]:
            raise ValueError("rho holds %d values for %d leaves" % (rho.numel(), lv.shape[0]))
        ptr, on_dev = _dptr(rho, name="rho"), 1
    else:
        keep = np.ascontiguousarray(rho.cpu().numpy() if isinstance(rho, torch.Tensor) else rho, dtype=np.float32)
        if keep.size != lv.shape[0]:
            raise ValueError("rho holds %d values for %d leaves" % (keep.size, lv.shape[0]))
        ptr, on_dev = keep.ctypes.data, 0
    if ix.shape[0] != lv.shape[0]:
        raise ValueError("ijk holds %d rows for %d leaves" % (ix.shape[0], lv.shape[0]))
    h = ctypes.c_void_p()
    _check(load().cd_build_tree_amr(int(base_level), int(max_level), float(box_cm), lv.shape[0],
                                    lv.ctypes.data_as(ctypes.c_void_p), ix.ctypes.data_as(ctypes.c_void_p),
                                    ctypes.c_void_p(ptr), on_dev, ctypes.c_void_p(_stream_ptr(stream)),
                                    ctypes.byref(h)))
    return Tree(h.value)


def tree_update(tree: Tree, rho, stream=None) -> Tree:
    """cd_tree_update: new leaf densities for an existing uniform tree."""
    import torch
    if isinstance(rho, torch.Tensor) and rho.is_cuda:
        if rho.numel() != tree.n_leaf:
            raise ValueError("rho holds %d values for %d leaves" % (rho.numel(), tree.n_leaf))
        ptr, on_dev = _dptr(rho, device=tree.device, name="rho"), 1
    else:
        keep = np.ascontiguousarray(rho.cpu().numpy() if isinstance(rho, torch.Tensor) else rho, dtype=np.float32)
        if keep.size != tree.n_leaf:
            raise ValueError("rho holds %d values for %d leaves" % (keep.size, tree.n_leaf))
        ptr, on_dev = keep.ctypes.data, 0
    _check(load().cd_tree_update(tree.handle, ctypes.c_void_p(ptr), on_dev, ctypes.c_void_p(_stream_ptr(stream))))
    return tree


def device_status(stream=None):
    """cd_device_status: raises ColdenError(CD_ETIMEOUT) if a kernel gave up a bounded wait."""
    _check(load().cd_device_status(ctypes.c_void_p(_stream_ptr(stream))))


def debug_wait_polls(polls: int):
    """cd_debug_wait_polls (tests only): cap the BF16 leaf kernel's pipeline
    waits at `polls` polls (0: they give up at once); negative restores the
    default."""
    load().cd_debug_wait_polls(int(polls))


def checked_status():
    """cd_checked_status: (site, index) of the first out-of-bounds gather the
    checked build recorded since the last call, (0, 0) when none."""
    site, index = ctypes.c_int(), ctypes.c_int64()
    _check(load().cd_checked_status(ctypes.byref(site), ctypes.byref(index)))
    return site.value, index.value


def debug_check_probe(i: int, stream=None):
    """cd_debug_check_probe (checked build): a read of element i of a 4-element array through the check."""
    _check(load().cd_debug_check_probe(int(i), ctypes.c_void_p(_stream_ptr(stream))))


def debug_batch_form(form: int):
    """cd_debug_batch_form (tests only): 0 = later Batch objects use the per-box
    form, 1 = the persistent form where supported, negative = the autotuner
    chooses."""
    load().cd_debug_batch_form(int(form))


def debug_leaf_span(rows: int):
    """cd_debug_leaf_span (tests only): the widest parent span an AMR list
    tile stages as one copy; 0 forces one row per oct, negative restores 16."""
    load().cd_debug_leaf_span(int(rows))


def stats_reset(timing: bool = False):
    load().cd_stats_reset(1 if timing else 0)


def stats_flops(kind: int) -> float:
    """Dense tensor-core flops issued by one kernel kind since the last reset."""
    f = ctypes.c_double()
    _check(load().cd_stats_flops(int(kind), ctypes.byref(f)))
    return f.value


def stats_get(kind: int):
    """(launches, milliseconds) of one kernel kind since the last reset."""
    n, ms = ctypes.c_int64(), ctypes.c_double()
    _check(load().cd_stats_get(int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def tree_image(tree: Tree, stream=None) -> bytes:
    """cd_tree_save: the tree's checkpoint image (mesh and current densities)."""
    size = ctypes.c_size_t()
    _check(load().cd_tree_save(tree.handle, None, 0, ctypes.byref(size), ctypes.c_void_p(_stream_ptr(stream))))
    buf = ctypes.create_string_buffer(size.value)
    _check(load().cd_tree_save(tree.handle, buf, size.value, ctypes.byref(size), ctypes.c_void_p(_stream_ptr(stream))))
    return buf.raw


def tree_from_image(image: bytes, stream=None) -> Tree:
    """cd_tree_load."""
    h = ctypes.c_void_p()
    _check(load().cd_tree_load(image, len(image), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return Tree(h.value)


def geometry_image(geom: Geometry) -> bytes:
    """cd_geom_save: the geometry's checkpoint image."""
    size = ctypes.c_size_t()
    _check(load().cd_geom_save(geom.handle, None, 0, ctypes.byref(size)))
    buf = ctypes.create_string_buffer(size.value)
    _check(load().cd_geom_save(geom.handle, buf, size.value, ctypes.byref(size)))
    return buf.raw


def geometry_from_image(image: bytes, stream=None) -> Geometry:
    """cd_geom_load: rebuilds the geometry and checks its direction and table hashes."""
    h = ctypes.c_void_p()
    _check(load().cd_geom_load(image, len(image), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return Geometry(h.value)


def geometry_hash(geom: Geometry):
    """cd_geom_hash: (hash of the direction set and mode, hash of the tables)."""
    d, t = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().cd_geom_hash(geom.handle, ctypes.byref(d), ctypes.byref(t)))
    return d.value, t.value


def save_tree(tree: Tree, path: str, stream=None):
    with open(path, "wb") as f:
        f.write(tree_image(tree, stream))


def load_tree(path: str, stream=None) -> Tree:
    with open(path, "rb") as f:
        return tree_from_image(f.read(), stream)


def save_geometry(geom: Geometry, path: str):
    with open(path, "wb") as f:
        f.write(geometry_image(geom))


def load_geometry(path: str, stream=None) -> Geometry:
    with open(path, "rb") as f:
        return geometry_from_image(f.read(), stream)


def fnv1a64(data: bytes) -> int:
    """cd_fnv1a64 (the checksum that ends every checkpoint image)."""
    return load().cd_fnv1a64(data, len(data))


def precompute_geometry(scheme="healpix", p0: int = 1, p1: int = 0, dirs=None, mode: int = MODE_PREC,
                        stream=None) -> Geometry:
    """cd_precompute_geometry.  scheme: 'healpix' (p0 = Nside), 'mxn' (p0 = M,
    p1 = N), 'axes', 'custom' (dirs: [n, 3]); mode: MODE_PREC, MODE_INSITU or
    MODE_CONE (weights averaged over each direction's cone)."""
    code = {"healpix": DIRS_HEALPIX, "mxn": DIRS_MXN, "axes": DIRS_AXES, "custom": DIRS_CUSTOM}[scheme] \
        if isinstance(scheme, str) else int(scheme)
    arr, n = None, 0
    if code == DIRS_CUSTOM:
        arr = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        n = arr.shape[0]
    h = ctypes.c_void_p()
    _check(load().cd_precompute_geometry(code, int(p0), int(p1),
                                         arr.ctypes.data_as(ctypes.c_void_p) if arr is not None else None, n,
                                         int(mode), ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
    return Geometry(h.value)


def column_density(tree: Tree, geom: Geometry, n_h=None, a_v=None, shield=None, precision: int = FP32,
                   av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5, net=None, stream=None):
    """cd_column_density into caller-owned CUDA float32 tensors (any may be
    None).  net: a Net for the learned form."""
    o = opts_default()
    o.net = net.handle.value if net is not None else None
    o.precision = int(precision)
    o.av_per_nh = float(av_per_nh)
    o.shield_k = float(shield_k)
    ptrs = _outputs(tree, geom, n_h, a_v, shield)
    _check(load().cd_column_density(tree.handle, geom.handle, ctypes.byref(o), *ptrs,
                                    ctypes.c_void_p(_stream_ptr(stream))))
    return n_h, a_v, shield


def _hptr(x, numel, name):
    """Host pointer of a contiguous float32 CPU tensor or numpy array (or None)."""
    if x is None:
        return None
    import torch
    if isinstance(x, torch.Tensor):
        if x.is_cuda or x.dtype != torch.float32 or not x.is_contiguous():
            raise ValueError("%s must be a contiguous float32 CPU tensor" % name)
        n, ptr = x.numel(), x.data_ptr()
    else:
        if not isinstance(x, np.ndarray) or x.dtype != np.float32 or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("%s must be a C-contiguous float32 numpy array" % name)
        n, ptr = x.size, x.ctypes.data
    if n < numel:
        raise ValueError("%s holds %d floats, %d needed" % (name, n, numel))
    return ptr


def column_density_host(tree: Tree, geom: Geometry, rho=None, n_h=None, a_v=None, shield=None,
                        precision: int = FP32, av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5,
                        stream=None):
    """cd_column_density_host: densities from and results to HOST memory (CPU
    tensors, pinned for asynchronous copies, or numpy arrays).  rho (or
    None): as for tree_update; n_h / a_v: n_leaf * n_dir floats, shield:
    n_leaf.  The host buffers are complete once `stream` is synchronised."""
    o = opts_default()
    o.precision, o.av_per_nh, o.shield_k = int(precision), float(av_per_nh), float(shield_k)
    nd = tree.n_leaf * geom.n_dir
    ptrs = [_hptr(rho, tree.n_leaf, "rho"), _hptr(n_h, nd, "n_h"), _hptr(a_v, nd, "a_v"),
            _hptr(shield, tree.n_leaf, "shield")]
    _check(load().cd_column_density_host(tree.handle, geom.handle, ctypes.byref(o),
                                         *[ctypes.c_void_p(p) for p in ptrs], ctypes.c_void_p(_stream_ptr(stream))))
    return n_h, a_v, shield


def _outputs(tree: Tree, geom: Geometry, n_h, a_v, shield, box=None):
    """Checked device pointers of one box's outputs: n_h and a_v need
    n_leaf * n_dir floats, shield n_leaf, all on the tree's device."""
    tag = "" if box is None else " of box %d" % box
    nd = tree.n_leaf * geom.n_dir
    return (_dptr(n_h, nd, tree.device, "n_h" + tag), _dptr(a_v, nd, tree.device, "a_v" + tag),
            _dptr(shield, tree.n_leaf, tree.device, "shield" + tag))


def heating(tree: Tree, chi, T=None, n_e=None, G0: float = 1.7, g0_eff=None, gamma_uv=None, gamma_cr=None,
            stream=None):
    """cd_heating: G0_eff = chi G0, the photoelectric rate (needs T and n_e)
    and the cosmic-ray rate per leaf, into caller-owned CUDA float32 tensors
    (any may be None)."""
    n, dev = tree.n_leaf, tree.device
    ins = [_dptr(v, n, dev, k) for k, v in (("chi", chi), ("T", T), ("n_e", n_e))]
    outs = [_dptr(v, n, dev, k) for k, v in (("g0_eff", g0_eff), ("gamma_uv", gamma_uv), ("gamma_cr", gamma_cr))]
    _check(load().cd_heating(tree.handle, *ins, float(G0), *outs, ctypes.c_void_p(_stream_ptr(stream))))
    return g0_eff, gamma_uv, gamma_cr


def column_density_noalloc(tree: Tree, geom: Geometry, n_h=None, a_v=None, shield=None,
                           av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5, stream=None):
    """cd_column_density_noalloc: FP32 evaluation whose scratch is a fixed
    16 MiB device array inside the library, for callers that must not
    allocate device memory once their time-step loop runs (small trees only,
    see include/colden.h)."""
    o = opts_default()
    o.precision = FP32
    o.av_per_nh = float(av_per_nh)
    o.shield_k = float(shield_k)
    ptrs = _outputs(tree, geom, n_h, a_v, shield)
    _check(load().cd_column_density_noalloc(tree.handle, geom.handle, ctypes.byref(o), *ptrs,
                                            ctypes.c_void_p(_stream_ptr(stream))))
    return n_h, a_v, shield


def _ptr_array(items, get):
    arr = (ctypes.c_void_p * len(items))()
    for i, x in enumerate(items):
        arr[i] = get(x)
    return arr


def _batch_outputs(trees, geoms, n_h, a_v, shield):
    """Per-box checked pointer arrays (ctypes) for the batch entry points, or
    None where the caller gives no list."""
    n = len(trees)
    if len(geoms) != n:
        raise ValueError("%d trees but %d geometries" % (n, len(geoms)))
    for name, ts in (("n_h", n_h), ("a_v", a_v), ("shield", shield)):
        if ts is not None and len(ts) != n:
            raise ValueError("%s lists %d buffers for %d boxes" % (name, len(ts), n))
    cols = [[None] * n, [None] * n, [None] * n]
    for i in range(n):
        pick = lambda ts: ts[i] if ts is not None else None
        for j, p in enumerate(_outputs(trees[i], geoms[i], pick(n_h), pick(a_v), pick(shield), box=i)):
            cols[j][i] = p
    return tuple(None if ts is None else _ptr_array(c, lambda p: p) for ts, c in zip((n_h, a_v, shield), cols))


def column_density_batch(trees, geoms, n_h=None, a_v=None, shield=None, precision: int = FP32,
                         av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5, stream=None):
    """cd_column_density_batch: the boxes one after another (per-box launches)."""
    n = len(trees)
    o = opts_default()
    o.precision, o.av_per_nh, o.shield_k = int(precision), float(av_per_nh), float(shield_k)
    outs = _batch_outputs(trees, geoms, n_h, a_v, shield)
    _check(load().cd_column_density_batch(n, _ptr_array(trees, lambda t: t.handle.value),
                                          _ptr_array(geoms, lambda g: g.handle.value), ctypes.byref(o),
                                          *outs, ctypes.c_void_p(_stream_ptr(stream))))


class EvalGraph:
    """cd_eval_graph: one step (the update from the device buffer rho, if
    given, then the evaluation into n_h / a_v / shield) captured once as a
    CUDA graph; launch() replays it (see include/colden.h)."""

    def __init__(self, tree: Tree, geom: Geometry, rho=None, n_h=None, a_v=None, shield=None,
                 precision: int = FP32, av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5, net=None,
                 stream=None):
        self._keep = (tree, geom, rho, n_h, a_v, shield, net)
        o = opts_default()
        o.net = net.handle.value if net is not None else None
        o.precision, o.av_per_nh, o.shield_k = int(precision), float(av_per_nh), float(shield_k)
        outs = _outputs(tree, geom, n_h, a_v, shield)
        r = _dptr(rho, tree.n_leaf, tree.device, "rho")
        h = ctypes.c_void_p()
        _check(load().cd_eval_graph_create(tree.handle, geom.handle, ctypes.byref(o), r, *outs,
                                           ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(load().cd_eval_graph_launch(self._h, ctypes.c_void_p(_stream_ptr(stream))))

    def kernels(self) -> int:
        n = ctypes.c_int64()
        _check(load().cd_eval_graph_info(self._h, ctypes.byref(n)))
        return n.value

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cd_eval_graph_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Batch:
    """cd_batch: the boxes captured once into one CUDA graph (see include/colden.h)."""

    def __init__(self, trees, geoms, n_h=None, a_v=None, shield=None, precision: int = FP32,
                 av_per_nh: float = 1.0 / 1.87e21, shield_k: float = 2.5, stream=None):
        self._keep = (list(trees), list(geoms), n_h, a_v, shield)
        n = len(trees)
        o = opts_default()
        o.precision, o.av_per_nh, o.shield_k = int(precision), float(av_per_nh), float(shield_k)
        outs = _batch_outputs(trees, geoms, n_h, a_v, shield)
        h = ctypes.c_void_p()
        _check(load().cd_batch_create(n, _ptr_array(trees, lambda t: t.handle.value),
                                      _ptr_array(geoms, lambda g: g.handle.value), ctypes.byref(o),
                                      *outs, ctypes.c_void_p(_stream_ptr(stream)), ctypes.byref(h)))
        self._h = h

    def run(self, stream=None):
        _check(load().cd_batch_run(self._h, ctypes.c_void_p(_stream_ptr(stream))))

    def info(self):
        w, nodes = ctypes.c_int(), ctypes.c_int64()
        ms = (ctypes.c_double * 4)()
        _check(load().cd_batch_info(self._h, ctypes.byref(w), ms, ctypes.byref(nodes)))
        per, full, ctas = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        pms = (ctypes.c_double * 4)()
        _check(load().cd_batch_plan(self._h, ctypes.byref(per), ctypes.byref(full), ctypes.byref(ctas), pms))
        shapes = (("half", 1), ("half", 2), ("full", 1), ("full", 2))
        return {"width": w.value, "ms_tried": {W: ms[i] for i, W in enumerate((1, 2, 4, 8)) if ms[i] >= 0},
                "kernel_nodes": nodes.value, "persistent": bool(per.value),
                "full_tiles": bool(full.value), "ctas_per_sm": ctas.value,
                "plan_ms": {"%s/%d" % sh: pms[i] for i, sh in enumerate(shapes) if pms[i] >= 0}}

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cd_batch_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Learned correction (include/colden_learned.h)
# ---------------------------------------------------------------------------

SLOTS = 8


def _iptr(t, numel=None, device=None, name="index buffer"):
    """Device pointer of a contiguous int64 CUDA tensor (or None); raises
    ValueError as _dptr does."""
    return _checked_ptr(t, "int64", numel, device, name)


def net_num_params(n_dir: int, hidden: int) -> int:
    return int(load().cd_net_num_params(int(n_dir), int(hidden)))


def adam_default() -> Adam:
    a = Adam()
    load().cd_adam_default(ctypes.byref(a))
    return a


def raymarch(tree: Tree, geom: Geometry, n_ray, leaves=None, stream=None):
    """cd_raymarch: exact columns [n, n_dir] from the centres of `leaves`
    (int64 CUDA tensor, or None for the first n_ray.shape[0] leaves)."""
    n = n_ray.shape[0]
    _check(load().cd_raymarch(tree.handle, geom.handle, n, _iptr(leaves, n, tree.device, "leaves"),
                              _dptr(n_ray, n * geom.n_dir, tree.device, "n_ray"),
                              ctypes.c_void_p(_stream_ptr(stream))))
    return n_ray


def learned_features(tree: Tree, geom: Geometry, x, n_tree=None, leaves=None, stream=None):
    """cd_learned_features: network inputs x [n, 8 n_dir + 1] and (optionally)
    the plain column n_tree [n, n_dir] of `leaves` (None: the first n)."""
    n = x.shape[0]
    dev = tree.device
    _check(load().cd_learned_features(tree.handle, geom.handle, n, _iptr(leaves, n, dev, "leaves"),
                                      _dptr(x, n * (SLOTS * geom.n_dir + 1), dev, "x"),
                                      _dptr(n_tree, n * geom.n_dir, dev, "n_tree"),
                                      ctypes.c_void_p(_stream_ptr(stream))))
    return x, n_tree


def learned_targets(n_ray, n_tree, y, stream=None):
    """cd_learned_targets: y = ln(n_ray / n_tree)."""
    n = n_ray.numel()
    _check(load().cd_learned_targets(n, _dptr(n_ray, n, None, "n_ray"), _dptr(n_tree, n, None, "n_tree"),
                                     _dptr(y, n, None, "y"), ctypes.c_void_p(_stream_ptr(stream))))
    return y


class Net:
    """cd_net: the learned correction's network (weights on the device)."""

    def __init__(self, n_dir: int, hidden: int, params):
        p = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if p.size != net_num_params(n_dir, hidden):
            raise ValueError("expected %d parameters, got %d" % (net_num_params(n_dir, hidden), p.size))
        h = ctypes.c_void_p()
        _check(load().cd_net_create(int(n_dir), int(hidden), p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(h)))
        self._h = h
        self.n_dir, self.hidden = int(n_dir), int(hidden)
        self.n_params = p.size
        self.n_in = SLOTS * self.n_dir + 1

    @property
    def handle(self):
        return self._h

    def fit_normaliser(self, x, stream=None):
        _check(load().cd_net_fit_normaliser(self._h, x.shape[0], _dptr(x), ctypes.c_void_p(_stream_ptr(stream))))

    def forward(self, x, delta, stream=None):
        _check(load().cd_net_forward(self._h, x.shape[0], _dptr(x), _dptr(delta),
                                     ctypes.c_void_p(_stream_ptr(stream))))
        return delta

    def loss_grad(self, x, y, loss, grad=None, rows=None, batch=None, stream=None):
        B = int(batch if batch is not None else (rows.numel() if rows is not None else x.shape[0]))
        _check(load().cd_net_loss_grad(self._h, B, _dptr(x), _dptr(y), _iptr(rows), _dptr(loss), _dptr(grad),
                                       ctypes.c_void_p(_stream_ptr(stream))))

    def train_step(self, x, y, rows=None, batch=None, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=None,
                   stream=None):
        B = int(batch if batch is not None else (rows.numel() if rows is not None else x.shape[0]))
        hp = Adam(float(lr), float(beta1), float(beta2), float(eps))
        _check(load().cd_net_train_step(self._h, B, _dptr(x), _dptr(y), _iptr(rows), ctypes.byref(hp),
                                        _dptr(loss), ctypes.c_void_p(_stream_ptr(stream))))

    def set_delta_range(self, lo: float, hi: float):
        """Trusted range of delta: outside [lo, hi] the plain column is kept."""
        _check(load().cd_net_set_delta_range(self._h, float(lo), float(hi)))

    def delta_range(self):
        lo, hi = ctypes.c_double(), ctypes.c_double()
        _check(load().cd_net_get_delta_range(self._h, ctypes.byref(lo), ctypes.byref(hi)))
        return lo.value, hi.value

    def fit_delta_range(self, y, margin: float, stream=None):
        """Trusted range = the finite targets' range widened by margin."""
        _check(load().cd_net_fit_delta_range(self._h, y.numel(), _dptr(y), float(margin),
                                             ctypes.c_void_p(_stream_ptr(stream))))
        return self.delta_range()

    def state(self) -> dict:
        """Checkpoint of the whole state (host numpy arrays), with the
        trusted delta range."""
        P, I = self.n_params, self.n_in
        out = {k: np.zeros(n, dtype=np.float32) for k, n in
               (("params", P), ("mu", I), ("sinv", I), ("adam_m", P), ("adam_v", P))}
        step = ctypes.c_int64()
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().cd_net_get_state(self._h, c(out["params"]), c(out["mu"]), c(out["sinv"]), c(out["adam_m"]),
                                       c(out["adam_v"]), ctypes.byref(step)))
        out["step"] = step.value
        out["delta_range"] = np.array(self.delta_range())
        return out

    def load_state(self, st: dict):
        arr = {k: np.ascontiguousarray(st[k], dtype=np.float32) for k in ("params", "mu", "sinv", "adam_m", "adam_v")}
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(load().cd_net_set_state(self._h, c(arr["params"]), c(arr["mu"]), c(arr["sinv"]), c(arr["adam_m"]),
                                       c(arr["adam_v"]), int(st.get("step", 0))))
        if "delta_range" in st:
            self.set_delta_range(*[float(v) for v in np.asarray(st["delta_range"]).reshape(2)])

    def save(self, path: str):
        np.savez(path, n_dir=self.n_dir, hidden=self.hidden, **self.state())

    @classmethod
    def load(cls, path: str) -> "Net":
        z = np.load(path)
        net = cls(int(z["n_dir"]), int(z["hidden"]), z["params"])
        net.load_state({k: z[k] for k in z.files})
        return net

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load().cd_net_free(self._h)
        self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def train(net: Net, x, y, steps: int, batch: int = 4096, lr: float = 1e-3, seed: int = 0, lr_final: float = None,
          val=None, eval_every: int = 250, row_weights=None, stream=None):
    """Adam training loop over the rows of (x, y) (CUDA tensors): a seeded
    permutation per epoch, minibatches of `batch` rows, optional cosine decay
    of the step size to lr_final.  With val = (x_val, y_val), the loss on
    those rows (cd_net_loss_grad, no update) is taken every `eval_every`
    steps and at the end, and the network is left in the state of the lowest
    one (the training stop chosen on held-out rows, e.g. of a field at the
    resolution the network will serve); val may instead be a function of
    the network returning the score to minimise (e.g. the mean |A_V| error
    on held-out leaves).  net.val_history then lists (step, score).
    With row_weights (one non-negative weight per row), each epoch draws its
    rows with replacement with probabilities proportional to the weights
    instead of a permutation, which weights the loss by them in expectation
    (e.g. by the squared column, so that the fit follows the absolute A_V
    error rather than the log error alone).  Returns the per-step training loss (host array).
    Orchestration only: every step is cd_net_train_step."""
    import math
    import torch
    n = x.shape[0]
    g = torch.Generator(device="cpu")
    g.manual_seed(seed)
    loss = torch.zeros(steps, device=x.device, dtype=torch.float32)
    vbuf = torch.zeros(1, device=x.device, dtype=torch.float32)
    best, best_state, hist = None, None, []

    def check(step):
        nonlocal best, best_state
        if callable(val):
            v = float(val(net))
        else:
            net.loss_grad(val[0], val[1], vbuf, stream=stream)
            v = float(vbuf.item())
        hist.append((step, v))
        if best is None or v < best:
            best, best_state = v, net.state()

    cdf = None if row_weights is None else torch.cumsum(row_weights.detach().double().cpu(), 0)

    def epoch():
        if cdf is None:
            return torch.randperm(n, generator=g)
        # n draws with replacement by inverse transform of the weights' cumulative sum
        u = torch.rand(n, generator=g, dtype=torch.float64) * cdf[-1]
        return torch.searchsorted(cdf, u, right=True).clamp_(max=n - 1)

    perm = None
    pos = n
    for it in range(steps):
        if val is not None and it > 0 and it % eval_every == 0:
            check(it)
        if pos + batch > n:
            perm = epoch().to(device=x.device, dtype=torch.int64)
            pos = 0
        rows = perm[pos:pos + min(batch, n)]
        pos += batch
        cur = lr if lr_final is None else lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * it / steps))
        net.train_step(x, y, rows=rows, lr=cur, loss=loss[it:it + 1], stream=stream)
    if val is not None:
        check(steps)
        if best_state is not None and hist[-1][1] > best:
            net.load_state(best_state)
        net.val_history = hist
    return loss.cpu().numpy()
