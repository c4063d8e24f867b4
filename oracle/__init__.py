"""FP64 CPU oracle of the tree-based column-density method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does: it has
no CPU fallback and shares no code with this oracle.

The arithmetic lives in ``oracle.c`` (plain C, FP64, OpenMP over targets); this
module compiles it with gcc on first use and wraps it with numpy-friendly
functions.  Every function cites the passage of Valdivia & Hennebelle it
follows (section / equation numbers of the paper).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

MODE_PREC = 0     # two-level approximation of the precalculation module (§3.3)
MODE_INSITU = 1   # every contribution from the oct centre, no approximation (§4.3)

# Extinction constants of the hot path: A_V = N_H / 1.87e21 cm^-2 and the
# screening factor <exp(-2.5 A_V)>; the paper's own attenuation uses
# sigma = 2e-21 cm^2 in chi = <exp(-sigma N)> (Eqs. eq_chi, eq_tau, chi_discret).
AV_PER_NH = 1.0 / 1.87e21
SHIELD_K = 2.5
SIGMA_PAPER = 2e-21


def build(force: bool = False) -> str:
    """Compile oracle.c into _build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fopenmp", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            L.or_dirs_mxn.argtypes = [ctypes.c_int, ctypes.c_int, P]
            L.or_dirs_healpix.argtypes = [ctypes.c_int, P]
            L.or_dirs_axes.argtypes = [P]
            L.or_dirs_custom.argtypes = [ctypes.c_int, P, P]
            L.or_ray_cube.argtypes = [P, P, P, ctypes.c_double]
            L.or_ray_cube.restype = ctypes.c_double
            L.or_tree_uniform.argtypes = [ctypes.c_int, ctypes.c_double, P]
            L.or_tree_uniform.restype = P
            L.or_tree_amr.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, i64, P, P, P,
                                      ctypes.c_char_p, ctypes.c_int]
            L.or_tree_amr.restype = P
            L.or_tree_free.argtypes = [P]
            L.or_colden.argtypes = [P, ctypes.c_int, P, ctypes.c_int, i64, P, P, P, ctypes.c_int, P]
            L.or_raymarch.argtypes = [P, ctypes.c_int, P, i64, P, P, P]
            L.or_raysum_allcells.argtypes = [P, ctypes.c_int, P, P, P]
            L.or_pref.argtypes = [ctypes.c_double, ctypes.c_int, i64, i64, i64, ctypes.c_int,
                                  ctypes.c_int, P]
            L.or_rho_many.argtypes = [P, i64, P, P, P]
            _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# Directions (§3.2 eqs. theta and phi; §4.3 six rays; HEALPix, Gorski et al. 2005)
# ----------------------------------------------------------------------------

def dirs_mxn(M: int, N: int) -> np.ndarray:
    """theta_m = arccos(1 + (1-2m)/M), phi_n = 2 pi (n-1)/N; index (m-1)N + (n-1)."""
    out = np.zeros((M * N, 3))
    lib().or_dirs_mxn(M, N, _p(out))
    return out


def dirs_healpix(nside: int) -> np.ndarray:
    """HEALPix ring-scheme pixel centres, 12 nside^2 unit vectors."""
    out = np.zeros((12 * nside * nside, 3))
    lib().or_dirs_healpix(nside, _p(out))
    return out


def dirs_axes() -> np.ndarray:
    """The six-ray set +x, -x, +y, -y, +z, -z (§4.3)."""
    out = np.zeros((6, 3))
    lib().or_dirs_axes(_p(out))
    return out


def dirs_custom(d) -> np.ndarray:
    d = np.ascontiguousarray(d, dtype=np.float64).reshape(-1, 3)
    out = np.zeros_like(d)
    if lib().or_dirs_custom(d.shape[0], _p(d), _p(out)) < 0:
        raise ValueError("zero-length direction")
    return out


CONE_RINGS, CONE_AZIMUTHS = 4, 8


def cone_rays(dirs, n_bins: int = None, rings: int = CONE_RINGS, azimuths: int = CONE_AZIMUTHS,
              cos_alpha: float = None) -> np.ndarray:
    """Sub-rays of the cone of each direction, shape [nd, rings * azimuths, 3].

    A direction stands for a bin of solid angle 4 pi / n_bins (§3.2: the
    directions split the sphere into equal solid angles).  Its cone is the
    circular cap of that solid angle around u, cos(alpha) = 1 - 2 / n_bins
    (n_bins defaults to the number of directions).  The cap is cut into
    `rings` bands of equal solid angle (equal steps in cos theta) and every band
    into `azimuths` equal sectors; one sub-ray passes through the middle of
    each piece:
        cos theta_r = 1 - (r + 1/2) (1 - cos alpha) / rings
        phi_rj      = 2 pi (j + [r odd] / 2) / azimuths
        v = cos theta_r u + sin theta_r (cos phi_rj e1 + sin phi_rj e2)
    with e1 = unit(e_a x u), a the first axis whose |u_a| is within 1e-9 of
    the smallest (so that exact ties, e.g. |u_x| = |u_y| at 45 degrees, pick
    the same axis whatever the last bit of the vector), and e2 = u x e1.
    Sub-ray index r * azimuths + j.  Components below 1e-14 in magnitude are
    zeroed and the vector renormalised, as for the directions.  The pieces have equal solid angle, so the cone average of
    a quantity is the plain mean over the sub-rays (a midpoint rule for the
    integral over the cap)."""
    u = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
    nd = u.shape[0]
    if cos_alpha is None:
        cos_alpha = 1.0 - 2.0 / float(n_bins if n_bins is not None else nd)
    au = np.abs(u)
    axis = np.argmax(au <= au.min(axis=1, keepdims=True) + 1e-9, axis=1)
    e1 = np.cross(np.eye(3)[axis], u)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(u, e1)
    out = np.zeros((nd, rings * azimuths, 3))
    for r in range(rings):
        c = 1.0 - (r + 0.5) * (1.0 - cos_alpha) / rings
        sn = np.sqrt(max(0.0, 1.0 - c * c))
        for j in range(azimuths):
            phi = 2.0 * np.pi * (j + 0.5 * (r & 1)) / azimuths
            v = c * u + sn * (np.cos(phi) * e1 + np.sin(phi) * e2)
            v[np.abs(v) < 1e-14] = 0.0
            out[:, r * azimuths + j] = v / np.linalg.norm(v, axis=1, keepdims=True)
    return out


def ray_cube(p, d, lo, h) -> float:
    """Length of the ray {p + s d, s >= 0} inside the cube [lo, lo+h]^3."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    d = np.ascontiguousarray(d, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.float64)
    return lib().or_ray_cube(_p(p), _p(d), _p(lo), float(h))


def pref(box: float, l0: int, ijk, l: int, mode: int = MODE_PREC) -> np.ndarray:
    """Reference point of the shell at level l for target (l0, ijk) (§3.3)."""
    out = np.zeros(3)
    lib().or_pref(float(box), int(l0), int(ijk[0]), int(ijk[1]), int(ijk[2]), int(l), int(mode),
                  _p(out))
    return out


# ----------------------------------------------------------------------------
# Tree (§3 intro: octs, levels, dx_l = 0.5^l L; coarse density = volume mean)
# ----------------------------------------------------------------------------

class Tree:
    """An octree whose cell values are volume means of the leaf field."""

    def __init__(self, handle, box, base, lmax):
        self._h = handle
        self.box = float(box)
        self.base = base
        self.lmax = lmax

    @classmethod
    def uniform(cls, rho: np.ndarray, box: float) -> "Tree":
        """rho: [n, n, n] indexed [z, y, x] (x fastest), n = 2^L."""
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        n = rho.shape[0]
        L = int(round(np.log2(n)))
        assert rho.shape == (n, n, n) and (1 << L) == n
        h = lib().or_tree_uniform(L, float(box), _p(rho))
        if not h:
            raise ValueError("bad uniform tree")
        return cls(h, box, L, L)

    @classmethod
    def amr(cls, base: int, lmax: int, box: float, lvl, ijk, rho) -> "Tree":
        lvl = np.ascontiguousarray(lvl, dtype=np.int8)
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        rho = np.ascontiguousarray(rho, dtype=np.float32)
        err = ctypes.create_string_buffer(256)
        h = lib().or_tree_amr(int(base), int(lmax), float(box), lvl.shape[0], _p(lvl), _p(ijk),
                              _p(rho), err, 256)
        if not h:
            raise ValueError(err.value.decode())
        return cls(h, box, base, lmax)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_tree_free(self._h)
            self._h = None

    def rho(self, lvl, ijk) -> np.ndarray:
        lvl = np.ascontiguousarray(lvl, dtype=np.int32).reshape(-1)
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        out = np.zeros(lvl.shape[0])
        lib().or_rho_many(self._h, lvl.shape[0], _p(lvl), _p(ijk), _p(out))
        return out

    def column_density(self, dirs, lvl, ijk, mode: int = MODE_PREC, per_level: int = 0):
        """Tree-method N_H (cm^-2) for targets (lvl[t], ijk[t]); shape [n, ndir].

        Follows Eq. N_discret1 for the central region and Eq. N_discret for the
        shells (§3.2, §3.3).  With per_level = S > 0 it also returns the
        contribution of every shell, shape [n, S, ndir] (slot 0: internal +
        local; slot q: the shell at level l0 - q)."""
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        lvl = np.ascontiguousarray(lvl, dtype=np.int32).reshape(-1)
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        n, nd = lvl.shape[0], dirs.shape[0]
        out = np.zeros((n, nd))
        pl = np.zeros((n, per_level, nd)) if per_level else None
        rc = lib().or_colden(self._h, nd, _p(dirs), int(mode), n, _p(lvl), _p(ijk), _p(out),
                             int(per_level), _p(pl) if per_level else None)
        if rc != 0:
            raise ValueError("bad target level")
        return (out, pl) if per_level else out

    def column_density_cone(self, dirs, lvl, ijk, n_bins: int = None, rings: int = CONE_RINGS,
                            azimuths: int = CONE_AZIMUTHS, mode: int = MODE_PREC) -> np.ndarray:
        """Cone-averaged tree-method N_H, shape [n, ndir]: the mean of the
        single-ray column (Eqs. N_discret1 and N_discret) over the sub-rays of
        cone_rays.  The geometric factors K enter the column linearly, so this
        equals the column computed with K averaged over each cone."""
        rays = cone_rays(dirs, n_bins, rings, azimuths)
        nd, ns = rays.shape[0], rays.shape[1]
        N = self.column_density(rays.reshape(-1, 3), lvl, ijk, mode=mode)
        return N.reshape(N.shape[0], nd, ns).mean(axis=2)

    def raymarch(self, dirs, lvl, ijk) -> np.ndarray:
        """Exact column from each target centre to the box edge (§4 reference)."""
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        lvl = np.ascontiguousarray(lvl, dtype=np.int32).reshape(-1)
        ijk = np.ascontiguousarray(ijk, dtype=np.int32).reshape(-1, 3)
        out = np.zeros((lvl.shape[0], dirs.shape[0]))
        lib().or_raymarch(self._h, dirs.shape[0], _p(dirs), lvl.shape[0], _p(lvl), _p(ijk), _p(out))
        return out

    def raysum_allcells(self, dirs, x0) -> np.ndarray:
        dirs = np.ascontiguousarray(dirs, dtype=np.float64).reshape(-1, 3)
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        out = np.zeros(dirs.shape[0])
        lib().or_raysum_allcells(self._h, dirs.shape[0], _p(dirs), _p(x0), _p(out))
        return out


# ----------------------------------------------------------------------------
# Epilogue (Eqs. eq_chi, eq_tau, chi_discret)
# ----------------------------------------------------------------------------

def a_v(N: np.ndarray, av_per_nh: float = AV_PER_NH) -> np.ndarray:
    return np.asarray(N, dtype=np.float64) * av_per_nh


def shield(N: np.ndarray, av_per_nh: float = AV_PER_NH, k: float = SHIELD_K) -> np.ndarray:
    """Direction average of exp(-k A_V): equal solid angles, so a plain mean."""
    return np.mean(np.exp(-k * a_v(N, av_per_nh)), axis=-1)


def chi(N: np.ndarray, sigma: float = SIGMA_PAPER) -> np.ndarray:
    """The paper's attenuation factor chi = (1/MN) sum exp(-sigma N(m,n))."""
    return np.mean(np.exp(-sigma * np.asarray(N, dtype=np.float64)), axis=-1)


# ----------------------------------------------------------------------------
# Heating of the application (§5, Eqs. G0_eff, gamma_uv, gamma_cr)
# ----------------------------------------------------------------------------

G0_DRAINE = 1.7   # the background UV field of §5, in Habing units


def heating_efficiency(g0_eff, T, n_e):
    """Photoelectric efficiency of Wolfire et al. (1995) as §5 states it, with
    x = G0_eff sqrt(T) / n_e:
        eps = 4.9e-2 / (1 + (x / 1925)^0.73) + 3.7e-2 (T / 1e4)^0.7 / (1 + x / 5000)."""
    g0_eff, T, n_e = (np.asarray(a, dtype=np.float64) for a in (g0_eff, T, n_e))
    x = g0_eff * np.sqrt(T) / n_e
    return 4.9e-2 / (1.0 + (x / 1925.0) ** 0.73) + 3.7e-2 * (T / 1e4) ** 0.7 / (1.0 + x / 5000.0)


def heating(chi_, n, T, n_e, G0: float = G0_DRAINE):
    """Per-cell heating of §5: G0_eff = chi G0 (Eq. G0_eff), the photoelectric
    rate Gamma_UV = 1e-24 eps G0_eff n (Eq. gamma_uv) and the cosmic-ray rate
    Gamma_CR = 1e-27 n (Eq. gamma_cr), in erg cm^-3 s^-1.  Returns
    (G0_eff, Gamma_UV, Gamma_CR)."""
    chi_, n = np.asarray(chi_, dtype=np.float64), np.asarray(n, dtype=np.float64)
    g0 = chi_ * G0
    return g0, 1e-24 * heating_efficiency(g0, T, n_e) * g0 * n, 1e-27 * n


# ----------------------------------------------------------------------------
# Leaf order helpers (plain bit interleaving; octant bits x=1, y=2, z=4)
# ----------------------------------------------------------------------------

def morton_ijk(level: int) -> np.ndarray:
    """ijk of every cell of a uniform level in Morton depth-first order."""
    n = 1 << level
    m = np.arange(n ** 3, dtype=np.int64)
    ijk = np.zeros((n ** 3, 3), dtype=np.int32)
    for b in range(level):
        for a in range(3):
            ijk[:, a] |= (((m >> (3 * b + a)) & 1) << b).astype(np.int32)
    return ijk
