"""FP64 oracle of the learned correction to the tree method (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The product library shares no code with it.

The paper stops at the tree method and its comparison with exact ray tracing
(§4, §6: errors of order ten per cent).  The learned form adds a small network
that reads, for one leaf, the method's own intermediate terms -- the
contribution of every tree level along every direction -- and predicts a
per-direction log correction toward the exactly ray-traced column:

    c[s, d]   contribution of the shells Delta_l = s levels above the leaf
              (s = 0: the leaf's own oct, internal + local term of §3.2;
              s = 1..6: the shell Delta_l = s of Eq. N_discret; s = 7: the sum
              of every coarser shell)
    x         [ln max(c[s, d], C_FLOOR) for s in 0..7, d in 0..n_dir-1 (s-major),
               ln max(n_t, N_FLOOR)]
    u         clip((x - mu) * sinv, -8, 8)          (fixed input standardisation)
    z1 = W1 u + b1,  a1 = gelu(z1)
    z2 = W2 a1 + b2, a2 = gelu(z2)
    delta = W3 a2 + b3                              (one value per direction)
    N_learned[d] = N_tree[d] * exp(delta[d]),  N_tree[d] = sum_s c[s, d]
                   (N_tree itself where delta[d] is not finite, or lies
                   outside the trusted range [lo, hi]: by default the whole
                   line; after training, the range of the targets the
                   network was fitted to, widened by a margin, so that a
                   finite but untrained correction falls back to the plain
                   method)

Training minimises the mean squared error of delta against
y = ln(N_ray / N_tree) with Adam (Kingma & Ba 2015, Algorithm 1).  GELU is the
tanh form of Hendrycks & Gimpel (2016).  Every function is a direct, unblocked
statement of these definitions; the matrix products are numpy's.

Parameter packing (the order the library also uses): W1 [H, n_in] row-major,
b1 [H], W2 [H, H], b2 [H], W3 [n_dir, H], b3 [n_dir].
"""
from __future__ import annotations

import math

import numpy as np

SLOTS = 8
C_FLOOR = 1e16      # cm^-2: floor under a level's contribution before the log
N_FLOOR = 1e-10     # cm^-3: floor under the leaf density before the log
GELU_C = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def n_inputs(n_dir: int) -> int:
    return SLOTS * n_dir + 1


def shapes(n_dir: int, hidden: int):
    n_in = n_inputs(n_dir)
    return [("W1", (hidden, n_in)), ("b1", (hidden,)), ("W2", (hidden, hidden)), ("b2", (hidden,)),
            ("W3", (n_dir, hidden)), ("b3", (n_dir,))]


def n_params(n_dir: int, hidden: int) -> int:
    return sum(int(np.prod(s)) for _, s in shapes(n_dir, hidden))


def unpack(p: np.ndarray, n_dir: int, hidden: int) -> dict:
    out, o = {}, 0
    for name, s in shapes(n_dir, hidden):
        k = int(np.prod(s))
        out[name] = np.asarray(p[o:o + k], dtype=np.float64).reshape(s)
        o += k
    return out


def pack(d: dict) -> np.ndarray:
    return np.concatenate([np.asarray(d[k], dtype=np.float64).ravel() for k in ("W1", "b1", "W2", "b2", "W3", "b3")])


# ---------------------------------------------------------------------------
# Features from the tree method's per-level terms
# ---------------------------------------------------------------------------

def slots_from_levels(per_level: np.ndarray) -> np.ndarray:
    """per_level [n, S_in, n_dir] indexed by Delta_l (0 = own oct) -> the eight
    slots [n, 8, n_dir]: Delta_l = 0..6 kept apart, every coarser level summed
    into slot 7 (zero when the tree has no such level)."""
    n, s_in, nd = per_level.shape
    out = np.zeros((n, SLOTS, nd))
    k = min(s_in, SLOTS - 1)
    out[:, :k] = per_level[:, :k]
    if s_in > SLOTS - 1:
        out[:, SLOTS - 1] = per_level[:, SLOTS - 1:].sum(axis=1)
    return out


def features(slots: np.ndarray, n_leaf: np.ndarray) -> np.ndarray:
    """slots [n, 8, n_dir], leaf densities [n] -> x [n, 8 n_dir + 1]."""
    n = slots.shape[0]
    x = np.empty((n, slots.shape[1] * slots.shape[2] + 1))
    x[:, :-1] = np.log(np.maximum(slots, C_FLOOR)).reshape(n, -1)
    x[:, -1] = np.log(np.maximum(np.asarray(n_leaf, dtype=np.float64), N_FLOOR))
    return x


def tree_total(slots: np.ndarray) -> np.ndarray:
    """N_tree [n, n_dir]: the plain method's column, the sum over slots."""
    return slots.sum(axis=1)


def targets(n_ray: np.ndarray, n_tree: np.ndarray) -> np.ndarray:
    """y = ln(N_ray / N_tree): the log correction the network learns."""
    return np.log(n_ray / n_tree)


SD_MIN = 1e-3       # columns with less spread than this (ln units) are ignored
U_MAX = 8.0         # standardised inputs are clipped to [-U_MAX, U_MAX]


def normaliser(x: np.ndarray):
    """Column mean and inverse standard deviation of a training set.  A column
    whose standard deviation is at most SD_MIN carried no information in
    training (an empty slot is ln of the floor in every row): it gets
    sinv = 0, so the network ignores it instead of extrapolating when a
    deeper tree fills that slot."""
    mu = x.mean(axis=0)
    sd = np.sqrt(((x - mu) ** 2).mean(axis=0))
    sinv = np.where(sd > SD_MIN, 1.0 / np.where(sd > SD_MIN, sd, 1.0), 0.0)
    return mu, sinv


def standardise(x, mu, sinv):
    """u = (x - mu) sinv, clipped to [-U_MAX, U_MAX]."""
    return np.clip((x - mu) * sinv, -U_MAX, U_MAX)


# ---------------------------------------------------------------------------
# The network
# ---------------------------------------------------------------------------

def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(GELU_C * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_C * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_C * (1.0 + 3.0 * GELU_A * z * z)


def forward(p: dict, mu, sinv, x: np.ndarray):
    """delta [n, n_dir] and the intermediates the backward pass needs."""
    u = standardise(x, mu, sinv)
    z1 = u @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    delta = a2 @ p["W3"].T + p["b3"]
    return delta, (u, z1, a1, z2, a2)


def loss(p: dict, mu, sinv, x, y) -> float:
    delta, _ = forward(p, mu, sinv, x)
    return float(np.mean((delta - y) ** 2))


def loss_grad(p: dict, mu, sinv, x, y):
    """Mean squared error over every (leaf, direction) and its gradient with
    respect to every parameter (reverse-mode chain rule, layer by layer)."""
    delta, (u, z1, a1, z2, a2) = forward(p, mu, sinv, x)
    r = delta - y
    L = float(np.mean(r * r))
    g_delta = 2.0 * r / r.size
    g = {"W3": g_delta.T @ a2, "b3": g_delta.sum(axis=0)}
    g_z2 = (g_delta @ p["W3"]) * gelu_grad(z2)
    g["W2"] = g_z2.T @ a1
    g["b2"] = g_z2.sum(axis=0)
    g_z1 = (g_z2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = g_z1.T @ u
    g["b1"] = g_z1.sum(axis=0)
    return L, g


def adam(p: np.ndarray, g: np.ndarray, m: np.ndarray, v: np.ndarray, t: int, lr: float,
         beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma & Ba 2015, Algorithm 1) of the packed parameters.
    t is the 1-based step number.  Returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mhat = m / (1.0 - beta1 ** t)
    vhat = v / (1.0 - beta2 ** t)
    return p - lr * mhat / (np.sqrt(vhat) + eps), m, v


def apply(n_tree: np.ndarray, delta: np.ndarray, lo: float = -math.inf, hi: float = math.inf) -> np.ndarray:
    """N_learned = N_tree exp(delta); the plain method where delta is not
    finite or lies outside the closed range [lo, hi] (lo > hi: everywhere)."""
    with np.errstate(over="ignore", invalid="ignore"):
        out = n_tree * np.exp(delta)
        keep = np.isfinite(delta) & (delta >= lo) & (delta <= hi)
    return np.where(keep, out, n_tree)


def delta_range(y: np.ndarray, margin: float):
    """The trusted range of a network trained on targets y: [min y - margin,
    max y + margin] over the finite entries ((+inf, -inf), an empty range,
    when there are none)."""
    f = np.asarray(y, dtype=np.float64).reshape(-1)
    f = f[np.isfinite(f)]
    if f.size == 0:
        return math.inf, -math.inf
    return float(f.min()) - margin, float(f.max()) + margin

