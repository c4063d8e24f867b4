/*
 * colden_learned.h -- the learned correction of libcolden, and the exact
 * ray-marcher that supplies its training targets.
 *
 * The paper's method stops at the tree sum of Eq. N_discret and measures its
 * error against exact ray tracing of the same field (§2 and §4: ray tracing
 * with 50 rays; §4 and §6: errors of order ten per cent).  The learned correction is an extension the
 * paper does not have: a small network reads, for one leaf t, the tree
 * method's own terms and predicts one log correction per direction.
 *
 *   c[s][d]  (cm^-2) contribution of the shells Delta_l = s levels above the
 *            leaf along direction d: s = 0 is the internal + local term of the
 *            leaf's own oct (§3.2), s = 1..6 the shell of level l0 - s
 *            (Eq. N_discret with the two-level approximation of §3.3), s = 7
 *            the sum of every coarser shell.
 *   x        x[s * n_dir + d] = ln max(c[s][d], 1e16 cm^-2) for s = 0..7,
 *            x[8 n_dir] = ln max(n_t, 1e-10 cm^-3)         (n_in = 8 n_dir + 1)
 *   u        clip((x - mu) * sinv, -8, 8)   (fixed per-input standardisation)
 *   delta    W3 gelu(W2 gelu(W1 u + b1) + b2) + b3       (n_dir values)
 *            gelu(z) = z/2 (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))
 *   N        N_tree[d] exp(delta[d]),  N_tree[d] = sum_s c[s][d] (the plain
 *            method's column); N_tree[d] itself where delta[d] is not finite
 *            or lies outside the network's trusted range [lo, hi]
 *            (cd_net_set_delta_range; the whole line by default).
 *
 * Training minimises the mean over rows and directions of
 * (delta - y)^2 with y = ln(N_ray / N_tree), N_ray from cd_raymarch, by Adam
 * (Kingma & Ba 2015) on FP32 master weights.
 *
 * Parameters are packed in this order (FP32): W1 [hidden][n_in] row-major,
 * b1 [hidden], W2 [hidden][hidden], b2 [hidden], W3 [n_dir][hidden],
 * b3 [n_dir].
 *
 * Conventions are those of colden.h (status codes, cd_last_error, stream
 * semantics, leaf order).  Row-major device arrays, float32 unless stated.
 * The library serves uniform trees (cd_build_tree_uniform) in these entry
 * points; an AMR tree returns CD_EUNSUPPORTED.
 */
#ifndef COLDEN_LEARNED_H
#define COLDEN_LEARNED_H

#include "colden.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cd_net_s *cd_net;

#define CD_NET_SLOTS 8

/* Adam hyper-parameters (Kingma & Ba 2015, Algorithm 1). */
typedef struct {
    double lr;       /* step size, default 1e-3 */
    double beta1;    /* default 0.9 */
    double beta2;    /* default 0.999 */
    double eps;      /* default 1e-8 */
} cd_adam;

/* Fills *a with the defaults above. */
void cd_adam_default(cd_adam *a);

/* Number of packed FP32 parameters of a network for n_dir directions and
 * `hidden` units per hidden layer: hidden (8 n_dir + 1) + hidden + hidden^2
 * + hidden + n_dir hidden + n_dir.  Returns -1 for sizes outside
 * 1 <= n_dir <= 768, 1 <= hidden <= 1024. */
int64_t cd_net_num_params(int n_dir, int hidden);

/* Exact column from the centre of each listed leaf to the box edge along every
 * direction of geom: the line integral of the leaf density field, cell by
 * cell (a 3-D DDA over the leaf grid; §2's ray-tracing reference, with the
 * same directions as the tree method).  FP32.
 *   leaves   device int64 [n]: leaf indices in the output order of the tree,
 *            or NULL for leaves 0 .. n-1
 *   n_ray    device [n][n_dir] (cm^-2), caller-owned
 * Errors: CD_EINVAL (NULL handle, n < 0, n > n_leaf with leaves == NULL),
 * CD_EUNSUPPORTED (AMR tree), CD_ECUDA.  Out-of-range entries of `leaves` are
 * not detected on the device: their rows are written as 0. */
cd_status cd_raymarch(cd_tree tree, cd_geom geom, int64_t n, const int64_t *leaves, float *n_ray, void *stream);

/* Network inputs of the listed leaves (definition at the top of this file),
 * from the tree method evaluated level by level in FP32 (every shell of
 * Eq. N_discret kept apart instead of summed).
 *   x        device [n][8 n_dir + 1]
 *   n_tree   device [n][n_dir] or NULL: N_tree = sum over the 8 slots (cm^-2)
 * The per-level sums are kept in the tree's workspace between calls that use
 * the same geometry; a cd_tree_update makes the next call recompute them.
 * Errors as cd_raymarch. */
cd_status cd_learned_features(cd_tree tree, cd_geom geom, int64_t n, const int64_t *leaves, float *x,
                              float *n_tree, void *stream);

/* Training targets y = ln(n_ray / n_tree), elementwise over n values. */
cd_status cd_learned_targets(int64_t n, const float *n_ray, const float *n_tree, float *y, void *stream);

/* Creates a network on the current device.
 *   params   host [cd_net_num_params(n_dir, hidden)] initial weights (copied)
 * The standardisation starts as mu = 0, sinv = 1 (see cd_net_fit_normaliser);
 * the Adam moments start at 0 and the step count at 0.
 * Errors: CD_EINVAL (sizes, NULL), CD_ENOMEM, CD_ECUDA. */
cd_status cd_net_create(int n_dir, int hidden, const float *params, cd_net *out);

/* Sets mu and sinv to the column mean and 1 / standard deviation of the n
 * rows of x (device [n][n_in]); a column whose standard deviation is at most
 * 1e-3 (an empty slot: ln of the floor in every row) gets sinv = 0, so the
 * network ignores that input.
 * Deterministic.  Errors: CD_EINVAL (n < 1), CD_ENOMEM, CD_ECUDA. */
cd_status cd_net_fit_normaliser(cd_net net, int64_t n, const float *x, void *stream);

/* delta for n input rows, FP32 on the CUDA cores.
 *   x        device [n][n_in];  delta  device [n][n_dir] */
cd_status cd_net_forward(cd_net net, int64_t n, const float *x, float *delta, void *stream);

/* Loss and gradient without an update.
 *   rows     device int64 [B]: rows of x and y that form the batch, or NULL
 *            for rows 0 .. B-1 (values must lie in the arrays; not checked)
 *   loss     device float [1]: mean over B x n_dir of (delta - y)^2
 *   grad     device [num_params] in packing order, or NULL
 * Reductions run in a fixed order: repeated calls give identical bits. */
cd_status cd_net_loss_grad(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows,
                           float *loss, float *grad, void *stream);

/* One Adam step on the batch (loss and gradient as cd_net_loss_grad, then the
 * update of the FP32 master weights).  hp NULL = defaults.  loss may be NULL. */
cd_status cd_net_train_step(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows,
                            const cd_adam *hp, float *loss, void *stream);

/* Checkpoint: copies the whole state to (get) or from (set) host buffers,
 * synchronously: params and the two Adam moments [num_params], mu and sinv
 * [n_in], and the Adam step count.  Any pointer may be NULL to skip it. */
cd_status cd_net_get_state(cd_net net, float *params, float *mu, float *sinv, float *adam_m, float *adam_v,
                           int64_t *step);
cd_status cd_net_set_state(cd_net net, const float *params, const float *mu, const float *sinv,
                           const float *adam_m, const float *adam_v, int64_t step);

/* The trusted range of the correction: where delta[d] lies outside the
 * closed range [lo, hi] (or is not finite) the learned form returns the plain
 * column N_tree[d], so that a finite correction the network was never trained
 * to make falls back to the tree method.  lo > hi makes the range empty (the
 * plain method everywhere).  A new network's range is [-inf, +inf].  The
 * bounds are kept in FP32; the BF16 form compares delta log2(e) with the
 * bounds times log2(e), so a delta within a rounding of an end point may be
 * decided either way.  Not part of cd_net_get_state / cd_net_set_state.
 * Errors: CD_EINVAL (NULL handle, a NaN end). */
cd_status cd_net_set_delta_range(cd_net net, double lo, double hi);
cd_status cd_net_get_delta_range(cd_net net, double *lo, double *hi);

/* Sets the trusted range to [min y - margin, max y + margin] over the finite
 * entries of the n training targets y (device [n], e.g. from
 * cd_learned_targets); an empty range when none is finite.  Synchronises the
 * stream.  Errors: CD_EINVAL (n < 1, NULL y, margin negative or not finite),
 * CD_ENOMEM, CD_ECUDA. */
cd_status cd_net_fit_delta_range(cd_net net, int64_t n, const float *y, double margin, void *stream);

/* The network's direction count, hidden width and parameter count (any
 * pointer may be NULL); CD_EINVAL for a NULL handle. */
cd_status cd_net_info(cd_net net, int *n_dir, int *hidden, int64_t *num_params);

/* Frees the network (synchronises the device first). */
void cd_net_free(cd_net net);

/* The learned form of cd_column_density: set cd_opts.net to a cd_net whose
 * n_dir equals the geometry's.  CD_FP32 runs features, the FP32 network and
 * the correction in chunks of leaves; CD_BF16 runs them in one fused kernel
 * on the tcgen05 tensor cores (BF16 weights and activations, FP32
 * accumulation) where the sizes allow (see colden.h, cd_column_density). */

#ifdef __cplusplus
}
#endif

#endif /* COLDEN_LEARNED_H */
