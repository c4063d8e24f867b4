/*
 * colden.h -- C ABI of libcolden.so, a GB300 (sm_103a) implementation of the
 * tree-based column-density method of Valdivia & Hennebelle, "A fast
 * tree-based method for estimating column densities in Adaptive Mesh
 * Refinement codes" (A&A, arXiv:1410.0624).
 *
 * For every leaf cell t of a fully threaded octree and every direction d of a
 * sphere partition the library computes
 *
 *   N_H[t,d] = sum_i n_i dx_i(d)                               (Eq. N_discret1)
 *            = internal + local (the target and its oct, §3.2)
 *            + sum_l dx_l sum_{i in C_l} n_i K(r_i - r_t, d, dl)   (Eq. N_discret)
 *
 * where C_l is the cubic shell of level l, K the precomputed geometric factor
 * of the precalculation module (§3.3), then A_V = N_H * av_per_nh and the
 * direction-averaged screening factor shield[t] = (1/N_dir) sum_d exp(-k A_V)
 * (Eqs. eq_chi and chi_discret with equal solid angles).
 *
 * Conventions shared by every entry point
 *   - Status codes, never aborts.  cd_last_error() returns a thread-local
 *     message describing the last failure of the calling thread.
 *   - Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous unless stated otherwise.  Device errors of
 *     kernels surface as CD_ECUDA from a later call on the same device.
 *   - The box is [0, box_cm]^3, non-periodic; density outside it is zero.
 *     Level l has cells of size dx_l = box_cm / 2^l (§3.2, "dx_l = 0.5^l L").
 *   - Octant code of a cell with integer index (i, j, k) at its level:
 *     (i & 1) + 2 (j & 1) + 4 (k & 1).  Leaves are numbered in Morton
 *     depth-first order (children visited in octant order); cd_tree_leaves()
 *     returns each leaf's level and index in that order.
 *   - Units: n in cm^-3, lengths in cm, N_H in cm^-2.
 *   - Handles (cd_tree, cd_geom) are owned by the library and freed with the
 *     matching *_free call, which synchronises the device first.
 *   - All entry points are callable from several host threads on different
 *     handles; one handle must not be used by two threads at once.
 */
#ifndef COLDEN_H
#define COLDEN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cd_tree_s *cd_tree;
typedef struct cd_geom_s *cd_geom;
typedef struct cd_batch_s *cd_batch;

typedef enum {
    CD_OK = 0,
    CD_EINVAL = -1,        /* bad argument: message in cd_last_error() */
    CD_ENOMEM = -2,        /* device allocation failed */
    CD_ECUDA = -3,         /* a CUDA runtime call failed */
    CD_ETIMEOUT = -4,      /* a bounded device-side wait gave up */
    CD_EUNSUPPORTED = -5   /* valid request the library does not provide */
} cd_status;

/* Direction sets (§3.2). */
enum {
    CD_DIRS_HEALPIX = 0,   /* HEALPix ring-scheme pixel centres (Gorski et al. 2005): p0 = Nside, 12 Nside^2 dirs */
    CD_DIRS_MXN = 1,       /* the paper's equal-area set: p0 = M, p1 = N; theta_m = arccos(1 + (1-2m)/M),
                              phi_n = 2 pi (n-1)/N, direction index (m-1) N + (n-1) */
    CD_DIRS_AXES = 2,      /* the six-ray set of §4.3: +x, -x, +y, -y, +z, -z */
    CD_DIRS_CUSTOM = 3     /* caller's list of n_custom vectors (normalised by the library) */
};

/* Reference point of the external rays (§3.3 vs §4.3). */
enum {
    CD_MODE_PREC = 0,      /* precalculation module, two-level approximation: the shell at level l is seen from
                              the centre of the target's ancestor at level min(l+2, l0-1) */
    CD_MODE_INSITU = 1,    /* every shell seen from the oct centre: an exact walk over each shell's cells per
                              (oct, direction) on the CUDA cores, FP32 whatever cd_opts.precision says; no far-shell
                              sharing, so it costs more (§4.3, Table 1) */
    CD_MODE_CONE = 2       /* as CD_MODE_PREC, but every geometric factor (shell tables, Kloc, BF16 operands) is
                              the mean over the 32 sub-rays of the direction's cone (below) instead of the value
                              of one ray; the evaluation costs the same, only wider rows of the FP32 tables */
};

/* Cone of a direction (CD_MODE_CONE).  Each of the n_dir directions stands
 * for a bin of 4 pi / n_dir steradians (§3.2: the directions split the sphere
 * into equal solid angles).  Its cone is the circular cap of that solid angle
 * around the direction u, cos(alpha) = 1 - 2 / n_dir, cut into 4 rings of equal
 * solid angle (equal steps in cos theta) and each ring into 8 equal sectors;
 * sub-ray (r, j), index 8 r + j, passes through the middle of its piece:
 *   cos theta_r = 1 - (r + 1/2) (1 - cos alpha) / 4,
 *   phi_rj      = 2 pi (j + 1/2 if r is odd) / 8,
 *   v = cos theta_r u + sin theta_r (cos phi_rj e1 + sin phi_rj e2),
 * with e1 = unit(e_a x u), a the first axis whose |u_a| is within 1e-9 of the
 * smallest, e2 = u x e1; components below 1e-14 are zeroed and v renormalised.
 * The pieces have equal solid angle, so the averaged factor is the midpoint
 * rule for the mean of K over the cap.  The column is linear in K, so N_H is
 * the mean over the sub-rays of the single-ray column.  The in-situ walk and
 * the learned correction are defined for single rays only (CD_EUNSUPPORTED). */
#define CD_CONE_SUBRAYS 32

/* Arithmetic of the shell contraction. */
enum {
    CD_FP32 = 0,           /* FP32 CUDA-core contraction against FP32 sparse weights (<= 1e-5 rel. vs FP64) */
    CD_BF16 = 1            /* BF16 densities x BF16 weights on the tcgen05 tensor cores, FP32 accumulate */
};

typedef struct {
    int precision;         /* CD_FP32 or CD_BF16 */
    int reserved0;
    double av_per_nh;      /* A_V = N_H * av_per_nh; default 1 / 1.87e21 cm^2 */
    double shield_k;       /* shield = <exp(-shield_k A_V)>; default 2.5 */
    const void *net;       /* NULL, or a cd_net (colden_learned.h): the learned correction */
} cd_opts;

/* Fills *o with the defaults above. */
void cd_opts_default(cd_opts *o);

/* Builds the octree of a uniform grid of 2^leaf_level leaves per axis
 * (§3 intro: octs of 2^3 cells, levels 0..leaf_level) and every coarse level
 * by the volume mean of its eight children (the coarse density "corresponds
 * to a mean", §3.2).
 *   leaf_level     1 .. 10
 *   box_cm         box edge in cm, > 0
 *   rho            (2^L)^3 floats, index (k * 2^L + j) * 2^L + i (x fastest),
 *                  finite and >= 0; a device pointer if rho_on_device != 0,
 *                  else host memory (copied before return)
 *   *out           receives the new tree
 * Errors: CD_EINVAL for bad sizes or a NULL pointer; CD_ENOMEM; CD_ECUDA.
 * A negative or non-finite density is not detected on the device path. */
cd_status cd_build_tree_uniform(int leaf_level, double box_cm, const float *rho, int rho_on_device,
                                void *stream, cd_tree *out);

/* Builds an adaptive (AMR) octree from its leaves (§3 intro: refinement cell
 * by cell; fully threaded tree).  Leaf i has level level[i] in
 * [base_level, max_level], integer index (ijk[3i], ijk[3i+1], ijk[3i+2]) at
 * its own level and density rho[i]; the leaves must tile the box exactly
 * (no gap, no overlap).  Coarse levels hold volume means of the leaf field: a
 * region inside a coarser leaf takes that leaf's value (§3.2).
 *   1 <= base_level <= max_level <= 11; level and ijk are host arrays; rho
 *   is a device pointer if rho_on_device != 0, else host memory.
 * Output rows follow the depth-first (Morton) order of the leaves;
 * cd_tree_leaves() returns it.  The mesh description is built on the host
 * (synchronous); the density-dependent part runs on `stream`.
 * Errors: CD_EINVAL (bad level or index, overlap, gap), CD_ENOMEM, CD_ECUDA. */
cd_status cd_build_tree_amr(int base_level, int max_level, double box_cm, int64_t n_leaf, const int8_t *level,
                            const int32_t *ijk, const float *rho, int rho_on_device, void *stream, cd_tree *out);

/* Replaces the leaf densities of an existing tree and recomputes every coarse
 * level.  Uniform trees: same layout and rules as cd_build_tree_uniform.  AMR
 * trees: n_leaf values in the caller's original leaf order (the order given
 * to cd_build_tree_amr).  This is the per-step call of a simulation whose density
 * changes but whose mesh does not; it allocates nothing.  Asynchronous for a
 * device pointer; for host memory the data are copied before return. */
cd_status cd_tree_update(cd_tree tree, const float *rho, int rho_on_device, void *stream);

/* Precomputes the geometric factors of the precalculation module (§3.3) in
 * FP64 on the device and stores them in FP32 (sparse lists) and BF16 (dense
 * GEMM operands):
 *   K1[o][d][s]       shell of level l0-1, seen from the oct centre (8 configs)
 *   K2[o1 o2][d][s]   shell of level l0-2, seen from the oct centre (64)
 *   K3[o1 o2 o3][d][s] shells of level l <= l0-3, seen from the centre of
 *                      the ancestor at level l+2 (512)
 *   Kloc[t][s][d]     rays from the centre of oct child t through child s
 * s runs over the 6x6x6 level-l cells covering the 3x3x3 neighbourhood of the
 * level-(l-1) ancestor; cells of the inner region get 0.
 *   scheme         CD_DIRS_*; p0, p1 as documented there
 *   dirs           CD_DIRS_CUSTOM only: n_custom x 3 doubles (host)
 *   mode           CD_MODE_PREC, CD_MODE_INSITU (the tables are built either way; in-situ
 *                  evaluations use only the local ones) or CD_MODE_CONE (tables averaged
 *                  over each direction's cone)
 * 1 <= number of directions <= 768.  Components below 1e-14 in magnitude are
 * set to zero and each vector renormalised.  The tables are built on
 * `stream` and the call returns once they are complete (synchronous), so the
 * geometry may serve evaluations on any stream. */
cd_status cd_precompute_geometry(int scheme, int p0, int p1, const double *dirs, int n_custom, int mode,
                                 void *stream, cd_geom *out);

/* The hot path.  For every leaf t (Morton order) and direction d:
 *   n_h[t * n_dir + d]   N_H in cm^-2 (or NULL)
 *   a_v[t * n_dir + d]   N_H * av_per_nh (or NULL)
 *   shield[t]            (1/n_dir) sum_d exp(-shield_k * A_V) (or NULL)
 * All three are caller-owned DEVICE buffers.  opts may be NULL (defaults).
 * Scratch (per-level partial sums) and two side streams are owned by the
 * tree and reused; the first call on a tree (which allocates them) must not
 * run while `stream` is capturing.  The call's work starts after what was
 * enqueued on `stream` before it, and what is enqueued on `stream` after it
 * waits for all of it, side streams included.  Two evaluations of one tree
 * must not overlap on the GPU (other streams or host threads): serialise
 * them.
 * With opts->net set, N_H is the learned form N_tree exp(delta) of
 * colden_learned.h (uniform trees; the network's n_dir must equal the
 * geometry's, else CD_EINVAL; an AMR tree returns CD_EUNSUPPORTED). */
cd_status cd_column_density(cd_tree tree, cd_geom geom, const cd_opts *opts, float *n_h, float *a_v,
                            float *shield, void *stream);

/* Batched evaluation of n independent boxes (trees of any kind and size,
 * each with its own geometry and outputs, all with the same opts): the boxes
 * one after another on `stream`.  Entries of n_h / a_v / shield may be NULL;
 * the arrays themselves may be NULL when no box wants that output. */
cd_status cd_column_density_batch(int n, const cd_tree *trees, const cd_geom *geoms, const cd_opts *opts,
                                  float *const *n_h, float *const *a_v, float *const *shield, void *stream);

/* cd_column_density for a caller whose data live in HOST memory: rho (or
 * NULL to keep the tree's densities) is uploaded and applied as by
 * cd_tree_update (same layout and order; not validated, as on the device
 * path), then the evaluation runs and n_h, a_v and shield (host buffers of
 * the sizes above, any may be NULL) receive the results.  On a uniform tree of
 * 128 or more octs the leaf stage runs in 8 Morton chunks of whole 16-oct
 * tiles and each chunk's rows are copied to the host on an internal copy
 * stream while the next chunk is computed; otherwise the copies follow the
 * evaluation.  Device staging (densities, outputs) is owned by the tree,
 * allocated by the first call that needs it and kept until cd_tree_free, so
 * that first call must not run while `stream` is capturing.  Asynchronous
 * like cd_column_density: the host buffers are complete once `stream` has
 * completed the call's work (e.g. cudaStreamSynchronize).  Page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) keeps the copies asynchronous;
 * pageable memory works but the runtime may stage it.
 * Errors: as cd_column_density, CD_ENOMEM for the staging buffers. */
cd_status cd_column_density_host(cd_tree tree, cd_geom geom, const cd_opts *opts, const float *rho, float *n_h,
                                 float *a_v, float *shield, void *stream);

/* One evaluation step captured once as a CUDA graph and replayed by one
 * launch (csrc/graph.cu).  cd_eval_graph_create runs the step once eagerly on
 * `stream` (allocating every buffer the library allocates on first use) and
 * synchronises it, then captures on a private stream: cd_tree_update(tree,
 * rho, device) when rho is not NULL, then cd_column_density(tree, geom, opts,
 * n_h, a_v, shield), with the evaluation's fork and join over the tree's side
 * streams.  cd_eval_graph_launch enqueues the whole step on `stream` as one
 * graph launch: the same kernels with the same arguments, so the outputs are
 * bitwise those of the eager calls on the densities that rho holds at the
 * time of the launch (without rho, on the tree's current densities).
 *   rho      device [n_leaf] in cd_tree_update's layout (a uniform tree's
 *            [z][y][x] grid, an AMR tree's original leaf order), or NULL;
 *            read by every launch, caller-owned, must stay allocated
 *   n_h, a_v, shield   as cd_column_density; caller-owned, must stay allocated
 * The graph holds the device pointers of the tree, the geometry and the
 * network as they were at capture.  Every free of library-owned device memory
 * (a tree, geometry, network or batch freed; a tree's workspace reallocated by
 * an evaluation with another direction count; a network's scratch grown) makes
 * every later launch of every graph return CD_EINVAL without launching
 * anything, as does a change of the network's parameters (training,
 * cd_net_set_state) or trusted range; create the graph again.  A learned
 * graph (opts->net) must hold the update (rho != NULL), because the learned
 * form reuses its per-level sums while the host records them as current.
 * Launches add the recorded kernels to cd_stats_get's counts (not their
 * times); the capture itself counts nothing.  Creation must not happen while
 * `stream` is capturing.
 * Errors: CD_EINVAL (NULL handles or out, another current device, a learned
 * graph without rho), the errors of the eager step, CD_ECUDA when the capture
 * or the instantiation fails. */
typedef struct cd_eval_graph_s *cd_eval_graph;
cd_status cd_eval_graph_create(cd_tree tree, cd_geom geom, const cd_opts *opts, const float *rho, float *n_h,
                               float *a_v, float *shield, void *stream, cd_eval_graph *out);
cd_status cd_eval_graph_launch(cd_eval_graph graph, void *stream);
/* Kernels one launch runs (any pointer may be NULL). */
cd_status cd_eval_graph_info(cd_eval_graph graph, int64_t *kernels);
/* Synchronises the device, then frees the graph; NULL is ignored. */
void cd_eval_graph_free(cd_eval_graph graph);

/* A batch captured once into a single CUDA graph.  cd_batch_create evaluates
 * the batch once eagerly (allocating every box's scratch), then autotunes it:
 * each candidate form is captured into a graph and its replay timed, and the
 * fastest graph is kept.  The candidates are the persistent form below (BF16
 * batches it serves, each shell tile shape and CTA count) and every box's own
 * kernels on W forked streams, W in {1, 2, 4, 8} (boxes placed largest first
 * on the least loaded branch).  It synchronises and returns with the outputs
 * of the last replay.  cd_batch_run launches the graph
 * on `stream`: one launch evaluates every box with its tree's current
 * densities (cd_tree_update between runs is seen).  The trees, geometries and
 * output buffers given at creation must stay alive and must not be resized
 * until cd_batch_free.  Creation must not happen while `stream` is capturing.
 * The graph holds each tree's scratch buffers, so while the batch lives they
 * are pinned: cd_column_density on one of its trees with a geometry of
 * another direction count (which would reallocate them) returns CD_EINVAL.
 * Errors at creation: CD_EINVAL for NULL entries or a tree listed twice with
 * geometries of different direction counts; CD_EUNSUPPORTED for a learned
 * correction in opts (its cached per-level sums are not replay-safe: use
 * cd_column_density_batch). */
cd_status cd_batch_create(int n, const cd_tree *trees, const cd_geom *geoms, const cd_opts *opts, float *const *n_h,
                          float *const *a_v, float *const *shield, void *stream, cd_batch *out);
cd_status cd_batch_run(cd_batch batch, void *stream);
/* Chosen branch count (per-box form), graph replay milliseconds measured for
 * W = 1, 2, 4, 8 (-1 where not tried; any pointer may be NULL) and the kernel
 * launches one run contains. */
cd_status cd_batch_info(cd_batch batch, int *width, double *ms_tried, int64_t *kernel_nodes);
/* The persistent form (BF16 batches the tensor-core path serves: see below).
 * *persistent = 1 when the graph holds the persistent launches, 0 when it
 * holds every box's kernels (then the other outputs are 0 / -1).  The
 * autotuner's choice: *full_tiles = 1 when shell tiles cover all 8 children
 * (N = 8 n_dir, boxes with n_dir <= 32), 0 for half the children (N = 4 n_dir);
 * *ctas_per_sm = 1 or 2 persistent shell CTAs per SM; ms_tried[4] = graph
 * replay milliseconds for (half, 1), (half, 2), (full, 1), (full, 2), -1
 * where not tried.  Any pointer may be NULL.
 *
 * Persistent form.  Per batch: one FP32 launch for the level-3 far shells of
 * every box; one persistent tensor-core launch over a device work list of
 * (box, level, tile) for every shell of levels >= 4 (the far shells level by
 * level, each adding its box's S_{k-1} once that level is complete, then the
 * oct levels); one persistent leaf launch per direction set over (box, tile).
 * The waits between levels are bounded spins on per-job counters inside the
 * launch; a spin that runs out sets the flag cd_device_status reports as
 * CD_ETIMEOUT (it can only run out if other work holds SMs for seconds while
 * the batch runs).  Results agree with per-box evaluation within the BF16
 * tolerance, not bitwise: the level-3 shells of uniform boxes go through the
 * list kernel and the local term carries dx in the epilogue instead of the
 * BF16 operand. */
cd_status cd_batch_plan(cd_batch batch, int *persistent, int *full_tiles, int *ctas_per_sm, double *ms_tried);
/* Releases the graph and the internal streams (synchronises the device first);
 * the trees, geometries and outputs stay the caller's.  NULL is ignored. */
void cd_batch_free(cd_batch batch);

/* Same evaluation as cd_column_density (FP32, uniform trees), but its scratch
 * lives in a fixed 16 MiB device array compiled into the library, so the call
 * allocates and frees nothing.  The paper has no counterpart: this serves
 * simulation codes that reserve all device memory once at start-up and must
 * not allocate inside their time-step loop (allocation calls may synchronise
 * the device and stall an asynchronous step loop).  Build the tree and the
 * geometry during set-up, then call this every step.
 *   Limit: n_dir * (8^3 + ... + 8^(L-2) + 8^(L-1)) floats (plus 256-byte
 *   rounding) must fit in 4 Mi floats, e.g. L <= 6 with 48 directions; larger
 *   trees get CD_EINVAL with the required size in cd_last_error().
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current.  That lookup is also
 *   what makes the CUDA runtime load the library's module holding the array
 *   on that device (modules load lazily), i.e. where the 16 MiB are taken.
 *   So make one call during set-up, before the time-step loop and before any
 *   stream capture: a call with all three outputs NULL does the lookup and
 *   enqueues nothing.
 *   Every call on a device shares the one array and leaves its contents
 *   behind; nothing in it needs clearing (each element read is written
 *   earlier in the same call).  Calls that overlap on the GPU (different
 *   streams or host threads) race on the array: serialise them.
 *   Every GPU that loads the library holds the 16 MiB until the process exits.
 * Other arguments, outputs and errors as for cd_column_density;
 * CD_EUNSUPPORTED for BF16, AMR trees or a learned correction. */
cd_status cd_column_density_noalloc(cd_tree tree, cd_geom geom, const cd_opts *opts, float *n_h, float *a_v,
                                    float *shield, void *stream);

/* The heating of the application (§5) for every leaf, in the output order
 * (the order of cd_column_density's shield):
 *   g0_eff[i]   = chi[i] G0                                      (Eq. G0_eff)
 *   gamma_uv[i] = 1e-24 eps G0_eff n   erg cm^-3 s^-1            (Eq. gamma_uv)
 *   gamma_cr[i] = 1e-27 n              erg cm^-3 s^-1            (Eq. gamma_cr)
 * with n the tree's leaf density (cm^-3, as last built or updated) and the
 * photoelectric efficiency of Wolfire et al. (1995), x = G0_eff sqrt(T) / n_e:
 *   eps = 4.9e-2 / (1 + (x / 1925)^0.73) + 3.7e-2 (T / 1e4)^0.7 / (1 + x / 5000).
 *   chi        n_leaf floats (device): the attenuation factor; the paper's
 *              chi = <exp(-2e-21 N)> is cd_column_density's shield with
 *              av_per_nh = 1 and shield_k = 2e-21
 *   T, n_e     n_leaf floats (device): temperature (K, >= 0) and electron
 *              density (cm^-3, > 0; §5 takes it from Wolfire et al. 2003, which
 *              the paper does not restate, so the caller supplies it); needed
 *              only for gamma_uv, may be NULL otherwise
 *   G0         the unscreened field in Habing units (§5: 1.7), finite, >= 0
 *   g0_eff, gamma_uv, gamma_cr   caller-owned device outputs of n_leaf
 *              floats, each may be NULL
 * FP32 arithmetic (powf, sqrtf).  Errors: CD_EINVAL (NULL tree or chi,
 * gamma_uv without T or n_e, bad G0).  Asynchronous on `stream`. */
cd_status cd_heating(cd_tree tree, const float *chi, const float *T, const float *n_e, double G0, float *g0_eff,
                     float *gamma_uv, float *gamma_cr, void *stream);

/* Sizes of a tree: number of leaves, finest level, base level, number of
 * leaf-bearing octs.  Any pointer may be NULL. */
cd_status cd_tree_info(cd_tree tree, int64_t *n_leaf, int *max_level, int *base_level, int64_t *n_oct);

/* Level and (i, j, k) index of every leaf in output order, written to host
 * arrays of n_leaf and 3 n_leaf elements.  Synchronous. */
cd_status cd_tree_leaves(cd_tree tree, int8_t *level, int32_t *ijk);

/* Number of directions and, if dirs != NULL, the n_dir x 3 unit vectors (host). */
cd_status cd_geom_info(cd_geom geom, int *n_dir, double *dirs);

/* Rays the geometric factors average over: *n_sub per direction (1 unless the
 * geometry's mode is CD_MODE_CONE, then CD_CONE_SUBRAYS) and, if rays != NULL,
 * the n_dir x n_sub x 3 unit vectors (host), direction-major. */
cd_status cd_geom_rays(cd_geom geom, int *n_sub, double *rays);

/* Checkpoint images (no counterpart in the paper, which restarts from its
 * simulation's own outputs).  An image is a flat little-endian byte string
 * that ends in the FNV-1a 64-bit hash (cd_fnv1a64) of every byte before it.
 *
 * cd_tree_save: the mesh and its current densities, leaves in output order:
 *   "CDTREE01" | int32 amr, base_level, max_level | float64 box_cm |
 *   int64 n_leaf | int8 level[n] | int32 ijk[3 n] | float32 rho[n] | uint64 hash
 * *size receives the image's size; with buf == NULL nothing else happens,
 * else the image is written to buf (cap bytes; CD_EINVAL if too small).
 * Synchronises `stream` (it reads the densities after the work on it).
 * cd_tree_load builds the tree again (as cd_build_tree_uniform or
 * cd_build_tree_amr, on `stream`).  An AMR tree loaded this way takes
 * cd_tree_update densities in output order (the order it was saved in).
 * CD_EINVAL for a damaged image (hash), a wrong magic or inconsistent sizes.
 *
 * cd_geom_save: how the direction set was made and what it holds:
 *   "CDGEOM01" | int32 scheme, p0, p1, mode, n_dir, n_custom |
 *   float64 custom[3 n_custom] (CD_DIRS_CUSTOM: the vectors as given) |
 *   float64 dirs[3 n_dir] | uint64 dirs_hash | uint64 table_hash | uint64 hash
 * (same size / buffer convention; synchronous).  cd_geom_load rebuilds the
 * geometry with cd_precompute_geometry from the recorded construction and
 * returns CD_EINVAL unless the rebuilt directions equal the saved ones bit for
 * bit and the rebuilt tables have the saved table hash (an image from a
 * library whose direction sets or tables differ is refused).
 * cd_geom_hash: dirs_hash = FNV-1a of (int32 mode, int32 n_dir, dirs);
 * table_hash = FNV-1a of int32 maxe followed by every table the evaluation
 * reads (Kloc, the FP32 shell tables and counts, the BF16 operands) as stored
 * on the device.  Either pointer may be NULL. */
cd_status cd_tree_save(cd_tree tree, void *buf, size_t cap, size_t *size, void *stream);
cd_status cd_tree_load(const void *buf, size_t size, void *stream, cd_tree *out);
cd_status cd_geom_save(cd_geom geom, void *buf, size_t cap, size_t *size);
cd_status cd_geom_load(const void *buf, size_t size, void *stream, cd_geom *out);
cd_status cd_geom_hash(cd_geom geom, uint64_t *dirs_hash, uint64_t *table_hash);
/* FNV-1a, 64 bits (Fowler, Noll, Vo): h = 14695981039346656037; for each
 * byte b: h = (h ^ b) * 1099511628211 mod 2^64. */
uint64_t cd_fnv1a64(const void *data, size_t n);

/* Synchronises `stream` and reports whether any library kernel on the current
 * device gave up a bounded wait since the last call: CD_ETIMEOUT (flag
 * cleared, message in cd_last_error()) or CD_OK.  Kernels never trap; a wait
 * that runs out of polls records this flag and the kernel returns early, so
 * its outputs are then incomplete. */
cd_status cd_device_status(void *stream);

/* Testing hook of the failure detection above (no counterpart in the paper).
 * polls >= 0 caps the pipeline waits of the tensor-core leaf kernel (the
 * BF16 leaf epilogue: its input copies landing, its product completing) at
 * `polls` polls; with
 * 0 they give up at once, so every CTA takes the timeout path: it records the
 * flag, still waits (with the full limit) for the copies and products it has
 * issued, frees its tensor memory and returns, and cd_device_status then
 * reports CD_ETIMEOUT while the context stays usable.  polls < 0 restores the
 * default limit.  Process-wide; applies to launches enqueued after the call.
 * Never set it outside tests: the outputs of capped launches are incomplete. */
void cd_debug_wait_polls(int64_t polls);

/* Testing hook (no counterpart in the paper).  On AMR trees the BF16 leaf
 * kernel adds each oct's far-shell prefix row (S of the parent level, §3.3)
 * itself: a tile of 16 consecutive octs stages its parents' rows, which form
 * one contiguous span of S, with one copy when the span is at most `rows`
 * rows (16 by default, the staging capacity), else one row per oct.  rows = 0
 * forces the per-oct form everywhere; the results do not change.  rows < 0 or
 * > 16 restores the default.  Process-wide; applies to later launches. */
void cd_debug_leaf_span(int rows);

/* Bounds-checked build (no counterpart in the paper).  Built with
 * -DCOLDEN_CHECKED (libcolden_checked.so, a test build), the kernels check the
 * indices of their gathers and stores before each access; one that falls
 * outside what it addresses is skipped and recorded (first failure wins) in
 * a device error word, with no trap.  Sites:
 *   11 FP32 shell kernel: stencil offset from the tables within the staged
 *      density region;  12: output row;  13: far-shell prefix row
 *   21 tensor-core shell kernel: brick index of an A-operand gather
 *   31 tensor-core leaf kernel: a tile's octs (E, densities) and parents (S)
 *   32 tensor-core leaf kernel: output row (N_H, A_V, screening factor)
 *   41 FP32 leaf kernel: a batch's octs and parents
 *   51 AMR list shell kernel: stencil offset within the stencil region
 *    1 cd_debug_check_probe
 * cd_checked_status synchronises the device and returns, in *site and
 * *index, the first failure since the last call (0 and 0 when none), then
 * clears it.  cd_debug_check_probe(i) reads element i of a 4-element device
 * array through the check (i outside 0..3 must be recorded as site 1, not
 * read).  Both return CD_EUNSUPPORTED from the normal library. */
cd_status cd_checked_status(int *site, int64_t *index);
cd_status cd_debug_check_probe(int64_t i, void *stream);

/* Testing hook of the batch autotuner (no counterpart in the paper): form = 0
 * restricts later cd_batch_create calls to the per-box form, 1 to the
 * persistent form where the batch supports it (else the per-box form), < 0
 * restores the autotuner's choice between them.  Process-wide. */
void cd_debug_batch_form(int form);

/* Launch statistics of this process, for benchmarks.  Kernel kinds: */
enum {
    CD_K_RESTRICT = 0,     /* level restriction and leaf reordering */
    CD_K_SHELL = 1,        /* shell contraction of one level (FP32 or tensor core) */
    CD_K_LEAF = 2,         /* per-leaf combine + epilogue */
    CD_K_OTHER = 3,        /* geometry precompute and the rest */
    CD_K_NET = 4,          /* the learned correction's network: FP32 GEMMs, Adam, per-oct tensor-core layer 1 */
    CD_K_FEATURES = 5,     /* per-level inputs of the network and the FP32 learned combine */
    CD_K_RAYMARCH = 6,     /* exact ray-marcher */
    CD_K_LEARNED = 7,      /* fused per-leaf learned kernel (BF16 tensor cores) */
    CD_K_HEATING = 8,      /* the heating epilogue (cd_heating) */
    CD_K_COUNT = 9
};
/* Resets the counters; with timing != 0 later launches also record CUDA
 * events on their stream (a synchronisation happens in cd_stats_get).  An
 * evaluation normally runs its independent steps (the far-shell prefix
 * chain, the oct shells, the leaves of each AMR level) concurrently on two
 * internal side streams joined back into the caller's stream; while timing
 * is on it runs every launch in order on the caller's stream instead, so
 * that each launch's events time that launch alone. */
void cd_stats_reset(int timing);
/* Number of kernel launches of one kind since the reset and, if timing was
 * on, their summed device time in milliseconds (synchronises the device). */
cd_status cd_stats_get(int kind, int64_t *launches, double *ms);
/* Dense tensor-core work, in flops, that the launches of one kind issued
 * since the reset: 2 M N K summed over their tcgen05 MMAs, zero rows and
 * columns of padded tiles included (0 for kinds that run on the CUDA cores).
 * Counted on the host at launch time, so launches replayed from a CUDA graph
 * (cd_batch_run) are not counted. */
cd_status cd_stats_flops(int kind, double *flops);

/* Release a handle and every device buffer, stream and event it owns, after
 * synchronising the device (work still enqueued on it finishes first).  NULL
 * is ignored; a handle must not be used after it is freed. */
void cd_tree_free(cd_tree tree);
void cd_geom_free(cd_geom geom);
/* The message of the last failed call on this host thread (thread-local,
 * library-owned, valid until the thread's next failing call). */
const char *cd_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* COLDEN_H */
