/*
 * FP64 CPU oracle of the tree-based column-density method of Valdivia & Hennebelle
 * ("A fast tree-based method for estimating column densities in AMR codes").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * What it computes, step by step and in the paper's order (§3.2 and §3.3):
 *   - the tree: the value of a cell at level l is the volume mean of the leaf
 *     field over that cell (the coarse-level density "corresponds to a mean",
 *     §3.2); a region inside a coarser leaf takes that leaf's value;
 *   - directions: the equal-area M x N set (§3.2, eqs. theta/phi), HEALPix ring
 *     pixel centres (Gorski et al. 2005), the six axis rays (§4.3), or a list;
 *   - for every target leaf t at level l0 and direction d, the column
 *     N(m,n) = sum_i n_i dx_i(m,n)  (Eq. N_discret1):
 *       internal + local: a ray from the centre of t through t and its seven
 *         siblings, each path length computed by a slab intersection;
 *       external (Eqs. N_discret0, deltax, N_discret): for every shell level
 *         l = l0-1 ... 1 the level-l cells of the 3x3x3 block of level-(l-1)
 *         cells around the ancestor A_{l-1}, minus the inner region (the cell
 *         A_{l0-1} for the first shell, the 3x3x3 level-l block around A_l for
 *         the others), each weighted by the length of a ray from the reference
 *         point p_ref(l) through it.  p_ref(l) is the centre of
 *         A_{min(l+2, l0-1)} under the two-level approximation of §3.3, and the
 *         centre of A_{l0-1} (the oct centre) in the in-situ variant of §4.3.
 *     The oracle loops over the cells of each shell directly: no table, no
 *     GEMM, no sharing between targets.
 *   - the brute-force reference: an exact line integral of the leaf field from
 *     the centre of t to the box edge, marched cell by cell on the finest grid
 *     (the ray-tracing reference of §4).
 *
 * Readings of points the paper leaves open (all listed in the design notes):
 *   box [0, L]^3, non-periodic, density zero outside; octant code
 *   ix&1 + 2(iy&1) + 4(iz&1); direction components below 1e-14 in magnitude are
 *   set to zero and the vector renormalised.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define OR_MAXL 20

/* ------------------------------------------------------------------------- */
/* Directions                                                                */
/* ------------------------------------------------------------------------- */

static void snap_normalise(double *v)
{
    for (int a = 0; a < 3; ++a)
        if (fabs(v[a]) < 1e-14) v[a] = 0.0;
    double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    for (int a = 0; a < 3; ++a) v[a] /= n;
}

static void from_angles(double theta, double phi, double *v)
{
    v[0] = sin(theta) * cos(phi);
    v[1] = sin(theta) * sin(phi);
    v[2] = cos(theta);
    snap_normalise(v);
}

/* Equal-area M x N set of §3.2: theta_m = arccos(1 + (1-2m)/M),
 * phi_n = 2 pi (n-1)/N, m in [1,M], n in [1,N].  Output index (m-1)*N + (n-1). */
int or_dirs_mxn(int M, int N, double *out)
{
    if (M < 1 || N < 1) return -1;
    for (int m = 1; m <= M; ++m)
        for (int n = 1; n <= N; ++n) {
            double theta = acos(1.0 + (double)(1 - 2 * m) / (double)M);
            double phi = 2.0 * M_PI * (double)(n - 1) / (double)N;
            from_angles(theta, phi, out + 3 * ((m - 1) * N + (n - 1)));
        }
    return M * N;
}

/* HEALPix ring-scheme pixel centres (Gorski et al. 2005, ApJ 622, 759, Sect. 4):
 * rings i = 1 .. 4 Nside - 1 from north to south, pixels by increasing phi. */
int or_dirs_healpix(int nside, double *out)
{
    if (nside < 1) return -1;
    int p = 0;
    double ns = (double)nside;
    for (int i = 1; i <= 4 * nside - 1; ++i) {
        if (i < nside || i > 3 * nside) {
            int ic = (i < nside) ? i : 4 * nside - i; /* polar-cap ring index */
            double z = 1.0 - (double)ic * (double)ic / (3.0 * ns * ns);
            if (i > 3 * nside) z = -z;
            for (int j = 1; j <= 4 * ic; ++j) {
                double phi = M_PI / (2.0 * ic) * ((double)j - 0.5);
                from_angles(acos(z), phi, out + 3 * p);
                ++p;
            }
        } else {
            double z = 4.0 / 3.0 - 2.0 * (double)i / (3.0 * ns);
            int s = (i - nside + 1) % 2;
            for (int j = 1; j <= 4 * nside; ++j) {
                double phi = M_PI / (2.0 * ns) * ((double)j - 0.5 * (double)s);
                from_angles(acos(z), phi, out + 3 * p);
                ++p;
            }
        }
    }
    return p;
}

/* The six-ray set of §4.3: +x, -x, +y, -y, +z, -z. */
int or_dirs_axes(double *out)
{
    static const double ax[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0},
                                    {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
    memcpy(out, ax, sizeof(ax));
    return 6;
}

/* A caller-supplied list, normalised and snapped like the others. */
int or_dirs_custom(int n, const double *in, double *out)
{
    for (int i = 0; i < n; ++i) {
        double v[3] = {in[3 * i], in[3 * i + 1], in[3 * i + 2]};
        double nn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        if (!(nn > 0.0)) return -1;
        for (int a = 0; a < 3; ++a) v[a] /= nn;
        snap_normalise(v);
        memcpy(out + 3 * i, v, sizeof(v));
    }
    return n;
}

/* ------------------------------------------------------------------------- */
/* Geometry: length of the ray {p + s d, s >= 0} inside an axis-aligned cube */
/* ------------------------------------------------------------------------- */

double or_ray_cube(const double *p, const double *d, const double *lo, double h)
{
    double t0 = 0.0, t1 = INFINITY;
    for (int a = 0; a < 3; ++a) {
        double lo_a = lo[a], hi_a = lo[a] + h;
        if (d[a] == 0.0) {
            if (p[a] < lo_a || p[a] > hi_a) return 0.0;
            continue;
        }
        double ta = (lo_a - p[a]) / d[a];
        double tb = (hi_a - p[a]) / d[a];
        if (ta > tb) { double x = ta; ta = tb; tb = x; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    return (t1 > t0) ? (t1 - t0) : 0.0;
}

/* ------------------------------------------------------------------------- */
/* Tree: volume means at every level                                         */
/* ------------------------------------------------------------------------- */

typedef struct {
    int base, lmax;
    double box;
    double *dense[OR_MAXL + 1];   /* levels 0..base: row-major, x fastest */
    int64_t nsp[OR_MAXL + 1];     /* levels base+1..lmax: cells that exist */
    uint64_t *key[OR_MAXL + 1];   /* sorted row-major keys */
    double *val[OR_MAXL + 1];
    uint8_t *isleaf[OR_MAXL + 1];
} or_tree;

static uint64_t key_of(int l, int64_t i, int64_t j, int64_t k)
{
    return ((uint64_t)k << (2 * l)) | ((uint64_t)j << l) | (uint64_t)i;
}

static int64_t find_key(const uint64_t *keys, int64_t n, uint64_t k)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        if (keys[mid] == k) return mid;
        if (keys[mid] < k) lo = mid + 1; else hi = mid - 1;
    }
    return -1;
}

/* Volume-mean density of cell (i,j,k) at level l; zero outside the box. */
double or_rho(const or_tree *T, int l, int64_t i, int64_t j, int64_t k)
{
    int64_t n = (int64_t)1 << l;
    if (i < 0 || j < 0 || k < 0 || i >= n || j >= n || k >= n) return 0.0;
    if (l <= T->base) return T->dense[l][(k * n + j) * n + i];
    int64_t at = find_key(T->key[l], T->nsp[l], key_of(l, i, j, k));
    if (at >= 0) return T->val[l][at];
    /* not refined to level l: the region lies inside a coarser leaf */
    return or_rho(T, l - 1, i >> 1, j >> 1, k >> 1);
}

static void dense_means_below(or_tree *T)
{
    for (int l = T->base - 1; l >= 0; --l) {
        int64_t n = (int64_t)1 << l, nc = 2 * n;
        T->dense[l] = (double *)malloc(sizeof(double) * n * n * n);
        const double *c = T->dense[l + 1];
        for (int64_t k = 0; k < n; ++k)
            for (int64_t j = 0; j < n; ++j)
                for (int64_t i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int o = 0; o < 8; ++o) {
                        int64_t ci = 2 * i + (o & 1), cj = 2 * j + ((o >> 1) & 1),
                                ck = 2 * k + ((o >> 2) & 1);
                        s += c[(ck * nc + cj) * nc + ci];
                    }
                    T->dense[l][(k * n + j) * n + i] = s / 8.0;
                }
    }
}

void or_tree_free(or_tree *T)
{
    if (!T) return;
    for (int l = 0; l <= OR_MAXL; ++l) {
        free(T->dense[l]);
        free(T->key[l]);
        free(T->val[l]);
        free(T->isleaf[l]);
    }
    free(T);
}

/* Uniform grid of 2^L cells per axis, rho row-major (x fastest). */
or_tree *or_tree_uniform(int L, double box, const float *rho)
{
    if (L < 0 || L > 10) return NULL;
    or_tree *T = (or_tree *)calloc(1, sizeof(or_tree));
    T->base = T->lmax = L;
    T->box = box;
    int64_t n = (int64_t)1 << L, N = n * n * n;
    T->dense[L] = (double *)malloc(sizeof(double) * N);
    for (int64_t x = 0; x < N; ++x) T->dense[L][x] = (double)rho[x];
    dense_means_below(T);
    return T;
}

typedef struct { uint64_t key; double val; uint8_t leaf; } entry;

static int cmp_entry(const void *a, const void *b)
{
    uint64_t x = ((const entry *)a)->key, y = ((const entry *)b)->key;
    return (x > y) - (x < y);
}

/* AMR tree: n leaves with level lvl[i] in [base, lmax], integer index
 * ijk[3i..3i+2] at their own level, density rho[i].  The leaves must tile the
 * box exactly.  Returns NULL and writes a message to err on failure. */
or_tree *or_tree_amr(int base, int lmax, double box, int64_t n, const int8_t *lvl,
                     const int32_t *ijk, const float *rho, char *err, int errlen)
{
    if (base < 0 || lmax < base || lmax > OR_MAXL || base > 10) {
        snprintf(err, errlen, "bad levels");
        return NULL;
    }
    or_tree *T = (or_tree *)calloc(1, sizeof(or_tree));
    T->base = base;
    T->lmax = lmax;
    T->box = box;
    /* per-level entry lists, built from the finest level up */
    entry *lists[OR_MAXL + 1] = {0};
    int64_t cnt[OR_MAXL + 1] = {0}, cap[OR_MAXL + 1] = {0};
    for (int64_t x = 0; x < n; ++x) {
        int l = lvl[x];
        if (l < base || l > lmax) { snprintf(err, errlen, "leaf level out of range"); goto fail; }
        int64_t m = (int64_t)1 << l;
        if (ijk[3 * x] < 0 || ijk[3 * x + 1] < 0 || ijk[3 * x + 2] < 0 ||
            ijk[3 * x] >= m || ijk[3 * x + 1] >= m || ijk[3 * x + 2] >= m) {
            snprintf(err, errlen, "leaf index outside the box");
            goto fail;
        }
        if (cnt[l] == cap[l]) {
            cap[l] = cap[l] ? 2 * cap[l] : 1024;
            lists[l] = (entry *)realloc(lists[l], sizeof(entry) * cap[l]);
        }
        entry e = {key_of(l, ijk[3 * x], ijk[3 * x + 1], ijk[3 * x + 2]), (double)rho[x], 1};
        lists[l][cnt[l]++] = e;
    }
    for (int l = lmax; l >= base; --l) {
        if (l < lmax) {
            /* parents of the level-(l+1) cells are refined cells at level l */
            int64_t m1 = (int64_t)1 << (l + 1);
            for (int64_t x = 0; x < T->nsp[l + 1]; ++x) {
                uint64_t k1 = T->key[l + 1][x];
                int64_t i = (int64_t)(k1 % (uint64_t)m1), j = (int64_t)((k1 / (uint64_t)m1) % (uint64_t)m1),
                        k = (int64_t)(k1 / ((uint64_t)m1 * (uint64_t)m1));
                if (cnt[l] == cap[l]) {
                    cap[l] = cap[l] ? 2 * cap[l] : 1024;
                    lists[l] = (entry *)realloc(lists[l], sizeof(entry) * cap[l]);
                }
                entry e = {key_of(l, i >> 1, j >> 1, k >> 1), 0.0, 0};
                lists[l][cnt[l]++] = e;
            }
        }
        qsort(lists[l], cnt[l], sizeof(entry), cmp_entry);
        /* deduplicate refined cells; a key that is both a leaf and refined is an overlap */
        int64_t w = 0;
        for (int64_t x = 0; x < cnt[l]; ++x) {
            if (w > 0 && lists[l][w - 1].key == lists[l][x].key) {
                if (lists[l][w - 1].leaf || lists[l][x].leaf) {
                    snprintf(err, errlen, "overlapping leaves at level %d", l);
                    goto fail;
                }
                continue;
            }
            lists[l][w++] = lists[l][x];
        }
        cnt[l] = w;
        T->nsp[l] = w;
        T->key[l] = (uint64_t *)malloc(sizeof(uint64_t) * (w ? w : 1));
        T->val[l] = (double *)malloc(sizeof(double) * (w ? w : 1));
        T->isleaf[l] = (uint8_t *)malloc(w ? w : 1);
        for (int64_t x = 0; x < w; ++x) {
            T->key[l][x] = lists[l][x].key;
            T->isleaf[l][x] = lists[l][x].leaf;
            if (lists[l][x].leaf) {
                T->val[l][x] = lists[l][x].val;
            } else {
                /* refined: the volume mean of its eight children (all must exist) */
                int64_t m = (int64_t)1 << l;
                uint64_t kk = lists[l][x].key;
                int64_t i = (int64_t)(kk % (uint64_t)m), j = (int64_t)((kk / (uint64_t)m) % (uint64_t)m),
                        k = (int64_t)(kk / ((uint64_t)m * (uint64_t)m));
                double s = 0.0;
                for (int o = 0; o < 8; ++o) {
                    int64_t at = find_key(T->key[l + 1], T->nsp[l + 1],
                                          key_of(l + 1, 2 * i + (o & 1), 2 * j + ((o >> 1) & 1),
                                                 2 * k + ((o >> 2) & 1)));
                    if (at < 0) { snprintf(err, errlen, "incomplete oct at level %d", l + 1); goto fail; }
                    s += T->val[l + 1][at];
                }
                T->val[l][x] = s / 8.0;
            }
        }
    }
    /* the base level is dense and every base cell must exist */
    {
        int64_t m = (int64_t)1 << base, N = m * m * m;
        if (T->nsp[base] != N) { snprintf(err, errlen, "leaves do not cover the box"); goto fail; }
        T->dense[base] = (double *)malloc(sizeof(double) * N);
        for (int64_t x = 0; x < N; ++x) T->dense[base][T->key[base][x]] = T->val[base][x];
        free(T->key[base]); free(T->val[base]); free(T->isleaf[base]);
        T->key[base] = NULL; T->val[base] = NULL; T->isleaf[base] = NULL;
        T->nsp[base] = 0;
    }
    dense_means_below(T);
    for (int l = 0; l <= OR_MAXL; ++l) free(lists[l]);
    return T;
fail:
    for (int l = 0; l <= OR_MAXL; ++l) free(lists[l]);
    or_tree_free(T);
    return NULL;
}

/* ------------------------------------------------------------------------- */
/* The tree method for one target leaf                                       */
/* ------------------------------------------------------------------------- */

enum { OR_MODE_PREC = 0, OR_MODE_INSITU = 1 };

/* Writes N[d] (cm^-2) for the leaf at level l0, index (i,j,k).  If per_level is
 * not NULL it receives the contribution of every shell as well:
 * per_level[(l0 - l) * ndir + d] for l = l0-1..1 at slot l0-l, and the
 * internal+local part at slot 0 (l0 slots in total). */
static void colden_one(const or_tree *T, int l0, int64_t i, int64_t j, int64_t k, int ndir,
                       const double *dirs, int mode, double *out, double *per_level)
{
    const double box = T->box;
    double dx0 = box / (double)((int64_t)1 << l0);
    double xt[3] = {((double)i + 0.5) * dx0, ((double)j + 0.5) * dx0, ((double)k + 0.5) * dx0};
    for (int d = 0; d < ndir; ++d) out[d] = 0.0;
    if (per_level) memset(per_level, 0, sizeof(double) * (size_t)ndir * (size_t)(l0 > 0 ? l0 : 1));

    /* internal and local contributions: rays from the target centre through the
     * target and its siblings (the cells of its oct), at level l0 */
    int64_t oi = i & ~(int64_t)1, oj = j & ~(int64_t)1, ok = k & ~(int64_t)1;
    for (int s = 0; s < 8; ++s) {
        int64_t ci = oi + (s & 1), cj = oj + ((s >> 1) & 1), ck = ok + ((s >> 2) & 1);
        double r = or_rho(T, l0, ci, cj, ck);
        double lo[3] = {(double)ci * dx0, (double)cj * dx0, (double)ck * dx0};
        for (int d = 0; d < ndir; ++d) {
            double c = r * or_ray_cube(xt, dirs + 3 * d, lo, dx0);
            out[d] += c;
            if (per_level) per_level[d] += c;
        }
    }

    /* external contribution: one concentric cubic shell per level l < l0 */
    for (int l = l0 - 1; l >= 1; --l) {
        double dxl = box / (double)((int64_t)1 << l);
        int r = (mode == OR_MODE_INSITU) ? (l0 - 1) : ((l + 2 < l0 - 1) ? l + 2 : l0 - 1);
        double dxr = box / (double)((int64_t)1 << r);
        double p[3] = {((double)(i >> (l0 - r)) + 0.5) * dxr, ((double)(j >> (l0 - r)) + 0.5) * dxr,
                       ((double)(k >> (l0 - r)) + 0.5) * dxr};
        int64_t ai = i >> (l0 - l), aj = j >> (l0 - l), ak = k >> (l0 - l);              /* A_l */
        int64_t pi = i >> (l0 - l + 1), pj = j >> (l0 - l + 1), pk = k >> (l0 - l + 1);  /* A_{l-1} */
        for (int nz = -1; nz <= 1; ++nz)
            for (int ny = -1; ny <= 1; ++ny)
                for (int nx = -1; nx <= 1; ++nx)
                    for (int ch = 0; ch < 8; ++ch) {
                        int64_t ci = 2 * (pi + nx) + (ch & 1), cj = 2 * (pj + ny) + ((ch >> 1) & 1),
                                ck = 2 * (pk + nz) + ((ch >> 2) & 1);
                        int inner;
                        if (l == l0 - 1)
                            inner = (ci == ai && cj == aj && ck == ak);
                        else
                            inner = (llabs(ci - ai) <= 1 && llabs(cj - aj) <= 1 && llabs(ck - ak) <= 1);
                        if (inner) continue;
                        double rho = or_rho(T, l, ci, cj, ck);
                        if (rho == 0.0) continue;
                        double lo[3] = {(double)ci * dxl, (double)cj * dxl, (double)ck * dxl};
                        for (int d = 0; d < ndir; ++d) {
                            double c = rho * or_ray_cube(p, dirs + 3 * d, lo, dxl);
                            out[d] += c;
                            if (per_level) per_level[(size_t)(l0 - l) * ndir + d] += c;
                        }
                    }
    }
}

/* Tree-method columns for n targets (level lvl[t], index ijk[3t..]); out is
 * n x ndir.  per_level (optional) is n x maxslots x ndir with maxslots >= l0. */
int or_colden(const or_tree *T, int ndir, const double *dirs, int mode, int64_t n, const int32_t *lvl,
              const int32_t *ijk, double *out, int maxslots, double *per_level)
{
    int bad = 0;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n; ++t) {
        int l0 = lvl[t];
        if (l0 < 0 || l0 > T->lmax || (per_level && l0 > maxslots)) { bad = 1; continue; }
        colden_one(T, l0, ijk[3 * t], ijk[3 * t + 1], ijk[3 * t + 2], ndir, dirs, mode,
                   out + (size_t)t * ndir, per_level ? per_level + (size_t)t * maxslots * ndir : NULL);
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------------- */
/* Brute-force reference: exact line integral to the box edge                */
/* ------------------------------------------------------------------------- */

/* Marches the finest grid (level lmax) cell by cell (Amanatides & Woo 1987)
 * from point x0 along unit vector d until the ray leaves the box.  Every leaf
 * is a union of finest cells, so the sum of rho_leaf x segment is exact. */
static double march(const or_tree *T, const double *x0, const double *d)
{
    int lf = T->lmax;
    int64_t m = (int64_t)1 << lf;
    double h = T->box / (double)m;
    int64_t c[3];
    double tnext[3], tdelta[3];
    int step[3];
    for (int a = 0; a < 3; ++a) {
        c[a] = (int64_t)floor(x0[a] / h);
        if (c[a] >= m) c[a] = m - 1;
        if (c[a] < 0) c[a] = 0;
        if (d[a] > 0.0) {
            step[a] = 1;
            tnext[a] = ((double)(c[a] + 1) * h - x0[a]) / d[a];
            tdelta[a] = h / d[a];
        } else if (d[a] < 0.0) {
            step[a] = -1;
            tnext[a] = ((double)c[a] * h - x0[a]) / d[a];
            tdelta[a] = -h / d[a];
        } else {
            step[a] = 0;
            tnext[a] = INFINITY;
            tdelta[a] = INFINITY;
        }
    }
    double t = 0.0, sum = 0.0;
    for (;;) {
        int a = 0;
        if (tnext[1] < tnext[a]) a = 1;
        if (tnext[2] < tnext[a]) a = 2;
        double tn = tnext[a];
        sum += or_rho(T, lf, c[0], c[1], c[2]) * (tn - t);
        t = tn;
        c[a] += step[a];
        tnext[a] += tdelta[a];
        if (c[a] < 0 || c[a] >= m) break;
    }
    return sum;
}

int or_raymarch(const or_tree *T, int ndir, const double *dirs, int64_t n, const int32_t *lvl,
                const int32_t *ijk, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t t = 0; t < n; ++t) {
        int l0 = lvl[t];
        double dx0 = T->box / (double)((int64_t)1 << l0);
        double x0[3] = {((double)ijk[3 * t] + 0.5) * dx0, ((double)ijk[3 * t + 1] + 0.5) * dx0,
                        ((double)ijk[3 * t + 2] + 0.5) * dx0};
        for (int d = 0; d < ndir; ++d) out[(size_t)t * ndir + d] = march(T, x0, dirs + 3 * d);
    }
    return 0;
}

/* Line integral to the box edge by summing, over every finest cell, density x
 * the ray's length inside it.  O(cells) per ray: tiny grids only. */
int or_raysum_allcells(const or_tree *T, int ndir, const double *dirs, const double *x0, double *out)
{
    int lf = T->lmax;
    int64_t m = (int64_t)1 << lf;
    double h = T->box / (double)m;
    for (int d = 0; d < ndir; ++d) {
        double s = 0.0;
        for (int64_t k = 0; k < m; ++k)
            for (int64_t j = 0; j < m; ++j)
                for (int64_t i = 0; i < m; ++i) {
                    double lo[3] = {(double)i * h, (double)j * h, (double)k * h};
                    double len = or_ray_cube(x0, dirs + 3 * d, lo, h);
                    if (len > 0.0) s += or_rho(T, lf, i, j, k) * len;
                }
        out[d] = s;
    }
    return 0;
}

/* Reference point of the shell at level l for a target at level l0, index
 * (i,j,k): writes its coordinates in box units (cm).  Exposed for the test of
 * the configuration count of §3.3. */
void or_pref(double box, int l0, int64_t i, int64_t j, int64_t k, int l, int mode, double *p)
{
    int r = (mode == OR_MODE_INSITU) ? (l0 - 1) : ((l + 2 < l0 - 1) ? l + 2 : l0 - 1);
    double dxr = box / (double)((int64_t)1 << r);
    p[0] = ((double)(i >> (l0 - r)) + 0.5) * dxr;
    p[1] = ((double)(j >> (l0 - r)) + 0.5) * dxr;
    p[2] = ((double)(k >> (l0 - r)) + 0.5) * dxr;
}

int or_tree_levels(const or_tree *T, int *base, int *lmax)
{
    *base = T->base;
    *lmax = T->lmax;
    return 0;
}

/* Batched lookup of volume-mean densities (for tests). */
void or_rho_many(const or_tree *T, int64_t n, const int32_t *lvl, const int32_t *ijk, double *out)
{
    for (int64_t x = 0; x < n; ++x) out[x] = or_rho(T, lvl[x], ijk[3 * x], ijk[3 * x + 1], ijk[3 * x + 2]);
}
