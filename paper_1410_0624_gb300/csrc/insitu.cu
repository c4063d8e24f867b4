// The in-situ variant of the tree method (§4.3): every shell is seen from the
// centre of the target's oct, with no precalculated two-level approximation.
//
// From the oct centre p, the shell of level l (the 6^3 level-l cells covering
// the 3^3 block of level l-1 around the ancestor A_{l-1}, minus the inner
// region: the oct itself at l = l0-1, the 3^3 level-l block around A_l below,
// both clipped to the box; Eq. N_discret) meets the ray p + s u (s >= 0) in the
// single segment between the ray's exits from the two nested boxes, since
// both contain p.  The contribution sum_i n_i dx_i of the shell is therefore
// the line integral of the level-l density over that segment, which a short
// cell-by-cell walk (DDA) over the level-l grid computes exactly: each
// crossing is recomputed from its cell face, so nothing accumulates.  One
// thread per (oct, direction) sums the shells of every level into the oct's
// external column E; the leaf kernels add the internal and local terms as in
// the precalculated form.
#include <algorithm>

#include "common.cuh"

namespace cd {
namespace {

struct InsituArgs {
    int64_t n;               // octs
    const uint64_t *keys;    // Morton keys of the octs at level k, or NULL: octs 0 .. n-1
    int k;                   // level of the octs (their children are the leaves, l0 = k + 1)
    int nd;
    const double *dirs;      // [nd][3]
    const float *lvl[CD_MAXL + 1];   // dense row-major volume means of levels 0 .. k
    float box;               // cm
    float *out;              // [n][nd], cm^-2
};

// exit distance of the ray p + s u from the box [lo, hi] (which contains p)
__device__ __forceinline__ float box_exit(const float p[3], const float u[3], const float inv[3], const float lo[3],
                                          const float hi[3])
{
    float t = INFINITY;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (u[a] > 0.f) t = fminf(t, (hi[a] - p[a]) * inv[a]);
        else if (u[a] < 0.f) t = fminf(t, (lo[a] - p[a]) * inv[a]);
    }
    return t;
}

__global__ void __launch_bounds__(256) insitu_external(InsituArgs A)
{
    const int nd = A.nd;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < A.n * nd;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = e / nd;
        const int d = (int)(e - o * nd);
        const uint64_t key = A.keys ? A.keys[o] : (uint64_t)o;
        const int k = A.k;
        const int oc[3] = {(int)compact3(key), (int)compact3(key >> 1), (int)compact3(key >> 2)};
        float u[3], inv[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            u[a] = (float)A.dirs[3 * d + a];
            inv[a] = u[a] != 0.f ? 1.f / u[a] : 0.f;
        }
        // coordinates in units of the box; the oct centre
        const float hk = 1.f / (float)(1 << k);
        const float p[3] = {((float)oc[0] + 0.5f) * hk, ((float)oc[1] + 0.5f) * hk, ((float)oc[2] + 0.5f) * hk};
        float total = 0.f;
        for (int l = k; l >= 1; --l) {
            const int n = 1 << l;
            const float h = 1.f / (float)n;
            int al[3], am[3];
            float olo[3], ohi[3], ilo[3], ihi[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                al[a] = oc[a] >> (k - l);        // A_l
                am[a] = al[a] >> 1;              // A_{l-1}
                olo[a] = (float)max(2 * (am[a] - 1), 0) * h;
                ohi[a] = (float)min(2 * (am[a] + 2), n) * h;
                if (l == k) {
                    ilo[a] = (float)al[a] * h;
                    ihi[a] = (float)(al[a] + 1) * h;
                } else {
                    ilo[a] = (float)max(al[a] - 1, 0) * h;
                    ihi[a] = (float)min(al[a] + 2, n) * h;
                }
            }
            const float t0 = box_exit(p, u, inv, ilo, ihi), t1 = box_exit(p, u, inv, olo, ohi);
            if (!(t1 > t0)) continue;
            // first cell: the one the ray enters at t0
            int c[3], step[3];
            float tnext[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float q = (p[a] + t0 * u[a]) * (float)n;
                if (u[a] > 0.f) {
                    c[a] = (int)floorf(q);
                    step[a] = 1;
                } else if (u[a] < 0.f) {
                    c[a] = (int)ceilf(q) - 1;
                    step[a] = -1;
                } else {
                    c[a] = (int)floorf(q);
                    step[a] = 0;
                }
                c[a] = min(max(c[a], 0), n - 1);
                tnext[a] = step[a] ? ((float)(c[a] + (step[a] > 0)) * h - p[a]) * inv[a] : INFINITY;
            }
            const float *rho = A.lvl[l];
            float t = t0, sum = 0.f;
            for (int it = 0; it < 24 && t < t1; ++it) {
                int a = 0;
                if (tnext[1] < tnext[a]) a = 1;
                if (tnext[2] < tnext[a]) a = 2;
                const float tn = fminf(tnext[a], t1);
                sum = fmaf(rho[((int64_t)c[2] * n + c[1]) * n + c[0]], tn - t, sum);
                t = tn;
                c[a] += step[a];
                if (c[a] < 0 || c[a] >= n) break;
                tnext[a] = ((float)(c[a] + (step[a] > 0)) * h - p[a]) * inv[a];
            }
            total += sum;
        }
        A.out[e] = total * A.box;
    }
}

}  // namespace

cd_status launch_insitu(cd_tree t, cd_geom g, int k, int64_t n, const uint64_t *keys, float *out, cudaStream_t s)
{
    if (n == 0) return CD_OK;
    InsituArgs A = {};
    A.n = n;
    A.keys = keys;
    A.k = k;
    A.nd = g->n_dir;
    A.dirs = g->dirs_dev;
    for (int l = 0; l <= k && l <= CD_MAXL; ++l) A.lvl[l] = t->rho_lvl[l];
    A.box = (float)t->box_cm;
    A.out = out;
    const int64_t blocks = std::min<int64_t>((n * g->n_dir + 255) / 256, 152 * 32);
    LaunchScope ls(CD_K_SHELL, s);
    insitu_external<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(A);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

}  // namespace cd
