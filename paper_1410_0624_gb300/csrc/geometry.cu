// Direction sets (§3.2) and the precalculation module of §3.3: the geometric
// factors K of Eq. N_discret, computed once in FP64 on the device.
//
// Stencil frame.  A shell of level l is handled per ancestor P = A_{l-1} of the
// target: its 3x3x3 level-(l-1) neighbourhood is 6x6x6 level-l cells, numbered
// s = a + 6 b + 36 c with (a, b, c) in [0,6)^3 and unit cubes [a, a+1] x ...
// (units of dx_l, origin 2 (P - 1)).  The child of P on the target's path,
// A_l, sits at (2 + ox, 2 + oy, 2 + oz) for its octant o.
//
// Table t (t = 1, 2, 3) serves the cell A_k, k = l + t - 1, that receives the
// shell sum.  Its configuration index is the Morton tail of A_k,
//   cfg = sum_{j=0}^{t-1} oct(A_{k-j}) 8^j,
// i.e. the octants of A_l (most significant) .. A_k (least significant).
// The ray origin is the centre of A_k:
//   p = 2 + sum_{j=0}^{t-1} o(A_{l+j}) 2^-j + 2^-t   (per axis).
// Under the two-level approximation A_k = A_{min(l+2, l0-1)}, so t = 1, 2, 3
// are the shells l0-1, l0-2 and l <= l0-3 (exact for the first three, §3.3).
// Inner region (cells with K = 0): A_l alone for t = 1 (the first shell's inner
// limit is the oct, §3.2 "central region"); the 3x3x3 level-l block around A_l
// for t >= 2 (the previous shell's outer limit).
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "geom_device.cuh"

namespace cd {

// ---- directions (host) --------------------------------------------------------

static void unit(double *v)
{
    for (int a = 0; a < 3; ++a)
        if (fabs(v[a]) < 1e-14) v[a] = 0.0;
    const double n = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= n;
    v[1] /= n;
    v[2] /= n;
}

static void polar(double cos_theta, double phi, double *v)
{
    const double st = sqrt(fmax(0.0, 1.0 - cos_theta * cos_theta));
    v[0] = st * cos(phi);
    v[1] = st * sin(phi);
    v[2] = cos_theta;
    unit(v);
}

int make_directions(int scheme, int p0, int p1, const double *custom, int n_custom, double *out)
{
    int n = 0;
    switch (scheme) {
    case CD_DIRS_HEALPIX: {
        // Gorski et al. (2005), ring scheme: rings r = 1 .. 4 Nside - 1.
        const int ns = p0;
        if (ns < 1 || 12 * ns * ns > CD_MAXDIR) return -1;
        for (int r = 1; r < 4 * ns; ++r) {
            const bool north = r < ns, south = r > 3 * ns;
            if (north || south) {
                const int q = north ? r : 4 * ns - r;
                double z = 1.0 - (double)(q * q) / (3.0 * ns * ns);
                if (south) z = -z;
                for (int j = 0; j < 4 * q; ++j, ++n)
                    polar(z, (M_PI / 2.0) * (j + 0.5) / q, out + 3 * n);
            } else {
                const double z = (4.0 * ns - 2.0 * r) / (3.0 * ns);
                const double shift = ((r - ns) & 1) ? 0.0 : 0.5;  // odd rings offset by half a pixel
                for (int j = 0; j < 4 * ns; ++j, ++n)
                    polar(z, (M_PI / 2.0) * (j + 1 - shift) / ns, out + 3 * n);
            }
        }
        return n;
    }
    case CD_DIRS_MXN: {
        const int M = p0, N = p1;
        if (M < 1 || N < 1 || (int64_t)M * N > CD_MAXDIR) return -1;
        for (int m = 1; m <= M; ++m)
            for (int k = 1; k <= N; ++k, ++n)
                polar(1.0 - (2.0 * m - 1.0) / M, 2.0 * M_PI * (k - 1) / N, out + 3 * n);
        return n;
    }
    case CD_DIRS_AXES: {
        const double a[18] = {1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1, 0, 0, 0, 1, 0, 0, -1};
        memcpy(out, a, sizeof(a));
        return 6;
    }
    case CD_DIRS_CUSTOM: {
        if (!custom || n_custom < 1 || n_custom > CD_MAXDIR) return -1;
        for (int i = 0; i < n_custom; ++i) {
            double v[3] = {custom[3 * i], custom[3 * i + 1], custom[3 * i + 2]};
            const double l = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            if (!(l > 0.0) || !isfinite(l)) return -1;
            v[0] /= l;
            v[1] /= l;
            v[2] /= l;
            unit(v);
            memcpy(out + 3 * i, v, sizeof(v));
        }
        return n_custom;
    }
    default:
        return -1;
    }
}

// Sub-rays of a direction's cone.  Direction d stands for a bin of 4 pi / nd
// steradians (§3.2: equal solid angles); its cone is the circular cap of that
// solid angle around u, cos(alpha) = 1 - 2 / nd.  The cap is cut into
// CD_CONE_RINGS bands of equal solid angle (equal steps in cos theta) and each
// band into CD_CONE_AZ equal sectors; sub-ray (r, j) goes through the middle of
// its piece: cos theta = 1 - (r + 1/2) (1 - cos alpha) / CD_CONE_RINGS,
// phi = 2 pi (j + 1/2 if r is odd) / CD_CONE_AZ, around the frame
// e1 = unit(e_a x u) (a: the first axis whose |u_a| is within 1e-9 of the
// smallest, so that a tie such as |u_x| = |u_y| picks the same axis whatever
// the last bit of u), e2 = u x e1.  The pieces have equal solid angle, so a cone average is the
// plain mean over the sub-rays.
void make_cone_rays(const double *dirs, int nd, double *out)
{
    const double cos_a = 1.0 - 2.0 / (double)nd;
    const int ns = CD_CONE_RINGS * CD_CONE_AZ;
    for (int d = 0; d < nd; ++d) {
        const double *u = dirs + 3 * d;
        const double amin = fmin(fabs(u[0]), fmin(fabs(u[1]), fabs(u[2])));
        int ax = 0;
        while (ax < 2 && !(fabs(u[ax]) <= amin + 1e-9)) ++ax;
        // e1 = e_ax x u, normalised; e2 = u x e1
        double e1[3] = {0.0, 0.0, 0.0};
        const int a1 = (ax + 1) % 3, a2 = (ax + 2) % 3;
        e1[a1] = -u[a2];
        e1[a2] = u[a1];
        const double n1 = sqrt(e1[a1] * e1[a1] + e1[a2] * e1[a2]);
        e1[a1] /= n1;
        e1[a2] /= n1;
        const double e2[3] = {u[1] * e1[2] - u[2] * e1[1], u[2] * e1[0] - u[0] * e1[2], u[0] * e1[1] - u[1] * e1[0]};
        for (int r = 0; r < CD_CONE_RINGS; ++r) {
            const double c = 1.0 - (r + 0.5) * (1.0 - cos_a) / CD_CONE_RINGS;
            const double sn = sqrt(fmax(0.0, 1.0 - c * c));
            for (int j = 0; j < CD_CONE_AZ; ++j) {
                const double phi = 2.0 * M_PI * (j + 0.5 * (r & 1)) / CD_CONE_AZ;
                const double cp = cos(phi), sp = sin(phi);
                double *v = out + 3 * ((size_t)d * ns + r * CD_CONE_AZ + j);
                for (int a = 0; a < 3; ++a) v[a] = c * u[a] + sn * (cp * e1[a] + sp * e2[a]);
                unit(v);
            }
        }
    }
}

// ---- FP64 geometry (device) ------------------------------------------------------

namespace {

// Sparse table t: the non-zero weights of every (cfg, d), averaged over the ns
// rays of direction d (rays[d][0 .. ns-1]).  With tab == NULL only the counts
// are taken (the table width maxe is not known before).
__global__ void shell_tables(int t, int nd, const double *__restrict__ rays, int ns, int2 *__restrict__ tab, int maxe,
                             int *__restrict__ cmax, int *__restrict__ max_count)
{
    const int ncfg = 1 << (3 * t);
    const int R = region_side(t);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncfg * nd; e += gridDim.x * blockDim.x) {
        const int cfg = e / nd, d = e - cfg * nd;
        const double *u = rays + (size_t)3 * ns * d;
        int2 *row = tab ? tab + (size_t)cfg * maxe * nd + d : nullptr;
        int n = 0;
        for (int s = 0; s < CD_STENCIL; ++s) {
            const double len = shell_weight_avg(t, cfg, s, u, ns);
            if (len > 0.0) {
                const int a = s % 6, b = (s / 6) % 6, c = s / 36;
                if (row && n < maxe) row[(size_t)n * nd] = make_int2(a + R * (b + R * c), __float_as_int((float)len));
                ++n;
            }
        }
        if (row) {
            for (int m = n; m < maxe; ++m) row[(size_t)m * nd] = make_int2(0, 0);
            atomicMax(&cmax[cfg], n < maxe ? n : maxe);
        }
        atomicMax(max_count, n);
    }
}

// Kloc[t][s][d]: ray from the centre of child t of an oct through child s,
// in units of the child size (internal contribution for s = t, local otherwise).
// (averaged over the ns rays of each direction, as the shell tables)
__global__ void local_table(int nd, const double *__restrict__ rays, int ns, float *__restrict__ kloc)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * nd; e += gridDim.x * blockDim.x) {
        const int ts = e / nd, d = e - ts * nd;
        const int t = ts >> 3, s = ts & 7;
        const double p[3] = {(t & 1) + 0.5, ((t >> 1) & 1) + 0.5, ((t >> 2) & 1) + 0.5};
        double acc = 0.0;
        for (int j = 0; j < ns; ++j)
            acc += path_in_cube(p, rays + 3 * ((size_t)ns * d + j), s & 1, (s >> 1) & 1, (s >> 2) & 1);
        kloc[e] = (float)(acc / ns);
    }
}

}  // namespace

cd_status build_geometry_tables(cd_geom g, cudaStream_t s)
{
    const int nd = g->n_dir, ns = g->n_sub;
    int *d_max = nullptr;
    CD_CUDA(cudaMallocAsync(&d_max, sizeof(int), s));
    CD_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), s));
    // pass 1: the largest non-zero count fixes the table width
    for (int t = 1; t <= 3; ++t) {
        const int n = (1 << (3 * t)) * nd;
        LaunchScope ls(CD_K_OTHER, s);
        shell_tables<<<(n + 127) / 128, 128, 0, s>>>(t, nd, g->rays_dev, ns, nullptr, 0, nullptr, d_max);
        CD_CHECK_LAUNCH();
    }
    int hmax = 0;
    CD_CUDA(cudaMemcpyAsync(&hmax, d_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    const int maxe = hmax > 0 ? hmax : 1;
    for (int t = 1; t <= 3; ++t) {
        const size_t ncfg = (size_t)1 << (3 * t);
        if (cudaMalloc(&g->tab[t], ncfg * maxe * nd * sizeof(int2)) != cudaSuccess ||
            cudaMalloc(&g->cmax[t], ncfg * sizeof(int)) != cudaSuccess) {
            cudaGetLastError();
            cudaFreeAsync(d_max, s);
            set_error("cannot allocate the shell tables (%d entries per row)", maxe);
            return CD_ENOMEM;
        }
    }
    g->maxe = maxe;
    // pass 2: the entries
    CD_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), s));
    for (int t = 1; t <= 3; ++t) {
        const int n = (1 << (3 * t)) * nd;
        CD_CUDA(cudaMemsetAsync(g->cmax[t], 0, sizeof(int) << (3 * t), s));
        LaunchScope ls(CD_K_OTHER, s);
        shell_tables<<<(n + 127) / 128, 128, 0, s>>>(t, nd, g->rays_dev, ns, g->tab[t], maxe, g->cmax[t], d_max);
        CD_CHECK_LAUNCH();
    }
    {
        LaunchScope ls(CD_K_OTHER, s);
        local_table<<<(64 * nd + 127) / 128, 128, 0, s>>>(nd, g->rays_dev, ns, g->kloc);
    }
    CD_CHECK_LAUNCH();
    int hmax2 = 0;
    CD_CUDA(cudaMemcpyAsync(&hmax2, d_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    CD_CUDA(cudaFreeAsync(d_max, s));
    if (hmax2 != hmax) {
        set_error("shell table counts changed between passes (%d, %d)", hmax, hmax2);
        return CD_ECUDA;
    }
    return CD_OK;
}

}  // namespace cd
