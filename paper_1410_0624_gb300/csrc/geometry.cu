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

// ---- FP64 geometry (device) ------------------------------------------------------

namespace {

__global__ void shell_tables(int t, int nd, const double *__restrict__ dirs, int2 *__restrict__ tab,
                             int *__restrict__ cmax, int *__restrict__ max_count)
{
    const int ncfg = 1 << (3 * t);
    const int R = region_side(t);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ncfg * nd; e += gridDim.x * blockDim.x) {
        const int cfg = e / nd, d = e - cfg * nd;
        const double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
        int2 *row = tab + (size_t)cfg * CD_MAXE * nd + d;
        int n = 0;
        for (int s = 0; s < CD_STENCIL; ++s) {
            const double len = shell_weight(t, cfg, s, u);
            if (len > 0.0) {
                const int a = s % 6, b = (s / 6) % 6, c = s / 36;
                if (n < CD_MAXE) row[(size_t)n * nd] = make_int2(a + R * (b + R * c), __float_as_int((float)len));
                ++n;
            }
        }
        for (int m = n; m < CD_MAXE; ++m) row[(size_t)m * nd] = make_int2(0, 0);
        atomicMax(&cmax[cfg], n < CD_MAXE ? n : CD_MAXE);
        atomicMax(max_count, n);
    }
}

// Kloc[t][s][d]: ray from the centre of child t of an oct through child s,
// in units of the child size (internal contribution for s = t, local otherwise).
__global__ void local_table(int nd, const double *__restrict__ dirs, float *__restrict__ kloc)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 64 * nd; e += gridDim.x * blockDim.x) {
        const int ts = e / nd, d = e - ts * nd;
        const int t = ts >> 3, s = ts & 7;
        const double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
        const double p[3] = {(t & 1) + 0.5, ((t >> 1) & 1) + 0.5, ((t >> 2) & 1) + 0.5};
        kloc[e] = (float)path_in_cube(p, u, s & 1, (s >> 1) & 1, (s >> 2) & 1);
    }
}

}  // namespace

cd_status build_geometry_tables(cd_geom g, cudaStream_t s)
{
    const int nd = g->n_dir;
    int *d_max = nullptr;
    CD_CUDA(cudaMallocAsync(&d_max, sizeof(int), s));
    CD_CUDA(cudaMemsetAsync(d_max, 0, sizeof(int), s));
    for (int t = 1; t <= 3; ++t) {
        const int n = (1 << (3 * t)) * nd;
        CD_CUDA(cudaMemsetAsync(g->cmax[t], 0, sizeof(int) << (3 * t), s));
        LaunchScope ls(CD_K_OTHER, s);
        shell_tables<<<(n + 127) / 128, 128, 0, s>>>(t, nd, g->dirs_dev, g->tab[t], g->cmax[t], d_max);
        CD_CHECK_LAUNCH();
    }
    {
        LaunchScope ls(CD_K_OTHER, s);
        local_table<<<(64 * nd + 127) / 128, 128, 0, s>>>(nd, g->dirs_dev, g->kloc);
    }
    CD_CHECK_LAUNCH();
    int hmax = 0;
    CD_CUDA(cudaMemcpyAsync(&hmax, d_max, sizeof(int), cudaMemcpyDeviceToHost, s));
    CD_CUDA(cudaStreamSynchronize(s));
    CD_CUDA(cudaFreeAsync(d_max, s));
    g->max_entries = hmax;
    if (hmax > CD_MAXE) {
        set_error("a ray crosses %d stencil cells, more than the %d the tables hold", hmax, CD_MAXE);
        return CD_EINVAL;
    }
    return CD_OK;
}

}  // namespace cd
