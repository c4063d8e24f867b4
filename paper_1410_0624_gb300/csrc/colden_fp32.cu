// FP32 CUDA-core form of the shell contraction (Eq. N_discret, one level of
// receiving cells per launch).  For every cell c at level k and direction d:
//   out[c][d] = prefix_in[parent(c)][d]
//             + sum_{t in tmask} dx_{k-t+1} sum_s rho_{k-t+1}(stencil_t(c), s) K_t[cfg_t(c)][d][s]
// with the 6^3 stencil of table t anchored at the ancestor A_{k-t} of c and
// cfg_t(c) the Morton tail of c (geometry.cu).
//
// One CTA takes the 8^span descendants of one level-q cell (q = k - span,
// span <= 3, smaller on coarse levels so that every launch has at least two
// CTAs per SM): a Morton-contiguous run, so the output rows are written
// coalesced.  The
// density regions its stencils touch (at most 12^3, 8^3 and 6^3 cells for
// tables 1, 2, 3) are staged once in shared memory, zero outside the box
// (§3.2: the shells stop at the box border).  Lanes walk consecutive (cell,
// direction) pairs; the sparse weights are stored [cfg][entry][direction] as
// {shared-memory offset, weight} pairs, so a warp's loads of one entry are
// contiguous, and each (cfg) row is walked to the largest non-zero count of
// its directions (padding entries have weight 0).
#include "common.cuh"

namespace cd {
namespace {

constexpr int kExtThreads = 256;

struct ExtArgs {
    ExtLaunch a;
    int span;
    const int2 *tab[4];
    const int *cmax[4];
    int maxe;           // entries per table row
};

__global__ void __launch_bounds__(kExtThreads) shell_sum_fp32(ExtArgs P)
{
    __shared__ float s_rho[kRegionTotal];

    const int k = P.a.k, nd = P.a.nd;
    const int span = P.span;                                  // levels below the CTA root
    const uint64_t root = blockIdx.x;                         // Morton index at level k - span
    const uint32_t Qx = compact3(root), Qy = compact3(root >> 1), Qz = compact3(root >> 2);

    // stage the density regions (level k - t + 1, origin 2 (P_min - 1))
    for (int t = 1; t <= 3; ++t) {
        if (!(P.a.tmask & (1 << (t - 1)))) continue;
        const int l = k - t + 1;
        const int64_t n = (int64_t)1 << l;
        // ancestors A_{k-t} of the CTA's cells: nP per axis from P_min
        const int nP = span >= t ? 1 << (span - t) : 1;
        const int ext = 2 * nP + 4, R = region_side(t);
        const int64_t ox = 2 * ((((int64_t)Qx << span) >> t) - 1), oy = 2 * ((((int64_t)Qy << span) >> t) - 1),
                      oz = 2 * ((((int64_t)Qz << span) >> t) - 1);
        const float *rho = P.a.rho[t];
        for (int r = threadIdx.x; r < R * R * R; r += blockDim.x) {
            const int rx = r % R, ry = (r / R) % R, rz = r / (R * R);
            const int64_t gx = ox + rx, gy = oy + ry, gz = oz + rz;
            float v = 0.f;
            if (rx < ext && ry < ext && rz < ext && gx >= 0 && gy >= 0 && gz >= 0 && gx < n && gy < n && gz < n)
                v = rho[(gz * n + gy) * n + gx];
            s_rho[region_base(t) + r] = v;
        }
    }
    __syncthreads();

    const int ncell = 1 << (3 * span);
    const uint64_t first = root << (3 * span);
    for (int p = threadIdx.x; p < ncell * nd; p += blockDim.x) {
        const int j = p / nd, d = p - j * nd;
        const uint64_t m = first + (uint64_t)j;
        const uint32_t cx = compact3((uint64_t)j), cy = compact3((uint64_t)j >> 1), cz = compact3((uint64_t)j >> 2);
        float acc = P.a.prefix_in && in_bounds((long long)(m >> 3), 1ll << (3 * (k - 1)), kCheckFp32Prefix)
                        ? P.a.prefix_in[(m >> 3) * nd + d]
                        : 0.f;
#pragma unroll
        for (int t = 1; t <= 3; ++t) {
            if (!(P.a.tmask & (1 << (t - 1)))) continue;
            const int R = region_side(t);
            // stencil origin of A_{k-t} relative to the staged region
            const int ax = span >= t ? 2 * (cx >> t) : 0, ay = span >= t ? 2 * (cy >> t) : 0,
                      az = span >= t ? 2 * (cz >> t) : 0;
            const int anchor = region_base(t) + ax + R * (ay + R * az);
            const int cfg = (int)(m & ((1u << (3 * t)) - 1));
            const int2 *row = P.tab[t] + (size_t)cfg * P.maxe * nd + d;
            const int n = P.cmax[t][cfg];
            float part = 0.f;
            for (int e = 0; e < n; ++e) {
                const int2 v = row[(size_t)e * nd];
                if (in_bounds(anchor + v.x - region_base(t), R * R * R, kCheckFp32Region))
                    part = fmaf(s_rho[anchor + v.x], __int_as_float(v.y), part);
            }
            acc = fmaf(P.a.dx[t], part, acc);
        }
        if (in_bounds((long long)m, 1ll << (3 * k), kCheckFp32Out)) P.a.out[m * nd + d] = acc;
    }
}

}  // namespace

cd_status launch_ext_fp32(const ExtLaunch &a, cd_geom g, cudaStream_t s)
{
    ExtArgs P;
    P.a = a;
    // largest span <= min(3, k) that still gives >= 304 CTAs (2 per SM)
    int span = a.k < 3 ? a.k : 3;
    while (span > 0 && (1ull << (3 * (a.k - span))) < 304ull) --span;
    P.span = span;
    for (int t = 0; t < 4; ++t) {
        P.tab[t] = g->tab[t];
        P.cmax[t] = g->cmax[t];
    }
    P.maxe = g->maxe;
    const uint64_t nblk = 1ull << (3 * (a.k - span));
    LaunchScope ls(CD_K_SHELL, s);
    shell_sum_fp32<<<(unsigned)nblk, kExtThreads, 0, s>>>(P);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

}  // namespace cd
