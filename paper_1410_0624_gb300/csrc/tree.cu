// Tree construction for a uniform leaf grid: Morton-ordered leaf densities and
// every coarse level as the volume mean of its eight children (§3 intro: octs
// of 2^3 cells; §3.2: the density of a coarse cell "corresponds to a mean").
//
// Layout in HBM
//   rho_leaf            n_leaf floats, Morton depth-first order (8 siblings contiguous)
//   rho_lvl[l], l < L   (2^l)^3 floats, row-major (x fastest): dense levels are
//                       addressed by stencil offsets in the shell kernels
//   rho_brick[l]        BF16 copy of level l in brick order: the 8 children of
//                       level-(l-1) cell p (row-major) at [8p .. 8p+7], octant order
#include "common.cuh"

namespace cd {
namespace {

// Each block takes a B x B x B patch of one dense level m (B = 2^b <= 8, one
// thread per cell) and reduces it b times inside shared memory: at every
// reduction the cells of level m-1 in the patch take the mean of their 8
// children (summed in octant order, then x 1/8) and the children are written
// as the BF16 brick of their parent.  So one launch writes b coarser levels and
// b brick levels, where separate launches per level cost mostly launch time.
//   top != 0: level m is L - 1 and each thread first reads its 8 leaves from the
//   row-major input, writes them to the Morton leaf array and their mean to m.
struct PatchPtrs {
    float *lvl[CD_MAXL + 1];
    __nv_bfloat16 *brick[CD_MAXL + 1];
};

template <bool top>
__global__ void __launch_bounds__(512) restrict_patch(const float *__restrict__ in, int m, int b,
                                                      float *__restrict__ leaf, const __grid_constant__ PatchPtrs P)
{
    __shared__ float s_val[2][512];
    const int B = 1 << b;
    const int t = threadIdx.x;
    const int64_t nm = (int64_t)1 << m;                                   // cells per axis at level m
    const int64_t nb = nm >> b;                                           // patches per axis
    const int64_t bx = blockIdx.x % nb, by = (blockIdx.x / nb) % nb, bz = blockIdx.x / (nb * nb);
    if (t < B * B * B) {
        const int tx = t & (B - 1), ty = (t >> b) & (B - 1), tz = t >> (2 * b);
        const int64_t x = bx * B + tx, y = by * B + ty, z = bz * B + tz;
        float v;
        if (top) {
            const int64_t nl = nm * 2;
            float c[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int64_t cx = 2 * x + (o & 1), cy = 2 * y + ((o >> 1) & 1), cz = 2 * z + ((o >> 2) & 1);
                c[o] = in[(cz * nl + cy) * nl + cx];
            }
            float sum = 0.f;
#pragma unroll
            for (int o = 0; o < 8; ++o) sum += c[o];
            v = sum * 0.125f;
            float4 *dst = reinterpret_cast<float4 *>(leaf + 8 * morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
            dst[0] = make_float4(c[0], c[1], c[2], c[3]);
            dst[1] = make_float4(c[4], c[5], c[6], c[7]);
            P.lvl[m][(z * nm + y) * nm + x] = v;
        } else {
            v = P.lvl[m][(z * nm + y) * nm + x];
        }
        s_val[0][t] = v;
    }
    __syncthreads();
    int cur = 0;
    for (int r = 0, n = B; r < b; ++r, n >>= 1) {
        const int h = n >> 1, lh = b - r - 1;                             // parent patch edge 2^lh
        const int lc = m - r;                                             // child level
        if (t < h * h * h) {
            const int px = t & (h - 1), py = (t >> lh) & (h - 1), pz = t >> (2 * lh);
            __align__(16) __nv_bfloat16 bv[8];
            float sum = 0.f;
#pragma unroll
            for (int o = 0; o < 8; ++o) {
                const int cx = 2 * px + (o & 1), cy = 2 * py + ((o >> 1) & 1), cz = 2 * pz + ((o >> 2) & 1);
                const float c = s_val[cur][(cz * n + cy) * n + cx];
                sum += c;
                bv[o] = __float2bfloat16_rn(c);
            }
            const float v = sum * 0.125f;
            const int64_t np = (int64_t)1 << (lc - 1);
            const int64_t gx = (bx * B >> (r + 1)) + px, gy = (by * B >> (r + 1)) + py, gz = (bz * B >> (r + 1)) + pz;
            const int64_t gp = (gz * np + gy) * np + gx;
            P.lvl[lc - 1][gp] = v;
            *reinterpret_cast<uint4 *>(P.brick[lc] + 8 * gp) = *reinterpret_cast<const uint4 *>(bv);
            s_val[cur ^ 1][t] = v;
        }
        __syncthreads();
        cur ^= 1;
    }
}

PatchPtrs patch_ptrs(cd_tree t)
{
    PatchPtrs P;
    for (int l = 0; l <= CD_MAXL; ++l) {
        P.lvl[l] = t->rho_lvl[l];
        P.brick[l] = t->rho_brick[l];
    }
    return P;
}

// Patches of level m down to level 0: each launch reduces min(3, m) levels.
cd_status restrict_from(cd_tree t, int m, cudaStream_t s)
{
    const PatchPtrs P = patch_ptrs(t);
    while (m >= 1) {
        const int b = m < 3 ? m : 3;
        const int64_t nb = (int64_t)1 << (m - b);
        LaunchScope ls(CD_K_RESTRICT, s);
        restrict_patch<false><<<(unsigned)(nb * nb * nb), 1 << (3 * b), 0, s>>>(nullptr, m, b, nullptr, P);
        CD_CHECK_LAUNCH();
        m -= b;
    }
    return CD_OK;
}

}  // namespace

// Leaves -> level L-1 (and the Morton leaf array) in the same launch as the
// first reductions, then the coarser levels.
cd_status restrict_uniform(cd_tree t, const float *rho_dev, cudaStream_t s)
{
    const int L = t->L, m = L - 1;
    const int b = m < 3 ? m : 3;
    const int64_t nb = (int64_t)1 << (m - b);
    {
        LaunchScope ls(CD_K_RESTRICT, s);
        restrict_patch<true><<<(unsigned)(nb * nb * nb), 1 << (3 * b), 0, s>>>(rho_dev, m, b, t->rho_leaf,
                                                                             patch_ptrs(t));
    }
    CD_CHECK_LAUNCH();
    return restrict_from(t, m - b, s);
}

cd_status restrict_dense(cd_tree t, int top, cudaStream_t s)
{
    return restrict_from(t, top, s);
}

}  // namespace cd
