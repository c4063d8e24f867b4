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

// A block takes a B x B x B patch of level m-1 (B = 2^b <= 8), one thread per
// cell: each thread reads its 8 children at level m (the row-major leaves when
// top, else dense level m), writes their mean (summed in octant order, then
// x 1/8) and, below the leaves, the children as the cell's BF16 brick of level
// m.  The patch is then reduced b more times in shared memory, writing levels
// m-2 .. m-1-b and bricks m-1 .. m-b.  One launch thus writes b + 1 levels;
// per-level launches cost mostly launch time on the small levels.
//   top: the children are the leaves; their Morton-order copy is written too.
struct PatchPtrs {
    float *lvl[CD_MAXL + 1];
    __nv_bfloat16 *brick[CD_MAXL + 1];
};

template <bool top>
__global__ void __launch_bounds__(512) restrict_patch(const float *__restrict__ in, int m, int b, int vec2,
                                                      float *__restrict__ leaf, const __grid_constant__ PatchPtrs P)
{
    __shared__ float s_val[2][512];
    const int B = 1 << b;
    const int t = threadIdx.x;
    const int64_t np = (int64_t)1 << (m - 1);                             // cells per axis at level m-1
    const int64_t nb = np >> b;                                           // patches per axis
    const int64_t bx = blockIdx.x % nb, by = (blockIdx.x / nb) % nb, bz = blockIdx.x / (nb * nb);
    if (t < B * B * B) {
        const int tx = t & (B - 1), ty = (t >> b) & (B - 1), tz = t >> (2 * b);
        const int64_t x = bx * B + tx, y = by * B + ty, z = bz * B + tz;
        const int64_t nc = np * 2;
        const float *src = top ? in : P.lvl[m];
        float c[8];
#pragma unroll
        for (int o = 0; o < 8; o += 2) {
            const int64_t cy = 2 * y + ((o >> 1) & 1), cz = 2 * z + ((o >> 2) & 1);
            const float *row = src + (cz * nc + cy) * nc + 2 * x;
            if (vec2) {                           // the input is 8-byte aligned
                const float2 pr = *reinterpret_cast<const float2 *>(row);
                c[o] = pr.x;
                c[o + 1] = pr.y;
            } else {
                c[o] = row[0];
                c[o + 1] = row[1];
            }
        }
        float sum = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) sum += c[o];
        const float v = sum * 0.125f;
        const int64_t gp = (z * np + y) * np + x;
        P.lvl[m - 1][gp] = v;
        if (top) {
            float4 *dst = reinterpret_cast<float4 *>(leaf + 8 * morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
            dst[0] = make_float4(c[0], c[1], c[2], c[3]);
            dst[1] = make_float4(c[4], c[5], c[6], c[7]);
        } else {
            __align__(16) __nv_bfloat16 bv[8];
#pragma unroll
            for (int o = 0; o < 8; ++o) bv[o] = __float2bfloat16_rn(c[o]);
            *reinterpret_cast<uint4 *>(P.brick[m] + 8 * gp) = *reinterpret_cast<const uint4 *>(bv);
        }
        s_val[0][t] = v;
    }
    __syncthreads();
    int cur = 0;
    for (int r = 0, n = B; r < b; ++r, n >>= 1) {
        const int h = n >> 1, lh = b - r - 1;                             // parent patch edge 2^lh
        const int lc = m - 1 - r;                                         // child level
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
            const int64_t npp = (int64_t)1 << (lc - 1);
            const int64_t gx = (bx * B >> (r + 1)) + px, gy = (by * B >> (r + 1)) + py, gz = (bz * B >> (r + 1)) + pz;
            const int64_t gp = (gz * npp + gy) * npp + gx;
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

// Children at level m (the leaves when top): writes levels m-1 .. 0 and bricks
// m-1 .. 1 (and brick m below the leaves), 1 + min(3, m-1) levels per launch.
cd_status restrict_launches(cd_tree t, const float *leaves, int m, cudaStream_t s)
{
    const PatchPtrs P = patch_ptrs(t);
    bool top = leaves != nullptr;
    while (m >= 1) {
        const int b = m - 1 < 3 ? m - 1 : 3;
        const int64_t nb = (int64_t)1 << (m - 1 - b);
        LaunchScope ls(CD_K_RESTRICT, s);
        if (top)
            restrict_patch<true><<<(unsigned)(nb * nb * nb), 1 << (3 * b), 0, s>>>(
                leaves, m, b, ((uintptr_t)leaves & 7) == 0, t->rho_leaf, P);
        else
            restrict_patch<false><<<(unsigned)(nb * nb * nb), 1 << (3 * b), 0, s>>>(nullptr, m, b, 1, nullptr, P);
        CD_CHECK_LAUNCH();
        top = false;
        m -= 1 + b;
    }
    return CD_OK;
}

}  // namespace

cd_status restrict_uniform(cd_tree t, const float *rho_dev, cudaStream_t s)
{
    return restrict_launches(t, rho_dev, t->L, s);
}

cd_status restrict_dense(cd_tree t, int top, cudaStream_t s)
{
    return restrict_launches(t, nullptr, top, s);
}

}  // namespace cd
