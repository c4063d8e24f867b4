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

// One thread per level-(L-1) cell: reads its 8 leaves from the row-major input,
// writes them to the Morton leaf array and their mean to level L-1.
__global__ void restrict_from_leaves(const float *__restrict__ in, int L, float *__restrict__ leaf,
                                     float *__restrict__ parent)
{
    const int64_t np = (int64_t)1 << (L - 1);
    const int64_t total = np * np * np;
    const int64_t nl = np * 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t x = (uint32_t)(p % np), y = (uint32_t)((p / np) % np), z = (uint32_t)(p / (np * np));
        float c[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int64_t cx = 2 * x + (o & 1), cy = 2 * y + ((o >> 1) & 1), cz = 2 * z + ((o >> 2) & 1);
            c[o] = in[(cz * nl + cy) * nl + cx];
        }
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) s += c[o];
        parent[p] = s * 0.125f;
        float4 *dst = reinterpret_cast<float4 *>(leaf + 8 * morton3(x, y, z));
        dst[0] = make_float4(c[0], c[1], c[2], c[3]);
        dst[1] = make_float4(c[4], c[5], c[6], c[7]);
    }
}

// One thread per level-(l-1) cell: mean of its 8 children at level l.
__global__ void restrict_level(const float *__restrict__ child, int l, float *__restrict__ parent)
{
    const int64_t np = (int64_t)1 << (l - 1);
    const int64_t total = np * np * np;
    const int64_t nc = np * 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = p % np, y = (p / np) % np, z = p / (np * np);
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int64_t cx = 2 * x + (o & 1), cy = 2 * y + ((o >> 1) & 1), cz = 2 * z + ((o >> 2) & 1);
            s += child[(cz * nc + cy) * nc + cx];
        }
        parent[p] = s * 0.125f;
    }
}

// BF16 brick copy of a dense level (l >= 1): brick p = the 8 children of
// level-(l-1) cell p, 16 bytes, octant order.
__global__ void to_bricks(const float *__restrict__ lvl, int l, __nv_bfloat16 *__restrict__ brick)
{
    const int64_t np = (int64_t)1 << (l - 1);
    const int64_t total = np * np * np;
    const int64_t nc = np * 2;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < total;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = p % np, y = (p / np) % np, z = p / (np * np);
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            const int64_t cx = 2 * x + (o & 1), cy = 2 * y + ((o >> 1) & 1), cz = 2 * z + ((o >> 2) & 1);
            v[o] = __float2bfloat16_rn(lvl[(cz * nc + cy) * nc + cx]);
        }
        *reinterpret_cast<uint4 *>(brick + 8 * p) = *reinterpret_cast<uint4 *>(v);
    }
}

inline unsigned grid_for(int64_t n, int block)
{
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

cd_status restrict_uniform(cd_tree t, const float *rho_dev, cudaStream_t s)
{
    const int L = t->L;
    const int64_t np = (int64_t)1 << (L - 1);
    {
        LaunchScope ls(CD_K_RESTRICT, s);
        restrict_from_leaves<<<grid_for(np * np * np, 256), 256, 0, s>>>(rho_dev, L, t->rho_leaf, t->rho_lvl[L - 1]);
    }
    CD_CHECK_LAUNCH();
    return restrict_dense(t, L - 1, s);
}

cd_status restrict_dense(cd_tree t, int top, cudaStream_t s)
{
    for (int l = top; l >= 1; --l) {
        const int64_t n = (int64_t)1 << (l - 1);
        LaunchScope ls(CD_K_RESTRICT, s);
        restrict_level<<<grid_for(n * n * n, 256), 256, 0, s>>>(t->rho_lvl[l], l, t->rho_lvl[l - 1]);
        CD_CHECK_LAUNCH();
    }
    for (int l = 1; l <= top; ++l) {
        const int64_t n = (int64_t)1 << (l - 1);
        LaunchScope ls(CD_K_RESTRICT, s);
        to_bricks<<<grid_for(n * n * n, 256), 256, 0, s>>>(t->rho_lvl[l], l, t->rho_brick[l]);
        CD_CHECK_LAUNCH();
    }
    return CD_OK;
}

}  // namespace cd
