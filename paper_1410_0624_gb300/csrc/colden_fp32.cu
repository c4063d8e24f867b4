// FP32 CUDA-core forms of the shell contraction and the per-leaf epilogue.
//
// Shell kernel (Eq. N_discret, one level of receiving cells at a time).  For
// every cell c at level k and direction d:
//   out[c][d] = prefix_in[parent(c)][d]
//             + sum_{t in tmask} dx_{k-t+1} sum_s rho_{k-t+1}(stencil_t(c), s) K_t[cfg_t(c)][d][s]
// with the stencil of table t anchored at the ancestor A_{k-t} of c.  The
// cells of one CTA are the 8^(k-q) descendants of one level-q cell
// (q = max(k-3, 0)): a Morton-contiguous run, so every output row is written
// coalesced.  The density regions the CTA's stencils touch are staged once in
// shared memory (zero outside the box, §3.2: the sum runs to the box border)
// and the sparse weights of each (cfg, d) are walked from L1/L2.
//
// Leaf kernel (§3.2 internal + local contributions, Eqs. eq_chi / chi_discret).
// One warp per oct:
//   N_H[t][d] = E[oct][d] + dx_L sum_s rho_leaf[oct][s] Kloc[t][s][d]
//   A_V = N_H av_per_nh,  shield[t] = (1/nd) sum_d exp(-k A_V).
#include "common.cuh"

namespace cd {
namespace {

constexpr int kExtThreads = 256;
constexpr int kRegion1 = 12 * 12 * 12;  // table 1: 4^3 ancestors -> (2*4+4)^3 cells
constexpr int kRegion2 = 8 * 8 * 8;
constexpr int kRegion3 = 6 * 6 * 6;

struct ExtArgs {
    ExtLaunch a;
    int q;
    const uint8_t *cnt[4];
    const uint8_t *idx[4];
    const float *w[4];
};

__global__ void __launch_bounds__(kExtThreads) shell_sum_fp32(ExtArgs P)
{
    __shared__ float s_rho[kRegion1 + kRegion2 + kRegion3];
    __shared__ int s_off[4][CD_STENCIL];

    const int k = P.a.k, q = P.q, nd = P.a.nd;
    const int span = k - q;                                   // levels below the CTA root
    const uint64_t root = blockIdx.x;                         // Morton index at level q
    const uint32_t Qx = compact3(root), Qy = compact3(root >> 1), Qz = compact3(root >> 2);

    int R[4] = {0, 0, 0, 0}, base[4] = {0, 0, 0, 0};
    {
        int off = 0;
        for (int t = 1; t <= 3; ++t) {
            if (!(P.a.tmask & (1 << (t - 1)))) continue;
            const int nP = 1 << (span - t);                   // ancestors per axis in the CTA
            R[t] = 2 * nP + 4;
            base[t] = off;
            off += R[t] * R[t] * R[t];
        }
    }
    // stage the density regions (level k - t + 1, origin 2 (P_min - 1))
    for (int t = 1; t <= 3; ++t) {
        if (!R[t]) continue;
        const int l = k - t + 1;
        const int64_t n = (int64_t)1 << l;
        const int nP = 1 << (span - t);
        const int64_t ox = 2 * ((int64_t)Qx * nP - 1), oy = 2 * ((int64_t)Qy * nP - 1), oz = 2 * ((int64_t)Qz * nP - 1);
        const int Rt = R[t], vol = Rt * Rt * Rt;
        const float *rho = P.a.rho[t];
        for (int r = threadIdx.x; r < vol; r += blockDim.x) {
            const int rx = r % Rt, ry = (r / Rt) % Rt, rz = r / (Rt * Rt);
            const int64_t gx = ox + rx, gy = oy + ry, gz = oz + rz;
            float v = 0.f;
            if (gx >= 0 && gy >= 0 && gz >= 0 && gx < n && gy < n && gz < n) v = rho[(gz * n + gy) * n + gx];
            s_rho[base[t] + r] = v;
        }
        for (int s = threadIdx.x; s < CD_STENCIL; s += blockDim.x)
            s_off[t][s] = base[t] + (s % 6) + Rt * (((s / 6) % 6) + Rt * (s / 36));
    }
    __syncthreads();

    const int ncell = 1 << (3 * span);
    const uint64_t first = root << (3 * span);
    for (int e = threadIdx.x; e < ncell * nd; e += blockDim.x) {
        const int j = e / nd, d = e - j * nd;
        const uint64_t m = first + (uint64_t)j;
        const uint32_t cx = compact3((uint64_t)j), cy = compact3((uint64_t)j >> 1), cz = compact3((uint64_t)j >> 2);
        float acc = P.a.prefix_in ? P.a.prefix_in[(m >> 3) * nd + d] : 0.f;
        for (int t = 1; t <= 3; ++t) {
            if (!R[t]) continue;
            const int Rt = R[t];
            const int anchor = 2 * (cx >> t) + Rt * (2 * (cy >> t) + Rt * (2 * (cz >> t)));
            const int cfg = (int)(m & ((1u << (3 * t)) - 1));
            const size_t row = (size_t)cfg * nd + d;
            const int n = P.cnt[t][row];
            const uint8_t *ix = P.idx[t] + row * CD_MAXE;
            const float *wt = P.w[t] + row * CD_MAXE;
            float part = 0.f;
            for (int i = 0; i < n; ++i) part = fmaf(s_rho[anchor + s_off[t][ix[i]]], wt[i], part);
            acc = fmaf(P.a.dx[t], part, acc);
        }
        P.a.out[m * nd + d] = acc;
    }
}

__global__ void __launch_bounds__(256) leaf_epilogue(LeafLaunch P)
{
    extern __shared__ float s_kloc[];                 // [8][8][nd]
    __shared__ float s_sum[8][8];
    const int nd = P.nd;
    for (int i = threadIdx.x; i < 64 * nd; i += blockDim.x) s_kloc[i] = P.kloc[i];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * 8;
    for (int64_t oct = (int64_t)blockIdx.x * 8 + warp; oct < P.n_oct; oct += stride) {
        const float r = P.rho_leaf[oct * 8 + (lane & 7)];
        float rs[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) rs[s] = __shfl_sync(0xffffffffu, r, s);
        if (lane < 8) s_sum[warp][lane] = 0.f;
        __syncwarp();
        const float *E = P.E ? P.E + oct * nd : nullptr;
        const int64_t obase = oct * 8 * nd;
        for (int f = lane; f < 8 * nd; f += 32) {
            const int t = f / nd, d = f - t * nd;
            const float *kl = s_kloc + t * 8 * nd + d;
            float loc = 0.f;
#pragma unroll
            for (int s = 0; s < 8; ++s) loc = fmaf(rs[s], kl[s * nd], loc);
            const float N = (E ? E[d] : 0.f) + P.dx_leaf * loc;
            if (P.n_h) P.n_h[obase + f] = N;
            const float av = N * P.av_per_nh;
            if (P.a_v) P.a_v[obase + f] = av;
            if (P.shield) atomicAdd(&s_sum[warp][t], expf(-P.shield_k * av));
        }
        __syncwarp();
        if (P.shield && lane < 8) P.shield[oct * 8 + lane] = s_sum[warp][lane] / (float)nd;
        __syncwarp();
    }
}

}  // namespace

cd_status launch_ext_fp32(const ExtLaunch &a, cd_geom g, cudaStream_t s)
{
    ExtArgs P;
    P.a = a;
    P.q = a.k > 3 ? a.k - 3 : 0;
    for (int t = 0; t < 4; ++t) {
        P.cnt[t] = g->cnt[t];
        P.idx[t] = g->idx[t];
        P.w[t] = g->w[t];
    }
    const uint64_t nblk = 1ull << (3 * P.q);
    LaunchScope ls(CD_K_SHELL, s);
    shell_sum_fp32<<<(unsigned)nblk, kExtThreads, 0, s>>>(P);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status launch_leaf(const LeafLaunch &a, cudaStream_t s)
{
    int64_t blocks = (a.n_oct + 7) / 8;
    if (blocks > 152 * 16) blocks = 152 * 16;
    const size_t smem = sizeof(float) * 64 * a.nd;
    if (smem > 48 * 1024) {
        CD_CUDA(cudaFuncSetAttribute(leaf_epilogue, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    LaunchScope ls(CD_K_LEAF, s);
    leaf_epilogue<<<(unsigned)blocks, 256, smem, s>>>(a);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

}  // namespace cd
