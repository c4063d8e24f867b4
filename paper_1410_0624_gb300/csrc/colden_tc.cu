// BF16 tensor-core (tcgen05) form of the shell contraction (Eq. N_discret).
//
// GEMM framing.  For a receiving level k (k >= 4) every shell table t reads a
// 6x6x6 stencil of level k-t+1 around the ancestor A_{k-t}; the stencil of
// table 1 sits around the parent P = A_{k-1} of the receiving cell c and is
// shared by the 8 children of P.  One GEMM row is one parent P:
//   A[P, (t, q, ch)] = rho_{k-t+1}(child ch of neighbour q of A_{k-t}(P))
//   B[(t, q, ch), (o, d)] = 2^(t-1) K_t[cfg_t(P, o)][s(q, ch)][d]
//   E[8P + o][d] = dx_k D[P, (o, d)] + S_{k-1}[P][d]
// with q over the 27 level-(k-t) neighbours (+1 zero brick: 28 per table),
// ch over their 8 children and o over the children of P.  cfg_t depends on
// the octants of P and of its parent, so the 64 classes (oct(par P), oct(P))
// each get their own B and a tile holds 128 parents of one class.  Powers
// of two fold dx_{k-t+1} = 2^(t-1) dx_k into B exactly.
//
// Densities are stored per level as BF16 "bricks" (the 8 children of one
// coarser cell, 16 bytes), so an A row is 84 bricks and one brick is exactly
// one row of an 8x16-byte core matrix: cp.async 16-byte copies place them
// straight into the K-major no-swizzle operand layout.  B is precomputed in
// global memory in that layout per K-chunk, so each chunk is one bulk copy.
//
// CTA (256 threads): warp 0 issues the MMAs (M = 128, N = 8 nd split in n_mma
// instructions, K = 16) and owns the TMEM accumulator; warp 1 bulk-copies B;
// warps 2-3 gather A; warps 4-7 drain TMEM (lane quarter = warp % 4) into E.
// A 4-stage mbarrier pipeline couples them; every wait is bounded and a
// timeout sets a device flag instead of trapping.
#include <algorithm>

#include "common.cuh"
#include "geom_device.cuh"
#include "umma.cuh"

namespace cd {
namespace {

constexpr int kStages = 4;
constexpr int kChunkBricks = 4;                 // K = 32 per chunk (2 MMA K-steps)
constexpr int kBricksPerTable = 28;             // 27 neighbours + 1 zero brick
constexpr int kChunks = 3 * kBricksPerTable / kChunkBricks;  // 21
constexpr int kThreads = 256;
constexpr uint32_t kMaxPolls = 1u << 26;
constexpr uint32_t kAStageBytes = 128 * kChunkBricks * 16;   // 8 KB

static __device__ int g_tc_fault;

struct TcArgs {
    int k;                       // receiving level (>= 4)
    int nd, N, n_mma, Nh;        // directions, N = 8 nd, MMAs per K-step, columns per MMA
    int c0, c1;                  // chunk range (tables 1..3 -> 0..21, table 3 only -> 14..21)
    const __nv_bfloat16 *brick[4];   // brick arrays of levels k, k-1, k-2 (tables 1, 2, 3)
    const __nv_bfloat16 *B;      // [64 class][21 chunk][N/8][4][8][8]
    const float *prefix_in;      // S_{k-1} [8^(k-1)][nd] or NULL
    float *out;                  // [8^k][nd]
    float dx_k;
    int64_t nG;                  // 8^(k-3)
    int64_t ntiles;              // 64 * ceil(nG / 128)
};

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity)
{
    return mbar_wait_bounded(bar, parity, kMaxPolls);
}

__global__ void __launch_bounds__(kThreads, 1) shell_sum_tc(TcArgs P)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t bstage = (uint32_t)P.N * kChunkBricks * 16;       // N/8 groups x 4 bricks x 128 B
    unsigned char *sA = smem;                                        // [kStages][8 KB]
    unsigned char *sB = smem + kStages * kAStageBytes;               // [kStages][bstage]
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + kStages * bstage);
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;
    uint64_t *acc_empty = acc_full + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc_empty + 1);
    __shared__ int s_fault;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nchunk = P.c1 - P.c0;

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 64 + 1);       // 64 gather threads + the B producer
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, 4);               // one arrival per epilogue warp
        fence_mbar_init();
        s_fault = 0;
    }
    if (warp == 0) tmem_alloc(tslot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    bool fault = false;
    if (warp == 0) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            uint32_t q = 0;
            int u = 0;
            for (int64_t tile = blockIdx.x; tile < P.ntiles && !fault; tile += gridDim.x, ++u) {
                if (!wait_bar(acc_empty, (u & 1) ^ 1)) { fault = true; break; }
                tc_fence_after();
                for (int j = 0; j < nchunk; ++j, ++q) {
                    const int s = q % kStages;
                    if (!wait_bar(&full[s], (q / kStages) & 1)) { fault = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kAStageBytes), b0 = smem_u32(sB + s * bstage);
#pragma unroll
                    for (int ks = 0; ks < kChunkBricks / 2; ++ks) {
                        const uint64_t ad = umma_smem_desc(a0 + ks * 256, 128, kChunkBricks * 128);
                        for (int h = 0; h < P.n_mma; ++h) {
                            const uint64_t bd =
                                umma_smem_desc(b0 + h * (P.Nh / 8) * (kChunkBricks * 128) + ks * 256, 128,
                                               kChunkBricks * 128);
                            umma_bf16(tbase + h * P.Nh, ad, bd, umma_idesc_bf16(128, P.Nh), (j > 0 || ks > 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (fault) break;
                umma_commit(acc_full);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- B producer ----------------
        if (lane == 0) {
            uint32_t q = 0;
            for (int64_t tile = blockIdx.x; tile < P.ntiles && !fault; tile += gridDim.x) {
                const int cls = (int)(tile % 64);
                const unsigned char *Bc = reinterpret_cast<const unsigned char *>(P.B) + (size_t)cls * kChunks * bstage;
                for (int j = 0; j < nchunk; ++j, ++q) {
                    const int s = q % kStages;
                    if (!wait_bar(&empty[s], ((q / kStages) & 1) ^ 1)) { fault = true; break; }
                    mbar_expect_tx(&full[s], bstage);
                    bulk_g2s(sB + s * bstage, Bc + (size_t)(P.c0 + j) * bstage, bstage, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp < 4) {
        // ---------------- A gather (64 threads, 8 bricks each per chunk) ----------------
        const int g = tid - 64;                  // 0..63
        uint32_t q = 0;
        for (int64_t tile = blockIdx.x; tile < P.ntiles && !fault; tile += gridDim.x) {
            const int cls = (int)(tile % 64);
            const int64_t gb = tile / 64;
            // this thread's two rows m = g, g + 64: parent P = (G << 6) | cls
            int64_t acx[2][3], acy[2][3], acz[2][3];   // anchors A_{k-t}(P) for t = 1..3
            bool valid[2];
            for (int r = 0; r < 2; ++r) {
                const int64_t G = gb * 128 + g + 64 * r;
                valid[r] = G < P.nG;
                const uint64_t Pm = ((uint64_t)(valid[r] ? G : 0) << 6) | (uint64_t)cls;
                const int64_t px = compact3(Pm), py = compact3(Pm >> 1), pz = compact3(Pm >> 2);
                for (int t = 0; t < 3; ++t) {
                    acx[r][t] = px >> t;
                    acy[r][t] = py >> t;
                    acz[r][t] = pz >> t;
                }
            }
            for (int j = 0; j < nchunk; ++j, ++q) {
                const int s = q % kStages;
                bool ok = true;
                if (lane == 0) ok = wait_bar(&empty[s], ((q / kStages) & 1) ^ 1);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { fault = true; break; }
                unsigned char *dst = sA + s * kAStageBytes;
                const int c = P.c0 + j;
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int m = g + 64 * r;
#pragma unroll
                    for (int b = 0; b < kChunkBricks; ++b) {
                        const int kb = c * kChunkBricks + b;             // 0..83
                        const int t = kb / kBricksPerTable, nq = kb % kBricksPerTable;
                        const int lvl_side_log = P.k - t - 1;            // neighbours live at level k-t-1
                        const int64_t n = (int64_t)1 << lvl_side_log;
                        const int64_t x = acx[r][t] + (nq % 3) - 1, y = acy[r][t] + (nq / 3) % 3 - 1,
                                      z = acz[r][t] + nq / 9 - 1;
                        const bool in = valid[r] && nq < 27 && x >= 0 && y >= 0 && z >= 0 && x < n && y < n && z < n;
                        const __nv_bfloat16 *src = P.brick[t + 1] + (in ? 8 * ((z * n + y) * n + x) : 0);
                        // core matrix (m / 8, b) of the stage, row m % 8
                        cp_async16(dst + ((m >> 3) * kChunkBricks + b) * 128 + (m & 7) * 16, src, in ? 16u : 0u);
                    }
                }
                cp_async_arrive(&full[s]);
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        // ---------------- epilogue: TMEM -> E ----------------
        const int quarter = warp & 3;             // TMEM lanes 32 quarter .. +31
        const int m = quarter * 32 + lane;
        int u = 0;
        for (int64_t tile = blockIdx.x; tile < P.ntiles && !fault; tile += gridDim.x, ++u) {
            const int cls = (int)(tile % 64);
            const int64_t G = (tile / 64) * 128 + m;
            const bool valid = G < P.nG;
            const int64_t Pm = ((valid ? G : 0) << 6) | cls;
            bool ok = true;
            if (lane == 0) ok = wait_bar(acc_full, u & 1);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) { fault = true; break; }
            tc_fence_after();
            float *orow = P.out + (size_t)Pm * 8 * P.nd;
            const float *pre = P.prefix_in ? P.prefix_in + (size_t)Pm * P.nd : nullptr;
            int o_d = 0;                          // running direction index of column c
            for (int c = 0; c < P.N; c += 32) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
                tmem_ld_wait();
                if (valid) {
                    float o[32];
                    int d = o_d;
#pragma unroll
                    for (int i = 0; i < 32; ++i) {
                        o[i] = P.dx_k * __uint_as_float(v[i]) + (pre ? pre[d] : 0.f);
                        d = (d + 1 == P.nd) ? 0 : d + 1;
                    }
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *reinterpret_cast<float4 *>(orow + c + i) = make_float4(o[i], o[i + 1], o[i + 2], o[i + 3]);
                }
                o_d = (o_d + 32) % P.nd;
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
        }
    }

    if (fault) {
        s_fault = 1;
        atomicExch(&g_tc_fault, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        if (s_fault && lane == 0) {
            // let issued MMAs finish before the accumulator is released
            umma_commit(acc_full);
            mbar_wait_bounded(acc_full, 0, kMaxPolls);
            mbar_wait_bounded(acc_full, 1, kMaxPolls);
        }
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

// ---- B operand construction (FP64 geometry, stored BF16) -----------------------

__global__ void build_b(int nd, const double *__restrict__ dirs, __nv_bfloat16 *__restrict__ B)
{
    const int N = 8 * nd;
    const int64_t total = (int64_t)64 * kChunks * kChunkBricks * 8 * N;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        // layout [cls][chunk][ng][b][n8][ch]
        const int ch = (int)(e & 7);
        const int n8 = (int)((e >> 3) & 7);
        const int b = (int)((e >> 6) % kChunkBricks);
        int64_t rest = (e >> 6) / kChunkBricks;
        const int ng = (int)(rest % (N / 8));
        rest /= (N / 8);
        const int chunk = (int)(rest % kChunks);
        const int cls = (int)(rest / kChunks);
        const int n = ng * 8 + n8, o = n / nd, d = n % nd;
        const int kb = chunk * kChunkBricks + b;
        const int t = kb / kBricksPerTable + 1, q = kb % kBricksPerTable;
        float v = 0.f;
        if (q < 27) {
            const int a = 2 * (q % 3) + (ch & 1), bb = 2 * ((q / 3) % 3) + ((ch >> 1) & 1),
                      cc = 2 * (q / 9) + ((ch >> 2) & 1);
            const int s = a + 6 * bb + 36 * cc;
            const int oP = cls & 7, opP = cls >> 3;
            const int cfg = t == 1 ? o : t == 2 ? (oP << 3) | o : (opP << 6) | (oP << 3) | o;
            const double u[3] = {dirs[3 * d], dirs[3 * d + 1], dirs[3 * d + 2]};
            v = (float)(shell_weight(t, cfg, s, u) * (double)(1 << (t - 1)));
        }
        B[e] = __float2bfloat16_rn(v);
    }
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

}  // namespace

// N = 8 nd accumulator columns: at most 512 (TMEM), a multiple of 32 (the
// epilogue drains 32 columns per load) and at most two MMAs of N/2 <= 256.
bool tc_supported(int nd)
{
    const int N = 8 * nd;
    return N <= 512 && N % 32 == 0;
}

cd_status build_tc_tables(cd_geom g, cudaStream_t s)
{
    const int nd = g->n_dir;
    if (!tc_supported(nd)) return CD_OK;
    const size_t elems = (size_t)64 * kChunks * kChunkBricks * 8 * 8 * nd;
    if (!g->wb) {
        if (cudaMalloc(&g->wb, elems * sizeof(__nv_bfloat16)) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate the BF16 weight operands (%zu bytes)", elems * 2);
            return CD_ENOMEM;
        }
        g->wb_bytes = elems * sizeof(__nv_bfloat16);
    }
    LaunchScope ls(CD_K_OTHER, s);
    build_b<<<num_sms() * 8, 256, 0, s>>>(nd, g->dirs_dev, g->wb);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status launch_ext_tc(const ExtLaunch &a, const __nv_bfloat16 *const *brick, cd_geom g, cudaStream_t s)
{
    if (a.k < 4 || !g->wb || !tc_supported(a.nd)) {
        set_error("tensor-core shell needs level >= 4 and a supported direction count");
        return CD_EUNSUPPORTED;
    }
    TcArgs P;
    P.k = a.k;
    P.nd = a.nd;
    P.N = 8 * a.nd;
    P.n_mma = P.N > 256 ? 2 : 1;
    P.Nh = P.N / P.n_mma;
    const bool all3 = (a.tmask & 7) == 7;
    if (!all3 && a.tmask != 4) {
        set_error("tensor-core shell serves tables {1,2,3} or {3}");
        return CD_EUNSUPPORTED;
    }
    P.c0 = all3 ? 0 : 2 * kBricksPerTable / kChunkBricks;
    P.c1 = kChunks;
    P.brick[0] = nullptr;
    P.brick[1] = brick[a.k];
    P.brick[2] = brick[a.k - 1];
    P.brick[3] = brick[a.k - 2];
    P.B = g->wb;
    P.prefix_in = a.prefix_in;
    P.out = a.out;
    P.dx_k = a.dx[1] > 0.f ? a.dx[1] : a.dx[3] * 0.25f;
    P.nG = (int64_t)1 << (3 * (a.k - 3));
    P.ntiles = 64 * ((P.nG + 127) / 128);
    const size_t bstage = (size_t)P.N * kChunkBricks * 16;
    const size_t smem = kStages * (kAStageBytes + bstage) + (2 * kStages + 2) * 8 + 16;
    CD_CUDA(cudaFuncSetAttribute(shell_sum_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::min<int64_t>(P.ntiles, num_sms());
    LaunchScope ls(CD_K_SHELL, s);
    shell_sum_tc<<<(unsigned)grid, kThreads, smem, s>>>(P);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status tc_fault_check()
{
    int v = 0;
    CD_CUDA(cudaMemcpyFromSymbol(&v, g_tc_fault, sizeof(int)));
    if (v) {
        const int zero = 0;
        CD_CUDA(cudaMemcpyToSymbol(g_tc_fault, &zero, sizeof(int)));
        set_error("a tensor-core shell kernel gave up a bounded wait");
        return CD_ETIMEOUT;
    }
    return CD_OK;
}

}  // namespace cd
