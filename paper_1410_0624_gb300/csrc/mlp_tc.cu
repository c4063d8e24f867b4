// The learned form of cd_column_density in BF16 on the tcgen05 tensor cores
// (weights and activations BF16, accumulation FP32 in tensor memory).
//
// Layer 1 is split along its inputs.  The external slots (Delta_l = 1..7, 7
// n_dir inputs) are the same for the 8 leaves of an oct, so
//   z1[leaf] = W1c u_cell[leaf] + h[oct],   h[oct] = W1e u_ext[oct] + b1
// with u_cell = the standardised own-oct slot (n_dir inputs) and ln n.  Two
// kernels:
//   learned_oct_tc   one GEMM row per oct: builds u_ext from the per-level
//                    sums (ln, standardise, BF16) straight into the operand
//                    layout in shared memory, one MMA chain of K = 7 n_dir
//                    against the resident W1e, writes h (BF16) and the oct's
//                    external column sum_s c[s] (FP32).
//   learned_cell_tc  one GEMM row per leaf, 128 leaves per tile: the internal +
//                    local term as a small MMA (the oct's 8 densities against
//                    dx K_loc), u_cell on the CUDA cores, then
//                    MMA1 (W1c, + h) -> GELU -> MMA2 (W2, + b2) -> GELU ->
//                    MMA3 (W3, + b3) = delta log2(e) -> N = N_tree 2^(...),
//                    A_V and the shield; the tile's N rows leave as one bulk
//                    copy.  Two independent groups
//                    of four warps share the weights, so one group's CUDA-core
//                    work overlaps the other's MMAs.
//
// Additions folded into the MMAs.  Every chain ends with one extra K-step of
// 16 whose A is a constant one-hot block, A1h[m][k] = (k == m / 8): row m
// (leaf m of the tile) selects column m / 8, its oct.  With B[n][k] = h[oct
// k][n] this adds h[oct(m)][n] (the tile's 16 layer-1 parts, which
// learned_oct_tc writes directly in this operand layout); with B[n][k] = b[n]
// for every k it adds the bias b[n].
//
// Every operand is K-major without swizzle: element (row, k) of a [rows x K]
// tile sits at byte (row/8) (K/8) 128 + (k/8) 128 + (row%8) 16 + (k%8) 2,
// i.e. LBO = 128 bytes along K and SBO = 16 K bytes between 8-row groups.
// Waits on the tensor cores are bounded; a timeout sets a device flag
// (cd_device_status) and the kernel leaves its loop with all threads together.
#include <algorithm>
#include <vector>

#include "learned.cuh"
#include "umma.cuh"

namespace cd {
namespace {

constexpr int kH = 128;                     // hidden width of the tensor-core form
constexpr int kKW = kH + 16;                // K of the W2 / W3 images: 128 inputs + the bias block
constexpr int kMaxNd = 48;
constexpr uint32_t kMaxPolls = 1u << 26;
constexpr float kGeluC = 0.7978845608028654f;
constexpr float kGeluA = 0.044715f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr int kHBlock = 128 * 16;           // BF16 elements of one tile's layer-1 block (16 octs)

static __device__ int g_ltc_fault;

__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }
__host__ __device__ constexpr size_t align128(size_t v) { return (v + 127) & ~(size_t)127; }

__host__ __device__ inline uint32_t op_off(int row, int k, int K)
{
    return (uint32_t)((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// Byte offsets of the packed tensor-core weights in one device buffer.
struct TcLayout {
    int nd, NP, KC, KE, n_in;
    size_t w1c, w1e, w2, w3;           // BF16 operand images [128 x KC], [128 x KE], [128 x kKW], [NP x kKW]
    size_t b1;                         // FP32 [128]
    size_t muc, sic, mue, sie;         // FP32 standardisation u = a lg2(x) + b: a then b for the cell inputs
                                       // [KC] and for the external inputs [KE]
    size_t total;
};

TcLayout make_layout(int nd)
{
    TcLayout T;
    T.nd = nd;
    T.NP = round16(nd);
    T.KC = round16(nd + 1);
    T.KE = round16(7 * nd);
    T.n_in = kSlots * nd + 1;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t r = o; o = align128(o + bytes); return r; };
    T.w1c = take((size_t)kH * T.KC * 2);
    T.w1e = take((size_t)kH * T.KE * 2);
    T.w2 = take((size_t)kH * kKW * 2);
    T.w3 = take((size_t)T.NP * kKW * 2);
    T.b1 = take(kH * 4);
    T.muc = take((size_t)T.KC * 4);
    T.sic = take((size_t)T.KC * 4);
    T.mue = take((size_t)T.KE * 4);
    T.sie = take((size_t)T.KE * 4);
    T.total = o;
    return T;
}

struct TcState {
    TcLayout lay;
    unsigned char *buf = nullptr;
    __nv_bfloat16 *h = nullptr;        // per-leaf-tile blocks [128 n x 16 octs] of the layer-1 parts
    float *ext = nullptr;              // [n_oct][nd] external column
    int64_t cap = 0;                   // octs h / ext hold
};

// ---- packing of the FP32 master parameters ----------------------------------

struct PackArgs {
    TcLayout T;
    const float *p;        // packed FP32 parameters
    const float *mu, *sinv;
    NetLayout N;
    unsigned char *buf;
};

// W3 and b3 are scaled by log2(e) so that the last chain gives delta log2(e)
// and N = N_tree 2^(that).
__global__ void pack_tc(PackArgs A)
{
    const TcLayout &T = A.T;
    const NetLayout &N = A.N;
    const int nd = T.nd;
    const float *W1 = A.p + N.W1, *W2 = A.p + N.W2, *W3 = A.p + N.W3;
    const int64_t n1c = (int64_t)kH * T.KC, n1e = (int64_t)kH * T.KE, n2 = (int64_t)kH * kKW,
                  n3 = (int64_t)T.NP * kKW;
    const int64_t total = n1c + n1e + n2 + n3 + kH + 2 * T.KC + 2 * T.KE;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        int64_t i = e;
        if (i < n1c) {
            const int n = (int)(i / T.KC), k = (int)(i % T.KC);
            const float v = k < nd ? W1[(int64_t)n * N.n_in + k] : (k == nd ? W1[(int64_t)n * N.n_in + kSlots * nd] : 0.f);
            reinterpret_cast<__nv_bfloat16 *>(A.buf + T.w1c + op_off(n, k, T.KC))[0] = __float2bfloat16_rn(v);
            continue;
        }
        i -= n1c;
        if (i < n1e) {
            const int n = (int)(i / T.KE), k = (int)(i % T.KE);
            const float v = k < 7 * nd ? W1[(int64_t)n * N.n_in + nd + k] : 0.f;
            reinterpret_cast<__nv_bfloat16 *>(A.buf + T.w1e + op_off(n, k, T.KE))[0] = __float2bfloat16_rn(v);
            continue;
        }
        i -= n1e;
        if (i < n2) {
            const int n = (int)(i / kKW), k = (int)(i % kKW);
            const float v = k < kH ? W2[(int64_t)n * kH + k] : A.p[N.b2 + n];
            reinterpret_cast<__nv_bfloat16 *>(A.buf + T.w2 + op_off(n, k, kKW))[0] = __float2bfloat16_rn(v);
            continue;
        }
        i -= n2;
        if (i < n3) {
            const int n = (int)(i / kKW), k = (int)(i % kKW);
            const float v = n >= nd ? 0.f : kLog2e * (k < kH ? W3[(int64_t)n * kH + k] : A.p[N.b3 + n]);
            reinterpret_cast<__nv_bfloat16 *>(A.buf + T.w3 + op_off(n, k, kKW))[0] = __float2bfloat16_rn(v);
            continue;
        }
        i -= n3;
        if (i < kH) { reinterpret_cast<float *>(A.buf + T.b1)[i] = A.p[N.b1 + i]; continue; }
        i -= kH;
        // standardisation as u = a lg2(x) + b: a = ln(2) sinv, b = -mu sinv
        if (i < 2 * T.KC) {
            const int k = (int)(i % T.KC);
            const int src = k < nd ? k : (k == nd ? kSlots * nd : -1);
            const bool is_a = i < T.KC;
            const float v = src < 0 ? 0.f : (is_a ? kLn2 * A.sinv[src] : -A.mu[src] * A.sinv[src]);
            reinterpret_cast<float *>(A.buf + (is_a ? T.muc : T.sic))[k] = v;
            continue;
        }
        i -= 2 * T.KC;
        {
            const int k = (int)(i % T.KE);
            const bool is_a = i < T.KE;
            const float v = k < 7 * nd ? (is_a ? kLn2 * A.sinv[nd + k] : -A.mu[nd + k] * A.sinv[nd + k]) : 0.f;
            reinterpret_cast<float *>(A.buf + (is_a ? T.mue : T.sie))[k] = v;
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ uint32_t bf2(float v)   // a BF16 constant in both halves
{
    return pack_bf16x2(v, v);
}

// GELU (tanh form) of two BF16 values in packed BF16 arithmetic:
// g = z/2 (1 + tanh(z (c + c a z^2))).  The result is an operand of the next
// BF16 product either way.
__device__ __forceinline__ uint32_t gelu_bf16x2(uint32_t z)
{
    uint32_t z2, p, inner, t, hz, g;
    const uint32_t ca = bf2(kGeluC * kGeluA), c = bf2(kGeluC), half = bf2(0.5f);
    asm("mul.rn.bf16x2 %0, %1, %1;" : "=r"(z2) : "r"(z));
    asm("fma.rn.bf16x2 %0, %1, %2, %3;" : "=r"(p) : "r"(z2), "r"(ca), "r"(c));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(inner) : "r"(p), "r"(z));
    asm("tanh.approx.bf16x2 %0, %1;" : "=r"(t) : "r"(inner));
    asm("mul.rn.bf16x2 %0, %1, %2;" : "=r"(hz) : "r"(z), "r"(half));
    asm("fma.rn.bf16x2 %0, %1, %2, %1;" : "=r"(g) : "r"(hz), "r"(t));
    return g;
}

__device__ __forceinline__ float fast_log2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// standardised, clipped input from a positive quantity: a lg2(max(x, floor)) + b
__device__ __forceinline__ float std_input(float x, float floor_, float a, float b)
{
    return fminf(fmaxf(fmaf(a, fast_log2(fmaxf(x, floor_)), b), -kUMax), kUMax);
}

__device__ __forceinline__ float fast_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void named_barrier(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// D (+)= A[128 x K] * B[N x K]^T over K-steps of 16; A and B are K-major
// images whose K (hence SBO) may differ.
__device__ __forceinline__ void mma_steps(uint32_t tmem_d, uint32_t a0, int Ka, uint32_t b0, int Kb, int steps, int N,
                                          bool accumulate_first)
{
    const uint32_t idesc = umma_idesc_bf16(128, N);
    for (int ks = 0; ks < steps; ++ks)
        umma_bf16(tmem_d, umma_smem_desc(a0 + ks * 256, 128, (uint32_t)Ka * 16),
                  umma_smem_desc(b0 + ks * 256, 128, (uint32_t)Kb * 16), idesc, (ks > 0 || accumulate_first) ? 1u : 0u);
}

// ---- per-oct part ---------------------------------------------------------------

struct OctArgs {
    TcLayout T;
    const unsigned char *tc;
    int64_t n_oct, ntiles;
    int L;
    const float *Et[4];
    const float *C[CD_MAXL + 1];
    __nv_bfloat16 *h;      // layer-1 blocks, kHBlock elements per 16 octs
    float *ext;            // [n_oct][nd]
};

constexpr int kOctThreads = 384;                              // 12 warps
constexpr int kOctUnits = 128 * kMaxNd / 8 / kOctThreads;   // (row, 8 directions) units per thread: 2

// Far slots of a tile of 128 consecutive octs o0 .. o0+127 (o0 a multiple of
// 128): Delta_l = 4 reads the 16 parents o0/8 + r/8, Delta_l = 5 the 2
// grandparents, every coarser level one ancestor; rows 0-15, 16-17, 18 and 19
// (the tail, Delta_l >= 7 summed) of sT.
__device__ __forceinline__ float far_slot_entry(const OctArgs &A, int64_t o0, int row, int d, int nd)
{
    const int L = A.L;
    if (row < 16) return L >= 5 ? A.C[L - 2][((o0 >> 3) + row) * nd + d] : 0.f;
    if (row < 18) return L >= 6 ? A.C[L - 3][((o0 >> 6) + row - 16) * nd + d] : 0.f;
    if (row == 18) return L >= 7 ? A.C[L - 4][(o0 >> 9) * nd + d] : 0.f;
    float t = 0.f;
    for (int dl = 7; dl <= L - 1; ++dl) t += A.C[L - dl + 2][(o0 >> (3 * (dl - 3))) * nd + d];
    return t;
}

size_t oct_smem(const TcLayout &T)
{
    return 2 * align128((size_t)128 * T.KE * 2) + (size_t)8 * kHBlock * 2 +
           (size_t)(2 * T.KE + kH + 20 * T.nd) * 4 + 2 * 8 + 16;
}

__global__ void __launch_bounds__(kOctThreads, 1) learned_oct_tc(OctArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcLayout &T = A.T;
    const int nd = T.nd, KE = T.KE;
    unsigned char *sA = smem;                                    // [128 x KE] BF16 operand
    unsigned char *sB = sA + align128((size_t)128 * KE * 2);     // W1e image
    __nv_bfloat16 *sHb = reinterpret_cast<__nv_bfloat16 *>(sB + align128((size_t)128 * KE * 2));  // 8 h blocks
    float *sMu = reinterpret_cast<float *>(sHb + 8 * kHBlock);  // [KE] standardisation a
    float *sSi = sMu + KE;                                       // [KE] standardisation b
    float *sB1 = sSi + KE;                                       // [128]
    float *sT = sB1 + kH;                                        // [20][nd] far slots of the tile
    uint64_t *bar = reinterpret_cast<uint64_t *>(sT + 20 * nd);  // [0] weights, [1] MMA
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    int *sflag = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
        *sflag = 0;
    }
    for (int i = tid; i < KE; i += kOctThreads) {
        sMu[i] = reinterpret_cast<const float *>(A.tc + T.mue)[i];
        sSi[i] = reinterpret_cast<const float *>(A.tc + T.sie)[i];
    }
    for (int i = tid; i < kH; i += kOctThreads) sB1[i] = reinterpret_cast<const float *>(A.tc + T.b1)[i];
    if (warp == 0) tmem_alloc(tslot, 128);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    if (tid == 0) {
        const uint32_t bytes = (uint32_t)(128 * KE * 2);
        mbar_expect_tx(&bar[0], bytes);
        bulk_g2s(sB, A.tc + T.w1e, bytes, &bar[0]);
    }
    bool weights_ready = false;
    uint32_t phase = 0;
    const int units = 128 * (nd / 8);

    // Software pipeline over tiles: the loads of tile k+1 (near slots into
    // registers, far slots into registers) are issued right after tile k's
    // operand is built, so they are in flight during tile k's MMA and epilogue.
    float c[kOctUnits][3][8];
    float fs[(20 * kMaxNd + kOctThreads - 1) / kOctThreads];
    auto issue_loads = [&](int64_t tile) {
        const int64_t o0 = tile * 128;
        const int rows = (int)std::min<int64_t>(128, A.n_oct - o0);
        // near slots (Delta_l = 1..3) of this thread's units: lanes take
        // consecutive octs, each 8 consecutive directions (two 16-byte loads
        // per table)
#pragma unroll
        for (int j = 0; j < kOctUnits; ++j) {
            const int u = tid + j * kOctThreads;
            const int r = u & 127, d0 = (u >> 7) * 8;
            const bool ok = u < units && r < rows;
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (ok && t + 1 <= A.L - 1) {
                    const float4 *src = reinterpret_cast<const float4 *>(A.Et[t + 1] + (o0 + r) * nd + d0);
                    const float4 a = src[0], b = src[1];
                    c[j][t][0] = a.x; c[j][t][1] = a.y; c[j][t][2] = a.z; c[j][t][3] = a.w;
                    c[j][t][4] = b.x; c[j][t][5] = b.y; c[j][t][6] = b.z; c[j][t][7] = b.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) c[j][t][q] = 0.f;
                }
            }
        }
        // far slots shared by the tile
#pragma unroll
        for (int q = 0; q < (20 * kMaxNd + kOctThreads - 1) / kOctThreads; ++q) {
            const int e = tid + q * kOctThreads;
            fs[q] = e < 20 * nd ? far_slot_entry(A, o0, e / nd, e % nd, nd) : 0.f;
        }
    };
    if (blockIdx.x < A.ntiles) issue_loads(blockIdx.x);

    for (int64_t tile = blockIdx.x; tile < A.ntiles; tile += gridDim.x) {
        const int64_t o0 = tile * 128;
        const int rows = (int)std::min<int64_t>(128, A.n_oct - o0);
#pragma unroll
        for (int q = 0; q < (20 * kMaxNd + kOctThreads - 1) / kOctThreads; ++q) {
            const int e = tid + q * kOctThreads;
            if (e < 20 * nd) sT[e] = fs[q];
        }
        // the previous tile's h blocks must have been read out of sHb
        if (tid == 0) bulk_wait_read<0>();
        __syncthreads();
        // 3. u_ext -> operand rows (16-byte stores, lanes on consecutive rows),
        //    external column -> HBM
#pragma unroll
        for (int j = 0; j < kOctUnits; ++j) {
            const int u = tid + j * kOctThreads;
            if (u >= units) continue;
            const int r = u & 127, d0 = (u >> 7) * 8;
            const bool ok = r < rows;
            float tot[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) tot[q] = 0.f;
#pragma unroll
            for (int s = 0; s < 7; ++s) {
                float cv[8], a[8], b[8], v[8];
                if (s < 3) {
#pragma unroll
                    for (int q = 0; q < 8; ++q) cv[q] = c[j][s][q];
                } else {
                    const int row = s == 3 ? (r >> 3) : s == 4 ? 16 + (r >> 6) : s == 5 ? 18 : 19;
                    const float4 x0 = *reinterpret_cast<const float4 *>(sT + row * nd + d0);
                    const float4 x1 = *reinterpret_cast<const float4 *>(sT + row * nd + d0 + 4);
                    cv[0] = x0.x; cv[1] = x0.y; cv[2] = x0.z; cv[3] = x0.w;
                    cv[4] = x1.x; cv[5] = x1.y; cv[6] = x1.z; cv[7] = x1.w;
                }
                {
                    const int k = s * nd + d0;
                    const float4 a0 = *reinterpret_cast<const float4 *>(sMu + k), a1 = *reinterpret_cast<const float4 *>(sMu + k + 4);
                    const float4 b0 = *reinterpret_cast<const float4 *>(sSi + k), b1 = *reinterpret_cast<const float4 *>(sSi + k + 4);
                    a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w; a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
                    b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w; b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
                }
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    tot[q] += cv[q];
                    v[q] = ok ? std_input(cv[q], kCFloor, a[q], b[q]) : 0.f;
                }
                *reinterpret_cast<uint4 *>(sA + op_off(r, s * nd + d0, KE)) =
                    make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                               pack_bf16x2(v[6], v[7]));
            }
            if (ok) {
                float4 *dst = reinterpret_cast<float4 *>(A.ext + (o0 + r) * nd + d0);
                dst[0] = make_float4(tot[0], tot[1], tot[2], tot[3]);
                dst[1] = make_float4(tot[4], tot[5], tot[6], tot[7]);
            }
        }
        for (int e = tid; e < 128 * (KE - 7 * nd); e += kOctThreads)   // K padding
            *reinterpret_cast<__nv_bfloat16 *>(sA + op_off(e & 127, 7 * nd + (e >> 7), KE)) = __float2bfloat16_rn(0.f);
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tile + gridDim.x < A.ntiles) issue_loads(tile + gridDim.x);   // in flight during MMA + epilogue
        if (tid == 0) {
            bool ok = true;
            if (!weights_ready) ok = weights_ready = mbar_wait_bounded(&bar[0], 0, kMaxPolls);
            if (ok) {
                tc_fence_after();
                mma_steps(tbase, smem_u32(sA), KE, smem_u32(sB), KE, KE / 16, kH, false);
                umma_commit(&bar[1]);
                ok = mbar_wait_bounded(&bar[1], phase, kMaxPolls);
            }
            if (!ok) *sflag = 1;
        }
        phase ^= 1;
        __syncthreads();
        if (*sflag) break;
        tc_fence_after();
        // 4. h = D + b1 -> the B-operand blocks of the per-leaf kernel: block
        //    r / 16, element (n, r % 16); rows past the end are zero (a 0 x NaN
        //    in the product would poison a real row).  Warps w, w + 4, w + 8
        //    share TMEM lanes 32 (w % 4) .., taking columns 0-63, 64-95, 96-127.
        {
            const int quarter = warp & 3, part = warp >> 2;
            const int r = quarter * 32 + lane;
            unsigned char *blk = reinterpret_cast<unsigned char *>(sHb + (r >> 4) * kHBlock);
            const int cbeg = part == 0 ? 0 : part == 1 ? 64 : 96, cend = part == 0 ? 64 : part == 1 ? 96 : 128;
#pragma unroll 1
            for (int c0 = cbeg; c0 < cend; c0 += 32) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, v);
                tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int n = c0 + q;
                    const float hv = r < rows ? __uint_as_float(v[q]) + sB1[n] : 0.f;
                    *reinterpret_cast<__nv_bfloat16 *>(blk + op_off(n, r & 15, 16)) = __float2bfloat16_rn(hv);
                }
            }
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            const int nblk = (rows + 15) / 16;
            bulk_s2g(A.h + (o0 >> 4) * kHBlock, sHb, (uint32_t)(nblk * kHBlock * 2));
            bulk_commit();
        }
    }
    if (*sflag && tid == 0) {
        atomicExch(&g_ltc_fault, 1);
        mbar_wait_bounded(&bar[1], phase ^ 1, kMaxPolls);   // let an issued chain finish
    }
    if (tid == 0) bulk_wait_all<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 128);
    }
}

// ---- per-leaf part --------------------------------------------------------------

struct CellArgs {
    TcLayout T;
    const unsigned char *tc;
    int64_t n_leaf, ntiles;
    float dx_leaf, av_per_nh, c2;    // c2 = -shield_k av_per_nh log2(e)
    float dlo2, dhi2;                // trusted delta range x log2(e)
    const float *rho_leaf;           // Morton
    const float *kloc;               // [8][8][nd]
    const __nv_bfloat16 *h;          // layer-1 blocks
    const float *ext;                // [n_oct][nd]
    float *n_h, *a_v, *shield;
    int vec;                         // n_h is 16-byte aligned: a tile's rows leave as one bulk copy
};

constexpr int kCellThreads = 512;   // two groups of 256: two threads per leaf row, each half the columns

// Shared memory of learned_cell_tc.  Shared: the weight images, the one-hot
// block, the local-term operand B_loc [NP x 64] = dx K_loc[t][s][d] at
// k = 8 t + s, the cell standardisation.  Per group: the operand buffer (the
// leaf inputs [128 x KC] for MMA1, then the activations [128 x 128] for MMA2
// and MMA3, then the tile's N rows [128 x nd] FP32 on their way out), the
// local-term operand A_loc [128 x 64] (row m holds its oct's 8 densities in
// block t = m % 8, zero elsewhere), and two stages of the tile's inputs that
// bulk copies bring in one tile ahead (the 16 octs' layer-1 block, which MMA1
// reads in place, densities of the 128 leaves and external columns of their
// 16 octs).
struct CellSmem {
    size_t w1c, w2, w3, onehot, bloc, muc, sic, bar, grp, grp_stride, a, aloc, stage, stage_bytes, st_rho, st_ext,
        st_h, total;
};

__host__ __device__ inline CellSmem cell_smem(const TcLayout &T)
{
    CellSmem S;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t r = o; o = align128(o + bytes); return r; };
    S.w1c = take((size_t)kH * T.KC * 2);
    S.w2 = take((size_t)kH * kKW * 2);
    S.w3 = take((size_t)T.NP * kKW * 2);
    S.onehot = take((size_t)kHBlock * 2);
    S.bloc = take((size_t)T.NP * 64 * 2);
    S.muc = take((size_t)T.KC * 4);
    S.sic = take((size_t)T.KC * 4);
    S.bar = take(128);
    S.grp = o;
    S.a = 0;
    S.aloc = align128((size_t)128 * kH * 2);
    S.st_h = 0;
    S.st_rho = (size_t)kHBlock * 2;
    S.st_ext = S.st_rho + 128 * 4;
    S.stage_bytes = align128(S.st_ext + (size_t)16 * T.nd * 4);
    S.stage = S.aloc + (size_t)128 * 64 * 2;
    S.grp_stride = S.stage + 2 * S.stage_bytes;
    S.total = S.grp + 2 * S.grp_stride;
    return S;
}

// a tile's inputs: the layer-1 block, 128 densities, 16 external columns
__device__ __forceinline__ void prefetch_tile(const CellArgs &A, const CellSmem &S, int64_t tile, unsigned char *st,
                                              uint64_t *bar)
{
    const int64_t c0 = tile * 128;
    const int rows = (int)(A.n_leaf - c0 < 128 ? A.n_leaf - c0 : 128);   // a multiple of 8
    const uint32_t b_rho = (uint32_t)rows * 4, b_ext = (uint32_t)(rows / 8) * A.T.nd * 4, b_h = kHBlock * 2;
    mbar_expect_tx(bar, b_rho + b_ext + b_h);
    bulk_g2s(st + S.st_h, A.h + tile * kHBlock, b_h, bar);
    bulk_g2s(st + S.st_rho, A.rho_leaf + c0, b_rho, bar);
    bulk_g2s(st + S.st_ext, A.ext + (c0 >> 3) * A.T.nd, b_ext, bar);
}

__global__ void __launch_bounds__(kCellThreads, 1) learned_cell_tc(CellArgs A)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcLayout &T = A.T;
    const CellSmem S = cell_smem(T);
    const int nd = T.nd, KC = T.KC, NP = T.NP;
    const int tid = threadIdx.x, warp = tid >> 5;
    // group g (warps 8g .. 8g+7); row i (TMEM lane quarter warp % 4); half of the columns
    const int g = warp >> 3, quarter = warp & 3, half = (warp >> 2) & 1, i = quarter * 32 + (tid & 31);
    const bool lead = half == 0 && i == 0;     // issues the group's copies and MMAs
    const float *sMu = reinterpret_cast<const float *>(smem + S.muc);
    const float *sSi = reinterpret_cast<const float *>(smem + S.sic);
    // [0] weights, [1 + g] group MMAs, [3 + 2 g + stage] group input stages
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S.bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 7);
    int *sflag = reinterpret_cast<int *>(tslot + 1);                  // [2] per-group fault flags
    unsigned char *G = smem + S.grp + g * S.grp_stride;
    unsigned char *sOp = G + S.a;
    unsigned char *sAloc = G + S.aloc;
    __shared__ float sAcc[2 * 2 * 128];         // [group][half][row] screening partial sums

    if (tid == 0) {
        for (int b = 0; b < 7; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
        sflag[0] = sflag[1] = 0;
    }
    // B_loc[d][8 t + s] = dx K_loc[t][s][d] (directions past nd are zero)
    for (int e = tid; e < NP * 64; e += kCellThreads) {
        const int n = e >> 6, k = e & 63;
        const float v = n < nd ? A.dx_leaf * A.kloc[(k >> 3) * 8 * nd + (k & 7) * nd + n] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(smem + S.bloc + op_off(n, k, 64)) = __float2bfloat16_rn(v);
    }
    // A_loc starts all zero; each tile rewrites only its rows' own blocks
    for (int e = tid; e < 2 * 128 * 64 / 8; e += kCellThreads) {
        const int gg = e / (128 * 8), r = e % (128 * 8);
        reinterpret_cast<uint4 *>(smem + S.grp + gg * S.grp_stride + S.aloc)[r] = make_uint4(0, 0, 0, 0);
    }
    for (int k = tid; k < KC; k += kCellThreads) {
        reinterpret_cast<float *>(smem + S.muc)[k] = reinterpret_cast<const float *>(A.tc + T.muc)[k];
        reinterpret_cast<float *>(smem + S.sic)[k] = reinterpret_cast<const float *>(A.tc + T.sic)[k];
    }
    for (int e = tid; e < kHBlock; e += kCellThreads) {   // one-hot: row m selects column m / 8
        const int m = e >> 4, k = e & 15;
        *reinterpret_cast<__nv_bfloat16 *>(smem + S.onehot + op_off(m, k, 16)) =
            __float2bfloat16_rn(k == (m >> 3) ? 1.f : 0.f);
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(tslot, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;
    if (tid == 0) {
        const uint32_t b1 = (uint32_t)(kH * KC * 2), b2 = (uint32_t)(kH * kKW * 2), b3 = (uint32_t)(NP * kKW * 2);
        mbar_expect_tx(&bar[0], b1 + b2 + b3);
        bulk_g2s(smem + S.w1c, A.tc + T.w1c, b1, &bar[0]);
        bulk_g2s(smem + S.w2, A.tc + T.w2, b2, &bar[0]);
        bulk_g2s(smem + S.w3, A.tc + T.w3, b3, &bar[0]);
    }
    // per group 256 TMEM columns: D (128: D1, D2, D3 in turn, each read out
    // before the next chain) and the local term (NP columns, alive through the tile)
    const uint32_t tD = tbase + (uint32_t)(g * 256), tL = tD + 128;
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const uint32_t a_op = smem_u32(sOp), a_1h = smem_u32(smem + S.onehot);
    const int bid = 1 + g;                                               // named barrier of the group
    const int64_t first = 2 * (int64_t)blockIdx.x + g, stride = 2 * (int64_t)gridDim.x;
    bool weights_ready = false;
    uint32_t phase = 0, sphase[2] = {0, 0};
    bool pending[2] = {false, false};          // leader: a prefetch into the stage has not been waited for
    bool fault = false;
    if (lead && first < A.ntiles) {
        prefetch_tile(A, S, first, G + S.stage, &bar[3 + 2 * g]);
        pending[0] = true;
    }

    const bool bulk_out = A.n_h && A.vec;
    // leader of the group: issue, commit and wait (bounded); everyone learns
    // the outcome after the group barrier.  layer 0 = the local term.
    auto issue_and_wait = [&](int layer, uint32_t h_block) {
        if (lead) {
            // the previous tile's N rows must have left the operand buffer
            // before anyone writes it again (right after the local term)
            if (layer == 0 && bulk_out) bulk_wait_read<0>();
            bool ok = true;
            if (!weights_ready) ok = weights_ready = mbar_wait_bounded(&bar[0], 0, kMaxPolls);
            if (ok) {
                tc_fence_after();
                if (layer == 0) {
                    mma_steps(tL, smem_u32(sAloc), 64, smem_u32(smem + S.bloc), 64, 4, NP, false);
                } else if (layer == 1) {
                    mma_steps(tD, a_op, KC, smem_u32(smem + S.w1c), KC, KC / 16, kH, false);
                    mma_steps(tD, a_1h, 16, h_block, 16, 1, kH, true);
                } else {
                    const uint32_t w = smem_u32(smem + (layer == 2 ? S.w2 : S.w3));
                    const int N = layer == 2 ? kH : NP;
                    mma_steps(tD, a_op, kH, w, kKW, kH / 16, N, false);
                    mma_steps(tD, a_1h, 16, w + (kH / 16) * 256, kKW, 1, N, true);
                }
                umma_commit(&bar[1 + g]);
                ok = mbar_wait_bounded(&bar[1 + g], phase, kMaxPolls);
            }
            if (!ok) sflag[g] = 1;
        }
        phase ^= 1;
        named_barrier(bid, 256);
        fault = sflag[g] != 0;
        tc_fence_after();
    };

    // GELU of a 128-column accumulator row -> the operand buffer; two 32-column
    // loads in flight per wait
    auto gelu_row = [&]() {
#pragma unroll 1
        for (int c = 64 * half; c < 64 * half + 64; c += 32) {
            uint32_t v[32];
            tmem_ld32(tD + lane_off + (uint32_t)c, v);
            tmem_ld_wait();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t o[4];
#pragma unroll
                for (int p2 = 0; p2 < 4; ++p2)
                    o[p2] = gelu_bf16x2(pack_bf16x2(__uint_as_float(v[8 * q + 2 * p2]),
                                                    __uint_as_float(v[8 * q + 2 * p2 + 1])));
                *reinterpret_cast<uint4 *>(sOp + op_off(i, c + 8 * q, kH)) = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
    };
    // the row's 8-direction groups this thread takes: [gq0, gq1) of nd / 8
    const int ngq = nd >> 3, gq0 = half * ((ngq + 1) >> 1), gq1 = half ? ngq : (ngq + 1) >> 1;

    int stg = 0;
    for (int64_t tile = first; tile < A.ntiles && !fault; tile += stride, stg ^= 1) {
        const int64_t c0 = tile * 128;
        const int rows = (int)std::min<int64_t>(128, A.n_leaf - c0);
        const int64_t m = c0 + i;
        const bool valid = i < rows;
        unsigned char *st = G + S.stage + stg * S.stage_bytes;
        // the next tile's inputs go to the other stage (its last reader was the
        // previous tile, finished at that tile's final barrier); the previous
        // tile's N rows must have left the operand buffer
        if (lead) {
            if (tile + stride < A.ntiles) {
                prefetch_tile(A, S, tile + stride, G + S.stage + (stg ^ 1) * S.stage_bytes,
                              &bar[3 + 2 * g + (stg ^ 1)]);
                pending[stg ^ 1] = true;
            }
            if (mbar_wait_bounded(&bar[3 + 2 * g + stg], sphase[stg], kMaxPolls)) pending[stg] = false;
            else sflag[g] = 1;
        }
        sphase[stg] ^= 1;
        named_barrier(bid, 256);
        if (sflag[g]) {
            fault = true;
            break;
        }
        const float *sR = reinterpret_cast<const float *>(st + S.st_rho);
        const float *sE = reinterpret_cast<const float *>(st + S.st_ext) + (i >> 3) * nd;

        // ---- local term on the tensor cores: A_loc row = the oct's 8 densities ----
        if (half == 0) {
            const float4 r0 = *reinterpret_cast<const float4 *>(sR + (i & ~7));
            const float4 r1 = *reinterpret_cast<const float4 *>(sR + (i & ~7) + 4);
            const uint4 w = valid ? make_uint4(pack_bf16x2(r0.x, r0.y), pack_bf16x2(r0.z, r0.w),
                                               pack_bf16x2(r1.x, r1.y), pack_bf16x2(r1.z, r1.w))
                                  : make_uint4(0, 0, 0, 0);
            *reinterpret_cast<uint4 *>(sAloc + op_off(i, 8 * (i & 7), 64)) = w;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 256);
        issue_and_wait(0, 0);
        if (fault) break;

        // ---- u_cell = standardised ln(local term) (8 directions per 16-byte
        //      store), then ln n and the K padding ----
#pragma unroll 1
        for (int q = gq0; q < gq1; ++q) {
            const int d0 = 8 * q;
            uint32_t v[8];
            tmem_ld8(tL + lane_off + (uint32_t)d0, v);
            tmem_ld_wait();
            const float4 a0 = *reinterpret_cast<const float4 *>(sMu + d0), a1 = *reinterpret_cast<const float4 *>(sMu + d0 + 4);
            const float4 b0 = *reinterpret_cast<const float4 *>(sSi + d0), b1 = *reinterpret_cast<const float4 *>(sSi + d0 + 4);
            const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
            float u[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) u[j] = valid ? std_input(__uint_as_float(v[j]), kCFloor, a[j], b[j]) : 0.f;
            *reinterpret_cast<uint4 *>(sOp + op_off(i, d0, KC)) =
                make_uint4(pack_bf16x2(u[0], u[1]), pack_bf16x2(u[2], u[3]), pack_bf16x2(u[4], u[5]),
                           pack_bf16x2(u[6], u[7]));
        }
        for (int d0 = nd + 8 * half; d0 < KC; d0 += 16) {      // ln n at column nd, zeros after it
            const float un = valid && d0 == nd ? std_input(sR[i], kNFloor, sMu[nd], sSi[nd]) : 0.f;
            *reinterpret_cast<uint4 *>(sOp + op_off(i, d0, KC)) = make_uint4(pack_bf16x2(un, 0.f), 0, 0, 0);
        }
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 256);
        issue_and_wait(1, smem_u32(st + S.st_h));
        if (fault) break;

        // ---- a1 = gelu(D1) (D1 includes h[oct] + b1) ----
        gelu_row();
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 256);
        issue_and_wait(2, 0);
        if (fault) break;

        // ---- a2 = gelu(D2) (D2 includes b2; MMA2 has finished reading a1) ----
        gelu_row();
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 256);
        issue_and_wait(3, 0);
        if (fault) break;

        // ---- N = (local + external) 2^D3 -> the operand buffer as FP32 rows; shield ----
        {
            float *nrow = reinterpret_cast<float *>(sOp) + (size_t)i * nd;
            float *av = A.a_v && valid ? A.a_v + m * nd : nullptr;
            float *nh = A.n_h && valid && !bulk_out ? A.n_h + m * nd : nullptr;
            float acc = 0.f;
#pragma unroll 1
            for (int q8 = gq0; q8 < gq1; ++q8) {
                const int c = 8 * q8;
                uint32_t v[8], w[8];
                tmem_ld8(tD + lane_off + (uint32_t)c, v);
                tmem_ld8(tL + lane_off + (uint32_t)c, w);
                tmem_ld_wait();
#pragma unroll
                for (int j4 = 0; j4 < 8; j4 += 4) {
                    const float4 e4 = *reinterpret_cast<const float4 *>(sE + c + j4);
                    const float ev[4] = {e4.x, e4.y, e4.z, e4.w};
                    float N[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const float dl = __uint_as_float(v[j4 + q]);
                        const float nt = __uint_as_float(w[j4 + q]) + ev[q];
                        N[q] = isfinite(dl) && dl >= A.dlo2 && dl <= A.dhi2 ? nt * fast_exp2(dl) : nt;
                        acc += fast_exp2(A.c2 * N[q]);
                    }
                    *reinterpret_cast<float4 *>(nrow + c + j4) = make_float4(N[0], N[1], N[2], N[3]);
                    if (nh)
#pragma unroll
                        for (int q = 0; q < 4; ++q) nh[c + j4 + q] = N[q];
                    if (av)
#pragma unroll
                        for (int q = 0; q < 4; ++q) av[c + j4 + q] = N[q] * A.av_per_nh;
                }
            }
            sAcc[(g * 2 + half) * 128 + i] = acc;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 256);     // the stage is rewritten by later tiles
        // the row's screening factor: the two halves' sums, in a fixed order
        if (half == 0 && A.shield && valid) A.shield[m] = (sAcc[(g * 2) * 128 + i] + sAcc[(g * 2 + 1) * 128 + i]) / (float)nd;
        if (bulk_out && lead) {
            bulk_s2g(A.n_h + c0 * nd, sOp, (uint32_t)(rows * nd * 4));
            bulk_commit();
        }
    }
    if (fault && lead) {
        atomicExch(&g_ltc_fault, 1);
        mbar_wait_bounded(&bar[1 + g], phase ^ 1, kMaxPolls);   // let an issued chain finish
    }
    // a prefetch still in flight must land, and the output copies must have
    // read the operand buffer, before the CTA exits
    if (lead) {
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait_bounded(&bar[3 + 2 * g + b], sphase[b], kMaxPolls);
        bulk_wait_all<0>();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    }
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

int max_smem_optin()
{
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// Packs the BF16 operands when the master weights changed since the last pack.
cd_status ensure_packed(cd_net net, cudaStream_t s)
{
    TcState *st = static_cast<TcState *>(net->tc);
    if (!st) {
        st = new TcState();
        st->lay = make_layout(net->lay.nd);
        if (cudaMalloc(&st->buf, st->lay.total) != cudaSuccess) {
            cudaGetLastError();
            delete st;
            set_error("cannot allocate the packed tensor-core weights");
            return CD_ENOMEM;
        }
        net->tc = st;
        net->tc_version = 0;
    }
    if (net->tc_version == net->version) return CD_OK;
    PackArgs P;
    P.T = st->lay;
    P.p = net->p;
    P.mu = net->mu;
    P.sinv = net->sinv;
    P.N = net->lay;
    P.buf = st->buf;
    LaunchScope ls(CD_K_NET, s);
    pack_tc<<<num_sms() * 4, 256, 0, s>>>(P);
    CD_CHECK_LAUNCH();
    net->tc_version = net->version;
    return CD_OK;
}

}  // namespace

bool learned_tc_supported(int nd, int hidden) { return hidden == kH && nd >= 8 && nd <= kMaxNd && nd % 8 == 0; }

cd_status column_density_learned_tc(cd_tree t, cd_geom g, const cd_opts &o, float *n_h, float *a_v, float *shield,
                                    cudaStream_t s)
{
    cd_net net = (cd_net)o.net;
    const int nd = g->n_dir;
    if (!learned_tc_supported(nd, net->lay.H)) {
        set_error("the BF16 learned form needs hidden = %d and n_dir a multiple of 8 up to %d (got %d, %d); "
                  "use CD_FP32", kH, kMaxNd, net->lay.H, nd);
        return CD_EUNSUPPORTED;
    }
    if (t->L < 2) {
        set_error("the BF16 learned form needs at least two tree levels");
        return CD_EUNSUPPORTED;
    }
    const int sms = num_sms(), smax = max_smem_optin();
    const TcLayout lay = make_layout(nd);
    const size_t smem_oct = oct_smem(lay), smem_cell = cell_smem(lay).total;
    if ((int)smem_oct > smax || (int)smem_cell > smax) {
        set_error("the learned kernels need %zu / %zu bytes of shared memory, the device offers %d", smem_oct,
                  smem_cell, smax);
        return CD_EUNSUPPORTED;
    }
    cd_status st = ensure_level_sums(t, g, CD_BF16, s);
    if (st != CD_OK) return st;
    if ((st = ensure_packed(net, s)) != CD_OK) return st;
    TcState *ts = static_cast<TcState *>(net->tc);
    const TcLayout &T = ts->lay;
    const int64_t n_blocks = (t->n_oct + 15) / 16;
    if (ts->cap < t->n_oct) {
        if (ts->h) cd::lib_free(ts->h);
        if (ts->ext) cd::lib_free(ts->ext);
        ts->h = nullptr;
        ts->ext = nullptr;
        ts->cap = 0;
        if (cudaMalloc(&ts->h, (size_t)n_blocks * kHBlock * 2) != cudaSuccess ||
            cudaMalloc(&ts->ext, (size_t)t->n_oct * nd * 4) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate the per-oct buffers of the learned form");
            return CD_ENOMEM;
        }
        ts->cap = t->n_oct;
    }
    {
        OctArgs A = {};
        A.T = T;
        A.tc = ts->buf;
        A.n_oct = t->n_oct;
        A.ntiles = (t->n_oct + 127) / 128;
        A.L = t->L;
        for (int i = 0; i < 4; ++i) A.Et[i] = t->lv.Et[i];
        for (int k = 0; k <= CD_MAXL; ++k) A.C[k] = t->lv.C[k];
        A.h = ts->h;
        A.ext = ts->ext;
        CD_CUDA(cudaFuncSetAttribute(learned_oct_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_oct));
        const int grid = (int)std::min<int64_t>(A.ntiles, sms);
        LaunchScope ls(CD_K_NET, s);
        learned_oct_tc<<<grid, kOctThreads, smem_oct, s>>>(A);
        CD_CHECK_LAUNCH();
    }
    {
        CellArgs A = {};
        A.T = T;
        A.tc = ts->buf;
        A.n_leaf = t->n_leaf;
        A.ntiles = (t->n_leaf + 127) / 128;
        A.dx_leaf = (float)(t->box_cm / (double)((int64_t)1 << t->L));
        A.av_per_nh = (float)o.av_per_nh;
        A.c2 = (float)(-o.shield_k * o.av_per_nh * 1.4426950408889634);
        A.dlo2 = (float)((double)net->dlo * 1.4426950408889634);
        A.dhi2 = (float)((double)net->dhi * 1.4426950408889634);
        A.rho_leaf = t->rho_leaf;
        A.kloc = g->kloc;
        A.h = ts->h;
        A.ext = ts->ext;
        A.n_h = n_h;
        A.a_v = a_v;
        A.shield = shield;
        A.vec = (uintptr_t)n_h % 16 == 0;
        CD_CUDA(cudaFuncSetAttribute(learned_cell_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_cell));
        const int grid = (int)std::min<int64_t>((A.ntiles + 1) / 2, sms);
        LaunchScope ls(CD_K_LEARNED, s);
        learned_cell_tc<<<grid, kCellThreads, smem_cell, s>>>(A);
        CD_CHECK_LAUNCH();
    }
    return CD_OK;
}

cd_status learned_tc_fault_check()
{
    int v = 0;
    CD_CUDA(cudaMemcpyFromSymbol(&v, g_ltc_fault, sizeof(int)));
    if (v) {
        const int zero = 0;
        CD_CUDA(cudaMemcpyToSymbol(g_ltc_fault, &zero, sizeof(int)));
        set_error("a learned tensor-core kernel gave up a bounded wait");
        return CD_ETIMEOUT;
    }
    return CD_OK;
}

void net_free_tc(cd_net net)
{
    TcState *st = static_cast<TcState *>(net->tc);
    if (!st) return;
    if (st->buf) cd::lib_free(st->buf);
    if (st->h) cd::lib_free(st->h);
    if (st->ext) cd::lib_free(st->ext);
    delete st;
    net->tc = nullptr;
}

}  // namespace cd
