// Per-leaf combine and epilogue (§3.2 internal + local contributions; Eqs.
// eq_chi / chi_discret for the direction average):
//   N_H[t][d] = E[oct][d] + Sp[oct / 8][d] + sum_s rho_leaf[oct][s] dx_L Kloc[t][s][d]
//   A_V = N_H av_per_nh,   shield[t] = (1/nd) sum_d exp(-k A_V)
// This kernel writes the N_H array, the dominant HBM traffic of the path
// (4 bytes per cell-direction), so it is built as a streaming pipeline:
//
//   - persistent CTAs, each walking batches of B consecutive octs (Morton
//     order, so every batch is one contiguous span of E, rho and N_H);
//   - E, Sp and rho of the next batch arrive by bulk asynchronous copies (TMA,
//     cp.async.bulk) into a double-buffered shared-memory stage, completed on
//     an mbarrier, while the current batch is computed;
//   - every thread owns one fixed (child t, four directions) slot of the oct,
//     so its 8 x 4 local weights sit in registers for the whole kernel;
//   - results are staged in shared memory in output layout and leave by bulk
//     stores, so HBM sees full-line writes;
//   - the direction sum of the screening factor goes through a shared-memory
//     partial array (no atomics).
// A generic one-thread-per-leaf kernel covers direction counts that are not a
// multiple of four and unaligned output pointers.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "ptx.cuh"

namespace cd {
namespace {

constexpr uint32_t kMaxPolls = 1u << 26;   // bounded mbarrier waits (seconds at worst)

static __device__ int g_leaf_fault;         // set when a bounded wait gives up

constexpr int kLoadStages = 4;             // E / rho batches in flight per CTA

struct LeafTmaArgs {
    LeafLaunch a;
    int G;           // thread groups; one group = 2 nd threads = one oct at a time
    int B;           // octs per batch
    int prows;       // parent rows a batch can touch: B / 8 + 2
    int64_t nbatch;
    float c_exp2;    // base-2 exponent per unit N_H: -shield_k * av_per_nh * log2(e)
    float inv_nd;
};

// W = lanes pre-reduced by shuffles before the shared-memory add of the
// screening sum (a leaf's 4-direction slots are W-aligned runs of lanes).
// W = lanes pre-reduced by shuffles before a leaf's screening partial goes to
// shared memory (a leaf's 4-direction slots are W-aligned runs of lanes).  The
// partials of batch i are summed in a fixed order while batch i+1 is computed
// and their store trails the N_H store by one batch, so results are bitwise
// reproducible with two barriers per batch.
// ND > 0 fixes the direction count at compile time (every offset folds to an
// immediate); ND = 0 reads it from the arguments.
template <int ND, int W>
__global__ void __launch_bounds__(384, 2) leaf_tma(LeafTmaArgs P)
{
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int kG = ND ? (384 / (2 * ND) > 1 ? 384 / (2 * ND) : 1) : 0;
    const int nd = ND ? ND : P.a.nd;
    const int G = ND ? kG : P.G;
    const int B = ND ? 4 * kG : P.B;
    const int prows = ND ? (4 * kG) / 8 + 2 : P.prows;
    const int q4 = nd >> 2, slots = 2 * nd, pw = slots / W, lw = q4 / W;
    const bool want_nh = P.a.n_h != nullptr, want_sh = P.a.shield != nullptr;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
    float *Eb = reinterpret_cast<float *>(smem + 128);      // [kLoadStages][B nd]
    float *Rb = Eb + kLoadStages * B * nd;                  // [kLoadStages][B 8]
    float *Pb = Rb + kLoadStages * B * 8;                   // [kLoadStages][(B/8 + 2) nd] parent rows
    float *Sb = Pb + kLoadStages * prows * nd;              // [3][B 8]
    float *part = Sb + 3 * B * 8;                           // [2][B][slots / W]
    float *Ob = part + 2 * B * pw;                          // [2][B 8 nd]

    const int tid = threadIdx.x;
    const int g = tid / slots, r = tid - g * slots;
    const int t = r / q4, d0 = 4 * (r - t * q4);
    // dx_L * Kloc[t][s][d0 + i] for sibling pairs j = (2j, 2j+1) and directions i
    float2 KP[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i)
            KP[j][i] = make_float2(P.a.dx_leaf * P.a.kloc[(t * 8 + 2 * j) * nd + d0 + i],
                                   P.a.dx_leaf * P.a.kloc[(t * 8 + 2 * j + 1) * nd + d0 + i]);

    // this thread's offsets in the stages (oct g of the batch) and the strides
    // to its next octs g + G, g + 2G, g + 3G (B = 4G)
    const bool has_E = P.a.E != nullptr, has_Sp = P.a.Sp != nullptr;
    const int eoff = g * nd + d0, roff = g * 8, ooff = (g * 8 + t) * nd + d0, poff = g * pw + r / W;
    const int sE = G * nd, sR = G * 8, sO = G * 8 * nd, sP = G * pw;

    const int64_t n_oct = P.a.n_oct;
    const int64_t first = blockIdx.x, stride = gridDim.x;
    const int n_iter = first < P.nbatch ? (int)((P.nbatch - first + stride - 1) / stride) : 0;
    auto batch_o0 = [&](int it) { return (first + (int64_t)it * stride) * B; };
    auto batch_nb = [&](int it) {
        const int64_t o0 = batch_o0(it);
        return (int)(n_oct - o0 < (int64_t)B ? n_oct - o0 : (int64_t)B);
    };

    auto issue = [&](int it) {
        const int st = it % kLoadStages;
        const int64_t o0 = batch_o0(it);
        const int nb = batch_nb(it);
        const uint32_t eb = P.a.E ? (uint32_t)nb * nd * 4 : 0u;
        const int64_t p0 = o0 >> 3;
        const uint32_t pb = P.a.Sp ? (uint32_t)(((o0 + nb - 1) >> 3) - p0 + 1) * nd * 4 : 0u;
        // checked builds: a batch outside the octs (or their parents) copies nothing
        if (!(in_bounds(o0, n_oct, kCheckLeafIn) && in_bounds(o0 + nb - 1, n_oct, kCheckLeafIn) &&
              (!P.a.Sp || in_bounds((o0 + nb - 1) >> 3, (n_oct + 7) / 8, kCheckLeafIn)))) {
            mbar_expect_tx(&bar[st], 0);
            return;
        }
        mbar_expect_tx(&bar[st], eb + pb + (uint32_t)nb * 32);
        if (P.a.E) bulk_g2s(Eb + st * B * nd, P.a.E + o0 * nd, eb, &bar[st]);
        if (P.a.Sp) bulk_g2s(Pb + st * prows * nd, P.a.Sp + p0 * nd, pb, &bar[st]);
        bulk_g2s(Rb + st * B * 8, P.a.rho_leaf + o0 * 8, (uint32_t)nb * 32, &bar[st]);
    };
    // screening factor of batch `it` from its partials, in a fixed order
    auto shield_sum = [&](int it) {
        const float *pp = part + (it & 1) * B * pw;
        float *S = Sb + (it % 3) * B * 8;
        for (int j = tid; j < batch_nb(it) * 8; j += blockDim.x) {
            const float *p = pp + (j >> 3) * pw + (j & 7) * lw;
            float acc = 0.f;
            for (int q = 0; q < lw; ++q) acc += p[q];
            S[j] = acc * P.inv_nd;
        }
    };

    if (tid == 0) {
        for (int s = 0; s < kLoadStages; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
        for (int it = 0; it < kLoadStages - 1 && it < n_iter; ++it) issue(it);
    }
    __syncthreads();

    int it = 0;
    bool fault = false;
    for (; it < n_iter; ++it) {
        const int ls = it % kLoadStages, os = it & 1;
        if (tid == 0) {
            if (it + kLoadStages - 1 < n_iter) issue(it + kLoadStages - 1);
            bulk_wait_read<1>();   // stores issued two iterations ago have read O[os] and their S
        }
        // one thread polls; the others sleep in the hardware barrier
        bool ok = true;
        if (tid == 0) ok = mbar_wait_bounded(&bar[ls], (it / kLoadStages) & 1, kMaxPolls);
        if (__syncthreads_or(!ok)) {
            fault = true;
            break;
        }
        if (want_sh && it > 0) shield_sum(it - 1);

        const int64_t o0 = batch_o0(it);
        const int nb = batch_nb(it);
        // 32-bit shared-memory bases of this thread's slot in every stage
        const float *E = Eb + ls * B * nd + eoff;
        const float *Spr = Pb + ls * prows * nd + d0;
        const float *R = Rb + ls * B * 8 + roff;
        float *O = Ob + os * B * 8 * nd + ooff;
        float *pp = part + (it & 1) * B * pw + poff;
        const int par0 = (int)(o0 & 7);           // parent row of oct b: (par0 + b) >> 3
        float *AV = P.a.a_v ? P.a.a_v + o0 * 8 * nd + ooff : nullptr;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = g + k * G;
            const bool live = nb == B || b < nb;
            float2 n01 = make_float2(0.f, 0.f), n23 = make_float2(0.f, 0.f);
            if (live) {
                if (has_E) {
                    const float4 e4 = *reinterpret_cast<const float4 *>(E + k * sE);
                    n01 = make_float2(e4.x, e4.y);
                    n23 = make_float2(e4.z, e4.w);
                }
                if (has_Sp) {
                    const float4 p4 = *reinterpret_cast<const float4 *>(Spr + ((par0 + b) >> 3) * nd);
                    n01 = __fadd2_rn(n01, make_float2(p4.x, p4.y));
                    n23 = __fadd2_rn(n23, make_float2(p4.z, p4.w));
                }
                const float4 r0 = *reinterpret_cast<const float4 *>(R + k * sR);
                const float4 r1 = *reinterpret_cast<const float4 *>(R + k * sR + 4);
                // packed FP32x2 FMAs over sibling pairs (s, s+1): acc[i] holds the
                // even- and odd-sibling partial sums of direction d0 + i
                const float2 rp[4] = {make_float2(r0.x, r0.y), make_float2(r0.z, r0.w), make_float2(r1.x, r1.y),
                                      make_float2(r1.z, r1.w)};
                float2 acc[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    acc[i] = __fmul2_rn(rp[0], KP[0][i]);
#pragma unroll
                    for (int j = 1; j < 4; ++j) acc[i] = __ffma2_rn(rp[j], KP[j][i], acc[i]);
                }
                n01.x += acc[0].x + acc[0].y;
                n01.y += acc[1].x + acc[1].y;
                n23.x += acc[2].x + acc[2].y;
                n23.y += acc[3].x + acc[3].y;
                if (want_nh) *reinterpret_cast<float4 *>(O + k * sO) = make_float4(n01.x, n01.y, n23.x, n23.y);
                if (AV) {
                    const float2 a2 = make_float2(P.a.av_per_nh, P.a.av_per_nh);
                    const float2 x = __fmul2_rn(n01, a2), y = __fmul2_rn(n23, a2);
                    *reinterpret_cast<float4 *>(AV + k * sO) = make_float4(x.x, x.y, y.x, y.y);
                }
            }
            if (want_sh) {
                // exp(-k A_V) = 2^(c2 N_H), c2 = -k av log2(e) precomputed on the host
                const float2 c2 = make_float2(P.c_exp2, P.c_exp2);
                const float2 a = __fmul2_rn(c2, n01), bb = __fmul2_rn(c2, n23);
                float e = (exp2f(a.x) + exp2f(a.y)) + (exp2f(bb.x) + exp2f(bb.y));
#pragma unroll
                for (int w = 1; w < W; w <<= 1) e += __shfl_xor_sync(0xffffffffu, e, w);
                pp[k * sP] = e;
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            if (want_nh) bulk_s2g(P.a.n_h + o0 * 8 * nd, O, (uint32_t)nb * 32 * nd);
            if (want_sh && it > 0)
                bulk_s2g(P.a.shield + batch_o0(it - 1) * 8, Sb + ((it - 1) % 3) * B * 8, (uint32_t)batch_nb(it - 1) * 32);
            bulk_commit();
        }
    }
    if (!fault && want_sh && n_iter > 0) {
        // the last batch's screening factor
        if (tid == 0) bulk_wait_read<1>();
        __syncthreads();
        shield_sum(n_iter - 1);
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            bulk_s2g(P.a.shield + batch_o0(n_iter - 1) * 8, Sb + ((n_iter - 1) % 3) * B * 8,
                     (uint32_t)batch_nb(n_iter - 1) * 32);
            bulk_commit();
        }
    }
    if (tid == 0) {
        if (fault) {
            atomicExch(&g_leaf_fault, 1);
            // let the loads already issued land before shared memory is released
            for (int j = it; j < it + kLoadStages - 1 && j < n_iter; ++j)
                mbar_wait_bounded(&bar[j % kLoadStages], (j / kLoadStages) & 1, kMaxPolls);
        }
        bulk_wait_all<0>();
    }
}

// One thread per leaf; any direction count and alignment.
__global__ void __launch_bounds__(256) leaf_generic(LeafLaunch P, float c_exp, float inv_nd)
{
    extern __shared__ float s_k[];   // [8 s][nd][8 t], times dx
    const int nd = P.nd;
    for (int i = threadIdx.x; i < 64 * nd; i += blockDim.x) {
        const int t = i & 7, sd = i >> 3, s = sd / nd, d = sd - s * nd;
        s_k[i] = P.dx_leaf * P.kloc[(t * 8 + s) * nd + d];
    }
    __syncthreads();
    const int64_t n_leaf = P.n_oct * 8;
    for (int64_t leaf = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; leaf < n_leaf;
         leaf += (int64_t)gridDim.x * blockDim.x) {
        const int64_t oct = leaf >> 3;
        const int t = (int)(leaf & 7);
        float rs[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) rs[s] = P.rho_leaf[oct * 8 + s];
        float acc = 0.f;
        for (int d = 0; d < nd; ++d) {
            float n = P.E ? P.E[oct * nd + d] : 0.f;
            if (P.Sp) n += P.Sp[(oct >> 3) * nd + d];
#pragma unroll
            for (int s = 0; s < 8; ++s) n = fmaf(rs[s], s_k[(s * nd + d) * 8 + t], n);
            if (P.n_h) P.n_h[leaf * nd + d] = n;
            if (P.a_v) P.a_v[leaf * nd + d] = n * P.av_per_nh;
            acc += __expf(c_exp * n);
        }
        if (P.shield) P.shield[leaf] = acc * inv_nd;
    }
}

struct DevInfo {
    int sms = 0;
};
std::mutex g_mu;
DevInfo g_dev[64];

int sm_count()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 152;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev[dev].sms) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_dev[dev].sms = n > 0 ? n : 152;
    }
    return g_dev[dev].sms;
}

bool aligned16(const void *p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

}  // namespace

cd_status launch_leaf(const LeafLaunch &a, cudaStream_t s)
{
    const int nd = a.nd;
    const float c_exp = -a.shield_k * a.av_per_nh;
    const float inv_nd = 1.0f / (float)nd;
    const bool tma = (nd % 4 == 0) && 2 * nd <= 384 && aligned16(a.n_h) && aligned16(a.a_v) &&
                     aligned16(a.shield) && aligned16(a.E) && aligned16(a.Sp) && aligned16(a.rho_leaf);
    if (tma) {
        const int W = 1;
        auto kern = nd == 48 ? leaf_tma<48, 1> : nd == 12 ? leaf_tma<12, 1> : leaf_tma<0, 1>;
        LeafTmaArgs P;
        P.a = a;
        P.G = std::max(1, 384 / (2 * nd));
        P.B = 4 * P.G;
        P.prows = P.B / 8 + 2;
        P.nbatch = (a.n_oct + P.B - 1) / P.B;
        P.c_exp2 = (float)(-(double)a.shield_k * (double)a.av_per_nh * 1.4426950408889634);
        P.inv_nd = inv_nd;
        const int threads = P.G * 2 * nd;
        const size_t smem = 128 + sizeof(float) * ((size_t)kLoadStages * (P.B * (nd + 8) + (size_t)P.prows * nd) + 3 * P.B * 8 +
                                                   (size_t)2 * P.B * (2 * nd / W) +
                                                   (a.n_h ? (size_t)2 * P.B * 8 * nd : 0));
        CD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        CD_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem));
        if (per_sm < 1) per_sm = 1;
        const int64_t grid = std::min<int64_t>(P.nbatch, (int64_t)per_sm * sm_count());
        LaunchScope ls(CD_K_LEAF, s);
        kern<<<(unsigned)grid, threads, smem, s>>>(P);
        CD_CHECK_LAUNCH();
        return CD_OK;
    }
    const size_t smem = sizeof(float) * 64 * nd;
    if (smem > 48 * 1024) {
        CD_CUDA(cudaFuncSetAttribute(leaf_generic, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    int64_t blocks = (a.n_oct * 8 + 255) / 256;
    blocks = std::min<int64_t>(blocks, (int64_t)sm_count() * 8);
    LaunchScope ls(CD_K_LEAF, s);
    leaf_generic<<<(unsigned)std::max<int64_t>(blocks, 1), 256, smem, s>>>(a, c_exp, inv_nd);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

// Returns CD_ETIMEOUT (and clears the flag) if a leaf kernel gave up a wait.
cd_status leaf_fault_check()
{
    int v = 0;
    CD_CUDA(cudaMemcpyFromSymbol(&v, g_leaf_fault, sizeof(int)));
    if (v) {
        const int zero = 0;
        CD_CUDA(cudaMemcpyToSymbol(g_leaf_fault, &zero, sizeof(int)));
        set_error("a leaf kernel gave up waiting for its input copies");
        return CD_ETIMEOUT;
    }
    return CD_OK;
}

}  // namespace cd
