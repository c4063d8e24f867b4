// Per-leaf combine and epilogue of the BF16 form, with the internal + local
// term (§3.2) on the tensor cores:
//   loc[t][d] = dx_L sum_s rho[oct][s] Kloc[t][s][d]
// is one small product per tile of 128 leaves (16 octs).  Row m of the A
// operand holds the oct's eight densities (BF16) in the block of its own
// octant t = m % 8 (K = 8 blocks x 8; zeros elsewhere, written once);
// B[d][8 t + s] = dx_L Kloc[t][s][d] in BF16.  The product lands in TMEM
// (FP32): the local term carries at most 2^-8 relative error from the two
// roundings, which enters N_H weighted by its share of the column (measured:
// the BF16 path's largest N_H error is unchanged).  The epilogue adds the oct's
// external column E and the parent's far-shell prefix Sp (§3.3), forms the
// screening factor (Eqs. eq_chi, chi_discret) and stages the tile's N_H rows
// for one bulk store.
//
// Tiles are 128 consecutive leaves in Morton order, so E, Sp, the densities and
// the N_H rows of a tile are contiguous spans; bulk copies bring the next
// tile's inputs in while the current one is computed.  Groups of four warps
// (four per CTA when shared memory allows) work on independent tiles so that
// one group's epilogue overlaps another's MMA.  Every wait is bounded; a
// timeout sets a device flag (cd_device_status).
#include <algorithm>
#include <atomic>
#include <string.h>

#include "common.cuh"
#include "umma.cuh"

namespace cd {
namespace {

constexpr uint32_t kMaxPolls = 1u << 26;
constexpr int kK = 64;                  // 8 octant blocks x 8 siblings

static __device__ int g_leaftc_fault;
// cd_debug_wait_polls: < 0 = the default limit
static std::atomic<int64_t> g_pipe_polls{-1};
// cd_debug_leaf_span: list tiles stage their parents' prefix rows as one span
// of up to this many rows (else one row per oct)
constexpr int kSpanRows = 16;
static std::atomic<int> g_span_max{kSpanRows};

__host__ __device__ constexpr size_t align128(size_t v) { return (v + 127) & ~(size_t)127; }
__host__ __device__ constexpr int round16(int v) { return (v + 15) & ~15; }

__host__ __device__ inline uint32_t op_off(int row, int k, int K)
{
    return (uint32_t)((row >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

struct LeafTcArgs {
    LeafLaunch a;
    int NP, G;                 // padded directions (MMA N), groups of 128 threads
    int64_t n_leaf, ntiles;
    float c2;                  // -shield_k av_per_nh log2(e)
    int out_bulk;              // n_h is 16-byte aligned: tile rows leave by bulk copies
    int list;                  // AMR list mode (a.oleaf): tiles of 16 octs, rows scattered
    uint32_t pipe_polls;       // poll limit of the pipeline waits (cd_debug_wait_polls); the exit
                               // waits for the CTA's own copies and products keep kMaxPolls
    int form;                  // kForm* bits; batched: the same for every job of the launch
    int span_max;              // list tiles with Sp: the widest parent span staged as one copy (<= 16)
};

// what a leaf row reads and writes: the parent prefix, staged rows (bulk
// stores) or direct n_h rows, A_V, the screening factor, list tiles
constexpr int kFormSp = 1, kFormBulk = 2, kFormNh = 4, kFormAv = 8, kFormShield = 16, kFormList = 32;

__host__ __device__ inline int leaf_form(const LeafLaunch &a, bool out_bulk, bool list)
{
    return (a.Sp ? kFormSp : 0) | (out_bulk ? kFormBulk : (a.n_h ? kFormNh : 0)) | (a.a_v ? kFormAv : 0) |
           (a.shield ? kFormShield : 0) | (list ? kFormList : 0);
}

struct LeafTcSmem {
    size_t bloc, bar, grp, grp_stride, aloc, out, stage, stage_bytes, st_e, st_p, st_r, st_l, total;
};

__host__ __device__ inline LeafTcSmem leaf_tc_smem(int nd, int NP, int G, bool list)
{
    LeafTcSmem S;
    size_t o = 0;
    auto take = [&](size_t bytes) { const size_t r = o; o = align128(o + bytes); return r; };
    S.bloc = take((size_t)NP * kK * 2);
    S.bar = take(128);
    S.grp = o;
    S.aloc = 0;
    S.out = align128((size_t)128 * kK * 2);
    S.st_e = 0;
    S.st_p = align128((size_t)16 * nd * 4);
    S.st_r = S.st_p + align128((size_t)(list ? 16 : 2) * nd * 4);   // list tiles: up to 16 parent rows
    S.st_l = S.st_r + 128 * 4;                     // list mode: the 16 octs' leaf rows
    S.stage_bytes = align128(S.st_l + (list ? 128 * 4 : 0));
    S.stage = S.out + align128((size_t)128 * nd * 4);
    S.grp_stride = S.stage + 2 * S.stage_bytes;
    S.total = S.grp + (size_t)G * S.grp_stride;
    return S;
}

__device__ __forceinline__ float fast_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ void named_barrier(int id, int threads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// octs in a tile (16, fewer in a list's last tile)
__device__ __forceinline__ int tile_octs(const LeafTcArgs &P, int64_t tile, bool list)
{
    if (!list) return 16;
    const int64_t left = P.a.n_oct - tile * 16;
    return left < 16 ? (int)left : 16;
}

// a tile's inputs: E rows of its 16 octs, Sp rows of their 2 parents, 128
// densities (list mode: plus the octs' 128 leaf rows, and with Sp the parent
// rows of the tile's octs: the span pf .. pl in one copy when it is at most
// 16 rows, else one row per oct; returns the first staged row, or -1 for the
// per-oct layout)
__device__ __forceinline__ int prefetch(const LeafTcArgs &P, const LeafTcSmem &S, int64_t tile, unsigned char *st,
                                        uint64_t *bar, bool list, int pf = 0, int pl = 0)
{
    const int nd = P.a.nd;
    const uint32_t nb = (uint32_t)tile_octs(P, tile, list);
    const bool lsp = list && P.a.Sp;
    const bool per_oct = lsp && pl - pf >= P.span_max;
    // checked builds: a tile outside its job's octs (or parents) copies nothing
    const int64_t o0 = tile * 16, n_oct = P.a.n_oct;
    bool sp_ok = true;
    if (lsp && !per_oct)
        sp_ok = pf <= pl && in_bounds(pf, P.a.n_sp, kCheckLeafTcIn) && in_bounds(pl, P.a.n_sp, kCheckLeafTcIn);
    else if (P.a.Sp && !list)
        sp_ok = in_bounds(tile * 2 + 1, n_oct / 8, kCheckLeafTcIn);
    if (!(in_bounds(o0, n_oct, kCheckLeafTcIn) && in_bounds(o0 + nb - 1, n_oct, kCheckLeafTcIn) && sp_ok)) {
        mbar_expect_tx(bar, 0);
        return pf;
    }
    const uint32_t bp = !P.a.Sp ? 0u : !list ? 2u * nd * 4 : per_oct ? nb * nd * 4 : (uint32_t)(pl - pf + 1) * nd * 4;
    const uint32_t be = nb * nd * 4, br = nb * 32, bl = list ? nb * 32 : 0u;
    mbar_expect_tx(bar, be + bp + br + bl);
    bulk_g2s(st + S.st_e, P.a.E + tile * 16 * nd, be, bar);
    if (per_oct) {
        // a span with parents that have no octs of this level in it: row by row
        for (uint32_t o = 0; o < nb; ++o) {
            int r = __ldg(P.a.oparent + o0 + o);
            if (!in_bounds(r, P.a.n_sp, kCheckLeafTcIn)) r = 0;
            bulk_g2s(st + S.st_p + (size_t)o * nd * 4, P.a.Sp + (int64_t)r * nd, nd * 4, bar);
        }
    } else if (P.a.Sp) {
        bulk_g2s(st + S.st_p, P.a.Sp + (list ? (int64_t)pf : tile * 2) * nd, bp, bar);
    }
    bulk_g2s(st + S.st_r, P.a.rho_leaf + tile * 128, br, bar);
    if (list) bulk_g2s(st + S.st_l, P.a.oleaf + tile * 128, bl, bar);
    return per_oct ? -1 : pf;
}

// Leaf jobs of many boxes (cd_batch) walked by one persistent launch: global
// tile g is tile tile_ref[g].y of job tile_ref[g].x.  All jobs
// of a launch share the direction set; their leaf cell sizes differ, so the
// local-term operand holds Kloc in units of dx and the epilogue scales it.
struct LeafBatch {
    const LeafTcArgs *jobs;
    const int2 *tile_ref;        // global tile -> {job, tile within the job}
    int64_t total;
};

template <class T>
__device__ __forceinline__ T ldg_copy(const T *p)
{
    static_assert(sizeof(T) % 8 == 0, "8-byte words");
    T v;
    const unsigned long long *src = reinterpret_cast<const unsigned long long *>(p);
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(&v);
#pragma unroll
    for (int i = 0; i < (int)(sizeof(T) / 8); ++i) dst[i] = __ldg(src + i);
    return v;
}

// One leaf row of a tile: N_H[d] = loc[d] (x dx when kScale) + E[d] (+ Sp[d]),
// written to the staging row (kOut 1) or straight to n_h (kOut 2, rows with
// ok only), optionally A_V = N_H av_per_nh; returns sum_d 2^(c2 N_H[d]).  All
// 32 lanes of a warp take the same instance (the form is a launch constant).
template <bool kSp, int kOut, bool kAv, bool kScale>
__device__ __forceinline__ float leaf_rows(uint32_t taddr, int nd, const float *Ei, const float *Pi, float *orow,
                                           float *nh, float *av, bool ok, float c2, float avk, float dxs)
{
    float acc = 0.f;
#pragma unroll 1
    for (int c = 0; c < nd; c += 32) {
        uint32_t v[32];
        tmem_ld32(taddr + (uint32_t)c, v);
        tmem_ld_wait();
#pragma unroll
        for (int j4 = 0; j4 < 32; j4 += 4) {
            if (c + j4 >= nd) break;       // nd is a multiple of 4
            float4 e = *reinterpret_cast<const float4 *>(Ei + c + j4);
            if (kSp) {
                const float4 p = *reinterpret_cast<const float4 *>(Pi + c + j4);
                e.x += p.x;
                e.y += p.y;
                e.z += p.z;
                e.w += p.w;
            }
            float4 N;
            if (kScale) {
                N = make_float4(fmaf(__uint_as_float(v[j4]), dxs, e.x), fmaf(__uint_as_float(v[j4 + 1]), dxs, e.y),
                                fmaf(__uint_as_float(v[j4 + 2]), dxs, e.z), fmaf(__uint_as_float(v[j4 + 3]), dxs, e.w));
            } else {
                N = make_float4(__uint_as_float(v[j4]) + e.x, __uint_as_float(v[j4 + 1]) + e.y,
                                __uint_as_float(v[j4 + 2]) + e.z, __uint_as_float(v[j4 + 3]) + e.w);
            }
            acc += (fast_exp2(c2 * N.x) + fast_exp2(c2 * N.y)) + (fast_exp2(c2 * N.z) + fast_exp2(c2 * N.w));
            if (kOut == 1) *reinterpret_cast<float4 *>(orow + c + j4) = N;
            if (kOut == 2 && ok) {
                nh[c + j4] = N.x;
                nh[c + j4 + 1] = N.y;
                nh[c + j4 + 2] = N.z;
                nh[c + j4 + 3] = N.w;
            }
            if (kAv && ok) {
                av[c + j4] = N.x * avk;
                av[c + j4 + 1] = N.y * avk;
                av[c + j4 + 2] = N.z * avk;
                av[c + j4 + 3] = N.w * avk;
            }
        }
    }
    return acc;
}

// kMode 0: uniform tiles (P0); 1: list tiles (P0); 2: the jobs of Bt (P0 holds
// the launch-wide nd, NP, G, kloc and screening constant)
template <int kMode>
__global__ void __launch_bounds__(512, 1) leaf_tc(LeafTcArgs P0, LeafBatch Bt)
{
    constexpr bool kList = kMode == 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int nd = P0.a.nd, NP = P0.NP, G = P0.G;
    const LeafTcSmem S = leaf_tc_smem(nd, NP, G, kMode != 0);
    const int64_t total = kMode == 2 ? Bt.total : P0.ntiles;
    // global tile -> its job's arguments, the tile within the job and its kind
    auto job_of = [&](int64_t gt, int64_t &lt, bool &list) -> LeafTcArgs {
        if (kMode == 2) {
            const int2 ref = __ldg(Bt.tile_ref + gt);
            lt = ref.y;
            const LeafTcArgs J = ldg_copy(Bt.jobs + ref.x);
            list = J.list != 0;
            return J;
        }
        lt = gt;
        list = kList;
        return P0;
    };
    const int tid = threadIdx.x, warp = tid >> 5;
    const int g = warp >> 2, quarter = warp & 3, i = tid & 127;   // group, TMEM lane quarter, row
    // batched: job arguments and tile index per group in three rotating slots
    // (iteration n uses slot n % 3; during n the group's thread 0 fills slot
    // (n + 1) % 3 for the next tile's prefetch while threads finishing n - 1
    // may still read slot (n - 1) % 3); a job's arguments are copied only when
    // the slot held another job
    __shared__ LeafTcArgs s_job[kMode == 2 ? 4 : 1][3];
    __shared__ int s_job_id[kMode == 2 ? 4 : 1][3];
    __shared__ int s_tile[kMode == 2 ? 4 : 1][3];
    __shared__ int s_run[4][4];                  // list tiles: per group and warp, rows form one run
    // [0 .. G) group MMAs, [G + 2 g + stage] input stages
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + S.bar);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 3 * G);
    int *sflag = reinterpret_cast<int *>(tslot + 1);
    unsigned char *Gb = smem + S.grp + (size_t)g * S.grp_stride;
    unsigned char *sA = Gb + S.aloc;
    float *sO = reinterpret_cast<float *>(Gb + S.out);

    if (tid == 0) {
        for (int b = 0; b < 3 * G; ++b) mbar_init(&bar[b], 1);
        fence_mbar_init();
        for (int q = 0; q < G; ++q) sflag[q] = 0;
    }
    // B[d][8 t + s] = dx Kloc[t][s][d] (BF16; batched: dx = 1, the epilogue scales), directions past nd zero
    for (int e = tid; e < NP * kK; e += blockDim.x) {
        const int n = e / kK, k = e % kK;
        const int t = k >> 3, s = k & 7;
        const float v = n < nd ? (kMode == 2 ? 1.f : P0.a.dx_leaf) * P0.a.kloc[(t * 8 + s) * nd + n] : 0.f;
        *reinterpret_cast<__nv_bfloat16 *>(smem + S.bloc + op_off(n, k, kK)) = __float2bfloat16_rn(v);
    }
    // every group's A starts all zero; a tile rewrites only each row's own block
    for (int e = tid; e < G * 128 * kK / 8; e += blockDim.x) {
        const int gg = e / (128 * kK / 8), r = e % (128 * kK / 8);
        reinterpret_cast<uint4 *>(smem + S.grp + (size_t)gg * S.grp_stride + S.aloc)[r] = make_uint4(0, 0, 0, 0);
    }
    fence_proxy_async_smem();
    if (warp == 0) tmem_alloc(tslot, 256);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tD = *tslot + (uint32_t)(g * 64);
    const uint32_t lane_off = (uint32_t)(quarter * 32) << 16;
    const int bid = 1 + g;
    const int64_t first = (int64_t)blockIdx.x * G + g, stride = (int64_t)gridDim.x * G;
    const uint32_t idesc = umma_idesc_bf16(128, NP);
    uint32_t phase = 0, sphase[2] = {0, 0};
    bool pending[2] = {false, false};
    bool fault = false;
    // thread 0 (batched): the reference of the tile after the next one
    int2 ref_next = make_int2(0, 0);
    auto fill_slot = [&](int sl, int2 ref) {   // thread 0, batched
        if (s_job_id[g][sl] != ref.x) {
            s_job[g][sl] = ldg_copy(Bt.jobs + ref.x);
            s_job_id[g][sl] = ref.x;
        }
        s_tile[g][sl] = ref.y;
    };
    // list tiles with a parent prefix: thread 0 reads the span of parent rows of
    // a tile one tile before its prefetch, so that the loads' latency hides
    // behind the current tile; s_pf holds each stage's first staged row
    const bool lsp = kMode == 1 && P0.a.Sp != nullptr;
    __shared__ int s_pf[4][2];
    int pf_next = 0, pl_next = 0;
    auto span = [&](int64_t t, int &pf, int &pl) {
        const int nb = tile_octs(P0, t, true);
        pf = __ldg(P0.a.oparent + t * 16);
        pl = __ldg(P0.a.oparent + t * 16 + nb - 1);
    };
    if (i == 0 && first < total) {
        if (kMode == 2) {
            for (int sl = 0; sl < 3; ++sl) s_job_id[g][sl] = -1;
            fill_slot(0, __ldg(Bt.tile_ref + first));
            prefetch(s_job[g][0], S, s_tile[g][0], Gb + S.stage, &bar[G + 2 * g], P0.list != 0);
            if (first + stride < total) ref_next = __ldg(Bt.tile_ref + first + stride);
        } else {
            int64_t lt;
            bool lst;
            const LeafTcArgs J = job_of(first, lt, lst);
            int pf = 0, pl = 0;
            if (lsp) {
                span(lt, pf, pl);
                if (first + stride < total) span(first + stride, pf_next, pl_next);
            }
            s_pf[g][0] = prefetch(J, S, lt, Gb + S.stage, &bar[G + 2 * g], lst, pf, pl);
        }
        pending[0] = true;
    }

    int stg = 0, it = 0;
    for (int64_t gt = first; gt < total && !fault; gt += stride, stg ^= 1, ++it) {
        int64_t tile;
        bool lst;
        const int slot = it % 3;
        const LeafTcArgs &P = kMode == 2 ? s_job[g][slot] : P0;
        unsigned char *st = Gb + S.stage + stg * S.stage_bytes;
        if (i == 0) {
            if (gt + stride < total) {
                if (kMode == 2) {
                    const int nsl = (it + 1) % 3;
                    fill_slot(nsl, ref_next);
                    prefetch(s_job[g][nsl], S, s_tile[g][nsl], Gb + S.stage + (stg ^ 1) * S.stage_bytes,
                             &bar[G + 2 * g + (stg ^ 1)], P0.list != 0);
                    if (gt + 2 * stride < total) ref_next = __ldg(Bt.tile_ref + gt + 2 * stride);
                } else {
                    int64_t lt;
                    bool ln;
                    const LeafTcArgs J = job_of(gt + stride, lt, ln);
                    const int pf = pf_next, pl = pl_next;
                    if (lsp && gt + 2 * stride < total) span(gt + 2 * stride, pf_next, pl_next);
                    s_pf[g][stg ^ 1] = prefetch(J, S, lt, Gb + S.stage + (stg ^ 1) * S.stage_bytes,
                                                &bar[G + 2 * g + (stg ^ 1)], ln, pf, pl);
                }
                pending[stg ^ 1] = true;
            }
            // the phase bit advances only once the copy has landed: after a
            // timeout the exit below still waits for this stage's copy
            if (mbar_wait_bounded(&bar[G + 2 * g + stg], sphase[stg], P0.pipe_polls)) {
                pending[stg] = false;
                sphase[stg] ^= 1;
            } else {
                sflag[g] = 1;
            }
        }
        named_barrier(bid, 128);
        if (sflag[g]) {
            fault = true;
            break;
        }
        // read after the barrier: thread 0 filled this tile's slot
        lst = kMode == 2 ? P0.list != 0 : kList;
        tile = kMode == 2 ? (int64_t)s_tile[g][slot] : gt;
        const float *sR = reinterpret_cast<const float *>(st + S.st_r);
        // list tiles with a parent prefix: this row's parent row (its load overlaps the product)
        const int par = lsp && (i >> 3) < tile_octs(P, tile, true) ? __ldg(P0.a.oparent + tile * 16 + (i >> 3)) : 0;
        // ---- A row: the oct's densities in block t ----
        {
            const float4 r0 = *reinterpret_cast<const float4 *>(sR + (i & ~7));
            const float4 r1 = *reinterpret_cast<const float4 *>(sR + (i & ~7) + 4);
            *reinterpret_cast<uint4 *>(sA + op_off(i, 8 * (i & 7), kK)) =
                make_uint4(pack_bf16x2(r0.x, r0.y), pack_bf16x2(r0.z, r0.w), pack_bf16x2(r1.x, r1.y),
                           pack_bf16x2(r1.z, r1.w));
        }
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 128);
        if (i == 0) {
            tc_fence_after();
            const uint32_t a0 = smem_u32(sA), b0 = smem_u32(smem + S.bloc);
            for (int ks = 0; ks < kK / 16; ++ks)
                umma_bf16(tD, umma_smem_desc(a0 + ks * 256, 128, kK * 16), umma_smem_desc(b0 + ks * 256, 128, kK * 16),
                          idesc, ks > 0 ? 1u : 0u);
            umma_commit(&bar[g]);
            if (!mbar_wait_bounded(&bar[g], phase, P0.pipe_polls)) sflag[g] = 1;
            // the previous tile's rows must have left the output buffer
            if (P0.out_bulk && !(kMode == 2 ? P0.list != 0 : kList)) bulk_wait_read<0>();
        }
        // each oct's copies were issued by thread i (list tiles)
        if (P0.out_bulk && (kMode == 2 ? P0.list != 0 : kList) && i < 16) bulk_wait_read<0>();
        phase ^= 1;
        named_barrier(bid, 128);
        if (sflag[g]) {
            fault = true;
            break;
        }
        tc_fence_after();
        // ---- N_H = loc + E[oct] + Sp[parent]; screening factor ----
        const int32_t *sL = reinterpret_cast<const int32_t *>(st + S.st_l);
        const int nb = tile_octs(P, tile, lst);
        const float dxs = kMode == 2 ? P.a.dx_leaf : 1.f;   // batched: Kloc in units of dx
        {
            // output row of this leaf: Morton position, or the list's row (-1: none)
            const int64_t m = lst ? ((i >> 3) < nb ? (int64_t)sL[i] : -1) : tile * 128 + i;
            const bool ok = m >= 0 && in_bounds(m, lst ? P.a.n_rows : 8 * P.a.n_oct, kCheckLeafTcOut);
            const int64_t mr = ok ? m : 0;
            const float *Ei = reinterpret_cast<const float *>(st + S.st_e) + (i >> 3) * nd;
            // the row's parent row among the staged ones: uniform tiles hold 2 parents;
            // list tiles the span from s_pf (at most 16 rows), or one row per oct (-1)
            int prow = i >> 6;
            if (lsp) {
                const int f = s_pf[g][stg];
                prow = f < 0 ? (i >> 3) : min(max(par - f, 0), 15);
            }
            const float *Pi = reinterpret_cast<const float *>(st + S.st_p) + prow * nd;
            float *orow = sO + (size_t)i * nd;
            const float c2 = P.c2, avk = P.a.av_per_nh;
            // the output form is a launch constant (kernel parameter): pick the
            // loop once, outside the per-direction work
            const int fm = P0.form;
            float *av = (fm & kFormAv) ? P.a.a_v + mr * nd : nullptr;
            float *nh = (fm & kFormNh) ? P.a.n_h + mr * nd : nullptr;
            float *shp = (fm & kFormShield) ? P.a.shield + mr : nullptr;
            const int form = fm & (kFormSp | kFormBulk | kFormNh | kFormAv);
            const uint32_t taddr = tD + lane_off;
            float acc;
            __syncwarp();
            switch (form) {
            case 0: acc = leaf_rows<false, 0, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 1: acc = leaf_rows<true, 0, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 2: acc = leaf_rows<false, 1, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 3: acc = leaf_rows<true, 1, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 4: acc = leaf_rows<false, 2, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 5: acc = leaf_rows<true, 2, false, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 8: acc = leaf_rows<false, 0, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 9: acc = leaf_rows<true, 0, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 10: acc = leaf_rows<false, 1, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 11: acc = leaf_rows<true, 1, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            case 12: acc = leaf_rows<false, 2, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            default: acc = leaf_rows<true, 2, true, kMode == 2>(taddr, nd, Ei, Pi, orow, nh, av, ok, c2, avk, dxs); break;
            }
            if ((fm & kFormShield) && ok) *shp = acc / (float)nd;
        }
        // list tiles: do the tile's leaf rows form one run (row of leaf i = row of leaf 0 + i)?
        // then one bulk copy sends the tile, as for Morton tiles (octs whose children are all
        // leaves lie next to each other in the depth-first order)
        if (lst && P0.out_bulk) {
            const bool in_run = (i >> 3) >= nb || sL[i] == sL[0] + i;
            const bool all = __all_sync(0xffffffffu, in_run);
            if ((i & 31) == 0) s_run[g][quarter] = all ? 1 : 0;
        }
        // list tiles: the rows the copies below need, read from the stage before the
        // barrier (after it, thread 0 may already prefetch the tile after next into
        // this stage)
        int lrow[8];
        const int lrow0 = lst ? sL[0] : 0;
        if (lst && i < nb) {
#pragma unroll
            for (int t = 0; t < 8; ++t) lrow[t] = sL[8 * i + t];
        }
        fence_proxy_async_smem();
        tc_fence_before();
        named_barrier(bid, 128);
        if (P0.out_bulk && !lst && i == 0 && in_bounds(tile * 128 + 127, 8 * P.a.n_oct, kCheckLeafTcOut)) {
            bulk_s2g(P.a.n_h + tile * 128 * nd, sO, (uint32_t)(128 * nd * 4));
            bulk_commit();
        }
        const bool tile_run = lst && P0.out_bulk && lrow0 >= 0 && s_run[g][0] && s_run[g][1] && s_run[g][2] &&
                              s_run[g][3] && in_bounds(lrow0 + 8 * nb - 1, P.a.n_rows, kCheckLeafTcOut);
        if (tile_run && i == 0) {
            bulk_s2g(P.a.n_h + (int64_t)lrow0 * nd, sO, (uint32_t)(8 * nb * nd * 4));
            bulk_commit();
        }
        if (lst && P0.out_bulk && i < nb && !tile_run) {
            // oct i's children: one copy when their rows are consecutive, else one per leaf row
            const int r0 = lrow[0];
            bool run = r0 >= 0 && in_bounds(r0 + 7, P.a.n_rows, kCheckLeafTcOut);
#pragma unroll
            for (int t = 1; t < 8; ++t) run = run && lrow[t] == r0 + t;
            if (run) {
                bulk_s2g(P.a.n_h + (int64_t)r0 * nd, sO + (size_t)8 * i * nd, (uint32_t)(8 * nd * 4));
            } else {
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int r = lrow[t];
                    if (r >= 0 && in_bounds(r, P.a.n_rows, kCheckLeafTcOut))
                        bulk_s2g(P.a.n_h + (int64_t)r * nd, sO + (size_t)(8 * i + t) * nd, (uint32_t)(nd * 4));
                }
            }
            bulk_commit();
        }
    }
    if (fault && i == 0) {
        atomicExch(&g_leaftc_fault, 1);
        mbar_wait_bounded(&bar[g], phase ^ 1, kMaxPolls);   // let an issued product finish
    }
    if (i == 0)
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait_bounded(&bar[G + 2 * g + b], sphase[b], kMaxPolls);
    if (i == 0 || (kMode != 0 && i < 16)) bulk_wait_all<0>();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(*tslot, 256);
    }
}

int sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace

// The tensor-core leaf kernel serves uniform trees with at least one full tile
// (128 leaves), n_dir a multiple of 4 up to 64, 16-byte aligned inputs.
cd_status launch_leaf_tc(const LeafLaunch &a, cudaStream_t s)
{
    const int nd = a.nd;
    const int64_t n_leaf = a.n_oct * 8;
    const bool list = a.oleaf != nullptr;
    if (nd % 4 != 0 || nd > 64 || !aligned16(a.E) || !aligned16(a.Sp) || !aligned16(a.rho_leaf) || !a.E)
        return CD_EUNSUPPORTED;
    if (!list && (n_leaf < 128 || n_leaf % 128 != 0)) return CD_EUNSUPPORTED;
    if (list && ((a.Sp && !a.oparent) || !aligned16(a.oleaf) || (a.n_h && !aligned16(a.n_h)))) return CD_EUNSUPPORTED;
    if (n_leaf == 0) return CD_OK;
    LeafTcArgs P;
    P.a = a;
    P.list = list;
    P.NP = round16(nd);
    P.n_leaf = n_leaf;
    P.ntiles = (a.n_oct + 15) / 16;
    P.c2 = (float)(-(double)a.shield_k * (double)a.av_per_nh * 1.4426950408889634);
    P.out_bulk = a.n_h && aligned16(a.n_h);
    P.form = leaf_form(a, P.out_bulk, list);
    {
        const int64_t cap = g_pipe_polls.load();
        P.pipe_polls = cap < 0 ? kMaxPolls : (uint32_t)std::min<int64_t>(cap, kMaxPolls);
    }
    P.span_max = g_span_max.load();
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    P.G = 4;
    while (P.G > 1 && (int)leaf_tc_smem(nd, P.NP, P.G, list).total > smax) --P.G;
    const size_t smem = leaf_tc_smem(nd, P.NP, P.G, list).total;
    if ((int)smem > smax) return CD_EUNSUPPORTED;
    const auto kern = list ? leaf_tc<1> : leaf_tc<0>;
    CD_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::min<int64_t>((P.ntiles + P.G - 1) / P.G, sms());
    LaunchScope ls(CD_K_LEAF, s, 2.0 * (double)P.ntiles * 128.0 * kK * P.NP);
    kern<<<(unsigned)grid, 128 * P.G, smem, s>>>(P, LeafBatch{});
    CD_CHECK_LAUNCH();
    return CD_OK;
}

size_t leaf_tc_job_bytes() { return sizeof(LeafTcArgs); }

int64_t leaf_tc_job_fill(const LeafLaunch &a, void *dst)
{
    const int nd = a.nd;
    const int64_t n_leaf = a.n_oct * 8;
    const bool list = a.oleaf != nullptr;
    if (nd % 4 != 0 || nd > 64 || !aligned16(a.E) || !aligned16(a.Sp) || !aligned16(a.rho_leaf) || !a.E) return -1;
    if (!list && (n_leaf < 128 || n_leaf % 128 != 0)) return -1;
    if (list && (a.Sp || !aligned16(a.oleaf) || (a.n_h && !aligned16(a.n_h)))) return -1;
    LeafTcArgs P = {};
    P.a = a;
    P.list = list;
    P.NP = round16(nd);
    P.n_leaf = n_leaf;
    P.ntiles = (a.n_oct + 15) / 16;
    P.c2 = (float)(-(double)a.shield_k * (double)a.av_per_nh * 1.4426950408889634);
    P.out_bulk = a.n_h && aligned16(a.n_h);
    P.form = leaf_form(a, P.out_bulk, list);
    P.pipe_polls = kMaxPolls;
    memcpy(dst, &P, sizeof(P));
    return P.ntiles;
}

int leaf_tc_job_form(const void *job)
{
    LeafTcArgs P;
    memcpy(&P, job, sizeof(P));
    return P.form;
}

cd_status launch_leaf_tc_batch(const void *jobs, const int2 *tile_ref, int64_t total, int nd, const float *kloc,
                               int form, double flops, cudaStream_t s)
{
    if (total <= 0) return CD_OK;
    LeafTcArgs P = {};
    P.a.nd = nd;
    P.a.kloc = kloc;
    P.NP = round16(nd);
    P.form = form;
    P.list = (form & kFormList) != 0;
    P.out_bulk = (form & kFormBulk) != 0;
    {
        const int64_t cap = g_pipe_polls.load();
        P.pipe_polls = cap < 0 ? kMaxPolls : (uint32_t)std::min<int64_t>(cap, kMaxPolls);
    }
    int dev = 0, smax = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    P.G = 4;
    while (P.G > 1 && (int)leaf_tc_smem(nd, P.NP, P.G, true).total > smax) --P.G;
    const size_t smem = leaf_tc_smem(nd, P.NP, P.G, true).total;   // the kernel's layout (mode 2) has the list rows
    if ((int)smem > smax) {
        set_error("the batched leaf kernel needs %zu bytes of shared memory", smem);
        return CD_EUNSUPPORTED;
    }
    LeafBatch Bt;
    Bt.jobs = static_cast<const LeafTcArgs *>(jobs);
    Bt.tile_ref = tile_ref;
    Bt.total = total;
    CD_CUDA(cudaFuncSetAttribute(leaf_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int64_t grid = std::min<int64_t>((total + P.G - 1) / P.G, sms());
    LaunchScope ls(CD_K_LEAF, s, flops);
    leaf_tc<2><<<(unsigned)grid, 128 * P.G, smem, s>>>(P, Bt);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

double leaf_tc_job_flops(const void *job)
{
    LeafTcArgs P;
    memcpy(&P, job, sizeof(P));
    return 2.0 * (double)P.ntiles * 128.0 * kK * P.NP;
}

void set_leaf_tc_wait_polls(int64_t polls) { g_pipe_polls.store(polls < 0 ? -1 : polls); }

void set_leaf_tc_span_max(int rows) { g_span_max.store(rows < 0 || rows > kSpanRows ? kSpanRows : rows); }

cd_status leaf_tc_fault_check()
{
    int v = 0;
    CD_CUDA(cudaMemcpyFromSymbol(&v, g_leaftc_fault, sizeof(int)));
    if (v) {
        const int zero = 0;
        CD_CUDA(cudaMemcpyToSymbol(g_leaftc_fault, &zero, sizeof(int)));
        set_error("a tensor-core leaf kernel gave up a bounded wait");
        return CD_ETIMEOUT;
    }
    return CD_OK;
}

}  // namespace cd
