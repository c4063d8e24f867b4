// BF16 tensor-core (tcgen05) form of the shell contraction (Eq. N_discret).
//
// GEMM framing.  For a receiving level k (k >= 4) every shell table t reads a
// 6x6x6 stencil of level k-t+1 around the ancestor A_{k-t}; the stencil of
// table 1 sits around the parent P = A_{k-1} of the receiving cell c and is
// shared by the 8 children of P.  One GEMM row is one parent P:
//   A[P, (t, q, ch)] = rho_{k-t+1}(child ch of neighbour q of A_{k-t}(P))
//   B[(t, q, ch), (o, d)] = 2^(t-1) K_t[cfg_t(P, o)][s(q, ch)][d]
//   E[8P + o][d] = dx_k D[P, (o, d)] + S_{k-1}[P][d]
// with q over the 27 level-(k-t) neighbours (+3 zero bricks: 30 per table),
// ch over their 8 children and o over the children of P.  cfg_t depends on
// the octants of P and of its parent, so the 64 classes (oct(par P), oct(P))
// each get their own B and a tile holds 128 parents of one class.  Powers
// of two fold dx_{k-t+1} = 2^(t-1) dx_k into B exactly.
//
// Densities are stored per level as BF16 "bricks" (the 8 children of one
// coarser cell, 16 bytes), so an A row is 90 bricks and one brick is exactly
// one row of an 8x16-byte core matrix: cp.async 16-byte copies place them
// straight into the K-major no-swizzle operand layout.  A K-chunk is 6 bricks,
// i.e. two x-runs of 3 neighbours (48 contiguous bytes each), and consecutive
// lanes copy consecutive bricks of a row, so one warp instruction touches few
// lines.  B is precomputed in global memory in the operand layout per K-chunk,
// so each chunk is one bulk copy.
//
// CTA (448 threads, two per SM): warp 0 issues the MMAs (M = 128, N = 4 nd,
// K = 16) and owns the TMEM accumulator; warp 1 bulk-copies B; warps 2-5
// gather A (one row each); warps 6-13 drain TMEM into E, two per lane quarter
// (warp % 4), each half of the columns (the epilogue is on the critical path:
// eight drain warps with two stages measured faster than four with three, as
// shared memory holds only one of the two at two CTAs per SM).  A 2-stage
// mbarrier pipeline couples them; every wait is bounded and a timeout sets a
// device flag instead of trapping.
#include <algorithm>
#include <string.h>

#include "common.cuh"
#include "geom_device.cuh"
#include "umma.cuh"

namespace cd {
namespace {

constexpr int kStages = 2;
constexpr int kChunkBricks = 6;                 // K = 48 per chunk (3 MMA K-steps)
constexpr int kBricksPerTable = 30;             // 27 neighbours + 3 zero bricks
constexpr int kChunks = 3 * kBricksPerTable / kChunkBricks;  // 15
constexpr int kThreads = 448;                   // 14 warps
constexpr int kEpiWarps = 8;                    // two per TMEM lane quarter, each half of the columns
constexpr uint32_t kMaxPolls = 1u << 26;
// A stage: core matrix (row group mg, brick b) at mg * kASbo + b * kALbo; the
// 144-byte K stride puts the bricks of one row in different bank quads
constexpr uint32_t kALbo = 144, kASbo = kChunkBricks * kALbo;
constexpr uint32_t kAStageBytes = 16 * kASbo;                // 13.5 KB
constexpr int kTmemCols = 256;

static __device__ int g_tc_fault;

struct TcArgs {
    int k;                       // receiving level (>= 4)
    int nd, N, Nt;               // directions, N = 8 nd, Nt = N / 2 columns per tile (children 4h .. 4h+3)
    int c0, c1;                  // chunk range: table t is chunks 5 (t-1) .. 5 t
    const __nv_bfloat16 *brick[4];   // brick arrays of levels k, k-1, k-2 (tables 1, 2, 3)
    const __nv_bfloat16 *B;      // [64 class][15 chunk][N/8][6][8][8]
    float *out;                  // [8^k][nd]: the shell sum of this launch (no far-field prefix)
    float dx_k;
    int64_t nG;                  // 8^(k-3)
    int64_t ntiles;              // 2 * 64 * ceil(nG / 128), or the list's tile count
    // list mode (tiles != NULL, AMR meshes): tile i = {class, first row, rows,
    // half} over row_key (parent Morton keys grouped by class); the output row
    // of child o of row r is row_out[8 r + o] (-1: not a receiver)
    const int4 *tiles;
    const uint64_t *row_key;
    const int32_t *row_out;
    // batched evaluation (cd_batch) only:
    int full;                    // 1: a tile covers all 8 children (Nt = N, list tiles: the h = 0 entry)
    const float *prefix;         // added to every output row in the epilogue (S_{k-1}), or NULL
    const int32_t *prefix_row;   // list mode: prefix row of output row i; uniform: the parent P
    int wait_job;                // job whose tiles must be complete before `prefix` is read (-1: none)
    int wait_count;              // that job's completion count when it is done (8 per tile)
    int signal;                  // another job waits on this one: count its finished tiles
    int pad0;
};

// A batch of shell jobs (one per box, level and table run) walked by one
// persistent launch: global tile g is tile tile_ref[g].y of job
// tile_ref[g].x; done[job] counts the epilogue warps (8 per tile) that have
// finished a tile of that job.  CTAs take tiles from the work counter `claim`
// in increasing order, so every tile a wait depends on (a lower one) has been
// taken by a CTA that is running: progress never depends on how many CTAs an
// SM holds at once.
struct TcBatch {
    const TcArgs *jobs;
    const int2 *tile_ref;        // global tile -> {job, tile within the job}
    int64_t total;
    int *done;
    int *claim;                  // work counter: the next global tile to hand out
    uint32_t bstage_max;         // largest B stage of any job (Nt x 96 bytes)
};
constexpr int kRing = 8;         // claimed tiles a CTA's roles may be apart (at most 3 in practice)

// copy of a job's arguments through the read-only path
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

// tile -> (row block gb, class cls, half h); uniform half tiles: the two halves
// of one row block are consecutive tiles; full tiles: one per (row block,
// class); list tiles: {class, first row, rows, half} entries in pairs
__device__ __forceinline__ void tile_coords(const TcArgs &P, int64_t tile, int64_t &gb, int &cls, int &h, int4 &tt)
{
    tt = make_int4(0, 0, 0, 0);
    if (P.tiles) {
        tt = P.tiles[P.full ? 2 * tile : tile];
        cls = tt.x;
        h = P.full ? 0 : tt.w;
        gb = 0;
    } else if (P.full) {
        h = 0;
        cls = (int)(tile & 63);
        gb = tile >> 6;
    } else {
        h = (int)(tile & 1);
        cls = (int)((tile >> 1) & 63);
        gb = tile >> 7;
    }
}

__device__ __forceinline__ int ld_acquire(const int *p)
{
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Waits until *cnt >= target (another CTA's tiles of the same launch); false
// after the poll limit.  Tiles are ordered so that a wait only ever depends on
// tiles of lower global index, which resident CTAs finish first.
__device__ __forceinline__ bool wait_count(const int *cnt, int target)
{
    for (uint32_t i = 0; i < (1u << 24); ++i) {
        if (ld_acquire(cnt) >= target) return true;
        __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ bool wait_bar(uint64_t *bar, uint32_t parity)
{
    return mbar_wait_bounded(bar, parity, kMaxPolls);
}

// kBatch = false: one launch of one level (P0; Bt unused).  kBatch = true:
// the jobs of Bt, each tile with its own job's arguments.
template <bool kBatch>
__global__ void __maxnreg__(64) shell_sum_tc(TcArgs P0, TcBatch Bt)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    // B stages sized for the widest tile (Nt/8 groups x 6 bricks x 128 B)
    const uint32_t bstage_max = kBatch ? Bt.bstage_max : (uint32_t)P0.Nt * kChunkBricks * 16;
    unsigned char *sA = smem;                                        // [kStages][13.5 KB]
    unsigned char *sB = smem + kStages * kAStageBytes;               // [kStages][bstage_max]
    float *sT = reinterpret_cast<float *>(sB + kStages * bstage_max);    // [8 warps][32][33] transpose
    int32_t *sOut = reinterpret_cast<int32_t *>(sT + kEpiWarps * 32 * 33);   // batched list mode: [8 warps][32][8]
    uint64_t *full = reinterpret_cast<uint64_t *>(sOut + (kBatch ? kEpiWarps * 32 * 8 : 0));
    uint64_t *empty = full + kStages;
    uint64_t *acc_full = empty + kStages;
    uint64_t *acc_empty = acc_full + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc_empty + 1);
    __shared__ int s_fault;
    // batched: the tiles this CTA claimed, in order, and one mbarrier each
    __shared__ int64_t s_ring[kBatch ? kRing : 1];
    __shared__ uint64_t s_ring_bar[kBatch ? kRing : 1];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = kBatch ? Bt.total : P0.ntiles;
    // the CTA's n-th tile: static stride (one launch of one level), or the
    // n-th claimed tile (batched: the B producer claims, every role reads the
    // ring).  False at the end, or with *bad set when a wait runs out.
    auto tile_n = [&](int n, int64_t &g, bool &bad) -> bool {
        bad = false;
        if (!kBatch) {
            g = blockIdx.x + (int64_t)n * gridDim.x;
            return g < total;
        }
        const int r = n % kRing;
        if (!mbar_wait_bounded(&s_ring_bar[r], (uint32_t)((n / kRing) & 1), kMaxPolls)) {
            bad = true;
            return false;
        }
        g = s_ring[r];
        return g >= 0;
    };
    auto claim_n = [&](int n) {   // the B producer's lane 0: hand the CTA its n-th tile
        if (!kBatch) return;
        const int64_t c = atomicAdd(Bt.claim, 1);
        s_ring[n % kRing] = c < total ? c : -1;
        mbar_arrive(&s_ring_bar[n % kRing]);   // release: the entry is visible to the waiters
    };
    // global tile g -> its job's arguments (a copy: the kernel's stores must
    // not force reloads from the job table) and the tile's index within the job
    auto job_of = [&](int64_t g, int &job, int64_t &tile) -> TcArgs {
        if (kBatch) {
            const int2 ref = __ldg(Bt.tile_ref + g);
            job = ref.x;
            tile = ref.y;
            return ldg_copy(Bt.jobs + job);
        }
        job = 0;
        tile = g;
        return P0;
    };

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 128 + 1);      // 128 gather threads + the B producer
            mbar_init(&empty[s], 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, kEpiWarps);       // one arrival per epilogue warp
        if (kBatch)
            for (int r = 0; r < kRing; ++r) mbar_init(&s_ring_bar[r], 1);
        fence_mbar_init();
        s_fault = 0;
    }
    if (warp == 0) tmem_alloc(tslot, kTmemCols);
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
            for (int n = 0; !fault; ++n, ++u) {
                int64_t g;
                bool bad;
                if (!tile_n(n, g, bad)) {
                    fault = bad;
                    break;
                }
                int job;
                int64_t tile;
                const TcArgs P = job_of(g, job, tile);
                const uint32_t idesc = umma_idesc_bf16(128, P.Nt);
                const int nchunk = P.c1 - P.c0;
                if (!wait_bar(acc_empty, (u & 1) ^ 1)) { fault = true; break; }
                tc_fence_after();
                for (int j = 0; j < nchunk; ++j, ++q) {
                    const int s = q % kStages;
                    if (!wait_bar(&full[s], (q / kStages) & 1)) { fault = true; break; }
                    tc_fence_after();
                    const uint32_t a0 = smem_u32(sA + s * kAStageBytes), b0 = smem_u32(sB + s * bstage_max);
#pragma unroll
                    for (int ks = 0; ks < kChunkBricks / 2; ++ks)
                        umma_bf16(tbase, umma_smem_desc(a0 + ks * 2 * kALbo, kALbo, kASbo),
                                  umma_smem_desc(b0 + ks * 256, 128, kChunkBricks * 128), idesc,
                                  (j > 0 || ks > 0) ? 1u : 0u);
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
            for (int n = 0; !fault; ++n) {
                claim_n(n);
                int64_t g;
                bool bad;
                if (!tile_n(n, g, bad)) {
                    fault = bad;
                    break;
                }
                int job;
                int64_t tile;
                const TcArgs P = job_of(g, job, tile);
                const int nchunk = P.c1 - P.c0;
                const uint32_t bstage = (uint32_t)P.Nt * kChunkBricks * 16;
                const uint32_t bhalf = (uint32_t)P.N * kChunkBricks * 16;    // one chunk of the global B
                int64_t gb;
                int cls, h;
                int4 tt;
                tile_coords(P, tile, gb, cls, h, tt);
                const unsigned char *Bc = reinterpret_cast<const unsigned char *>(P.B) + (size_t)cls * kChunks * bhalf +
                                          (size_t)h * bstage;
                for (int j = 0; j < nchunk; ++j, ++q) {
                    const int s = q % kStages;
                    if (!wait_bar(&empty[s], ((q / kStages) & 1) ^ 1)) { fault = true; break; }
                    mbar_expect_tx(&full[s], bstage);
                    bulk_g2s(sB + s * bstage_max, Bc + (size_t)(P.c0 + j) * bhalf, bstage, &full[s]);
                }
            }
        }
        __syncwarp();
    } else if (warp < 6) {
        // ---------------- A gather (128 threads, one row each) ----------------
        // Per tile a thread keeps, for each table, a pointer to the brick of its
        // (-1,-1,-1) neighbour and a 27-bit in-box mask; per chunk the six
        // neighbour offsets are uniform, so each brick is an add, a bit test and
        // one 16-byte cp.async.
        const int m = tid - 64;
        unsigned char *dst_row = sA + (m >> 3) * kASbo + (m & 7) * 16;
        uint32_t q = 0;
        for (int n = 0; !fault; ++n) {
            int64_t g;
            bool bad;
            if (!tile_n(n, g, bad)) {
                fault = bad;
                break;
            }
            int job;
            int64_t tile;
            const TcArgs P = job_of(g, job, tile);
            int64_t gb;
            int cls, h;
            int4 tt;
            tile_coords(P, tile, gb, cls, h, tt);
            const int64_t G = gb * 128 + m;
            bool valid = G < P.nG;
            uint64_t Pm = ((uint64_t)(valid ? G : 0) << 6) | (uint64_t)cls;
            if (P.tiles) {
                valid = m < tt.z;
                Pm = P.row_key[tt.y + (valid ? m : 0)];
            }
            const int px = (int)compact3(Pm), py = (int)compact3(Pm >> 1), pz = (int)compact3(Pm >> 2);
            const __nv_bfloat16 *corner[3];
            uint32_t mask[3];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                const int n = 1 << (P.k - 1 - t);
                const int ax = (px >> t) - 1, ay = (py >> t) - 1, az = (pz >> t) - 1;
                corner[t] = P.brick[t + 1] + ((int64_t)((int64_t)az * n + ay) * n + ax) * 8;
                uint32_t mx = 0, my = 0, mz = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    mx |= (uint32_t)(ax + d >= 0 && ax + d < n) << d;
                    my |= (uint32_t)(ay + d >= 0 && ay + d < n) << d;
                    mz |= (uint32_t)(az + d >= 0 && az + d < n) << d;
                }
                uint32_t mm = 0;
#pragma unroll
                for (int nq = 0; nq < 27; ++nq)
                    mm |= ((mx >> (nq % 3)) & (my >> ((nq / 3) % 3)) & (mz >> (nq / 9)) & 1u) << nq;
                mask[t] = valid ? mm : 0u;
            }
            // the 15 chunks unrolled: chunk j is table t = j / 5, neighbours
            // 6 (j % 5) .. + 5, so every neighbour offset is a constant
            // (dz, dy, dx) scaled by the level's side 2^e (a uniform shift);
            // chunks outside [c0, c1) are skipped
            const int e0 = P.k - 1;
#pragma unroll
            for (int j = 0; j < kChunks; ++j) {
                if (j < P.c0 || j >= P.c1) continue;
                const int s = q % kStages;
                bool ok = true;
                if (lane == 0) ok = wait_bar(&empty[s], ((q / kStages) & 1) ^ 1);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) { fault = true; break; }
                constexpr int kPerTable = kBricksPerTable / kChunkBricks;
                const int t = j / kPerTable, nq0 = (j % kPerTable) * kChunkBricks;
                const int e = e0 - t;                                 // level side n = 2^e
                const __nv_bfloat16 *cor = corner[t];
                const uint32_t mk = mask[t];
                unsigned char *dst = dst_row + s * kAStageBytes;
#pragma unroll
                for (int b = 0; b < kChunkBricks; ++b) {
                    const int nq = nq0 + b;
                    if (nq >= 27) {                                    // the zero bricks of the table
                        cp_async16_ca(dst + b * kALbo, P.brick[1], 0u);
                        continue;
                    }
                    const int64_t off = ((int64_t)(nq / 9) << (2 * e + 3)) + ((int64_t)((nq / 3) % 3) << (e + 3)) +
                                        (int64_t)((nq % 3) << 3);
                    const bool in = ((mk >> nq) & 1u) &&
                                    in_bounds((cor - P.brick[t + 1]) / 8 + off / 8, 1ll << (3 * e), kCheckTcBrick);
                    cp_async16_ca(dst + b * kALbo, in ? cor + off : P.brick[1], in ? 16u : 0u);
                }
                cp_async_arrive(&full[s]);
                ++q;
            }
        }
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else {
        // ---------------- epilogue: TMEM -> E (warps 6..13, TMEM lane quarter warp % 4) ----------------
        const int ew = warp - 6;
        const int chalf = ew >> 2;             // this warp's half of the columns
        const int quarter = warp & 3;
        float *T = sT + ew * 32 * 33;
        int32_t *my_rows = sOut + ew * 32 * 8;  // batched list mode: output row of child j of row r at [8 r + j]
        int u = 0;
        for (int n = 0; !fault; ++n, ++u) {
            int64_t g;
            bool bad;
            if (!tile_n(n, g, bad)) {
                fault = bad;
                break;
            }
            int job;
            int64_t tile;
            const TcArgs P = job_of(g, job, tile);
            int64_t gb;
            int cls, h;
            int4 tt;
            tile_coords(P, tile, gb, cls, h, tt);
            const int Nt = P.Nt, nd = P.nd;
            const float dx_k = P.dx_k;
            const int64_t G0 = gb * 128 + quarter * 32;               // the warp's first row
            int nrows = (int)(P.nG - G0 < 32 ? (P.nG - G0 > 0 ? P.nG - G0 : 0) : 32);
            int my_out[4] = {-1, -1, -1, -1};   // list mode: output rows of this lane's row, children 4h .. 4h+3
            if (P.tiles) {
                nrows = tt.z - quarter * 32;
                nrows = nrows < 0 ? 0 : (nrows > 32 ? 32 : nrows);
                if (kBatch) {
                    // this lane's row: its children's output rows (looked up once per tile)
                    const int nch = P.full ? 8 : 4;
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const int dst = (lane < nrows && j < nch)
                                            ? __ldg(P.row_out + 8 * (int64_t)(tt.y + quarter * 32 + lane) + 4 * h + j)
                                            : -1;
                        my_rows[lane * 8 + j] = dst;
                    }
                    __syncwarp();
                } else if (lane < nrows) {
#pragma unroll
                    for (int j = 0; j < 4; ++j)
                        my_out[j] = P.row_out[8 * (int64_t)(tt.y + quarter * 32 + lane) + 4 * h + j];
                }
            }
            // row r of the warp is parent P = ((G0 + r) << 6) | cls; its columns of
            // this tile are the contiguous run out[(8P + 4h) nd .. + Nt)
            float *row0 = P.out + (size_t)((((G0 << 6) | cls) * 8) + 4 * h) * nd;
            const size_t rstride = (size_t)64 * 8 * nd;
            bool ok = true;
            if (lane == 0) ok = wait_bar(acc_full, u & 1);
            // batched: the prefix rows of this job are complete once the job they come from is
            if (kBatch && P.prefix && P.wait_job >= 0 && lane == 0 && ok)
                ok = wait_count(Bt.done + P.wait_job, P.wait_count);
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) { fault = true; break; }
            if (kBatch && P.prefix) __syncwarp();   // the lanes' prefix loads come after lane 0's acquire
            tc_fence_after();
            const int cmid = ((Nt >> 1) + 31) & ~31;   // the halves split on a 32-column chunk boundary
            for (int c = chalf ? cmid : 0; c < (chalf ? Nt : cmid); c += 32) {
                uint32_t v[32];
                tmem_ld32(tbase + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, v);
                tmem_ld_wait();
#pragma unroll
                for (int i = 0; i < 32; ++i) T[lane * 33 + i] = __uint_as_float(v[i]);
                __syncwarp();
                const int col = c + lane;
                if (kBatch) {
                    // dx D (+ prefix): two roundings, as the separate prefix pass of one evaluation
                    const int j = col < Nt ? col / nd : 0, d = col - j * nd;
                    const float *pre = P.prefix;
                    if (!P.tiles && col < Nt) {
                        // uniform tile: row r's output and prefix rows advance by fixed strides
                        float *o = row0 + col;
                        if (pre) {
                            const float *pp = pre + ((G0 << 6) | cls) * nd + d;
#pragma unroll 4
                            for (int r = 0; r < nrows; ++r, o += rstride, pp += 64 * nd)
                                *o = __fadd_rn(__fmul_rn(dx_k, T[r * 33 + lane]), __ldg(pp));
                        } else {
#pragma unroll 4
                            for (int r = 0; r < nrows; ++r, o += rstride) *o = __fmul_rn(dx_k, T[r * 33 + lane]);
                        }
                    } else if (P.tiles) {
#pragma unroll 4
                        for (int r = 0; r < nrows; ++r) {
                            const int dst = my_rows[r * 8 + j];
                            if (col < Nt && dst >= 0) {
                                float val = __fmul_rn(dx_k, T[r * 33 + lane]);
                                if (pre) val = __fadd_rn(val, __ldg(pre + (int64_t)__ldg(P.prefix_row + dst) * nd + d));
                                P.out[(int64_t)dst * nd + d] = val;
                            }
                        }
                    }
                } else if (col < Nt && !P.tiles) {
                    float *o = row0 + col;
#pragma unroll 4
                    for (int r = 0; r < nrows; ++r, o += rstride) *o = dx_k * T[r * 33 + lane];
                } else if (P.tiles) {
                    // row r's output row for this lane's child, broadcast from lane r; when
                    // the chunk's 32 columns span at most two children j0 and j0 + 1, two
                    // shuffles a row select it
                    const int j = col < Nt ? col / nd : 0, d = col - j * nd;
                    const int j0 = c / nd, jl = (c + 31 < Nt ? c + 31 : Nt - 1) / nd;
                    const int j1 = j0 + 1 < 4 ? j0 + 1 : 3;
                    const int s0 = j0 == 0 ? my_out[0] : j0 == 1 ? my_out[1] : j0 == 2 ? my_out[2] : my_out[3];
                    const int s1 = j1 == 1 ? my_out[1] : j1 == 2 ? my_out[2] : my_out[3];
                    if (jl - j0 <= 1) {
                        for (int r = 0; r < nrows; ++r) {
                            const int a0 = __shfl_sync(0xffffffffu, s0, r), a1 = __shfl_sync(0xffffffffu, s1, r);
                            const int dst = j == j0 ? a0 : a1;
                            if (col < Nt && dst >= 0) P.out[(int64_t)dst * nd + d] = dx_k * T[r * 33 + lane];
                        }
                    } else {
                        for (int r = 0; r < nrows; ++r) {
                            const int o0 = __shfl_sync(0xffffffffu, my_out[0], r),
                                      o1 = __shfl_sync(0xffffffffu, my_out[1], r),
                                      o2 = __shfl_sync(0xffffffffu, my_out[2], r),
                                      o3 = __shfl_sync(0xffffffffu, my_out[3], r);
                            const int dst = j == 0 ? o0 : j == 1 ? o1 : j == 2 ? o2 : o3;
                            if (col < Nt && dst >= 0) P.out[(int64_t)dst * nd + d] = dx_k * T[r * 33 + lane];
                        }
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acc_empty);
            if (kBatch && P.signal) {
                // this warp's rows of the tile are written: count it for the job that waits on this
                // one (the warp barrier orders the lanes' stores before lane 0's release)
                __syncwarp();
                if (lane == 0) {
                    __threadfence();
                    atomicAdd(Bt.done + job, 1);
                }
            }
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
        tmem_dealloc(tbase, kTmemCols);
    }
}

// ---- B operand construction (FP64 geometry, stored BF16) -----------------------

__global__ void build_b(int nd, const double *__restrict__ rays, int ns, __nv_bfloat16 *__restrict__ B)
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
            v = (float)(shell_weight_avg(t, cfg, s, rays + (size_t)3 * ns * d, ns) * (double)(1 << (t - 1)));
        }
        B[e] = __float2bfloat16_rn(v);
    }
}

// out[c][d] += parent[c >> 3][d] over n = 8^k nd elements (nd % 4 == 0).
__global__ void add_parent_rows(float *__restrict__ out, const float *__restrict__ parent, int nd, int64_t n)
{
    for (int64_t e = 4 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x); e < n; e += 4 * (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / nd;
        const int d = (int)(e - c * nd);
        float4 v = *reinterpret_cast<float4 *>(out + e);
        const float4 p = *reinterpret_cast<const float4 *>(parent + (c >> 3) * nd + d);
        v.x += p.x;
        v.y += p.y;
        v.z += p.z;
        v.w += p.w;
        *reinterpret_cast<float4 *>(out + e) = v;
    }
}

// out[i][d] += prefix[parent[i]][d] over n = n_recv nd elements
__global__ void add_parent_list(float *__restrict__ out, const float *__restrict__ prefix,
                                const int32_t *__restrict__ parent, int nd, int64_t n)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nd;
        out[e] += prefix[(int64_t)parent[i] * nd + (e - i * nd)];
    }
}

// dynamic shared memory of the shell kernel for B stages of bstage bytes
size_t tc_smem_bytes(size_t bstage, bool batch)
{
    return kStages * (kAStageBytes + bstage) + sizeof(float) * kEpiWarps * 32 * 33 +
           (batch ? sizeof(int32_t) * kEpiWarps * 32 * 8 : 0) + (2 * kStages + 2) * 8 + 16;
}

int num_sms()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 152;
}

}  // namespace

// A tile holds half the children of its parents: Nt = 4 nd accumulator
// columns, one MMA of N = Nt (a multiple of 16, at most 256 = the TMEM
// columns of one of the two CTAs an SM runs).
bool tc_supported(int nd)
{
    const int Nt = 4 * nd;
    return Nt <= 256 && Nt % 16 == 0;
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
    build_b<<<num_sms() * 8, 256, 0, s>>>(nd, g->rays_dev, g->n_sub, g->wb);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status launch_ext_tc(const ExtLaunch &a, const __nv_bfloat16 *const *brick, cd_geom g, cudaStream_t s)
{
    if (a.k < 4 || !g->wb || !tc_supported(a.nd)) {
        set_error("tensor-core shell needs level >= 4 and a supported direction count");
        return CD_EUNSUPPORTED;
    }
    TcArgs P = {};
    P.k = a.k;
    P.nd = a.nd;
    P.N = 8 * a.nd;
    P.Nt = 4 * a.nd;
    // any contiguous run of tables t0..t1: chunks [(t0-1) 5, t1 5)
    int t0 = 0, t1 = 0;
    for (int t = 1; t <= 3; ++t)
        if (a.tmask & (1 << (t - 1))) {
            if (!t0) t0 = t;
            t1 = t;
        }
    const int run = t0 ? ((1 << t1) - 1) & ~((1 << (t0 - 1)) - 1) : 0;
    if (!t0 || a.tmask != run) {
        set_error("tensor-core shell serves a contiguous run of tables (mask %d)", a.tmask);
        return CD_EUNSUPPORTED;
    }
    constexpr int kChunksPerTable = kBricksPerTable / kChunkBricks;
    P.c0 = (t0 - 1) * kChunksPerTable;
    P.c1 = t1 * kChunksPerTable;
    P.brick[0] = nullptr;
    P.brick[1] = brick[a.k];
    P.brick[2] = brick[a.k - 1];
    P.brick[3] = brick[a.k - 2];
    P.B = g->wb;
    P.out = a.out;
    P.dx_k = a.dx[t0] / (float)(1 << (t0 - 1));   // dx of table t's level = 2^(t-1) dx_k
    P.nG = (int64_t)1 << (3 * (a.k - 3));
    P.ntiles = 2 * 64 * ((P.nG + 127) / 128);
    P.tiles = nullptr;
    P.row_key = nullptr;
    P.row_out = nullptr;
    if (a.list) {
        P.tiles = a.list->tiles;
        P.row_key = a.list->key;
        P.row_out = a.list->out;
        P.ntiles = a.list->ntiles;
        if (P.ntiles == 0) return CD_OK;
    }
    const size_t smem = tc_smem_bytes((size_t)P.Nt * kChunkBricks * 16, false);
    CD_CUDA(cudaFuncSetAttribute(shell_sum_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // persistent CTAs hold every SM until the last tile; n tiles per CTA let the
    // CTAs of other streams' launches in as these retire
    const int64_t grid = a.tiles_per_cta > 0 ? (P.ntiles + a.tiles_per_cta - 1) / a.tiles_per_cta
                                             : std::min<int64_t>(P.ntiles, 2 * (int64_t)num_sms());
    {
        // every tile runs its chunks' MMAs over 128 rows and Nt columns, K = 48 a chunk
        LaunchScope ls(CD_K_SHELL, s, 2.0 * (double)P.ntiles * 128.0 * (P.c1 - P.c0) * (kChunkBricks * 8) * P.Nt);
        shell_sum_tc<false><<<(unsigned)grid, kThreads, smem, s>>>(P, TcBatch{});
    }
    CD_CHECK_LAUNCH();
    if (a.prefix_in && a.list) {
        // S_k[i] += S_{k-1}[parent index of receiver i]
        const cd_status st = launch_add_parent_list(a.out, a.prefix_in, a.list->recv_parent, a.nd, a.list->n_recv, s);
        if (st != CD_OK) return st;
    } else if (a.prefix_in) {
        // S_k[c] += S_{k-1}[parent c]
        const int64_t n = ((int64_t)1 << (3 * a.k)) * a.nd;
        LaunchScope ls(CD_K_SHELL, s);
        add_parent_rows<<<(unsigned)std::min<int64_t>((n / 4 + 255) / 256, 152 * 16), 256, 0, s>>>(a.out, a.prefix_in, a.nd, n);
        CD_CHECK_LAUNCH();
    }
    return CD_OK;
}

size_t tc_job_bytes() { return sizeof(TcArgs); }

int64_t tc_job_fill(const TcJobDesc &d, const __nv_bfloat16 *const *brick, cd_geom g, void *dst)
{
    const ExtLaunch &a = d.a;
    if (a.k < 4 || !g->wb || !tc_supported(a.nd)) return -1;
    if (d.full && !(8 * a.nd <= 256 && (8 * a.nd) % 16 == 0)) return -1;
    int t0 = 0, t1 = 0;
    for (int t = 1; t <= 3; ++t)
        if (a.tmask & (1 << (t - 1))) {
            if (!t0) t0 = t;
            t1 = t;
        }
    const int run = t0 ? ((1 << t1) - 1) & ~((1 << (t0 - 1)) - 1) : 0;
    if (!t0 || a.tmask != run) return -1;
    constexpr int kChunksPerTable = kBricksPerTable / kChunkBricks;
    TcArgs P = {};
    P.k = a.k;
    P.nd = a.nd;
    P.N = 8 * a.nd;
    P.full = d.full ? 1 : 0;
    P.Nt = d.full ? 8 * a.nd : 4 * a.nd;
    P.c0 = (t0 - 1) * kChunksPerTable;
    P.c1 = t1 * kChunksPerTable;
    P.brick[1] = brick[a.k];
    P.brick[2] = brick[a.k - 1];
    P.brick[3] = brick[a.k - 2];
    P.B = g->wb;
    P.out = a.out;
    P.dx_k = a.dx[t0] / (float)(1 << (t0 - 1));
    P.nG = (int64_t)1 << (3 * (a.k - 3));
    P.ntiles = (d.full ? 64 : 128) * ((P.nG + 127) / 128);
    if (a.list) {
        P.tiles = a.list->tiles;
        P.row_key = a.list->key;
        P.row_out = a.list->out;
        P.ntiles = d.full ? a.list->ntiles / 2 : a.list->ntiles;
    }
    P.prefix = d.prefix;
    P.prefix_row = d.prefix_row;
    P.wait_job = d.wait_job;
    P.wait_count = d.wait_count;
    memcpy(dst, &P, sizeof(P));
    return P.ntiles;
}

double tc_job_flops(const void *job)
{
    TcArgs P;
    memcpy(&P, job, sizeof(P));
    return 2.0 * (double)P.ntiles * 128.0 * (P.c1 - P.c0) * (kChunkBricks * 8) * P.Nt;
}

uint32_t tc_job_bstage(const void *job)
{
    TcArgs P;
    memcpy(&P, job, sizeof(P));
    return (uint32_t)P.Nt * kChunkBricks * 16;
}

void tc_job_set_signal(void *job)
{
    TcArgs *P = static_cast<TcArgs *>(job);
    P->signal = 1;
}

cd_status launch_tc_batch(const void *jobs, const int2 *tile_ref, int64_t total, int *done, int *claim,
                          uint32_t bstage_max, int ctas_per_sm, double flops, cudaStream_t s, int *ctas_used)
{
    if (ctas_used) *ctas_used = 0;
    if (total <= 0) return CD_OK;
    TcBatch Bt;
    Bt.jobs = static_cast<const TcArgs *>(jobs);
    Bt.tile_ref = tile_ref;
    Bt.total = total;
    Bt.done = done;
    Bt.claim = claim;
    Bt.bstage_max = bstage_max;
    const size_t smem = tc_smem_bytes(bstage_max, true);
    CD_CUDA(cudaFuncSetAttribute(shell_sum_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // two CTAs per SM need the largest shared-memory carveout
    CD_CUDA(cudaFuncSetAttribute(shell_sum_tc<true>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared));
    // CTAs claim tiles from the work counter, so the grid need not be resident
    // at once (the runtime's occupancy figure counts one CTA per SM for any
    // kernel that allocates tensor memory; two of these fit an SM's registers,
    // shared memory and tensor memory)
    if (2 * (smem + 2048) > 233472) ctas_per_sm = 1;
    const int per_sm = std::max(1, std::min(2, ctas_per_sm));
    if (ctas_used) *ctas_used = per_sm;
    const int64_t grid = std::min<int64_t>(total, (int64_t)per_sm * num_sms());
    LaunchScope ls(CD_K_SHELL, s, flops);
    shell_sum_tc<true><<<(unsigned)grid, kThreads, smem, s>>>(TcArgs{}, Bt);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

// out[i][4j .. 4j+3] += prefix[parent[i]][4j .. 4j+3]: one float4 per thread
// (nd % 4 == 0, 16-byte aligned rows)
__global__ void add_parent_list4(float *__restrict__ out, const float *__restrict__ prefix,
                                 const int32_t *__restrict__ parent, int nq, int64_t n4)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n4; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / nq;
        float4 v = reinterpret_cast<float4 *>(out)[e];
        const float4 p = reinterpret_cast<const float4 *>(prefix)[(int64_t)parent[i] * nq + (e - i * nq)];
        v.x += p.x;
        v.y += p.y;
        v.z += p.z;
        v.w += p.w;
        reinterpret_cast<float4 *>(out)[e] = v;
    }
}

cd_status launch_add_parent_list(float *out, const float *prefix, const int32_t *parent, int nd, int64_t rows,
                                 cudaStream_t s)
{
    const int64_t n = rows * nd;
    if (n == 0) return CD_OK;
    LaunchScope ls(CD_K_SHELL, s);
    if (nd % 4 == 0 && ((uintptr_t)out & 15) == 0 && ((uintptr_t)prefix & 15) == 0) {
        const int64_t n4 = n / 4;
        add_parent_list4<<<(unsigned)std::min<int64_t>((n4 + 255) / 256, 152 * 32), 256, 0, s>>>(out, prefix, parent,
                                                                                                 nd / 4, n4);
    } else {
        add_parent_list<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, s>>>(out, prefix, parent,
                                                                                               nd, n);
    }
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
