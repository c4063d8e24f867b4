// Adaptive (AMR) octrees: leaves at levels base .. lmax that tile the box.
//
// Build (host, once per mesh): leaves are validated, ordered depth-first
// (Morton key of their first finest cell), checked to tile the box exactly,
// and the mesh is described per level by
//   - the refined cells of level k (sorted Morton keys, parent index in level
//     k-1): they receive the far-shell prefix S_k (§3.3, two-level
//     approximation for Δl >= 3);
//   - the leaf-bearing octs of level k (refined cells with at least one leaf
//     child at k+1): they receive the three nearest shells E, and their leaf
//     children get the internal and local terms (§3.2).
// Update (device, every step): the leaf densities are permuted into output
// order, the dense volume-mean arrays of levels 0 .. lmax-1 are rebuilt (a
// cell inside a coarser leaf takes that leaf's value, a refined cell the mean
// of its children: the coarse density "corresponds to a mean", §3.2) --
// top-down from the base level to the finest dense level, then the
// restriction below it -- and the per-oct sibling densities are gathered.
//
// Shells and leaves run over these lists with the same tables as the uniform
// tree; the stencil densities come from the dense level arrays.
#include <algorithm>
#include <numeric>
#include <vector>

#include <string.h>

#include "common.cuh"

namespace cd {
namespace {

inline unsigned grid_for(int64_t n, int block, int cap = 152 * 32)
{
    int64_t g = (n + block - 1) / block;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// ---- update kernels ------------------------------------------------------------

// The dense level arrays above the base are built top-down: a cell inside a
// leaf of a coarser level takes the value its parent already holds (a
// coalesced pass per level), the leaves of the level are scattered in, and a
// cell refined at that level is marked NaN until its mean arrives (from
// mean_finest at the finest dense level, from the restriction below it).
// Leaf densities are finite (checked on the host path), so NaN is free as a
// marker.

// Dense levels whose leaves take their values in the gather below: bit l of
// mask set for every level that no prolongation writes afterwards
struct LeafScatter {
    float *dense[CD_MAXL + 1];
    uint32_t mask;
};

// One launch for two independent passes over disjoint arrays: entries [0, n)
// gather the caller's leaf densities into output order (and into the dense
// array of the leaf's level when D.mask has it), entries [n, n + nr) mark the
// base level's refined cells NaN
__global__ void gather_and_mark(const float *__restrict__ in, const int64_t *__restrict__ src, int64_t n,
                                float *__restrict__ out, const uint64_t *__restrict__ keys, int64_t nr, int l,
                                float *__restrict__ dense, const uint64_t *__restrict__ lkey,
                                const int8_t *__restrict__ llvl, const __grid_constant__ LeafScatter D,
                                const int32_t *__restrict__ slot, float *__restrict__ rho8)
{
    const int64_t side = (int64_t)1 << l;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n + nr; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n) {
            const float v = in[src[i]];
            out[i] = v;
            const int32_t sl = slot[i];   // the leaf as child of its oct (-1: no oct)
            if (sl >= 0) rho8[sl] = v;
            const int lv = llvl[i];
            if ((D.mask >> lv) & 1u) {
                const uint64_t m = lkey[i];
                const int64_t sd = (int64_t)1 << lv;
                D.dense[lv][((int64_t)compact3(m >> 2) * sd + compact3(m >> 1)) * sd + compact3(m)] = v;
            }
        } else {
            const uint64_t m = keys[i - n];
            dense[((int64_t)compact3(m >> 2) * side + compact3(m >> 1)) * side + compact3(m)] = __int_as_float(0x7fc00000);
        }
    }
}

// The leaves of level l, from the leaf-bearing octs of level l - 1: entry e is
// child e % 8 of oct e / 8 (row -1: refined, left as it is).
__global__ void scatter_octs(const float *__restrict__ rho, const uint64_t *__restrict__ okey,
                             const int32_t *__restrict__ oleaf, int64_t n, int l, float *__restrict__ dense)
{
    const int64_t side = (int64_t)1 << l;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < 8 * n; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = oleaf[e];
        if (r < 0) continue;
        const uint64_t m = (okey[e >> 3] << 3) | (uint64_t)(e & 7);
        dense[((int64_t)compact3(m >> 2) * side + compact3(m >> 1)) * side + compact3(m)] = rho[r];
    }
}

// Four cells of a row per thread (side >= 4): the parents of x .. x+3 are
// x/2 and x/2 + 1, so one float4 store takes (a, a, b, b).
__global__ void prolong4(const float *__restrict__ coarse, int l, float *__restrict__ fine)
{
    const int64_t side = (int64_t)1 << l, n4 = side * side * side / 4;
    const int sh = l;
    const int64_t hs = side >> 1;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = 4 * q;
        const int64_t x = c & (side - 1), y = (c >> sh) & (side - 1), z = c >> (2 * sh);
        const float *row = coarse + ((z >> 1) * hs + (y >> 1)) * hs + (x >> 1);
        const float a = row[0], b = row[1];
        reinterpret_cast<float4 *>(fine)[q] = make_float4(a, a, b, b);
    }
}

// fine[c] = coarse[parent c] over the row-major level l (NaN propagates: the
// children of a refined cell are leaves or refined cells of level l).
__global__ void prolong(const float *__restrict__ coarse, int l, float *__restrict__ fine)
{
    const int64_t side = (int64_t)1 << l, n = side * side * side;
    const int sh = l;                     // log2 side
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n; c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t x = c & (side - 1), y = (c >> sh) & (side - 1), z = c >> (2 * sh);
        const int64_t hs = side >> 1;
        fine[c] = coarse[((z >> 1) * hs + (y >> 1)) * hs + (x >> 1)];
    }
}

// Octs of level lf whose 8 children are leaves of level lf + 1: the cell value
// is the mean of the children (same order and rounding as the restriction).
__global__ void mean_finest(const float *__restrict__ rho, const uint64_t *__restrict__ okey,
                            const int32_t *__restrict__ oleaf, int64_t n, int lf, float *__restrict__ out)
{
    const int64_t side = (int64_t)1 << lf;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = okey[i];
        float s = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o) s += rho[oleaf[8 * i + o]];
        out[((int64_t)compact3(m >> 2) * side + compact3(m >> 1)) * side + compact3(m)] = s * 0.125f;
    }
}

// Refined cells of level l take the mean of their 8 children at level l + 1
// (octant order, then x 1/8, as the restriction): the children are leaves or
// refined cells, all written before.
__global__ void fill_refined(const uint64_t *__restrict__ keys, int64_t n, int l, const float *__restrict__ child,
                             float *__restrict__ dense)
{
    const int64_t side = (int64_t)1 << l, cs = side * 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = keys[i];
        const int64_t x = compact3(m), y = compact3(m >> 1), z = compact3(m >> 2);
        float sum = 0.f;
#pragma unroll
        for (int o = 0; o < 8; ++o)
            sum += child[((2 * z + ((o >> 2) & 1)) * cs + 2 * y + ((o >> 1) & 1)) * cs + 2 * x + (o & 1)];
        dense[(z * side + y) * side + x] = sum * 0.125f;
    }
}

// The read part of the sparse finest level lf: for each listed cell of level
// lf - 1, paint its 8 children with its value unless it is refined (then they
// hold leaves and means already), and write their BF16 brick.
__global__ void fill_deep(const uint64_t *__restrict__ keys, const int8_t *__restrict__ paint, int64_t n, int lf,
                          const float *__restrict__ parent, float *__restrict__ fine, __nv_bfloat16 *__restrict__ brick)
{
    const int64_t ps = (int64_t)1 << (lf - 1), fs = ps * 2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t m = keys[i];
        const int64_t x = compact3(m), y = compact3(m >> 1), z = compact3(m >> 2);
        const int64_t p = (z * ps + y) * ps + x;
        const float v = parent[p];
        __align__(16) __nv_bfloat16 bv[8];
#pragma unroll
        for (int o = 0; o < 8; ++o) {
            float *c = fine + ((2 * z + ((o >> 2) & 1)) * fs + 2 * y + ((o >> 1) & 1)) * fs + 2 * x + (o & 1);
            if (paint[i]) *c = v;
            bv[o] = __float2bfloat16_rn(*c);
        }
        *reinterpret_cast<uint4 *>(brick + 8 * p) = *reinterpret_cast<const uint4 *>(bv);
    }
}

// Sibling densities of every oct (oct_rho8, [n_oct][8]): a leaf child's own
// density is written by gather_and_mark (through leaf_slot); this launch
// takes the refined children, each the volume mean at level k+1 from the
// dense array (ref8 lists their slots 8 oct + child; the octs are stored
// level by level, oct_begin[k] .. oct_begin[k+1]).
struct Rho8Args {
    const uint64_t *okey;
    const int32_t *ref8;
    float *rho8;
    int64_t n;                           // refined children
    int nlev;                            // levels 0 .. nlev-1 hold octs
    int64_t begin[CD_MAXL + 2];          // oct_begin
    const float *dense[CD_MAXL + 1];     // level k+1 as a dense array
};

__global__ void gather_rho8(const __grid_constant__ Rho8Args A)
{
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < A.n; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = A.ref8[q];
        const int64_t i = e >> 3;
        const int o = (int)(e & 7);
        int k = 0;
        while (k + 1 < A.nlev && i >= A.begin[k + 1]) ++k;
        const int64_t side = (int64_t)1 << (k + 1);
        const uint64_t m = A.okey[i];
        const int64_t x = 2 * (int64_t)compact3(m) + (o & 1), y = 2 * (int64_t)compact3(m >> 1) + ((o >> 1) & 1),
                      z = 2 * (int64_t)compact3(m >> 2) + ((o >> 2) & 1);
        A.rho8[e] = A.dense[k][(z * side + y) * side + x];
    }
}

// ---- list kernels --------------------------------------------------------------

struct ShellListArgs {
    int k, nd, tmask;
    const float *lvl[4];         // dense level arrays of the shell level of table t (k - t + 1)
    float dx[4];
    const uint64_t *keys;        // receiving cells (Morton keys at level k)
    int64_t n;
    const int32_t *parent;       // index of each receiver's parent in the prefix rows
    const float *prefix;         // S_{k-1} rows or NULL
    float *out;                  // [n][nd]
    const int2 *tab[4];
    const int *cmax[4];
    int maxe;                    // entries per table row
};

// Eq. N_discret for a list of receiving cells: thread per (cell, direction),
// stencil densities read from the dense level arrays (zero outside the box).
__device__ __forceinline__ void shell_list_body(const ShellListArgs &P, int64_t e0, int64_t step)
{
    const int nd = P.nd;
    for (int64_t e = e0; e < P.n * nd; e += step) {
        const int64_t i = e / nd;
        const int d = (int)(e - i * nd);
        const uint64_t m = P.keys[i];
        const int64_t cx = compact3(m), cy = compact3(m >> 1), cz = compact3(m >> 2);
        float acc = P.prefix ? P.prefix[(int64_t)P.parent[i] * nd + d] : 0.f;
        for (int t = 1; t <= 3; ++t) {
            if (!(P.tmask & (1 << (t - 1)))) continue;
            const int64_t side = (int64_t)1 << (P.k - t + 1);
            const int R = region_side(t);
            const int64_t ox = 2 * ((cx >> t) - 1), oy = 2 * ((cy >> t) - 1), oz = 2 * ((cz >> t) - 1);
            const int cfg = (int)(m & ((1u << (3 * t)) - 1));
            const int2 *row = P.tab[t] + (size_t)cfg * P.maxe * nd + d;
            const int cnt = P.cmax[t][cfg];
            const float *rho = P.lvl[t];
            float part = 0.f;
            for (int q = 0; q < cnt; ++q) {
                const int2 v = row[(size_t)q * nd];
                const int a = v.x % R, b = (v.x / R) % R, c = v.x / (R * R);
                const int64_t gx = ox + a, gy = oy + b, gz = oz + c;
                if (gx >= 0 && gy >= 0 && gz >= 0 && gx < side && gy < side && gz < side &&
                    in_bounds(v.x, R * R * R, kCheckListLevel))
                    part = fmaf(rho[(gz * side + gy) * side + gx], __int_as_float(v.y), part);
            }
            acc = fmaf(P.dx[t], part, acc);
        }
        P.out[e] = acc;
    }
}

__global__ void __launch_bounds__(256) shell_list_fp32(ShellListArgs P)
{
    shell_list_body(P, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// many lists in one launch: blockIdx.y selects the list (cd_batch)
__global__ void __launch_bounds__(256) shell_list_fp32_batch(const ShellListArgs *jobs)
{
    const ShellListArgs P = jobs[blockIdx.y];
    shell_list_body(P, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

struct LeafListArgs {
    int64_t n;                   // octs of this level
    int nd;
    float dx_leaf, av_per_nh, c_exp2, inv_nd;
    const float *rho8;           // [n][8]
    const int32_t *oleaf;        // [n][8] leaf rows, -1 for refined children
    const float *E;              // [n][nd]
    const float *Sp;             // parent prefix rows or NULL
    const int32_t *oparent;      // [n]
    const float *kloc;
    float *n_h, *a_v, *shield;
};

// Internal + local terms and the epilogue for the leaf children of a list of
// octs: one warp per oct, its lanes over (child t, 4 directions) units in
// child-major order, so that consecutive lanes write consecutive 16-byte
// pieces of the children's rows (an oct's leaf rows are consecutive unless a
// refined sibling's subtree lies between them).  The oct's 8 densities and leaf
// rows are read once per warp and broadcast by shuffles; the external and
// prefix rows are shared by the 8 children (L1 hits); the local weights come
// from shared memory.  The screening sum of a child adds its units' partial
// sums in a fixed order through shared memory.
// Directions are a multiple of 4 here (leaf_list_scalar serves the rest).
__global__ void __launch_bounds__(256) leaf_list(LeafListArgs P)
{
    extern __shared__ float sm[];
    const int nd = P.nd, nq = nd >> 2, nu = 8 * nq;
    float *s_k = sm;                          // [8 t][8 s][nd], times dx
    for (int i = threadIdx.x; i < 64 * nd; i += blockDim.x) s_k[i] = P.dx_leaf * P.kloc[i];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *s_e = sm + 64 * nd + w * nu;       // this warp's per-unit screening partial sums
    const int iters = (nu + 31) >> 5;
    for (int64_t ii = (int64_t)blockIdx.x * 8 + w; ii < P.n; ii += (int64_t)gridDim.x * 8) {
        const float r = P.rho8[8 * ii + (lane & 7)];
        const int row_l = P.oleaf[8 * ii + (lane & 7)];
        float rho[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) rho[s] = __shfl_sync(0xffffffffu, r, s);
        const float *E = P.E + ii * nd;
        const float *Sp = P.Sp ? P.Sp + (int64_t)P.oparent[ii] * nd : nullptr;
        for (int j = 0; j < iters; ++j) {
            const int u = lane + 32 * j;
            const bool valid = u < nu;
            const int t = valid ? u / nq : 0, d = 4 * (u - t * nq);
            const int row = __shfl_sync(0xffffffffu, row_l, t);
            if (!valid) continue;
            float e = 0.f;
            if (row >= 0) {
                float4 nv = *reinterpret_cast<const float4 *>(E + d);
                if (Sp) {
                    const float4 p = *reinterpret_cast<const float4 *>(Sp + d);
                    nv.x += p.x;
                    nv.y += p.y;
                    nv.z += p.z;
                    nv.w += p.w;
                }
                const float *kt = s_k + t * 8 * nd + d;
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const float4 k4 = *reinterpret_cast<const float4 *>(kt + s * nd);
                    nv.x = fmaf(rho[s], k4.x, nv.x);
                    nv.y = fmaf(rho[s], k4.y, nv.y);
                    nv.z = fmaf(rho[s], k4.z, nv.z);
                    nv.w = fmaf(rho[s], k4.w, nv.w);
                }
                const int64_t o = (int64_t)row * nd + d;
                if (P.n_h) *reinterpret_cast<float4 *>(P.n_h + o) = nv;
                if (P.a_v)
                    *reinterpret_cast<float4 *>(P.a_v + o) =
                        make_float4(nv.x * P.av_per_nh, nv.y * P.av_per_nh, nv.z * P.av_per_nh, nv.w * P.av_per_nh);
                e = (exp2f(P.c_exp2 * nv.x) + exp2f(P.c_exp2 * nv.y)) + (exp2f(P.c_exp2 * nv.z) + exp2f(P.c_exp2 * nv.w));
            }
            s_e[u] = e;
        }
        __syncwarp();
        if (lane < 8 && P.shield && row_l >= 0) {
            float a = 0.f;
            for (int q = 0; q < nq; ++q) a += s_e[lane * nq + q];
            P.shield[row_l] = a * P.inv_nd;
        }
        __syncwarp();
    }
}

// Same work for direction counts that are not a multiple of 4 (one warp per
// oct, lanes over (child, direction)); the screening sum in a fixed order.
__global__ void __launch_bounds__(256) leaf_list_scalar(LeafListArgs P)
{
    extern __shared__ float sm[];
    const int nd = P.nd;
    float *s_k = sm;                          // [8 t][8 s][nd], times dx
    float *s_e = sm + 64 * nd;                // [8 warps][8 nd]
    __shared__ int s_row[8][8];
    for (int i = threadIdx.x; i < 64 * nd; i += blockDim.x) s_k[i] = P.dx_leaf * P.kloc[i];
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *e_w = s_e + w * 8 * nd;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < P.n; i += (int64_t)gridDim.x * 8) {
        const float r = P.rho8[8 * i + (lane & 7)];
        float rs[8];
#pragma unroll
        for (int s = 0; s < 8; ++s) rs[s] = __shfl_sync(0xffffffffu, r, s);
        if (lane < 8) s_row[w][lane] = P.oleaf[8 * i + lane];
        __syncwarp();
        const float *E = P.E + i * nd;
        const float *Sp = P.Sp ? P.Sp + (int64_t)P.oparent[i] * nd : nullptr;
        for (int f = lane; f < 8 * nd; f += 32) {
            const int t = f / nd, d = f - t * nd;
            const int row = s_row[w][t];
            if (row < 0) continue;
            float nv = E[d] + (Sp ? Sp[d] : 0.f);
            const float *kl = s_k + t * 8 * nd + d;
#pragma unroll
            for (int s = 0; s < 8; ++s) nv = fmaf(rs[s], kl[s * nd], nv);
            if (P.n_h) P.n_h[(int64_t)row * nd + d] = nv;
            if (P.a_v) P.a_v[(int64_t)row * nd + d] = nv * P.av_per_nh;
            e_w[f] = exp2f(P.c_exp2 * nv);
        }
        __syncwarp();
        if (P.shield && lane < 8 && s_row[w][lane] >= 0) {
            float acc = 0.f;
            for (int d = 0; d < nd; ++d) acc += e_w[lane * nd + d];
            P.shield[s_row[w][lane]] = acc * P.inv_nd;
        }
        __syncwarp();
    }
}

}  // namespace

// ---- tensor-core lists -------------------------------------------------------------

// Receivers (sorted Morton keys of one level, output row = position) -> their
// distinct parents grouped by class (low six Morton bits) with the output row
// of each child, and the tiles (128 rows, two halves) over each class.
static cd_status build_tc_list(const std::vector<uint64_t> &recv, int32_t *recv_parent, TcList &L)
{
    L = TcList();
    L.n_recv = (int64_t)recv.size();
    L.recv_parent = recv_parent;
    if (recv.empty()) return CD_OK;
    std::vector<uint64_t> key;
    std::vector<int32_t> out;
    for (size_t i = 0; i < recv.size(); ++i) {
        const uint64_t p = recv[i] >> 3;
        if (key.empty() || key.back() != p) {
            key.push_back(p);
            out.insert(out.end(), 8, -1);
        }
        out[8 * (key.size() - 1) + (recv[i] & 7)] = (int32_t)i;
    }
    std::vector<size_t> ord(key.size());
    std::iota(ord.begin(), ord.end(), (size_t)0);
    std::stable_sort(ord.begin(), ord.end(), [&](size_t a, size_t b) { return (key[a] & 63) < (key[b] & 63); });
    std::vector<uint64_t> skey(key.size());
    std::vector<int32_t> sout(out.size());
    for (size_t r = 0; r < ord.size(); ++r) {
        skey[r] = key[ord[r]];
        for (int o = 0; o < 8; ++o) sout[8 * r + o] = out[8 * ord[r] + o];
    }
    std::vector<int4> tiles;
    for (size_t i = 0; i < skey.size();) {
        const int cls = (int)(skey[i] & 63);
        size_t j = i;
        while (j < skey.size() && (int)(skey[j] & 63) == cls) ++j;
        for (size_t b = i; b < j; b += 128)
            for (int h = 0; h < 2; ++h) tiles.push_back(make_int4(cls, (int)b, (int)std::min<size_t>(128, j - b), h));
        i = j;
    }
    L.nrows = (int64_t)skey.size();
    L.ntiles = (int64_t)tiles.size();
    if (cudaMalloc(&L.key, skey.size() * 8) != cudaSuccess || cudaMalloc(&L.out, sout.size() * 4) != cudaSuccess ||
        cudaMalloc(&L.tiles, tiles.size() * sizeof(int4)) != cudaSuccess) {
        cudaGetLastError();
        set_error("tensor-core list allocation failed");
        return CD_ENOMEM;
    }
    if (cudaMemcpy(L.key, skey.data(), skey.size() * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(L.out, sout.data(), sout.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(L.tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("tensor-core list upload failed");
        return CD_ECUDA;
    }
    return CD_OK;
}

// ---- host build ------------------------------------------------------------------

cd_status build_amr(cd_tree t, int base, int lmax, int64_t n, const int8_t *level, const int32_t *ijk)
{
    if (base < 1 || lmax < base || lmax > 11) {
        set_error("AMR levels must satisfy 1 <= base <= max_level <= 11 (got %d, %d)", base, lmax);
        return CD_EINVAL;
    }
    if (n < 1) {
        set_error("no leaves");
        return CD_EINVAL;
    }
    // depth-first order: Morton key of the first finest cell
    std::vector<uint64_t> fine(n), key(n);
    for (int64_t i = 0; i < n; ++i) {
        const int l = level[i];
        if (l < base || l > lmax) {
            set_error("leaf %lld has level %d outside [%d, %d]", (long long)i, l, base, lmax);
            return CD_EINVAL;
        }
        const int64_t side = (int64_t)1 << l;
        const int64_t x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
        if (x < 0 || y < 0 || z < 0 || x >= side || y >= side || z >= side) {
            set_error("leaf %lld index (%lld, %lld, %lld) outside its level", (long long)i, (long long)x, (long long)y,
                      (long long)z);
            return CD_EINVAL;
        }
        key[i] = morton3((uint32_t)x, (uint32_t)y, (uint32_t)z);
        fine[i] = key[i] << (3 * (lmax - l));
    }
    std::vector<int64_t> ord(n);
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int64_t a, int64_t b) { return fine[a] < fine[b]; });
    // exact tiling: consecutive leaves abut and cover 8^lmax finest cells
    uint64_t expect = 0;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t i = ord[r];
        if (fine[i] != expect) {
            set_error(fine[i] < expect ? "leaves overlap (near leaf %lld)" : "leaves leave a gap (near leaf %lld)",
                      (long long)i);
            return CD_EINVAL;
        }
        expect += (uint64_t)1 << (3 * (lmax - level[i]));
    }
    if (expect != (uint64_t)1 << (3 * lmax)) {
        set_error("leaves do not cover the box");
        return CD_EINVAL;
    }
    // output-order arrays (host)
    t->leaf_level_h = new int8_t[n];
    t->leaf_ijk_h = new int32_t[3 * n];
    t->leaf_src_h = new int64_t[n];
    std::vector<uint64_t> okey(n);
    std::vector<int8_t> olvl(n);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t i = ord[r];
        t->leaf_level_h[r] = level[i];
        for (int a = 0; a < 3; ++a) t->leaf_ijk_h[3 * r + a] = ijk[3 * i + a];
        t->leaf_src_h[r] = i;
        okey[r] = key[i];
        olvl[r] = level[i];
    }
    // refined cells per level: all cells below base; ancestors of deeper leaves from base on
    std::vector<std::vector<uint64_t>> ref(lmax + 1);
    for (int k = 0; k < base; ++k) {
        ref[k].resize((size_t)1 << (3 * k));
        std::iota(ref[k].begin(), ref[k].end(), (uint64_t)0);
    }
    for (int64_t r = 0; r < n; ++r)
        for (int k = base; k < olvl[r]; ++k) {
            const uint64_t a = okey[r] >> (3 * (olvl[r] - k));
            if (ref[k].empty() || ref[k].back() != a) ref[k].push_back(a);   // leaves are in depth-first order
        }
    for (int k = base; k <= lmax; ++k) {
        std::sort(ref[k].begin(), ref[k].end());
        ref[k].erase(std::unique(ref[k].begin(), ref[k].end()), ref[k].end());
    }
    // leaf-bearing octs, grouped by level, depth-first within a level
    std::vector<std::vector<uint64_t>> oct(lmax + 1);
    std::vector<std::vector<int32_t>> oleaf(lmax + 1);
    {
        std::vector<std::vector<std::pair<uint64_t, int64_t>>> tmp(lmax + 1);
        for (int64_t r = 0; r < n; ++r) tmp[olvl[r] - 1].push_back({okey[r], r});
        for (int k = 0; k < lmax; ++k) {
            auto &v = tmp[k];
            std::sort(v.begin(), v.end());
            for (size_t j = 0; j < v.size(); ++j) {
                const uint64_t p = v[j].first >> 3;
                if (oct[k].empty() || oct[k].back() != p) {
                    oct[k].push_back(p);
                    oleaf[k].insert(oleaf[k].end(), 8, -1);
                }
                oleaf[k][8 * (oct[k].size() - 1) + (v[j].first & 7)] = (int32_t)v[j].second;
            }
        }
    }
    // parents
    auto parent_index = [&](int k, uint64_t cellkey) -> int32_t {
        if (k < 1) return -1;
        const auto &v = ref[k - 1];
        auto it = std::lower_bound(v.begin(), v.end(), cellkey >> 3);
        return (it != v.end() && *it == (cellkey >> 3)) ? (int32_t)(it - v.begin()) : -1;
    };
    // upload
    cd_status st = CD_OK;
    auto up = [&](void **dst, const void *src, size_t bytes) -> bool {
        if (bytes == 0) return true;
        if (cudaMalloc(dst, bytes) != cudaSuccess) {
            cudaGetLastError();
            set_error("AMR tree allocation failed (%zu bytes)", bytes);
            st = CD_ENOMEM;
            return false;
        }
        if (src && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            set_error("AMR tree upload failed");
            st = CD_ECUDA;
            return false;
        }
        return true;
    };
    for (int k = 0; k <= lmax; ++k) {
        t->n_ref[k] = (int64_t)ref[k].size();
        if (!t->n_ref[k]) continue;
        std::vector<int32_t> par(ref[k].size());
        for (size_t j = 0; j < ref[k].size(); ++j) par[j] = parent_index(k, ref[k][j]);
        if (!up((void **)&t->ref_key[k], ref[k].data(), ref[k].size() * 8)) return st;
        if (!up((void **)&t->ref_parent[k], par.data(), par.size() * 4)) return st;
    }
    std::vector<uint64_t> allkey;
    std::vector<int32_t> allpar, allleaf;
    for (int k = 0; k <= lmax; ++k) {
        t->oct_begin[k] = (int64_t)allkey.size();
        for (size_t j = 0; j < oct[k].size(); ++j) {
            allkey.push_back(oct[k][j]);
            allpar.push_back(parent_index(k, oct[k][j]));
        }
        allleaf.insert(allleaf.end(), oleaf[k].begin(), oleaf[k].end());
    }
    t->oct_begin[lmax + 1] = (int64_t)allkey.size();
    t->n_oct = (int64_t)allkey.size();
    if (!up((void **)&t->oct_key, allkey.data(), allkey.size() * 8)) return st;
    if (!up((void **)&t->oct_parent, allpar.data(), allpar.size() * 4)) return st;
    if (!up((void **)&t->oct_leaf, allleaf.data(), allleaf.size() * 4)) return st;
    {
        // each leaf's slot among its oct's children, and the refined children's slots
        std::vector<int32_t> slot(n, -1), ref8;
        for (size_t j = 0; j < allleaf.size(); ++j) {
            if (allleaf[j] >= 0) slot[allleaf[j]] = (int32_t)j;
            else ref8.push_back((int32_t)j);
        }
        t->n_ref8 = (int64_t)ref8.size();
        if (!up((void **)&t->leaf_slot, slot.data(), n * 4)) return st;
        if (!up((void **)&t->ref8, ref8.data(), ref8.size() * 4)) return st;
    }
    if (!up((void **)&t->oct_rho8, nullptr, allkey.size() * 8 * 4)) return st;
    if (!up((void **)&t->leaf_key, okey.data(), n * 8)) return st;
    if (!up((void **)&t->leaf_lvl, olvl.data(), n)) return st;
    if (!up((void **)&t->leaf_src, t->leaf_src_h, n * 8)) return st;
    if (!up((void **)&t->rho_leaf, nullptr, n * 4)) return st;
    for (int l = 0; l <= lmax - 1; ++l) {
        const size_t cells = (size_t)1 << (3 * l);
        if (!up((void **)&t->rho_lvl[l], nullptr, cells * 4)) return st;
        if (l >= 1 && !up((void **)&t->rho_brick[l], nullptr, cells * 2)) return st;
    }
    // the read part of the finest dense level (see cd_tree_s): level-(lf-1) cells
    // around the parents of the octs of level lf
    if (lmax - 1 > base && lmax - 1 >= 1 && !oct[lmax - 1].empty()) {
        const int lf = lmax - 1;
        const int64_t ps = (int64_t)1 << (lf - 1);
        std::vector<uint64_t> deep;
        for (uint64_t o : oct[lf]) {
            const uint64_t a = o >> 3;
            const int64_t ax = compact3(a), ay = compact3(a >> 1), az = compact3(a >> 2);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t x = ax + dx, y = ay + dy, z = az + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= ps || y >= ps || z >= ps) continue;
                        deep.push_back(morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
                    }
        }
        std::sort(deep.begin(), deep.end());
        deep.erase(std::unique(deep.begin(), deep.end()), deep.end());
        std::vector<int8_t> paint(deep.size());
        for (size_t j = 0; j < deep.size(); ++j)
            paint[j] = std::binary_search(ref[lf - 1].begin(), ref[lf - 1].end(), deep[j]) ? 0 : 1;
        t->n_deep = (int64_t)deep.size();
        if (!up((void **)&t->deep_key, deep.data(), deep.size() * 8)) return st;
        if (!up((void **)&t->deep_paint, paint.data(), paint.size())) return st;
        t->sparse_finest = 1;
    }
    // the read part of level lm = lf-1 when it lies above the base level:
    // level-(lm-1) cells around the parents of the octs of level lm and around
    // the grandparents of the octs of level lf
    if (t->sparse_finest && lmax - 2 > base) {
        const int lm = lmax - 2;
        const int64_t ps = (int64_t)1 << (lm - 1);
        std::vector<uint64_t> mid;
        auto around = [&](uint64_t a) {
            const int64_t ax = compact3(a), ay = compact3(a >> 1), az = compact3(a >> 2);
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        const int64_t x = ax + dx, y = ay + dy, z = az + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= ps || y >= ps || z >= ps) continue;
                        mid.push_back(morton3((uint32_t)x, (uint32_t)y, (uint32_t)z));
                    }
        };
        for (uint64_t o : oct[lm]) around(o >> 3);
        for (uint64_t o : oct[lm + 1]) around(o >> 6);
        std::sort(mid.begin(), mid.end());
        mid.erase(std::unique(mid.begin(), mid.end()), mid.end());
        std::vector<int8_t> paint(mid.size());
        for (size_t j = 0; j < mid.size(); ++j)
            paint[j] = std::binary_search(ref[lm - 1].begin(), ref[lm - 1].end(), mid[j]) ? 0 : 1;
        t->n_mid = (int64_t)mid.size();
        if (!up((void **)&t->mid_key, mid.data(), mid.size() * 8)) return st;
        if (!up((void **)&t->mid_paint, paint.data(), paint.size())) return st;
        const size_t cells = (size_t)1 << (3 * lm);
        // (memsets are ordered on the legacy stream only: finished here, before any
        // stream writes the painted part)
        if (cudaMemset(t->rho_lvl[lm], 0xff, cells * 4) != cudaSuccess ||
            cudaMemset(t->rho_brick[lm], 0xff, cells * 2) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            set_error("AMR tree initialisation failed");
            return CD_ECUDA;
        }
        t->sparse_mid = 1;
    }
    // tensor-core lists of the levels the BF16 contraction serves (receiving level >= 4)
    for (int k = 4; k <= lmax - 1; ++k) {
        if (k <= lmax - 2 && (st = build_tc_list(ref[k], t->ref_parent[k], t->tc_ref[k])) != CD_OK) return st;
        if ((st = build_tc_list(oct[k], nullptr, t->tc_oct[k])) != CD_OK) return st;
    }
    t->amr = 1;
    t->L = lmax;
    t->base = base;
    t->n_leaf = n;
    return CD_OK;
}

void free_tc_lists(cd_tree t)
{
    for (int k = 0; k <= CD_MAXL; ++k)
        for (TcList *L : {&t->tc_ref[k], &t->tc_oct[k]}) {
            if (L->key) cd::lib_free(L->key);
            if (L->out) cd::lib_free(L->out);
            if (L->tiles) cd::lib_free(L->tiles);
            *L = TcList();
        }
}

// rho: leaf densities in the caller's order (device).
cd_status update_amr(cd_tree t, const float *rho_dev, cudaStream_t s)
{
    const int lmax = t->L, lf = lmax - 1;
    // levels that no prolongation writes: their leaves go in with the gather
    const auto prolonged = [&](int l) {
        return l != t->base && !(t->sparse_finest && l == lf) && !(t->sparse_mid && l == lf - 1);
    };
    LeafScatter D = {};
    for (int l = t->base; l <= lf; ++l) {
        D.dense[l] = t->rho_lvl[l];
        if (!prolonged(l)) D.mask |= 1u << l;
    }
    {
        // leaves into output order (and into the unprolonged dense levels), and
        // the base level's refined cells marked NaN
        const int64_t nr = t->n_ref[t->base];
        LaunchScope ls(CD_K_RESTRICT, s);
        gather_and_mark<<<grid_for(t->n_leaf + nr, 256), 256, 0, s>>>(
            rho_dev, t->leaf_src, t->n_leaf, t->rho_leaf, t->ref_key[t->base], nr, t->base, t->rho_lvl[t->base],
            t->leaf_key, t->leaf_lvl, D, t->leaf_slot, t->oct_rho8);
    }
    CD_CHECK_LAUNCH();
    // dense levels base .. lf, top-down
    for (int l = t->base; l <= lf; ++l) {
        if (l == t->base) {
            // done above
        } else if (!prolonged(l)) {
            // no prolongation into the finest dense levels: fill_deep paints the part that is read
        } else if (l >= 2) {
            LaunchScope ls(CD_K_RESTRICT, s);
            prolong4<<<grid_for((int64_t)1 << (3 * l - 2), 256, 152 * 64), 256, 0, s>>>(t->rho_lvl[l - 1], l,
                                                                                       t->rho_lvl[l]);
        } else {
            LaunchScope ls(CD_K_RESTRICT, s);
            prolong<<<grid_for((int64_t)1 << (3 * l), 256, 152 * 64), 256, 0, s>>>(t->rho_lvl[l - 1], l, t->rho_lvl[l]);
        }
        CD_CHECK_LAUNCH();
        const int64_t no = t->oct_begin[l] - t->oct_begin[l - 1];   // octs of level l - 1: their leaf children
        if (no > 0 && prolonged(l)) {
            LaunchScope ls(CD_K_RESTRICT, s);
            scatter_octs<<<grid_for(8 * no, 256), 256, 0, s>>>(t->rho_leaf, t->oct_key + t->oct_begin[l - 1],
                                                               t->oct_leaf + 8 * t->oct_begin[l - 1], no, l,
                                                               t->rho_lvl[l]);
            CD_CHECK_LAUNCH();
        }
    }
    const int64_t nfin = t->oct_begin[lf + 1] - t->oct_begin[lf];
    if (nfin > 0) {
        LaunchScope ls(CD_K_RESTRICT, s);
        mean_finest<<<grid_for(nfin, 256), 256, 0, s>>>(t->rho_leaf, t->oct_key + t->oct_begin[lf],
                                                        t->oct_leaf + 8 * t->oct_begin[lf], nfin, lf, t->rho_lvl[lf]);
    }
    CD_CHECK_LAUNCH();
    cd_status st = CD_OK;
    if (t->sparse_finest) {
        if (t->n_ref[lf - 1]) {
            LaunchScope ls(CD_K_RESTRICT, s);
            fill_refined<<<grid_for(t->n_ref[lf - 1], 256), 256, 0, s>>>(t->ref_key[lf - 1], t->n_ref[lf - 1], lf - 1,
                                                                         t->rho_lvl[lf], t->rho_lvl[lf - 1]);
            CD_CHECK_LAUNCH();
        }
        if (t->sparse_mid) {
            // level lf-2 complete (its refined cells from lf-1), restricted from
            // there; then the read part of lf-1 and its bricks
            if (t->n_ref[lf - 2]) {
                LaunchScope ls(CD_K_RESTRICT, s);
                fill_refined<<<grid_for(t->n_ref[lf - 2], 256), 256, 0, s>>>(t->ref_key[lf - 2], t->n_ref[lf - 2],
                                                                             lf - 2, t->rho_lvl[lf - 1],
                                                                             t->rho_lvl[lf - 2]);
                CD_CHECK_LAUNCH();
            }
            if ((st = restrict_dense(t, lf - 2, s)) != CD_OK) return st;
            if (t->n_mid) {
                LaunchScope ls(CD_K_RESTRICT, s);
                fill_deep<<<grid_for(t->n_mid, 256), 256, 0, s>>>(t->mid_key, t->mid_paint, t->n_mid, lf - 1,
                                                                  t->rho_lvl[lf - 2], t->rho_lvl[lf - 1],
                                                                  t->rho_brick[lf - 1]);
                CD_CHECK_LAUNCH();
            }
        } else if ((st = restrict_dense(t, lf - 1, s)) != CD_OK) {
            return st;
        }
        if (t->n_deep) {
            LaunchScope ls(CD_K_RESTRICT, s);
            fill_deep<<<grid_for(t->n_deep, 256), 256, 0, s>>>(t->deep_key, t->deep_paint, t->n_deep, lf,
                                                               t->rho_lvl[lf - 1], t->rho_lvl[lf], t->rho_brick[lf]);
            CD_CHECK_LAUNCH();
        }
    } else if ((st = restrict_dense(t, lf, s)) != CD_OK) {
        return st;
    }
    Rho8Args R = {};
    R.okey = t->oct_key;
    R.ref8 = t->ref8;
    R.rho8 = t->oct_rho8;
    R.n = t->n_ref8;
    R.nlev = lmax;
    for (int k = 0; k <= lmax; ++k) R.begin[k] = t->oct_begin[k];
    for (int k = 0; k < lmax; ++k) R.dense[k] = k + 1 <= lf ? t->rho_lvl[k + 1] : nullptr;
    if (R.n > 0) {
        LaunchScope ls(CD_K_RESTRICT, s);
        gather_rho8<<<grid_for(R.n, 256), 256, 0, s>>>(R);
        CD_CHECK_LAUNCH();
    }
    return CD_OK;
}

size_t list_job_bytes() { return sizeof(ShellListArgs); }

void list_job_fill_far3(cd_tree t, cd_geom g, const uint64_t *keys512, void *dst)
{
    ShellListArgs A = {};
    A.k = 3;
    A.nd = g->n_dir;
    A.tmask = 4;
    A.lvl[3] = t->rho_lvl[1];
    A.dx[3] = (float)(t->box_cm / 2.0);
    A.keys = keys512;
    A.n = 512;
    A.parent = nullptr;
    A.prefix = nullptr;
    A.out = t->ws.S[3];
    for (int q = 0; q < 4; ++q) {
        A.tab[q] = g->tab[q];
        A.cmax[q] = g->cmax[q];
    }
    A.maxe = g->maxe;
    memcpy(dst, &A, sizeof(A));
}

cd_status launch_list_batch(const void *jobs, int n_jobs, int64_t max_elems, cudaStream_t s)
{
    if (n_jobs <= 0) return CD_OK;
    LaunchScope ls(CD_K_SHELL, s);
    const dim3 grid((unsigned)((max_elems + 255) / 256), (unsigned)n_jobs);
    shell_list_fp32_batch<<<grid, 256, 0, s>>>(static_cast<const ShellListArgs *>(jobs));
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status column_density_amr(cd_tree t, cd_geom g, const cd_opts &opts, float *n_h, float *a_v, float *shield,
                             cudaStream_t s)
{
    const int nd = g->n_dir, L = t->L;
    // workspace: S_k over the refined cells of levels 3 .. L-2, E over all octs
    if (t->ws.ndir != nd) {
        const cd_status pin = check_workspace_pinned(t, nd);
        if (pin != CD_OK) return pin;
        for (int k = 0; k <= CD_MAXL; ++k) {
            if (t->ws.S[k]) cd::lib_free(t->ws.S[k]);
            t->ws.S[k] = nullptr;
        }
        if (t->ws.E) cd::lib_free(t->ws.E);
        t->ws.E = nullptr;
        t->ws.ndir = 0;
        for (int k = 3; k <= L - 2; ++k)
            if (t->n_ref[k] && cudaMalloc(&t->ws.S[k], sizeof(float) * t->n_ref[k] * nd) != cudaSuccess) {
                cudaGetLastError();
                set_error("AMR workspace allocation failed");
                return CD_ENOMEM;
            }
        if (cudaMalloc(&t->ws.E, sizeof(float) * std::max<int64_t>(t->n_oct, 1) * nd) != cudaSuccess) {
            cudaGetLastError();
            set_error("AMR workspace allocation failed");
            return CD_ENOMEM;
        }
        t->ws.ndir = nd;
    }
    const auto dx = [&](int l) { return (float)(t->box_cm / (double)((int64_t)1 << l)); };
    // in-situ variant: every oct's shells from its centre (insitu.cu), no prefixes
    const bool insitu = g->mode == CD_MODE_INSITU;
    // BF16: the tensor-core contraction over the level's receiver lists where it serves
    const bool tc = !insitu && opts.precision == CD_BF16 && tc_supported(nd) && g->wb != nullptr;
    ShellListArgs A;
    for (int q = 0; q < 4; ++q) {
        A.tab[q] = g->tab[q];
        A.cmax[q] = g->cmax[q];
    }
    A.maxe = g->maxe;
    A.nd = nd;
    // The far-shell prefix chain (S_k needs S_{k-1}) runs on s; the oct shells
    // of every level, which need only the densities, on side stream 0; the
    // leaves of level k+1 on side stream 1 once E of level k and S_{k-1} are
    // done.  Small launches of one branch fill the SMs another leaves idle.
    SideFork fork(t, s);
    if (fork.status() != CD_OK) return fork.status();
    cudaStream_t s_oct = fork.side(0), s_leaf = fork.side(1);
    bool have_S[CD_MAXL + 1] = {}, have_E[CD_MAXL + 1] = {};
    // far-shell prefixes of the refined cells
    for (int k = 3; k <= L - 2 && !insitu; ++k) {
        if (!t->n_ref[k]) continue;
        if (tc && k >= 4 && t->tc_ref[k].ntiles) {
            ExtLaunch e = {};
            e.k = k;
            e.nd = nd;
            e.tmask = 4;
            e.dx[3] = dx(k - 2);
            e.prefix_in = (k - 1 >= 3) ? t->ws.S[k - 1] : nullptr;
            e.out = t->ws.S[k];
            // a fully refined level (below the base level) keeps every cell in Morton
            // order, so it takes the whole-level tiles of a uniform tree
            e.list = t->n_ref[k] == ((int64_t)1 << (3 * k)) ? nullptr : &t->tc_ref[k];
            cd_status st = launch_ext_tc(e, t->rho_brick, g, s);
            if (st != CD_OK) return st;
            CD_CUDA(cudaEventRecord(t->ev_S[k], s));
            have_S[k] = true;
            continue;
        }
        A.k = k;
        A.tmask = 4;
        for (int q = 0; q < 4; ++q) {
            A.lvl[q] = nullptr;
            A.dx[q] = 0.f;
        }
        A.lvl[3] = t->rho_lvl[k - 2];
        A.dx[3] = dx(k - 2);
        A.keys = t->ref_key[k];
        A.n = t->n_ref[k];
        A.parent = t->ref_parent[k];
        A.prefix = (k - 1 >= 3) ? t->ws.S[k - 1] : nullptr;
        A.out = t->ws.S[k];
        {
            LaunchScope ls(CD_K_SHELL, s);
            shell_list_fp32<<<grid_for(A.n * nd, 256), 256, 0, s>>>(A);
            CD_CHECK_LAUNCH();
        }
        CD_CUDA(cudaEventRecord(t->ev_S[k], s));
        have_S[k] = true;
    }
    // the three nearest shells of every oct, level by level
    for (int k = 0; k <= L - 1; ++k) {
        const int64_t no = t->oct_begin[k + 1] - t->oct_begin[k];
        if (!no) continue;
        if (insitu) {
            cd_status st =
                launch_insitu(t, g, k, no, t->oct_key + t->oct_begin[k], t->ws.E + t->oct_begin[k] * nd, s_oct);
            if (st != CD_OK) return st;
            CD_CUDA(cudaEventRecord(t->ev_E[k], s_oct));
            have_E[k] = true;
            continue;
        }
        if (tc && k >= 4 && t->tc_oct[k].ntiles) {
            ExtLaunch e = {};
            e.k = k;
            e.nd = nd;
            e.tmask = 7;
            for (int q = 1; q <= 3; ++q) e.dx[q] = dx(k - q + 1);
            e.out = t->ws.E + t->oct_begin[k] * nd;
            e.list = &t->tc_oct[k];
            cd_status st = launch_ext_tc(e, t->rho_brick, g, s_oct);
            if (st != CD_OK) return st;
            CD_CUDA(cudaEventRecord(t->ev_E[k], s_oct));
            have_E[k] = true;
            continue;
        }
        A.k = k;
        A.tmask = 0;
        for (int q = 0; q < 4; ++q) {
            A.lvl[q] = nullptr;
            A.dx[q] = 0.f;
        }
        for (int q = 1; q <= 3 && q <= k; ++q) {
            A.tmask |= 1 << (q - 1);
            A.lvl[q] = t->rho_lvl[k - q + 1];
            A.dx[q] = dx(k - q + 1);
        }
        A.keys = t->oct_key + t->oct_begin[k];
        A.n = no;
        A.parent = nullptr;
        A.prefix = nullptr;
        A.out = t->ws.E + t->oct_begin[k] * nd;
        {
            LaunchScope ls(CD_K_SHELL, s_oct);
            shell_list_fp32<<<grid_for(no * nd, 256), 256, 0, s_oct>>>(A);
            CD_CHECK_LAUNCH();
        }
        CD_CUDA(cudaEventRecord(t->ev_E[k], s_oct));
        have_E[k] = true;
    }
    // leaves: the 16-lanes-per-oct kernel when 16-byte rows are possible
    const bool vec = nd % 4 == 0 && (uintptr_t)n_h % 16 == 0 && (uintptr_t)a_v % 16 == 0;
    const size_t smem = sizeof(float) * (vec ? 64 * nd + 8 * 2 * nd : 64 * nd + 64 * nd);
    if (smem > 48 * 1024)
        CD_CUDA(cudaFuncSetAttribute(vec ? leaf_list : leaf_list_scalar, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    for (int k = 0; k <= L - 1; ++k) {
        const int64_t no = t->oct_begin[k + 1] - t->oct_begin[k];
        if (!no) continue;
        LeafListArgs B;
        B.n = no;
        B.nd = nd;
        B.dx_leaf = dx(k + 1);
        B.av_per_nh = (float)opts.av_per_nh;
        B.c_exp2 = (float)(-opts.shield_k * opts.av_per_nh * 1.4426950408889634);
        B.inv_nd = 1.0f / (float)nd;
        B.rho8 = t->oct_rho8 + 8 * t->oct_begin[k];
        B.oleaf = t->oct_leaf + 8 * t->oct_begin[k];
        B.E = t->ws.E + t->oct_begin[k] * nd;
        B.Sp = (!insitu && k - 1 >= 3) ? t->ws.S[k - 1] : nullptr;
        B.oparent = t->oct_parent + t->oct_begin[k];
        B.kloc = g->kloc;
        B.n_h = n_h;
        B.a_v = a_v;
        B.shield = shield;
        if (have_E[k]) CD_CUDA(cudaStreamWaitEvent(s_leaf, t->ev_E[k], 0));
        if (B.Sp && have_S[k - 1]) CD_CUDA(cudaStreamWaitEvent(s_leaf, t->ev_S[k - 1], 0));
        if (tc) {
            // BF16: the tensor-core leaf kernel takes the level's octs in tiles of
            // 16 (csrc/leaf_tc.cu) and adds each oct's parent prefix row itself
            float *Ek = t->ws.E + t->oct_begin[k] * nd;
            LeafLaunch b = {};
            b.n_oct = no;
            b.nd = nd;
            b.dx_leaf = B.dx_leaf;
            b.av_per_nh = B.av_per_nh;
            b.shield_k = (float)opts.shield_k;
            b.rho_leaf = B.rho8;
            b.E = Ek;
            b.Sp = B.Sp;
            b.oparent = B.Sp ? B.oparent : nullptr;
            b.n_sp = B.Sp ? t->n_ref[k - 1] : 0;
            b.kloc = g->kloc;
            b.n_h = n_h;
            b.a_v = a_v;
            b.shield = shield;
            b.oleaf = B.oleaf;
            b.n_rows = t->n_leaf;
            cd_status st = launch_leaf_tc(b, s_leaf);
            if (st == CD_OK) continue;
            if (st != CD_EUNSUPPORTED) return st;
        }
        LaunchScope ls(CD_K_LEAF, s_leaf);
        if (vec) leaf_list<<<grid_for(no, 8, 152 * 16), 256, smem, s_leaf>>>(B);
        else leaf_list_scalar<<<grid_for(no, 8, 152 * 16), 256, smem, s_leaf>>>(B);
        CD_CHECK_LAUNCH();
    }
    return fork.join();
}

}  // namespace cd
