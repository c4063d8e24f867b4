// The learned correction (include/colden_learned.h): the tree method's terms
// level by level, the exact ray-marcher that gives the training targets, the
// combine N = N_tree exp(delta), the network handle and the FP32 learned form
// of cd_column_density.
//
// Per-level terms.  The plain evaluation folds the far shells into prefix
// sums; here every shell stays apart.  For a uniform tree with leaves at level
// L (octs at L-1) the shell Delta_l = L - l of leaf m comes from
//   Delta_l = 1, 2, 3:  Et[Delta_l][m >> 3]    (oct level, table Delta_l alone)
//   Delta_l >= 4:       C[k][m >> 3 (L - k)]   with k = L - Delta_l + 2
// (C[k] = shell of level k - 2 seen from the centre of the level-k ancestor,
// table 3, §3.3), and Delta_l = 0 is the internal + local term of §3.2.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "learned.cuh"

namespace cd {
namespace {

constexpr int kThreads = 256;
constexpr int64_t kChunkRows = 1 << 20;   // leaves per chunk of the FP32 learned path

float dx_of(const cd_tree t, int l) { return (float)(t->box_cm / (double)((int64_t)1 << l)); }

int grid_for(int64_t n, int threads)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

struct FeatArgs {
    int64_t n, first, n_leaf;
    const int64_t *leaves;
    int L, nd;
    float dx_leaf;
    const float *rho_leaf;          // Morton
    const float *kloc;              // [8][8][nd], units of dx
    const float *Et[4];             // [n_oct][nd] or NULL
    const float *C[CD_MAXL + 1];    // [8^k][nd] or NULL
    float *x;                       // [n][8 nd + 1]
    float *n_tree;                  // [n][nd] or NULL
};

// One thread per (row, direction).
__global__ void __launch_bounds__(kThreads) learned_features(FeatArgs A)
{
    const int nd = A.nd, n_in = kSlots * nd + 1;
    const int64_t total = A.n * nd;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / nd;
        const int d = (int)(e - r * nd);
        const int64_t m = A.leaves ? A.leaves[r] : A.first + r;
        float *xr = A.x + r * n_in;
        if (m < 0 || m >= A.n_leaf) {
            for (int sl = 0; sl < kSlots; ++sl) xr[sl * nd + d] = 0.f;
            if (d == 0) xr[kSlots * nd] = 0.f;
            if (A.n_tree) A.n_tree[r * nd + d] = 0.f;
            continue;
        }
        const int t = (int)(m & 7);
        const int64_t oct = m >> 3;
        float c[kSlots];
        // Delta_l = 0: internal + local (§3.2)
        float loc = 0.f;
        for (int sib = 0; sib < 8; ++sib)
            loc = fmaf(A.rho_leaf[oct * 8 + sib], A.kloc[(t * 8 + sib) * nd + d], loc);
        c[0] = A.dx_leaf * loc;
        for (int sl = 1; sl < kSlots; ++sl) c[sl] = 0.f;
#pragma unroll
        for (int dl = 1; dl < CD_MAXL; ++dl) {      // dl constant after unrolling
            if (dl > A.L - 1) break;
            const float v = dl <= 3 ? A.Et[dl][oct * nd + d] : A.C[A.L - dl + 2][(m >> (3 * (dl - 2))) * nd + d];
            c[dl < kSlots ? dl : kSlots - 1] += v;
        }
        float tot = 0.f;
        for (int sl = 0; sl < kSlots; ++sl) {
            tot += c[sl];
            xr[sl * nd + d] = logf(fmaxf(c[sl], kCFloor));
        }
        if (d == 0) xr[kSlots * nd] = logf(fmaxf(A.rho_leaf[m], kNFloor));
        if (A.n_tree) A.n_tree[r * nd + d] = tot;
    }
}

struct MarchArgs {
    int64_t n, n_leaf;
    const int64_t *leaves;
    int L, nd;
    float dx_leaf;
    const float *rho_leaf;    // Morton
    const double *dirs;       // [nd][3]
    float *out;               // [n][nd]
};

constexpr uint64_t kDil = 0x1249249249249249ull;   // bits of the x coordinate in a Morton code

// Exact column from the leaf centre to the box edge: Amanatides-Woo DDA over
// the leaf grid in cell units.  Each boundary crossing is computed afresh as
// (boundary - x0) / d, so no error accumulates along the ray; the Morton index
// of the current cell is stepped by dilated-integer addition.
__global__ void __launch_bounds__(kThreads) raymarch(MarchArgs A)
{
    const int nd = A.nd;
    const int64_t total = A.n * nd;
    const int nside = 1 << A.L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / nd;
        const int d = (int)(e - r * nd);
        const int64_t m0 = A.leaves ? A.leaves[r] : r;
        if (m0 < 0 || m0 >= A.n_leaf) {
            A.out[e] = 0.f;
            continue;
        }
        int c[3] = {(int)compact3((uint64_t)m0), (int)compact3((uint64_t)m0 >> 1), (int)compact3((uint64_t)m0 >> 2)};
        float dir[3], inv[3], tnext[3], bnd[3], x0[3];
        int step[3];
        for (int a = 0; a < 3; ++a) {
            dir[a] = (float)A.dirs[3 * d + a];
            x0[a] = (float)c[a] + 0.5f;
            step[a] = dir[a] > 0.f ? 1 : (dir[a] < 0.f ? -1 : 0);
            inv[a] = step[a] ? 1.f / dir[a] : 0.f;
            bnd[a] = (float)(c[a] + (step[a] > 0 ? 1 : 0));
            tnext[a] = step[a] ? (bnd[a] - x0[a]) * inv[a] : INFINITY;
        }
        uint64_t m = (uint64_t)m0;
        float t = 0.f, sum = 0.f;
        for (int it = 0; it < 3 * nside; ++it) {
            int a = 0;
            if (tnext[1] < tnext[a]) a = 1;
            if (tnext[2] < tnext[a]) a = 2;
            const float tn = tnext[a];
            sum = fmaf(A.rho_leaf[m], tn - t, sum);
            t = tn;
            c[a] += step[a];
            if (c[a] < 0 || c[a] >= nside) break;
            const uint64_t mask = kDil << a;
            const uint64_t part = step[a] > 0 ? (((m & mask) | ~mask) + 1) & mask : ((m & mask) - 1) & mask;
            m = (m & ~mask) | part;
            bnd[a] += (float)step[a];
            tnext[a] = (bnd[a] - x0[a]) * inv[a];
        }
        A.out[e] = sum * A.dx_leaf;
    }
}

__global__ void targets(int64_t n, const float *__restrict__ n_ray, const float *__restrict__ n_tree,
                        float *__restrict__ y)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] = logf(n_ray[i] / n_tree[i]);
}

// per-block minimum and maximum of the finite entries of y (+inf / -inf
// where a block saw none)
__global__ void __launch_bounds__(256) finite_range(int64_t n, const float *__restrict__ y, float *__restrict__ part)
{
    __shared__ float smin[256], smax[256];
    float lo = INFINITY, hi = -INFINITY;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float v = y[i];
        if (isfinite(v)) {
            lo = fminf(lo, v);
            hi = fmaxf(hi, v);
        }
    }
    smin[threadIdx.x] = lo;
    smax[threadIdx.x] = hi;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            smin[threadIdx.x] = fminf(smin[threadIdx.x], smin[threadIdx.x + w]);
            smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = smin[0];
        part[2 * blockIdx.x + 1] = smax[0];
    }
}

// N = N_tree exp(delta) (N_tree where delta is not finite or outside
// [dlo, dhi]), A_V and the shield; one warp per leaf, the shield summed by a
// fixed butterfly.
__global__ void __launch_bounds__(kThreads) learned_combine(int64_t n, int nd, const float *__restrict__ n_tree,
                                                            const float *__restrict__ delta, float dlo, float dhi,
                                                            float av_per_nh,
                                                            float shield_k, float *__restrict__ n_h,
                                                            float *__restrict__ a_v, float *__restrict__ shield)
{
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = blockIdx.x * (int64_t)(blockDim.x / 32) + (threadIdx.x >> 5); r < n; r += warps) {
        float acc = 0.f;
        for (int d = lane; d < nd; d += 32) {
            const int64_t o = r * nd + d;
            const float dl = delta[o], nt = n_tree[o];
            const float N = isfinite(dl) && dl >= dlo && dl <= dhi ? nt * expf(dl) : nt;
            const float av = N * av_per_nh;
            if (n_h) n_h[o] = N;
            if (a_v) a_v[o] = av;
            acc += expf(-shield_k * av);
        }
        for (int w = 16; w > 0; w >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
        if (shield && lane == 0) shield[r] = acc / (float)nd;
    }
}

cd_status check_tree_geom(cd_tree t, cd_geom g)
{
    if (!t || !g) {
        set_error("tree or geometry is NULL");
        return CD_EINVAL;
    }
    if (t->amr) {
        set_error("the learned form and the ray-marcher serve uniform trees only");
        return CD_EUNSUPPORTED;
    }
    return CD_OK;
}

template <typename T>
cd_status alloc(T **p, size_t count)
{
    if (cudaMalloc(p, count * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("device allocation of %zu bytes failed", count * sizeof(T));
        return CD_ENOMEM;
    }
    return CD_OK;
}

cd_status launch_features(cd_tree t, cd_geom g, int64_t n, int64_t first, const int64_t *leaves, float *x,
                          float *n_tree, cudaStream_t s)
{
    FeatArgs A = {};
    A.n = n;
    A.first = first;
    A.n_leaf = t->n_leaf;
    A.leaves = leaves;
    A.L = t->L;
    A.nd = g->n_dir;
    A.dx_leaf = dx_of(t, t->L);
    A.rho_leaf = t->rho_leaf;
    A.kloc = g->kloc;
    for (int i = 0; i < 4; ++i) A.Et[i] = t->lv.Et[i];
    for (int k = 0; k <= CD_MAXL; ++k) A.C[k] = t->lv.C[k];
    A.x = x;
    A.n_tree = n_tree;
    if (n == 0) return CD_OK;
    LaunchScope ls(CD_K_FEATURES, s);
    learned_features<<<grid_for(n * g->n_dir, kThreads), kThreads, 0, s>>>(A);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status check_net(cd_net net)
{
    if (!net) {
        set_error("network is NULL");
        return CD_EINVAL;
    }
    return CD_OK;
}

}  // namespace

// Computes (or reuses) every shell's sum kept apart: C[k] for k = 3 .. L-2 and
// Et[t] at the oct level.
cd_status ensure_level_sums(cd_tree t, cd_geom g, int precision, cudaStream_t s)
{
    LevelSums &lv = t->lv;
    const int nd = g->n_dir, L = t->L;
    if (lv.ndir == nd && lv.geom_uid == g->uid && lv.rho_version == t->rho_version && lv.precision == precision)
        return CD_OK;
    // BF16: the tensor-core contraction (one table per launch) where it serves
    const bool tc = precision == CD_BF16 && tc_supported(nd) && g->wb != nullptr;
    if (lv.ndir != nd) {
        free_level_sums(t);
        for (int k = 3; k <= L - 2; ++k)
            if (alloc(&lv.C[k], ((size_t)1 << (3 * k)) * nd) != CD_OK) return CD_ENOMEM;
        for (int tt = 1; tt <= 3 && tt <= L - 1; ++tt)
            if (alloc(&lv.Et[tt], (size_t)t->n_oct * nd) != CD_OK) return CD_ENOMEM;
        lv.ndir = nd;
    }
    lv.rho_version = -1;
    for (int k = 3; k <= L - 2; ++k) {
        ExtLaunch a = {};
        a.k = k;
        a.nd = nd;
        a.tmask = 4;
        a.rho[3] = t->rho_lvl[k - 2];
        a.dx[3] = dx_of(t, k - 2);
        a.out = lv.C[k];
        cd_status st = tc && k >= 4 ? launch_ext_tc(a, t->rho_brick, g, s) : launch_ext_fp32(a, g, s);
        if (st != CD_OK) return st;
    }
    const int k = L - 1;
    for (int tt = 1; tt <= 3 && tt <= k; ++tt) {
        ExtLaunch a = {};
        a.k = k;
        a.nd = nd;
        a.tmask = 1 << (tt - 1);
        a.rho[tt] = t->rho_lvl[k - tt + 1];
        a.dx[tt] = dx_of(t, k - tt + 1);
        a.out = lv.Et[tt];
        cd_status st = tc && k >= 4 ? launch_ext_tc(a, t->rho_brick, g, s) : launch_ext_fp32(a, g, s);
        if (st != CD_OK) return st;
    }
    lv.geom_uid = g->uid;
    lv.rho_version = t->rho_version;
    lv.precision = precision;
    return CD_OK;
}

void free_level_sums(cd_tree t)
{
    LevelSums &lv = t->lv;
    for (int k = 0; k <= CD_MAXL; ++k) {
        if (lv.C[k]) cd::lib_free(lv.C[k]);
        lv.C[k] = nullptr;
    }
    for (int i = 0; i < 4; ++i) {
        if (lv.Et[i]) cd::lib_free(lv.Et[i]);
        lv.Et[i] = nullptr;
    }
    for (float **p : {&lv.x, &lv.n_tree, &lv.delta}) {
        if (*p) cd::lib_free(*p);
        *p = nullptr;
    }
    lv.rows = 0;
    lv.ndir = 0;
    lv.geom_uid = 0;
    lv.rho_version = -1;
    lv.precision = -1;
}

cd_status column_density_learned(cd_tree t, cd_geom g, const cd_opts &o, float *n_h, float *a_v, float *shield,
                                 cudaStream_t s)
{
    cd_status st = check_tree_geom(t, g);
    if (st != CD_OK) return st;
    if (o.precision != CD_FP32 && o.precision != CD_BF16) {
        set_error("unknown precision %d", o.precision);
        return CD_EINVAL;
    }
    cd_net net = (cd_net)o.net;
    const int nd = g->n_dir;
    if (o.precision == CD_BF16) return column_density_learned_tc(t, g, o, n_h, a_v, shield, s);
    if (net->lay.nd != nd) {
        set_error("the network has %d directions, the geometry %d", net->lay.nd, nd);
        return CD_EINVAL;
    }
    if ((st = ensure_level_sums(t, g, CD_FP32, s)) != CD_OK) return st;
    LevelSums &lv = t->lv;
    const int64_t chunk = std::min<int64_t>(kChunkRows, t->n_leaf);
    if (lv.rows < chunk) {
        for (float **p : {&lv.x, &lv.n_tree, &lv.delta}) {
            if (*p) cd::lib_free(*p);
            *p = nullptr;
        }
        lv.rows = 0;
        if (alloc(&lv.x, (size_t)chunk * net->lay.n_in) != CD_OK || alloc(&lv.n_tree, (size_t)chunk * nd) != CD_OK ||
            alloc(&lv.delta, (size_t)chunk * nd) != CD_OK)
            return CD_ENOMEM;
        lv.rows = chunk;
    }
    for (int64_t c0 = 0; c0 < t->n_leaf; c0 += chunk) {
        const int64_t cn = std::min(chunk, t->n_leaf - c0);
        if ((st = launch_features(t, g, cn, c0, nullptr, lv.x, lv.n_tree, s)) != CD_OK) return st;
        if ((st = mlp_forward(net, cn, lv.x, nullptr, lv.delta, s)) != CD_OK) return st;
        LaunchScope ls(CD_K_FEATURES, s);
        learned_combine<<<grid_for(cn * 32, kThreads), kThreads, 0, s>>>(
            cn, nd, lv.n_tree, lv.delta, net->dlo, net->dhi, (float)o.av_per_nh, (float)o.shield_k, n_h ? n_h + c0 * nd : nullptr,
            a_v ? a_v + c0 * nd : nullptr, shield ? shield + c0 : nullptr);
        CD_CHECK_LAUNCH();
    }
    return CD_OK;
}

}  // namespace cd

using namespace cd;

extern "C" {

void cd_adam_default(cd_adam *a)
{
    if (!a) return;
    a->lr = 1e-3;
    a->beta1 = 0.9;
    a->beta2 = 0.999;
    a->eps = 1e-8;
}

int64_t cd_net_num_params(int n_dir, int hidden)
{
    if (n_dir < 1 || n_dir > CD_MAXDIR || hidden < 1 || hidden > 1024) return -1;
    return NetLayout(n_dir, hidden).total;
}

cd_status cd_raymarch(cd_tree tree, cd_geom geom, int64_t n, const int64_t *leaves, float *n_ray, void *stream)
{
    NvtxRange nvtx_range("colden:raymarch");
    cd_status st = check_tree_geom(tree, geom);
    if (st != CD_OK) return st;
    if (n < 0 || !n_ray || (!leaves && n > tree->n_leaf)) {
        set_error("bad ray-march arguments (n = %lld)", (long long)n);
        return CD_EINVAL;
    }
    if (n == 0) return CD_OK;
    MarchArgs A = {};
    A.n = n;
    A.n_leaf = tree->n_leaf;
    A.leaves = leaves;
    A.L = tree->L;
    A.nd = geom->n_dir;
    A.dx_leaf = dx_of(tree, tree->L);
    A.rho_leaf = tree->rho_leaf;
    A.dirs = geom->dirs_dev;
    A.out = n_ray;
    cudaStream_t s = (cudaStream_t)stream;
    LaunchScope ls(CD_K_RAYMARCH, s);
    raymarch<<<grid_for(n * geom->n_dir, kThreads), kThreads, 0, s>>>(A);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status cd_learned_features(cd_tree tree, cd_geom geom, int64_t n, const int64_t *leaves, float *x, float *n_tree,
                              void *stream)
{
    NvtxRange nvtx_range("colden:learned_features");
    cd_status st = check_tree_geom(tree, geom);
    if (st != CD_OK) return st;
    if (geom->mode != CD_MODE_PREC) {
        set_error("the learned inputs are defined on the single-ray precalculated form");
        return CD_EUNSUPPORTED;
    }
    if (n < 0 || !x || (!leaves && n > tree->n_leaf)) {
        set_error("bad feature arguments (n = %lld)", (long long)n);
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_level_sums(tree, geom, CD_FP32, s)) != CD_OK) return st;
    return launch_features(tree, geom, n, 0, leaves, x, n_tree, s);
}

cd_status cd_learned_targets(int64_t n, const float *n_ray, const float *n_tree, float *y, void *stream)
{
    NvtxRange nvtx_range("colden:learned_targets");
    if (n < 0 || (n > 0 && (!n_ray || !n_tree || !y))) {
        set_error("bad target arguments");
        return CD_EINVAL;
    }
    if (n == 0) return CD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    LaunchScope ls(CD_K_FEATURES, s);
    targets<<<grid_for(n, kThreads), kThreads, 0, s>>>(n, n_ray, n_tree, y);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

cd_status cd_net_create(int n_dir, int hidden, const float *params, cd_net *out)
{
    if (!out) {
        set_error("out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (cd_net_num_params(n_dir, hidden) < 0 || !params) {
        set_error("bad network sizes (n_dir %d, hidden %d) or NULL params", n_dir, hidden);
        return CD_EINVAL;
    }
    cd_net net = new cd_net_s();
    net->lay = NetLayout(n_dir, hidden);
    cudaGetDevice(&net->dev);
    const size_t P = (size_t)net->lay.total, I = (size_t)net->lay.n_in;
    bool ok = alloc(&net->p, P) == CD_OK && alloc(&net->m, P) == CD_OK && alloc(&net->v, P) == CD_OK &&
              alloc(&net->grad, P) == CD_OK && alloc(&net->mu, I) == CD_OK && alloc(&net->sinv, I) == CD_OK;
    if (!ok) {
        cd_net_free(net);
        return CD_ENOMEM;
    }
    std::vector<float> ones(I, 1.f);
    ok = cudaMemcpy(net->p, params, P * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemset(net->m, 0, P * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->v, 0, P * sizeof(float)) == cudaSuccess &&
         cudaMemset(net->mu, 0, I * sizeof(float)) == cudaSuccess &&
         cudaMemcpy(net->sinv, ones.data(), I * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
         // pageable uploads and memsets may return before they land, ordered only
         // on the legacy default stream: finish them before any stream reads the net
         cudaDeviceSynchronize() == cudaSuccess;
    if (!ok) {
        set_error("network upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        cd_net_free(net);
        return CD_ECUDA;
    }
    *out = net;
    return CD_OK;
}

cd_status cd_net_fit_normaliser(cd_net net, int64_t n, const float *x, void *stream)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (n < 1 || !x) {
        set_error("the normaliser needs at least one row");
        return CD_EINVAL;
    }
    return mlp_fit_normaliser(net, n, x, (cudaStream_t)stream);
}

cd_status cd_net_forward(cd_net net, int64_t n, const float *x, float *delta, void *stream)
{
    NvtxRange nvtx_range("colden:net_forward");
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (n < 0 || (n > 0 && (!x || !delta))) {
        set_error("bad forward arguments");
        return CD_EINVAL;
    }
    const NetLayout &L = net->lay;
    cudaStream_t s = (cudaStream_t)stream;
    for (int64_t c0 = 0; c0 < n; c0 += kChunkRows) {
        const int64_t cn = std::min<int64_t>(kChunkRows, n - c0);
        if ((st = mlp_forward(net, cn, x + c0 * L.n_in, nullptr, delta + c0 * L.nd, s)) != CD_OK) return st;
    }
    return CD_OK;
}

cd_status cd_net_loss_grad(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows, float *loss,
                           float *grad, void *stream)
{
    NvtxRange nvtx_range("colden:net_loss_grad");
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (B < 1 || B > kChunkRows * 4 || !x || !y) {
        set_error("batch size %lld outside 1 .. %lld or NULL data", (long long)B, (long long)kChunkRows * 4);
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = mlp_loss_grad(net, B, x, y, rows, loss, s)) != CD_OK) return st;
    if (grad) CD_CUDA(cudaMemcpyAsync(grad, net->grad, sizeof(float) * net->lay.total, cudaMemcpyDeviceToDevice, s));
    return CD_OK;
}

cd_status cd_net_train_step(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows,
                            const cd_adam *hp, float *loss, void *stream)
{
    NvtxRange nvtx_range("colden:net_train_step");
    cd_status st = cd_net_loss_grad(net, B, x, y, rows, loss, nullptr, stream);
    if (st != CD_OK) return st;
    cd_adam h;
    if (hp) h = *hp; else cd_adam_default(&h);
    return mlp_adam(net, h, (cudaStream_t)stream);
}

cd_status cd_net_get_state(cd_net net, float *params, float *mu, float *sinv, float *adam_m, float *adam_v,
                           int64_t *step)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    CD_CUDA(cudaDeviceSynchronize());
    const size_t P = sizeof(float) * net->lay.total, I = sizeof(float) * net->lay.n_in;
    if (params) CD_CUDA(cudaMemcpy(params, net->p, P, cudaMemcpyDeviceToHost));
    if (adam_m) CD_CUDA(cudaMemcpy(adam_m, net->m, P, cudaMemcpyDeviceToHost));
    if (adam_v) CD_CUDA(cudaMemcpy(adam_v, net->v, P, cudaMemcpyDeviceToHost));
    if (mu) CD_CUDA(cudaMemcpy(mu, net->mu, I, cudaMemcpyDeviceToHost));
    if (sinv) CD_CUDA(cudaMemcpy(sinv, net->sinv, I, cudaMemcpyDeviceToHost));
    if (step) *step = net->step;
    return CD_OK;
}

cd_status cd_net_set_state(cd_net net, const float *params, const float *mu, const float *sinv, const float *adam_m,
                           const float *adam_v, int64_t step)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (step < 0) {
        set_error("negative step count");
        return CD_EINVAL;
    }
    CD_CUDA(cudaDeviceSynchronize());
    const size_t P = sizeof(float) * net->lay.total, I = sizeof(float) * net->lay.n_in;
    if (params) CD_CUDA(cudaMemcpy(net->p, params, P, cudaMemcpyHostToDevice));
    if (adam_m) CD_CUDA(cudaMemcpy(net->m, adam_m, P, cudaMemcpyHostToDevice));
    if (adam_v) CD_CUDA(cudaMemcpy(net->v, adam_v, P, cudaMemcpyHostToDevice));
    if (mu) CD_CUDA(cudaMemcpy(net->mu, mu, I, cudaMemcpyHostToDevice));
    if (sinv) CD_CUDA(cudaMemcpy(net->sinv, sinv, I, cudaMemcpyHostToDevice));
    CD_CUDA(cudaDeviceSynchronize());   // the pageable uploads have landed
    net->step = step;
    net->version += 1;
    return CD_OK;
}

cd_status cd_net_set_delta_range(cd_net net, double lo, double hi)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (std::isnan(lo) || std::isnan(hi)) {
        set_error("the delta range has a NaN end");
        return CD_EINVAL;
    }
    net->dlo = (float)lo;
    net->dhi = (float)hi;
    return CD_OK;
}

cd_status cd_net_get_delta_range(cd_net net, double *lo, double *hi)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (lo) *lo = net->dlo;
    if (hi) *hi = net->dhi;
    return CD_OK;
}

cd_status cd_net_fit_delta_range(cd_net net, int64_t n, const float *y, double margin, void *stream)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (n < 1 || !y || !(margin >= 0.0) || std::isinf(margin)) {
        set_error("the delta range needs n >= 1 targets and a finite margin >= 0");
        return CD_EINVAL;
    }
    constexpr int kBlocks = 256;
    float *part = nullptr;
    if (alloc(&part, 2 * kBlocks) != CD_OK) return CD_ENOMEM;
    cudaStream_t s = (cudaStream_t)stream;
    float h[2 * kBlocks];
    finite_range<<<kBlocks, 256, 0, s>>>(n, y, part);
    const bool ok = cudaGetLastError() == cudaSuccess &&
                    cudaMemcpyAsync(h, part, sizeof(h), cudaMemcpyDeviceToHost, s) == cudaSuccess &&
                    cudaStreamSynchronize(s) == cudaSuccess;
    cd::lib_free(part);
    if (!ok) {
        set_error("delta range reduction failed: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    float lo = INFINITY, hi = -INFINITY;
    for (int b = 0; b < kBlocks; ++b) {
        lo = std::min(lo, h[2 * b]);
        hi = std::max(hi, h[2 * b + 1]);
    }
    if (lo > hi) {   // no finite target: an empty range, the plain method everywhere
        net->dlo = INFINITY;
        net->dhi = -INFINITY;
    } else {
        net->dlo = (float)((double)lo - margin);
        net->dhi = (float)((double)hi + margin);
    }
    return CD_OK;
}

cd_status cd_net_info(cd_net net, int *n_dir, int *hidden, int64_t *num_params)
{
    cd_status st = check_net(net);
    if (st != CD_OK) return st;
    if (n_dir) *n_dir = net->lay.nd;
    if (hidden) *hidden = net->lay.H;
    if (num_params) *num_params = net->lay.total;
    return CD_OK;
}

void cd_net_free(cd_net net)
{
    if (!net) return;
    cudaDeviceSynchronize();
    for (float *p : {net->p, net->m, net->v, net->grad, net->mu, net->sinv, net->act.U, net->act.Z1, net->act.A1,
                     net->act.Z2, net->act.A2, net->act.D, net->act.G, net->act.part, net->act.red})
        if (p) cd::lib_free(p);
    net_free_tc(net);
    delete net;
}

}  // extern "C"
