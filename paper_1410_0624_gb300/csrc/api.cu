// C ABI of libcolden: argument checking, handle lifetime, workspace and the
// order in which the kernels of one column-density evaluation run.
//
// Evaluation order for a tree whose leaves sit at level L (prec mode, §3.3):
//   1. k = 3 .. L-2: S_k[c] = S_{k-1}[parent c] + far shell of level k-2 seen
//      from the centre of c (table 3).  S_k holds, for every level-k cell, the
//      summed shells l <= k-2 it shares with all its descendants' octs.
//   2. k = L-1 (the octs): E[c] = shells L-3 (table 3), L-2 (table 2) and
//      L-1 (table 1), all seen from the oct centre.
//   3. leaves: N_H = E[oct] + S_{L-2}[parent oct] + internal + local, then A_V
//      and the shield.
// Every shell l = 1 .. L-1 enters exactly once (Eq. N_discret).  Step 2 needs
// only the densities, so it runs on a side stream of the tree while step 1
// runs on the tree's high-priority side stream; step 3 waits for both
// (SideFork).
#include <algorithm>
#include <atomic>
#include <vector>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>
#include <math.h>

#include "learned.cuh"

namespace cd {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

static void free_workspace(cd_tree t)
{
    for (int l = 0; l <= CD_MAXL; ++l) {
        if (t->ws.S[l]) cd::lib_free(t->ws.S[l]);
        t->ws.S[l] = nullptr;
    }
    if (t->ws.E) cd::lib_free(t->ws.E);
    t->ws.E = nullptr;
    t->ws.ndir = 0;
}

cd_status check_workspace_pinned(cd_tree t, int nd)
{
    if (t->ws.ndir == nd || t->batch_refs == 0) return CD_OK;
    set_error("the tree's scratch is sized for %d directions and held by %d live batch object(s); an evaluation "
              "with %d directions would reallocate it under the batch's graph (free the batch first)",
              t->ws.ndir, t->batch_refs, nd);
    return CD_EINVAL;
}

static cd_status ensure_workspace(cd_tree t, int nd)
{
    if (t->ws.ndir == nd) return CD_OK;
    cd_status pin = check_workspace_pinned(t, nd);
    if (pin != CD_OK) return pin;
    free_workspace(t);
    for (int k = 3; k <= t->L - 2; ++k) {
        const size_t bytes = sizeof(float) * ((size_t)1 << (3 * k)) * nd;
        if (cudaMalloc(&t->ws.S[k], bytes) != cudaSuccess) {
            cudaGetLastError();
            free_workspace(t);
            set_error("workspace allocation failed (%zu bytes)", bytes);
            return CD_ENOMEM;
        }
    }
    if (t->L >= 2) {
        const size_t bytes = sizeof(float) * (size_t)t->n_oct * nd;
        if (cudaMalloc(&t->ws.E, bytes) != cudaSuccess) {
            cudaGetLastError();
            free_workspace(t);
            set_error("workspace allocation failed (%zu bytes)", bytes);
            return CD_ENOMEM;
        }
    }
    t->ws.ndir = nd;
    return CD_OK;
}

static float dx_of(const cd_tree t, int l) { return (float)(t->box_cm / (double)((int64_t)1 << l)); }

// tiles per CTA of the oct level's tensor-core shells in a concurrent evaluation
constexpr int kOctTilesPerCta = 8;

static void free_side_streams(cd_tree t)
{
    for (int i = 0; i < 2; ++i) {
        if (t->side[i]) cudaStreamDestroy(t->side[i]);
        if (t->ev_done[i]) cudaEventDestroy(t->ev_done[i]);
        t->side[i] = nullptr;
        t->ev_done[i] = nullptr;
    }
    for (int l = 0; l <= CD_MAXL; ++l) {
        if (t->ev_S[l]) cudaEventDestroy(t->ev_S[l]);
        if (t->ev_E[l]) cudaEventDestroy(t->ev_E[l]);
        t->ev_S[l] = t->ev_E[l] = nullptr;
    }
    if (t->ev_fork) cudaEventDestroy(t->ev_fork);
    t->ev_fork = nullptr;
}

// non-blocking streams (no implicit order with the legacy default stream: the
// fork and the join order them explicitly) and timing-free events
static cd_status ensure_side_streams(cd_tree t)
{
    if (t->ev_fork) return CD_OK;
    // side stream 1 at the highest priority: its pending CTAs are placed first
    // when CTAs of other launches retire
    int least = 0, greatest = 0;
    bool ok = cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess;
    for (int i = 0; i < 2 && ok; ++i)
        ok = cudaStreamCreateWithPriority(&t->side[i], cudaStreamNonBlocking, i == 1 ? greatest : least) ==
                 cudaSuccess &&
             cudaEventCreateWithFlags(&t->ev_done[i], cudaEventDisableTiming) == cudaSuccess;
    for (int l = 0; l <= CD_MAXL && ok; ++l)
        ok = cudaEventCreateWithFlags(&t->ev_S[l], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&t->ev_E[l], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&t->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        free_side_streams(t);
        set_error("cannot create the tree's side streams");
        return CD_ECUDA;
    }
    return CD_OK;
}

SideFork::SideFork(cd_tree t, cudaStream_t s) : t_(t), s_(s)
{
    // the events exist in both modes: the callers record and wait on them
    // unconditionally (on s alone they order nothing new)
    st_ = ensure_side_streams(t);
    serial_ = stats_timing();
    if (st_ != CD_OK || serial_) {
        joined_ = true;   // nothing was forked
        return;
    }
    if (cudaEventRecord(t->ev_fork, s) != cudaSuccess || cudaStreamWaitEvent(t->side[0], t->ev_fork, 0) != cudaSuccess ||
        cudaStreamWaitEvent(t->side[1], t->ev_fork, 0) != cudaSuccess) {
        set_error("cannot order the side streams after the caller's stream: %s", cudaGetErrorString(cudaGetLastError()));
        st_ = CD_ECUDA;
    }
}

cd_status SideFork::join()
{
    if (joined_) return CD_OK;
    joined_ = true;
    for (int i = 0; i < 2; ++i)
        if (cudaEventRecord(t_->ev_done[i], t_->side[i]) != cudaSuccess ||
            cudaStreamWaitEvent(s_, t_->ev_done[i], 0) != cudaSuccess) {
            set_error("cannot join the side streams: %s", cudaGetErrorString(cudaGetLastError()));
            return CD_ECUDA;
        }
    return CD_OK;
}

cudaStream_t SideFork::side(int i) const { return serial_ ? s_ : t_->side[i]; }

SideFork::~SideFork() { join(); }

void free_host_io(cd_tree t)
{
    cd_tree_s::HostIO &h = t->hio;
    for (float *p : {h.rho, h.nh, h.av, h.sh})
        if (p) cd::lib_free(p);
    if (h.copy) cudaStreamDestroy(h.copy);
    for (cudaEvent_t e : h.ev)
        if (e) cudaEventDestroy(e);
    h = cd_tree_s::HostIO();
}

// the staging buffers cd_column_density_host needs (kept by the tree, grown on demand)
cd_status ensure_host_io(cd_tree t, int64_t nh_elems, bool rho, bool nh, bool av, bool sh)
{
    cd_tree_s::HostIO &h = t->hio;
    if (h.nh_elems < nh_elems) {
        for (float **p : {&h.nh, &h.av}) {
            if (*p) cd::lib_free(*p);
            *p = nullptr;
        }
        h.nh_elems = nh_elems;
    }
    bool ok = true;
    if (!h.copy) {
        ok = cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t &e : h.ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    }
    auto take = [&](float *&p, bool want, int64_t n) {
        if (ok && want && !p) ok = cudaMalloc(&p, sizeof(float) * n) == cudaSuccess;
    };
    take(h.rho, rho, t->n_leaf);
    take(h.nh, nh, nh_elems);
    take(h.av, av, nh_elems);
    take(h.sh, sh, t->n_leaf);
    if (!ok) {
        cudaGetLastError();
        set_error("cannot allocate the host-output staging buffers");
        return CD_ENOMEM;
    }
    return CD_OK;
}

#ifdef COLDEN_CHECKED
// every translation unit's check-word reader (registered at load time)
static std::vector<CheckReader> &check_readers()
{
    static std::vector<CheckReader> v;
    return v;
}

int register_check_reader(CheckReader r)
{
    check_readers().push_back(r);
    return 1;
}

// cd_debug_check_probe: reads a[i] of a 4-element array through the check
__global__ void check_probe(const float *a, int64_t i, float *out)
{
    *out = in_bounds(i, 4, kCheckProbe) ? a[i] : -1.f;
}
#endif

}  // namespace cd

using namespace cd;

extern "C" {

void cd_opts_default(cd_opts *o)
{
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = CD_FP32;
    o->av_per_nh = 1.0 / 1.87e21;
    o->shield_k = 2.5;
    o->net = nullptr;
}

const char *cd_last_error(void) { return g_err; }

cd_status cd_build_tree_uniform(int leaf_level, double box_cm, const float *rho, int rho_on_device, void *stream,
                                cd_tree *out)
{
    NvtxRange nvtx_range("colden:build_tree_uniform");
    if (!out) {
        set_error("out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (leaf_level < 1 || leaf_level > 10) {
        set_error("leaf_level %d outside 1..10", leaf_level);
        return CD_EINVAL;
    }
    if (!(box_cm > 0.0) || !isfinite(box_cm)) {
        set_error("box_cm must be finite and > 0");
        return CD_EINVAL;
    }
    if (!rho) {
        set_error("rho is NULL");
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int L = leaf_level;
    const int64_t n = (int64_t)1 << L, N = n * n * n;
    if (!rho_on_device) {
        for (int64_t i = 0; i < N; ++i)
            if (!(rho[i] >= 0.f) || !isfinite(rho[i])) {
                set_error("rho[%lld] = %g is negative or not finite", (long long)i, (double)rho[i]);
                return CD_EINVAL;
            }
    }
    cd_tree t = new cd_tree_s();
    cudaGetDevice(&t->dev);
    t->L = L;
    t->base = L;
    t->box_cm = box_cm;
    t->n_leaf = N;
    t->n_oct = N / 8;
    cd_status st = CD_OK;
    float *staging = nullptr;
    auto fail = [&](cd_status code) {
        if (staging) cd::lib_free(staging);
        cd_tree_free(t);
        return code;
    };
    if (cudaMalloc(&t->rho_leaf, sizeof(float) * N) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate %lld leaves", (long long)N);
        return fail(CD_ENOMEM);
    }
    for (int l = 0; l <= L - 1; ++l) {
        const int64_t m = (int64_t)1 << l;
        if (cudaMalloc(&t->rho_lvl[l], sizeof(float) * m * m * m) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate level %d", l);
            return fail(CD_ENOMEM);
        }
        if (l >= 1 && cudaMalloc(&t->rho_brick[l], sizeof(__nv_bfloat16) * m * m * m) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate level %d bricks", l);
            return fail(CD_ENOMEM);
        }
    }
    const float *src = rho;
    if (!rho_on_device) {
        if (cudaMalloc(&staging, sizeof(float) * N) != cudaSuccess) {
            cudaGetLastError();
            set_error("cannot allocate the upload buffer");
            return fail(CD_ENOMEM);
        }
        if (cudaMemcpyAsync(staging, rho, sizeof(float) * N, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            set_error("upload failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(CD_ECUDA);
        }
        src = staging;
    }
    st = restrict_uniform(t, src, s);
    if (st != CD_OK) return fail(st);
    if (staging) {
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            set_error("tree build failed: %s", cudaGetErrorString(cudaGetLastError()));
            return fail(CD_ECUDA);
        }
        cd::lib_free(staging);
        staging = nullptr;
    }
    *out = t;
    return CD_OK;
}

cd_status cd_build_tree_amr(int base_level, int max_level, double box_cm, int64_t n_leaf, const int8_t *level,
                            const int32_t *ijk, const float *rho, int rho_on_device, void *stream, cd_tree *out)
{
    NvtxRange nvtx_range("colden:build_tree_amr");
    if (!out) {
        set_error("out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (!level || !ijk || !rho) {
        set_error("level, ijk or rho is NULL");
        return CD_EINVAL;
    }
    if (!(box_cm > 0.0) || !isfinite(box_cm)) {
        set_error("box_cm must be finite and > 0");
        return CD_EINVAL;
    }
    cd_tree t = new cd_tree_s();
    cudaGetDevice(&t->dev);
    t->box_cm = box_cm;
    cd_status st = build_amr(t, base_level, max_level, n_leaf, level, ijk);
    // the index arrays went up by cudaMemcpy from pageable memory, which may
    // return before its DMA lands and orders it only on the legacy default
    // stream: finish it before work on any other stream reads them
    if (st == CD_OK && cudaDeviceSynchronize() != cudaSuccess) {
        set_error("AMR tree upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = CD_ECUDA;
    }
    if (st == CD_OK) st = cd_tree_update(t, rho, rho_on_device, stream);
    if (st != CD_OK) {
        cd_tree_free(t);
        return st;
    }
    *out = t;
    return CD_OK;
}

cd_status cd_tree_update(cd_tree t, const float *rho, int rho_on_device, void *stream)
{
    NvtxRange nvtx_range("colden:tree_update");
    if (!t || !rho) {
        set_error("tree or rho is NULL");
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = t->n_leaf;
    ++t->rho_version;
    const auto apply = [&](const float *dev) { return t->amr ? update_amr(t, dev, s) : restrict_uniform(t, dev, s); };
    if (rho_on_device) return apply(rho);
    for (int64_t i = 0; i < N; ++i)
        if (!(rho[i] >= 0.f) || !isfinite(rho[i])) {
            set_error("rho[%lld] = %g is negative or not finite", (long long)i, (double)rho[i]);
            return CD_EINVAL;
        }
    // host data goes through a temporary device buffer
    float *staging = nullptr;
    if (cudaMallocAsync(&staging, sizeof(float) * N, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate the upload buffer");
        return CD_ENOMEM;
    }
    cd_status st = CD_OK;
    if (cudaMemcpyAsync(staging, rho, sizeof(float) * N, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        set_error("upload failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = CD_ECUDA;
    }
    if (st == CD_OK) st = apply(staging);
    cudaFreeAsync(staging, s);
    if (st == CD_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("tree update failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = CD_ECUDA;
    }
    return st;
}

cd_status cd_precompute_geometry(int scheme, int p0, int p1, const double *dirs, int n_custom, int mode,
                                 void *stream, cd_geom *out)
{
    NvtxRange nvtx_range("colden:precompute_geometry");
    if (!out) {
        set_error("out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (mode != CD_MODE_PREC && mode != CD_MODE_INSITU && mode != CD_MODE_CONE) {
        set_error("unknown mode %d", mode);
        return CD_EINVAL;
    }
    static thread_local double buf[3 * CD_MAXDIR];
    const int nd = make_directions(scheme, p0, p1, dirs, n_custom, buf);
    if (nd < 1) {
        set_error("bad direction set (scheme %d, p0 %d, p1 %d, n_custom %d)", scheme, p0, p1, n_custom);
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cd_geom g = new cd_geom_s();
    static std::atomic<int64_t> next_uid{1};
    g->uid = next_uid++;
    cudaGetDevice(&g->dev);
    g->n_dir = nd;
    g->mode = mode;
    g->scheme = scheme;
    g->p0 = p0;
    g->p1 = p1;
    if (scheme == CD_DIRS_CUSTOM) {
        g->n_custom = n_custom;
        g->custom = new double[3 * (size_t)n_custom];
        memcpy(g->custom, dirs, sizeof(double) * 3 * n_custom);
    }
    g->dirs_host = new double[3 * nd];
    memcpy(g->dirs_host, buf, sizeof(double) * 3 * nd);
    static_assert(CD_CONE_RINGS * CD_CONE_AZ == CD_CONE_SUBRAYS, "sub-ray count of colden.h");
    g->n_sub = mode == CD_MODE_CONE ? CD_CONE_SUBRAYS : 1;
    if (g->n_sub > 1) {
        g->rays_host = new double[(size_t)3 * nd * g->n_sub];
        make_cone_rays(g->dirs_host, nd, g->rays_host);
    } else {
        g->rays_host = g->dirs_host;
    }
    auto fail = [&](cd_status code) {
        cd_geom_free(g);
        return code;
    };
    bool ok = cudaMalloc(&g->dirs_dev, sizeof(double) * 3 * nd) == cudaSuccess;
    if (ok && g->n_sub > 1) ok = cudaMalloc(&g->rays_dev, sizeof(double) * 3 * nd * g->n_sub) == cudaSuccess;
    else g->rays_dev = g->dirs_dev;
    ok = ok && cudaMalloc(&g->kloc, sizeof(float) * 64 * nd) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error("geometry allocation failed");
        return fail(CD_ENOMEM);
    }
    if (cudaMemcpyAsync(g->dirs_dev, g->dirs_host, sizeof(double) * 3 * nd, cudaMemcpyHostToDevice, s) !=
            cudaSuccess ||
        (g->n_sub > 1 && cudaMemcpyAsync(g->rays_dev, g->rays_host, sizeof(double) * 3 * nd * g->n_sub,
                                         cudaMemcpyHostToDevice, s) != cudaSuccess)) {
        set_error("direction upload failed");
        return fail(CD_ECUDA);
    }
    cd_status st = build_geometry_tables(g, s);
    if (st != CD_OK) return fail(st);
    if ((st = build_tc_tables(g, s)) != CD_OK) return fail(st);
    // the tables are complete on return, so evaluations on any stream (not
    // only those ordered after `stream`) may read them
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("geometry build failed: %s", cudaGetErrorString(cudaGetLastError()));
        return fail(CD_ECUDA);
    }
    *out = g;
    return CD_OK;
}

// cd_column_density_host: the leaf stage of a uniform tree runs in Morton
// chunks and each chunk's rows go to the host on the copy stream while the
// next chunk is computed
constexpr int kHostChunks = 8;
struct LeafSink {
    float *h_nh, *h_av, *h_sh;     // host destinations (NULL: not wanted)
    cudaStream_t copy;
    cudaEvent_t *ev;               // kHostChunks + 1
    bool used;                     // the leaf stage copied its rows out itself
};

static cd_status evaluate(cd_tree tree, cd_geom geom, const cd_opts *opts_in, float *n_h, float *a_v, float *shield,
                          void *stream, LeafSink *sink)
{
    if (!tree || !geom) {
        set_error("tree or geometry is NULL");
        return CD_EINVAL;
    }
    cd_opts opts;
    if (opts_in) opts = *opts_in; else cd_opts_default(&opts);
    if (opts.precision != CD_FP32 && opts.precision != CD_BF16) {
        set_error("unknown precision %d", opts.precision);
        return CD_EINVAL;
    }
    if (!n_h && !a_v && !shield) return CD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool insitu = geom->mode == CD_MODE_INSITU;
    if (opts.net) {
        if (geom->mode != CD_MODE_PREC) {
            set_error("the learned correction is defined on the single-ray precalculated form");
            return CD_EUNSUPPORTED;
        }
        return column_density_learned(tree, geom, opts, n_h, a_v, shield, s);
    }
    if (tree->amr) return column_density_amr(tree, geom, opts, n_h, a_v, shield, s);
    const int nd = geom->n_dir, L = tree->L;
    cd_status st = ensure_workspace(tree, nd);
    if (st != CD_OK) return st;
    if (insitu) {
        // every shell from the oct centre (an exact walk per level), then the leaves
        if (L >= 2 && (st = launch_insitu(tree, geom, L - 1, tree->n_oct, nullptr, tree->ws.E, s)) != CD_OK) return st;
        LeafLaunch b = {};
        b.n_oct = tree->n_oct;
        b.nd = nd;
        b.dx_leaf = dx_of(tree, L);
        b.av_per_nh = (float)opts.av_per_nh;
        b.shield_k = (float)opts.shield_k;
        b.rho_leaf = tree->rho_leaf;
        b.E = L >= 2 ? tree->ws.E : nullptr;
        b.Sp = nullptr;
        b.kloc = geom->kloc;
        b.n_h = n_h;
        b.a_v = a_v;
        b.shield = shield;
        return launch_leaf(b, s);
    }
    // BF16 tensor cores for receiving levels >= 4 when the direction count
    // fits the accumulator; the few cells of coarser levels stay FP32
    const bool bf16 = opts.precision == CD_BF16 && tc_supported(nd) && geom->wb != nullptr;
    const auto use_tc = [&](int k) { return bf16 && k >= 4; };

    // The oct level's shells need only the densities: they run on side stream
    // 0 in launches of kOctTilesPerCta tiles per CTA, while the far-shell prefix
    // chain (S_k needs S_{k-1}) runs on side stream 1, the high-priority one, so
    // its CTAs take SMs as the oct level's retire; the leaves wait for both.
    SideFork fork(tree, s);
    if ((st = fork.status()) != CD_OK) return st;
    cudaStream_t s_oct = fork.side(0), s_chain = fork.side(1);
    for (int k = 3; k <= L - 2; ++k) {
        ExtLaunch a = {};
        a.k = k;
        a.nd = nd;
        a.tmask = 4;
        a.rho[3] = tree->rho_lvl[k - 2];
        a.dx[3] = dx_of(tree, k - 2);
        a.prefix_in = (k > 3) ? tree->ws.S[k - 1] : nullptr;
        a.out = tree->ws.S[k];
        st = use_tc(k) ? launch_ext_tc(a, tree->rho_brick, geom, s_chain) : launch_ext_fp32(a, geom, s_chain);
        if (st != CD_OK) return st;
    }
    if (L >= 2) {
        ExtLaunch a = {};
        const int k = L - 1;
        a.k = k;
        a.nd = nd;
        for (int t = 1; t <= 3 && t <= k; ++t) {
            a.tmask |= 1 << (t - 1);
            a.rho[t] = tree->rho_lvl[k - t + 1];
            a.dx[t] = dx_of(tree, k - t + 1);
        }
        a.prefix_in = nullptr;   // the leaf kernel adds S_{L-2}[parent]
        a.out = tree->ws.E;
        a.tiles_per_cta = fork.serial() ? 0 : kOctTilesPerCta;
        st = use_tc(k) ? launch_ext_tc(a, tree->rho_brick, geom, s_oct) : launch_ext_fp32(a, geom, s_oct);
        if (st != CD_OK) return st;
    }
    if ((st = fork.join()) != CD_OK) return st;
    LeafLaunch b = {};
    b.n_oct = tree->n_oct;
    b.nd = nd;
    b.dx_leaf = dx_of(tree, L);
    b.av_per_nh = (float)opts.av_per_nh;
    b.shield_k = (float)opts.shield_k;
    b.rho_leaf = tree->rho_leaf;
    b.E = tree->ws.E;
    b.Sp = (L - 2 >= 3) ? tree->ws.S[L - 2] : nullptr;
    b.kloc = geom->kloc;
    b.n_h = n_h;
    b.a_v = a_v;
    b.shield = shield;
    auto leaf = [&](const LeafLaunch &x) {
        if (bf16) {
            const cd_status r = launch_leaf_tc(x, s);
            if (r != CD_EUNSUPPORTED) return r;
        }
        return launch_leaf(x, s);
    };
    if (!sink || tree->n_oct < 16 * kHostChunks) return leaf(b);
    // chunks of whole 16-oct tiles (whole parents too), each copied out once written
    const int64_t per = (tree->n_oct / kHostChunks + 15) & ~(int64_t)15;
    int c = 0;
    for (int64_t o0 = 0; o0 < tree->n_oct; o0 += per, ++c) {
        const int64_t no = std::min(per, tree->n_oct - o0), r0 = 8 * o0, nr = 8 * no;
        LeafLaunch x = b;
        x.n_oct = no;
        x.rho_leaf += r0;
        x.E += o0 * nd;
        if (x.Sp) x.Sp += (o0 / 8) * nd;
        if (x.n_h) x.n_h += r0 * nd;
        if (x.a_v) x.a_v += r0 * nd;
        if (x.shield) x.shield += r0;
        if ((st = leaf(x)) != CD_OK) return st;
        CD_CUDA(cudaEventRecord(sink->ev[c], s));
        CD_CUDA(cudaStreamWaitEvent(sink->copy, sink->ev[c], 0));
        if (sink->h_nh)
            CD_CUDA(cudaMemcpyAsync(sink->h_nh + r0 * nd, x.n_h, sizeof(float) * nr * nd, cudaMemcpyDeviceToHost,
                                    sink->copy));
        if (sink->h_av)
            CD_CUDA(cudaMemcpyAsync(sink->h_av + r0 * nd, x.a_v, sizeof(float) * nr * nd, cudaMemcpyDeviceToHost,
                                    sink->copy));
        if (sink->h_sh)
            CD_CUDA(cudaMemcpyAsync(sink->h_sh + r0, x.shield, sizeof(float) * nr, cudaMemcpyDeviceToHost,
                                    sink->copy));
    }
    CD_CUDA(cudaEventRecord(sink->ev[kHostChunks], sink->copy));
    CD_CUDA(cudaStreamWaitEvent(s, sink->ev[kHostChunks], 0));
    sink->used = true;
    return CD_OK;
}

cd_status cd_column_density(cd_tree tree, cd_geom geom, const cd_opts *opts_in, float *n_h, float *a_v,
                            float *shield, void *stream)
{
    NvtxRange nvtx_range("colden:column_density");
    return evaluate(tree, geom, opts_in, n_h, a_v, shield, stream, nullptr);
}

cd_status cd_column_density_host(cd_tree tree, cd_geom geom, const cd_opts *opts, const float *rho, float *n_h,
                                 float *a_v, float *shield, void *stream)
{
    NvtxRange nvtx_range("colden:column_density_host");
    if (!tree || !geom) {
        set_error("tree or geometry is NULL");
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = tree->n_leaf, nd = geom->n_dir;
    cd_tree_s::HostIO &h = tree->hio;
    cd_status st = ensure_host_io(tree, N * nd, rho != nullptr, n_h != nullptr, a_v != nullptr, shield != nullptr);
    if (st != CD_OK) return st;
    if (rho) {
        CD_CUDA(cudaMemcpyAsync(h.rho, rho, sizeof(float) * N, cudaMemcpyHostToDevice, s));
        if ((st = cd_tree_update(tree, h.rho, 1, stream)) != CD_OK) return st;
    }
    if (!n_h && !a_v && !shield) return CD_OK;
    LeafSink sink = {n_h, a_v, shield, h.copy, h.ev, false};
    if ((st = evaluate(tree, geom, opts, n_h ? h.nh : nullptr, a_v ? h.av : nullptr, shield ? h.sh : nullptr, stream,
                       &sink)) != CD_OK)
        return st;
    if (!sink.used) {
        if (n_h) CD_CUDA(cudaMemcpyAsync(n_h, h.nh, sizeof(float) * N * nd, cudaMemcpyDeviceToHost, s));
        if (a_v) CD_CUDA(cudaMemcpyAsync(a_v, h.av, sizeof(float) * N * nd, cudaMemcpyDeviceToHost, s));
        if (shield) CD_CUDA(cudaMemcpyAsync(shield, h.sh, sizeof(float) * N, cudaMemcpyDeviceToHost, s));
    }
    return CD_OK;
}

void cd_debug_wait_polls(int64_t polls) { set_leaf_tc_wait_polls(polls); }

void cd_debug_leaf_span(int rows) { set_leaf_tc_span_max(rows); }

cd_status cd_checked_status(int *site, int64_t *index)
{
#ifndef COLDEN_CHECKED
    (void)site;
    (void)index;
    set_error("this library was built without COLDEN_CHECKED");
    return CD_EUNSUPPORTED;
#else
    CD_CUDA(cudaDeviceSynchronize());
    int s0 = 0;
    int64_t i0 = 0;
    for (CheckReader r : check_readers()) {
        CheckWord w = {};
        if (!r(&w)) {
            set_error("reading a check word failed: %s", cudaGetErrorString(cudaGetLastError()));
            return CD_ECUDA;
        }
        if (w.site && !s0) {
            s0 = w.site;
            i0 = w.index;
        }
    }
    if (site) *site = s0;
    if (index) *index = i0;
    return CD_OK;
#endif
}

cd_status cd_debug_check_probe(int64_t i, void *stream)
{
#ifndef COLDEN_CHECKED
    (void)i;
    (void)stream;
    set_error("this library was built without COLDEN_CHECKED");
    return CD_EUNSUPPORTED;
#else
    cudaStream_t s = (cudaStream_t)stream;
    float *buf = nullptr;
    if (cudaMallocAsync(&buf, 5 * sizeof(float), s) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate the probe buffer");
        return CD_ENOMEM;
    }
    CD_CUDA(cudaMemsetAsync(buf, 0, 5 * sizeof(float), s));
    {
        LaunchScope ls(CD_K_OTHER, s);
        check_probe<<<1, 1, 0, s>>>(buf, i, buf + 4);
    }
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(buf, s);
    if (e != cudaSuccess) {
        set_error("probe launch failed: %s", cudaGetErrorString(e));
        return CD_ECUDA;
    }
    CD_CUDA(cudaStreamSynchronize(s));
    return CD_OK;
#endif
}

cd_status cd_device_status(void *stream)
{
    CD_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    cd_status a = leaf_fault_check();
    cd_status b = tc_fault_check();
    cd_status c = learned_tc_fault_check();
    cd_status d = leaf_tc_fault_check();
    return a != CD_OK ? a : b != CD_OK ? b : c != CD_OK ? c : d;
}

cd_status cd_tree_info(cd_tree t, int64_t *n_leaf, int *max_level, int *base_level, int64_t *n_oct)
{
    if (!t) {
        set_error("tree is NULL");
        return CD_EINVAL;
    }
    if (n_leaf) *n_leaf = t->n_leaf;
    if (max_level) *max_level = t->L;
    if (base_level) *base_level = t->base;
    if (n_oct) *n_oct = t->n_oct;
    return CD_OK;
}

cd_status cd_tree_leaves(cd_tree t, int8_t *level, int32_t *ijk)
{
    if (!t) {
        set_error("tree is NULL");
        return CD_EINVAL;
    }
    if (t->amr) {
        if (level) memcpy(level, t->leaf_level_h, t->n_leaf);
        if (ijk) memcpy(ijk, t->leaf_ijk_h, sizeof(int32_t) * 3 * t->n_leaf);
        return CD_OK;
    }
    for (int64_t i = 0; i < t->n_leaf; ++i) {
        if (level) level[i] = (int8_t)t->L;
        if (ijk) {
            ijk[3 * i] = (int32_t)compact3((uint64_t)i);
            ijk[3 * i + 1] = (int32_t)compact3((uint64_t)i >> 1);
            ijk[3 * i + 2] = (int32_t)compact3((uint64_t)i >> 2);
        }
    }
    return CD_OK;
}

cd_status cd_geom_info(cd_geom g, int *n_dir, double *dirs)
{
    if (!g) {
        set_error("geometry is NULL");
        return CD_EINVAL;
    }
    if (n_dir) *n_dir = g->n_dir;
    if (dirs) memcpy(dirs, g->dirs_host, sizeof(double) * 3 * g->n_dir);
    return CD_OK;
}

cd_status cd_geom_rays(cd_geom g, int *n_sub, double *rays)
{
    if (!g) {
        set_error("geometry is NULL");
        return CD_EINVAL;
    }
    if (n_sub) *n_sub = g->n_sub;
    if (rays) memcpy(rays, g->rays_host, sizeof(double) * 3 * g->n_dir * g->n_sub);
    return CD_OK;
}

void cd_tree_free(cd_tree t)
{
    if (!t) return;
    cudaDeviceSynchronize();
    free_workspace(t);
    free_side_streams(t);
    free_host_io(t);
    free_level_sums(t);
    free_tc_lists(t);
    for (int l = 0; l <= CD_MAXL; ++l) {
        if (t->rho_lvl[l]) cd::lib_free(t->rho_lvl[l]);
        if (t->rho_brick[l]) cd::lib_free(t->rho_brick[l]);
    }
    if (t->rho_leaf) cd::lib_free(t->rho_leaf);
    for (int l = 0; l <= CD_MAXL; ++l) {
        if (t->ref_key[l]) cd::lib_free(t->ref_key[l]);
        if (t->ref_parent[l]) cd::lib_free(t->ref_parent[l]);
    }
    for (void *p : {(void *)t->deep_key, (void *)t->deep_paint, (void *)t->mid_key, (void *)t->mid_paint,
                    (void *)t->oct_key, (void *)t->oct_parent,
                    (void *)t->oct_leaf, (void *)t->oct_rho8, (void *)t->leaf_slot, (void *)t->ref8,
                    (void *)t->leaf_key, (void *)t->leaf_lvl, (void *)t->leaf_src})
        if (p) cd::lib_free(p);
    delete[] t->leaf_level_h;
    delete[] t->leaf_ijk_h;
    delete[] t->leaf_src_h;
    delete t;
}

void cd_geom_free(cd_geom g)
{
    if (!g) return;
    cudaDeviceSynchronize();
    if (g->rays_dev && g->rays_dev != g->dirs_dev) cd::lib_free(g->rays_dev);
    if (g->dirs_dev) cd::lib_free(g->dirs_dev);
    for (int t = 0; t < 4; ++t) {
        if (g->tab[t]) cd::lib_free(g->tab[t]);
        if (g->cmax[t]) cd::lib_free(g->cmax[t]);
    }
    if (g->kloc) cd::lib_free(g->kloc);
    if (g->wb) cd::lib_free(g->wb);
    if (g->rays_host != g->dirs_host) delete[] g->rays_host;
    delete[] g->dirs_host;
    delete[] g->custom;
    delete g;
}

}  // extern "C"
