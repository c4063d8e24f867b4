// Many independent boxes in one launch.
//
// cd_column_density_batch: the boxes one after another on one stream (the
// per-box-launch baseline).
//
// cd_batch_*: a batch object that owns one CUDA graph.  For BF16 batches of
// boxes the tensor-core path serves (the usual case), the graph holds a few
// persistent launches over work lists instead of every box's kernels:
//   1. one FP32 launch for the far shells of level 3 of every box (one list
//      of 512 cells per box, blockIdx.y = box);
//   2. one persistent tensor-core launch over every (box, level, tile) of
//      the shell contraction: the far shells of levels 4 .. L-2 (table 3) in
//      order of level, then every oct level (tables 1-3, uniform tiles or the
//      AMR receiver lists).  A far tile of level k adds S_{k-1} of its box in
//      its epilogue once that box's level k-1 is complete (a counter per job,
//      bounded spin; every wait points at lower tiles, which resident CTAs
//      finish first); an AMR oct tile adds S_{k-1} the same way;
//   3. one persistent leaf launch per direction set over every (box, tile)
//      of the leaf epilogue (uniform 128-leaf tiles, AMR 16-oct list tiles).
// An autotuner times the live batch at creation over the shell tile shape
// (half the children, N = 4 nd, or all 8, N = 8 nd, where nd <= 32) and the
// shell CTAs per SM (1 or 2), keeps the fastest and captures it.  Other
// batches (FP32, in-situ geometry, small or shallow trees) fall back to a
// graph of every box's own kernels over W forked streams, W tuned over 1, 2,
// 4, 8 (boxes assigned largest first to the least loaded stream).  Either way
// the graph reads the trees' current densities at every replay (cd_tree_update
// between replays is seen), but it holds the trees, geometries and output
// pointers given at creation: they must outlive the batch.  While a batch
// lives, its trees' scratch is pinned: an evaluation that would reallocate it
// (another direction count) returns CD_EINVAL.
#include <algorithm>
#include <atomic>
#include <map>
#include <numeric>
#include <tuple>
#include <vector>

#include "common.cuh"

namespace cd {
namespace {

// The persistent form of one batch: device job tables and the chosen shapes.
struct Plan {
    int full = 0;                    // shell tiles cover all 8 children where nd <= 32
    int ctas = 2;                    // shell CTAs per SM requested
    int ctas_used = 0;               // and launched (at most what fits an SM)
    void *tc_jobs = nullptr;
    int2 *tc_tile_ref = nullptr;
    int *tc_done = nullptr;
    int n_tc = 0;
    int64_t tc_total = 0;
    uint32_t bstage_max = 0;
    double tc_flops = 0.0;
    void *list_jobs = nullptr;
    int n_list = 0;
    struct Leaf {
        int nd;
        const float *kloc;
        void *jobs;
        int2 *tile_ref;
        int64_t total;
        int form;                    // output form shared by the launch's jobs
        double flops;
    };
    std::vector<Leaf> leaves;
    std::vector<void *> allocs;
};

}  // namespace
}  // namespace cd

struct cd_batch_s {
    std::vector<cd_tree> trees;
    std::vector<cd_geom> geoms;
    std::vector<float *> n_h, a_v, shield;
    cd_opts opts;
    int width = 1;
    double ms_tried[4] = {-1, -1, -1, -1};   // eager ms for W = 1, 2, 4, 8
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t main = nullptr;             // branch 0 during tuning and capture
    std::vector<cudaStream_t> streams;       // W - 1 side streams
    std::vector<cudaEvent_t> events;
    int64_t kernel_nodes = 0;
    bool pinned = false;                     // batch_refs of the distinct trees were raised
    bool persistent = false;                 // the graph holds the persistent launches of `plan`
    cd::Plan plan;
    double plan_ms[4] = {-1, -1, -1, -1};    // eager ms for (half, 1), (half, 2), (full, 1), (full, 2)
    uint64_t *keys512 = nullptr;             // Morton keys 0 .. 511 (level-3 lists)
};

namespace cd {
namespace {

// largest work first onto the least loaded branch
std::vector<int> assign(const cd_batch_s &b, int W)
{
    const int n = (int)b.trees.size();
    std::vector<int> ord(n), branch(n);
    std::vector<double> work(n), load(W, 0.0);
    for (int i = 0; i < n; ++i) work[i] = (double)b.trees[i]->n_leaf * b.geoms[i]->n_dir;
    std::iota(ord.begin(), ord.end(), 0);
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return work[x] > work[y]; });
    for (int i : ord) {
        const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        branch[i] = w;
        load[w] += work[i];
    }
    return branch;
}

// Enqueues the whole batch over W branches (stream s + W-1 side streams).
cd_status enqueue(cd_batch_s &b, int W, cudaStream_t s)
{
    const auto branch = assign(b, W);
    CD_CUDA(cudaEventRecord(b.events[0], s));
    for (int w = 1; w < W; ++w) CD_CUDA(cudaStreamWaitEvent(b.streams[w - 1], b.events[0], 0));
    for (size_t i = 0; i < b.trees.size(); ++i) {
        cudaStream_t si = branch[i] == 0 ? s : b.streams[branch[i] - 1];
        cd_status st = cd_column_density(b.trees[i], b.geoms[i], &b.opts, b.n_h[i], b.a_v[i], b.shield[i], si);
        if (st != CD_OK) return st;
    }
    for (int w = 1; w < W; ++w) {
        CD_CUDA(cudaEventRecord(b.events[w], b.streams[w - 1]));
        CD_CUDA(cudaStreamWaitEvent(s, b.events[w], 0));
    }
    return CD_OK;
}

void plan_free(Plan &P)
{
    for (void *p : P.allocs)
        if (p) cd::lib_free(p);
    P = Plan();
}

template <typename T>
cd_status upload(Plan &P, T **dst, const void *src, size_t bytes)
{
    *dst = nullptr;
    if (bytes == 0) return CD_OK;
    void *d = nullptr;
    if (cudaMalloc(&d, bytes) != cudaSuccess) {
        cudaGetLastError();
        set_error("cannot allocate the batch work lists (%zu bytes)", bytes);
        return CD_ENOMEM;
    }
    P.allocs.push_back(d);
    if (cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        set_error("batch work-list upload failed");
        return CD_ECUDA;
    }
    *dst = static_cast<T *>(d);
    return CD_OK;
}

float dx_at(const cd_tree t, int l) { return (float)(t->box_cm / (double)((int64_t)1 << l)); }

// Whether every box takes the persistent form: BF16 tensor-core shells at
// every level from 4 up, level 3 complete, leaves on the tensor-core leaf
// kernel.  The eager warm-up has sized every tree's scratch for its geometry.
bool plan_supported(const cd_batch_s &b)
{
    if (b.opts.precision != CD_BF16 || b.opts.net) return false;
    for (size_t i = 0; i < b.trees.size(); ++i) {
        const cd_tree t = b.trees[i];
        const cd_geom g = b.geoms[i];
        const int nd = g->n_dir;
        if (g->mode == CD_MODE_INSITU || !tc_supported(nd) || !g->wb || t->ws.ndir != nd || nd % 4 != 0) return false;
        if (b.n_h[i] && ((uintptr_t)b.n_h[i] & 15)) return false;
        if (b.a_v[i] && ((uintptr_t)b.a_v[i] & 15)) return false;
        if (!t->amr) {
            if (t->L < 5) return false;
            continue;
        }
        if (t->base < 5) return false;
        for (int k = 4; k <= t->L - 2; ++k)
            if (t->n_ref[k] && t->n_ref[k] != ((int64_t)1 << (3 * k)) && !t->tc_ref[k].ntiles) return false;
        for (int k = 0; k <= t->L - 1; ++k)
            if (t->oct_begin[k + 1] > t->oct_begin[k] && (k < 4 || !t->tc_oct[k].ntiles)) return false;
    }
    return true;
}

// Builds the work lists of the persistent form with the given shapes.
cd_status plan_build(cd_batch_s &b, int full, int ctas, Plan &P)
{
    P = Plan();
    P.full = full;
    P.ctas = ctas;
    const size_t tcb = tc_job_bytes(), lfb = leaf_tc_job_bytes(), lsb = list_job_bytes();
    // shell jobs: far levels by level, then oct levels; (box, level) -> job for the waits
    struct Pending {
        int level;       // far level, or 100 + level for an oct level
        size_t box;
        TcJobDesc d;
        int waits_on_level;   // far level whose job this one waits for (-1: none)
    };
    std::vector<Pending> pend;
    std::vector<unsigned char> lists;
    // leaf launches: one per direction table (kloc) and output form
    using LeafKey = std::tuple<const float *, int, int>;   // kloc, nd, form
    std::map<LeafKey, std::vector<unsigned char>> leaf_jobs;
    std::map<LeafKey, double> leaf_flops;
    std::map<LeafKey, std::vector<int64_t>> leaf_tiles;
    for (size_t i = 0; i < b.trees.size(); ++i) {
        const cd_tree t = b.trees[i];
        const cd_geom g = b.geoms[i];
        const int nd = g->n_dir, L = t->L;
        const bool fl = full && 8 * nd <= 256;
        // level 3: FP32 list over the 512 cells
        lists.resize(lists.size() + lsb);
        list_job_fill_far3(t, g, b.keys512, lists.data() + lists.size() - lsb);
        ++P.n_list;
        for (int k = 4; k <= L - 2; ++k) {
            if (t->amr && !t->n_ref[k]) break;
            Pending q = {};
            q.level = k;
            q.box = i;
            q.d.a.k = k;
            q.d.a.nd = nd;
            q.d.a.tmask = 4;
            q.d.a.dx[3] = dx_at(t, k - 2);
            q.d.a.out = t->ws.S[k];
            q.d.a.list = (!t->amr || t->n_ref[k] == ((int64_t)1 << (3 * k))) ? nullptr : &t->tc_ref[k];
            q.d.full = fl;
            q.d.prefix = t->ws.S[k - 1];
            q.d.prefix_row = q.d.a.list ? q.d.a.list->recv_parent : nullptr;
            q.waits_on_level = k - 1 >= 4 ? k - 1 : -1;
            pend.push_back(q);
        }
        auto oct_job = [&](int k, float *out, const TcList *list, const float *prefix, const int32_t *prow) {
            Pending q = {};
            q.level = 100 + k;
            q.box = i;
            q.d.a.k = k;
            q.d.a.nd = nd;
            q.d.a.tmask = 7;
            for (int tt = 1; tt <= 3; ++tt) q.d.a.dx[tt] = dx_at(t, k - tt + 1);
            q.d.a.out = out;
            q.d.a.list = list;
            q.d.full = fl;
            q.d.prefix = prefix;
            q.d.prefix_row = prow;
            q.waits_on_level = prefix && k - 1 >= 4 ? k - 1 : -1;
            pend.push_back(q);
        };
        auto add_leaf = [&](const LeafLaunch &a) {
            std::vector<unsigned char> job(lfb);
            const int64_t nt = leaf_tc_job_fill(a, job.data());
            if (nt < 0) return false;
            const LeafKey key(a.kloc, nd, leaf_tc_job_form(job.data()));
            std::vector<unsigned char> &v = leaf_jobs[key];
            v.insert(v.end(), job.begin(), job.end());
            leaf_tiles[key].push_back(nt);
            leaf_flops[key] += leaf_tc_job_flops(job.data());
            return true;
        };
        LeafLaunch lb = {};
        lb.nd = nd;
        lb.av_per_nh = (float)b.opts.av_per_nh;
        lb.shield_k = (float)b.opts.shield_k;
        lb.kloc = g->kloc;
        lb.n_h = b.n_h[i];
        lb.a_v = b.a_v[i];
        lb.shield = b.shield[i];
        lb.n_rows = t->n_leaf;
        if (!t->amr) {
            oct_job(L - 1, t->ws.E, nullptr, nullptr, nullptr);
            lb.n_oct = t->n_oct;
            lb.dx_leaf = dx_at(t, L);
            lb.rho_leaf = t->rho_leaf;
            lb.E = t->ws.E;
            lb.Sp = t->ws.S[L - 2];
            if (!add_leaf(lb)) return CD_EUNSUPPORTED;
            continue;
        }
        for (int k = 4; k <= L - 1; ++k) {
            const int64_t no = t->oct_begin[k + 1] - t->oct_begin[k];
            if (!no) continue;
            float *Ek = t->ws.E + t->oct_begin[k] * nd;
            const bool pre = k - 1 >= 3;
            oct_job(k, Ek, &t->tc_oct[k], pre ? t->ws.S[k - 1] : nullptr, pre ? t->oct_parent + t->oct_begin[k] : nullptr);
            LeafLaunch a = lb;
            a.n_oct = no;
            a.dx_leaf = dx_at(t, k + 1);
            a.rho_leaf = t->oct_rho8 + 8 * t->oct_begin[k];
            a.E = Ek;
            a.Sp = nullptr;
            a.oleaf = t->oct_leaf + 8 * t->oct_begin[k];
            if (!add_leaf(a)) return CD_EUNSUPPORTED;
        }
    }
    std::stable_sort(pend.begin(), pend.end(), [](const Pending &x, const Pending &y) { return x.level < y.level; });
    std::map<std::pair<size_t, int>, int> job_of;   // (box, far level) -> job
    std::vector<unsigned char> jobs(pend.size() * tcb);
    std::vector<int64_t> first(pend.size() + 1, 0), ntiles(pend.size(), 0);
    for (size_t j = 0; j < pend.size(); ++j) {
        Pending &q = pend[j];
        if (q.waits_on_level >= 0) {
            const auto it = job_of.find({q.box, q.waits_on_level});
            if (it == job_of.end()) return CD_EUNSUPPORTED;
            q.d.wait_job = it->second;
            q.d.wait_count = (int)(8 * ntiles[it->second]);
        } else {
            q.d.wait_job = -1;
        }
        const int64_t nt = tc_job_fill(q.d, b.trees[q.box]->rho_brick, b.geoms[q.box], jobs.data() + j * tcb);
        if (nt < 0) return CD_EUNSUPPORTED;
        ntiles[j] = nt;
        first[j + 1] = first[j] + nt;
        if (q.level < 100) job_of[{q.box, q.level}] = (int)j;
        P.tc_flops += tc_job_flops(jobs.data() + j * tcb);
        P.bstage_max = std::max(P.bstage_max, tc_job_bstage(jobs.data() + j * tcb));
    }
    for (size_t j = 0; j < pend.size(); ++j)
        if (pend[j].d.wait_job >= 0) tc_job_set_signal(jobs.data() + (size_t)pend[j].d.wait_job * tcb);
    P.n_tc = (int)pend.size();
    P.tc_total = first.back();
    std::vector<int2> tile_ref((size_t)P.tc_total);
    for (size_t j = 0; j < pend.size(); ++j)
        for (int64_t g = first[j]; g < first[j + 1]; ++g) tile_ref[(size_t)g] = make_int2((int)j, (int)(g - first[j]));
    cd_status st;
    if ((st = upload(P, &P.tc_jobs, jobs.data(), jobs.size())) != CD_OK) return st;
    if ((st = upload(P, &P.tc_tile_ref, tile_ref.data(), tile_ref.size() * sizeof(int2))) != CD_OK) return st;
    // done[job] per job, then the work counter
    std::vector<int> zeros(std::max(1, P.n_tc) + 1, 0);
    if ((st = upload(P, &P.tc_done, zeros.data(), zeros.size() * 4)) != CD_OK) return st;
    if ((st = upload(P, &P.list_jobs, lists.data(), lists.size())) != CD_OK) return st;
    for (auto &kv : leaf_jobs) {
        Plan::Leaf lf = {};
        lf.kloc = std::get<0>(kv.first);
        lf.nd = std::get<1>(kv.first);
        lf.form = std::get<2>(kv.first);
        lf.flops = leaf_flops[kv.first];
        const std::vector<int64_t> &nts = leaf_tiles[kv.first];
        std::vector<int64_t> lfirst(nts.size() + 1, 0);
        for (size_t j = 0; j < nts.size(); ++j) lfirst[j + 1] = lfirst[j] + nts[j];
        lf.total = lfirst.back();
        std::vector<int2> ltile((size_t)lf.total);
        for (size_t j = 0; j < nts.size(); ++j)
            for (int64_t g = lfirst[j]; g < lfirst[j + 1]; ++g) ltile[(size_t)g] = make_int2((int)j, (int)(g - lfirst[j]));
        if ((st = upload(P, &lf.jobs, kv.second.data(), kv.second.size())) != CD_OK) return st;
        if ((st = upload(P, &lf.tile_ref, ltile.data(), ltile.size() * sizeof(int2))) != CD_OK) return st;
        P.leaves.push_back(lf);
    }
    return CD_OK;
}

// The persistent form on stream s: counters cleared, level 3, the shell
// launch, one leaf launch per direction set.
cd_status plan_enqueue(Plan &P, cudaStream_t s)
{
    CD_CUDA(cudaMemsetAsync(P.tc_done, 0, sizeof(int) * (std::max(1, P.n_tc) + 1), s));
    cd_status st = launch_list_batch(P.list_jobs, P.n_list, (int64_t)512 * 64, s);
    if (st != CD_OK) return st;
    if ((st = launch_tc_batch(P.tc_jobs, P.tc_tile_ref, P.tc_total, P.tc_done, P.tc_done + std::max(1, P.n_tc),
                              P.bstage_max, P.ctas, P.tc_flops, s, &P.ctas_used)) != CD_OK)
        return st;
    for (const Plan::Leaf &lf : P.leaves)
        if ((st = launch_leaf_tc_batch(lf.jobs, lf.tile_ref, lf.total, lf.nd, lf.kloc, lf.form, lf.flops, s)) != CD_OK)
            return st;
    return CD_OK;
}

// cd_debug_batch_form: -1 the autotuner picks, 0 per-box launches only, 1 the
// persistent form where the batch supports it
std::atomic<int> g_batch_form{-1};

// A candidate form of the batch, captured and instantiated, with its replay time.
struct Tuned {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    double ms = 1e30;
};

void tuned_free(Tuned &t)
{
    if (t.exec) cudaGraphExecDestroy(t.exec);
    if (t.graph) cudaGraphDestroy(t.graph);
    t = Tuned();
}

// Capture enq(s) into a graph, replay it once as a warm-up, then time two
// replays (CUDA events on s).  Errors: the enqueue's own status, CD_ECUDA for
// a failed capture, instantiation or replay.
template <class F>
cd_status tune_form(cudaStream_t s, F &&enq, Tuned &out)
{
    out = Tuned();
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        set_error("stream capture could not start (is the stream already capturing?)");
        return CD_ECUDA;
    }
    const cd_status st = enq(s);
    const cudaError_t ce = cudaStreamEndCapture(s, &out.graph);
    if (st != CD_OK || ce != cudaSuccess) {
        tuned_free(out);
        if (st == CD_OK) set_error("stream capture failed: %s", cudaGetErrorString(ce));
        return st != CD_OK ? st : CD_ECUDA;
    }
    if (cudaGraphInstantiate(&out.exec, out.graph, 0) != cudaSuccess) {
        tuned_free(out);
        set_error("graph instantiation failed");
        return CD_ECUDA;
    }
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    float ms = 0.f;
    bool ok = cudaEventCreate(&t0) == cudaSuccess && cudaEventCreate(&t1) == cudaSuccess &&
              cudaGraphLaunch(out.exec, s) == cudaSuccess && cudaEventRecord(t0, s) == cudaSuccess &&
              cudaGraphLaunch(out.exec, s) == cudaSuccess && cudaGraphLaunch(out.exec, s) == cudaSuccess &&
              cudaEventRecord(t1, s) == cudaSuccess && cudaEventSynchronize(t1) == cudaSuccess &&
              cudaEventElapsedTime(&ms, t0, t1) == cudaSuccess;
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (!ok) {
        tuned_free(out);
        set_error("batch tuning replay failed: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    // the kernels' own bounded waits report through the device flags
    cd_status fs = cd_device_status(s);
    if (fs != CD_OK) {
        tuned_free(out);
        return fs;
    }
    out.ms = ms / 2.0;
    return CD_OK;
}

void destroy(cd_batch_s *b)
{
    plan_free(b->plan);
    if (b->keys512) cd::lib_free(b->keys512);
    if (b->pinned)
        for (size_t i = 0; i < b->trees.size(); ++i)
            if (std::find(b->trees.begin(), b->trees.begin() + i, b->trees[i]) == b->trees.begin() + i)
                --b->trees[i]->batch_refs;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->streams) cudaStreamDestroy(s);
    if (b->main) cudaStreamDestroy(b->main);
    for (auto e : b->events) cudaEventDestroy(e);
    delete b;
}

}  // namespace
}  // namespace cd

using namespace cd;

extern "C" {

cd_status cd_column_density_batch(int n, const cd_tree *trees, const cd_geom *geoms, const cd_opts *opts,
                                  float *const *n_h, float *const *a_v, float *const *shield, void *stream)
{
    NvtxRange nvtx_range("colden:column_density_batch");
    if (n < 0 || (n > 0 && (!trees || !geoms))) {
        set_error("bad batch arguments");
        return CD_EINVAL;
    }
    for (int i = 0; i < n; ++i) {
        cd_status st = cd_column_density(trees[i], geoms[i], opts, n_h ? n_h[i] : nullptr, a_v ? a_v[i] : nullptr,
                                         shield ? shield[i] : nullptr, stream);
        if (st != CD_OK) return st;
    }
    return CD_OK;
}

cd_status cd_batch_create(int n, const cd_tree *trees, const cd_geom *geoms, const cd_opts *opts, float *const *n_h,
                          float *const *a_v, float *const *shield, void *stream, cd_batch *out)
{
    NvtxRange nvtx_range("colden:batch_create");
    if (!out || n < 1 || !trees || !geoms) {
        set_error("bad batch arguments");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (opts && opts->net) {
        // the learned form caches per-level sums between calls and skips their
        // launches when the densities have not changed, so a captured graph
        // would replay stale sums after cd_tree_update
        set_error("batches evaluate the plain tree method; call cd_column_density_batch for the learned form");
        return CD_EUNSUPPORTED;
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < i; ++j)
            if (trees[i] && trees[i] == trees[j] && geoms[i] && geoms[j] && geoms[i]->n_dir != geoms[j]->n_dir) {
                // one scratch per tree: the graph would hold the one sized last
                set_error("batch entries %d and %d share a tree with %d and %d directions", j, i, geoms[j]->n_dir,
                          geoms[i]->n_dir);
                return CD_EINVAL;
            }
    cd_batch_s *b = new cd_batch_s();
    if (opts) b->opts = *opts; else cd_opts_default(&b->opts);
    for (int i = 0; i < n; ++i) {
        if (!trees[i] || !geoms[i]) {
            delete b;
            set_error("batch entry %d has no tree or geometry", i);
            return CD_EINVAL;
        }
        b->trees.push_back(trees[i]);
        b->geoms.push_back(geoms[i]);
        b->n_h.push_back(n_h ? n_h[i] : nullptr);
        b->a_v.push_back(a_v ? a_v[i] : nullptr);
        b->shield.push_back(shield ? shield[i] : nullptr);
    }
    // tuning and capture run on an internal stream ordered after the caller's
    // (the legacy default stream cannot be captured)
    cudaStream_t user = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        set_error("stream creation failed");
        return CD_ECUDA;
    }
    cudaStream_t s = b->main;
    const int wmax = std::min(8, n);
    for (int w = 1; w < wmax; ++w) {
        cudaStream_t x;
        if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) {
            destroy(b);
            set_error("stream creation failed");
            return CD_ECUDA;
        }
        b->streams.push_back(x);
    }
    for (int w = 0; w < 8; ++w) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            destroy(b);
            set_error("event creation failed");
            return CD_ECUDA;
        }
        b->events.push_back(e);
    }
    // one eager warm-up (allocates every box's workspace outside any capture)
    cd_status st = CD_OK;
    if (cudaEventRecord(b->events[0], user) != cudaSuccess || cudaStreamWaitEvent(s, b->events[0], 0) != cudaSuccess) {
        set_error("cannot order the batch after the caller's stream");
        st = CD_ECUDA;
    }
    if (st == CD_OK) st = enqueue(*b, 1, s);
    if (st == CD_OK && cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("batch warm-up failed: %s", cudaGetErrorString(cudaGetLastError()));
        st = CD_ECUDA;
    }
    if (st != CD_OK) {
        destroy(b);
        return st;
    }
    // autotune: every candidate form is captured into a graph and its replay
    // timed; the fastest graph is kept.  Candidates: the persistent form with
    // each shell tile shape (half / all children) x CTAs per SM, and the
    // per-box launches fanned out over W = 1, 2, 4, 8 streams.
    Tuned best;
    const int forced = g_batch_form.load();
    if (forced != 0 && plan_supported(*b)) {
        std::vector<uint64_t> keys(512);
        for (int c = 0; c < 512; ++c) keys[c] = (uint64_t)c;
        if (cudaMalloc(&b->keys512, 512 * 8) != cudaSuccess ||
            cudaMemcpy(b->keys512, keys.data(), 512 * 8, cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            destroy(b);
            set_error("cannot allocate the batch work lists");
            return CD_ENOMEM;
        }
        bool narrow = false;   // a box whose tiles can cover all 8 children
        for (auto g : b->geoms) narrow = narrow || 8 * g->n_dir <= 256;
        for (int full = 0; full <= (narrow ? 1 : 0); ++full)
            for (int ctas = 1; ctas <= 2; ++ctas) {
                Plan P;
                cd_status ps = plan_build(*b, full, ctas, P);
                Tuned c;
                if (ps == CD_OK) ps = tune_form(s, [&](cudaStream_t x) { return plan_enqueue(P, x); }, c);
                if (ps == CD_ECUDA || ps == CD_ETIMEOUT) {   // a device error: do not go on
                    plan_free(P);
                    tuned_free(best);
                    destroy(b);
                    return ps;
                }
                if (ps != CD_OK) {
                    cudaGetLastError();
                    plan_free(P);
                    continue;
                }
                b->plan_ms[2 * full + ctas - 1] = c.ms;
                if (c.ms < best.ms) {
                    tuned_free(best);
                    best = c;
                    plan_free(b->plan);
                    b->plan = P;
                    b->persistent = true;
                } else {
                    tuned_free(c);
                    plan_free(P);
                }
            }
    }
    const int cand[4] = {1, 2, 4, 8};
    for (int c = 0; c < 4 && cand[c] <= wmax && !(forced == 1 && b->persistent); ++c) {
        const int W = cand[c];
        Tuned t;
        st = tune_form(s, [&](cudaStream_t x) { return enqueue(*b, W, x); }, t);
        if (st != CD_OK) break;
        b->ms_tried[c] = t.ms;
        if (t.ms < best.ms) {
            tuned_free(best);
            best = t;
            b->persistent = false;
            b->width = W;
        } else {
            tuned_free(t);
        }
    }
    if (st != CD_OK || !best.exec) {
        tuned_free(best);
        destroy(b);
        if (st == CD_OK) {
            set_error("no batch form could be captured");
            st = CD_ECUDA;
        }
        return st;
    }
    if (!b->persistent) plan_free(b->plan);
    b->graph = best.graph;
    b->exec = best.exec;
    size_t nn = 0;
    if (cudaGraphGetNodes(b->graph, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(b->graph, nodes.data(), &nn);
        for (auto nd : nodes) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++b->kernel_nodes;
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        destroy(b);
        set_error("batch tuning failed: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    // the graph now holds every tree's scratch pointers: pin them
    for (size_t i = 0; i < b->trees.size(); ++i)
        if (std::find(b->trees.begin(), b->trees.begin() + i, b->trees[i]) == b->trees.begin() + i)
            ++b->trees[i]->batch_refs;
    b->pinned = true;
    *out = b;
    return CD_OK;
}

void cd_debug_batch_form(int form) { cd::g_batch_form.store(form < 0 ? -1 : form > 1 ? 1 : form); }

cd_status cd_batch_run(cd_batch b, void *stream)
{
    NvtxRange nvtx_range("colden:batch_run");
    if (!b) {
        set_error("batch is NULL");
        return CD_EINVAL;
    }
    // while per-launch timing is on, the launches go out directly (a graph
    // replay would hide them from the per-kind timers)
    if (stats_timing()) return b->persistent ? plan_enqueue(b->plan, (cudaStream_t)stream)
                                             : enqueue(*b, 1, (cudaStream_t)stream);
    LaunchScope ls(CD_K_OTHER, (cudaStream_t)stream);
    CD_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
    return CD_OK;
}

cd_status cd_batch_plan(cd_batch b, int *persistent, int *full_tiles, int *ctas_per_sm, double *ms_tried)
{
    if (!b) {
        set_error("batch is NULL");
        return CD_EINVAL;
    }
    if (persistent) *persistent = b->persistent ? 1 : 0;
    if (full_tiles) *full_tiles = b->persistent ? b->plan.full : 0;
    if (ctas_per_sm) *ctas_per_sm = b->persistent ? b->plan.ctas_used : 0;
    if (ms_tried)
        for (int c = 0; c < 4; ++c) ms_tried[c] = b->plan_ms[c];
    return CD_OK;
}

cd_status cd_batch_info(cd_batch b, int *width, double *ms_tried, int64_t *kernel_nodes)
{
    if (!b) {
        set_error("batch is NULL");
        return CD_EINVAL;
    }
    if (width) *width = b->width;
    if (kernel_nodes) *kernel_nodes = b->kernel_nodes;
    if (ms_tried)
        for (int c = 0; c < 4; ++c) ms_tried[c] = b->ms_tried[c];
    return CD_OK;
}

void cd_batch_free(cd_batch b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    destroy(b);
}

}  // extern "C"
