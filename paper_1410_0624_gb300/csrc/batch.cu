// Many independent boxes in one launch.
//
// cd_column_density_batch: the boxes one after another on one stream (the
// per-box-launch baseline).
//
// cd_batch_*: a batch object that owns one CUDA graph holding every kernel of
// every box.  At creation an autotuner times the batch run eagerly over
// W = 1, 2, 4, 8 concurrent streams (boxes assigned largest first to the least
// loaded stream) and keeps the fastest W; the per-box pipelines are then
// captured on W forked streams and joined back, so one cudaGraphLaunch runs
// the whole batch with independent boxes overlapping on the GPU.  The graph
// reads the trees' current densities at every replay (cd_tree_update between
// replays is seen), but it holds the trees, geometries and output pointers
// given at creation: they must outlive the batch.  While a batch lives, its
// trees' scratch is pinned: an evaluation that would reallocate it (another
// direction count) returns CD_EINVAL.
#include <algorithm>
#include <numeric>
#include <vector>

#include "common.cuh"

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

void destroy(cd_batch_s *b)
{
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
    // autotune the branch count: one eager warm-up (allocates every box's
    // workspace outside the capture), then time W = 1, 2, 4, 8
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    cd_status st = CD_OK;
    if (cudaEventRecord(b->events[0], user) != cudaSuccess || cudaStreamWaitEvent(s, b->events[0], 0) != cudaSuccess) {
        set_error("cannot order the batch after the caller's stream");
        st = CD_ECUDA;
    }
    if (st == CD_OK) st = enqueue(*b, 1, s);
    double best = 1e30;
    const int cand[4] = {1, 2, 4, 8};
    for (int c = 0; c < 4 && st == CD_OK; ++c) {
        const int W = cand[c];
        if (W > wmax) break;
        float ms = 0.f;
        if (cudaEventRecord(t0, s) != cudaSuccess) { st = CD_ECUDA; break; }
        st = enqueue(*b, W, s);
        if (st != CD_OK) break;
        if (cudaEventRecord(t1, s) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess) {
            st = CD_ECUDA;
            break;
        }
        b->ms_tried[c] = ms;
        if (ms < best) {
            best = ms;
            b->width = W;
        }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != CD_OK) {
        destroy(b);
        return st;
    }
    // capture the chosen fan-out into one graph
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        destroy(b);
        set_error("stream capture could not start (is the stream already capturing?)");
        return CD_ECUDA;
    }
    st = enqueue(*b, b->width, s);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    if (st != CD_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        destroy(b);
        if (st == CD_OK) set_error("stream capture failed: %s", cudaGetErrorString(ce));
        return st != CD_OK ? st : CD_ECUDA;
    }
    b->graph = g;
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
        destroy(b);
        set_error("graph instantiation failed");
        return CD_ECUDA;
    }
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        cudaGraphGetNodes(g, nodes.data(), &nn);
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

cd_status cd_batch_run(cd_batch b, void *stream)
{
    if (!b) {
        set_error("batch is NULL");
        return CD_EINVAL;
    }
    LaunchScope ls(CD_K_OTHER, (cudaStream_t)stream);
    CD_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
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
