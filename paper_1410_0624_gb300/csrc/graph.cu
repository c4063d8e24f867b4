// One evaluation step captured as a CUDA graph (cd_eval_graph_*): the density
// update (cd_tree_update from a device buffer) and cd_column_density are
// enqueued once on a private stream under capture, with the side-stream fork
// and join of the evaluation, and every launch replays the recorded kernels
// on the caller's stream.  A replay costs one graph launch instead of one
// host call per kernel, and the GPU runs the dependent launches back to back.
//
// The graph holds raw device pointers of the tree's, the geometry's and the
// network's buffers as they were at capture.  Any free of library-owned
// device memory advances a process-wide count (lib_free), and a launch after
// such a free is refused, so a replay can never touch a buffer that a later
// call reallocated.  Host-side state that the capture baked in is checked
// the same way: the network's parameters and trusted range.  The learned form
// skips its per-level sums when the host records them as current, so a
// learned graph must hold the density update: every replay then recomputes
// the sums it reads.
#include <cstring>

#include "learned.cuh"

struct cd_eval_graph_s {
    cudaGraphExec_t exec = nullptr;
    int dev = 0;
    int64_t gen = 0;                   // free_generation() at capture
    cd_net net = nullptr;
    int64_t net_version = 0;
    float dlo = 0.f, dhi = 0.f;
    int64_t count[CD_K_COUNT] = {};    // kernels and flops one replay launches, by kind
    double flops[CD_K_COUNT] = {};
};

using namespace cd;

extern "C" {

cd_status cd_eval_graph_create(cd_tree tree, cd_geom geom, const cd_opts *opts, const float *rho, float *n_h,
                               float *a_v, float *shield, void *stream, cd_eval_graph *out)
{
    NvtxRange nvtx_range("colden:eval_graph_create");
    if (!out) {
        set_error("out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    if (!tree || !geom) {
        set_error("tree or geometry is NULL");
        return CD_EINVAL;
    }
    int dev = 0;
    CD_CUDA(cudaGetDevice(&dev));
    if (dev != tree->dev || dev != geom->dev) {
        set_error("the current device (%d) is not the tree's (%d) or the geometry's (%d)", dev, tree->dev, geom->dev);
        return CD_EINVAL;
    }
    if (opts && opts->net && !rho) {
        set_error("a learned graph must hold the density update (rho != NULL)");
        return CD_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    CD_CUDA(cudaStreamIsCapturing(s, &cap));
    if (cap != cudaStreamCaptureStatusNone) {
        set_error("the stream is capturing: the graph's eager first step cannot run inside a capture");
        return CD_EINVAL;
    }
    // one eager step first: every buffer that the library allocates on first
    // use exists before the capture (no allocation may happen inside it)
    cd_status st = CD_OK;
    if (rho && (st = cd_tree_update(tree, rho, 1, stream)) != CD_OK) return st;
    if ((st = cd_column_density(tree, geom, opts, n_h, a_v, shield, stream)) != CD_OK) return st;
    CD_CUDA(cudaStreamSynchronize(s));

    cd_eval_graph g = new cd_eval_graph_s();
    g->dev = dev;
    g->net = opts ? (cd_net)opts->net : nullptr;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
        delete g;
        set_error("cannot create the capture stream: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    g->gen = free_generation();
    int64_t c0[CD_K_COUNT];
    double f0[CD_K_COUNT];
    stats_snapshot(c0, f0);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (rho) st = cd_tree_update(tree, rho, 1, cs);
        if (st == CD_OK) st = cd_column_density(tree, geom, opts, n_h, a_v, shield, cs);
        e = cudaStreamEndCapture(cs, &graph);   // ends the capture whatever happened inside it
    }
    cudaStreamDestroy(cs);
    int64_t c1[CD_K_COUNT];
    double f1[CD_K_COUNT];
    stats_snapshot(c1, f1);
    if (st == CD_OK && e == cudaSuccess && free_generation() != g->gen) {
        set_error("a library buffer was freed during the capture");
        st = CD_ECUDA;
    }
    if (st == CD_OK && e == cudaSuccess) e = cudaGraphInstantiate(&g->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != CD_OK || e != cudaSuccess) {
        if (st == CD_OK) {
            set_error("graph capture failed: %s", cudaGetErrorString(e));
            st = CD_ECUDA;
        }
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        delete g;
        return st;
    }
    for (int k = 0; k < CD_K_COUNT; ++k) {
        g->count[k] = c1[k] - c0[k];
        g->flops[k] = f1[k] - f0[k];
    }
    // the capture advanced the host-side counters without running anything
    stats_add(g->count, g->flops, -1);
    if (g->net) {
        g->net_version = g->net->version;
        g->dlo = g->net->dlo;
        g->dhi = g->net->dhi;
    }
    *out = g;
    return CD_OK;
}

cd_status cd_eval_graph_launch(cd_eval_graph g, void *stream)
{
    if (!g) {
        set_error("graph is NULL");
        return CD_EINVAL;
    }
    // checked before anything the graph names is read: a freed tree, geometry
    // or network advanced the count
    if (free_generation() != g->gen) {
        set_error("a library buffer was freed or reallocated since the capture (a tree, geometry or network "
                  "freed, or a workspace grown by another call): create the graph again");
        return CD_EINVAL;
    }
    if (g->net && (g->net->version != g->net_version || g->net->dlo != g->dlo || g->net->dhi != g->dhi)) {
        set_error("the network's parameters or trusted range changed since the capture: create the graph again");
        return CD_EINVAL;
    }
    int dev = 0;
    CD_CUDA(cudaGetDevice(&dev));
    if (dev != g->dev) {
        set_error("the graph belongs to device %d, the current device is %d", g->dev, dev);
        return CD_EINVAL;
    }
    CD_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    stats_add(g->count, g->flops);
    return CD_OK;
}

cd_status cd_eval_graph_info(cd_eval_graph g, int64_t *kernels)
{
    if (!g) {
        set_error("graph is NULL");
        return CD_EINVAL;
    }
    int64_t n = 0;
    for (int k = 0; k < CD_K_COUNT; ++k) n += g->count[k];
    if (kernels) *kernels = n;
    return CD_OK;
}

void cd_eval_graph_free(cd_eval_graph g)
{
    if (!g) return;
    if (g->exec) {
        cudaDeviceSynchronize();   // no replay may still be running
        cudaGraphExecDestroy(g->exec);
    }
    delete g;
}

}  // extern "C"
