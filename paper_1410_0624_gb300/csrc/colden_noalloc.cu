// cd_column_density_noalloc: the FP32 column-density evaluation with its
// scratch (the per-level partial sums S_k and the per-oct external column E)
// placed in a fixed, file-scope device array instead of memory the library
// allocates.
//
// Who needs it: simulation codes that reserve all their device memory once at
// start-up (a fixed budget shared with the hydro solver) and must not allocate
// or free device memory inside the time-step loop, for instance because
// allocation calls may synchronise the device and stall their asynchronous
// step loop.  They build the tree and the geometry tables once during set-up
// and then call this entry point every step.
//
// The scratch array is 16 MiB.  Every GPU that loads the library holds it
// until the process exits.  The module holding it is loaded on a device the
// first time its address is looked up there (lazy module loading), which is
// the first call of this entry point on that device, outputs or not: callers
// make that call during set-up.
#include <mutex>

#include "common.cuh"

namespace cd {
namespace {

constexpr size_t kScratchFloats = (size_t)4 << 20;   // 16 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_scratch[kScratchFloats];

std::mutex g_mu;
float *g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device, looked up once per device.
cd_status scratch_address(float **out)
{
    int dev = 0;
    CD_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("device ordinal %d beyond the %d this entry point tracks", dev, kMaxDevices);
        return CD_EUNSUPPORTED;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p) {
            set_error("cudaGetSymbolAddress(g_scratch) failed: %s", cudaGetErrorString(e));
            return CD_ECUDA;
        }
        g_scratch_addr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_addr[dev];
    return CD_OK;
}

size_t round_up(size_t n) { return (n + 63) & ~(size_t)63; }   // 256-byte sub-buffers

}  // namespace
}  // namespace cd

using namespace cd;

extern "C" cd_status cd_column_density_noalloc(cd_tree tree, cd_geom geom, const cd_opts *opts_in, float *n_h,
                                               float *a_v, float *shield, void *stream)
{
    if (!tree || !geom) {
        set_error("tree or geometry is NULL");
        return CD_EINVAL;
    }
    cd_opts opts;
    if (opts_in) opts = *opts_in; else cd_opts_default(&opts);
    if (opts.precision != CD_FP32) {
        set_error("cd_column_density_noalloc computes in FP32 only");
        return CD_EUNSUPPORTED;
    }
    if (opts.net || tree->amr || geom->mode == CD_MODE_INSITU) {
        set_error("cd_column_density_noalloc serves uniform trees in the precalculated form without a learned correction");
        return CD_EUNSUPPORTED;
    }
    // the lookup loads this file's module (and its array) on the device, so a
    // set-up call with no outputs already takes the 16 MiB
    float *base = nullptr;
    cd_status st = scratch_address(&base);
    if (st != CD_OK) return st;
    if (!n_h && !a_v && !shield) return CD_OK;
    const int nd = geom->n_dir, L = tree->L;

    // scratch layout: S_3 .. S_{L-2}, then E
    size_t off[CD_MAXL + 2] = {};
    size_t need = 0;
    for (int k = 3; k <= L - 2; ++k) {
        off[k] = need;
        need += round_up(((size_t)1 << (3 * k)) * nd);
    }
    const size_t offE = need;
    if (L >= 2) need += round_up((size_t)tree->n_oct * nd);
    if (need > kScratchFloats) {
        set_error("this tree needs %zu scratch floats (%.1f MiB) but the fixed scratch holds %zu (16 MiB); "
                  "use cd_column_density or fewer levels / directions",
                  need, need * 4.0 / (1 << 20), kScratchFloats);
        return CD_EINVAL;
    }
    // Every scratch element the kernels read is written earlier in this call,
    // so nothing needs clearing between calls.
    cudaStream_t s = (cudaStream_t)stream;
    const auto dx = [&](int l) { return (float)(tree->box_cm / (double)((int64_t)1 << l)); };
    for (int k = 3; k <= L - 2; ++k) {
        ExtLaunch a = {};
        a.k = k;
        a.nd = nd;
        a.tmask = 4;
        a.rho[3] = tree->rho_lvl[k - 2];
        a.dx[3] = dx(k - 2);
        a.prefix_in = (k > 3) ? base + off[k - 1] : nullptr;
        a.out = base + off[k];
        if ((st = launch_ext_fp32(a, geom, s)) != CD_OK) return st;
    }
    if (L >= 2) {
        ExtLaunch a = {};
        const int k = L - 1;
        a.k = k;
        a.nd = nd;
        for (int t = 1; t <= 3 && t <= k; ++t) {
            a.tmask |= 1 << (t - 1);
            a.rho[t] = tree->rho_lvl[k - t + 1];
            a.dx[t] = dx(k - t + 1);
        }
        a.prefix_in = nullptr;   // the leaf kernel adds S_{L-2}[parent]
        a.out = base + offE;
        if ((st = launch_ext_fp32(a, geom, s)) != CD_OK) return st;
    }
    LeafLaunch b = {};
    b.n_oct = tree->n_oct;
    b.nd = nd;
    b.dx_leaf = dx(L);
    b.av_per_nh = (float)opts.av_per_nh;
    b.shield_k = (float)opts.shield_k;
    b.rho_leaf = tree->rho_leaf;
    b.E = (L >= 2) ? base + offE : nullptr;
    b.Sp = (L - 2 >= 3) ? base + off[L - 2] : nullptr;
    b.kloc = geom->kloc;
    b.n_h = n_h;
    b.a_v = a_v;
    b.shield = shield;
    return launch_leaf(b, s);
}
