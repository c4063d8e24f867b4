// Internal declarations of libcolden: handle layouts, error plumbing, Morton
// helpers and the kernel launchers each translation unit provides.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>

#include "../../include/colden.h"

#define CD_MAXL 16          // deepest level a tree may have
#define CD_STENCIL 216      // 6 x 6 x 6 level-l cells around a level-(l-1) ancestor
#define CD_CONE_RINGS 4     // sub-ray pattern of CD_MODE_CONE: rings of equal solid angle ...
#define CD_CONE_AZ 8        // ... times azimuths per ring
#define CD_MAXDIR 768       // the leaf kernel stages 64 * n_dir floats in shared memory

namespace cd {

void set_error(const char *fmt, ...);

// ---- bounds-checked builds (COLDEN_CHECKED) ---------------------------------
// Built with -DCOLDEN_CHECKED (libcolden_checked.so), the gathers of the shell
// and leaf kernels test each index against the extent of what they read or
// write: in_bounds(i, n, site) is true for 0 <= i < n; otherwise it records
// (site, i) in this translation unit's check word (the first failure wins),
// returns false and the caller skips the access (or issues an empty copy).
// Nothing traps.  cd_checked_status collects and clears every unit's word.
// In the normal build in_bounds is the constant true and the checks vanish.
#ifdef COLDEN_CHECKED
struct CheckWord {
    int site;
    int pad;
    long long index;
};
using CheckReader = bool (*)(CheckWord *);
int register_check_reader(CheckReader r);   // api.cu
namespace {
__device__ CheckWord g_check_word;
__device__ __noinline__ bool check_fail(long long i, int site)
{
    if (atomicCAS(&g_check_word.site, 0, site) == 0) *(volatile long long *)&g_check_word.index = i;
    return false;
}
__device__ __forceinline__ bool in_bounds(long long i, long long n, int site)
{
    return (i >= 0 && i < n) ? true : check_fail(i, site);
}
bool read_check_word(CheckWord *w)
{
    const CheckWord zero = {};
    return cudaMemcpyFromSymbol(w, g_check_word, sizeof(CheckWord)) == cudaSuccess &&
           cudaMemcpyToSymbol(g_check_word, &zero, sizeof(CheckWord)) == cudaSuccess;
}
const int g_check_registered = register_check_reader(read_check_word);
}  // namespace
#else
__device__ __forceinline__ constexpr bool in_bounds(long long, long long, int) { return true; }
#endif
// check sites (cd_checked_status reports the code)
enum {
    kCheckProbe = 1,
    kCheckFp32Region = 11, kCheckFp32Out = 12, kCheckFp32Prefix = 13,
    kCheckTcBrick = 21,
    kCheckLeafTcIn = 31, kCheckLeafTcOut = 32,
    kCheckLeafIn = 41,
    kCheckListLevel = 51,
};

// Shared-memory staging of the shell kernels: the density region read by
// table t is a cube of side kRegionSide[t] level-(k-t+1) cells (6 + 2 x the
// ancestors per axis of one CTA) starting at kRegionBase[t].
__host__ __device__ constexpr int region_side(int t) { return t == 1 ? 12 : t == 2 ? 8 : t == 3 ? 6 : 0; }
__host__ __device__ constexpr int region_base(int t) { return t == 2 ? 12 * 12 * 12 : t == 3 ? 12 * 12 * 12 + 8 * 8 * 8 : 0; }
constexpr int kRegionTotal = 12 * 12 * 12 + 8 * 8 * 8 + 6 * 6 * 6;

#define CD_CUDA(call)                                                                  \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess) {                                                       \
            ::cd::set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                  \
                            cudaGetErrorString(e_));                                   \
            return CD_ECUDA;                                                           \
        }                                                                              \
    } while (0)

#define CD_CHECK_LAUNCH()                                                              \
    do {                                                                               \
        cudaError_t e_ = cudaGetLastError();                                           \
        if (e_ != cudaSuccess) {                                                       \
            ::cd::set_error("%s:%d kernel launch: %s", __FILE__, __LINE__,             \
                            cudaGetErrorString(e_));                                   \
            return CD_ECUDA;                                                           \
        }                                                                              \
    } while (0)

// ---- Morton (octant bits x = 1, y = 2, z = 4) --------------------------------

__host__ __device__ inline uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1fffff;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__host__ __device__ inline uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
    x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
    x = (x ^ (x >> 8)) & 0x1f0000ff0000ffull;
    x = (x ^ (x >> 16)) & 0x1f00000000ffffull;
    x = (x ^ (x >> 32)) & 0x1fffff;
    return (uint32_t)x;
}

__host__ __device__ inline uint64_t morton3(uint32_t x, uint32_t y, uint32_t z)
{
    return spread3(x) | (spread3(y) << 1) | (spread3(z) << 2);
}

// ---- handles -----------------------------------------------------------------

struct Workspace {
    int ndir = 0;
    float *S[CD_MAXL + 1] = {};  // prefix sums of the far shells, Morton order, [8^k][ndir]
    float *E = nullptr;          // external column of every oct, Morton order, [n_oct][ndir]
};

// The learned form's per-level sums (learned.cu): every shell kept apart.
struct LevelSums {
    int ndir = 0;
    int precision = -1;                       // CD_FP32, or CD_BF16 (tensor cores for levels >= 4)
    int64_t geom_uid = 0, rho_version = -1;   // what the sums were computed for
    float *C[CD_MAXL + 1] = {};   // shell of level k-2 seen from level-k cells, no prefix, [8^k][ndir]
    float *Et[4] = {};            // oct level, table t alone (shell of level L-t), [n_oct][ndir]
    float *x = nullptr, *n_tree = nullptr, *delta = nullptr;   // chunk buffers of the FP32 learned path
    int64_t rows = 0;
};

// A sparse set of receiving cells of one level (AMR meshes), arranged for the
// tensor-core shell contraction: the receivers' parents grouped by class
// (the low six Morton bits), and the tiles over those rows.
struct TcList {
    int64_t n_recv = 0;          // receivers (output rows 0 .. n_recv-1)
    int64_t nrows = 0;           // distinct parents
    int64_t ntiles = 0;
    uint64_t *key = nullptr;     // (device) [nrows] parent Morton keys, grouped by class
    int32_t *out = nullptr;      // (device) [nrows][8] output row of child o, -1 if not a receiver
    int4 *tiles = nullptr;       // (device) [ntiles] {class, first row, rows, half}
    int32_t *recv_parent = nullptr;   // (device, borrowed) prefix row of each receiver, or NULL
};


}  // namespace cd

struct cd_tree_s {
    int L = 0;                          // finest leaf level
    int base = 0;                       // base (coarsest leaf) level
    int amr = 0;
    double box_cm = 0;
    int64_t n_leaf = 0;
    int64_t n_oct = 0;                  // leaf-bearing octs (uniform: 8^(L-1))
    float *rho_lvl[CD_MAXL + 1] = {};   // dense row-major volume means, levels 0..L-1
    __nv_bfloat16 *rho_brick[CD_MAXL + 1] = {};  // BF16 copies in brick order (tensor path)
    float *rho_leaf = nullptr;          // leaf densities, Morton order
    cd::Workspace ws;
    cd::LevelSums lv;
    int64_t rho_version = 0;            // bumped by every density update
    int dev = 0;
    // AMR meshes (amr != 0); see amr.cu
    int64_t n_ref[CD_MAXL + 1] = {};      // refined cells of level k
    uint64_t *ref_key[CD_MAXL + 1] = {};  // their sorted Morton keys (device)
    int32_t *ref_parent[CD_MAXL + 1] = {};// index of each one's parent in level k-1 (device)
    int64_t oct_begin[CD_MAXL + 2] = {};  // leaf-bearing octs of level k: [oct_begin[k], oct_begin[k+1])
    uint64_t *oct_key = nullptr;          // (device) Morton key of every oct at its level
    int32_t *oct_parent = nullptr;        // (device) index of the oct's parent among the refined cells
    int32_t *oct_leaf = nullptr;          // (device) [n_oct][8] output row of child o, -1 if refined
    cd::TcList tc_ref[CD_MAXL + 1];       // tensor-core lists: refined cells of level k (far-shell prefixes)
    cd::TcList tc_oct[CD_MAXL + 1];       // tensor-core lists: leaf-bearing octs of level k
    float *oct_rho8 = nullptr;            // (device) [n_oct][8] volume-mean density of child o
    int32_t *leaf_slot = nullptr;         // (device) output order: 8 oct + child of the leaf (-1: no oct)
    int32_t *ref8 = nullptr;              // (device) the slots 8 oct + child of the refined children
    int64_t n_ref8 = 0;
    // The finest dense level lf = L-1 is filled only where it is read (when lf >
    // base): leaves and refined cells of lf, and the children of the level-(lf-1)
    // cells around the parents of the octs of level lf (their shells' stencils)
    int sparse_finest = 0;
    int64_t n_deep = 0;
    uint64_t *deep_key = nullptr;         // (device) those level-(lf-1) cells, sorted Morton keys
    int8_t *deep_paint = nullptr;         // (device) 1: not refined, its children take its value
    // The level below it, lm = lf-1, likewise when lm > base: leaves, refined
    // cells, and the children of the level-(lm-1) cells around the parents of
    // the octs of level lm and the grandparents of the octs of level lf (the
    // stencils of their shells, in-situ walks and of the deep cells' parents);
    // the rest of level lm holds NaN from the build on, so that a read outside
    // the painted part cannot pass unnoticed
    int sparse_mid = 0;
    int64_t n_mid = 0;
    uint64_t *mid_key = nullptr;          // (device) those level-(lm-1) cells, sorted Morton keys
    int8_t *mid_paint = nullptr;          // (device) 1: not refined, its children take its value
    uint64_t *leaf_key = nullptr;         // (device) output order: Morton key at the leaf's level
    int8_t *leaf_lvl = nullptr;           // (device) output order: level
    int64_t *leaf_src = nullptr;          // (device) output order: index in the caller's leaf arrays
    int8_t *leaf_level_h = nullptr;       // host copies of the output order
    int32_t *leaf_ijk_h = nullptr;
    int64_t *leaf_src_h = nullptr;
    // Two side streams of one evaluation: the steps that do not depend on one
    // another (the far-shell prefix chain, the oct shells of each level, the
    // leaves of each level) run on them concurrently, ordered by events and
    // joined back into the caller's stream before the call returns
    cudaStream_t side[2] = {};
    cudaEvent_t ev_fork = nullptr, ev_done[2] = {};
    // cd_column_density_host: device staging of the host densities and
    // outputs, the copy stream and one event per leaf chunk (api.cu)
    struct HostIO {
        float *rho = nullptr, *nh = nullptr, *av = nullptr, *sh = nullptr;
        int64_t nh_elems = 0;                 // n_h / a_v staging size (n_leaf x n_dir)
        cudaStream_t copy = nullptr;
        cudaEvent_t ev[9] = {};
    } hio;
    cudaEvent_t ev_S[CD_MAXL + 1] = {}, ev_E[CD_MAXL + 1] = {};
    // live cd_batch objects whose graph holds this tree's scratch pointers:
    // while it is non-zero an evaluation must not reallocate the scratch
    int batch_refs = 0;
};

struct cd_geom_s {
    int64_t uid = 0;                    // process-unique id (learned.cu caches per geometry)
    int n_dir = 0;
    int mode = 0;
    // how the direction set was made (cd_geom_save records it): scheme, p0,
    // p1 and, for CD_DIRS_CUSTOM, the caller's vectors as given
    int scheme = 0, p0 = 0, p1 = 0, n_custom = 0;
    double *custom = nullptr;
    double *dirs_host = nullptr;        // n_dir x 3
    double *dirs_dev = nullptr;
    // the rays the weights are averaged over: n_sub per direction, [nd][n_sub][3];
    // one (the direction itself, rays_dev == dirs_dev) unless the mode is CD_MODE_CONE
    int n_sub = 1;
    double *rays_host = nullptr;
    double *rays_dev = nullptr;
    // sparse FP32 shell tables, t = 1..3 (index 0 unused): entry e of (cfg, d)
    // at tab[t][(cfg * maxe + e) * nd + d] = {offset in the staged region of
    // table t, weight bits}; cmax[t][cfg] = largest non-zero count over d;
    // maxe = largest count over every table, configuration and direction
    int maxe = 0;
    int2 *tab[4] = {};
    int *cmax[4] = {};
    float *kloc = nullptr;              // [8 t][8 s][nd], units of dx
    // BF16 B operands for the tensor-core contraction (see colden_tc.cu)
    __nv_bfloat16 *wb = nullptr;
    size_t wb_bytes = 0;
    int dev = 0;
};

namespace cd {

// stats.cu: counts (and optionally times) one kernel launch on stream s for
// the lifetime of the scope; construct it right before the launch.  flops:
// the dense tensor-core work the launch issues (2 M N K per MMA, padding
// included), 0 for CUDA-core kernels.
class LaunchScope {
  public:
    LaunchScope(int kind, cudaStream_t s, double flops = 0.0);
    ~LaunchScope();
    LaunchScope(const LaunchScope &) = delete;
    LaunchScope &operator=(const LaunchScope &) = delete;

  private:
    int kind_;
    cudaStream_t s_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// stats.cu: an NVTX range (nvtxRangePushA / nvtxRangePop) for the lifetime of
// the scope; a no-op unless a tool (nsys, an NVTX injection library) is
// attached.  Every LaunchScope also opens one named after its kernel kind
// ("colden:shell", ...); the entry points open "colden:<entry point>".
class NvtxRange {
  public:
    explicit NvtxRange(const char *name);
    ~NvtxRange();
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// learned.cu: frees the tree's LevelSums
void free_level_sums(cd_tree t);

// stats.cu: per-launch timing is on (cd_stats_reset(1))
bool stats_timing();
// Frees library-owned device memory and advances a process-wide count, so
// that a captured evaluation graph (cd_eval_graph) refuses to replay once a
// buffer it may reference has been freed or reallocated.
cudaError_t lib_free(void *p);
int64_t free_generation();
// launch counters and flops by kind (CD_K_COUNT entries): a copy, and adding
// sign x counts (a graph replay adds what its capture recorded)
void stats_snapshot(int64_t *count, double *flops);
void stats_add(const int64_t *count, const double *flops, int sign = 1);

// api.cu: the side streams of a tree.  Fork makes both side streams wait for
// the work enqueued on s so far; join() (or the destructor, on an early
// return) makes s wait for everything enqueued on them since.  While
// per-launch timing is on, side(i) is s itself: the evaluation runs in
// order, so that each launch's events time that launch alone.
class SideFork {
  public:
    SideFork(cd_tree t, cudaStream_t s);
    ~SideFork();
    SideFork(const SideFork &) = delete;
    SideFork &operator=(const SideFork &) = delete;
    cd_status status() const { return st_; }   // CD_OK once both side streams are ordered after s
    cudaStream_t side(int i) const;
    bool serial() const { return serial_; }
    cd_status join();

  private:
    cd_tree t_;
    cudaStream_t s_;
    cd_status st_ = CD_OK;
    bool joined_ = false;
    bool serial_ = false;
};

// api.cu: CD_EINVAL (with a message) when the tree's scratch, sized for
// ws.ndir directions, would have to be reallocated for nd while a batch graph
// holds its pointers
cd_status check_workspace_pinned(cd_tree t, int nd);

// tree.cu
cd_status restrict_uniform(cd_tree t, const float *rho_dev, cudaStream_t s);
// levels top-1 .. 0 as means of top .. 1, then BF16 bricks of levels 1 .. top
cd_status restrict_dense(cd_tree t, int top, cudaStream_t s);

// amr.cu
void free_tc_lists(cd_tree t);
cd_status build_amr(cd_tree t, int base, int lmax, int64_t n, const int8_t *level, const int32_t *ijk);
cd_status update_amr(cd_tree t, const float *rho_dev, cudaStream_t s);
cd_status column_density_amr(cd_tree t, cd_geom g, const cd_opts &opts, float *n_h, float *a_v, float *shield,
                             cudaStream_t s);
// Batched FP32 list shells (cd_batch): the far shells of level 3 (table 3)
// of a tree whose level 3 is complete, into ws.S[3], over the 512 Morton keys
// keys512; many such lists run as one launch (blockIdx.y = list).
size_t list_job_bytes();
void list_job_fill_far3(cd_tree t, cd_geom g, const uint64_t *keys512, void *dst);
cd_status launch_list_batch(const void *jobs, int n_jobs, int64_t max_elems, cudaStream_t s);

// insitu.cu: the external column of n octs of level k (keys NULL: every oct of
// a uniform tree), every shell seen from the oct centre (§4.3)
cd_status launch_insitu(cd_tree t, cd_geom g, int k, int64_t n, const uint64_t *keys, float *out, cudaStream_t s);

// geometry.cu
int make_directions(int scheme, int p0, int p1, const double *custom, int n_custom, double *out);
// the CD_CONE_RINGS * CD_CONE_AZ sub-rays of each of the nd directions, out[nd][n_sub][3]
void make_cone_rays(const double *dirs, int nd, double *out);
cd_status build_geometry_tables(cd_geom g, cudaStream_t s);

// colden_fp32.cu
struct ExtLaunch {
    int k;                    // level of the cells that receive the sum
    int nd;
    int tmask;                // bit (t-1): table t contributes (shell level k - t + 1)
    const float *rho[4];      // dense level arrays of the shell level of each table
    float dx[4];              // dx of that shell level, cm
    const float *prefix_in;   // S_{k-1} (Morton) or NULL
    float *out;               // Morton [8^k][nd], or [n_recv][nd] with a list
    const TcList *list;       // tensor-core form only: receivers of an AMR level (NULL: every cell of level k)
    int tiles_per_cta;        // tensor-core form: 0 = persistent CTAs (two per SM); n = one CTA per n tiles
};
cd_status launch_ext_fp32(const ExtLaunch &a, cd_geom g, cudaStream_t s);

struct LeafLaunch {
    int64_t n_oct;
    int nd;
    float dx_leaf;
    float av_per_nh, shield_k;
    const float *rho_leaf;    // Morton, 8 per oct
    const float *E;           // [n_oct][nd] or NULL: shells l0-3 .. l0-1 of every oct
    const float *Sp;          // [n_oct / 8][nd] or NULL: far shells shared by the 8 octs of a parent
    const float *kloc;        // [8][8][nd]
    float *n_h, *a_v, *shield;
    // AMR list mode (leaf_tc only): oleaf[8 o + t] is the output row of child t
    // of oct o (-1: refined); rho_leaf then holds 8 densities per oct (in list
    // order).  The parent prefix is either already in E (Sp NULL) or row
    // oparent[o] of Sp (n_sp rows); oparent is non-decreasing along the list,
    // so a tile's parent rows are one contiguous span of Sp
    const int32_t *oleaf;
    int64_t n_rows;           // list mode: rows of n_h / a_v / shield (the tree's leaves; bounds checks)
    const int32_t *oparent;   // list mode with Sp: [n_oct] parent row of each oct
    int64_t n_sp;             // list mode with Sp: rows of Sp
};
cd_status launch_leaf(const LeafLaunch &a, cudaStream_t s);

// leaf.cu: CD_ETIMEOUT if a leaf kernel gave up a bounded wait (clears it)
cd_status leaf_fault_check();

// leaf_tc.cu: the BF16 form's leaf kernel with the local term on the tensor
// cores; CD_EUNSUPPORTED (no error text) when the sizes do not fit it
cd_status launch_leaf_tc(const LeafLaunch &a, cudaStream_t s);
cd_status leaf_tc_fault_check();
// Batched leaf jobs (batch.cu): one job is one launch_leaf_tc's worth (a
// uniform tree's leaves, or an AMR level's oct list); all jobs of one launch
// share the direction table (nd, kloc) and the output form (which of Sp,
// n_h, A_V and the screening factor the rows use, list or Morton tiles: the
// kernel branches on it as a launch constant).  tile counts as tc_job_fill.
size_t leaf_tc_job_bytes();
int64_t leaf_tc_job_fill(const LeafLaunch &a, void *dst);
int leaf_tc_job_form(const void *job);
double leaf_tc_job_flops(const void *job);
cd_status launch_leaf_tc_batch(const void *jobs, const int2 *tile_ref, int64_t total, int nd, const float *kloc,
                               int form, double flops, cudaStream_t s);
// cd_debug_wait_polls: poll limit of the BF16 leaf kernel's pipeline waits (< 0: default)
void set_leaf_tc_wait_polls(int64_t polls);
// cd_debug_leaf_span: widest parent span a list tile stages as one copy (< 0: default 16)
void set_leaf_tc_span_max(int rows);

// colden_tc.cu: BF16 tensor-core shell contraction for receiving levels >= 4
bool tc_supported(int nd);
cd_status build_tc_tables(cd_geom g, cudaStream_t s);
cd_status launch_ext_tc(const ExtLaunch &a, const __nv_bfloat16 *const *brick, cd_geom g, cudaStream_t s);
cd_status tc_fault_check();
// Batched shell jobs (batch.cu): one job is one launch's worth of
// launch_ext_tc (a level, a run of tables, uniform or list tiles), optionally
// with tiles covering all 8 children (N = 8 nd, nd <= 32) and the prefix rows
// S_{k-1} added in the epilogue once job wait_job is complete.
struct TcJobDesc {
    ExtLaunch a;
    int full;
    const float *prefix;         // or NULL
    const int32_t *prefix_row;   // list jobs: prefix row of each output row
    int wait_job, wait_count;
};
size_t tc_job_bytes();
// writes the job's kernel arguments to dst (tc_job_bytes() bytes of host
// memory); returns its tile count, or -1 if the tensor-core form cannot serve it
int64_t tc_job_fill(const TcJobDesc &d, const __nv_bfloat16 *const *brick, cd_geom g, void *dst);
double tc_job_flops(const void *job);
uint32_t tc_job_bstage(const void *job);
// marks a job that another job waits on (its tiles count themselves done)
void tc_job_set_signal(void *job);
// one persistent launch over `total` tiles of the device job array
// (tile_ref[g] = {job, tile within the job} of global tile g)
// (*ctas_used: the CTAs per SM launched, at most ctas_per_sm and what fits an SM)
// (*claim: the work counter, zero at the launch)
cd_status launch_tc_batch(const void *jobs, const int2 *tile_ref, int64_t total, int *done, int *claim,
                          uint32_t bstage_max, int ctas_per_sm, double flops, cudaStream_t s, int *ctas_used = nullptr);
// out[i][d] += prefix[parent[i]][d] for n = rows * nd elements
cd_status launch_add_parent_list(float *out, const float *prefix, const int32_t *parent, int nd, int64_t rows,
                                 cudaStream_t s);

}  // namespace cd
