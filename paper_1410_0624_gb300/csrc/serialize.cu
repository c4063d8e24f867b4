// Checkpoint images of a tree and of a geometry (cd_tree_save/load,
// cd_geom_save/load, cd_geom_hash).  The paper has no file format: a
// simulation restarts from its own outputs.  These images let a caller
// store the mesh, its densities and the direction set with the run and get
// the same columns back after a restart.
//
// Both images are flat little-endian byte strings (fields at fixed offsets,
// no padding) ending in the FNV-1a 64-bit hash of every byte before it
// (Fowler, Noll and Vo: offset basis 14695981039346656037, prime
// 1099511628211, one byte at a time: h ^= byte, h *= prime).
//
// Tree image:
//   "CDTREE01" | int32 amr, base, L | float64 box_cm | int64 n_leaf |
//   int8 level[n] | int32 ijk[3 n] | float32 rho[n] | uint64 hash
// leaves in output (Morton) order with the densities of the last update.
//
// Geometry image:
//   "CDGEOM01" | int32 scheme, p0, p1, mode, n_dir, n_custom |
//   float64 custom[3 n_custom] | float64 dirs[3 n_dir] | uint64 dirs_hash |
//   uint64 table_hash | uint64 hash
// A geometry is loaded by building it again from its recorded construction;
// the rebuilt directions must equal the stored ones bit for bit and the
// rebuilt tables must have the stored table hash, so an image from a library
// whose direction sets or tables differ is refused instead of giving other
// columns.
#include <string.h>

#include <vector>

#include "common.cuh"

namespace cd {
namespace {

constexpr uint64_t kFnvBasis = 14695981039346656037ull, kFnvPrime = 1099511628211ull;

uint64_t fnv(const void *p, size_t n, uint64_t h = kFnvBasis)
{
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= kFnvPrime;
    }
    return h;
}

// byte writer / reader at running offsets; the writer only counts when dst is NULL
struct Out {
    unsigned char *dst;
    size_t n = 0;
    void put(const void *p, size_t k)
    {
        if (dst) memcpy(dst + n, p, k);
        n += k;
    }
    template <class T>
    void val(T v) { put(&v, sizeof(T)); }
};

struct In {
    const unsigned char *src;
    size_t size, n = 0;
    bool ok = true;
    void get(void *p, size_t k)
    {
        if (!ok || k > size - n) {
            ok = false;
            return;
        }
        memcpy(p, src + n, k);
        n += k;
    }
    template <class T>
    T val()
    {
        T v{};
        get(&v, sizeof(T));
        return v;
    }
};

const char kTreeMagic[8] = {'C', 'D', 'T', 'R', 'E', 'E', '0', '1'};
const char kGeomMagic[8] = {'C', 'D', 'G', 'E', 'O', 'M', '0', '1'};

// hash of the direction set and mode (the identity of a geometry)
uint64_t dirs_hash(const cd_geom_s *g)
{
    uint64_t h = fnv(&g->mode, sizeof(int));
    h = fnv(&g->n_dir, sizeof(int), h);
    return fnv(g->dirs_host, sizeof(double) * 3 * g->n_dir, h);
}

// hash of every table the evaluation reads: Kloc, the sparse FP32 shell
// tables with their per-configuration counts, the BF16 operand images
cd_status table_hash(const cd_geom_s *g, uint64_t *out)
{
    const int nd = g->n_dir;
    std::vector<unsigned char> buf;
    auto add = [&](const void *dev, size_t bytes) {
        if (!dev || !bytes) return true;
        const size_t at = buf.size();
        buf.resize(at + bytes);
        return cudaMemcpy(buf.data() + at, dev, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    bool ok = add(g->kloc, sizeof(float) * 64 * nd);
    for (int t = 1; t <= 3 && ok; ++t) {
        const size_t ncfg = (size_t)1 << (3 * t);
        ok = add(g->tab[t], ncfg * g->maxe * nd * sizeof(int2)) && add(g->cmax[t], ncfg * sizeof(int));
    }
    ok = ok && add(g->wb, g->wb_bytes);
    if (!ok) {
        set_error("reading the geometry tables failed: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    uint64_t h = fnv(&g->maxe, sizeof(int));
    *out = fnv(buf.data(), buf.size(), h);
    return CD_OK;
}

cd_status geom_image(const cd_geom_s *g, unsigned char *dst, size_t *size, uint64_t th)
{
    Out o{dst};
    o.put(kGeomMagic, 8);
    o.val<int32_t>(g->scheme);
    o.val<int32_t>(g->p0);
    o.val<int32_t>(g->p1);
    o.val<int32_t>(g->mode);
    o.val<int32_t>(g->n_dir);
    o.val<int32_t>(g->n_custom);
    if (g->n_custom) o.put(g->custom, sizeof(double) * 3 * g->n_custom);
    o.put(g->dirs_host, sizeof(double) * 3 * g->n_dir);
    o.val<uint64_t>(dirs_hash(g));
    o.val<uint64_t>(th);
    if (dst) {
        const uint64_t h = fnv(dst, o.n);
        memcpy(dst + o.n, &h, 8);
    }
    *size = o.n + 8;
    return CD_OK;
}

}  // namespace
}  // namespace cd

using namespace cd;

extern "C" {

uint64_t cd_fnv1a64(const void *data, size_t n) { return fnv(data, n); }

cd_status cd_tree_save(cd_tree t, void *buf, size_t cap, size_t *size, void *stream)
{
    NvtxRange nvtx_range("colden:tree_save");
    if (!t || !size) {
        set_error("tree or size is NULL");
        return CD_EINVAL;
    }
    const int64_t n = t->n_leaf;
    const size_t need = 8 + 3 * 4 + 8 + 8 + (size_t)n * (1 + 12 + 4) + 8;
    *size = need;
    if (!buf) return CD_OK;
    if (cap < need) {
        set_error("buffer of %zu bytes, the image needs %zu", cap, need);
        return CD_EINVAL;
    }
    std::vector<int8_t> level((size_t)n);
    std::vector<int32_t> ijk((size_t)n * 3);
    std::vector<float> rho((size_t)n);
    cd_status st = cd_tree_leaves(t, level.data(), ijk.data());
    if (st != CD_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(rho.data(), t->rho_leaf, sizeof(float) * n, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        set_error("reading the leaf densities failed: %s", cudaGetErrorString(cudaGetLastError()));
        return CD_ECUDA;
    }
    Out o{static_cast<unsigned char *>(buf)};
    o.put(kTreeMagic, 8);
    o.val<int32_t>(t->amr);
    o.val<int32_t>(t->base);
    o.val<int32_t>(t->L);
    o.val<double>(t->box_cm);
    o.val<int64_t>(n);
    o.put(level.data(), (size_t)n);
    o.put(ijk.data(), sizeof(int32_t) * 3 * n);
    o.put(rho.data(), sizeof(float) * n);
    const uint64_t h = fnv(buf, o.n);
    o.val<uint64_t>(h);
    return CD_OK;
}

cd_status cd_tree_load(const void *buf, size_t size, void *stream, cd_tree *out)
{
    NvtxRange nvtx_range("colden:tree_load");
    if (!buf || !out) {
        set_error("buffer or out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    uint64_t stored = 0;
    if (size >= 16) memcpy(&stored, static_cast<const unsigned char *>(buf) + size - 8, 8);
    if (size < 16 || fnv(buf, size - 8) != stored) {
        set_error("not a tree image, or the image is damaged (hash mismatch)");
        return CD_EINVAL;
    }
    In r{static_cast<const unsigned char *>(buf), size - 8};
    char magic[8];
    r.get(magic, 8);
    const int amr = r.val<int32_t>(), base = r.val<int32_t>(), L = r.val<int32_t>();
    const double box = r.val<double>();
    const int64_t n = r.val<int64_t>();
    if (!r.ok || memcmp(magic, kTreeMagic, 8) != 0 || n < 1 || L < 1 || L > CD_MAXL || base < 1 || base > L ||
        (size_t)n > (size - 8 - r.n) / 17 || r.n + (size_t)n * 17 != size - 8) {
        set_error("malformed tree image");
        return CD_EINVAL;
    }
    std::vector<int8_t> level((size_t)n);
    std::vector<int32_t> ijk((size_t)n * 3);
    std::vector<float> rho((size_t)n);
    r.get(level.data(), (size_t)n);
    r.get(ijk.data(), sizeof(int32_t) * 3 * n);
    r.get(rho.data(), sizeof(float) * n);
    if (!amr) {
        // uniform: back to the builder's row-major order (x fastest)
        const int64_t m = (int64_t)1 << L;
        if (base != L || n != m * m * m) {
            set_error("malformed tree image (uniform sizes)");
            return CD_EINVAL;
        }
        std::vector<float> grid((size_t)n);
        for (int64_t i = 0; i < n; ++i) {
            const int64_t x = ijk[3 * i], y = ijk[3 * i + 1], z = ijk[3 * i + 2];
            if (level[i] != L || x < 0 || y < 0 || z < 0 || x >= m || y >= m || z >= m) {
                set_error("malformed tree image (leaf %lld)", (long long)i);
                return CD_EINVAL;
            }
            grid[(size_t)((z * m + y) * m + x)] = rho[i];
        }
        return cd_build_tree_uniform(L, box, grid.data(), 0, stream, out);
    }
    return cd_build_tree_amr(base, L, box, n, level.data(), ijk.data(), rho.data(), 0, stream, out);
}

cd_status cd_geom_hash(cd_geom g, uint64_t *dirs, uint64_t *tables)
{
    if (!g) {
        set_error("geometry is NULL");
        return CD_EINVAL;
    }
    if (dirs) *dirs = dirs_hash(g);
    if (tables) return table_hash(g, tables);
    return CD_OK;
}

cd_status cd_geom_save(cd_geom g, void *buf, size_t cap, size_t *size)
{
    NvtxRange nvtx_range("colden:geom_save");
    if (!g || !size) {
        set_error("geometry or size is NULL");
        return CD_EINVAL;
    }
    geom_image(g, nullptr, size, 0);
    if (!buf) return CD_OK;
    if (cap < *size) {
        set_error("buffer of %zu bytes, the image needs %zu", cap, *size);
        return CD_EINVAL;
    }
    uint64_t th = 0;
    cd_status st = table_hash(g, &th);
    if (st != CD_OK) return st;
    return geom_image(g, static_cast<unsigned char *>(buf), size, th);
}

cd_status cd_geom_load(const void *buf, size_t size, void *stream, cd_geom *out)
{
    NvtxRange nvtx_range("colden:geom_load");
    if (!buf || !out) {
        set_error("buffer or out is NULL");
        return CD_EINVAL;
    }
    *out = nullptr;
    uint64_t stored = 0;
    if (size >= 16) memcpy(&stored, static_cast<const unsigned char *>(buf) + size - 8, 8);
    if (size < 16 || fnv(buf, size - 8) != stored) {
        set_error("not a geometry image, or the image is damaged (hash mismatch)");
        return CD_EINVAL;
    }
    In r{static_cast<const unsigned char *>(buf), size - 8};
    char magic[8];
    r.get(magic, 8);
    const int scheme = r.val<int32_t>(), p0 = r.val<int32_t>(), p1 = r.val<int32_t>(), mode = r.val<int32_t>();
    const int nd = r.val<int32_t>(), nc = r.val<int32_t>();
    if (!r.ok || memcmp(magic, kGeomMagic, 8) != 0 || nd < 1 || nd > CD_MAXDIR || nc < 0 || nc > CD_MAXDIR ||
        r.n + 24 * (size_t)(nc + nd) + 16 != size - 8) {
        set_error("malformed geometry image");
        return CD_EINVAL;
    }
    std::vector<double> custom((size_t)3 * nc), dirs((size_t)3 * nd);
    if (nc) r.get(custom.data(), sizeof(double) * 3 * nc);
    r.get(dirs.data(), sizeof(double) * 3 * nd);
    const uint64_t dh = r.val<uint64_t>(), th = r.val<uint64_t>();
    cd_geom g = nullptr;
    cd_status st = cd_precompute_geometry(scheme, p0, p1, nc ? custom.data() : nullptr, nc, mode, stream, &g);
    if (st != CD_OK) return st;
    uint64_t th2 = 0;
    if (g->n_dir != nd || memcmp(g->dirs_host, dirs.data(), sizeof(double) * 3 * nd) != 0 || dirs_hash(g) != dh) {
        cd_geom_free(g);
        set_error("the rebuilt direction set differs from the saved one");
        return CD_EINVAL;
    }
    if ((st = table_hash(g, &th2)) != CD_OK) {
        cd_geom_free(g);
        return st;
    }
    if (th2 != th) {
        cd_geom_free(g);
        set_error("the rebuilt geometry tables differ from the saved ones (table hash %016llx, saved %016llx)",
                  (unsigned long long)th2, (unsigned long long)th);
        return CD_EINVAL;
    }
    *out = g;
    return CD_OK;
}

}  // extern "C"
