// Heating of the application (§5): the screened UV field, the photoelectric
// rate with the efficiency of Wolfire et al. (1995) and the cosmic-ray rate,
// per leaf in the output order (Eqs. G0_eff, gamma_uv, gamma_cr).
//
// An elementwise pass over the leaves: it reads chi, T, n_e and the tree's
// leaf density (16 B a leaf) and writes up to three floats, so it runs at the
// HBM rate; four leaves a thread (16-byte loads and stores) when every pointer
// allows it.
#include <algorithm>

#include "common.cuh"

namespace cd {
namespace {

struct HeatArgs {
    int64_t n;
    const float *chi, *T, *n_e, *rho;
    float G0;
    float *g0_eff, *gamma_uv, *gamma_cr;
};

__device__ __forceinline__ void heat_one(const HeatArgs &A, float chi, float T, float ne, float n, float &g,
                                         float &uv, float &cr)
{
    g = chi * A.G0;
    cr = 1e-27f * n;
    if (A.gamma_uv) {
        const float x = g * sqrtf(T) / ne;
        const float eps = 4.9e-2f / (1.f + powf(x * (1.f / 1925.f), 0.73f)) +
                          3.7e-2f * powf(T * 1e-4f, 0.7f) / (1.f + x * (1.f / 5000.f));
        uv = 1e-24f * eps * g * n;
    }
}

__global__ void __launch_bounds__(256) heating_scalar(HeatArgs A)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
        const float T = A.gamma_uv ? A.T[i] : 0.f, ne = A.gamma_uv ? A.n_e[i] : 1.f;
        float g, uv = 0.f, cr;
        heat_one(A, A.chi[i], T, ne, A.rho[i], g, uv, cr);
        if (A.g0_eff) A.g0_eff[i] = g;
        if (A.gamma_uv) A.gamma_uv[i] = uv;
        if (A.gamma_cr) A.gamma_cr[i] = cr;
    }
}

// n % 4 == 0 and every non-NULL pointer 16-byte aligned
__global__ void __launch_bounds__(256) heating_vec4(HeatArgs A)
{
    const int64_t n4 = A.n >> 2;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n4; q += (int64_t)gridDim.x * blockDim.x) {
        const float4 c = reinterpret_cast<const float4 *>(A.chi)[q];
        const float4 r = reinterpret_cast<const float4 *>(A.rho)[q];
        float4 T = make_float4(0.f, 0.f, 0.f, 0.f), ne = make_float4(1.f, 1.f, 1.f, 1.f);
        if (A.gamma_uv) {
            T = reinterpret_cast<const float4 *>(A.T)[q];
            ne = reinterpret_cast<const float4 *>(A.n_e)[q];
        }
        float4 g, uv = make_float4(0.f, 0.f, 0.f, 0.f), cr;
        heat_one(A, c.x, T.x, ne.x, r.x, g.x, uv.x, cr.x);
        heat_one(A, c.y, T.y, ne.y, r.y, g.y, uv.y, cr.y);
        heat_one(A, c.z, T.z, ne.z, r.z, g.z, uv.z, cr.z);
        heat_one(A, c.w, T.w, ne.w, r.w, g.w, uv.w, cr.w);
        if (A.g0_eff) reinterpret_cast<float4 *>(A.g0_eff)[q] = g;
        if (A.gamma_uv) reinterpret_cast<float4 *>(A.gamma_uv)[q] = uv;
        if (A.gamma_cr) reinterpret_cast<float4 *>(A.gamma_cr)[q] = cr;
    }
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15) == 0; }

}  // namespace
}  // namespace cd

using namespace cd;

extern "C" cd_status cd_heating(cd_tree tree, const float *chi, const float *T, const float *n_e, double G0,
                                float *g0_eff, float *gamma_uv, float *gamma_cr, void *stream)
{
    NvtxRange nvtx_range("colden:heating_entry");
    if (!tree || !chi) {
        set_error("tree or chi is NULL");
        return CD_EINVAL;
    }
    if (gamma_uv && (!T || !n_e)) {
        set_error("the photoelectric rate needs T and n_e");
        return CD_EINVAL;
    }
    if (!(G0 >= 0.0) || !(G0 < 3.4e38)) {
        set_error("G0 must be finite and >= 0 (got %g)", G0);
        return CD_EINVAL;
    }
    if (!g0_eff && !gamma_uv && !gamma_cr) return CD_OK;
    HeatArgs A;
    A.n = tree->n_leaf;
    A.chi = chi;
    A.T = T;
    A.n_e = n_e;
    A.rho = tree->rho_leaf;
    A.G0 = (float)G0;
    A.g0_eff = g0_eff;
    A.gamma_uv = gamma_uv;
    A.gamma_cr = gamma_cr;
    if (A.n == 0) return CD_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const bool vec = A.n % 4 == 0 && aligned16(chi) && aligned16(A.rho) && (!gamma_uv || (aligned16(T) && aligned16(n_e))) &&
                     (!g0_eff || aligned16(g0_eff)) && (!gamma_uv || aligned16(gamma_uv)) &&
                     (!gamma_cr || aligned16(gamma_cr));
    const int64_t work = vec ? A.n / 4 : A.n;
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((work + 255) / 256, (int64_t)152 * 64));
    LaunchScope ls(CD_K_HEATING, s);
    if (vec) heating_vec4<<<(unsigned)blocks, 256, 0, s>>>(A);
    else heating_scalar<<<(unsigned)blocks, 256, 0, s>>>(A);
    CD_CHECK_LAUNCH();
    return CD_OK;
}
