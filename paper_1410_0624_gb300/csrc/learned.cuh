// Internal declarations of the learned correction (include/colden_learned.h):
// the network handle and the launchers of mlp.cu, learned.cu and mlp_tc.cu.
#pragma once

#include "common.cuh"
#include "../../include/colden_learned.h"

namespace cd {

constexpr int kSlots = CD_NET_SLOTS;
constexpr float kCFloor = 1e16f;    // cm^-2, floor under a level's contribution
constexpr float kNFloor = 1e-10f;   // cm^-3, floor under the leaf density
constexpr float kUMax = 8.f;        // standardised inputs are clipped to [-kUMax, kUMax]

// Offsets of the packed parameters (floats).
struct NetLayout {
    int nd, H, n_in;
    int64_t W1, b1, W2, b2, W3, b3, total;
    NetLayout() = default;
    NetLayout(int nd_, int H_)
        : nd(nd_), H(H_), n_in(kSlots * nd_ + 1)
    {
        W1 = 0;
        b1 = W1 + (int64_t)H * n_in;
        W2 = b1 + H;
        b2 = W2 + (int64_t)H * H;
        W3 = b2 + H;
        b3 = W3 + (int64_t)nd * H;
        total = b3 + nd;
    }
};

// Activations of one batch: row-major [cap][...].
struct Activations {
    int64_t cap = 0;
    float *U = nullptr;     // standardised inputs [cap][n_in]
    float *Z1 = nullptr, *A1 = nullptr, *Z2 = nullptr, *A2 = nullptr;   // [cap][H]
    float *D = nullptr;     // delta, then d loss / d delta [cap][nd]
    float *G = nullptr;     // d loss / d (A or Z) scratch [cap][H]
    float *part = nullptr;  // split-K partial sums
    size_t part_cap = 0;
    float *red = nullptr;   // partial sums of the loss and the normaliser
    size_t red_cap = 0;
};

}  // namespace cd

struct cd_net_s {
    cd::NetLayout lay;
    float *p = nullptr;       // FP32 master parameters (device)
    float *mu = nullptr;      // [n_in]
    float *sinv = nullptr;    // [n_in]
    float *m = nullptr, *v = nullptr;   // Adam moments
    float *grad = nullptr;    // [total]
    int64_t step = 0;
    // trusted range of delta (cd_net_set_delta_range): outside it, or where
    // delta is not finite, the learned form returns the plain column
    float dlo = -INFINITY, dhi = INFINITY;
    int dev = 0;
    cd::Activations act;
    // BF16 operands of the tensor-core inference (mlp_tc.cu), rebuilt when
    // version != built_version
    void *tc = nullptr;
    int64_t version = 1, tc_version = 0;
};

namespace cd {

// mlp.cu
cd_status net_reserve(cd_net net, int64_t rows);
// delta [B][nd] of rows `rows` (NULL: 0..B-1) of x; keeps the activations
// (for a following backward) when keep != 0
cd_status mlp_forward(cd_net net, int64_t B, const float *x, const int64_t *rows, float *delta, cudaStream_t s);
// loss and gradient into net->grad; loss_out may be NULL
cd_status mlp_loss_grad(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows,
                        float *loss_out, cudaStream_t s);
cd_status mlp_adam(cd_net net, const cd_adam &hp, cudaStream_t s);
cd_status mlp_fit_normaliser(cd_net net, int64_t n, const float *x, cudaStream_t s);

// mlp_tc.cu: the fused BF16 tensor-core inference
cd_status column_density_learned_tc(cd_tree t, cd_geom g, const cd_opts &o, float *n_h, float *a_v, float *shield,
                                    cudaStream_t s);
void net_free_tc(cd_net net);
bool learned_tc_supported(int nd, int hidden);
// CD_ETIMEOUT if a learned tensor-core kernel gave up a bounded wait (clears it)
cd_status learned_tc_fault_check();

// learned.cu
// every shell's sum kept apart; precision CD_BF16 uses the tensor-core
// contraction for receiving levels >= 4
cd_status ensure_level_sums(cd_tree t, cd_geom g, int precision, cudaStream_t s);
cd_status column_density_learned(cd_tree t, cd_geom g, const cd_opts &o, float *n_h, float *a_v, float *shield,
                                 cudaStream_t s);

}  // namespace cd
