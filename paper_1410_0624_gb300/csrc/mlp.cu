// The learned correction's network on the CUDA cores, FP32: forward pass,
// mean-squared-error loss, backward pass (reverse-mode chain rule, layer by
// layer), Adam (Kingma & Ba 2015, Algorithm 1) and the input standardisation.
// Training runs here; so does the FP32 form of learned inference.
//
// Every product is one tiled SGEMM kernel with the transposes and the
// elementwise epilogue (bias, GELU, GELU') as template parameters.  Sums over
// the batch (weight and bias gradients) are split over CTAs into partial
// buffers and added in a fixed order by a second kernel, so the gradient is
// bit-for-bit repeatable (no atomics anywhere in training).
#include <algorithm>

#include "learned.cuh"

namespace cd {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, kGemmThreads = 256;
constexpr int kTargetCtas = 304;   // two per SM

enum { EPI_STORE = 0, EPI_BIAS = 1, EPI_BIAS_GELU = 2, EPI_GELU_BWD = 3 };

struct Gemm {
    int M, N, K;
    const float *A;
    int64_t lda;
    const float *B;
    int64_t ldb;
    float *C;
    int64_t ldc;
    const float *bias;     // EPI_BIAS, EPI_BIAS_GELU: [N]
    float *Z;              // EPI_BIAS_GELU: pre-activation out (ldc), may be NULL
    const float *Zin;      // EPI_GELU_BWD: pre-activation (ldc); may alias C
    int kps;               // K per split, a multiple of BK; blockIdx.z is the split
    int64_t split_stride;  // floats between consecutive splits' C blocks
};

constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)
constexpr float kGeluA = 0.044715f;

__device__ __forceinline__ float gelu_f(float z)
{
    return 0.5f * z * (1.f + tanhf(kGeluC * fmaf(kGeluA * z, z * z, z)));
}

__device__ __forceinline__ float gelu_grad_f(float z)
{
    const float t = tanhf(kGeluC * fmaf(kGeluA * z, z * z, z));
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * fmaf(3.f * kGeluA * z, z, 1.f);
}

// C = op(A) op(B) (+ epilogue), op(A)[m][k] = TA ? A[k lda + m] : A[m lda + k],
// op(B)[k][n] = TB ? B[n ldb + k] : B[k ldb + n].  64 x 64 tile per CTA,
// 4 x 4 outputs per thread, K in slabs of 16 staged in shared memory.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(kGemmThreads) sgemm(Gemm g)
{
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * g.kps, ke = min(g.K, kb + g.kps);
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int idx = tid + e * kGemmThreads;   // 0 .. 1023 = 64 x 16
            const int ka = TA ? idx >> 6 : idx & 15, ma = TA ? idx & 63 : idx >> 4;
            const int gm = m0 + ma, gka = k0 + ka;
            float a = 0.f;
            if (gm < g.M && gka < ke) a = TA ? g.A[(int64_t)gka * g.lda + gm] : g.A[(int64_t)gm * g.lda + gka];
            As[ka][ma] = a;
            const int kb_ = TB ? idx & 15 : idx >> 6, nb = TB ? idx >> 4 : idx & 63;
            const int gn = n0 + nb, gkb = k0 + kb_;
            float b = 0.f;
            if (gn < g.N && gkb < ke) b = TB ? g.B[(int64_t)gn * g.ldb + gkb] : g.B[(int64_t)gkb * g.ldb + gn];
            Bs[kb_][nb] = b;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 b = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        __syncthreads();
    }

    float *C = g.C + (int64_t)blockIdx.z * g.split_stride;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            const int64_t o = (int64_t)m * g.ldc + n;
            float v = acc[i][j];
            if (EPI == EPI_BIAS) v += g.bias[n];
            if (EPI == EPI_BIAS_GELU) {
                v += g.bias[n];
                if (g.Z) g.Z[o] = v;
                v = gelu_f(v);
            }
            if (EPI == EPI_GELU_BWD) v *= gelu_grad_f(g.Zin[o]);
            C[o] = v;
        }
    }
}

template <bool TA, bool TB, int EPI>
cd_status run_gemm(Gemm g, int splits, cudaStream_t s)
{
    if (g.M <= 0 || g.N <= 0) return CD_OK;
    const dim3 grid((unsigned)((g.N + BN - 1) / BN), (unsigned)((g.M + BM - 1) / BM), (unsigned)splits);
    if (grid.y > 65535u) {
        set_error("GEMM with %d rows exceeds one launch", g.M);
        return CD_EINVAL;
    }
    LaunchScope ls(CD_K_NET, s);
    sgemm<TA, TB, EPI><<<grid, kGemmThreads, 0, s>>>(g);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

// out[i] = sum_{z < Z} part[z n + i], z in increasing order
__global__ void reduce_splits(int64_t n, int Z, const float *__restrict__ part, float *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f;
        for (int z = 0; z < Z; ++z) acc += part[(int64_t)z * n + i];
        out[i] = acc;
    }
}

// U[r][i] = (X[row r][i] - mu[i]) sinv[i], clipped to [-kUMax, kUMax]
__global__ void gather_normalise(int64_t B, int n_in, const float *__restrict__ X, const int64_t *__restrict__ rows,
                                 const float *__restrict__ mu, const float *__restrict__ sinv, float *__restrict__ U)
{
    const int64_t total = B * n_in;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / n_in;
        const int i = (int)(e - r * n_in);
        const int64_t src = rows ? rows[r] : r;
        U[e] = fminf(fmaxf((X[src * n_in + i] - mu[i]) * sinv[i], -kUMax), kUMax);
    }
}

constexpr int kRedThreads = 256;

// G = scale (D - Y[rows]); partial[b] = sum over block b's elements of (D - Y)^2
// (G may alias D: each element is read and then written by one thread)
__global__ void __launch_bounds__(kRedThreads) residual(int64_t B, int nd, const float *D,
                                                        const float *__restrict__ Y, const int64_t *__restrict__ rows,
                                                        float scale, float *G, float *__restrict__ partial)
{
    __shared__ float sh[kRedThreads];
    const int64_t total = B * nd;
    float acc = 0.f;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / nd;
        const int d = (int)(e - r * nd);
        const int64_t src = rows ? rows[r] : r;
        const float res = D[e] - Y[src * nd + d];
        acc = fmaf(res, res, acc);
        G[e] = scale * res;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

// out[0] = scale * sum_b partial[b] (one CTA, fixed order)
__global__ void __launch_bounds__(kRedThreads) finish_sum(int n, const float *__restrict__ partial, float scale,
                                                          float *__restrict__ out)
{
    __shared__ float sh[kRedThreads];
    float acc = 0.f;
    for (int i = threadIdx.x; i < n; i += kRedThreads) acc += partial[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = kRedThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = scale * sh[0];
}

__global__ void fill(int64_t n, float v, float *__restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = v;
}

// Adam with bias corrections c1 = 1 / (1 - beta1^t), c2 = 1 / (1 - beta2^t)
__global__ void adam_update(int64_t n, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// Column sums of x (pass 0) or of (x - mu)^2 (pass 1) over a row range, in
// FP64: partial[split][col].  32 columns per CTA (one per lane), 8 warps
// striding the rows.
constexpr int kNormSplits = 128;

__global__ void __launch_bounds__(256) column_moments(int64_t n, int n_in, const float *__restrict__ x,
                                                      const float *__restrict__ mu, int pass,
                                                      double *__restrict__ partial)
{
    __shared__ double sh[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int col = blockIdx.x * 32 + lane;
    const int64_t per = (n + gridDim.y - 1) / gridDim.y;
    const int64_t r0 = blockIdx.y * per, r1 = min(n, r0 + per);
    double acc = 0.0;
    if (col < n_in) {
        const double m = pass ? (double)mu[col] : 0.0;
        for (int64_t r = r0 + w; r < r1; r += 8) {
            const double v = (double)x[r * n_in + col] - m;
            acc += pass ? v * v : v;
        }
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0 && col < n_in) {
        double t = 0.0;
        for (int i = 0; i < 8; ++i) t += sh[i][lane];
        partial[(int64_t)blockIdx.y * n_in + col] = t;
    }
}

// pass 0: mu = sum / n; pass 1: sinv = 1 / sqrt(sum / n), or 0 for a column
// whose spread is at most kSdMin (it carried no information: ignored)
constexpr double kSdMin = 1e-3;

__global__ void finish_moments(int n_in, int splits, int64_t n, const double *__restrict__ partial, int pass,
                               float *__restrict__ mu, float *__restrict__ sinv)
{
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    if (col >= n_in) return;
    double t = 0.0;
    for (int z = 0; z < splits; ++z) t += partial[(int64_t)z * n_in + col];
    t /= (double)n;
    if (pass == 0) {
        mu[col] = (float)t;
    } else {
        const double sd = sqrt(t);
        sinv[col] = sd > kSdMin ? (float)(1.0 / sd) : 0.f;
    }
}

int grid_for(int64_t n, int threads)
{
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// split count for a GEMM whose K is the batch: enough CTAs to fill the GPU
int splits_for(int M, int N, int K, int *kps)
{
    const int tiles = ((M + BM - 1) / BM) * ((N + BN - 1) / BN);
    const int kslabs = (K + BK - 1) / BK;
    int z = std::max(1, std::min(kslabs, (kTargetCtas + tiles - 1) / tiles));
    int per = (kslabs + z - 1) / z;
    z = (kslabs + per - 1) / per;
    *kps = per * BK;
    return z;
}

template <typename T>
cd_status grow(T **p, size_t *cap, size_t need)
{
    if (*cap >= need) return CD_OK;
    if (*p) cd::lib_free(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        set_error("device allocation of %zu bytes failed", need * sizeof(T));
        return CD_ENOMEM;
    }
    *cap = need;
    return CD_OK;
}

// weight-style gradient: out[M][N] = op(A)^T-batch product, split over the batch
template <bool TA, bool TB>
cd_status batch_reduce_gemm(cd_net net, Gemm g, float *out, cudaStream_t s)
{
    int kps = 0;
    const int z = splits_for(g.M, g.N, g.K, &kps);
    const size_t need = (size_t)z * g.M * g.N;
    cd_status st = grow(&net->act.part, &net->act.part_cap, need);
    if (st != CD_OK) return st;
    g.C = net->act.part;
    g.ldc = g.N;
    g.kps = kps;
    g.split_stride = (int64_t)g.M * g.N;
    if ((st = run_gemm<TA, TB, EPI_STORE>(g, z, s)) != CD_OK) return st;
    const int64_t n = (int64_t)g.M * g.N;
    LaunchScope ls(CD_K_NET, s);
    reduce_splits<<<grid_for(n, 256), 256, 0, s>>>(n, z, net->act.part, out);
    CD_CHECK_LAUNCH();
    return CD_OK;
}

}  // namespace

cd_status net_reserve(cd_net net, int64_t rows)
{
    Activations &a = net->act;
    if (a.cap >= rows) return CD_OK;
    for (float *p : {a.U, a.Z1, a.A1, a.Z2, a.A2, a.D, a.G})
        if (p) cd::lib_free(p);
    a.U = a.Z1 = a.A1 = a.Z2 = a.A2 = a.D = a.G = nullptr;
    a.cap = 0;
    const NetLayout &L = net->lay;
    const size_t r = (size_t)rows;
    bool ok = cudaMalloc(&a.U, r * L.n_in * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.Z1, r * L.H * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.A1, r * L.H * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.Z2, r * L.H * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.A2, r * L.H * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.D, r * std::max(L.nd, 1) * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&a.G, r * std::max(L.H, 1) * sizeof(float)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        set_error("activation buffers for %lld rows do not fit", (long long)rows);
        return CD_ENOMEM;
    }
    a.cap = rows;
    return CD_OK;
}

cd_status mlp_forward(cd_net net, int64_t B, const float *x, const int64_t *rows, float *delta, cudaStream_t s)
{
    const NetLayout &L = net->lay;
    if (B > 0x7fffffff / 2) {
        set_error("batch of %lld rows too large", (long long)B);
        return CD_EINVAL;
    }
    cd_status st = net_reserve(net, B);
    if (st != CD_OK) return st;
    Activations &a = net->act;
    {
        LaunchScope ls(CD_K_NET, s);
        gather_normalise<<<grid_for(B * L.n_in, 256), 256, 0, s>>>(B, L.n_in, x, rows, net->mu, net->sinv, a.U);
        CD_CHECK_LAUNCH();
    }
    const float *P = net->p;
    Gemm g = {};
    g.M = (int)B;
    g.kps = 1 << 30;
    // z1 = W1 u + b1, a1 = gelu(z1)
    g.N = L.H; g.K = L.n_in; g.A = a.U; g.lda = L.n_in; g.B = P + L.W1; g.ldb = L.n_in;
    g.C = a.A1; g.ldc = L.H; g.bias = P + L.b1; g.Z = a.Z1;
    if ((st = run_gemm<false, true, EPI_BIAS_GELU>(g, 1, s)) != CD_OK) return st;
    // z2 = W2 a1 + b2, a2 = gelu(z2)
    g.N = L.H; g.K = L.H; g.A = a.A1; g.lda = L.H; g.B = P + L.W2; g.ldb = L.H;
    g.C = a.A2; g.ldc = L.H; g.bias = P + L.b2; g.Z = a.Z2;
    if ((st = run_gemm<false, true, EPI_BIAS_GELU>(g, 1, s)) != CD_OK) return st;
    // delta = W3 a2 + b3
    g.N = L.nd; g.K = L.H; g.A = a.A2; g.lda = L.H; g.B = P + L.W3; g.ldb = L.H;
    g.C = delta ? delta : a.D; g.ldc = L.nd; g.bias = P + L.b3; g.Z = nullptr;
    return run_gemm<false, true, EPI_BIAS>(g, 1, s);
}

cd_status mlp_loss_grad(cd_net net, int64_t B, const float *x, const float *y, const int64_t *rows,
                        float *loss_out, cudaStream_t s)
{
    const NetLayout &L = net->lay;
    cd_status st = mlp_forward(net, B, x, rows, nullptr, s);
    if (st != CD_OK) return st;
    Activations &a = net->act;
    // reduction scratch: residual partials, then a ones vector of length B
    const int nblk = grid_for(B * L.nd, kRedThreads);
    if ((st = grow(&a.red, &a.red_cap, (size_t)nblk + 1 + (size_t)B)) != CD_OK) return st;
    float *partial = a.red, *ones = a.red + nblk + 1;
    {
        // d loss / d delta = 2 (delta - y) / (B nd), in place over delta
        LaunchScope ls(CD_K_NET, s);
        residual<<<nblk, kRedThreads, 0, s>>>(B, L.nd, a.D, y, rows, (float)(2.0 / ((double)B * L.nd)), a.D,
                                              partial);
        CD_CHECK_LAUNCH();
    }
    if (loss_out) {
        LaunchScope ls(CD_K_NET, s);
        finish_sum<<<1, kRedThreads, 0, s>>>(nblk, partial, (float)(1.0 / ((double)B * L.nd)), loss_out);
        CD_CHECK_LAUNCH();
    }
    {
        LaunchScope ls(CD_K_NET, s);
        fill<<<grid_for(B, 256), 256, 0, s>>>(B, 1.f, ones);
        CD_CHECK_LAUNCH();
    }
    const float *P = net->p;
    float *G = net->grad;
    Gemm g = {};
    // dW3 = G3^T a2, db3 = 1^T G3
    g = {};
    g.M = L.nd; g.N = L.H; g.K = (int)B; g.A = a.D; g.lda = L.nd; g.B = a.A2; g.ldb = L.H;
    if ((st = batch_reduce_gemm<true, false>(net, g, G + L.W3, s)) != CD_OK) return st;
    g = {};
    g.M = 1; g.N = L.nd; g.K = (int)B; g.A = ones; g.lda = 1; g.B = a.D; g.ldb = L.nd;
    if ((st = batch_reduce_gemm<true, false>(net, g, G + L.b3, s)) != CD_OK) return st;
    // dz2 = (G3 W3) * gelu'(z2)
    g = {};
    g.M = (int)B; g.N = L.H; g.K = L.nd; g.A = a.D; g.lda = L.nd; g.B = P + L.W3; g.ldb = L.H;
    g.C = a.G; g.ldc = L.H; g.Zin = a.Z2; g.kps = 1 << 30;
    if ((st = run_gemm<false, false, EPI_GELU_BWD>(g, 1, s)) != CD_OK) return st;
    // dW2 = dz2^T a1, db2 = 1^T dz2
    g = {};
    g.M = L.H; g.N = L.H; g.K = (int)B; g.A = a.G; g.lda = L.H; g.B = a.A1; g.ldb = L.H;
    if ((st = batch_reduce_gemm<true, false>(net, g, G + L.W2, s)) != CD_OK) return st;
    g = {};
    g.M = 1; g.N = L.H; g.K = (int)B; g.A = ones; g.lda = 1; g.B = a.G; g.ldb = L.H;
    if ((st = batch_reduce_gemm<true, false>(net, g, G + L.b2, s)) != CD_OK) return st;
    // dz1 = (dz2 W2) * gelu'(z1), written over z1
    g = {};
    g.M = (int)B; g.N = L.H; g.K = L.H; g.A = a.G; g.lda = L.H; g.B = P + L.W2; g.ldb = L.H;
    g.C = a.Z1; g.ldc = L.H; g.Zin = a.Z1; g.kps = 1 << 30;
    if ((st = run_gemm<false, false, EPI_GELU_BWD>(g, 1, s)) != CD_OK) return st;
    // dW1 = dz1^T u, db1 = 1^T dz1
    g = {};
    g.M = L.H; g.N = L.n_in; g.K = (int)B; g.A = a.Z1; g.lda = L.H; g.B = a.U; g.ldb = L.n_in;
    if ((st = batch_reduce_gemm<true, false>(net, g, G + L.W1, s)) != CD_OK) return st;
    g = {};
    g.M = 1; g.N = L.H; g.K = (int)B; g.A = ones; g.lda = 1; g.B = a.Z1; g.ldb = L.H;
    return batch_reduce_gemm<true, false>(net, g, G + L.b1, s);
}

cd_status mlp_adam(cd_net net, const cd_adam &hp, cudaStream_t s)
{
    net->step += 1;
    const double t = (double)net->step;
    const float c1 = (float)(1.0 / (1.0 - pow(hp.beta1, t)));
    const float c2 = (float)(1.0 / (1.0 - pow(hp.beta2, t)));
    const int64_t n = net->lay.total;
    LaunchScope ls(CD_K_NET, s);
    adam_update<<<grid_for(n, 256), 256, 0, s>>>(n, net->p, net->grad, net->m, net->v, (float)hp.lr,
                                                 (float)hp.beta1, (float)hp.beta2, (float)hp.eps, c1, c2);
    CD_CHECK_LAUNCH();
    net->version += 1;
    return CD_OK;
}

cd_status mlp_fit_normaliser(cd_net net, int64_t n, const float *x, cudaStream_t s)
{
    const int n_in = net->lay.n_in;
    const int splits = (int)std::min<int64_t>(kNormSplits, std::max<int64_t>(1, n / 64));
    double *partial = nullptr;
    if (cudaMallocAsync(&partial, sizeof(double) * splits * n_in, s) != cudaSuccess) {
        cudaGetLastError();
        set_error("normaliser scratch allocation failed");
        return CD_ENOMEM;
    }
    const dim3 grid((unsigned)((n_in + 31) / 32), (unsigned)splits);
    for (int pass = 0; pass < 2; ++pass) {
        {
            LaunchScope ls(CD_K_NET, s);
            column_moments<<<grid, 256, 0, s>>>(n, n_in, x, net->mu, pass, partial);
        }
        LaunchScope ls(CD_K_NET, s);
        finish_moments<<<(n_in + 127) / 128, 128, 0, s>>>(n_in, splits, n, partial, pass, net->mu, net->sinv);
    }
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(partial, s);
    if (e != cudaSuccess) {
        set_error("normaliser launch: %s", cudaGetErrorString(e));
        return CD_ECUDA;
    }
    net->version += 1;
    return CD_OK;
}

}  // namespace cd
