// Learned local-field correction (no counterpart in the paper): a network
// 6 -> 128 -> 128 -> 128 -> 2 with SiLU hidden activations that maps
// (|q|/q_max, q direction, w/w_max, ln(L_noLFE)/10) to (mu, s): mu estimates
// log(L_LFE / L_noLFE) of the loss-function heads and s = log sigma^2 its
// uncertainty.  Loss: the Gaussian negative log-likelihood
// (s + (y - mu)^2 e^-s) / 2 averaged over the batch; optimiser: Adam.
//
// Precision: FP32 master weights; BF16 compute copies of the weight
// matrices (biases stay FP32); activations, accumulations and gradients in
// FP32.
//
// Kernels: k_mlp_tile runs one 16-sample tile per CTA with all weights
// resident in shared memory (rows padded to an odd word count so the row-
// and column-wise walks are both free of bank conflicts): thread j owns
// neuron j of a layer for the 16 samples.  In training mode it back-
// propagates and writes the tile's gradient into its own slot of a partial
// buffer (no atomics, so the sum is deterministic); k_mlp_update sums the
// slots, applies Adam to the FP32 masters and refreshes the BF16 copies.
// One epoch (a shuffled pass in steps of `batch` samples) is captured once as
// a CUDA graph and replayed per epoch; the shuffle (Fisher-Yates driven by
// SplitMix64) runs on the host and only the index list is uploaded.
#include "qcx_internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

namespace {

constexpr int NI = 6, H = 128, NO = 2, S = 16;
constexpr int OW1 = 0, OB1 = OW1 + H * NI, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H * H,
              OW4 = OB3 + H, OB4 = OW4 + NO * H, NP = OB4 + NO;
constexpr int WST = H + 2;   // padded row stride (BF16) of the 128 x 128 matrices in shared memory
static_assert(NP == 34178, "parameter layout");

struct Smem {
    __nv_bfloat16 W2[H][WST], W3[H][WST];
    __nv_bfloat16 W1[H][NI];
    __nv_bfloat16 W4[NO][H];
    float b1[H], b2[H], b3[H], b4[NO];
    float x[S][NI];
    float z1[S][H], z2[S][H], z3[S][H];   // pre-activations
    float a1[S][H], a2[S][H], a3[S][H];   // activations
    float d[2][S][H];                     // deltas (ping-pong)
    float out[S][NO], dout[S][NO];
    float lsum[S];
};

__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }
__device__ __forceinline__ float dsilu(float z) {
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

struct TileArgs {
    const float* theta;            // FP32 masters (biases read from here)
    const __nv_bfloat16* wbf;      // BF16 copies (same layout; bias slots unused)
    const float* X;                // [n][6]
    const float* y;                // [n] (training)
    const int* idx;                // sample order (training) or null (identity)
    int n, off, count;             // samples [off, off + count) of the order
    float inv_batch;               // 1 / samples in the step (mean loss)
    float* part;                   // [grid][NP] gradient slots (training)
    float* ploss;                  // [grid] loss sums (training)
    float* mu;                     // [n] (prediction)
    float* logvar;                 // [n]
};

// one layer 128 -> 128: z[s][j] = b[j] + sum_i W[j][i] a[s][i]
__device__ __forceinline__ void dense128(const __nv_bfloat16 (*W)[WST], const float* b, const float (*a)[H],
                                         float (*z)[H], float (*act)[H], int j) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = b[j];
    for (int i = 0; i < H; i += 2) {
        const float2 w = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&W[j][i]));
#pragma unroll
        for (int s = 0; s < S; ++s) {
            const float2 av = *reinterpret_cast<const float2*>(&a[s][i]);
            acc[s] = fmaf(w.x, av.x, fmaf(w.y, av.y, acc[s]));
        }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
        z[s][j] = acc[s];
        act[s][j] = silu(acc[s]);
    }
}

// delta of a 128-wide layer from the 128-wide layer above:
// din[s][i] = (sum_j W[j][i] dout[s][j]) * silu'(z[s][i])
__device__ __forceinline__ void back128(const __nv_bfloat16 (*W)[WST], const float (*dout)[H], const float (*z)[H],
                                        float (*din)[H], int i) {
    float acc[S];
#pragma unroll
    for (int s = 0; s < S; ++s) acc[s] = 0.0f;
    for (int j = 0; j < H; ++j) {
        const float w = __bfloat162float(W[j][i]);
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = fmaf(w, dout[s][j], acc[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) din[s][i] = acc[s] * dsilu(z[s][i]);
}

// gradient slot of a 128 x 128 layer: g[j][i] = sum_s d[s][j] a[s][i] (thread i, coalesced rows)
__device__ __forceinline__ void wgrad128(const float (*d)[H], const float (*a)[H], float* g, int i) {
    float av[S];
#pragma unroll
    for (int s = 0; s < S; ++s) av[s] = a[s][i];
    for (int j = 0; j < H; ++j) {
        float acc = 0.0f;
#pragma unroll
        for (int s = 0; s < S; ++s) acc = fmaf(d[s][j], av[s], acc);
        g[j * H + i] = acc;
    }
}

template <int TRAIN>
__global__ void __launch_bounds__(H) k_mlp_tile(TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& sm = *reinterpret_cast<Smem*>(smem_raw);
    const int t = threadIdx.x;
    const int first = a.off + blockIdx.x * S;
    // weights into shared memory
    for (int e = t; e < H * H / 2; e += H) {
        const int r = e / (H / 2), c = 2 * (e - r * (H / 2));
        *reinterpret_cast<__nv_bfloat162*>(&sm.W2[r][c]) =
            *reinterpret_cast<const __nv_bfloat162*>(a.wbf + OW2 + r * H + c);
        *reinterpret_cast<__nv_bfloat162*>(&sm.W3[r][c]) =
            *reinterpret_cast<const __nv_bfloat162*>(a.wbf + OW3 + r * H + c);
    }
    for (int e = t; e < H * NI; e += H) sm.W1[e / NI][e % NI] = a.wbf[OW1 + e];
    for (int e = t; e < NO * H; e += H) sm.W4[e / H][e % H] = a.wbf[OW4 + e];
    sm.b1[t] = a.theta[OB1 + t];
    sm.b2[t] = a.theta[OB2 + t];
    sm.b3[t] = a.theta[OB3 + t];
    if (t < NO) sm.b4[t] = a.theta[OB4 + t];
    // inputs (rows past the end are zero and carry no loss)
    for (int e = t; e < S * NI; e += H) {
        const int s = e / NI, i = e - s * NI;
        const int k = first + s;
        float v = 0.0f;
        if (k < a.off + a.count) v = a.X[(size_t)(a.idx ? a.idx[k] : k) * NI + i];
        sm.x[s][i] = v;
    }
    __syncthreads();
    // ---------------------------------------------------------------- forward
    {
        float acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) acc[s] = sm.b1[t];
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const float w = __bfloat162float(sm.W1[t][i]);
#pragma unroll
            for (int s = 0; s < S; ++s) acc[s] = fmaf(w, sm.x[s][i], acc[s]);
        }
#pragma unroll
        for (int s = 0; s < S; ++s) {
            sm.z1[s][t] = acc[s];
            sm.a1[s][t] = silu(acc[s]);
        }
    }
    __syncthreads();
    dense128(sm.W2, sm.b2, sm.a1, sm.z2, sm.a2, t);
    __syncthreads();
    dense128(sm.W3, sm.b3, sm.a2, sm.z3, sm.a3, t);
    __syncthreads();
    if (t < NO * S) {
        const int o = t / S, s = t - o * S;
        float acc = sm.b4[o];
        for (int i = 0; i < H; ++i) acc = fmaf(__bfloat162float(sm.W4[o][i]), sm.a3[s][i], acc);
        sm.out[s][o] = acc;
    }
    __syncthreads();
    if (!TRAIN) {
        if (t < S && first + t < a.off + a.count) {
            a.mu[first + t] = sm.out[t][0];
            a.logvar[first + t] = sm.out[t][1];
        }
        return;
    }
    // --------------------------------------------------------------- backward
    if (t < S) {
        const int k = first + t;
        float d0 = 0.0f, d1 = 0.0f, l = 0.0f;
        if (k < a.off + a.count) {
            const float yv = a.y[a.idx ? a.idx[k] : k];
            const float mu = sm.out[t][0], s = sm.out[t][1];
            const float r = yv - mu, e = expf(-s);
            l = 0.5f * (s + r * r * e);
            d0 = -r * e * a.inv_batch;
            d1 = 0.5f * (1.0f - r * r * e) * a.inv_batch;
        }
        sm.dout[t][0] = d0;
        sm.dout[t][1] = d1;
        sm.lsum[t] = l;
    }
    __syncthreads();
    float* g = a.part + (size_t)blockIdx.x * NP;
    // output layer: dW4[o][i], db4, and the delta of layer 3
    {
        float g0 = 0.0f, g1 = 0.0f, acc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
            g0 = fmaf(sm.dout[s][0], sm.a3[s][t], g0);
            g1 = fmaf(sm.dout[s][1], sm.a3[s][t], g1);
            acc[s] = (__bfloat162float(sm.W4[0][t]) * sm.dout[s][0] + __bfloat162float(sm.W4[1][t]) * sm.dout[s][1]) *
                     dsilu(sm.z3[s][t]);
        }
        g[OW4 + t] = g0;
        g[OW4 + H + t] = g1;
#pragma unroll
        for (int s = 0; s < S; ++s) sm.d[0][s][t] = acc[s];
        if (t < NO) {
            float b = 0.0f;
            for (int s = 0; s < S; ++s) b += sm.dout[s][t];
            g[OB4 + t] = b;
        }
        if (t == 0) {
            float l = 0.0f;
            for (int s = 0; s < S; ++s) l += sm.lsum[s];
            a.ploss[blockIdx.x] = l;
        }
    }
    __syncthreads();
    // layer 3 (a2 -> z3): weights, bias, delta of layer 2
    wgrad128(sm.d[0], sm.a2, g + OW3, t);
    {
        float b = 0.0f;
        for (int s = 0; s < S; ++s) b += sm.d[0][s][t];
        g[OB3 + t] = b;
    }
    back128(sm.W3, sm.d[0], sm.z2, sm.d[1], t);
    __syncthreads();
    // layer 2 (a1 -> z2)
    wgrad128(sm.d[1], sm.a1, g + OW2, t);
    {
        float b = 0.0f;
        for (int s = 0; s < S; ++s) b += sm.d[1][s][t];
        g[OB2 + t] = b;
    }
    back128(sm.W2, sm.d[1], sm.z1, sm.d[0], t);
    __syncthreads();
    // layer 1 (x -> z1): thread j owns row j of W1
    {
        float gi[NI] = {0, 0, 0, 0, 0, 0}, b = 0.0f;
        for (int s = 0; s < S; ++s) {
            const float dj = sm.d[0][s][t];
            b += dj;
#pragma unroll
            for (int i = 0; i < NI; ++i) gi[i] = fmaf(dj, sm.x[s][i], gi[i]);
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) g[OW1 + t * NI + i] = gi[i];
        g[OB1 + t] = b;
    }
}

struct UpdArgs {
    float* theta;
    __nv_bfloat16* wbf;
    float* m;
    float* v;
    const float* part;
    const float* ploss;
    int nslot;
    float* grad_out;           // optional: summed gradient (no update when adam == 0)
    double* loss_acc;          // optional: += loss sum of the step
    const long long* tbase;    // Adam step count before this epoch
    int step;                  // step number inside the epoch (0-based)
    int adam;
    float lr, beta1, beta2, eps;
};

bool is_weight(int p) {
    return (p >= OW1 && p < OB1) || (p >= OW2 && p < OB2) || (p >= OW3 && p < OB3) || (p >= OW4 && p < OB4);
}

__device__ __forceinline__ bool d_is_weight(int p) {
    return (p < OB1) || (p >= OW2 && p < OB2) || (p >= OW3 && p < OB3) || (p >= OW4 && p < OB4);
}

__global__ void k_mlp_update(UpdArgs u) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p == 0 && u.loss_acc) {
        double l = 0.0;
        for (int c = 0; c < u.nslot; ++c) l += (double)u.ploss[c];
        *u.loss_acc += l;
    }
    if (p >= NP) return;
    float gsum = 0.0f;
    for (int c = 0; c < u.nslot; ++c) gsum += u.part[(size_t)c * NP + p];
    if (u.grad_out) u.grad_out[p] = gsum;
    if (!u.adam) return;
    const double t = (double)(*u.tbase + u.step + 1);
    const float m = u.beta1 * u.m[p] + (1.0f - u.beta1) * gsum;
    const float v = u.beta2 * u.v[p] + (1.0f - u.beta2) * gsum * gsum;
    u.m[p] = m;
    u.v[p] = v;
    const float mh = m / (float)(1.0 - pow((double)u.beta1, t));
    const float vh = v / (float)(1.0 - pow((double)u.beta2, t));
    const float th = u.theta[p] - u.lr * mh / (sqrtf(vh) + u.eps);
    u.theta[p] = th;
    if (d_is_weight(p)) u.wbf[p] = __float2bfloat16_rn(th);
}

__global__ void k_mlp_requant(const float* theta, __nv_bfloat16* wbf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) wbf[p] = __float2bfloat16_rn(theta[p]);
}

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace

struct MlpState {
    bool have = false;
    long long t = 0;            // Adam steps taken
    DevBuf theta, wbf, m, v, part, ploss, X, y, idx, mu, lv, grad, tbase, lacc;
    cudaGraphExec_t exec = nullptr;
    int g_n = 0, g_batch = 0;   // shape the captured epoch graph was built for
    float g_lr = 0, g_b1 = 0, g_b2 = 0, g_eps = 0;
    std::vector<const void*> g_ptrs;   // buffers the graph reads and writes (re-captured if any moved)
    std::vector<const void*> ptrs() const {
        return {theta.p, wbf.p, m.p, v.p, part.p, ploss.p, X.p, y.p, idx.p, lacc.p, tbase.p};
    }
    ~MlpState() {
        if (exec) cudaGraphExecDestroy(exec);
    }
};

void qcx_mlp_destroy(MlpState* m) { delete m; }

namespace {

size_t smem_bytes() { return sizeof(Smem); }

qcx_status need_params(qcx_ctx* ctx) {
    if (!ctx->mlp || !ctx->mlp->have) return ctx->fail(QCX_ERR_STATE, "mlp: no parameters set");
    return QCX_OK;
}

cudaError_t set_smem_attr() {
    cudaError_t e = cudaFuncSetAttribute((const void*)k_mlp_tile<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_bytes());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute((const void*)k_mlp_tile<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_bytes());
}

// forward + backward of samples [off, off + count) of the order, gradient slots per tile
cudaError_t launch_grad(qcx_ctx* ctx, MlpState& s, int n, int off, int count, int batch) {
    TileArgs a{};
    a.theta = s.theta.as<float>();
    a.wbf = s.wbf.as<__nv_bfloat16>();
    a.X = s.X.as<float>();
    a.y = s.y.as<float>();
    a.idx = s.idx.as<int>();
    a.n = n;
    a.off = off;
    a.count = count;
    a.inv_batch = 1.0f / (float)batch;
    a.part = s.part.as<float>();
    a.ploss = s.ploss.as<float>();
    const int grid = (count + S - 1) / S;
    k_mlp_tile<1><<<grid, H, smem_bytes(), ctx->stream>>>(a);
    return cudaGetLastError();
}

qcx_status load_data(qcx_ctx* ctx, MlpState& s, int n, const float* X, const float* y, bool identity) {
    CUDA_OR_FAIL(s.X.ensure(sizeof(float) * NI * (size_t)n), "alloc");
    CUDA_OR_FAIL(qcx_copy_in(ctx, s.X.p, X, sizeof(float) * NI * (size_t)n), "copy X");
    if (y) {
        CUDA_OR_FAIL(s.y.ensure(sizeof(float) * (size_t)n), "alloc");
        CUDA_OR_FAIL(qcx_copy_in(ctx, s.y.p, y, sizeof(float) * (size_t)n), "copy y");
    }
    CUDA_OR_FAIL(s.idx.ensure(sizeof(int) * (size_t)n), "alloc");
    if (identity) {
        std::vector<int> id(n);
        for (int i = 0; i < n; ++i) id[i] = i;
        CUDA_OR_FAIL(cudaMemcpyAsync(s.idx.p, id.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream),
                     "copy order");
        CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    }
    return QCX_OK;
}

bool finite_f(const float* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

extern "C" {

int qcx_mlp_nparam(void) { return NP; }

qcx_status qcx_mlp_set_params(qcx_ctx* ctx, const float* params) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!params) return ctx->fail(QCX_ERR_ARG, "mlp_set_params: null");
    cudaSetDevice(ctx->device);
    if (!ctx->mlp) {
        ctx->mlp = new (std::nothrow) MlpState();
        if (!ctx->mlp) return ctx->fail(QCX_ERR_ALLOC, "mlp state");
    }
    MlpState& s = *ctx->mlp;
    CUDA_OR_FAIL(s.theta.ensure(sizeof(float) * NP), "alloc");
    CUDA_OR_FAIL(s.wbf.ensure(sizeof(__nv_bfloat16) * NP), "alloc");
    CUDA_OR_FAIL(s.m.ensure(sizeof(float) * NP), "alloc");
    CUDA_OR_FAIL(s.v.ensure(sizeof(float) * NP), "alloc");
    CUDA_OR_FAIL(s.tbase.ensure(sizeof(long long)), "alloc");
    CUDA_OR_FAIL(s.lacc.ensure(sizeof(double)), "alloc");
    CUDA_OR_FAIL(s.grad.ensure(sizeof(float) * NP), "alloc");
    CUDA_OR_FAIL(qcx_copy_in(ctx, s.theta.p, params, sizeof(float) * NP), "copy params");
    CUDA_OR_FAIL(cudaMemsetAsync(s.m.p, 0, sizeof(float) * NP, ctx->stream), "clear");
    CUDA_OR_FAIL(cudaMemsetAsync(s.v.p, 0, sizeof(float) * NP, ctx->stream), "clear");
    k_mlp_requant<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(s.theta.as<float>(), s.wbf.as<__nv_bfloat16>());
    CUDA_OR_FAIL(cudaGetLastError(), "requantise");
    std::vector<float> h(NP);
    CUDA_OR_FAIL(cudaMemcpyAsync(h.data(), s.theta.p, sizeof(float) * NP, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    if (!finite_f(h.data(), NP)) return ctx->fail(QCX_ERR_ARG, "mlp_set_params: non-finite parameter");
    CUDA_OR_FAIL(set_smem_attr(), "smem attribute");
    s.t = 0;
    s.have = true;
    return QCX_OK;
}

qcx_status qcx_mlp_get_params(qcx_ctx* ctx, float* out_params, float* out_compute) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    qcx_status st = need_params(ctx);
    if (st != QCX_OK) return st;
    cudaSetDevice(ctx->device);
    MlpState& s = *ctx->mlp;
    std::vector<float> th(NP);
    std::vector<__nv_bfloat16> wb(NP);
    CUDA_OR_FAIL(cudaMemcpyAsync(th.data(), s.theta.p, sizeof(float) * NP, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(wb.data(), s.wbf.p, sizeof(__nv_bfloat16) * NP, cudaMemcpyDeviceToHost, ctx->stream),
                 "copy");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    std::vector<float> comp(NP);
    for (int p = 0; p < NP; ++p) comp[p] = is_weight(p) ? __bfloat162float(wb[p]) : th[p];
    if (out_params) {
        if (qcx_is_device_ptr(out_params))
            CUDA_OR_FAIL(cudaMemcpy(out_params, th.data(), sizeof(float) * NP, cudaMemcpyHostToDevice), "copy out");
        else
            std::memcpy(out_params, th.data(), sizeof(float) * NP);
    }
    if (out_compute) {
        if (qcx_is_device_ptr(out_compute))
            CUDA_OR_FAIL(cudaMemcpy(out_compute, comp.data(), sizeof(float) * NP, cudaMemcpyHostToDevice), "copy out");
        else
            std::memcpy(out_compute, comp.data(), sizeof(float) * NP);
    }
    return QCX_OK;
}

qcx_status qcx_mlp_grad(qcx_ctx* ctx, int n, const float* X, const float* y, float* out_grad, double* out_loss) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    qcx_status st = need_params(ctx);
    if (st != QCX_OK) return st;
    if (n < 1 || n > (1 << 24) || !X || !y || !out_grad) return ctx->fail(QCX_ERR_ARG, "mlp_grad: bad arguments");
    cudaSetDevice(ctx->device);
    MlpState& s = *ctx->mlp;
    st = load_data(ctx, s, n, X, y, true);
    if (st != QCX_OK) return st;
    const int nslot = (n + S - 1) / S;
    CUDA_OR_FAIL(s.part.ensure(sizeof(float) * NP * (size_t)nslot), "alloc");
    CUDA_OR_FAIL(s.ploss.ensure(sizeof(float) * (size_t)nslot), "alloc");
    CUDA_OR_FAIL(cudaMemsetAsync(s.lacc.p, 0, sizeof(double), ctx->stream), "clear");
    CUDA_OR_FAIL(launch_grad(ctx, s, n, 0, n, n), "gradient kernel");
    UpdArgs u{};
    u.theta = s.theta.as<float>();
    u.wbf = s.wbf.as<__nv_bfloat16>();
    u.m = s.m.as<float>();
    u.v = s.v.as<float>();
    u.part = s.part.as<float>();
    u.ploss = s.ploss.as<float>();
    u.nslot = nslot;
    u.grad_out = s.grad.as<float>();
    u.loss_acc = s.lacc.as<double>();
    u.tbase = s.tbase.as<long long>();
    u.adam = 0;
    k_mlp_update<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(u);
    CUDA_OR_FAIL(cudaGetLastError(), "reduce kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_grad, s.grad.p, sizeof(float) * NP), "copy out");
    double l = 0.0;
    CUDA_OR_FAIL(cudaMemcpyAsync(&l, s.lacc.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    if (out_loss) *out_loss = l / n;
    return QCX_OK;
}

qcx_status qcx_mlp_train(qcx_ctx* ctx, int n, const float* X, const float* y, const qcx_mlp_opts* opts,
                         float* out_epoch_loss) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    qcx_status st = need_params(ctx);
    if (st != QCX_OK) return st;
    if (n < 1 || n > (1 << 24) || !X || !y || !opts || opts->epochs < 1 || opts->batch < 1 ||
        !(opts->lr > 0) || !(opts->beta1 >= 0 && opts->beta1 < 1) || !(opts->beta2 >= 0 && opts->beta2 < 1) ||
        !(opts->eps > 0))
        return ctx->fail(QCX_ERR_ARG, "mlp_train: bad arguments");
    cudaSetDevice(ctx->device);
    MlpState& s = *ctx->mlp;
    st = load_data(ctx, s, n, X, y, false);
    if (st != QCX_OK) return st;
    const int batch = std::min(opts->batch, n);
    const int nstep = (n + batch - 1) / batch;
    const int nslot = (batch + S - 1) / S;
    CUDA_OR_FAIL(s.part.ensure(sizeof(float) * NP * (size_t)nslot), "alloc");
    CUDA_OR_FAIL(s.ploss.ensure(sizeof(float) * (size_t)nslot), "alloc");
    // one epoch as a graph: per step the tile kernel and the reduction + Adam update
    if (!s.exec || s.g_n != n || s.g_batch != batch || s.g_lr != opts->lr || s.g_b1 != opts->beta1 ||
        s.g_b2 != opts->beta2 || s.g_eps != opts->eps || s.g_ptrs != s.ptrs()) {
        if (s.exec) cudaGraphExecDestroy(s.exec);
        s.exec = nullptr;
        cudaGraph_t g = nullptr;
        CUDA_OR_FAIL(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed), "capture");
        cudaError_t er = cudaSuccess;
        for (int k = 0; k < nstep && er == cudaSuccess; ++k) {
            const int off = k * batch, cnt = std::min(batch, n - off);
            er = launch_grad(ctx, s, n, off, cnt, cnt);
            if (er != cudaSuccess) break;
            UpdArgs u{};
            u.theta = s.theta.as<float>();
            u.wbf = s.wbf.as<__nv_bfloat16>();
            u.m = s.m.as<float>();
            u.v = s.v.as<float>();
            u.part = s.part.as<float>();
            u.ploss = s.ploss.as<float>();
            u.nslot = (cnt + S - 1) / S;
            u.grad_out = nullptr;
            u.loss_acc = s.lacc.as<double>();
            u.tbase = s.tbase.as<long long>();
            u.step = k;
            u.adam = 1;
            u.lr = opts->lr;
            u.beta1 = opts->beta1;
            u.beta2 = opts->beta2;
            u.eps = opts->eps;
            k_mlp_update<<<(NP + 255) / 256, 256, 0, ctx->stream>>>(u);
            er = cudaGetLastError();
        }
        cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g);
        if (er != cudaSuccess || ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            CUDA_OR_FAIL(er != cudaSuccess ? er : ec, "capture epoch");
        }
        cudaError_t ei = cudaGraphInstantiate(&s.exec, g, 0);
        cudaGraphDestroy(g);
        CUDA_OR_FAIL(ei, "instantiate epoch graph");
        s.g_ptrs = s.ptrs();
        s.g_n = n;
        s.g_batch = batch;
        s.g_lr = opts->lr;
        s.g_b1 = opts->beta1;
        s.g_b2 = opts->beta2;
        s.g_eps = opts->eps;
    }
    uint64_t seed = opts->seed;
    std::vector<int> order(n);
    std::vector<double> eloss(opts->epochs);
    for (int ep = 0; ep < opts->epochs; ++ep) {
        for (int i = 0; i < n; ++i) order[i] = i;
        for (int i = n - 1; i > 0; --i) {
            const int j = (int)(splitmix64(seed) % (uint64_t)(i + 1));
            std::swap(order[i], order[j]);
        }
        CUDA_OR_FAIL(cudaMemcpyAsync(s.idx.p, order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, ctx->stream),
                     "copy order");
        CUDA_OR_FAIL(cudaMemcpyAsync(s.tbase.p, &s.t, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream),
                     "copy step");
        CUDA_OR_FAIL(cudaMemsetAsync(s.lacc.p, 0, sizeof(double), ctx->stream), "clear");
        CUDA_OR_FAIL(cudaGraphLaunch(s.exec, ctx->stream), "launch epoch");
        CUDA_OR_FAIL(cudaMemcpyAsync(&eloss[ep], s.lacc.p, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream),
                     "copy loss");
        CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");   // order and step buffers are reused
        s.t += nstep;
    }
    if (out_epoch_loss)
        for (int ep = 0; ep < opts->epochs; ++ep) out_epoch_loss[ep] = (float)(eloss[ep] / n);
    for (double l : eloss)
        if (!std::isfinite(l)) return ctx->fail(QCX_ERR_NOT_CONVERGED, "mlp_train: loss became non-finite");
    return QCX_OK;
}

qcx_status qcx_mlp_predict(qcx_ctx* ctx, int n, const float* X, float* out_mu, float* out_logvar) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    qcx_status st = need_params(ctx);
    if (st != QCX_OK) return st;
    if (n < 1 || n > (1 << 24) || !X || !out_mu || !out_logvar) return ctx->fail(QCX_ERR_ARG, "mlp_predict: bad arguments");
    cudaSetDevice(ctx->device);
    MlpState& s = *ctx->mlp;
    CUDA_OR_FAIL(s.X.ensure(sizeof(float) * NI * (size_t)n), "alloc");
    CUDA_OR_FAIL(qcx_copy_in(ctx, s.X.p, X, sizeof(float) * NI * (size_t)n), "copy X");
    CUDA_OR_FAIL(s.mu.ensure(sizeof(float) * (size_t)n), "alloc");
    CUDA_OR_FAIL(s.lv.ensure(sizeof(float) * (size_t)n), "alloc");
    TileArgs a{};
    a.theta = s.theta.as<float>();
    a.wbf = s.wbf.as<__nv_bfloat16>();
    a.X = s.X.as<float>();
    a.idx = nullptr;
    a.n = n;
    a.off = 0;
    a.count = n;
    a.mu = s.mu.as<float>();
    a.logvar = s.lv.as<float>();
    k_mlp_tile<0><<<(n + S - 1) / S, H, smem_bytes(), ctx->stream>>>(a);
    CUDA_OR_FAIL(cudaGetLastError(), "predict kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_mu, s.mu.p, sizeof(float) * (size_t)n), "copy out");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_logvar, s.lv.p, sizeof(float) * (size_t)n), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

}  // extern "C"
