// The surrogate route for the loss-function heads (no counterpart in the
// paper) and the cheap quantities it needs:
//
//  * qcx_head_nolfe: L_noLFE at the head, -Im 1/eps_00 with
//    eps_00 = 1 - v(q) chi0_00 (Eq. (eps_noLFE)): only rho_t(q + 0) is formed
//    (the pair-density kernel with one G) and chi0_00(w) =
//    2/(N_k V) sum_t W_t(w) |rho_t|^2 is one FP64 sum per frequency
//    (8 N_t flops per block instead of the 8 N_t N_G^2 of the Dyson route).
//  * qcx_surrogate_features: the network inputs (|q|/q_max, q/|q|,
//    w/w_max, ln(L_noLFE)/10).
//  * qcx_surrogate_heads: per (q, w) the network's (mu, s); the prediction
//    L_LFE = L_noLFE e^mu is accepted where sigma = e^(s/2) is below the
//    threshold; a seeded random fraction of the accepted samples is re-solved
//    by the Dyson route, and if any of them misses by more than the tolerance
//    in |log ratio| every sample of the call falls back; rejected samples are
//    always solved by the Dyson route (pair densities, chi0, inverse of the
//    per-q path, for just the frequencies that need it).
#include "qcx_internal.h"
#include "cplx.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

extern "C" qcx_status qcx_pair_density(qcx_ctx* ctx, int iq, int ng, const int* G_int, qcx_precision prec,
                                       qcx_c64* out_rho);
extern "C" qcx_status qcx_chi0(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, qcx_precision prec,
                               qcx_c64* out_chi0);
extern "C" qcx_status qcx_invert_eps(qcx_ctx* ctx, int iq, qcx_precision prec, qcx_c64* out_diag_inv,
                                     qcx_c64* out_eps_diag, double* out_resid);
extern "C" qcx_status qcx_mlp_predict(qcx_ctx* ctx, int n, const float* X, float* out_mu, float* out_logvar);

namespace {

constexpr int HC_THREADS = 256;

// chi0_00(w) for every frequency: one CTA per frequency, FP64 sum over t
__global__ void __launch_bounds__(HC_THREADS)
    k_head_chi(long long nt, int nv, int nc, const double* Ek, const double* Ekq, const double* w, double eta,
               const double2* rho, double pref, double vs0, double* out_L) {
    __shared__ double red[2][HC_THREADS / 32];
    const int iw = blockIdx.x;
    const double om = w[iw];
    const int nvc = nv * nc;
    double sr = 0.0, si = 0.0;
    for (long long t = threadIdx.x; t < nt; t += HC_THREADS) {
        const long long k = t / nvc;
        const int rem = (int)(t - k * nvc);
        const int v = rem / nc, c = rem - v * nc;
        const double dE = Ekq[k * nc + c] - Ek[k * nv + v];
        const double x1 = om - dE, x2 = om + dE;
        const double d1 = 1.0 / (x1 * x1 + eta * eta), d2 = 1.0 / (x2 * x2 + eta * eta);
        const double2 r = rho[t];
        const double m2 = r.x * r.x + r.y * r.y;
        sr = fma(x1 * d1 - x2 * d2, m2, sr);
        si = fma(eta * (d2 - d1), m2, si);
    }
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sr;
        red[1][threadIdx.x >> 5] = si;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        for (int i = 0; i < HC_THREADS / 32; ++i) {
            a += red[0][i];
            b += red[1][i];
        }
        const double v = vs0 * vs0 * pref;
        const double er = 1.0 - v * a, ei = -v * b;     // eps_00
        out_L[iw] = ei / (er * er + ei * ei);
    }
}

__global__ void k_features(int n, const double* q, const double* w, const double* L, double qmax, double wmax,
                           float* X, const double* L_lfe = nullptr, float* y = nullptr) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double qx = q[3 * i], qy = q[3 * i + 1], qz = q[3 * i + 2];
    const double qn = sqrt(qx * qx + qy * qy + qz * qz);
    float* x = X + 6 * (size_t)i;
    x[0] = (float)(qn / qmax);
    x[1] = (float)(qx / qn);
    x[2] = (float)(qy / qn);
    x[3] = (float)(qz / qn);
    x[4] = (float)(w[i] / wmax);
    x[5] = (float)(log(L[i]) / 10.0);
    if (y) y[i] = (float)log(L_lfe[i] / L[i]);     // training target log(L_LFE / L_noLFE)
}

double cell_volume(const double* L) {
    return std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                     L[2] * (L[3] * L[7] - L[4] * L[6]));
}

uint64_t splitmix(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// L_noLFE heads of q number iq for nw frequencies (device array d_w) into d_out
qcx_status head_nolfe_dev(qcx_ctx* ctx, int iq, int nw, const double* d_w, double eta, double* d_out) {
    const int G0[3] = {0, 0, 0};
    qcx_status st = qcx_pair_density(ctx, iq, 1, G0, QCX_FP64, nullptr);
    if (st != QCX_OK) return st;
    QSlot& s = ctx->slot[QCX_FP64];
    const double* q = &ctx->qpts[3 * iq];
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (!(qn > 0)) return ctx->fail(QCX_ERR_ARG, "head_nolfe: q = 0 needs the optical limit");
    const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    k_head_chi<<<nw, HC_THREADS, 0, ctx->stream>>>(nt, ctx->nv, ctx->nc, ctx->d_Ek.as<double>(),
                                                   ctx->d_Ekq.as<double>() + (size_t)iq * ctx->nk * ctx->nc, d_w,
                                                   eta, s.rho.as<double2>(), 2.0 / (ctx->nk * cell_volume(ctx->lattice)),
                                                   QCX_SQRT_4PI / qn, d_out);
    CUDA_OR_FAIL(cudaGetLastError(), "head chi0 kernel");
    // the slot now holds one G only: later per-q calls must recompute their pair densities
    s.have_rho = s.have_eps = false;
    s.iq = -1;
    return QCX_OK;
}

}  // namespace

extern "C" {

qcx_status qcx_head_nolfe(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, double* out_L_nolfe_head) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nq) return ctx->fail(QCX_ERR_STATE, "head_nolfe: no states");
    if (iq < 0 || iq >= ctx->nq || nw < 1 || !w || !out_L_nolfe_head || !(eta > 0) || !std::isfinite(eta))
        return ctx->fail(QCX_ERR_ARG, "head_nolfe: bad arguments");
    cudaSetDevice(ctx->device);
    // own buffer: the pair-density call below stages its G list in the context's scratch
    DevBuf buf;
    CUDA_OR_FAIL(buf.ensure(2 * sizeof(double) * nw), "alloc");
    double* d_w = buf.as<double>();
    CUDA_OR_FAIL(qcx_copy_in(ctx, d_w, w, sizeof(double) * nw), "copy w");
    qcx_status st = head_nolfe_dev(ctx, iq, nw, d_w, eta, d_w + nw);
    if (st != QCX_OK) return st;
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L_nolfe_head, d_w + nw, sizeof(double) * nw), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

qcx_status qcx_surrogate_features(qcx_ctx* ctx, int n, const double* qvec, const double* w, const double* L_nolfe,
                                  const double* L_lfe, double q_max, double w_max, float* out_X, float* out_y) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (n < 1 || !qvec || !w || !L_nolfe || !out_X || !(q_max > 0) || !(w_max > 0) || (!L_lfe != !out_y))
        return ctx->fail(QCX_ERR_ARG, "surrogate_features: bad arguments");
    cudaSetDevice(ctx->device);
    const size_t bq = 3 * sizeof(double) * n, bw = sizeof(double) * n, bx = 6 * sizeof(float) * n,
                 by = sizeof(float) * n;
    DevBuf buf;
    CUDA_OR_FAIL(buf.ensure(bq + 3 * bw + bx + by), "alloc");
    char* base = buf.as<char>();
    double* dq = reinterpret_cast<double*>(base);
    double* dw = reinterpret_cast<double*>(base + bq);
    double* dL = reinterpret_cast<double*>(base + bq + bw);
    double* dL1 = reinterpret_cast<double*>(base + bq + 2 * bw);
    float* X = reinterpret_cast<float*>(base + bq + 3 * bw);
    float* Y = reinterpret_cast<float*>(base + bq + 3 * bw + bx);
    CUDA_OR_FAIL(qcx_copy_in(ctx, dq, qvec, bq), "copy q");
    CUDA_OR_FAIL(qcx_copy_in(ctx, dw, w, bw), "copy w");
    CUDA_OR_FAIL(qcx_copy_in(ctx, dL, L_nolfe, bw), "copy L");
    if (L_lfe) CUDA_OR_FAIL(qcx_copy_in(ctx, dL1, L_lfe, bw), "copy L");
    k_features<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, dq, dw, dL, q_max, w_max, X, L_lfe ? dL1 : nullptr,
                                                         L_lfe ? Y : nullptr);
    CUDA_OR_FAIL(cudaGetLastError(), "features kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_X, X, bx), "copy out");
    if (out_y) CUDA_OR_FAIL(qcx_copy_out(ctx, out_y, Y, by), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

qcx_status qcx_surrogate_heads(qcx_ctx* ctx, int nsel, const int* iq_list, int ng, const int* G_int, int nw,
                               const double* w, double eta, qcx_precision fallback_prec,
                               const qcx_surrogate_opts* opts, double* out_L_lfe_head, double* out_L_nolfe_head,
                               int* out_source, double* out_check_err) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nq) return ctx->fail(QCX_ERR_STATE, "surrogate_heads: no states");
    if (!ctx->mlp) return ctx->fail(QCX_ERR_STATE, "surrogate_heads: no network parameters");
    if (nsel < 1 || !iq_list || ng < 1 || !G_int || nw < 1 || !w || !(eta > 0) || !opts || !out_L_lfe_head ||
        (fallback_prec != QCX_FP64 && fallback_prec != QCX_MIXED) || !(opts->q_max > 0) || !(opts->w_max > 0) ||
        !(opts->check_frac >= 0 && opts->check_frac <= 1) || !(opts->check_tol > 0))
        return ctx->fail(QCX_ERR_ARG, "surrogate_heads: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<int> iqs(iq_list, iq_list + nsel);
    std::vector<int> G(G_int, G_int + 3 * (size_t)ng);
    std::vector<double> wh(w, w + nw);
    int head = -1;
    for (int g = 0; g < ng; ++g)
        if (!G[3 * g] && !G[3 * g + 1] && !G[3 * g + 2]) head = g;
    if (head < 0) return ctx->fail(QCX_ERR_ARG, "surrogate_heads: G = 0 is not in the G list");
    for (int iq : iqs)
        if (iq < 0 || iq >= ctx->nq) return ctx->fail(QCX_ERR_ARG, "surrogate_heads: q index out of range");
    const size_t n = (size_t)nsel * nw;
    // 1) cheap heads, features, network
    DevBuf d_w, d_L, d_q, d_wall, d_X, d_mu, d_lv;
    CUDA_OR_FAIL(d_w.ensure(sizeof(double) * nw), "alloc");
    CUDA_OR_FAIL(d_L.ensure(sizeof(double) * n), "alloc");
    CUDA_OR_FAIL(d_q.ensure(3 * sizeof(double) * n), "alloc");
    CUDA_OR_FAIL(d_wall.ensure(sizeof(double) * n), "alloc");
    CUDA_OR_FAIL(d_X.ensure(6 * sizeof(float) * n), "alloc");
    CUDA_OR_FAIL(d_mu.ensure(sizeof(float) * n), "alloc");
    CUDA_OR_FAIL(d_lv.ensure(sizeof(float) * n), "alloc");
    CUDA_OR_FAIL(cudaMemcpyAsync(d_w.p, wh.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, ctx->stream), "copy");
    std::vector<double> qall(3 * n), wall(n);
    for (int s = 0; s < nsel; ++s) {
        qcx_status st = head_nolfe_dev(ctx, iqs[s], nw, d_w.as<double>(), eta, d_L.as<double>() + (size_t)s * nw);
        if (st != QCX_OK) return st;
        for (int j = 0; j < nw; ++j) {
            std::memcpy(&qall[3 * ((size_t)s * nw + j)], &ctx->qpts[3 * iqs[s]], 3 * sizeof(double));
            wall[(size_t)s * nw + j] = wh[j];
        }
    }
    CUDA_OR_FAIL(cudaMemcpyAsync(d_q.p, qall.data(), 3 * sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(d_wall.p, wall.data(), sizeof(double) * n, cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    k_features<<<(int)((n + 255) / 256), 256, 0, ctx->stream>>>((int)n, d_q.as<double>(), d_wall.as<double>(),
                                                                d_L.as<double>(), opts->q_max, opts->w_max,
                                                                d_X.as<float>());
    CUDA_OR_FAIL(cudaGetLastError(), "features kernel");
    qcx_status st = qcx_mlp_predict(ctx, (int)n, d_X.as<float>(), d_mu.as<float>(), d_lv.as<float>());
    if (st != QCX_OK) return st;
    std::vector<double> Lno(n);
    std::vector<float> mu(n), lv(n);
    CUDA_OR_FAIL(cudaMemcpyAsync(Lno.data(), d_L.p, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(mu.data(), d_mu.p, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(lv.data(), d_lv.p, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    // 2) acceptance and the spot check
    std::vector<int> src(n, 1);
    std::vector<size_t> acc;
    for (size_t i = 0; i < n; ++i) {
        const double sig = std::exp(0.5 * (double)lv[i]);
        if (std::isfinite(mu[i]) && sig < opts->sigma_accept && Lno[i] > 0 && std::isfinite(Lno[i])) {
            src[i] = 0;
            acc.push_back(i);
        }
    }
    size_t nchk = acc.empty() ? 0 : (size_t)std::ceil(opts->check_frac * (double)acc.size());
    uint64_t seed = opts->seed;
    for (size_t k = 0; k < nchk; ++k) {   // partial Fisher-Yates: the first nchk of a seeded shuffle
        const size_t j = k + (size_t)(splitmix(seed) % (uint64_t)(acc.size() - k));
        std::swap(acc[k], acc[j]);
        src[acc[k]] = 2;
    }
    std::vector<double> Lout(n, 0.0);
    // 3) the Dyson route for every sample with src != 0, one q at a time
    DevBuf d_diag;
    auto dyson = [&](void) -> qcx_status {
        for (int s = 0; s < nsel; ++s) {
            std::vector<int> js;
            for (int j = 0; j < nw; ++j)
                if (src[(size_t)s * nw + j] != 0 && Lout[(size_t)s * nw + j] == 0.0) js.push_back(j);
            if (js.empty()) continue;
            std::vector<double> wsub(js.size());
            for (size_t k = 0; k < js.size(); ++k) wsub[k] = wh[js[k]];
            qcx_status r = qcx_pair_density(ctx, iqs[s], ng, G.data(), fallback_prec, nullptr);
            if (r == QCX_OK) r = qcx_chi0(ctx, iqs[s], (int)js.size(), wsub.data(), eta, fallback_prec, nullptr);
            std::vector<double> dg(2 * js.size() * (size_t)ng);
            if (r == QCX_OK)
                r = qcx_invert_eps(ctx, iqs[s], fallback_prec, reinterpret_cast<qcx_c64*>(dg.data()), nullptr,
                                   nullptr);
            if (r != QCX_OK) return r;
            for (size_t k = 0; k < js.size(); ++k) Lout[(size_t)s * nw + js[k]] = -dg[2 * (k * ng + head) + 1];
        }
        return QCX_OK;
    };
    st = dyson();
    if (st != QCX_OK) return st;
    double chk = 0.0;
    for (size_t i = 0; i < n; ++i)
        if (src[i] == 2) chk = std::max(chk, std::fabs((double)mu[i] - std::log(Lout[i] / Lno[i])));
    if (nchk && !(chk <= opts->check_tol)) {
        for (size_t i = 0; i < n; ++i)
            if (src[i] == 0) src[i] = 1;
        st = dyson();
        if (st != QCX_OK) return st;
    }
    for (size_t i = 0; i < n; ++i)
        if (src[i] == 0) Lout[i] = Lno[i] * std::exp((double)mu[i]);
    // outputs (host or device)
    auto put = [&](void* dst, const void* srcp, size_t bytes) -> cudaError_t {
        if (!dst) return cudaSuccess;
        if (qcx_is_device_ptr(dst)) return cudaMemcpy(dst, srcp, bytes, cudaMemcpyHostToDevice);
        std::memcpy(dst, srcp, bytes);
        return cudaSuccess;
    };
    CUDA_OR_FAIL(put(out_L_lfe_head, Lout.data(), sizeof(double) * n), "copy out");
    CUDA_OR_FAIL(put(out_L_nolfe_head, Lno.data(), sizeof(double) * n), "copy out");
    CUDA_OR_FAIL(put(out_source, src.data(), sizeof(int) * n), "copy out");
    if (out_check_err) *out_check_err = nchk ? chk : -1.0;
    return QCX_OK;
}

}  // extern "C"
