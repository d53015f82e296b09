// Plain FP64 path of Eq. (RPA):
//   chi0_GG'(w) = 2/(N_k V) sum_t W_t(w) conj(rho_t(G)) rho_t(G'),
//   W_t(w) = 1/(w - dE_t + i eta) - 1/(w + dE_t + i eta),  dE_t = E_c(k+q) - E_v(k),
// and the Dyson step eps = 1 - v^1/2 chi0 v^1/2 fused in the epilogue.
//
// Tiling: one CTA owns a 32 x 32 (G, G') tile for 4 frequencies; each of the
// 256 threads accumulates 2 x 2 x 4 complex entries in registers.  The
// transition axis is streamed through shared memory 16 at a time; the
// product conj(rho_G) rho_G' is formed once per t and reused for the 4
// frequencies.  The kernel is bound by the FP64 pipe.
#include "qcx_internal.h"
#include "cplx.cuh"

namespace {

constexpr int TG = 32;   // G tile
constexpr int TK = 16;   // transitions per stage
constexpr int TW = 4;    // frequencies per CTA

struct Chi64Args {
    const double2* R;     // [ng][nt]
    long long nt;
    int ng, nw, nv, nc;
    const double* Ek;     // [nk][nv]
    const double* Ekq;    // [nk][nc]
    const double* w;      // [nw]
    double eta, pref;
    const double* vs;     // [ng]
    double2* eps;         // [nw][ng][ng]
    double2* chi;         // optional [nw][ng][ng]
};

__device__ __forceinline__ double2 weight(double om, double dE, double eta) {
    const double a = om - dE, b = om + dE;
    const double d1 = 1.0 / (a * a + eta * eta), d2 = 1.0 / (b * b + eta * eta);
    return make_double2(a * d1 - b * d2, eta * (d2 - d1));
}

__global__ void __launch_bounds__(256) k_chi0_fp64(Chi64Args a) {
    __shared__ double2 As[TK][TG + 1];
    __shared__ double2 Bs[TK][TG + 1];
    __shared__ double2 Ws[TW][TK];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int G0 = blockIdx.y * TG, H0 = blockIdx.x * TG, W0 = blockIdx.z * TW;
    double2 acc[TW][2][2];
#pragma unroll
    for (int w = 0; w < TW; ++w)
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < 2; ++j) acc[w][i][j] = make_double2(0.0, 0.0);

    const int nvc = a.nv * a.nc;
    for (long long t0 = 0; t0 < a.nt; t0 += TK) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = threadIdx.x + 256 * r;
            const int tt = i & (TK - 1), gg = i >> 4;
            const long long t = t0 + tt;
            double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
            if (t < a.nt) {
                if (G0 + gg < a.ng) {
                    va = a.R[(long long)(G0 + gg) * a.nt + t];
                    va.y = -va.y;
                }
                if (H0 + gg < a.ng) vb = a.R[(long long)(H0 + gg) * a.nt + t];
            }
            As[tt][gg] = va;
            Bs[tt][gg] = vb;
        }
        if (threadIdx.x < TW * TK) {
            const int ww = threadIdx.x / TK, tt = threadIdx.x % TK;
            const long long t = t0 + tt;
            double2 wt = make_double2(0.0, 0.0);
            if (t < a.nt && W0 + ww < a.nw) {
                const long long k = t / nvc;
                const int rem = (int)(t - k * nvc);
                const int v = rem / a.nc, c = rem - v * a.nc;
                const double dE = a.Ekq[k * a.nc + c] - a.Ek[k * a.nv + v];
                wt = weight(a.w[W0 + ww], dE, a.eta);
            }
            Ws[ww][tt] = wt;
        }
        __syncthreads();
#pragma unroll 4
        for (int tt = 0; tt < TK; ++tt) {
            const double2 a0 = As[tt][ty], a1 = As[tt][ty + 16];
            const double2 b0 = Bs[tt][tx], b1 = Bs[tt][tx + 16];
            double2 p[2][2];
            p[0][0] = cmul(a0, b0);
            p[0][1] = cmul(a0, b1);
            p[1][0] = cmul(a1, b0);
            p[1][1] = cmul(a1, b1);
#pragma unroll
            for (int w = 0; w < TW; ++w) {
                const double2 wt = Ws[w][tt];
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int j = 0; j < 2; ++j) cfma(acc[w][i][j], wt, p[i][j]);
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int w = 0; w < TW; ++w) {
        const int iw = W0 + w;
        if (iw >= a.nw) continue;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int G = G0 + ty + 16 * i;
            if (G >= a.ng) continue;
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                const int H = H0 + tx + 16 * j;
                if (H >= a.ng) continue;
                const double2 ch = make_double2(a.pref * acc[w][i][j].x, a.pref * acc[w][i][j].y);
                const double vv = a.vs[G] * a.vs[H];
                const long long o = ((long long)iw * a.ng + G) * a.ng + H;
                a.eps[o] = make_double2((G == H ? 1.0 : 0.0) - vv * ch.x, -vv * ch.y);
                if (a.chi) a.chi[o] = ch;
            }
        }
    }
}

}  // namespace

cudaError_t qcx_launch_chi0_fp64(qcx_ctx* ctx, QSlot& s, int iq, double2* d_chi0_out) {
    Chi64Args a;
    a.R = s.rho.as<double2>();
    a.nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    a.ng = s.ng;
    a.nw = s.nw;
    a.nv = ctx->nv;
    a.nc = ctx->nc;
    a.Ek = ctx->d_Ek.as<double>();
    a.Ekq = ctx->d_Ekq.as<double>() + (size_t)iq * ctx->nk * ctx->nc;
    a.w = s.w.as<double>();
    a.eta = s.eta;
    const double* L = ctx->lattice;
    const double vol = fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                            L[2] * (L[3] * L[7] - L[4] * L[6]));
    a.pref = 2.0 / (ctx->nk * vol);
    a.vs = s.vs.as<double>();
    a.eps = s.eps.as<double2>();
    a.chi = d_chi0_out;
    dim3 grid((s.ng + TG - 1) / TG, (s.ng + TG - 1) / TG, (s.nw + TW - 1) / TW);
    k_chi0_fp64<<<grid, 256, 0, ctx->stream>>>(a);
    return cudaGetLastError();
}
