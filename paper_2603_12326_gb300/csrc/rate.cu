// Momentum binning of the loss tables and the nonrelativistic halo rate.
//
// dR/dw = (rho_chi/m_chi)(1/rho_T) sigma_e/(8 pi^2 alpha mu^2)
//         int dq q^3 |F_DM(q)|^2 Im[-1/eps(w,q)] eta(v_min),   v_min = q/(2 m_chi) + w/q
// (end of Appendix A with Eqs. (general_rate), (v_min), (F_DM)); eta is the
// mean inverse speed above v_min of the truncated Maxwellian halo.  The
// recoil spectrum is Eq. (excitation_rate) with the step ionisation model.
// Everything here is FP64: the rate accumulates over q and w.
#include "qcx_internal.h"

namespace {

// CODATA 2018 and unit conversions (natural units, eV)
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kMe = 510998.95000;            // eV
constexpr double kHbarC = 1.973269804e-5;       // eV cm
constexpr double kHbar = 6.582119569e-16;       // eV s
constexpr double kC = 299792.458;               // km/s
constexpr double kEvPerKg = 5.609588603804452e35;
constexpr double kYear = 365.25 * 24.0 * 3600.0;
constexpr double kHartree = 27.211386245988;    // eV
constexpr double kAme = kAlpha * kMe;           // eV per bohr^-1
constexpr double kPi = 3.141592653589793;

// mean inverse speed above vmin of f ~ exp(-|v + vE|^2/v0^2), |v + vE| < vesc (units of c)
__device__ double eta_halo(double vmin, double v0, double vesc, double vE) {
    const double x = vmin / v0, y = vE / v0, z = vesc / v0;
    const double nesc = erf(z) - 2.0 / sqrt(kPi) * z * exp(-z * z);
    const double pref = 1.0 / (2.0 * nesc * v0 * y);
    if (x < z - y) return pref * (erf(x + y) - erf(x - y) - 4.0 / sqrt(kPi) * y * exp(-z * z));
    if (x < z + y) return pref * (erf(z) - erf(x - y) - 2.0 / sqrt(kPi) * (z + y - x) * exp(-z * z));
    return 0.0;
}

__global__ void k_rate(int nq, const double* q_bohr, int nw, const double* w_ha, const double* L,
                       qcx_halo_params p, double* dRdw) {
    const int iw = blockIdx.x * blockDim.x + threadIdx.x;
    if (iw >= nw) return;
    const double v0 = p.v0_kms / kC, vesc = p.vesc_kms / kC, vE = p.vE_kms / kC;
    const double n_chi = p.rho_chi_GeV_cm3 * 1e9 / p.m_chi_eV * kHbarC * kHbarC * kHbarC;
    const double rho_T = p.rho_T_g_cm3 * kEvPerKg * 1e-3 * kHbarC * kHbarC * kHbarC;
    const double sigma = p.sigma_e_cm2 / (kHbarC * kHbarC);
    const double mu = p.m_chi_eV * kMe / (p.m_chi_eV + kMe);
    const double pref = n_chi / rho_T * sigma / (8.0 * kPi * kPi * kAlpha * mu * mu);
    const double wv = w_ha[iw] * kHartree;
    double acc = 0.0, gprev = 0.0, qprev = 0.0;
    for (int i = 0; i < nq; ++i) {
        const double qv = q_bohr[i] * kAme;
        double F2 = 1.0;
        if (p.m_med_eV >= 0.0) {
            const double f = (kAme * kAme + p.m_med_eV * p.m_med_eV) / (qv * qv + p.m_med_eV * p.m_med_eV);
            F2 = f * f;
        }
        const double vmin = qv / (2.0 * p.m_chi_eV) + wv / qv;
        const double g = qv * qv * qv * F2 * L[(size_t)i * nw + iw] * eta_halo(vmin, v0, vesc, vE);
        if (i > 0) acc += 0.5 * (g + gprev) * (qv - qprev);
        gprev = g;
        qprev = qv;
    }
    dRdw[iw] = pref * acc * kEvPerKg * (kYear / kHbar);
}

__global__ void k_recoil(int nw, const double* w_ha, const double* dRdw, double wgap, double wpp, int nQ,
                         double* out) {
    const int Q = blockIdx.x * blockDim.x + threadIdx.x + 1;
    if (Q > nQ) return;
    const double dw = (w_ha[1] - w_ha[0]) * kHartree;
    double acc = 0.0;
    for (int i = 0; i < nw; ++i) {
        const double wv = w_ha[i] * kHartree;
        if (wv < wgap) continue;
        const int Qi = 1 + (int)floor((wv - wgap) / wpp);
        if (Qi == Q) acc += dRdw[i] * dw;
    }
    out[Q - 1] = acc;
}

// out[bin][w] = mean over (q, G) with |q+G| in [edges[bin], edges[bin+1]) of L[which][w][G]
__global__ void k_bin(int nsel, const double* const* Ls, const double* const* qm, const int* ngs, int nw,
                      int which, int nbin, const double* edges, double* out, double* cnt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nbin * nw) return;
    const int bin = id / nw, iw = id - bin * nw;
    const double lo = edges[bin], hi = edges[bin + 1];
    double s = 0.0;
    int c = 0;
    for (int q = 0; q < nsel; ++q) {
        const int ng = ngs[q];
        const double* Lq = Ls[q] + ((size_t)which * nw + iw) * ng;
        for (int g = 0; g < ng; ++g) {
            const double m = qm[q][g];
            if (m >= lo && m < hi) {
                s += Lq[g];
                ++c;
            }
        }
    }
    out[id] = c ? s / c : 0.0;
    if (iw == 0) cnt[bin] = (double)c;
}

}  // namespace

cudaError_t qcx_launch_bin(qcx_ctx* ctx, int nsel, const double* const* d_L, const double* const* d_qmag,
                           const int* d_ng, int nw, int which, int nbin, const double* d_edges, double* d_out,
                           double* d_cnt) {
    const int n = nbin * nw;
    k_bin<<<(n + 127) / 128, 128, 0, ctx->stream>>>(nsel, d_L, d_qmag, d_ng, nw, which, nbin, d_edges, d_out,
                                                   d_cnt);
    return cudaGetLastError();
}

cudaError_t qcx_launch_recoil(cudaStream_t st, int nw, const double* d_w, const double* d_dRdw, double wgap_eV,
                              double wpp_eV, int nQ, double* d_dRQ) {
    k_recoil<<<(nQ + 63) / 64, 64, 0, st>>>(nw, d_w, d_dRdw, wgap_eV, wpp_eV, nQ, d_dRQ);
    return cudaGetLastError();
}

cudaError_t qcx_launch_rate(qcx_ctx* ctx, int nqbin, const double* d_q, int nw, const double* d_w,
                            const double* d_L, const qcx_halo_params& p, double* d_dRdw, int nQ,
                            double* d_dRQ) {
    k_rate<<<(nw + 127) / 128, 128, 0, ctx->stream>>>(nqbin, d_q, nw, d_w, d_L, p, d_dRdw);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || nQ <= 0) return e;
    k_recoil<<<(nQ + 63) / 64, 64, 0, ctx->stream>>>(nw, d_w, d_dRdw, p.w_gap_eV, p.w_pp_eV, nQ, d_dRQ);
    return cudaGetLastError();
}
