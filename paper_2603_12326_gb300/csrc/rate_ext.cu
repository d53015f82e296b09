// The rate end of the path beyond the |q+G| binning of rate.cu:
//  * the composite dielectric function (Eq. (e_comp)) of every stored q binned
//    in three-dimensional momentum space (spherical shells of width dq split
//    into N_theta x N_phi angular cells), empty bins filled by linear
//    interpolation in |q| between the nearest filled shells of the same cell;
//  * the isotropic loss function of such tables with the screening choices of
//    Section IV.C (Eq. (ELF_screening) with eps itself, 1, the modified
//    Thomas-Fermi model of Eq. (MTF) or the Lindhard function of Eq. (Lindhard));
//  * the general rate for a velocity flux with vector or scalar mediators
//    (Eqs. (general_rate), (H), (cross_section_iso), (v_min)), its recoil
//    spectrum (Eq. (excitation_rate)) and the reach (the cross section giving
//    a set number of events in an exposure).
// All of it in FP64.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <cmath>
#include <cstring>

namespace {

constexpr double kAlpha = 1.0 / 137.035999084;   // CODATA 2018
constexpr double kMe = 510998.95000;             // eV
constexpr double kHbarC = 1.973269804e-5;        // eV cm
constexpr double kHbar = 6.582119569e-16;        // eV s
constexpr double kEvPerKg = 5.609588603804452e35;
constexpr double kYear = 365.25 * 24.0 * 3600.0;
constexpr double kHartree = 27.211386245988;     // eV
constexpr double kAme = kAlpha * kMe;            // eV per bohr^-1
constexpr double kPi = 3.141592653589793;

__device__ __forceinline__ double2 cdiv1(double2 z) {       // 1 / z
    const double d = 1.0 / (z.x * z.x + z.y * z.y);
    return make_double2(z.x * d, -z.y * d);
}

// eps^LFE = 1/(Re [eps^-1]_GG - i L_LFE) (the stored loss keeps the imaginary part at full
// accuracy on the mixed path), eps^noLFE = eps_GG; out [2][nw][ng]
__global__ void k_store_eps(int n, const double2* dinv, const double2* ed, const double* L, double2* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        out[i] = cdiv1(make_double2(dinv[i].x, -L[i]));
        out[n + i] = ed[i];
    }
}

struct Bin3 {
    int nshell, nth, nph;
    double dq;
};

// (shell, theta cell, phi cell) flattened, or -1
__device__ int bin3_index(const double* k, const Bin3& b) {
    const double kk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    if (!(kk > 0.0)) return -1;
    const int s = (int)floor(kk / b.dq);
    if (s >= b.nshell) return -1;
    const double th = acos(fmax(-1.0, fmin(1.0, k[2] / kk)));
    const int it = min(b.nth - 1, (int)floor(th * b.nth / kPi));
    double ph = atan2(k[1], k[0]);
    if (ph < 0.0) ph += 2.0 * kPi;
    const int ip = min(b.nph - 1, (int)floor(ph * b.nph / (2.0 * kPi)));
    return (s * b.nth + it) * b.nph + ip;
}

// one thread per (selected q, G): sums of eps^comp over w and the count of its bin
__global__ void k_bin3d(int nsel, const double* const* kvec, const double2* const* eps, const int* ngs, int ngmax,
                        int nw, double q_lfe, Bin3 b, double2* sums, double* cnt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nsel * ngmax) return;
    const int q = id / ngmax, g = id - q * ngmax;
    const int ng = ngs[q];
    if (g >= ng) return;
    const double* k = kvec[q] + 3 * (size_t)g;
    const int bi = bin3_index(k, b);
    if (bi < 0) return;
    const double kk = sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
    // composite: the local-field value up to q_lfe, the diagonal one above (Eq. (e_comp))
    const double2* src = eps[q] + (kk <= q_lfe ? 0 : (size_t)nw * ng);
    atomicAdd(&cnt[bi], 1.0);
    for (int iw = 0; iw < nw; ++iw) {
        const double2 e = src[(size_t)iw * ng + g];
        atomicAdd(&sums[(size_t)bi * nw + iw].x, e.x);
        atomicAdd(&sums[(size_t)bi * nw + iw].y, e.y);
    }
}

__global__ void k_bin3d_mean(int nbin, int nw, double2* sums, const double* cnt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= nbin * nw) return;
    const double c = cnt[id / nw];
    if (c > 0.0) sums[id] = make_double2(sums[id].x / c, sums[id].y / c);
}

// one thread per (angular cell, w): empty shells between filled ones take the linear interpolation
// in |q| of the nearest filled shells; the w = 0 thread marks them (count -1)
__global__ void k_fill3d(Bin3 b, int nw, double2* eps, double* cnt) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    const int ncell = b.nth * b.nph;
    if (id >= ncell * nw) return;
    const int cell = id / nw, iw = id - cell * nw;
    int prev = -1;
    for (int s = 0; s < b.nshell; ++s) {
        const size_t bs = (size_t)s * ncell + cell;
        if (!(cnt[bs] > 0.0)) continue;
        if (prev >= 0 && s > prev + 1) {
            const double2 e0 = eps[((size_t)prev * ncell + cell) * nw + iw];
            const double2 e1 = eps[bs * nw + iw];
            for (int t = prev + 1; t < s; ++t) {
                const double x = (double)(t - prev) / (double)(s - prev);
                eps[((size_t)t * ncell + cell) * nw + iw] =
                    make_double2((1.0 - x) * e0.x + x * e1.x, (1.0 - x) * e0.y + x * e1.y);
                if (iw == 0) cnt[(size_t)t * ncell + cell] = -1.0;
            }
        }
        prev = s;
    }
}

// ----------------------------------------------------------- screening models
__device__ __forceinline__ double2 cmulz(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 clog(double2 z) {           // principal branch
    return make_double2(log(sqrt(z.x * z.x + z.y * z.y)), atan2(z.y, z.x));
}

// eps_MTF (Eq. (MTF)), real; w, q in eV
__device__ double eps_mtf(double w, double q, const qcx_screening& s) {
    const double d = 1.0 / (s.eps0 - 1.0) + s.tau * (q / s.qtf_eV) * (q / s.qtf_eV) +
                     q * q * q * q / (4.0 * kMe * kMe * s.wp_eV * s.wp_eV) - (w / s.wp_eV) * (w / s.wp_eV);
    return 1.0 + 1.0 / d;
}

// eps_Lindhard (Eq. (Lindhard)) of an electron gas of density ne (eV^3); w, q in eV
__device__ double2 eps_lindhard(double w, double q, double ne, double fp) {
    const double qf = cbrt(3.0 * kPi * kPi * ne);
    const double vf = qf / kMe;
    const double wp = sqrt(4.0 * kPi * kAlpha * ne / kMe);
    const double a = q / (2.0 * qf);
    const double2 b = make_double2(w / (q * vf), fp * wp / (q * vf));
    double2 tot = make_double2(0.5, 0.0);
    for (int sgn = 0; sgn < 2; ++sgn) {
        const double2 Q = sgn == 0 ? make_double2(a + b.x, b.y) : make_double2(a - b.x, -b.y);
        const double2 num = make_double2(Q.x + 1.0, Q.y), den = make_double2(Q.x - 1.0, Q.y);
        const double dd = 1.0 / (den.x * den.x + den.y * den.y);
        const double2 ratio = make_double2((num.x * den.x + num.y * den.y) * dd, (num.y * den.x - num.x * den.y) * dd);
        const double2 Q2 = cmulz(Q, Q);
        const double2 t = cmulz(make_double2(1.0 - Q2.x, -Q2.y), clog(ratio));
        const double c = qf / (4.0 * q);
        tot.x += c * t.x;
        tot.y += c * t.y;
    }
    const double f = 3.0 * wp * wp / (q * q * vf * vf);
    return make_double2(1.0 + f * tot.x, f * tot.y);
}

// one thread per (shell, w): mean over the cells with count != 0 of Im eps / |eps_scr|^2
__global__ void k_loss_iso(Bin3 b, int nw, const double* w_ha, const double2* eps, const double* cnt,
                           qcx_screening scr, double ne_ev3, double* L, double* ncell_out) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= b.nshell * nw) return;
    const int s = id / nw, iw = id - s * nw;
    const int ncell = b.nth * b.nph;
    const double qs = (s + 0.5) * b.dq * kAme, wv = w_ha[iw] * kHartree;
    double den_model = 1.0;
    if (scr.model == QCX_SCREEN_MTF) {
        const double e = eps_mtf(wv, qs, scr);
        den_model = e * e;
    } else if (scr.model == QCX_SCREEN_LINDHARD) {
        const double2 e = eps_lindhard(wv, qs, ne_ev3, scr.fp);
        den_model = e.x * e.x + e.y * e.y;
    }
    double acc = 0.0;
    int nc = 0;
    for (int c = 0; c < ncell; ++c) {
        const size_t bi = (size_t)s * ncell + c;
        if (cnt[bi] == 0.0) continue;
        const double2 e = eps[bi * nw + iw];
        const double den = scr.model == QCX_SCREEN_SELF ? e.x * e.x + e.y * e.y : den_model;
        acc += e.y / den;
        ++nc;
    }
    L[id] = nc ? acc / nc : 0.0;
    if (iw == 0) ncell_out[s] = nc;
}

// ----------------------------------------------------------------- general rate
struct RateArgs {
    int nq, nw, nv;
    const double* q;      // bohr^-1
    const double* w;      // Hartree
    const double* L;      // [nq][nw]
    const double* v;      // units of c
    const double* flux;   // 1/(cm^2 s) per unit v
    qcx_rate_params p;
    double* dRdw;
};

constexpr int RATE_THREADS = 256;

// trapezoid weight of node i of an ascending grid x[0..n)
__device__ __forceinline__ double trap_w(const double* x, int i, int n) {
    const double lo = i > 0 ? x[i] - x[i - 1] : 0.0, hi = i + 1 < n ? x[i + 1] - x[i] : 0.0;
    return 0.5 * (lo + hi);
}

// one block per w: threads over the velocity nodes, the q integral per node, a fixed-order reduction
__global__ void __launch_bounds__(RATE_THREADS) k_rate_general(RateArgs a) {
    const int iw = blockIdx.x;
    const double m = a.p.m_chi_eV;
    const double mu = m * kMe / (m + kMe);
    const double sigma = a.p.sigma_e_cm2 / (kHbarC * kHbarC);
    const double rho_T = a.p.rho_T_g_cm3 * kEvPerKg * 1e-3 * kHbarC * kHbarC * kHbarC;
    const double flux_unit = kHbarC * kHbarC * kHbar;                  // 1/(cm^2 s) in eV^3
    const double wv = a.w[iw] * kHartree;
    double part = 0.0;
    for (int iv = threadIdx.x; iv < a.nv; iv += RATE_THREADS) {
        const double vv = a.v[iv];
        if (!(vv > 0.0 && vv < 1.0)) continue;
        const double gam = 1.0 / sqrt(1.0 - vv * vv);
        const double E = gam * m, Ep = E - wv;
        if (!(Ep > m)) continue;
        double qint = 0.0;
        for (int iq = 0; iq < a.nq; ++iq) {
            const double qv = a.q[iq] * kAme;
            const double vmin = qv / (2.0 * gam * m) + wv / qv;
            if (vv < vmin) continue;
            const double H = a.p.mediator == 0 ? (E + Ep) * (E + Ep) - qv * qv
                                               : 4.0 * m * m - (E - Ep) * (E - Ep) + qv * qv;
            double F = 1.0;
            if (a.p.m_med_eV >= 0.0) {
                const double mm = a.p.m_med_eV * a.p.m_med_eV;
                const double num = mm + kAme * kAme, den = wv * wv - qv * qv - mm;
                F = num * num / (den * den);
            }
            const double S = qv * qv * a.L[(size_t)iq * a.nw + iw] / (2.0 * kPi * kAlpha);
            qint += trap_w(a.q, iq, a.nq) * kAme * qv * H * F * S / (vv * vv);
        }
        part += trap_w(a.v, iv, a.nv) * a.flux[iv] * flux_unit * sigma / (16.0 * kPi * mu * mu) / (E * Ep) * qint;
    }
    __shared__ double red[RATE_THREADS];
    red[threadIdx.x] = part;
    __syncthreads();
    for (int h = RATE_THREADS / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x == 0) a.dRdw[iw] = red[0] / rho_T * kEvPerKg * (kYear / kHbar);
}

// reach[Q - 1] = n_events sigma_e / (exposure sum_{Q' >= Q} dR_Q'), infinite where the tail is 0
__global__ void k_reach(int nQ, const double* dRQ, double sigma, double exposure, double nev, double* out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double tail = 0.0;
    for (int Q = nQ - 1; Q >= 0; --Q) {
        tail += dRQ[Q];
        out[Q] = tail > 0.0 ? nev * sigma / (exposure * tail) : INFINITY;
    }
}

}  // namespace

cudaError_t qcx_launch_store_eps(cudaStream_t st, int nw, int ng, const double2* diag_inv, const double2* eps_diag,
                                 const double* L_lfe, double2* out) {
    const int n = nw * ng;
    k_store_eps<<<(n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096, 256, 0, st>>>(n, diag_inv, eps_diag, L_lfe, out);
    return cudaGetLastError();
}

namespace {

inline int nblk(size_t n, int t) { return (int)((n + t - 1) / t); }

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

}  // namespace

extern "C" {

qcx_status qcx_bin_eps3d(qcx_ctx* ctx, int nsel, const int* iq_list, double q_lfe, int nshell, double dq,
                         int n_theta, int n_phi, int fill, qcx_c64* out_eps, double* out_count) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (nsel < 1 || !iq_list || nshell < 1 || n_theta < 1 || n_phi < 1 || !finite_pos(dq) || std::isnan(q_lfe) ||
        !out_eps || (long long)nshell * n_theta * n_phi > (1ll << 26))
        return ctx->fail(QCX_ERR_ARG, "bin_eps3d: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<int> iqs;
    CUDA_OR_FAIL(fetch(ctx, iqs, iq_list, nsel), "bin_eps3d iq list");
    std::vector<const double*> kp(nsel);
    std::vector<const double2*> ep(nsel);
    std::vector<int> ngs(nsel);
    int nw = -1, ngmax = 0;
    const std::vector<double>* wref = nullptr;
    for (int i = 0; i < nsel; ++i) {
        const int iq = iqs[i];
        if (iq < 0 || iq >= ctx->nq || !ctx->loss[iq] || !ctx->loss[iq]->valid)
            return ctx->fail(QCX_ERR_STATE, "bin_eps3d: q not inverted");
        LossTab* lt = ctx->loss[iq];
        if (nw < 0) {
            nw = lt->nw;
            wref = &lt->w;
        } else if (lt->nw != nw || lt->w != *wref) {
            return ctx->fail(QCX_ERR_ARG, "bin_eps3d: q tables use different frequency grids");
        }
        kp[i] = lt->kvec.as<double>();
        ep[i] = lt->eps.as<double2>();
        ngs[i] = lt->ng;
        ngmax = std::max(ngmax, lt->ng);
    }
    const size_t nbin = (size_t)nshell * n_theta * n_phi;
    const size_t off_k = 0, off_e = nsel * sizeof(void*), off_n = 2 * nsel * sizeof(void*);
    const size_t off_c = (off_n + nsel * sizeof(int) + 15) / 16 * 16;
    const size_t off_s = (off_c + nbin * sizeof(double) + 15) / 16 * 16;
    const size_t total = off_s + nbin * nw * sizeof(double2);
    CUDA_OR_FAIL(ctx->scratch2.ensure(total), "alloc");
    char* base = ctx->scratch2.as<char>();
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_k, kp.data(), nsel * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_e, ep.data(), nsel * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_n, ngs.data(), nsel * sizeof(int), cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    double* cnt = reinterpret_cast<double*>(base + off_c);
    double2* sums = reinterpret_cast<double2*>(base + off_s);
    CUDA_OR_FAIL(cudaMemsetAsync(cnt, 0, nbin * sizeof(double), ctx->stream), "clear");
    CUDA_OR_FAIL(cudaMemsetAsync(sums, 0, nbin * nw * sizeof(double2), ctx->stream), "clear");
    Bin3 b{nshell, n_theta, n_phi, dq};
    const size_t nth = (size_t)nsel * ngmax;
    k_bin3d<<<nblk(nth, 128), 128, 0, ctx->stream>>>(nsel, reinterpret_cast<const double* const*>(base + off_k),
                                                     reinterpret_cast<const double2* const*>(base + off_e),
                                                     reinterpret_cast<const int*>(base + off_n), ngmax, nw, q_lfe, b,
                                                     sums, cnt);
    k_bin3d_mean<<<nblk(nbin * nw, 256), 256, 0, ctx->stream>>>((int)nbin, nw, sums, cnt);
    if (fill) k_fill3d<<<nblk((size_t)n_theta * n_phi * nw, 128), 128, 0, ctx->stream>>>(b, nw, sums, cnt);
    CUDA_OR_FAIL(cudaGetLastError(), "bin_eps3d kernels");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_eps, sums, nbin * nw * sizeof(double2)), "copy out");
    if (out_count) CUDA_OR_FAIL(qcx_copy_out(ctx, out_count, cnt, nbin * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

qcx_status qcx_loss_isotropic(qcx_ctx* ctx, int nshell, int n_theta, int n_phi, int nw, const double* w, double dq,
                              const qcx_c64* eps, const double* count, const qcx_screening* scr, double* out_L,
                              double* out_ncell) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (nshell < 1 || n_theta < 1 || n_phi < 1 || nw < 1 || !w || !finite_pos(dq) || !eps || !count || !scr ||
        !out_L || (long long)nshell * n_theta * n_phi > (1ll << 26))
        return ctx->fail(QCX_ERR_ARG, "loss_isotropic: bad arguments");
    const qcx_screening s = *scr;
    if (s.model < QCX_SCREEN_SELF || s.model > QCX_SCREEN_LINDHARD)
        return ctx->fail(QCX_ERR_ARG, "loss_isotropic: unknown screening model");
    if (s.model == QCX_SCREEN_MTF && !(s.eps0 > 1.0 && finite_pos(s.wp_eV) && finite_pos(s.qtf_eV) && s.tau >= 0.0))
        return ctx->fail(QCX_ERR_ARG, "loss_isotropic: MTF parameters");
    if (s.model == QCX_SCREEN_LINDHARD && !(finite_pos(s.ne_bohr3) && finite_pos(s.fp)))
        return ctx->fail(QCX_ERR_ARG, "loss_isotropic: Lindhard parameters (density and f_p > 0)");
    cudaSetDevice(ctx->device);
    const size_t nbin = (size_t)nshell * n_theta * n_phi;
    const size_t oe = 0, oc = nbin * nw * sizeof(double2), ow = oc + nbin * sizeof(double);
    const size_t oL = ow + nw * sizeof(double), on = oL + (size_t)nshell * nw * sizeof(double);
    const size_t total = on + nshell * sizeof(double);
    CUDA_OR_FAIL(ctx->scratch2.ensure(total), "alloc");
    char* base = ctx->scratch2.as<char>();
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oe, eps, nbin * nw * sizeof(double2)), "copy eps");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oc, count, nbin * sizeof(double)), "copy count");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + ow, w, nw * sizeof(double)), "copy w");
    Bin3 b{nshell, n_theta, n_phi, dq};
    const double ne_ev3 = s.ne_bohr3 * kAme * kAme * kAme;
    k_loss_iso<<<nblk((size_t)nshell * nw, 128), 128, 0, ctx->stream>>>(
        b, nw, reinterpret_cast<const double*>(base + ow), reinterpret_cast<const double2*>(base + oe),
        reinterpret_cast<const double*>(base + oc), s, ne_ev3, reinterpret_cast<double*>(base + oL),
        reinterpret_cast<double*>(base + on));
    CUDA_OR_FAIL(cudaGetLastError(), "loss_isotropic kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L, base + oL, (size_t)nshell * nw * sizeof(double)), "copy out");
    if (out_ncell) CUDA_OR_FAIL(qcx_copy_out(ctx, out_ncell, base + on, nshell * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

qcx_status qcx_rate_general(qcx_ctx* ctx, int nqbin, const double* qbin, int nw, const double* w, const double* L,
                            int nv, const double* v, const double* dphidv, const qcx_rate_params* params,
                            double* out_dRdw, int nQ, double* out_dRQ, double* out_reach) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (nqbin < 2 || nw < 2 || nv < 2 || !qbin || !w || !L || !v || !dphidv || !params || !out_dRdw || nQ < 0 ||
        (nQ > 0 && !out_dRQ))
        return ctx->fail(QCX_ERR_ARG, "rate_general: bad arguments");
    const qcx_rate_params p = *params;
    if (!finite_pos(p.m_chi_eV) || !finite_pos(p.rho_T_g_cm3) || !finite_pos(p.w_pp_eV) ||
        (p.mediator != 0 && p.mediator != 1) || std::isnan(p.m_med_eV))
        return ctx->fail(QCX_ERR_ARG, "rate_general: non-physical parameters");
    if (out_reach && !(nQ > 0 && finite_pos(p.exposure_kg_yr) && finite_pos(p.n_events)))
        return ctx->fail(QCX_ERR_ARG, "rate_general: reach needs nQ > 0, an exposure and an event count");
    cudaSetDevice(ctx->device);
    const size_t oq = 0, ow = nqbin * sizeof(double), oL = ow + nw * sizeof(double);
    const size_t ov = oL + (size_t)nqbin * nw * sizeof(double), of = ov + nv * sizeof(double);
    const size_t oR = of + nv * sizeof(double), oQ = oR + nw * sizeof(double);
    const size_t oX = oQ + (nQ > 0 ? nQ : 1) * sizeof(double), total = oX + (nQ > 0 ? nQ : 1) * sizeof(double);
    CUDA_OR_FAIL(ctx->scratch2.ensure(total), "alloc");
    char* base = ctx->scratch2.as<char>();
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oq, qbin, nqbin * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + ow, w, nw * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oL, L, (size_t)nqbin * nw * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + ov, v, nv * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + of, dphidv, nv * sizeof(double)), "copy");
    RateArgs a{nqbin, nw, nv, reinterpret_cast<double*>(base + oq), reinterpret_cast<double*>(base + ow),
               reinterpret_cast<double*>(base + oL), reinterpret_cast<double*>(base + ov),
               reinterpret_cast<double*>(base + of), p, reinterpret_cast<double*>(base + oR)};
    k_rate_general<<<nw, RATE_THREADS, 0, ctx->stream>>>(a);
    CUDA_OR_FAIL(cudaGetLastError(), "rate kernel");
    if (nQ > 0) {
        CUDA_OR_FAIL(qcx_launch_recoil(ctx->stream, nw, a.w, a.dRdw, p.w_gap_eV, p.w_pp_eV, nQ,
                                       reinterpret_cast<double*>(base + oQ)),
                     "recoil kernel");
        if (out_reach) {
            k_reach<<<1, 32, 0, ctx->stream>>>(nQ, reinterpret_cast<double*>(base + oQ), p.sigma_e_cm2,
                                               p.exposure_kg_yr, p.n_events, reinterpret_cast<double*>(base + oX));
            CUDA_OR_FAIL(cudaGetLastError(), "reach kernel");
        }
    }
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_dRdw, base + oR, nw * sizeof(double)), "copy out");
    if (nQ > 0) CUDA_OR_FAIL(qcx_copy_out(ctx, out_dRQ, base + oQ, nQ * sizeof(double)), "copy out");
    if (out_reach) CUDA_OR_FAIL(qcx_copy_out(ctx, out_reach, base + oX, nQ * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

}  // extern "C"
