// Optical limit q -> 0 of the dielectric matrix (Appendix C): the momentum
// matrix elements <c k|grad|v k> of the Bloch sums and the G = 0 column of the
// pair densities that replaces rho_t(0)/|q| in the limit,
//
//   P_{mu nu}(k)  = sum_L e^{ik.L} int chi_mu(r - tau_mu) grad chi_nu(r - tau_nu - L) dr,
//   p_t           = <c k|grad|v k> = sum_{mu nu} conj(C_c[mu]) P_{mu nu}(k) C_v[nu],
//   rho~_t        = -i (qhat . p_t) / dE_t                 (Eq. (ol_overlap), m_e = 1),
//
// with v^1/2(0) |q| -> sqrt(4 pi), so that Eq. (RPA) with that column is the
// optical-limit matrix (head, wings and body) along qhat.
//
// Kernels:
//   k_momentum        one CTA per shell pair, one thread per k: the lattice sum of the
//                     closed-form one-dimensional overlap and derivative factors of the
//                     Cartesian s/p Gaussians (L kept where the Gaussian-product prefactor
//                     is at least e^{-46}), with the phase e^{ik.L};
//   k_momentum_elems  one CTA per k: Y = P C_v in shared memory, then p = C_c^H Y;
//   k_optical_column  rho~_t into the G = 0 row of the slot's pair densities (FP64 row or
//                     the three BF16 terms of the FP32 value), v^1/2 of that row set.
// All in FP64.
#include "qcx_internal.h"
#include "tc_ptx.cuh"

#include <cmath>
#include <vector>

namespace {

constexpr double kLatticeCut = 46.0;

struct MomPair {
    double A[3], B[3];        // centres (bohr)
    double ea, eb;            // exponents
    double r2;                // radius^2 of the kept lattice vectors around A - B
    int la, lb;               // 0 (s) or 1 (p)
    int mu0, nu0;             // first basis function of each shell
    int nmax[3];              // lattice box half widths
};

// the one-dimensional factors of one axis: S[i][j] = int (x-A)^i (x-B)^j e^{-a(x-A)^2 - b(x-B)^2}
// for i <= 1, j <= 2 without the Gaussian prefactor (applied once for the three axes), and
// D[i][j] = j S[i][j-1] - 2 b S[i][j+1] for j <= 1
__device__ __forceinline__ void axis_factors(double A, double B, double a, double b, double S[2][2], double D[2][2]) {
    const double p = a + b;
    const double P = (a * A + b * B) / p;
    const double PA = P - A, PB = P - B;
    const double m0 = sqrt(3.141592653589793 / p), m2 = m0 / (2.0 * p);
    const double s00 = m0, s01 = PB * m0, s02 = PB * PB * m0 + m2;
    const double s10 = PA * m0, s11 = PA * PB * m0 + m2, s12 = PA * PB * PB * m0 + 2.0 * PB * m2 + PA * m2;
    S[0][0] = s00;
    S[0][1] = s01;
    S[1][0] = s10;
    S[1][1] = s11;
    D[0][0] = -2.0 * b * s01;
    D[0][1] = s00 - 2.0 * b * s02;
    D[1][0] = -2.0 * b * s11;
    D[1][1] = s10 - 2.0 * b * s12;
}

__device__ __forceinline__ double prim_norm(double a, int l) {
    const double n = pow(2.0 * a / 3.141592653589793, 0.75);
    return l ? n * 2.0 * sqrt(a) : n;
}

// P[k][x][mu][nu] for the functions of one shell pair
__global__ void __launch_bounds__(128) k_momentum(const MomPair* pairs, double l00, double l01, double l02, double l10,
                                                  double l11, double l12, double l20, double l21, double l22, int nk,
                                                  const double* kpts, int nb, double2* P) {
    const MomPair pr = pairs[blockIdx.x];
    const int k = blockIdx.y * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const double kx = kpts[3 * k], ky = kpts[3 * k + 1], kz = kpts[3 * k + 2];
    const int na = pr.la ? 3 : 1, nbf = pr.lb ? 3 : 1;
    const double norm = prim_norm(pr.ea, pr.la) * prim_norm(pr.eb, pr.lb);
    const double mu_ab = pr.ea * pr.eb / (pr.ea + pr.eb);
    double2 acc[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int x = 0; x < 3; ++x) acc[i][j][x] = make_double2(0.0, 0.0);
    for (int n0 = -pr.nmax[0]; n0 <= pr.nmax[0]; ++n0)
        for (int n1 = -pr.nmax[1]; n1 <= pr.nmax[1]; ++n1)
            for (int n2 = -pr.nmax[2]; n2 <= pr.nmax[2]; ++n2) {
                const double Lx = n0 * l00 + n1 * l10 + n2 * l20;
                const double Ly = n0 * l01 + n1 * l11 + n2 * l21;
                const double Lz = n0 * l02 + n1 * l12 + n2 * l22;
                const double dx = pr.A[0] - pr.B[0] - Lx, dy = pr.A[1] - pr.B[1] - Ly, dz = pr.A[2] - pr.B[2] - Lz;
                const double d2 = dx * dx + dy * dy + dz * dz;
                if (d2 > pr.r2) continue;
                const double pref = norm * exp(-mu_ab * d2);
                double S[3][2][2], D[3][2][2];
                axis_factors(pr.A[0], pr.B[0] + Lx, pr.ea, pr.eb, S[0], D[0]);
                axis_factors(pr.A[1], pr.B[1] + Ly, pr.ea, pr.eb, S[1], D[1]);
                axis_factors(pr.A[2], pr.B[2] + Lz, pr.ea, pr.eb, S[2], D[2]);
                double sn, cs;
                sincos(kx * Lx + ky * Ly + kz * Lz, &sn, &cs);
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    if (i >= na) continue;
                    // angular momentum of function i of shell a along each axis
                    const int ia0 = pr.la && i == 0, ia1 = pr.la && i == 1, ia2 = pr.la && i == 2;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        if (j >= nbf) continue;
                        const int jb0 = pr.lb && j == 0, jb1 = pr.lb && j == 1, jb2 = pr.lb && j == 2;
                        const double sx = S[0][ia0][jb0], sy = S[1][ia1][jb1], sz = S[2][ia2][jb2];
                        const double v[3] = {pref * D[0][ia0][jb0] * sy * sz, pref * sx * D[1][ia1][jb1] * sz,
                                             pref * sx * sy * D[2][ia2][jb2]};
#pragma unroll
                        for (int x = 0; x < 3; ++x) {
                            acc[i][j][x].x += cs * v[x];
                            acc[i][j][x].y += sn * v[x];
                        }
                    }
                }
            }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int x = 0; x < 3; ++x)
                if (i < na && j < nbf) P[(((size_t)k * 3 + x) * nb + pr.mu0 + i) * nb + pr.nu0 + j] = acc[i][j][x];
}

// p[t][x] = <c k|d/dr_x|v k>, t = (k, v, c): Y = P(k) C_v in shared memory, then C_c^H Y
__global__ void __launch_bounds__(256) k_momentum_elems(int nb, int nv, int nc, const double2* P, const double2* Cv,
                                                        const double2* Cc, double2* p) {
    extern __shared__ double2 Y[];                 // [3][nb][nv]
    const int k = blockIdx.x;
    const double2* Pk = P + (size_t)k * 3 * nb * nb;
    const double2* Cvk = Cv + (size_t)k * nb * nv;
    const double2* Cck = Cc + (size_t)k * nb * nc;
    for (int i = threadIdx.x; i < 3 * nb * nv; i += blockDim.x) {
        const int v = i % nv, mu = (i / nv) % nb, x = i / (nv * nb);
        const double2* row = Pk + ((size_t)x * nb + mu) * nb;
        double2 s = make_double2(0.0, 0.0);
        for (int nu = 0; nu < nb; ++nu) {
            const double2 a = row[nu], b = Cvk[(size_t)nu * nv + v];
            s.x += a.x * b.x - a.y * b.y;
            s.y += a.x * b.y + a.y * b.x;
        }
        Y[i] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nv * nc * 3; i += blockDim.x) {
        const int x = i % 3, c = (i / 3) % nc, v = i / (3 * nc);
        double2 s = make_double2(0.0, 0.0);
        for (int mu = 0; mu < nb; ++mu) {
            const double2 a = Cck[(size_t)mu * nc + c], b = Y[((size_t)x * nb + mu) * nv + v];
            s.x += a.x * b.x + a.y * b.y;                 // conj(a) b
            s.y += a.x * b.y - a.y * b.x;
        }
        p[(((size_t)k * nv + v) * nc + c) * 3 + x] = s;
    }
}

// rho~_t = -i (qhat . p_t)/dE_t into row g0; status bit 1 where dE_t is zero
__global__ void k_optical_column(long long nt, int nv, int nc, const double* Ek, const double* Ekq, const double2* p,
                                 double q0, double q1, double q2, int g0, double2* R64, uint32_t* pl0, uint32_t* pl1,
                                 uint32_t* pl2, long long kp2, int* status) {
    const int nvc = nv * nc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / nvc;
        const int rem = (int)(t - k * nvc);
        const int v = rem / nc, c = rem - v * nc;
        const double dE = Ekq[k * nc + c] - Ek[k * nv + v];
        const double2 a0 = p[3 * t], a1 = p[3 * t + 1], a2 = p[3 * t + 2];
        const double ar = q0 * a0.x + q1 * a1.x + q2 * a2.x, ai = q0 * a0.y + q1 * a1.y + q2 * a2.y;
        double2 r = make_double2(0.0, 0.0);
        if (dE != 0.0) {
            r = make_double2(ai / dE, -ar / dE);
        } else {
            atomicOr(status, 1);
        }
        if (R64) {
            R64[(long long)g0 * nt + t] = r;
        } else {
            uint32_t u0, u1, u2;
            split3((float)r.x, (float)r.y, u0, u1, u2);
            const long long o = (long long)g0 * kp2 + t;
            pl0[o] = u0;
            pl1[o] = u1;
            pl2[o] = u2;
        }
    }
}

__global__ void k_set_head_vs(int g0, double* vs, float* vs32) {
    vs[g0] = QCX_SQRT_4PI;
    vs32[g0] = (float)QCX_SQRT_4PI;
}

}  // namespace

cudaError_t qcx_launch_optical(qcx_ctx* ctx, QSlot& s, int iq, int g0, const double qhat[3], qcx_precision prec,
                               int* d_status) {
    OpticalBufs& ob = ctx->optical;
    const int nk = ctx->nk, nb = ctx->nb, nv = ctx->nv, nc = ctx->nc;
    const long long nt = (long long)nk * nv * nc;
    cudaStream_t st = ctx->stream;
    cudaError_t e;
    if (ob.gen != ctx->gen || ob.nk != nk) {
        // shell pairs with their lattice boxes (the rule of the overlap's lattice sum)
        const double* Lm = ctx->lattice;
        const double det = Lm[0] * (Lm[4] * Lm[8] - Lm[5] * Lm[7]) - Lm[1] * (Lm[3] * Lm[8] - Lm[5] * Lm[6]) +
                           Lm[2] * (Lm[3] * Lm[7] - Lm[4] * Lm[6]);
        // rows of inv(lattice)^T: recip[i] . a_j = delta_ij
        double rc[3][3];
        rc[0][0] = (Lm[4] * Lm[8] - Lm[5] * Lm[7]) / det;
        rc[0][1] = (Lm[5] * Lm[6] - Lm[3] * Lm[8]) / det;
        rc[0][2] = (Lm[3] * Lm[7] - Lm[4] * Lm[6]) / det;
        rc[1][0] = (Lm[2] * Lm[7] - Lm[1] * Lm[8]) / det;
        rc[1][1] = (Lm[0] * Lm[8] - Lm[2] * Lm[6]) / det;
        rc[1][2] = (Lm[1] * Lm[6] - Lm[0] * Lm[7]) / det;
        rc[2][0] = (Lm[1] * Lm[5] - Lm[2] * Lm[4]) / det;
        rc[2][1] = (Lm[2] * Lm[3] - Lm[0] * Lm[5]) / det;
        rc[2][2] = (Lm[0] * Lm[4] - Lm[1] * Lm[3]) / det;
        std::vector<MomPair> pairs;
        const int ns = ctx->nshell;
        pairs.reserve((size_t)ns * ns);
        for (int a = 0; a < ns; ++a)
            for (int b = 0; b < ns; ++b) {
                MomPair pr;
                const double* A = &ctx->atom_xyz[3 * ctx->shell_atom[a]];
                const double* B = &ctx->atom_xyz[3 * ctx->shell_atom[b]];
                for (int x = 0; x < 3; ++x) {
                    pr.A[x] = A[x];
                    pr.B[x] = B[x];
                }
                pr.ea = ctx->shell_exp[a];
                pr.eb = ctx->shell_exp[b];
                pr.la = ctx->shell_l[a];
                pr.lb = ctx->shell_l[b];
                pr.mu0 = ctx->shell_mu0[a];
                pr.nu0 = ctx->shell_mu0[b];
                const double rad = std::sqrt(kLatticeCut * (pr.ea + pr.eb) / (pr.ea * pr.eb));
                pr.r2 = rad * rad;
                const double d[3] = {A[0] - B[0], A[1] - B[1], A[2] - B[2]};
                const double reach = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]) + rad;
                for (int i = 0; i < 3; ++i)
                    pr.nmax[i] =
                        (int)std::ceil(reach * std::sqrt(rc[i][0] * rc[i][0] + rc[i][1] * rc[i][1] + rc[i][2] * rc[i][2])) +
                        1;
                pairs.push_back(pr);
            }
        e = ob.pairs.ensure(sizeof(MomPair) * pairs.size());
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(ob.pairs.p, pairs.data(), sizeof(MomPair) * pairs.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return e;
        e = ob.P.ensure(sizeof(double2) * (size_t)nk * 3 * nb * nb);
        if (e != cudaSuccess) return e;
        k_momentum<<<dim3((unsigned)pairs.size(), (nk + 127) / 128), 128, 0, st>>>(
            ob.pairs.as<MomPair>(), Lm[0], Lm[1], Lm[2], Lm[3], Lm[4], Lm[5], Lm[6], Lm[7], Lm[8], nk,
            ctx->d_kpts.as<double>(), nb, ob.P.as<double2>());
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        ob.gen = ctx->gen;
        ob.nk = nk;
    }
    e = ob.p.ensure(sizeof(double2) * 3 * (size_t)nt);
    if (e != cudaSuccess) return e;
    const size_t ysm = sizeof(double2) * 3 * (size_t)nb * nv;
    if (ysm > 227 * 1024) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute((const void*)k_momentum_elems, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ysm);
    if (e != cudaSuccess) return e;
    k_momentum_elems<<<nk, 256, ysm, st>>>(nb, nv, nc, ob.P.as<double2>(), ctx->d_Ck64.as<double2>(),
                                          ctx->d_Ckq64.as<double2>() + (size_t)iq * nk * nb * nc, ob.p.as<double2>());
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    double2* R64 = nullptr;
    uint32_t *pl0 = nullptr, *pl1 = nullptr, *pl2 = nullptr;
    if (prec == QCX_FP64) {
        R64 = s.rho.as<double2>();
    } else {
        pl0 = reinterpret_cast<uint32_t*>(s.rho.p);
        pl1 = pl0 + (size_t)s.ngp * (s.kp / 2);
        pl2 = pl1 + (size_t)s.ngp * (s.kp / 2);
    }
    k_optical_column<<<(int)std::min<long long>((nt + 255) / 256, 16384), 256, 0, st>>>(
        nt, nv, nc, ctx->d_Ek.as<double>(), ctx->d_Ekq.as<double>() + (size_t)iq * nk * nc, ob.p.as<double2>(),
        qhat[0], qhat[1], qhat[2], g0, R64, pl0, pl1, pl2, s.kp / 2, d_status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_set_head_vs<<<1, 1, 0, st>>>(g0, s.vs.as<double>(), s.vs32.as<float>());
    return cudaGetLastError();
}
