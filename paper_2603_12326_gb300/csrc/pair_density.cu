// Pair densities rho_vck(q+G) = <c,k+q| e^{i(q+G).r} |v,k>  (Eq. (RPA) matrix
// elements; Bloch form of Appendix C) for Bloch sums of normalised Cartesian
// s/p Gaussians.
//
// Per (k, G) and shell pair (a on centre A, b on centre B):
//   B_ab(k; kappa) = sum_L e^{ik.L} int chi_a(r-A) e^{i kappa.r} chi_b(r-B-L) dr.
// With the Gaussian product theorem every term is a product over the three
// Cartesian axes.  The lattice is a sublattice of index m of h Z^3, so the
// sum over L is (1/m) sum_chi sum_{n in Z^3} chi(n) F(h n), and the Z^3 sum of
// a product is the product of three one-dimensional sums.  Per axis
//   sum_n e^{i theta n} w_n d_n^j ,  d_n = A_x - B_x - h n,  w_n = e^{-mu d_n^2},
//   theta = (k_x + (beta/p) kappa_x) h + 2 pi chi_x,   j = 0, 1, 2,
// gives the one-dimensional factors E(l_a, l_b) of the closed form
// (E(0,0) = 1, E(1,0) = PA + i kappa/2p, E(0,1) = PB + i kappa/2p,
//  E(1,1) = PA PB + (PA + PB) i kappa/2p + 1/2p - kappa^2/4p^2 with
//  PA = -(beta/p) d, PB = (alpha/p) d).
// Shells on the same centre with the same exponent (an s and a p shell) form
// one group, so the one-dimensional sums are formed once per group pair and
// give all 16 s/p components.  The contraction rho = C_kq^H B C_k runs in
// shared memory per (k, G).
#include "qcx_internal.h"
#include "cplx.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int PD_THREADS = 256;
constexpr int PDF_MAXT = 384;          // threads of the fused mixed-path kernel at most
constexpr double LATTICE_CUT = 46.0;   // Gaussian prefactors below e^-46 ~ 1e-20 are dropped

template <typename T> struct PDArgs {
    int nb, nv, nc, nk, ng, nt, ldB, ngrp;
    int row_s0[65];          // group row blocks: groups [row_s0[i], row_s0[i+1])
    int nblk;
    int max_rows;            // rows of the largest block (Bs holds max_rows * ldB entries)
    int g_per_cta;
    T h;
    T charre[4][3], charim[4][3];   // e^{2 pi i chi_x} per character and axis
    const int* grp_mu0;      // first basis function of each group (ngrp + 1 entries)
    const int* grp_mask;     // bit 0: has s, bit 1: has p
    const int* dir_off;      // [npair][3]
    const int* dir_cnt;
    const int* dir_nlo;
    const T* par;            // [npair][8]
    const cplx<T>* tab;      // terms {w_n, d_n}
    const T* kpts;           // [nk][3]
    const T* kappa;          // [ng][3]
    const cplx<T>* Ck;       // [nk][nb][nv]
    const cplx<T>* Ckq;      // [nk][nb][nc]
    double2* R64;            // FP64 output [ng][nt]
    __nv_bfloat162* R0;      // MIXED output: three BF16 planes [ngp][kp/2] (pairs re, im),
    __nv_bfloat162* R1;      // x = x0 + x1 + x2 with x0 = bf16(x), x1 = bf16(x - x0),
    __nv_bfloat162* R2;      // x2 = bf16(x - x0 - x1)
    long long kp2;           // row length of the BF16 planes in bf16x2 units
    cplx<T>* Sout;           // overlap mode: [nk][nb][nb]
    // tables of the mixed path (PdTab): one-dimensional factors per (pair, axis, k class, q+G
    // class) and the factor of (pair, G)
    const float2* ptab;      // [entries][NCH][4]
    const float2* pcmn;      // [npair][ng]
    const int* kidx;         // [nk][3]
    const int* gidx;         // [ng][3]
    int nkx[3], nqx[3];
    long long tbase[4];
};

// z^n for integer n (|n| small) by repeated squaring
template <typename C> __device__ __forceinline__ C cpow_int(C z, int n) {
    C r;
    r.x = 1;
    r.y = 0;
    int m = n < 0 ? -n : n;
    C b = z;
    while (m) {
        if (m & 1) r = cmul(r, b);
        b = cmul(b, b);
        m >>= 1;
    }
    if (n < 0) r.y = -r.y;     // |z| = 1: z^-n = conj(z^n)
    return r;
}

template <typename T, int NCH>
__device__ __forceinline__ void assemble_block(const PDArgs<T>& a, int ga, int gb, T p, T ap, T bp,
                                               const cplx<T>& common, const cplx<T> (&E)[3][NCH][4],
                                               cplx<T> (&out)[4][4]);

// One group pair's 4 x 4 block of B (components s, p_x, p_y, p_z of each group;
// absent components are left unset).
template <typename T, int NCH>
__device__ __forceinline__ void pair_block_vals(const PDArgs<T>& a, int ip, const T kk[3], const T kap[3], T k2,
                                                cplx<T> (&out)[4][4]) {
    using C = cplx<T>;
    const int ga = ip / a.ngrp, gb = ip % a.ngrp;
    const T* par = a.par + (size_t)ip * 8;
    const T p = par[0], ap = par[1], bp = par[2], pref = par[3];
    const T inv2p = T(0.5) / p;
    T s, c;
    sincos_t(kap[0] * par[4] + kap[1] * par[5] + kap[2] * par[6], &s, &c);
    const T amp = pref * exp_t(-k2 * T(0.25) / p) / T(NCH);
    const C common = mk<T>(amp * c, amp * s);

    C E[3][NCH][4];      // per axis and character: E(0,0), E(1,0), E(0,1), E(1,1)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const int di = ip * 3 + x;
        const int off = a.dir_off[di], cnt = a.dir_cnt[di], nlo = a.dir_nlo[di];
        const T theta = (kk[x] + bp * kap[x]) * a.h;
        const T tk = kap[x] * inv2p;
        T zs, zc;
        sincos_t(theta, &zs, &zc);
        const C z = mk<T>(zc, zs);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const C zch = ch ? cmul(z, mk<T>(a.charre[ch][x], a.charim[ch][x])) : z;
            C zn = cpow_int(zch, nlo);
            C M0 = mk<T>(0, 0), M1 = mk<T>(0, 0), M2 = mk<T>(0, 0);
            for (int j = 0; j < cnt; ++j) {
                const C wd = a.tab[off + j];
                const C t0 = cscale(zn, wd.x);
                M0 = cadd(M0, t0);
                const C t1 = cscale(t0, wd.y);
                M1 = cadd(M1, t1);
                M2 = cadd(M2, cscale(t1, wd.y));
                zn = cmul(zn, zch);
            }
            const C itkM0 = mk<T>(-tk * M0.y, tk * M0.x);
            const C itkM1 = mk<T>(-tk * M1.y, tk * M1.x);
            E[x][ch][0] = M0;
            E[x][ch][1] = cadd(cscale(M1, -bp), itkM0);                       // E(1,0)
            E[x][ch][2] = cadd(cscale(M1, ap), itkM0);                        // E(0,1)
            E[x][ch][3] = cadd(cadd(cscale(M2, -ap * bp), cscale(itkM1, ap - bp)),
                               cscale(M0, inv2p - tk * tk));                  // E(1,1)
        }
    }
    assemble_block<T, NCH>(a, ga, gb, p, ap, bp, common, E, out);
}

// The 4 x 4 block from the one-dimensional factors of the three axes: component (ca, cb) takes
// per axis the factor of its Cartesian powers, summed over the characters, times the common factor
// and the p normalisations.
template <typename T, int NCH>
__device__ __forceinline__ void assemble_block(const PDArgs<T>& a, int ga, int gb, T p, T ap, T bp,
                                               const cplx<T>& common, const cplx<T> (&E)[3][NCH][4],
                                               cplx<T> (&out)[4][4]) {
    using C = cplx<T>;
    // components: 0 = s, 1..3 = p_x, p_y, p_z
    const int ma = a.grp_mask[ga], mb = a.grp_mask[gb];
    const T fa = T(2) * sqrt(ap * p), fb = T(2) * sqrt(bp * p);   // p normalisation 2 sqrt(alpha)
#pragma unroll
    for (int ca = 0; ca < 4; ++ca) {
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
            const bool oka = ca == 0 ? (ma & 1) : (ma & 2);
            const bool okb = cb == 0 ? (mb & 1) : (mb & 2);
            if (oka && okb) {
                C val = mk<T>(0, 0);
#pragma unroll
                for (int ch = 0; ch < NCH; ++ch) {
                    C prod = E[0][ch][(ca == 1) + 2 * (cb == 1)];
                    prod = cmul(prod, E[1][ch][(ca == 2) + 2 * (cb == 2)]);
                    prod = cmul(prod, E[2][ch][(ca == 3) + 2 * (cb == 3)]);
                    val = cadd(val, prod);
                }
                const T f = (ca ? fa : T(1)) * (cb ? fb : T(1));
                out[ca][cb] = cscale(cmul(common, val), f);
            }
        }
    }
}

// One group pair's block of B into shared memory (row offset row0); present
// components map to consecutive basis rows and columns.
template <typename T, int NCH>
__device__ __forceinline__ void pair_block(const PDArgs<T>& a, int ip, const T kk[3], const T kap[3], T k2,
                                           cplx<T>* Bs, int row0) {
    cplx<T> blk[4][4];
    pair_block_vals<T, NCH>(a, ip, kk, kap, k2, blk);
    const int ga = ip / a.ngrp, gb = ip % a.ngrp;
    const int ma = a.grp_mask[ga], mb = a.grp_mask[gb];
    const int mu0 = a.grp_mu0[ga] - row0 - ((ma & 1) ? 0 : 1);
    const int nu0 = a.grp_mu0[gb] - ((mb & 1) ? 0 : 1);
#pragma unroll
    for (int ca = 0; ca < 4; ++ca)
#pragma unroll
        for (int cb = 0; cb < 4; ++cb) {
            const bool oka = ca == 0 ? (ma & 1) : (ma & 2);
            const bool okb = cb == 0 ? (mb & 1) : (mb & 2);
            if (oka && okb) Bs[(mu0 + ca) * a.ldB + nu0 + cb] = blk[ca][cb];
        }
}

// (re, im) of one FP32 pair density -> the three BF16 terms of each part, x = x0 + x1 + x2 with
// x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1) (round to nearest), written to the
// three planes
__device__ __forceinline__ void store_split3(float re, float im, __nv_bfloat162* R0, __nv_bfloat162* R1,
                                             __nv_bfloat162* R2, long long o) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(re, im);
    const float2 hf = __bfloat1622float2(h);
    const float rr = re - hf.x, ri = im - hf.y;
    const __nv_bfloat162 m = __floats2bfloat162_rn(rr, ri);
    const float2 mf = __bfloat1622float2(m);
    R0[o] = h;
    R1[o] = m;
    R2[o] = __floats2bfloat162_rn(rr - mf.x, ri - mf.y);
}

// Arguments of the table kernels (arithmetic in T, FP32 results).
template <typename T> struct PdTabArgs {
    const T* par;            // [npair][8]
    const cplx<T>* tab;      // lattice terms {w_n, d_n}
    const int* dir_off;
    const int* dir_cnt;
    const int* dir_nlo;
    T h;
    T charre[4][3], charim[4][3];
    const double* kval;      // k classes, axes concatenated
    const double* qval;      // q+G classes, axes concatenated
    const T* kappa;          // [ng][3] q + G
    int nkx[3], nqx[3], kofs[3], qofs[3];
    long long tbase[4];
    int npair, ng;
    float2* out;             // [entries][NCH][4]
    float2* cmn;             // [npair][ng]
};

// One entry of the one-dimensional table: for shell-group pair ip, axis x, the k component of
// class ik and the q+G component of class iq, the factors E(0,0), E(1,0), E(0,1), E(1,1) of every
// character, by the lattice sum of pair_block_vals (same operations, same order) in T.
template <typename T, int NCH> __global__ void k_pd_axis_table(PdTabArgs<T> a) {
    using C = cplx<T>;
    const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (e >= a.tbase[3]) return;
    const int x = e < a.tbase[1] ? 0 : (e < a.tbase[2] ? 1 : 2);
    long long r = e - a.tbase[x];
    const int iq = (int)(r % a.nqx[x]);
    r /= a.nqx[x];
    const int ik = (int)(r % a.nkx[x]);
    const int ip = (int)(r / a.nkx[x]);
    const T kk = (T)a.kval[a.kofs[x] + ik], kap = (T)a.qval[a.qofs[x] + iq];
    const T* par = a.par + (size_t)ip * 8;
    const T p = par[0], ap = par[1], bp = par[2];
    const T inv2p = T(0.5) / p;
    const int di = ip * 3 + x;
    const int off = a.dir_off[di], cnt = a.dir_cnt[di], nlo = a.dir_nlo[di];
    const T theta = (kk + bp * kap) * a.h;
    const T tk = kap * inv2p;
    T zs, zc;
    sincos_t(theta, &zs, &zc);
    const C z = mk<T>(zc, zs);
    float4* out = reinterpret_cast<float4*>(a.out + e * (NCH * 4));
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
        const C zch = ch ? cmul(z, mk<T>(a.charre[ch][x], a.charim[ch][x])) : z;
        C zn = cpow_int(zch, nlo);
        C M0 = mk<T>(0, 0), M1 = mk<T>(0, 0), M2 = mk<T>(0, 0);
        for (int j = 0; j < cnt; ++j) {
            const C wd = a.tab[off + j];
            const C t0 = cscale(zn, wd.x);
            M0 = cadd(M0, t0);
            const C t1 = cscale(t0, wd.y);
            M1 = cadd(M1, t1);
            M2 = cadd(M2, cscale(t1, wd.y));
            zn = cmul(zn, zch);
        }
        const C itkM0 = mk<T>(-tk * M0.y, tk * M0.x);
        const C itkM1 = mk<T>(-tk * M1.y, tk * M1.x);
        const C e10 = cadd(cscale(M1, -bp), itkM0);
        const C e01 = cadd(cscale(M1, ap), itkM0);
        const C e11 = cadd(cadd(cscale(M2, -ap * bp), cscale(itkM1, ap - bp)), cscale(M0, inv2p - tk * tk));
        out[2 * ch] = make_float4((float)M0.x, (float)M0.y, (float)e10.x, (float)e10.y);
        out[2 * ch + 1] = make_float4((float)e01.x, (float)e01.y, (float)e11.x, (float)e11.y);
    }
}

// The factor of pair ip and G: pref e^{-|q+G|^2/4p} e^{i (q+G).P} / (number of characters), in T.
template <typename T, int NCH> __global__ void k_pd_common(PdTabArgs<T> a) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)a.npair * a.ng) return;
    const int ip = (int)(i / a.ng), g = (int)(i - (long long)ip * a.ng);
    const T* par = a.par + (size_t)ip * 8;
    const T kap[3] = {a.kappa[3 * g], a.kappa[3 * g + 1], a.kappa[3 * g + 2]};
    const T k2 = kap[0] * kap[0] + kap[1] * kap[1] + kap[2] * kap[2];
    T s, c;
    sincos_t(kap[0] * par[4] + kap[1] * par[5] + kap[2] * par[6], &s, &c);
    const T amp = par[3] * exp_t(-k2 * T(0.25) / par[0]) / T(NCH);
    a.cmn[i] = make_float2((float)(amp * c), (float)(amp * s));
}

// One group pair's block from the tables (k classes kx, q+G classes gx of this thread's G).
template <int NCH>
__device__ __forceinline__ void pair_block_tab(const PDArgs<float>& a, int ip, int ga, int gb, const int (&kx)[3],
                                               const int (&gx)[3], int g, cplx<float> (&out)[4][4]) {
    using C = cplx<float>;
    const float* par = a.par + (size_t)ip * 8;
    const float2 cm = a.pcmn[(size_t)ip * a.ng + g];
    C E[3][NCH][4];
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const float4* src = reinterpret_cast<const float4*>(
            a.ptab + (a.tbase[x] + ((long long)ip * a.nkx[x] + kx[x]) * a.nqx[x] + gx[x]) * (NCH * 4));
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch) {
            const float4 u = src[2 * ch], v = src[2 * ch + 1];
            E[x][ch][0] = mk<float>(u.x, u.y);
            E[x][ch][1] = mk<float>(u.z, u.w);
            E[x][ch][2] = mk<float>(v.x, v.y);
            E[x][ch][3] = mk<float>(v.z, v.w);
        }
    }
    assemble_block<float, NCH>(a, ga, gb, par[0], par[1], par[2], mk<float>(cm.x, cm.y), E, out);
}

template <typename T, int NCH>
__global__ void __launch_bounds__(PD_THREADS) k_pair_density(PDArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Bs = reinterpret_cast<C*>(smem_raw);        // [max_rows][ldB]
    C* Cks = Bs + (size_t)a.max_rows * a.ldB;      // [nb][nv]
    C* Ys = Cks + (size_t)a.nb * a.nv;             // [nb][nv]

    const int k = blockIdx.x;
    for (int i = threadIdx.x; i < a.nb * a.nv; i += blockDim.x) Cks[i] = a.Ck[(size_t)k * a.nb * a.nv + i];
    const T kk[3] = {a.kpts[3 * k], a.kpts[3 * k + 1], a.kpts[3 * k + 2]};
    const C* Ckq = a.Ckq + (size_t)k * a.nb * a.nc;
    const int g0 = blockIdx.y * a.g_per_cta;
    const int g1 = min(a.ng, g0 + a.g_per_cta);

    for (int g = g0; g < g1; ++g) {
        const T kap[3] = {a.kappa[3 * g], a.kappa[3 * g + 1], a.kappa[3 * g + 2]};
        const T k2 = kap[0] * kap[0] + kap[1] * kap[1] + kap[2] * kap[2];
        for (int blk = 0; blk < a.nblk; ++blk) {
            const int s0 = a.row_s0[blk], s1 = a.row_s0[blk + 1];
            const int row0 = a.grp_mu0[s0];
            const int row1 = a.grp_mu0[s1];
            __syncthreads();  // Bs free, Cks staged
            const int p0 = s0 * a.ngrp, p1 = s1 * a.ngrp;
            for (int ip = p0 + threadIdx.x; ip < p1; ip += blockDim.x) pair_block<T, NCH>(a, ip, kk, kap, k2, Bs, row0);
            __syncthreads();
            const int rows = row1 - row0;
            for (int i = threadIdx.x; i < rows * a.nv; i += blockDim.x) {
                const int r = i / a.nv, v = i - r * a.nv;
                C acc = mk<T>(0, 0);
                const C* brow = Bs + (size_t)r * a.ldB;
                for (int nu = 0; nu < a.nb; ++nu) cfma(acc, brow[nu], Cks[nu * a.nv + v]);
                Ys[(row0 + r) * a.nv + v] = acc;
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < a.nv * a.nc; i += blockDim.x) {
            const int v = i / a.nc, c = i - v * a.nc;
            C acc = mk<T>(0, 0);
            for (int mu = 0; mu < a.nb; ++mu) cfmac(acc, Ckq[mu * a.nc + c], Ys[mu * a.nv + v]);
            const long long t = ((long long)k * a.nv + v) * a.nc + c;
            if (a.R64) {
                a.R64[(long long)g * a.nt + t] = make_double2((double)acc.x, (double)acc.y);
            } else {
                store_split3((float)acc.x, (float)acc.y, a.R0, a.R1, a.R2, (long long)g * a.kp2 + t);
            }
        }
    }
}

// Mixed path, fused: one thread per (G, group a) walks every group b, forms the
// 4 x 4 pair block in registers and adds it straight into its rows of
// Y = B C_k (NV >= nv columns in registers), so B never goes through shared
// memory.  Threads are ordered G fastest, so a warp holds one or two groups a
// and every thread of it runs the same pair's lattice sums.  Y then goes to
// shared memory and rho = C_kq^H Y is formed per (G, v, c).  The sums run in
// the same order as in k_pair_density.  With the tables of PdTab (TAB) the
// one-dimensional lattice sums and the (pair, G) factor are read, not formed
// per (k, G).
template <int NV> constexpr int pdf_maxt() { return NV <= 4 ? PDF_MAXT : (NV <= 8 ? 256 : 192); }

// TAB: the one-dimensional factors and the common factor come from the tables of this q (PdTab)
// instead of being formed per (k, G).
template <int NCH, int NV, bool TAB>
__global__ void __launch_bounds__(pdf_maxt<NV>()) k_pair_density_fused(PDArgs<float> a) {
    using C = cplx<float>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int nb = a.nb, nv = a.nv, nc = a.nc, gc = a.g_per_cta;
    C* Cks = reinterpret_cast<C*>(smem_raw);       // [nb][nv]
    C* Ckqs = Cks + (size_t)nb * nv;               // [nb][nc]
    C* Ys = Ckqs + (size_t)nb * nc;                // [gc][nb][nv]
    const int k = blockIdx.x;
    const int g0 = blockIdx.y * gc;
    const int ngl = min(gc, a.ng - g0);
    for (int i = threadIdx.x; i < nb * nv; i += blockDim.x) Cks[i] = a.Ck[(size_t)k * nb * nv + i];
    for (int i = threadIdx.x; i < nb * nc; i += blockDim.x) Ckqs[i] = a.Ckq[(size_t)k * nb * nc + i];
    const float kk[3] = {a.kpts[3 * k], a.kpts[3 * k + 1], a.kpts[3 * k + 2]};
    __syncthreads();

    const int ga = threadIdx.x / gc, gl = threadIdx.x - ga * gc;
    if (ga < a.ngrp && gl < ngl) {
        const int g = g0 + gl;
        const float kap[3] = {a.kappa[3 * g], a.kappa[3 * g + 1], a.kappa[3 * g + 2]};
        const float k2 = kap[0] * kap[0] + kap[1] * kap[1] + kap[2] * kap[2];
        int kx[3] = {0, 0, 0}, gx[3] = {0, 0, 0};
        if (TAB) {
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                kx[x] = a.kidx[3 * k + x];
                gx[x] = a.gidx[3 * g + x];
            }
        }
        C Y[4][NV];
#pragma unroll
        for (int ca = 0; ca < 4; ++ca)
#pragma unroll
            for (int v = 0; v < NV; ++v) Y[ca][v] = mk<float>(0, 0);
        for (int gb = 0; gb < a.ngrp; ++gb) {
            C blk[4][4];
            if (TAB)
                pair_block_tab<NCH>(a, ga * a.ngrp + gb, ga, gb, kx, gx, g, blk);
            else
                pair_block_vals<float, NCH>(a, ga * a.ngrp + gb, kk, kap, k2, blk);
            const int mb = a.grp_mask[gb];
            const int nu0 = a.grp_mu0[gb] - ((mb & 1) ? 0 : 1);
#pragma unroll
            for (int cb = 0; cb < 4; ++cb) {
                if (!(cb == 0 ? (mb & 1) : (mb & 2))) continue;
                const C* ck = Cks + (size_t)(nu0 + cb) * nv;
#pragma unroll
                for (int v = 0; v < NV; ++v) {
                    if (v < nv) {
                        const C c = ck[v];
#pragma unroll
                        for (int ca = 0; ca < 4; ++ca) cfma(Y[ca][v], blk[ca][cb], c);
                    }
                }
            }
        }
        const int ma = a.grp_mask[ga];
        const int mu0 = a.grp_mu0[ga] - ((ma & 1) ? 0 : 1);
        C* yrow = Ys + (size_t)gl * nb * nv;
#pragma unroll
        for (int ca = 0; ca < 4; ++ca) {
            if (!(ca == 0 ? (ma & 1) : (ma & 2))) continue;
#pragma unroll
            for (int v = 0; v < NV; ++v)
                if (v < nv) yrow[(size_t)(mu0 + ca) * nv + v] = Y[ca][v];
        }
    }
    __syncthreads();
    const int nvc = nv * nc;
    for (int i = threadIdx.x; i < ngl * nvc; i += blockDim.x) {
        const int l = i / nvc, rem = i - l * nvc;
        const int v = rem / nc, c = rem - v * nc;
        const C* yv = Ys + (size_t)l * nb * nv + v;
        C acc = mk<float>(0, 0);
        for (int mu = 0; mu < nb; ++mu) cfmac(acc, Ckqs[mu * nc + c], yv[(size_t)mu * nv]);
        const long long t = ((long long)k * nv + v) * nc + c;
        store_split3(acc.x, acc.y, a.R0, a.R1, a.R2, (long long)(g0 + l) * a.kp2 + t);
    }
}

// S(k) = B(k; 0): one CTA per k, full matrix written to Sout.
template <typename T, int NCH>
__global__ void __launch_bounds__(PD_THREADS) k_overlap(PDArgs<T> a) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Bs = reinterpret_cast<C*>(smem_raw);
    const int k = blockIdx.x;
    const T kk[3] = {a.kpts[3 * k], a.kpts[3 * k + 1], a.kpts[3 * k + 2]};
    const T kap[3] = {0, 0, 0};
    for (int blk = 0; blk < a.nblk; ++blk) {
        const int s0 = a.row_s0[blk], s1 = a.row_s0[blk + 1];
        const int row0 = a.grp_mu0[s0];
        const int row1 = a.grp_mu0[s1];
        __syncthreads();
        for (int ip = s0 * a.ngrp + threadIdx.x; ip < s1 * a.ngrp; ip += blockDim.x)
            pair_block<T, NCH>(a, ip, kk, kap, T(0), Bs, row0);
        __syncthreads();
        for (int i = threadIdx.x; i < (row1 - row0) * a.nb; i += blockDim.x) {
            const int r = i / a.nb, nu = i - r * a.nb;
            a.Sout[((size_t)k * a.nb + row0 + r) * a.nb + nu] = Bs[(size_t)r * a.ldB + nu];
        }
    }
}

__global__ void k_qsetup(const int* G, int ng, double q0, double q1, double q2, double b00, double b01,
                         double b02, double b10, double b11, double b12, double b20, double b21, double b22,
                         double* kappa, float* kappa32, double* vs, float* vs32) {
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ng; g += gridDim.x * blockDim.x) {
        const double n0 = G[3 * g], n1 = G[3 * g + 1], n2 = G[3 * g + 2];
        const double x = q0 + n0 * b00 + n1 * b10 + n2 * b20;
        const double y = q1 + n0 * b01 + n1 * b11 + n2 * b21;
        const double z = q2 + n0 * b02 + n1 * b12 + n2 * b22;
        kappa[3 * g] = x;
        kappa[3 * g + 1] = y;
        kappa[3 * g + 2] = z;
        kappa32[3 * g] = (float)x;
        kappa32[3 * g + 1] = (float)y;
        kappa32[3 * g + 2] = (float)z;
        const double v = QCX_SQRT_4PI / sqrt(x * x + y * y + z * z);
        vs[g] = v;
        vs32[g] = (float)v;
    }
}

template <typename T> void fill_common(qcx_ctx* ctx, PDArgs<T>& a) {
    a.nb = ctx->nb;
    a.ngrp = ctx->ngrp;
    a.h = (T)ctx->h;
    for (int c = 0; c < 4; ++c)
        for (int x = 0; x < 3; ++x) {
            a.charre[c][x] = (T)cos(2.0 * M_PI * ctx->chars[c][x]);
            a.charim[c][x] = (T)sin(2.0 * M_PI * ctx->chars[c][x]);
        }
    a.grp_mu0 = ctx->d_grp_mu0.as<int>();
    a.grp_mask = ctx->d_grp_mask.as<int>();
    const PairTables& pt = ctx->pairs;
    a.dir_off = pt.dir_off.as<int>();
    a.dir_cnt = pt.dir_cnt.as<int>();
    a.dir_nlo = pt.dir_nlo.as<int>();
}

// Row blocks of shells such that the B rows plus Ck and Y fit in `budget` bytes.
template <typename T> int plan_blocks(qcx_ctx* ctx, PDArgs<T>& a, int nv, size_t* smem) {
    const size_t cs = sizeof(cplx<T>);
    const size_t budget = 200 * 1024;
    const size_t fixed = 2 * (size_t)ctx->nb * nv * cs;
    const int ldB = ctx->nb + 1;
    if (fixed + 3 * ldB * cs > budget) return -1;
    const size_t max_rows = (budget - fixed) / (ldB * cs);
    a.ldB = ldB;
    int nblk = 0, s = 0, rows_max = 0;
    a.row_s0[0] = 0;
    while (s < ctx->ngrp) {
        int rows = 0, e = s;
        while (e < ctx->ngrp) {
            const int r = ctx->grp_mu0_h[e + 1] - ctx->grp_mu0_h[e];
            if (rows + r > (int)max_rows) break;
            rows += r;
            ++e;
        }
        if (e == s) return -1;
        if (nblk >= 64) return -1;
        a.row_s0[++nblk] = e;
        rows_max = rows > rows_max ? rows : rows_max;
        s = e;
    }
    a.nblk = nblk;
    a.max_rows = rows_max;
    *smem = fixed + (size_t)rows_max * ldB * cs;
    return 0;
}

template <typename T> cudaError_t set_smem(const void* fn, size_t smem) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename T, int NCH> cudaError_t launch_pd(qcx_ctx* ctx, PDArgs<T>& a, size_t smem, dim3 grid) {
    cudaError_t e = set_smem<T>((const void*)k_pair_density<T, NCH>, smem);
    if (e != cudaSuccess) return e;
    k_pair_density<T, NCH><<<grid, PD_THREADS, smem, ctx->stream>>>(a);
    return cudaGetLastError();
}

template <int NCH, int NV> cudaError_t launch_fused(qcx_ctx* ctx, PDArgs<float>& a, size_t smem, dim3 grid, int nthr) {
    cudaError_t e;
    if (a.ptab) {
        if ((e = set_smem<float>((const void*)k_pair_density_fused<NCH, NV, true>, smem)) != cudaSuccess) return e;
        k_pair_density_fused<NCH, NV, true><<<grid, nthr, smem, ctx->stream>>>(a);
        return cudaGetLastError();
    }
    if ((e = set_smem<float>((const void*)k_pair_density_fused<NCH, NV, false>, smem)) != cudaSuccess) return e;
    k_pair_density_fused<NCH, NV, false><<<grid, nthr, smem, ctx->stream>>>(a);
    return cudaGetLastError();
}
template <int NCH> cudaError_t launch_fused_nv(qcx_ctx* ctx, PDArgs<float>& a, size_t smem, dim3 grid, int nthr) {
    if (a.nv <= 4) return launch_fused<NCH, 4>(ctx, a, smem, grid, nthr);
    if (a.nv <= 8) return launch_fused<NCH, 8>(ctx, a, smem, grid, nthr);
    return launch_fused<NCH, 16>(ctx, a, smem, grid, nthr);
}

template <typename T, int NCH> cudaError_t launch_ov(qcx_ctx* ctx, PDArgs<T>& a, size_t smem, int nk) {
    cudaError_t e = set_smem<T>((const void*)k_overlap<T, NCH>, smem);
    if (e != cudaSuccess) return e;
    k_overlap<T, NCH><<<nk, PD_THREADS, smem, ctx->stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

// --------------------------------------------------------------------- host

// Recognise lattice subset h Z^3 and its characters; build the per-pair
// one-dimensional tables.  Returns QCX_OK or an error with ctx->err set.
qcx_status qcx_build_pair_tables(qcx_ctx* ctx) {
    const double* L = ctx->lattice;
    double hmin = 0.0;
    for (int i = 0; i < 9; ++i) {
        const double v = fabs(L[i]);
        if (v > 1e-9 && (hmin == 0.0 || v < hmin)) hmin = v;
    }
    if (hmin == 0.0) return ctx->fail(QCX_ERR_ARG, "lattice is zero");
    double h = 0.0;
    int M[9];
    for (int div = 1; div <= 6 && h == 0.0; ++div) {
        const double hc = hmin / div;
        bool ok = true;
        for (int i = 0; i < 9 && ok; ++i) {
            const double r = L[i] / hc;
            const double n = std::round(r);
            if (fabs(r - n) > 1e-8 * fmax(1.0, fabs(r))) ok = false;
            M[i] = (int)n;
        }
        if (ok) h = hc;
    }
    if (h == 0.0)
        return ctx->fail(QCX_ERR_UNSUPPORTED,
                         "lattice is not a sublattice of h Z^3 (needs cubic-frame SC/FCC/BCC-type lattices)");
    const long det = (long)M[0] * (M[4] * M[8] - M[5] * M[7]) - (long)M[1] * (M[3] * M[8] - M[5] * M[6]) +
                     (long)M[2] * (M[3] * M[7] - M[4] * M[6]);
    const int m = (int)labs(det);
    if (m < 1 || m > 4) return ctx->fail(QCX_ERR_UNSUPPORTED, "lattice index in h Z^3 must be 1..4");
    int nch = 0;
    for (int a0 = 0; a0 < m; ++a0)
        for (int a1 = 0; a1 < m; ++a1)
            for (int a2 = 0; a2 < m; ++a2) {
                bool ok = true;
                for (int r = 0; r < 3; ++r) {
                    const long s = (long)M[3 * r] * a0 + (long)M[3 * r + 1] * a1 + (long)M[3 * r + 2] * a2;
                    if (s % m != 0) ok = false;
                }
                if (ok && nch < 4) {
                    ctx->chars[nch][0] = (double)a0 / m;
                    ctx->chars[nch][1] = (double)a1 / m;
                    ctx->chars[nch][2] = (double)a2 / m;
                    ++nch;
                }
            }
    if (nch != m) return ctx->fail(QCX_ERR_UNSUPPORTED, "could not enumerate lattice characters");
    ctx->h = h;
    ctx->nchar = m;

    // groups: consecutive shells on the same atom with the same exponent (at most one s and one p)
    std::vector<int> gfirst, gmask, gmu0;
    int mu = 0;
    for (int sh = 0; sh < ctx->nshell;) {
        int mask = 0, e = sh;
        while (e < ctx->nshell && ctx->shell_atom[e] == ctx->shell_atom[sh] &&
               ctx->shell_exp[e] == ctx->shell_exp[sh] && !(mask & (1 << ctx->shell_l[e])) &&
               (e == sh || ctx->shell_l[e] > ctx->shell_l[e - 1])) {
            mask |= 1 << ctx->shell_l[e];
            ++e;
        }
        gfirst.push_back(sh);
        gmask.push_back(mask);
        gmu0.push_back(mu);
        mu += ((mask & 1) ? 1 : 0) + ((mask & 2) ? 3 : 0);
        sh = e;
    }
    gmu0.push_back(mu);
    const int ng_ = (int)gfirst.size();
    ctx->ngrp = ng_;
    ctx->grp_mu0_h = gmu0;
    const int npair = ng_ * ng_;
    std::vector<int> dir_off(npair * 3), dir_cnt(npair * 3), dir_nlo(npair * 3);
    std::vector<double> par(npair * 8);
    std::vector<double2> tab;
    for (int ga = 0; ga < ng_; ++ga) {
        const int sa = gfirst[ga];
        const double al = ctx->shell_exp[sa];
        const double* A = &ctx->atom_xyz[3 * ctx->shell_atom[sa]];
        const double na = pow(2.0 * al / M_PI, 0.75);      // the p factor 2 sqrt(a) is folded in below
        for (int gb = 0; gb < ng_; ++gb) {
            const int sb = gfirst[gb];
            const double be = ctx->shell_exp[sb];
            const double* B = &ctx->atom_xyz[3 * ctx->shell_atom[sb]];
            const double nbn = pow(2.0 * be / M_PI, 0.75);
            const int ip = ga * ng_ + gb;
            const double p = al + be, mu_ = al * be / p;
            par[ip * 8 + 0] = p;
            par[ip * 8 + 1] = al / p;
            par[ip * 8 + 2] = be / p;
            par[ip * 8 + 3] = na * nbn * pow(M_PI / p, 1.5);
            for (int x = 0; x < 3; ++x) par[ip * 8 + 4 + x] = (al * A[x] + be * B[x]) / p;
            par[ip * 8 + 7] = 0.0;
            const double R = sqrt(LATTICE_CUT / mu_);
            for (int x = 0; x < 3; ++x) {
                const double D = A[x] - B[x];
                const int nlo = (int)std::ceil((D - R) / h);
                const int nhi = (int)std::floor((D + R) / h);
                dir_off[ip * 3 + x] = (int)tab.size();
                dir_nlo[ip * 3 + x] = nlo;
                int cnt = 0;
                for (int n = nlo; n <= nhi; ++n) {
                    const double d = D - h * n;
                    tab.push_back(make_double2(exp(-mu_ * d * d), d));
                    ++cnt;
                }
                dir_cnt[ip * 3 + x] = cnt;
            }
        }
    }
    PairTables& pt = ctx->pairs;
    pt.npair = npair;
    std::vector<double> par32d(par.begin(), par.end());
    std::vector<float> par32(par.size());
    for (size_t i = 0; i < par.size(); ++i) par32[i] = (float)par[i];
    std::vector<float2> tab32(tab.size());
    for (size_t i = 0; i < tab.size(); ++i) tab32[i] = make_float2((float)tab[i].x, (float)tab[i].y);
    cudaError_t e;
#define UP(buf, vec, T)                                                                          \
    if ((e = buf.ensure(vec.size() * sizeof(T))) != cudaSuccess ||                                \
        (e = cudaMemcpy(buf.p, vec.data(), vec.size() * sizeof(T), cudaMemcpyHostToDevice)) != \
            cudaSuccess)                                                                         \
        return ctx->fail(QCX_ERR_CUDA, std::string("pair tables: ") + cudaGetErrorString(e));
    UP(pt.dir_off, dir_off, int)
    UP(pt.dir_cnt, dir_cnt, int)
    UP(pt.dir_nlo, dir_nlo, int)
    UP(pt.par64, par, double)
    UP(pt.par32, par32, float)
    UP(pt.tab64, tab, double2)
    UP(pt.tab32, tab32, float2)
    UP(ctx->d_grp_mu0, gmu0, int)
    UP(ctx->d_grp_mask, gmask, int)
#undef UP
    return QCX_OK;
}

cudaError_t qcx_launch_qsetup(qcx_ctx* ctx, QSlot& s, const int* d_G, int ng, const double* q) {
    // reciprocal basis b_i (rows) = 2 pi inv(A)^T
    const double* A = ctx->lattice;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    double inv[9];
    inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    double b[9];  // b[i][j] = 2 pi inv[j][i]
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
    k_qsetup<<<(ng + 127) / 128, 128, 0, ctx->stream>>>(d_G, ng, q[0], q[1], q[2], b[0], b[1], b[2], b[3], b[4],
                                                         b[5], b[6], b[7], b[8], s.kappa.as<double>(),
                                                         s.kappa32.as<float>(), s.vs.as<double>(),
                                                         s.vs32.as<float>());
    return cudaGetLastError();
}

// Classes of the components v[3 i + x] of n points along axis x: values equal to a class's first
// value within 1e-9 (relative) share it; idx[3 i + x] receives the class, vals the float values.
static void axis_classes(const double* v, int n, int x, std::vector<double>& vals, std::vector<int>& idx) {
    std::vector<int> ord(n);
    for (int i = 0; i < n; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int i, int j) { return v[3 * i + x] < v[3 * j + x]; });
    int cls = -1;
    double first = 0.0;
    for (int j = 0; j < n; ++j) {
        const double d = v[3 * ord[j] + x];
        if (cls < 0 || fabs(d - first) > 1e-9 * fmax(1.0, fabs(d))) {
            ++cls;
            first = d;
            vals.push_back(d);
        }
        idx[3 * ord[j] + x] = cls;
    }
}

cudaError_t qcx_pd_tab_prepare(qcx_ctx* ctx, QSlot& s, const int* G_host, int ng, int iq) {
    PdTab& t = s.pdt;
    t.valid = false;
    const int nk = ctx->nk, npair = ctx->ngrp * ctx->ngrp;
    if ((int)ctx->kpts_h.size() != 3 * nk || npair < 1) return cudaSuccess;
    // q + G in Cartesian components (reciprocal basis b_i = 2 pi inv(A)^T rows)
    const double* A = ctx->lattice;
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    const double inv[9] = {(A[4] * A[8] - A[5] * A[7]) / det, (A[2] * A[7] - A[1] * A[8]) / det,
                           (A[1] * A[5] - A[2] * A[4]) / det, (A[5] * A[6] - A[3] * A[8]) / det,
                           (A[0] * A[8] - A[2] * A[6]) / det, (A[2] * A[3] - A[0] * A[5]) / det,
                           (A[3] * A[7] - A[4] * A[6]) / det, (A[1] * A[6] - A[0] * A[7]) / det,
                           (A[0] * A[4] - A[1] * A[3]) / det};
    const double* q = &ctx->qpts[3 * iq];
    std::vector<double> kap(3 * (size_t)ng);
    for (int g = 0; g < ng; ++g)
        for (int x = 0; x < 3; ++x) {
            double v = q[x];
            for (int i = 0; i < 3; ++i) v += G_host[3 * g + i] * 2.0 * M_PI * inv[3 * x + i];
            kap[3 * g + x] = v;
        }
    std::vector<double> kval, qval;
    std::vector<int> kidx(3 * (size_t)nk), gidx(3 * (size_t)ng);
    long long cells = 0;
    for (int x = 0; x < 3; ++x) {
        t.kofs[x] = (int)kval.size();
        t.qofs[x] = (int)qval.size();
        axis_classes(ctx->kpts_h.data(), nk, x, kval, kidx);
        axis_classes(kap.data(), ng, x, qval, gidx);
        t.nkx[x] = (int)kval.size() - t.kofs[x];
        t.nqx[x] = (int)qval.size() - t.qofs[x];
        cells += (long long)t.nkx[x] * t.nqx[x];
    }
    // worth it only when the classes repeat (regular k grids, G shells); bounded memory
    const int nch = ctx->nchar;
    const size_t tab_bytes = (size_t)npair * cells * nch * 4 * sizeof(float2);
    if (4 * cells > 3LL * 3 * nk * ng || tab_bytes > ((size_t)512 << 20)) return cudaSuccess;
    for (int x = 0; x < 3; ++x) t.tbase[x + 1] = t.tbase[x] + (long long)npair * t.nkx[x] * t.nqx[x];
    cudaError_t e;
    if ((e = t.tab.ensure(tab_bytes)) != cudaSuccess) return e;
    if ((e = t.cmn.ensure((size_t)npair * ng * sizeof(float2))) != cudaSuccess) return e;
    if ((e = t.kidx.ensure(kidx.size() * sizeof(int))) != cudaSuccess) return e;
    if ((e = t.gidx.ensure(gidx.size() * sizeof(int))) != cudaSuccess) return e;
    if ((e = t.kval.ensure(kval.size() * sizeof(double))) != cudaSuccess) return e;
    if ((e = t.qval.ensure(qval.size() * sizeof(double))) != cudaSuccess) return e;
    const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
    if ((e = cudaMemcpyAsync(t.kidx.p, kidx.data(), kidx.size() * sizeof(int), h2d, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(t.gidx.p, gidx.data(), gidx.size() * sizeof(int), h2d, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(t.kval.p, kval.data(), kval.size() * sizeof(double), h2d, ctx->stream)) != cudaSuccess ||
        (e = cudaMemcpyAsync(t.qval.p, qval.data(), qval.size() * sizeof(double), h2d, ctx->stream)) != cudaSuccess)
        return e;
    t.valid = true;
    return cudaSuccess;
}

cudaError_t qcx_launch_pair_density(qcx_ctx* ctx, QSlot& s, int iq, qcx_precision prec) {
    const int nt = ctx->nk * ctx->nv * ctx->nc;
    const int gpc = 8;
    dim3 grid(ctx->nk, (s.ng + gpc - 1) / gpc);
    size_t smem = 0;
    if (prec == QCX_FP64) {
        PDArgs<double> a{};
        fill_common(ctx, a);
        if (plan_blocks(ctx, a, ctx->nv, &smem)) return cudaErrorInvalidValue;
        a.nv = ctx->nv;
        a.nc = ctx->nc;
        a.nk = ctx->nk;
        a.ng = s.ng;
        a.nt = nt;
        a.g_per_cta = gpc;
        a.par = ctx->pairs.par64.as<double>();
        a.tab = ctx->pairs.tab64.as<double2>();
        a.kpts = ctx->d_kpts.as<double>();
        a.kappa = s.kappa.as<double>();
        a.Ck = ctx->d_Ck64.as<double2>();
        a.Ckq = ctx->d_Ckq64.as<double2>() + (size_t)iq * ctx->nk * ctx->nb * ctx->nc;
        a.R64 = s.rho.as<double2>();
        switch (ctx->nchar) {
            case 1: return launch_pd<double, 1>(ctx, a, smem, grid);
            case 2: return launch_pd<double, 2>(ctx, a, smem, grid);
            default: return launch_pd<double, 4>(ctx, a, smem, grid);
        }
    }
    PDArgs<float> a{};
    fill_common(ctx, a);
    // fused kernel: threads = (G per CTA) x groups, Y = B C_k in registers (nv <= 16)
    int gcf = 0;
    size_t smem_f = 0;
    if (ctx->nv <= 16 && ctx->ngrp <= PDF_MAXT) {
        const int tmax = ctx->nv <= 4 ? pdf_maxt<4>() : (ctx->nv <= 8 ? pdf_maxt<8>() : pdf_maxt<16>());
        gcf = std::max(1, std::min(16, tmax / ctx->ngrp));
        auto need = [&](int gc) {
            return sizeof(cplx<float>) * ((size_t)ctx->nb * ctx->nv + (size_t)ctx->nb * ctx->nc +
                                          (size_t)gc * ctx->nb * ctx->nv);
        };
        while (gcf > 1 && need(gcf) > 200 * 1024) --gcf;
        smem_f = need(gcf);
        if (smem_f > 200 * 1024) gcf = 0;
    }
    if (!gcf && plan_blocks(ctx, a, ctx->nv, &smem)) return cudaErrorInvalidValue;
    a.nv = ctx->nv;
    a.nc = ctx->nc;
    a.nk = ctx->nk;
    a.ng = s.ng;
    a.nt = nt;
    a.g_per_cta = gpc;
    a.par = ctx->pairs.par32.as<float>();
    a.tab = ctx->pairs.tab32.as<float2>();
    a.kpts = ctx->d_kpts32.as<float>();
    a.kappa = s.kappa32.as<float>();
    a.Ck = ctx->d_Ck32.as<float2>();
    a.Ckq = ctx->d_Ckq32.as<float2>() + (size_t)iq * ctx->nk * ctx->nb * ctx->nc;
    a.R64 = nullptr;
    a.R0 = reinterpret_cast<__nv_bfloat162*>(s.rho.p);
    a.R1 = a.R0 + (size_t)s.ngp * (s.kp / 2);
    a.R2 = a.R1 + (size_t)s.ngp * (s.kp / 2);
    a.kp2 = s.kp / 2;
    if (gcf && s.pdt.valid) {
        // tables of this q first (FP32, the operations of pair_block_vals: FP64 tables were no more
        // accurate in the loss and cost ~2 ms per mid q at the GB300's FP64 rate): the one-dimensional
        // factors, then the factor of (pair, G)
        const PdTab& t = s.pdt;
        PdTabArgs<float> ta{};
        ta.par = ctx->pairs.par32.as<float>();
        ta.tab = ctx->pairs.tab32.as<float2>();
        ta.dir_off = ctx->pairs.dir_off.as<int>();
        ta.dir_cnt = ctx->pairs.dir_cnt.as<int>();
        ta.dir_nlo = ctx->pairs.dir_nlo.as<int>();
        ta.h = (float)ctx->h;
        for (int c = 0; c < 4; ++c)
            for (int x = 0; x < 3; ++x) {
                ta.charre[c][x] = (float)cos(2.0 * M_PI * ctx->chars[c][x]);
                ta.charim[c][x] = (float)sin(2.0 * M_PI * ctx->chars[c][x]);
            }
        ta.kval = t.kval.as<double>();
        ta.qval = t.qval.as<double>();
        ta.kappa = s.kappa32.as<float>();
        for (int x = 0; x < 3; ++x) {
            ta.nkx[x] = t.nkx[x];
            ta.nqx[x] = t.nqx[x];
            ta.kofs[x] = t.kofs[x];
            ta.qofs[x] = t.qofs[x];
        }
        for (int x = 0; x < 4; ++x) ta.tbase[x] = t.tbase[x];
        ta.npair = ctx->ngrp * ctx->ngrp;
        ta.ng = s.ng;
        ta.out = t.tab.as<float2>();
        ta.cmn = t.cmn.as<float2>();
        const unsigned gt = (unsigned)((t.tbase[3] + 255) / 256);
        const unsigned gcm = (unsigned)(((long long)ta.npair * s.ng + 255) / 256);
        switch (ctx->nchar) {
            case 1:
                k_pd_axis_table<float, 1><<<gt, 256, 0, ctx->stream>>>(ta);
                k_pd_common<float, 1><<<gcm, 256, 0, ctx->stream>>>(ta);
                break;
            case 2:
                k_pd_axis_table<float, 2><<<gt, 256, 0, ctx->stream>>>(ta);
                k_pd_common<float, 2><<<gcm, 256, 0, ctx->stream>>>(ta);
                break;
            default:
                k_pd_axis_table<float, 4><<<gt, 256, 0, ctx->stream>>>(ta);
                k_pd_common<float, 4><<<gcm, 256, 0, ctx->stream>>>(ta);
        }
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        a.ptab = t.tab.as<float2>();
        a.pcmn = t.cmn.as<float2>();
        a.kidx = t.kidx.as<int>();
        a.gidx = t.gidx.as<int>();
        for (int x = 0; x < 3; ++x) {
            a.nkx[x] = t.nkx[x];
            a.nqx[x] = t.nqx[x];
        }
        for (int x = 0; x < 4; ++x) a.tbase[x] = t.tbase[x];
    }
    if (gcf) {
        a.g_per_cta = gcf;
        const dim3 gridf(ctx->nk, (s.ng + gcf - 1) / gcf);
        const int nthr = gcf * ctx->ngrp;
        switch (ctx->nchar) {
            case 1: return launch_fused_nv<1>(ctx, a, smem_f, gridf, nthr);
            case 2: return launch_fused_nv<2>(ctx, a, smem_f, gridf, nthr);
            default: return launch_fused_nv<4>(ctx, a, smem_f, gridf, nthr);
        }
    }
    switch (ctx->nchar) {
        case 1: return launch_pd<float, 1>(ctx, a, smem, grid);
        case 2: return launch_pd<float, 2>(ctx, a, smem, grid);
        default: return launch_pd<float, 4>(ctx, a, smem, grid);
    }
}

cudaError_t qcx_launch_overlap(qcx_ctx* ctx, int nk, const double* d_kpts, double2* d_out) {
    PDArgs<double> a{};
    fill_common(ctx, a);
    size_t smem = 0;
    if (plan_blocks(ctx, a, 0, &smem)) return cudaErrorInvalidValue;
    a.par = ctx->pairs.par64.as<double>();
    a.tab = ctx->pairs.tab64.as<double2>();
    a.kpts = d_kpts;
    a.Sout = d_out;
    switch (ctx->nchar) {
        case 1: return launch_ov<double, 1>(ctx, a, smem, nk);
        case 2: return launch_ov<double, 2>(ctx, a, smem, nk);
        default: return launch_ov<double, 4>(ctx, a, smem, nk);
    }
}
