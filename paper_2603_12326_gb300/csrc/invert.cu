// Inverse of the dielectric matrices and the loss functions.
//
// eps(w, q+G) = 1/[eps^-1]_GG (Eq. (eps_LFE)); eps^noLFE = eps_GG
// (Eq. (eps_noLFE)); L = Im[-1/eps] (Eq. (dynamic_structure_factor)).
//
// One CTA per (q, w) block runs Gauss-Jordan elimination with partial
// (row) pivoting in place on a work copy of the matrix, then undoes the
// column permutation.  The FP64 path does this in double.  The mixed path
// does it in FP32 on the rounded copy of the FP64 matrix and records the
// condition estimate kappa_1 = |A|_1 |X|_1.  Blocks with kappa_1 above the
// context's threshold (default 1e4; the ill-conditioned ones, near the
// plasmon) then get one FP64 correction of the diagonal against the FP64
// matrix: with R = I - A X, [A^-1]_jj = X_jj + (X R)_jj + O(|R|^2).  The other
// blocks take L_LFE from the quadratic form below, which keeps the relative
// accuracy of X; on the 10 000 blocks of the 181-G workload the 981 with
// kappa_1 in (1e3, 1e4] agree with their FP64-corrected loss to 1.8e-5.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <cooperative_groups.h>

namespace {

constexpr int INV_THREADS = 512;

template <typename T> struct InvArgs {
    int ng, nw;
    const double2* eps64;      // FP64 input [nw][ng][ng]
    cplx<T>* X;                // work [nw][ng][ng]
    double* kappa;             // [nw] condition estimate (mixed path) or null
    double2* diag_inv;         // [nw][ng]
    double2* eps_diag;         // [nw][ng]
    double* L;                 // [2][nw][ng] (LFE, noLFE)
    int* flags;                // [nw]
};

template <typename T> __device__ __forceinline__ T cabs2(cplx<T> z) { return z.x * z.x + z.y * z.y; }

template <typename T>
__global__ void __launch_bounds__(INV_THREADS) k_gauss_jordan(InvArgs<T> a, int write_lfe) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = a.ng;
    C* rowk = reinterpret_cast<C*>(smem_raw);          // [n]
    C* colk = rowk + n;                                 // [n]
    int* piv = reinterpret_cast<int*>(colk + n);        // [n]
    int* idx = piv + n;                                 // [n]
    __shared__ T red_v[INV_THREADS / 32];
    __shared__ int red_i[INV_THREADS / 32];
    __shared__ int s_p;
    __shared__ int s_bad;

    const int b = blockIdx.x;
    C* X = a.X + (size_t)b * n * n;
    // load the matrix; record eps_GG and the loss without local fields
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const double2 z = a.eps64[(size_t)b * n * n + e];
        X[e] = mk<T>((T)z.x, (T)z.y);
        const int i = e / n;
        if (e == i * n + i) {
            const double re = z.x, im = z.y;
            a.eps_diag[(size_t)b * n + i] = make_double2(re, im);
            a.L[((size_t)a.nw + b) * n + i] = im / (re * re + im * im);
        }
    }
    __shared__ double s_norm;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_norm = 0.0;
    }
    __syncthreads();
    if (a.kappa) {
        // |A|_1: largest column sum of |A_ij|
        double best = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double cs = 0.0;
            for (int i = 0; i < n; ++i) {
                const double2 z = a.eps64[(size_t)b * n * n + (size_t)i * n + j];
                cs += sqrt(z.x * z.x + z.y * z.y);
            }
            best = fmax(best, cs);
        }
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(&s_norm), (unsigned long long)__double_as_longlong(best));
    }
    __syncthreads();

    for (int k = 0; k < n; ++k) {
        // pivot: largest |X_ik| over i >= k (smallest index on ties)
        T best = -1;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const T v = cabs2<T>(X[(size_t)i * n + k]);
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const T ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 0) {
            red_v[wid] = best;
            red_i[wid] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            T bv = red_v[0];
            int bix = red_i[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
                if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bix)) {
                    bv = red_v[w];
                    bix = red_i[w];
                }
            if (!(bv > 0) || bix >= n) {
                s_bad = 1;
                bix = k;
            }
            s_p = bix;
            piv[k] = bix;
        }
        __syncthreads();
        if (s_bad) break;
        const int p = s_p;
        // swap rows k and p, then load the (scaled) pivot row and column k
        if (p != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const C t = X[(size_t)k * n + j];
                X[(size_t)k * n + j] = X[(size_t)p * n + j];
                X[(size_t)p * n + j] = t;
            }
            __syncthreads();
        }
        const C pv = X[(size_t)k * n + k];
        const T d = (T)1 / cabs2<T>(pv);
        const C inv = mk<T>(pv.x * d, -pv.y * d);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const C v = (j == k) ? mk<T>(1, 0) : X[(size_t)k * n + j];
            rowk[j] = cmul(v, inv);
            colk[j] = (j == k) ? mk<T>(0, 0) : X[(size_t)j * n + k];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) X[(size_t)k * n + j] = rowk[j];
        // eliminate column k from every other row; X_ik itself becomes -colk_i * inv
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e - i * n;
            if (i == k) continue;
            const C f = colk[i];
            C x = (j == k) ? mk<T>(0, 0) : X[e];
            x.x -= f.x * rowk[j].x - f.y * rowk[j].y;
            x.y -= f.x * rowk[j].y + f.y * rowk[j].x;
            X[e] = x;
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0) a.flags[b] = 1;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            a.diag_inv[(size_t)b * n + j] = make_double2(0.0, 0.0);
            if (write_lfe) a.L[(size_t)b * n + j] = 0.0;
        }
        return;
    }
    // undo the column permutation: the inverse's column c is X's column idx[c]
    if (threadIdx.x == 0) {
        a.flags[b] = 0;
        for (int c = 0; c < n; ++c) idx[c] = c;
        for (int k = n - 1; k >= 0; --k) {
            const int t = idx[k];
            idx[k] = idx[piv[k]];
            idx[piv[k]] = t;
        }
    }
    __syncthreads();
    // write the permuted inverse back in place, row by row through shared memory
    for (int i = 0; i < n; ++i) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) rowk[j] = X[(size_t)i * n + idx[j]];
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) X[(size_t)i * n + j] = rowk[j];
        __syncthreads();
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const C z = X[(size_t)j * n + j];
        a.diag_inv[(size_t)b * n + j] = make_double2((double)z.x, (double)z.y);
        if (write_lfe) a.L[(size_t)b * n + j] = -(double)z.y;
    }
    if (a.kappa) {
        // |X|_1 of the computed inverse
        __shared__ double s_xnorm;
        if (threadIdx.x == 0) s_xnorm = 0.0;
        __syncthreads();
        double best = 0.0;
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            double cs = 0.0;
            for (int i = 0; i < n; ++i) {
                const C z = X[(size_t)i * n + j];
                cs += sqrt((double)z.x * z.x + (double)z.y * z.y);
            }
            best = fmax(best, cs);
        }
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
        if ((threadIdx.x & 31) == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(&s_xnorm), (unsigned long long)__double_as_longlong(best));
        __syncthreads();
        if (threadIdx.x == 0) a.kappa[b] = s_norm * s_xnorm;
    }
}

// Mixed path, N_G <= GJC_MAXN: the same elimination with the matrix resident
// in shared memory, split by columns over a cluster of GJC_CS CTAs (a 181 x 181
// FP32 complex matrix is 262 KB, more than one CTA holds; with four CTAs of
// 74 KB, three clusters' CTAs share an SM and hide each other's barriers).  Step k: the CTA
// owning column k picks the pivot row and publishes the row index, the pivot
// and column k after the row exchange (the multipliers) in its shared memory;
// after one cluster barrier the others read them through distributed shared
// memory; every CTA then exchanges rows, scales the pivot row and eliminates
// in its own columns.  The published values alternate between two slots, so
// the barrier of the next step also orders their reuse.  Warps take rows,
// lanes take columns.
constexpr int GJC_CS = 4;
constexpr int GJC_THREADS = 256;
constexpr int GJC_MAXN = 192;
constexpr int GJC_WARPS = GJC_THREADS / 32;

__global__ void __cluster_dims__(GJC_CS, 1, 1) __launch_bounds__(GJC_THREADS) k_gj_cluster(InvArgs<float> a) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int b = blockIdx.x / GJC_CS;
    const int n = a.ng;
    const int h = (n + GJC_CS - 1) / GJC_CS;
    const int c0 = rank * h;
    const int hn = max(0, min(h, n - c0));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* Xs = reinterpret_cast<float2*>(smem_raw);     // [n][h] my columns
    float2* F = Xs + (size_t)n * h;                        // [2][n] published multipliers
    float2* Fl = F + 2 * n;                                // [n] multipliers of this step
    float2* rowk = Fl + n;                                 // [h] scaled pivot row
    int* piv = reinterpret_cast<int*>(rowk + h);           // [n]
    int* idx = piv + n;                                    // [n]
    int* jof = idx + n;                                    // [n] inverse of idx
    __shared__ int s_p[2], s_bad[2];
    __shared__ float2 s_pv[2];
    __shared__ float red_v[GJC_WARPS];
    __shared__ int red_i[GJC_WARPS];
    __shared__ double s_anorm, s_xnorm;

    const double2* A = a.eps64 + (size_t)b * n * n;
    for (int i = warp; i < n; i += GJC_WARPS)
        for (int c = lane; c < hn; c += 32) {
            const double2 z = A[(size_t)i * n + c0 + c];
            Xs[i * h + c] = make_float2((float)z.x, (float)z.y);
            if (i == c0 + c) {
                a.eps_diag[(size_t)b * n + i] = z;
                a.L[((size_t)a.nw + b) * n + i] = z.y / (z.x * z.x + z.y * z.y);
            }
        }
    if (threadIdx.x == 0) {
        s_anorm = 0.0;
        s_xnorm = 0.0;
    }
    __syncthreads();
    if (a.kappa) {
        double best = 0.0;
        for (int c = threadIdx.x; c < hn; c += blockDim.x) {
            double cs = 0.0;
            for (int i = 0; i < n; ++i) {
                const double2 z = A[(size_t)i * n + c0 + c];
                cs += sqrt(z.x * z.x + z.y * z.y);
            }
            best = fmax(best, cs);
        }
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(&s_anorm), (unsigned long long)__double_as_longlong(best));
    }
    __syncthreads();

    int bad = 0;
    for (int k = 0; k < n; ++k) {
        const int owner = k / h, kc = k - owner * h, par = k & 1;
        if (rank == owner) {
            float best = -1.0f;
            int bi = n;
            for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
                const float2 z = Xs[i * h + kc];
                const float v = z.x * z.x + z.y * z.y;
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                const float ov = __shfl_down_sync(0xffffffffu, best, o);
                const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                red_v[warp] = best;
                red_i[warp] = bi;
            }
            __syncthreads();
            if (threadIdx.x == 0) {
                float bv = red_v[0];
                int bix = red_i[0];
                for (int w = 1; w < GJC_WARPS; ++w)
                    if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bix)) {
                        bv = red_v[w];
                        bix = red_i[w];
                    }
                const int sing = !(bv > 0.0f) || bix >= n;
                if (sing) bix = k;
                s_bad[par] = sing;
                s_p[par] = bix;
                s_pv[par] = Xs[bix * h + kc];
            }
            __syncthreads();
            const int p = s_p[par];
            for (int i = threadIdx.x; i < n; i += blockDim.x) {
                const int src = (i == k) ? p : (i == p ? k : i);
                F[par * n + i] = Xs[src * h + kc];
            }
        }
        cl.sync();
        const int p = cl.map_shared_rank(s_p, owner)[par];
        bad = cl.map_shared_rank(s_bad, owner)[par];
        const float2 pv = cl.map_shared_rank(s_pv, owner)[par];
        if (bad) break;
        const float2* Fr = cl.map_shared_rank(F, owner) + par * n;
        for (int i = threadIdx.x; i < n; i += blockDim.x) Fl[i] = Fr[i];
        if (threadIdx.x == 0) piv[k] = p;
        if (p != k)
            for (int c = threadIdx.x; c < hn; c += blockDim.x) {
                const float2 t = Xs[k * h + c];
                Xs[k * h + c] = Xs[p * h + c];
                Xs[p * h + c] = t;
            }
        __syncthreads();
        const float d = 1.0f / (pv.x * pv.x + pv.y * pv.y);
        const float2 inv = make_float2(pv.x * d, -pv.y * d);
        for (int c = threadIdx.x; c < hn; c += blockDim.x)
            rowk[c] = (rank == owner && c == kc) ? inv : cmul(Xs[k * h + c], inv);
        __syncthreads();
        for (int i = warp; i < n; i += GJC_WARPS) {
            const float2 f = Fl[i];
            for (int c = lane; c < hn; c += 32) {
                const float2 r = rowk[c];
                if (i == k) {
                    Xs[k * h + c] = r;
                } else {
                    float2 x = (rank == owner && c == kc) ? make_float2(0.f, 0.f) : Xs[i * h + c];
                    x.x -= f.x * r.x - f.y * r.y;
                    x.y -= f.x * r.y + f.y * r.x;
                    Xs[i * h + c] = x;
                }
            }
        }
        __syncthreads();
    }
    if (bad) {
        if (rank == 0) {
            if (threadIdx.x == 0) {
                a.flags[b] = 1;
                if (a.kappa) a.kappa[b] = 0.0;
            }
            for (int j = threadIdx.x; j < n; j += blockDim.x) a.diag_inv[(size_t)b * n + j] = make_double2(0.0, 0.0);
        }
        cl.sync();    // no CTA leaves while another may still read its shared memory
        return;
    }
    // the inverse's column j is the eliminated matrix's column idx[j]
    if (threadIdx.x == 0) {
        for (int c = 0; c < n; ++c) idx[c] = c;
        for (int kk = n - 1; kk >= 0; --kk) {
            const int t = idx[kk];
            idx[kk] = idx[piv[kk]];
            idx[piv[kk]] = t;
        }
        if (rank == 0) a.flags[b] = 0;
    }
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) jof[idx[j]] = j;
    __syncthreads();
    float2* Xg = a.X + (size_t)b * n * n;
    for (int i = warp; i < n; i += GJC_WARPS)
        for (int c = lane; c < hn; c += 32) Xg[(size_t)i * n + jof[c0 + c]] = Xs[i * h + c];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const int cgl = idx[j] - c0;
        if (cgl >= 0 && cgl < hn) {
            const float2 z = Xs[j * h + cgl];
            a.diag_inv[(size_t)b * n + j] = make_double2((double)z.x, (double)z.y);
        }
    }
    if (a.kappa) {
        double best = 0.0;
        for (int c = threadIdx.x; c < hn; c += blockDim.x) {
            double cs = 0.0;
            for (int i = 0; i < n; ++i) {
                const float2 z = Xs[i * h + c];
                cs += sqrt((double)z.x * z.x + (double)z.y * z.y);
            }
            best = fmax(best, cs);
        }
        for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
        if (lane == 0)
            atomicMax(reinterpret_cast<unsigned long long*>(&s_xnorm), (unsigned long long)__double_as_longlong(best));
    }
    cl.sync();
    if (a.kappa && rank == 0 && threadIdx.x == 0) {
        double an = 0.0, xn = 0.0;
        for (int r = 0; r < GJC_CS; ++r) {
            an = fmax(an, *cl.map_shared_rank(&s_anorm, r));
            xn = fmax(xn, *cl.map_shared_rank(&s_xnorm, r));
        }
        a.kappa[b] = an * xn;
    }
    cl.sync();    // rank 0 has read every CTA's norms
}

size_t gjc_smem(int n) {
    const int h = (n + GJC_CS - 1) / GJC_CS;
    return ((size_t)n * h + 3 * (size_t)n + h) * sizeof(float2) + 3 * (size_t)n * sizeof(int);
}

// FP64 correction of the diagonal of X ~ A^-1 for the blocks with kappa_1 above
// the threshold (A FP64, X FP32):  d_j = X_jj + sum_k X_jk (delta_kj - sum_l A_kl X_lj).
// Grid (block, 32-column panel).  The other blocks keep X_jj.
constexpr int RF_COLS = 32;
__global__ void __launch_bounds__(256) k_refine_diag(int n, const double2* Aall, const float2* Xall,
                                                     const int* flags, const double* kappa, double kappa_refine,
                                                     double2* diag_inv, double* L, double* resid) {
    __shared__ double2 s_d[RF_COLS];
    const int b = blockIdx.x, j0 = blockIdx.y * RF_COLS;
    if (flags[b] || j0 >= n) return;
    const float2* X = Xall + (size_t)b * n * n;
    if (!(kappa[b] > kappa_refine)) {
        if (threadIdx.x < RF_COLS && j0 + threadIdx.x < n) {
            const int j = j0 + threadIdx.x;
            const float2 x = X[(size_t)j * n + j];
            diag_inv[(size_t)b * n + j] = make_double2((double)x.x, (double)x.y);
            L[(size_t)b * n + j] = -(double)x.y;
        }
        return;
    }
    const double2* A = Aall + (size_t)b * n * n;
    if (threadIdx.x < RF_COLS) s_d[threadIdx.x] = make_double2(0.0, 0.0);
    __syncthreads();
    const int jl = threadIdx.x & (RF_COLS - 1);
    const int j = j0 + jl;
    double2 part = make_double2(0.0, 0.0);
    if (j < n) {
        for (int k = threadIdx.x / RF_COLS; k < n; k += blockDim.x / RF_COLS) {
            double yr = 0.0, yi = 0.0;          // sum_l A_kl X_lj in FP64
            for (int l = 0; l < n; ++l) {
                const double2 av = A[(size_t)k * n + l];
                const float2 x = X[(size_t)l * n + j];
                yr = fma(av.x, (double)x.x, yr);
                yr = fma(-av.y, (double)x.y, yr);
                yi = fma(av.x, (double)x.y, yi);
                yi = fma(av.y, (double)x.x, yi);
            }
            const double rr = (k == j ? 1.0 : 0.0) - yr, ri = -yi;
            const float2 xjk = X[(size_t)j * n + k];
            part.x += (double)xjk.x * rr - (double)xjk.y * ri;
            part.y += (double)xjk.x * ri + (double)xjk.y * rr;
        }
    }
    atomicAdd(&s_d[jl].x, part.x);
    atomicAdd(&s_d[jl].y, part.y);
    __syncthreads();
    if (threadIdx.x < RF_COLS && j0 + threadIdx.x < n) {
        const int jj = j0 + threadIdx.x;
        const float2 x = X[(size_t)jj * n + jj];
        const double dr = (double)x.x + s_d[threadIdx.x].x, di = (double)x.y + s_d[threadIdx.x].y;
        diag_inv[(size_t)b * n + jj] = make_double2(dr, di);
        L[(size_t)b * n + jj] = -di;
        const double mag = sqrt(dr * dr + di * di);
        const double rel = mag > 0 ? sqrt(s_d[threadIdx.x].x * s_d[threadIdx.x].x +
                                          s_d[threadIdx.x].y * s_d[threadIdx.x].y) / mag
                                   : 0.0;
        atomicMax(reinterpret_cast<unsigned long long*>(resid + b), (unsigned long long)__double_as_longlong(rel));
    }
}

// L_LFE of the mixed path without cancellation: for X = A^-1 (the FP32
// inverse) and B = (A - A^H)/(2i) the Hermitian form of A's anti-Hermitian
// part, -Im [A^-1]_jj = [X B X^H]_jj.  Where the loss is small against
// |[A^-1]_jj| (Im of an O(1) diagonal) the imaginary part of the FP32 diagonal
// loses its relative accuracy; the form builds L from the small B itself
// (B from the FP64 matrix in FP64, rounded once), so its relative error is
// that of X.  One CTA per (block, 32 rows j): T = X B in 32 x 32 tiles, then
// L_j = Re sum_l T_jl conj(X_jl); the imaginary part of the reported diagonal
// becomes -L_j.  Blocks corrected in FP64 keep their values.
constexpr int QF = 32;
__global__ void __launch_bounds__(256) k_loss_quadform(int n, const double2* Aall, const float2* Xall,
                                                       const int* flags, const double* kappa, double kappa_refine,
                                                       double2* diag_inv, double* L) {
    __shared__ float2 Xs[QF][QF + 1];
    __shared__ float2 Bs[QF][QF + 1];
    __shared__ double2 At[QF][QF + 1];       // A_lk tile, read along rows, used transposed
    __shared__ float Lrow[QF];
    const int b = blockIdx.x, j0 = blockIdx.y * QF;
    if (flags[b] || kappa[b] > kappa_refine) return;
    const double2* A = Aall + (size_t)b * n * n;
    const float2* X = Xall + (size_t)b * n * n;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (threadIdx.x < QF) Lrow[threadIdx.x] = 0.0f;
    for (int l0 = 0; l0 < n; l0 += QF) {
        float2 acc[2][2];
#pragma unroll
        for (int r = 0; r < 2; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c) acc[r][c] = make_float2(0.f, 0.f);
        for (int k0 = 0; k0 < n; k0 += QF) {
            for (int e = threadIdx.x; e < QF * QF; e += blockDim.x) {
                const int r = e / QF, c = e % QF;
                At[r][c] = (l0 + r < n && k0 + c < n) ? A[(size_t)(l0 + r) * n + k0 + c] : make_double2(0.0, 0.0);
            }
            __syncthreads();
            for (int e = threadIdx.x; e < QF * QF; e += blockDim.x) {
                const int r = e / QF, c = e % QF;
                const int j = j0 + r, kk = k0 + c;
                Xs[r][c] = (j < n && kk < n) ? X[(size_t)j * n + kk] : make_float2(0.f, 0.f);
                const int kr = k0 + r, lc = l0 + c;
                float2 bv = make_float2(0.f, 0.f);
                if (kr < n && lc < n) {
                    const double2 akl = A[(size_t)kr * n + lc], alk = At[c][r];
                    bv = make_float2((float)(0.5 * (akl.y + alk.y)), (float)(-0.5 * (akl.x - alk.x)));
                }
                Bs[r][c] = bv;
            }
            __syncthreads();
#pragma unroll 8
            for (int kk = 0; kk < QF; ++kk) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float2 x = Xs[ty + 16 * r][kk];
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float2 bb = Bs[kk][tx + 16 * c];
                        acc[r][c].x = fmaf(x.x, bb.x, fmaf(-x.y, bb.y, acc[r][c].x));
                        acc[r][c].y = fmaf(x.x, bb.y, fmaf(x.y, bb.x, acc[r][c].y));
                    }
                }
            }
            __syncthreads();
        }
        // L_j += Re sum_l T_jl conj(X_jl) over this column tile
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int j = j0 + ty + 16 * r;
            float part = 0.0f;
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                const int l = l0 + tx + 16 * c;
                if (j < n && l < n) {
                    const float2 x = X[(size_t)j * n + l];
                    part = fmaf(acc[r][c].x, x.x, fmaf(acc[r][c].y, x.y, part));
                }
            }
            for (int o = 8; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o, 16);
            if (tx == 0) Lrow[ty + 16 * r] += part;
        }
        __syncthreads();
    }
    if (threadIdx.x < QF && j0 + threadIdx.x < n) {
        const size_t o = (size_t)b * n + j0 + threadIdx.x;
        L[o] = (double)Lrow[threadIdx.x];
        diag_inv[o].y = -(double)Lrow[threadIdx.x];
    }
}

}  // namespace

cudaError_t qcx_launch_invert(qcx_ctx* ctx, QSlot& s, qcx_precision prec, double* d_loss_out) {
    const int n = s.ng;
    if (prec == QCX_FP64) {
        InvArgs<double> a{};
        a.ng = n;
        a.nw = s.nw;
        a.eps64 = s.eps.as<double2>();
        a.X = s.work.as<double2>();
        a.diag_inv = s.diag_inv.as<double2>();
        a.eps_diag = s.eps_diag.as<double2>();
        a.L = d_loss_out;
        a.flags = s.flags.as<int>();
        a.kappa = nullptr;
        const size_t smem = (size_t)n * 2 * sizeof(double2) + (size_t)n * 2 * sizeof(int);
        cudaError_t e = cudaFuncSetAttribute((const void*)k_gauss_jordan<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gauss_jordan<double><<<s.nw, INV_THREADS, smem, ctx->stream>>>(a, 1);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return cudaMemsetAsync(s.resid.p, 0, sizeof(double) * s.nw, ctx->stream);
    }
    InvArgs<float> a{};
    a.ng = n;
    a.nw = s.nw;
    a.eps64 = s.eps.as<double2>();
    a.X = s.work.as<float2>();
    cudaError_t e = s.kappa1.ensure(sizeof(double) * s.nw);
    if (e != cudaSuccess) return e;
    a.kappa = s.kappa1.as<double>();
    a.diag_inv = s.diag_inv.as<double2>();
    a.eps_diag = s.eps_diag.as<double2>();
    a.L = d_loss_out;
    a.flags = s.flags.as<int>();
    if (n <= GJC_MAXN) {
        // the matrix stays in the shared memory of a GJC_CS-CTA cluster
        const size_t smem = gjc_smem(n);
        e = cudaFuncSetAttribute((const void*)k_gj_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_gj_cluster<<<s.nw * GJC_CS, GJC_THREADS, smem, ctx->stream>>>(a);
    } else {
        const size_t smem = (size_t)n * 2 * sizeof(float2) + (size_t)n * 2 * sizeof(int);
        e = cudaFuncSetAttribute((const void*)k_gauss_jordan<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        k_gauss_jordan<float><<<s.nw, INV_THREADS, smem, ctx->stream>>>(a, 0);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.resid.p, 0, sizeof(double) * s.nw, ctx->stream);
    if (e != cudaSuccess) return e;
    dim3 grid(s.nw, (n + RF_COLS - 1) / RF_COLS);
    k_refine_diag<<<grid, 256, 0, ctx->stream>>>(n, a.eps64, a.X, a.flags, a.kappa, ctx->kappa_refine, a.diag_inv,
                                                  d_loss_out, s.resid.as<double>());
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 gq(s.nw, (n + QF - 1) / QF);
    k_loss_quadform<<<gq, 256, 0, ctx->stream>>>(n, a.eps64, a.X, a.flags, a.kappa, ctx->kappa_refine, a.diag_inv,
                                                  d_loss_out);
    return cudaGetLastError();
}

extern "C" qcx_status qcx_set_refine_threshold(qcx_ctx* ctx, double kappa1) {
    if (!ctx) return QCX_ERR_ARG;
    if (!(kappa1 >= 0.0)) return ctx->fail(QCX_ERR_ARG, "set_refine_threshold: kappa1 must be >= 0");
    ctx->kappa_refine = kappa1;
    return QCX_OK;
}
