// Spectral route to chi0: the spectral part of Eq. (RPA) (Eq. (eRPA_spectral)) put on a
// uniform energy grid E_b = E0 + b step, and the principal part from the Kramers-Kronig
// relations with the retarded broadening of the direct sum:
//
//   S_b[G][G'] = 2/(N_k V) sum_t phi_b(dE_t) conj(rho_t(G)) rho_t(G'),
//   chi0(w)    = sum_b S_b K(w, E_b),   K(w, E) = 1/(w - E + i eta) - 1/(w + E + i eta),
//   eps        = delta - v^1/2 chi0 v^1/2.
//
// phi_b is the hat function of grid point b: dE = E_b + x step (0 <= x < 1) gives the weight
// 1 - x to point b and x to point b + 1, which keeps the zeroth and first moments of the
// delta.  The spectral weights are formed once per q (each transition feeds two grid
// points), the frequency dependence enters only through K.
//
// Steps for one q:
//   k_spec_hat      b_t, x_t per transition (FP64) and the count of each grid point;
//   k_spec_scan     offsets of the groups (one block);
//   k_spec_place    transitions grouped by b (positions taken with atomics) ...
//   k_spec_order    ... and put in ascending t within a group, so every later sum runs in a
//                   fixed order;
//   k_spec_gather   pair densities and x in the grouped order;
//   k_spec_gram     S_b for each upper (G, G') tile pair of 32 x 32 from the groups of b - 1
//                   (weight x) and b (weight 1 - x); S_b is Hermitian, so tiles below the
//                   diagonal are not formed;
//   k_spec_kk       the contraction over b for 16 w x (8 x 32) (G, G') per CTA, a real GEMM
//                   in the four products of (Re K, Im K) with (Re S, Im S) that gives both
//                   chi0[G][G'] and chi0[G'][G] from one upper tile;
//   k_spec_dyson    eps in the layout of the slot (FP64: [w][G][G'], MIXED: [w][G'][G]).
//
// Precision: FP64 throughout (QCX_FP64), or FP32 pair densities (the sum of the three
// BF16 terms of the mixed path), FP32 spectral weights and the contraction on the tcgen05
// tensor cores in three-term split BF16 (spectral_tc.cu; QCX_MIXED); K and the grid are formed
// in FP64 in both.  The grid points are processed in chunks whose spectral weights fit a
// memory budget (at most 4096 points for the mixed route); chi0 is accumulated over the
// chunks in FP64.  The mixed contraction can also run on the CUDA cores in FP32
// (qcx_set_spectral_engine), summed in two levels: partial sums over 64 grid points added
// into a second FP32 accumulator.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <climits>
#include <cmath>
#include <vector>

namespace {

constexpr int SP_TILE = 32;            // (G, G') tile edge of the spectral weights
constexpr int SP_TILE2 = SP_TILE * SP_TILE;
constexpr int KK_TW = 16;              // frequencies per CTA of the contraction
constexpr int KK_RC = 8;               // tile rows per CTA of the contraction
constexpr int KK_NX = KK_RC * SP_TILE; // (G, G') pairs per CTA
constexpr int KK_THREADS = 256;
constexpr int KK_FLUSH = 64;           // MIXED: grid points per FP32 partial sum
constexpr int KK_F32_CHUNK = 4096;     // MIXED: grid points per chunk (64 partial sums at most)

template <typename R> struct KKCfg;
template <> struct KKCfg<double> { static constexpr int TB = 16; };   // grid points per stage
template <> struct KKCfg<float> { static constexpr int TB = 32; };

template <typename R> constexpr size_t kk_smem_bytes() {
    return 2 * ((size_t)KKCfg<R>::TB * KK_NX + (size_t)KK_TW * KKCfg<R>::TB) * sizeof(cplx<R>);
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// ------------------------------------------------------------------- grid and grouping
// min and max of dE_t over the transitions of one q (one block)
__global__ void __launch_bounds__(1024) k_spec_range(long long nt, int nv, int nc, const double* Ek,
                                                     const double* Ekq, double* out) {
    __shared__ double lo[1024], hi[1024];
    double mn = INFINITY, mx = -INFINITY;
    const int nvc = nv * nc;
    for (long long t = threadIdx.x; t < nt; t += 1024) {
        const long long k = t / nvc;
        const int rem = (int)(t - k * nvc);
        const int v = rem / nc, c = rem - v * nc;
        const double dE = Ekq[k * nc + c] - Ek[k * nv + v];
        mn = fmin(mn, dE);
        mx = fmax(mx, dE);
    }
    lo[threadIdx.x] = mn;
    hi[threadIdx.x] = mx;
    __syncthreads();
    for (int d = 512; d > 0; d >>= 1) {
        if (threadIdx.x < d) {
            lo[threadIdx.x] = fmin(lo[threadIdx.x], lo[threadIdx.x + d]);
            hi[threadIdx.x] = fmax(hi[threadIdx.x], hi[threadIdx.x + d]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = lo[0];
        out[1] = hi[0];
    }
}

// b_t = floor(u), x_t = u - b_t with u = (dE_t - E0)/step; b_t must lie in [0, nbin - 2]
// (else status bit 1 and b_t = -1); count[b] += 1
__global__ void k_spec_hat(long long nt, int nv, int nc, const double* Ek, const double* Ekq, double E0, double step,
                           int nbin, int* bin, double* x, int* cnt, int* status) {
    const int nvc = nv * nc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt;
         t += (long long)gridDim.x * blockDim.x) {
        const long long k = t / nvc;
        const int rem = (int)(t - k * nvc);
        const int v = rem / nc, c = rem - v * nc;
        const double dE = Ekq[k * nc + c] - Ek[k * nv + v];
        const double u = (dE - E0) / step;
        const double fb = floor(u);
        if (!(fb >= 0.0 && fb <= (double)(nbin - 2))) {
            atomicOr(status, 1);
            bin[t] = -1;
            x[t] = 0.0;
            continue;
        }
        const int b = (int)fb;
        bin[t] = b;
        x[t] = u - fb;
        atomicAdd(&cnt[b], 1);
    }
}

// off[b] = sum of cnt[0 .. b-1], off[n] = total (one block of 1024)
__global__ void __launch_bounds__(1024) k_spec_scan(int n, const int* cnt, int* off) {
    __shared__ int part[1024];
    const int per = (n + 1023) / 1024;
    const int lo = min(n, (int)threadIdx.x * per), hi = min(n, lo + per);
    int s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int d = 1; d < 1024; d <<= 1) {
        const int v = threadIdx.x >= (unsigned)d ? part[threadIdx.x - d] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    int run = threadIdx.x ? part[threadIdx.x - 1] : 0;
    for (int i = lo; i < hi; ++i) {
        off[i] = run;
        run += cnt[i];
    }
    if (threadIdx.x == 1023) off[n] = part[1023];
}

__global__ void k_spec_place(long long nt, const int* bin, const int* off, int* fill, int* perm0) {
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nt;
         t += (long long)gridDim.x * blockDim.x) {
        const int b = bin[t];
        if (b < 0) continue;
        perm0[off[b] + atomicAdd(&fill[b], 1)] = (int)t;
    }
}

// one warp per group: rank of each member among the group's (distinct) transition indices
__global__ void __launch_bounds__(256) k_spec_order(int nbin, const int* off, const int* perm0, int* perm) {
    const int b = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (b >= nbin) return;
    const int o = off[b], L = off[b + 1] - o;
    for (int i = lane; i < L; i += 32) {
        const int ti = perm0[o + i];
        int r = 0;
        for (int j = 0; j < L; ++j) r += perm0[o + j] < ti;
        perm[o + r] = ti;
    }
}

template <typename R> struct GatherArgs {
    const double2* r64;                  // FP64 pair densities [ng][nt], or null
    const __nv_bfloat162* p0;            // else the three BF16 planes [ngp][kp2]
    const __nv_bfloat162* p1;
    const __nv_bfloat162* p2;
    long long kp2;
    const int* perm;
    const double* x;
    long long nt;
    cplx<R>* out;                        // [ng][nt] in the grouped order
    R* xs;                               // [nt]
};

template <typename R> __global__ void k_spec_gather(GatherArgs<R> a) {
    const long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (j >= a.nt) return;
    const int G = blockIdx.y;
    const int t = a.perm[j];
    cplx<R> v;
    if (a.r64) {
        const double2 r = a.r64[(long long)G * a.nt + t];
        v.x = (R)r.x;
        v.y = (R)r.y;
    } else {
        const long long o = (long long)G * a.kp2 + t;
        const float2 f0 = __bfloat1622float2(a.p0[o]), f1 = __bfloat1622float2(a.p1[o]),
                     f2 = __bfloat1622float2(a.p2[o]);
        v.x = (R)((f0.x + f1.x) + f2.x);
        v.y = (R)((f0.y + f1.y) + f2.y);
    }
    a.out[(long long)G * a.nt + j] = v;
    if (G == 0) a.xs[j] = (R)a.x[t];
}

// ------------------------------------------------------------------- spectral weights
template <typename R> struct GramArgs {
    const cplx<R>* rho;                  // [ng][nt] grouped order
    const R* xs;                         // [nt]
    const int* off;                      // [nbin + 1]
    const int2* tp;                      // upper tile pairs (gi <= hi)
    long long nt;
    int ng, b0, nbc;
    R pref;
    cplx<R>* S;                          // [ntp][nbc][32][32]
};

// S_b for one upper tile pair and one grid point; thread (tx, ty) holds rows ty, ty + 16 and
// columns tx, tx + 16 of the tile; transitions are staged 16 at a time
template <typename R> __global__ void __launch_bounds__(256) k_spec_gram(GramArgs<R> a) {
    using C = cplx<R>;
    __shared__ C As[16][SP_TILE + 1];
    __shared__ C Bs[16][SP_TILE + 1];
    const int p = blockIdx.x, bl = blockIdx.y, b = a.b0 + bl;
    const int2 pr = a.tp[p];
    const int G0 = pr.x * SP_TILE, H0 = pr.y * SP_TILE;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int jlo = a.off[b > 0 ? b - 1 : 0], jmid = a.off[b], jhi = a.off[b + 1];
    C acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = mk<R>(0, 0);
    for (int j0 = jlo; j0 < jhi; j0 += 16) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = threadIdx.x + 256 * r;
            const int tt = i & 15, gg = i >> 4;
            const int j = j0 + tt;
            C va = mk<R>(0, 0), vb = mk<R>(0, 0);
            if (j < jhi) {
                const R phi = j < jmid ? a.xs[j] : (R)1 - a.xs[j];
                if (G0 + gg < a.ng) {
                    const C r0 = a.rho[(long long)(G0 + gg) * a.nt + j];
                    va = mk<R>(phi * r0.x, -phi * r0.y);
                }
                if (H0 + gg < a.ng) vb = a.rho[(long long)(H0 + gg) * a.nt + j];
            }
            As[tt][gg] = va;
            Bs[tt][gg] = vb;
        }
        __syncthreads();
#pragma unroll 4
        for (int tt = 0; tt < 16; ++tt) {
            const C a0 = As[tt][ty], a1 = As[tt][ty + 16];
            const C b0 = Bs[tt][tx], b1 = Bs[tt][tx + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][0], a1, b0);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
    // S_b is Hermitian: its diagonal is real, so the rounding left in the imaginary part there
    // (which Re K would carry into Im chi0_GG) is dropped
    C* out = a.S + ((size_t)p * a.nbc + bl) * SP_TILE2;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const bool diag = pr.x == pr.y && ty + 16 * i == tx + 16 * j;
            out[(ty + 16 * i) * SP_TILE + tx + 16 * j] = mk<R>(a.pref * acc[i][j].x, diag ? (R)0 : a.pref * acc[i][j].y);
        }
}

// full Hermitian S_b [b][G][G'] (FP64) from the upper tiles of one chunk
template <typename R>
__global__ void k_spec_export(int nb, int nbc, int ng, int T, const cplx<R>* S, double2* out) {
    const long long n = (long long)nb * ng * ng;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int bl = (int)(i / ((long long)ng * ng));
        const int r = (int)(i - (long long)bl * ng * ng);
        const int G = r / ng, H = r - G * ng;
        int gi = G / SP_TILE, hi = H / SP_TILE, gr = G % SP_TILE, hr = H % SP_TILE;
        const bool lower = gi > hi;
        if (lower) {
            const int t0 = gi, t1 = gr;
            gi = hi;
            hi = t0;
            gr = hr;
            hr = t1;
        }
        const int p = gi * T - gi * (gi - 1) / 2 + (hi - gi);
        const cplx<R> v = S[((size_t)p * nbc + bl) * SP_TILE2 + gr * SP_TILE + hr];
        out[i] = make_double2((double)v.x, lower ? -(double)v.y : (double)v.y);
    }
}

// ------------------------------------------------------------------- Kramers-Kronig
// K[w][b] = 1/(w - E_b + i eta) - 1/(w + E_b + i eta), E_b = E0 + b step (FP64, stored as R);
// zero for b >= nbin
template <typename R>
__global__ void k_spec_ktab(int nw, long long ld, int nbin, const double* w, double E0, double step, double eta,
                            cplx<R>* K) {
    const long long n = (long long)nw * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int iw = (int)(i / ld);
        const long long b = i - (long long)iw * ld;
        cplx<R> k = mk<R>(0, 0);
        if (b < nbin) {
            const double E = E0 + step * (double)b;
            const double am = w[iw] - E, ap = w[iw] + E;
            const double d1 = 1.0 / (am * am + eta * eta), d2 = 1.0 / (ap * ap + eta * eta);
            k = mk<R>((R)(am * d1 - ap * d2), (R)(eta * (d2 - d1)));
        }
        K[i] = k;
    }
}

template <typename R> struct KKArgs {
    const cplx<R>* S;                    // [ntp][nbc][32][32] spectral weights of the chunk
    const cplx<R>* K;                    // [nw][ldk]
    long long ldk;
    const int2* tp;
    int nbc, nb, b0;                     // chunk stride, grid points used, first grid point
    int nw, ng;
    int accumulate;                      // add to chi (later chunks) instead of storing
    double2* chi;                        // [nw][ng][ng]
};

// chi0 over the grid points of one chunk for 16 w x 256 (G, G') pairs (rows rg*8 .. rg*8+7
// of an upper tile pair); thread: 4 frequencies (wi*4 ..) x 4 pairs (xi + 64 x).  Per pair
// and frequency the four sums A = sum Kr Sr, B = sum Ki Si, Cs = sum Kr Si, D = sum Ki Sr
// give chi0[G][G'] = (A - B) + i (Cs + D) and chi0[G'][G] = (A + B) + i (D - Cs).
template <typename R> __global__ void __launch_bounds__(KK_THREADS, 1) k_spec_kk(KKArgs<R> a) {
    using C = cplx<R>;
    constexpr int TB = KKCfg<R>::TB;
    constexpr bool F32 = sizeof(R) == 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* Ss = reinterpret_cast<C*>(smem_raw);          // [2][TB][KK_NX]
    C* Ks = Ss + 2 * TB * KK_NX;                     // [2][KK_TW][TB]
    const int tid = threadIdx.x, xi = tid & 63, wi = tid >> 6;
    const int wg = blockIdx.x, rg = blockIdx.y, p = blockIdx.z;
    const int2 pr = a.tp[p];
    const C* Sp = a.S + (size_t)p * a.nbc * SP_TILE2 + rg * KK_NX;
    const int nstage = (a.nb + TB - 1) / TB;

    auto load = [&](int st, int buf) {
        constexpr int PER_BIN = (int)(KK_NX * sizeof(C) / 16);
        constexpr int SCH = TB * PER_BIN;
        char* sd = reinterpret_cast<char*>(Ss + buf * TB * KK_NX);
        for (int i = tid; i < SCH; i += KK_THREADS) {
            const int bb = i / PER_BIN, o = i - bb * PER_BIN;
            const int b = st * TB + bb;
            const bool ok = b < a.nb;
            const char* src = reinterpret_cast<const char*>(Sp + (size_t)(ok ? b : 0) * SP_TILE2) + o * 16;
            cp_async16(sd + (size_t)i * 16, src, ok ? 16 : 0);
        }
        constexpr int PER_ROW = (int)(TB * sizeof(C) / 16);
        constexpr int KCH = KK_TW * PER_ROW;
        char* kd = reinterpret_cast<char*>(Ks + buf * KK_TW * TB);
        for (int i = tid; i < KCH; i += KK_THREADS) {
            const int r = i / PER_ROW, o = i - r * PER_ROW;
            const int w = wg * KK_TW + r;
            const bool ok = w < a.nw;
            const char* src =
                reinterpret_cast<const char*>(a.K + (size_t)(ok ? w : 0) * a.ldk + a.b0 + st * TB) + o * 16;
            cp_async16(kd + (size_t)i * 16, src, ok ? 16 : 0);
        }
    };

    R acc[4][4][4];
    float part[F32 ? 4 : 1][4][4];           // MIXED: sum of the 64-point partial sums
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[m][x][c] = (R)0;
                if constexpr (F32) part[m][x][c] = 0.f;
            }

    if (nstage > 0) load(0, 0);
    cp_async_commit();
    for (int st = 0; st < nstage; ++st) {
        if (st + 1 < nstage) load(st + 1, (st + 1) & 1);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const C* Sb = Ss + (st & 1) * TB * KK_NX;
        const C* Kb = Ks + (st & 1) * KK_TW * TB;
#pragma unroll 2
        for (int bb = 0; bb < TB; ++bb) {
            C s[4], k[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) s[x] = Sb[bb * KK_NX + xi + 64 * x];
#pragma unroll
            for (int m = 0; m < 4; ++m) k[m] = Kb[(wi * 4 + m) * TB + bb];
#pragma unroll
            for (int m = 0; m < 4; ++m)
#pragma unroll
                for (int x = 0; x < 4; ++x) {
                    acc[m][x][0] = fma(k[m].x, s[x].x, acc[m][x][0]);
                    acc[m][x][1] = fma(k[m].y, s[x].y, acc[m][x][1]);
                    acc[m][x][2] = fma(k[m].x, s[x].y, acc[m][x][2]);
                    acc[m][x][3] = fma(k[m].y, s[x].x, acc[m][x][3]);
                }
        }
        __syncthreads();
        if constexpr (F32) {
            if (((st + 1) * TB) % KK_FLUSH == 0 || st == nstage - 1) {
#pragma unroll
                for (int m = 0; m < 4; ++m)
#pragma unroll
                    for (int x = 0; x < 4; ++x)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            part[m][x][c] += acc[m][x][c];
                            acc[m][x][c] = 0.f;
                        }
            }
        }
    }

#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const int w = wg * KK_TW + wi * 4 + m;
        if (w >= a.nw) continue;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int X = xi + 64 * x;
            const int G = pr.x * SP_TILE + rg * KK_RC + X / SP_TILE;
            const int H = pr.y * SP_TILE + X % SP_TILE;
            if (G >= a.ng || H >= a.ng) continue;
            double s4[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                if constexpr (F32)
                    s4[c] = (double)part[m][x][c];
                else
                    s4[c] = (double)acc[m][x][c];
            }
            const double2 gh = make_double2(s4[0] - s4[1], s4[2] + s4[3]);
            double2* d = a.chi + ((size_t)w * a.ng + G) * a.ng + H;
            if (a.accumulate) {
                d->x += gh.x;
                d->y += gh.y;
            } else {
                *d = gh;
            }
            if (pr.x != pr.y) {
                const double2 hg = make_double2(s4[0] + s4[1], s4[3] - s4[2]);
                double2* e = a.chi + ((size_t)w * a.ng + H) * a.ng + G;
                if (a.accumulate) {
                    e->x += hg.x;
                    e->y += hg.y;
                } else {
                    *e = hg;
                }
            }
        }
    }
}

// eps = delta - v^1/2 chi0 v^1/2 (FP64 slot: [w][G][G']; MIXED slot: [w][G'][G])
__global__ void k_spec_dyson(int nw, int ng, const double2* chi, const double* vs, int transpose, double2* eps,
                             double2* chi_out) {
    const long long n = (long long)nw * ng * ng;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int w = (int)(i / ((long long)ng * ng));
        const int r = (int)(i - (long long)w * ng * ng);
        const int G = r / ng, H = r - G * ng;
        const double2 ch = chi[i];
        const double vv = vs[G] * vs[H];
        const double2 e = make_double2((G == H ? 1.0 : 0.0) - vv * ch.x, -vv * ch.y);
        if (transpose)
            eps[((size_t)w * ng + H) * ng + G] = e;
        else
            eps[i] = e;
        if (chi_out) chi_out[i] = ch;
    }
}

inline int nblk(long long n, int t, int cap = 16384) { return (int)std::min<long long>((n + t - 1) / t, cap); }

double cell_volume(const qcx_ctx* ctx) {
    const double* L = ctx->lattice;
    return fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                L[2] * (L[3] * L[7] - L[4] * L[6]));
}

}  // namespace

namespace {

constexpr size_t kSpecChunkBytes = 4ull << 30;   // default budget of the spectral weights of one chunk

// The precision-dependent part: gather, K table, then per chunk of grid points the spectral
// weights and the contraction, then the Dyson step.
template <typename R>
qcx_status spectral_chi0(qcx_ctx* ctx, QSlot& s, bool mixed, int nw, double E0, double step, int nbin, long long nt,
                         double2* d_chi_out, qcx_c64* out_S) {
    using C = cplx<R>;
    SpecBufs& sp = ctx->spec;
    const int ng = s.ng;
    cudaStream_t st = ctx->stream;

    CUDA_OR_FAIL(sp.rhos.ensure(sizeof(C) * (size_t)ng * nt), "alloc grouped pair densities");
    CUDA_OR_FAIL(sp.xs.ensure(sizeof(R) * (size_t)nt), "alloc");
    GatherArgs<R> g{};
    if (mixed) {
        g.p0 = reinterpret_cast<const __nv_bfloat162*>(s.rho.p);
        g.p1 = g.p0 + (size_t)s.ngp * (s.kp / 2);
        g.p2 = g.p1 + (size_t)s.ngp * (s.kp / 2);
        g.kp2 = s.kp / 2;
    } else {
        g.r64 = s.rho.as<double2>();
    }
    g.perm = sp.perm.as<int>();
    g.x = sp.x.as<double>();
    g.nt = nt;
    g.out = sp.rhos.as<C>();
    g.xs = sp.xs.as<R>();
    k_spec_gather<R><<<dim3((unsigned)((nt + 255) / 256), ng), 256, 0, st>>>(g);
    CUDA_OR_FAIL(cudaGetLastError(), "gather kernel");

    const int T = (ng + SP_TILE - 1) / SP_TILE;
    const int ntp = T * (T + 1) / 2;
    std::vector<int2> tp;
    tp.reserve(ntp);
    for (int gi = 0; gi < T; ++gi)
        for (int hi = gi; hi < T; ++hi) tp.push_back(make_int2(gi, hi));
    CUDA_OR_FAIL(sp.tp.ensure(sizeof(int2) * ntp), "alloc");
    CUDA_OR_FAIL(cudaMemcpyAsync(sp.tp.p, tp.data(), sizeof(int2) * ntp, cudaMemcpyHostToDevice, st), "copy tiles");

    const long long ldk = (nbin + 31LL) / 32 * 32;
    CUDA_OR_FAIL(sp.ktab.ensure(sizeof(C) * (size_t)nw * ldk), "alloc K");
    k_spec_ktab<R><<<nblk((long long)nw * ldk, 256), 256, 0, st>>>(nw, ldk, nbin, s.w.as<double>(), E0, step, s.eta,
                                                                    sp.ktab.as<C>());
    CUDA_OR_FAIL(cudaGetLastError(), "K kernel");

    const size_t per_bin = (size_t)ntp * SP_TILE2 * sizeof(C);
    long long nbc = ctx->spec_chunk_bins > 0 ? ctx->spec_chunk_bins : (long long)(kSpecChunkBytes / per_bin);
    nbc = std::min<long long>(nbc, sizeof(R) == 4 ? KK_F32_CHUNK : 65504);
    nbc = std::max<long long>(32, nbc / 32 * 32);
    nbc = std::min<long long>(nbc, ldk);
    CUDA_OR_FAIL(sp.S.ensure(per_bin * nbc), "alloc spectral weights");
    CUDA_OR_FAIL(sp.chi.ensure(sizeof(double2) * (size_t)nw * ng * ng), "alloc chi0");
    const bool s_dev = out_S && qcx_is_device_ptr(out_S);
    if (out_S && !s_dev) CUDA_OR_FAIL(sp.Sout.ensure(sizeof(double2) * (size_t)nbc * ng * ng), "alloc");
    const size_t smem = kk_smem_bytes<R>();
    CUDA_OR_FAIL(cudaFuncSetAttribute((const void*)k_spec_kk<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem),
                 "contraction smem");
    const R pref = (R)(2.0 / (ctx->nk * cell_volume(ctx)));
    const int nchunk = (int)((nbin + nbc - 1) / nbc);
    // the mixed route's contraction on the tensor cores: K table and each chunk's weights as
    // three BF16 planes, K-major over the grid points
    const bool tc = mixed && !ctx->spec_cuda_cores;
    const int mtiles = (2 * nw + 127) / 128;
    const int ntiles = ntp * 16;                      // 2 x 1024 columns per tile pair, 128 per tile
    CUtensorMap kmaps[3], smaps[3];
    if (tc) {
        const size_t kn = (size_t)mtiles * 128 * ldk;
        const size_t sn = (size_t)ntiles * 128 * nbc;
        CUDA_OR_FAIL(sp.kplanes.ensure(3 * kn * sizeof(__nv_bfloat16)), "alloc K planes");
        CUDA_OR_FAIL(sp.splanes.ensure(3 * sn * sizeof(__nv_bfloat16)), "alloc weight planes");
        CUDA_OR_FAIL(qcx_spec_tc_ktab(st, nw, mtiles * 128, ldk, nbin, s.w.as<double>(), E0, step, s.eta,
                                      sp.kplanes.as<__nv_bfloat16>()),
                     "K planes kernel");
        for (int i = 0; i < 3; ++i)
            if (!qcx_make_bf16_map(&kmaps[i], sp.kplanes.as<__nv_bfloat16>() + i * kn, ldk, mtiles * 128, 128, 32) ||
                !qcx_make_bf16_map(&smaps[i], sp.splanes.as<__nv_bfloat16>() + i * sn, nbc, ntiles * 128, 128, 32))
                return ctx->fail(QCX_ERR_CUDA, "chi0_spectral: tensor map encoding failed");
        CUDA_OR_FAIL(cudaMemsetAsync(sp.status.p, 0, sizeof(int), st), "clear");
    }
    CUDA_OR_FAIL(sp.events(3 + 3 * (size_t)nchunk + 1), "events");
    CUDA_OR_FAIL(cudaEventRecord(sp.ev[2], st), "event");

    for (long long b0 = 0; b0 < nbin; b0 += nbc) {
        const int nb = (int)std::min<long long>(nbc, nbin - b0);
        cudaEvent_t* ce = &sp.ev[3 + 3 * (size_t)(b0 / nbc)];
        CUDA_OR_FAIL(cudaEventRecord(ce[0], st), "event");
        GramArgs<R> ga;
        ga.rho = sp.rhos.as<C>();
        ga.xs = sp.xs.as<R>();
        ga.off = sp.off.as<int>();
        ga.tp = sp.tp.as<int2>();
        ga.nt = nt;
        ga.ng = ng;
        ga.b0 = (int)b0;
        ga.nbc = (int)nbc;
        ga.pref = pref;
        ga.S = sp.S.as<C>();
        k_spec_gram<R><<<dim3(ntp, nb), 256, 0, st>>>(ga);
        CUDA_OR_FAIL(cudaGetLastError(), "spectral weight kernel");
        if (out_S) {
            const size_t nel = (size_t)nb * ng * ng;
            double2* dst = s_dev ? reinterpret_cast<double2*>(out_S) + (size_t)b0 * ng * ng : sp.Sout.as<double2>();
            k_spec_export<R><<<nblk((long long)nel, 256), 256, 0, st>>>(nb, (int)nbc, ng, T, sp.S.as<C>(), dst);
            CUDA_OR_FAIL(cudaGetLastError(), "export kernel");
            if (!s_dev)
                CUDA_OR_FAIL(qcx_copy_out(ctx, reinterpret_cast<double2*>(out_S) + (size_t)b0 * ng * ng, dst,
                                          nel * sizeof(double2)),
                             "copy out weights");
        }
        CUDA_OR_FAIL(cudaEventRecord(ce[1], st), "event");
        if (tc) {
            CUDA_OR_FAIL(qcx_spec_tc_contract(st, kmaps, smaps, mtiles, ntiles, nw, ng, (int)nbc, nb, (int)b0, nbc,
                                              reinterpret_cast<const float2*>(sp.S.p),
                                              sp.splanes.as<__nv_bfloat16>(), sp.tp.as<int2>(), b0 > 0 ? 1 : 0,
                                              sp.chi.as<double2>(), sp.status.as<int>(), ctx->wait_limit),
                         "tensor-core contraction");
            CUDA_OR_FAIL(cudaEventRecord(ce[2], st), "event");
            continue;
        }
        KKArgs<R> ka;
        ka.S = sp.S.as<C>();
        ka.K = sp.ktab.as<C>();
        ka.ldk = ldk;
        ka.tp = sp.tp.as<int2>();
        ka.nbc = (int)nbc;
        ka.nb = nb;
        ka.b0 = (int)b0;
        ka.nw = nw;
        ka.ng = ng;
        ka.accumulate = b0 > 0;
        ka.chi = sp.chi.as<double2>();
        k_spec_kk<R><<<dim3((nw + KK_TW - 1) / KK_TW, SP_TILE / KK_RC, ntp), KK_THREADS, smem, st>>>(ka);
        CUDA_OR_FAIL(cudaGetLastError(), "contraction kernel");
        CUDA_OR_FAIL(cudaEventRecord(ce[2], st), "event");
    }
    k_spec_dyson<<<nblk((long long)nw * ng * ng, 256), 256, 0, st>>>(nw, ng, sp.chi.as<double2>(), s.vs.as<double>(),
                                                                      mixed ? 1 : 0, s.eps.as<double2>(), d_chi_out);
    CUDA_OR_FAIL(cudaGetLastError(), "dyson kernel");
    cudaEvent_t end = sp.ev[3 + 3 * (size_t)nchunk];
    CUDA_OR_FAIL(cudaEventRecord(end, st), "event");
    CUDA_OR_FAIL(cudaEventSynchronize(end), "sync");
    float t = 0.f;
    double ms[5] = {0, 0, 0, 0, 0};
    CUDA_OR_FAIL(cudaEventElapsedTime(&t, sp.ev[0], sp.ev[1]), "timing");
    ms[0] = t;
    CUDA_OR_FAIL(cudaEventElapsedTime(&t, sp.ev[1], sp.ev[2]), "timing");
    ms[1] = t;
    for (int c = 0; c < nchunk; ++c) {
        const cudaEvent_t* ce = &sp.ev[3 + 3 * (size_t)c];
        CUDA_OR_FAIL(cudaEventElapsedTime(&t, ce[0], ce[1]), "timing");
        ms[2] += t;
        CUDA_OR_FAIL(cudaEventElapsedTime(&t, ce[1], ce[2]), "timing");
        ms[3] += t;
    }
    CUDA_OR_FAIL(cudaEventElapsedTime(&t, sp.ev[3 + 3 * (size_t)(nchunk - 1) + 2], end), "timing");
    ms[4] = t;
    for (int i = 0; i < 5; ++i) sp.ms[i] = ms[i];
    if (tc) {
        int bad = 0;
        CUDA_OR_FAIL(cudaMemcpyAsync(&bad, sp.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
        CUDA_OR_FAIL(cudaStreamSynchronize(st), "sync");
        if (bad) return ctx->fail(QCX_ERR_TIMEOUT, "chi0_spectral: a pipeline wait in the tensor-core kernel gave up");
    }
    return QCX_OK;
}

}  // namespace

extern "C" qcx_status qcx_spectral_grid(qcx_ctx* ctx, int iq, double step, double* E0, int* nbin) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!E0 || !nbin || !(step > 0.0) || !std::isfinite(step))
        return ctx->fail(QCX_ERR_ARG, "spectral_grid: bad arguments");
    if (iq < 0 || iq >= ctx->nq || ctx->nk < 1 || !ctx->d_Ekq.p)
        return ctx->fail(QCX_ERR_STATE, "spectral_grid: states of this q not set");
    cudaSetDevice(ctx->device);
    const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    CUDA_OR_FAIL(ctx->spec.range.ensure(2 * sizeof(double)), "alloc");
    k_spec_range<<<1, 1024, 0, ctx->stream>>>(nt, ctx->nv, ctx->nc, ctx->d_Ek.as<double>(),
                                              ctx->d_Ekq.as<double>() + (size_t)iq * ctx->nk * ctx->nc,
                                              ctx->spec.range.as<double>());
    CUDA_OR_FAIL(cudaGetLastError(), "range kernel");
    double mm[2];
    CUDA_OR_FAIL(cudaMemcpyAsync(mm, ctx->spec.range.p, sizeof(mm), cudaMemcpyDeviceToHost, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    if (!std::isfinite(mm[0]) || !std::isfinite(mm[1]))
        return ctx->fail(QCX_ERR_ARG, "spectral_grid: non-finite transition energies");
    const double e0 = step * std::floor(mm[0] / step) - step;
    const double nb = std::floor((mm[1] - e0) / step) + 3.0;
    if (!(nb <= (double)(INT_MAX / 2))) return ctx->fail(QCX_ERR_ARG, "spectral_grid: too many grid points");
    *E0 = e0;
    *nbin = (int)nb;
    return QCX_OK;
}

extern "C" qcx_status qcx_set_spectral_engine(qcx_ctx* ctx, int cuda_cores) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    ctx->spec_cuda_cores = cuda_cores ? 1 : 0;
    return QCX_OK;
}

extern "C" qcx_status qcx_set_spectral_chunk(qcx_ctx* ctx, int bins) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (bins < 0) return ctx->fail(QCX_ERR_ARG, "set_spectral_chunk: bins must be >= 0");
    ctx->spec_chunk_bins = bins;
    return QCX_OK;
}

extern "C" qcx_status qcx_chi0_spectral(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, double E0,
                                        double step, int nbin, qcx_precision prec, qcx_c64* out_chi0,
                                        qcx_c64* out_S) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (prec != QCX_FP64 && prec != QCX_MIXED) return ctx->fail(QCX_ERR_ARG, "chi0_spectral: bad precision");
    QSlot& s = ctx->slot[prec];
    if (!s.have_rho || s.iq != iq)
        return ctx->fail(QCX_ERR_STATE, "chi0_spectral: pair densities of this q not computed");
    if (nw < 1 || !w || !(eta > 0.0) || !std::isfinite(eta) || !(step > 0.0) || !std::isfinite(step) ||
        !std::isfinite(E0) || nbin < 2)
        return ctx->fail(QCX_ERR_ARG, "chi0_spectral: bad arguments");
    const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    if (nt > INT_MAX) return ctx->fail(QCX_ERR_UNSUPPORTED, "chi0_spectral: more than 2^31 - 1 transitions");
    cudaSetDevice(ctx->device);
    std::vector<double> wh;
    CUDA_OR_FAIL(fetch(ctx, wh, w, nw), "chi0_spectral w");
    for (double v : wh)
        if (!std::isfinite(v)) return ctx->fail(QCX_ERR_ARG, "chi0_spectral: non-finite frequency");
    s.nw = nw;
    s.eta = eta;
    s.have_eps = false;
    if (ctx->loss[iq]) ctx->loss[iq]->valid = false;
    const int ng = s.ng;
    cudaStream_t st = ctx->stream;
    CUDA_OR_FAIL(s.w.ensure(sizeof(double) * nw), "alloc");
    CUDA_OR_FAIL(cudaMemcpyAsync(s.w.p, wh.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, st), "copy w");
    const size_t nmat = (size_t)nw * ng * ng;
    CUDA_OR_FAIL(s.eps.ensure(nmat * sizeof(double2)), "alloc eps");

    // grid points of every transition, grouped by grid point
    SpecBufs& sp = ctx->spec;
    CUDA_OR_FAIL(sp.bin.ensure(sizeof(int) * nt), "alloc");
    CUDA_OR_FAIL(sp.x.ensure(sizeof(double) * nt), "alloc");
    CUDA_OR_FAIL(sp.perm0.ensure(sizeof(int) * nt), "alloc");
    CUDA_OR_FAIL(sp.perm.ensure(sizeof(int) * nt), "alloc");
    CUDA_OR_FAIL(sp.cnt.ensure(sizeof(int) * (size_t)nbin), "alloc");
    CUDA_OR_FAIL(sp.fill.ensure(sizeof(int) * (size_t)nbin), "alloc");
    CUDA_OR_FAIL(sp.off.ensure(sizeof(int) * ((size_t)nbin + 1)), "alloc");
    CUDA_OR_FAIL(sp.status.ensure(sizeof(int)), "alloc");
    CUDA_OR_FAIL(cudaMemsetAsync(sp.cnt.p, 0, sizeof(int) * (size_t)nbin, st), "clear");
    CUDA_OR_FAIL(cudaMemsetAsync(sp.fill.p, 0, sizeof(int) * (size_t)nbin, st), "clear");
    CUDA_OR_FAIL(cudaMemsetAsync(sp.status.p, 0, sizeof(int), st), "clear");
    CUDA_OR_FAIL(sp.events(3), "events");
    CUDA_OR_FAIL(cudaEventRecord(sp.ev[0], st), "event");
    k_spec_hat<<<nblk(nt, 256), 256, 0, st>>>(nt, ctx->nv, ctx->nc, ctx->d_Ek.as<double>(),
                                               ctx->d_Ekq.as<double>() + (size_t)iq * ctx->nk * ctx->nc, E0, step,
                                               nbin, sp.bin.as<int>(), sp.x.as<double>(), sp.cnt.as<int>(),
                                               sp.status.as<int>());
    CUDA_OR_FAIL(cudaGetLastError(), "grid kernel");
    k_spec_scan<<<1, 1024, 0, st>>>(nbin, sp.cnt.as<int>(), sp.off.as<int>());
    CUDA_OR_FAIL(cudaGetLastError(), "scan kernel");
    int bad = 0;
    CUDA_OR_FAIL(cudaMemcpyAsync(&bad, sp.status.p, sizeof(int), cudaMemcpyDeviceToHost, st), "status");
    CUDA_OR_FAIL(cudaStreamSynchronize(st), "sync");
    if (bad) return ctx->fail(QCX_ERR_ARG, "chi0_spectral: transition energies outside [E0, E0 + (nbin - 1) step)");
    k_spec_place<<<nblk(nt, 256), 256, 0, st>>>(nt, sp.bin.as<int>(), sp.off.as<int>(), sp.fill.as<int>(),
                                                 sp.perm0.as<int>());
    CUDA_OR_FAIL(cudaGetLastError(), "place kernel");
    k_spec_order<<<(nbin + 7) / 8, 256, 0, st>>>(nbin, sp.off.as<int>(), sp.perm0.as<int>(), sp.perm.as<int>());
    CUDA_OR_FAIL(cudaGetLastError(), "order kernel");
    CUDA_OR_FAIL(cudaEventRecord(sp.ev[1], st), "event");

    double2* chi = nullptr;
    if (out_chi0) {
        chi = qcx_is_device_ptr(out_chi0) ? reinterpret_cast<double2*>(out_chi0) : nullptr;
        if (!chi) {
            CUDA_OR_FAIL(ctx->scratch.ensure(nmat * sizeof(double2)), "alloc");
            chi = ctx->scratch.as<double2>();
        }
    }
    const qcx_status r = prec == QCX_FP64
                             ? spectral_chi0<double>(ctx, s, false, nw, E0, step, nbin, nt, chi, out_S)
                             : spectral_chi0<float>(ctx, s, true, nw, E0, step, nbin, nt, chi, out_S);
    if (r != QCX_OK) return r;
    if (out_chi0 && chi != reinterpret_cast<double2*>(out_chi0))
        CUDA_OR_FAIL(qcx_copy_out(ctx, out_chi0, chi, nmat * sizeof(double2)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(st), "sync");
    s.have_eps = true;
    return QCX_OK;
}

extern "C" qcx_status qcx_spectral_timings(qcx_ctx* ctx, double* ms) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ms) return ctx->fail(QCX_ERR_ARG, "spectral_timings: ms is NULL");
    for (int i = 0; i < 5; ++i) ms[i] = ctx->spec.ms[i];
    return QCX_OK;
}
