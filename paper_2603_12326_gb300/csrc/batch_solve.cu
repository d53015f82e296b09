// Heads of the inverse dielectric matrices of a batch of uneven (q, w)
// instances: L_LFE = -Im [eps^-1]_{00} (Eq. (eps_LFE)) and L_noLFE =
// -Im (1/eps_00) (Eq. (eps_noLFE)).
//
// Only the head of eps^-1 is needed, so no inverse is formed.  With the head
// row and column moved last (A' = P^T eps P), [eps^-1]_{00} is the last
// component of the solution of A' x = e_last; LU elimination with partial
// pivoting of the augmented matrix [A' | e_last] leaves that component as
// y_last / u_last,last, with no back substitution.
//
// k_lu_head: one CTA per instance at a time (instance lists per CTA are built
//   on the host, largest first, so the batch is one persistent launch).
//   Right-looking blocked LU on a work copy in global memory (L2-resident):
//   rows are never moved; a row map in shared memory records the pivot order
//   (logical row -> stored row).  Per panel of PB columns: the panel is
//   gathered into shared memory and factored there; the trailing columns
//   (right-hand side included) are processed CW at a time: U12 = L11^-1 A12
//   through the explicit inverse of the unit lower triangle L11, then the
//   rank-PB update A22 -= L21 U12 with U12 columns held in registers.
//   FP64 for the plain path; FP32 for the mixed path, which also back-
//   substitutes the whole solution x for the refinement.
// k_resid: r = e_last - A' x in FP64 from the FP64 eps (32 rows per CTA, all
//   instances at once, so the FP64 work is spread over the whole GPU).
// k_lu_correct: d = A'^-1 r with the stored FP32 factors (blocked forward
//   and back substitution), x += d in FP64; the head is x_last.
#include "qcx_internal.h"
#include "cplx.cuh"

namespace {

constexpr int LU_THREADS = 256;
constexpr int NWARP = LU_THREADS / 32;
constexpr int CW = 64;                       // trailing columns per chunk
constexpr int RG = LU_THREADS / CW;          // row groups of the trailing update
constexpr double REFINE_TOL = 1.0e-6;        // last relative correction that counts as converged

template <typename T> struct Pb;
template <> struct Pb<float> { static constexpr int v = 32; };
template <> struct Pb<double> { static constexpr int v = 16; };

// logical index -> index in eps with the head moved last
__device__ __forceinline__ int head_last(int i, int n, int h) { return i == n - 1 ? h : (i < h ? i : i + 1); }

template <typename C> __device__ __forceinline__ C czero() {
    C z;
    z.x = 0;
    z.y = 0;
    return z;
}
template <typename C> __device__ __forceinline__ C cinv(C a) {
    const auto d = 1 / (a.x * a.x + a.y * a.y);
    C z;
    z.x = a.x * d;
    z.y = -a.y * d;
    return z;
}
// acc -= a * b
template <typename C> __device__ __forceinline__ void cfms(C& acc, C a, C b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(LU_THREADS) k_lu_head(BatchSolveArgs a, int nmax, int want_x) {
    using C = cplx<T>;
    constexpr int PB = Pb<T>::v;
    extern __shared__ __align__(16) unsigned char sm[];
    C* P = reinterpret_cast<C*>(sm);                  // [nmax][PB] panel, logical row order
    C* Li = P + (size_t)nmax * PB;                    // [PB][PB] L11^-1 (then U blocks)
    C* As = Li + PB * PB;                             // [PB][CW] A12 chunk
    C* Ub = As + PB * CW;                             // [PB][CW] U12 chunk
    C* xs = Ub + PB * CW;                             // [nmax] solution
    int* rmap = reinterpret_cast<int*>(xs + nmax);    // [nmax]
    __shared__ T red_v[NWARP];
    __shared__ int red_i[NWARP];
    __shared__ C sblk[PB];
    __shared__ int s_p, s_bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int ii = a.cta_off[blockIdx.x]; ii < a.cta_off[blockIdx.x + 1]; ++ii) {
        const int id = a.cta_ids[ii];
        const BatchInst in = a.inst[id];
        const int n = in.ng, h = in.head, ld = n + 1;
        const double2* A = a.eps + in.eps_off;
        C* M = reinterpret_cast<C*>(a.work) + in.work_off;
        for (long long e = threadIdx.x; e < (long long)n * ld; e += LU_THREADS) {
            const int i = (int)(e / ld), j = (int)(e - (long long)i * ld);
            C v;
            if (j == n) {
                v.x = (i == n - 1) ? T(1) : T(0);
                v.y = 0;
            } else {
                const double2 z = A[(size_t)head_last(i, n, h) * n + head_last(j, n, h)];
                v.x = (T)z.x;
                v.y = (T)z.y;
            }
            M[e] = v;
        }
        for (int i = threadIdx.x; i < n; i += LU_THREADS) rmap[i] = i;
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();

        for (int k0 = 0; k0 < n; k0 += PB) {
            const int kb = min(PB, n - k0), R = n - k0;
            for (int e = threadIdx.x; e < R * PB; e += LU_THREADS) {
                const int r = e / PB, c = e - r * PB;
                P[e] = c < kb ? M[(size_t)rmap[k0 + r] * ld + k0 + c] : czero<C>();
            }
            __syncthreads();
            for (int kk = 0; kk < kb; ++kk) {
                // pivot: largest |P_r,kk| over r >= kk (smallest r on ties)
                T best = -1;
                int bi = R;
                for (int r = kk + threadIdx.x; r < R; r += LU_THREADS) {
                    const C z = P[r * PB + kk];
                    const T v = z.x * z.x + z.y * z.y;
                    if (v > best) {
                        best = v;
                        bi = r;
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
                if (lane == 0) {
                    red_v[warp] = best;
                    red_i[warp] = bi;
                }
                __syncthreads();
                if (threadIdx.x == 0) {
                    T bv = red_v[0];
                    int bix = red_i[0];
                    for (int w = 1; w < NWARP; ++w)
                        if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bix)) {
                            bv = red_v[w];
                            bix = red_i[w];
                        }
                    if (!(bv > 0) || bix >= R) {
                        s_bad = 1;
                        bix = kk;
                    }
                    s_p = bix;
                    if (bix != kk) {
                        const int t = rmap[k0 + kk];
                        rmap[k0 + kk] = rmap[k0 + bix];
                        rmap[k0 + bix] = t;
                    }
                }
                __syncthreads();
                if (s_bad) break;
                const int p = s_p;
                if (p != kk && threadIdx.x < PB) {
                    const C t = P[kk * PB + threadIdx.x];
                    P[kk * PB + threadIdx.x] = P[p * PB + threadIdx.x];
                    P[p * PB + threadIdx.x] = t;
                }
                __syncthreads();
                const C inv = cinv(P[kk * PB + kk]);
                for (int r = kk + 1 + threadIdx.x; r < R; r += LU_THREADS) {
                    const C l = cmul(P[r * PB + kk], inv);
                    P[r * PB + kk] = l;
                    for (int c = kk + 1; c < kb; ++c) cfms(P[r * PB + c], l, P[kk * PB + c]);
                }
                __syncthreads();
            }
            if (s_bad) break;
            for (int e = threadIdx.x; e < R * kb; e += LU_THREADS) {
                const int r = e / kb, c = e - r * kb;
                M[(size_t)rmap[k0 + r] * ld + k0 + c] = P[r * PB + c];
            }
            if (threadIdx.x < kb) {
                // column c of L11^-1 by forward substitution (unit diagonal)
                const int c = threadIdx.x;
                for (int i = 0; i < kb; ++i) {
                    C y = czero<C>();
                    if (i == c) y.x = 1;
                    else if (i > c)
                        for (int l = c; l < i; ++l) cfms(y, P[i * PB + l], Li[l * PB + c]);
                    Li[i * PB + c] = y;
                }
            }
            __syncthreads();
            for (int c0 = k0 + kb; c0 <= n; c0 += CW) {
                const int cw = min(CW, n + 1 - c0);
                for (int e = threadIdx.x; e < kb * CW; e += LU_THREADS) {
                    const int i = e / CW, c = e - i * CW;
                    As[e] = c < cw ? M[(size_t)rmap[k0 + i] * ld + c0 + c] : czero<C>();
                }
                __syncthreads();
                for (int e = threadIdx.x; e < kb * CW; e += LU_THREADS) {
                    const int i = e / CW, c = e - i * CW;
                    C s = czero<C>();
                    for (int l = 0; l <= i; ++l) cfma(s, Li[i * PB + l], As[l * CW + c]);
                    Ub[e] = s;
                    if (c < cw) M[(size_t)rmap[k0 + i] * ld + c0 + c] = s;
                }
                __syncthreads();
                const int c = threadIdx.x % CW, rg = threadIdx.x / CW;
                if (c < cw) {
                    C u[PB];
#pragma unroll
                    for (int l = 0; l < PB; ++l) u[l] = l < kb ? Ub[l * CW + c] : czero<C>();
                    for (int r = kb + rg; r < R; r += 4 * RG) {
                        C* dst[4];
                        C acc[4];
#pragma unroll
                        for (int v = 0; v < 4; ++v) {
                            const int rr = r + v * RG;
                            dst[v] = rr < R ? M + (size_t)rmap[k0 + rr] * ld + c0 + c : nullptr;
                            acc[v] = dst[v] ? *dst[v] : czero<C>();
                        }
#pragma unroll
                        for (int l = 0; l < PB; ++l)
#pragma unroll
                            for (int v = 0; v < 4; ++v) {
                                const int rr = min(r + v * RG, R - 1);
                                cfms(acc[v], P[rr * PB + l], u[l]);
                            }
#pragma unroll
                        for (int v = 0; v < 4; ++v)
                            if (dst[v]) *dst[v] = acc[v];
                    }
                }
                __syncthreads();
            }
        }
        const double2 ehh = A[(size_t)h * n + h];
        const double Lno = ehh.y / (ehh.x * ehh.x + ehh.y * ehh.y);
        if (s_bad) {
            if (threadIdx.x == 0) {
                a.flags[id] = 1;
                a.out[id] = 0.0;
                a.out[a.ninst + id] = Lno;
                a.out[2 * a.ninst + id] = 0.0;
            }
            __syncthreads();
            continue;
        }
        if (!want_x) {
            if (threadIdx.x == 0) {
                const C* rowp = M + (size_t)rmap[n - 1] * ld;
                const C xl = cmul(rowp[n], cinv(rowp[n - 1]));
                a.flags[id] = 0;
                a.out[id] = -(double)xl.y;
                a.out[a.ninst + id] = Lno;
                a.out[2 * a.ninst + id] = 0.0;
            }
            __syncthreads();
            continue;
        }
        // back substitution U x = y, PB rows at a time from the bottom
        for (int bk = ((n - 1) / PB) * PB; bk >= 0; bk -= PB) {
            const int kb = min(PB, n - bk);
            for (int i = warp; i < kb; i += NWARP) {
                const C* rowp = M + (size_t)rmap[bk + i] * ld;
                T sx = 0, sy = 0;
                for (int j = bk + kb + lane; j < n; j += 32) {
                    const C u = rowp[j], xv = xs[j];
                    sx = fma(u.x, xv.x, fma(-u.y, xv.y, sx));
                    sy = fma(u.x, xv.y, fma(u.y, xv.x, sy));
                }
                sx = warp_sum(sx);
                sy = warp_sum(sy);
                if (lane == 0) {
                    const C y = rowp[n];
                    C s;
                    s.x = y.x - sx;
                    s.y = y.y - sy;
                    sblk[i] = s;
                }
            }
            for (int e = threadIdx.x; e < kb * kb; e += LU_THREADS) {
                const int i = e / kb, j = e - i * kb;
                Li[i * PB + j] = M[(size_t)rmap[bk + i] * ld + bk + j];
            }
            __syncthreads();
            if (warp == 0) {
                // lane i keeps the running right-hand side of row bk + i
                C s = lane < kb ? sblk[lane] : czero<C>();
                for (int i = kb - 1; i >= 0; --i) {
                    C xi = czero<C>();
                    if (lane == i) xi = cmul(s, cinv(Li[i * PB + i]));
                    xi.x = __shfl_sync(0xffffffffu, xi.x, i);
                    xi.y = __shfl_sync(0xffffffffu, xi.y, i);
                    if (lane < i) cfms(s, Li[lane * PB + i], xi);
                    if (lane == i) s = xi;
                }
                if (lane < kb) xs[bk + lane] = s;
            }
            __syncthreads();
        }
        double2* xg = a.x + in.vec_off;
        int* rg = a.rowmap + in.vec_off;
        for (int i = threadIdx.x; i < n; i += LU_THREADS) {
            xg[i] = make_double2((double)xs[i].x, (double)xs[i].y);
            rg[i] = rmap[i];
        }
        if (threadIdx.x == 0) {
            a.flags[id] = 0;
            a.out[id] = -(double)xs[n - 1].y;
            a.out[a.ninst + id] = Lno;
            a.out[2 * a.ninst + id] = 0.0;
        }
        __syncthreads();
    }
}

// r = e_last - A' x in FP64; task = {instance, first of 32 rows}, 4 rows per warp
__global__ void __launch_bounds__(256) k_resid(BatchSolveArgs a, const int2* tasks) {
    const int2 tk = tasks[blockIdx.x];
    const BatchInst in = a.inst[tk.x];
    const int n = in.ng, h = in.head;
    const double2* A = a.eps + in.eps_off;
    const double2* x = a.x + in.vec_off;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (a.flags[tk.x] == 1) return;
    for (int v = 0; v < 4; ++v) {
        const int i = tk.y + warp * 4 + v;
        if (i >= n) break;
        const double2* row = A + (size_t)head_last(i, n, h) * n;
        double sx = 0.0, sy = 0.0;
        for (int j = lane; j < n; j += 32) {
            const double2 av = row[head_last(j, n, h)], xv = x[j];
            sx = fma(av.x, xv.x, fma(-av.y, xv.y, sx));
            sy = fma(av.x, xv.y, fma(av.y, xv.x, sy));
        }
        sx = warp_sum(sx);
        sy = warp_sum(sy);
        if (lane == 0) a.r[in.vec_off + i] = make_double2((i == n - 1 ? 1.0 : 0.0) - sx, -sy);
    }
}

// d = A'^-1 r with the stored FP32 factors; x += d
__global__ void __launch_bounds__(LU_THREADS) k_lu_correct(BatchSolveArgs a, int nmax, int last) {
    using C = float2;
    constexpr int PB = Pb<float>::v;
    extern __shared__ __align__(16) unsigned char sm[];
    C* b = reinterpret_cast<C*>(sm);                  // [nmax] right-hand side, stored-row order
    C* d = b + nmax;                                  // [nmax] forward then backward solution, logical order
    C* Lt = d + nmax;                                 // [PB][PB] diagonal block
    int* rmap = reinterpret_cast<int*>(Lt + PB * PB); // [nmax]
    __shared__ C sblk[PB];
    __shared__ float s_red[2][NWARP];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    for (int ii = a.cta_off[blockIdx.x]; ii < a.cta_off[blockIdx.x + 1]; ++ii) {
        const int id = a.cta_ids[ii];
        if (a.flags[id] == 1) continue;
        const BatchInst in = a.inst[id];
        const int n = in.ng, ld = n + 1;
        const C* M = reinterpret_cast<const C*>(a.work) + in.work_off;
        for (int i = threadIdx.x; i < n; i += LU_THREADS) {
            const double2 r = a.r[in.vec_off + i];
            b[i] = make_float2((float)r.x, (float)r.y);
            rmap[i] = a.rowmap[in.vec_off + i];
        }
        __syncthreads();
        // forward: L y = P b, one panel of PB columns at a time
        for (int k0 = 0; k0 < n; k0 += PB) {
            const int kb = min(PB, n - k0);
            for (int e = threadIdx.x; e < kb * kb; e += LU_THREADS) {
                const int i = e / kb, l = e - i * kb;
                Lt[i * PB + l] = M[(size_t)rmap[k0 + i] * ld + k0 + l];
            }
            __syncthreads();
            if (warp == 0) {
                C s = lane < kb ? b[rmap[k0 + lane]] : czero<C>();
                for (int l = 0; l < kb; ++l) {
                    C yl;
                    yl.x = __shfl_sync(0xffffffffu, s.x, l);
                    yl.y = __shfl_sync(0xffffffffu, s.y, l);
                    if (lane > l && lane < kb) cfms(s, Lt[lane * PB + l], yl);
                }
                if (lane < kb) d[k0 + lane] = s;
            }
            __syncthreads();
            for (int r = k0 + kb + threadIdx.x; r < n; r += LU_THREADS) {
                const C* rowp = M + (size_t)rmap[r] * ld + k0;
                C s = b[rmap[r]];
                for (int l = 0; l < kb; ++l) cfms(s, rowp[l], d[k0 + l]);
                b[rmap[r]] = s;
            }
            __syncthreads();
        }
        // backward: U d = y
        for (int bk = ((n - 1) / PB) * PB; bk >= 0; bk -= PB) {
            const int kb = min(PB, n - bk);
            for (int i = warp; i < kb; i += NWARP) {
                const C* rowp = M + (size_t)rmap[bk + i] * ld;
                float sx = 0.f, sy = 0.f;
                for (int j = bk + kb + lane; j < n; j += 32) {
                    const C u = rowp[j], xv = d[j];
                    sx = fmaf(u.x, xv.x, fmaf(-u.y, xv.y, sx));
                    sy = fmaf(u.x, xv.y, fmaf(u.y, xv.x, sy));
                }
                sx = warp_sum(sx);
                sy = warp_sum(sy);
                if (lane == 0) sblk[i] = make_float2(d[bk + i].x - sx, d[bk + i].y - sy);
            }
            for (int e = threadIdx.x; e < kb * kb; e += LU_THREADS) {
                const int i = e / kb, j = e - i * kb;
                Lt[i * PB + j] = M[(size_t)rmap[bk + i] * ld + bk + j];
            }
            __syncthreads();
            if (warp == 0) {
                C s = lane < kb ? sblk[lane] : czero<C>();
                for (int i = kb - 1; i >= 0; --i) {
                    C xi = czero<C>();
                    if (lane == i) xi = cmul(s, cinv(Lt[i * PB + i]));
                    xi.x = __shfl_sync(0xffffffffu, xi.x, i);
                    xi.y = __shfl_sync(0xffffffffu, xi.y, i);
                    if (lane < i) cfms(s, Lt[lane * PB + i], xi);
                    if (lane == i) s = xi;
                }
                if (lane < kb) d[bk + lane] = s;
            }
            __syncthreads();
        }
        // x += d; relative size of the correction
        double2* xg = a.x + in.vec_off;
        float dmax = 0.f, xmax = 0.f;
        for (int i = threadIdx.x; i < n; i += LU_THREADS) {
            double2 xv = xg[i];
            xv.x += (double)d[i].x;
            xv.y += (double)d[i].y;
            xg[i] = xv;
            dmax = fmaxf(dmax, hypotf(d[i].x, d[i].y));
            xmax = fmaxf(xmax, (float)hypot(xv.x, xv.y));
        }
        for (int o = 16; o > 0; o >>= 1) {
            dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
            xmax = fmaxf(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
        }
        if (lane == 0) {
            s_red[0][warp] = dmax;
            s_red[1][warp] = xmax;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            float dm = 0.f, xm = 0.f;
            for (int w = 0; w < NWARP; ++w) {
                dm = fmaxf(dm, s_red[0][w]);
                xm = fmaxf(xm, s_red[1][w]);
            }
            const double rel = xm > 0.f ? (double)dm / (double)xm : 0.0;
            const double2 xl = xg[n - 1];
            a.out[id] = -xl.y;
            a.out[2 * a.ninst + id] = rel;
            if (last) a.flags[id] = (rel > REFINE_TOL || !(rel == rel)) ? 2 : 0;
        }
        __syncthreads();
    }
}

template <typename T> size_t lu_smem(int nmax) {
    constexpr int PB = Pb<T>::v;
    return ((size_t)nmax * PB + PB * PB + 2 * PB * CW + nmax) * sizeof(cplx<T>) + nmax * sizeof(int);
}

}  // namespace

cudaError_t qcx_launch_lu_head(cudaStream_t st, const BatchSolveArgs& a, int grid, int nmax, bool fp64, bool want_x) {
    if (grid < 1 || nmax < 1) return cudaErrorInvalidValue;
    if (fp64) {
        const size_t smem = lu_smem<double>(nmax);
        cudaError_t e = cudaFuncSetAttribute((const void*)k_lu_head<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lu_head<double><<<grid, LU_THREADS, smem, st>>>(a, nmax, want_x ? 1 : 0);
    } else {
        const size_t smem = lu_smem<float>(nmax);
        cudaError_t e = cudaFuncSetAttribute((const void*)k_lu_head<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_lu_head<float><<<grid, LU_THREADS, smem, st>>>(a, nmax, want_x ? 1 : 0);
    }
    return cudaGetLastError();
}

cudaError_t qcx_launch_resid(cudaStream_t st, const BatchSolveArgs& a, const int2* tasks, int ntask) {
    if (ntask < 1) return cudaErrorInvalidValue;
    k_resid<<<ntask, 256, 0, st>>>(a, tasks);
    return cudaGetLastError();
}

cudaError_t qcx_launch_lu_correct(cudaStream_t st, const BatchSolveArgs& a, int grid, int nmax, int last) {
    if (grid < 1 || nmax < 1) return cudaErrorInvalidValue;
    constexpr int PB = Pb<float>::v;
    const size_t smem = (2 * (size_t)nmax + PB * PB) * sizeof(float2) + nmax * sizeof(int);
    cudaError_t e =
        cudaFuncSetAttribute((const void*)k_lu_correct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_lu_correct<<<grid, LU_THREADS, smem, st>>>(a, nmax, last);
    return cudaGetLastError();
}
