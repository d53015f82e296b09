// The Kramers-Kronig contraction of the spectral route (mixed precision) on the
// tcgen05 tensor cores:
//
//   chi0(w)[G][G'] = sum_b K(w, E_b) S_b[G][G'],   K(w, E) = 1/(w - E + i eta) - 1/(w + E + i eta),
//
// as one real GEMM per chunk of grid points,
//   D[m][n] = sum_b A[m][b] B[n][b],
//   m = 2 w + r      A = (Re K, Im K)(w, E_b)                       (r = 0, 1)
//   n = 2 X + c      B = (Re S, Im S)_b at the upper (G, G') pair X  (c = 0, 1)
// so that with Ar = D[2w][2X], Bi = D[2w+1][2X+1], Cs = D[2w][2X+1], Dr = D[2w+1][2X]
//   chi0[G][G'] = (Ar - Bi) + i (Cs + Dr),   chi0[G'][G] = (Ar + Bi) + i (Dr - Cs)
// (S_b is Hermitian; X runs over the 32 x 32 tiles with G-tile <= G'-tile, X = p 1024 + 32 r + c).
//
// Both operands are split into three BF16 terms (the six products of order <= 2 are
// accumulated, as in the direct route's kernel) and stored K-major: the K table as
// [2 N_w (padded)][grid points], the weights of one chunk as [2 x 1024 x tile pairs][chunk
// points], both loaded by TMA into 64-byte-swizzled stages.  FP32 accumulation in TMEM is
// restarted every two K stages (24 MMAs; the tensor core's FP32 sums truncate) and the window
// sums are added in FP32 registers, so a chunk is summed in two levels; chunks are added into
// an FP64 chi0 in the epilogue.
//
// CTA: one 128-row M tile (64 frequencies) x one 128-column N tile (64 pairs).  Warps: 0 TMA
// producer; 1 and 10 MMA issuers on alternate accumulation windows (TMEM buffers 0 and 1);
// 2-9 drain the accumulators and run the epilogue; 11 idles.  Every wait is bounded: on
// timeout the kernel records an error status, lets its own copies and MMAs finish, frees
// TMEM and returns.
#include "qcx_internal.h"
#include "tc_ptx.cuh"

namespace {

constexpr int SK_THREADS = 384;
constexpr int SK_MMA2 = 10;
constexpr int SK_NSTAGE = 4;
constexpr int SK_N = 128;                   // columns per CTA (64 pairs x re/im)
constexpr int SK_M = 128;                   // rows per CTA (64 frequencies x re/im)
constexpr int SK_PROMOTE = 2;               // K stages accumulated in one TMEM buffer
constexpr int SK_TILE = SK_M * ROWB;        // one 128-row operand piece (8 KB)
constexpr int SK_STAGE = 6 * SK_TILE;       // three A pieces and three B pieces
constexpr int SK_HALF = SK_N / 2;           // columns one drain thread owns

struct SkArgs {
    int nw, ng;
    int kstages;                            // K stages of 32 grid points in this chunk
    int kb0;                                // first grid point of the chunk (column of the K planes)
    const int2* tp;                         // upper tile pairs
    int accumulate;                         // add into chi (later chunks) instead of storing
    double2* chi;                           // [nw][ng][ng]
    int* status;
    long long wait_limit;
};

__global__ void __launch_bounds__(SK_THREADS, 1)
    k_spec_kk_tc(const __grid_constant__ CUtensorMap ka0, const __grid_constant__ CUtensorMap ka1,
                 const __grid_constant__ CUtensorMap ka2, const __grid_constant__ CUtensorMap sb0,
                 const __grid_constant__ CUtensorMap sb1, const __grid_constant__ CUtensorMap sb2, SkArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mt = blockIdx.x, nt = blockIdx.y;
    unsigned char* tail = base + SK_NSTAGE * SK_STAGE;
    // copy barriers of K stage it are number it mod 2 NSTAGE (ring slot it mod NSTAGE), so the
    // previous phase of one lies at least two accumulation windows back for an issuer
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail);
    uint64_t* full = bars;                          // [2 NSTAGE] both operands landed
    uint64_t* empty = bars + 2 * SK_NSTAGE;         // [NSTAGE] MMAs of the slot done
    uint64_t* acc_full = bars + 3 * SK_NSTAGE;      // [2] TMEM buffer holds a finished window
    uint64_t* drained = acc_full + 2;               // [2] TMEM buffer read out (8 warps)
    uint64_t* mma_done = drained + 2;               // every issued MMA finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < 2 * SK_NSTAGE; ++s) mbar_init(&full[s], 1);
        for (int s = 0; s < SK_NSTAGE; ++s) mbar_init(&empty[s], 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&drained[b], 8);
        }
        mbar_init(mma_done, 2);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, 2 * SK_N);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nwin = (a.kstages + SK_PROMOTE - 1) / SK_PROMOTE;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            int last = -1;
            for (int it = 0; it < a.kstages; ++it) {
                const int s = it % SK_NSTAGE;
                const uint32_t ph = (uint32_t)(it / SK_NSTAGE) & 1u;
                if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, a.status, a.wait_limit)) break;
                uint64_t* fb = &full[it % (2 * SK_NSTAGE)];
                unsigned char* st = base + s * SK_STAGE;
                mbar_arrive_tx(fb, SK_STAGE);
                const int xk = a.kb0 + it * KSTEP, xs = it * KSTEP;
                tma_load_2d(st, &ka0, fb, xk, mt * SK_M);
                tma_load_2d(st + SK_TILE, &ka1, fb, xk, mt * SK_M);
                tma_load_2d(st + 2 * SK_TILE, &ka2, fb, xk, mt * SK_M);
                tma_load_2d(st + 3 * SK_TILE, &sb0, fb, xs, nt * SK_N);
                tma_load_2d(st + 4 * SK_TILE, &sb1, fb, xs, nt * SK_N);
                tma_load_2d(st + 5 * SK_TILE, &sb2, fb, xs, nt * SK_N);
                last = it;
            }
            // let every copy still in flight (at most the last NSTAGE stages) land before the CTA can exit
            for (int it = max(0, last - SK_NSTAGE + 1); it <= last; ++it)
                mbar_wait(&full[it % (2 * SK_NSTAGE)], (uint32_t)(it / (2 * SK_NSTAGE)) & 1u, abort_flag, a.status,
                          CLEANUP_WAIT_LIMIT, false);
        }
    } else if (warp == 1 || warp == SK_MMA2) {
        // ---------------------------------------------------------------- MMA issuers
        if (lane == 0) {
            const int par = warp == 1 ? 0 : 1;
            const uint32_t idesc = make_idesc(SK_M, SK_N);
            bool ok = true;
            for (int win = par; win < nwin && ok; win += 2) {
                const int b = win & 1;
                if (win >= 2 &&
                    !mbar_wait(&drained[b], (uint32_t)((win - 2) >> 1) & 1u, abort_flag, a.status, a.wait_limit))
                    break;
                const int it1 = min((win + 1) * SK_PROMOTE, a.kstages);
                for (int it = win * SK_PROMOTE; it < it1; ++it) {
                    const int s = it % SK_NSTAGE;
                    const bool first = it == win * SK_PROMOTE;
                    if (!mbar_wait(&full[it % (2 * SK_NSTAGE)], (uint32_t)(it / (2 * SK_NSTAGE)) & 1u, abort_flag,
                                   a.status, a.wait_limit)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    unsigned char* st = base + s * SK_STAGE;
                    const uint32_t a0 = smem_u32(st), a1 = a0 + SK_TILE, a2 = a1 + SK_TILE;
                    const uint32_t b0 = a2 + SK_TILE, b1 = b0 + SK_TILE, b2 = b1 + SK_TILE;
                    const uint32_t d = tmem + (uint32_t)(b * SK_N);
#pragma unroll
                    for (int kk = 0; kk < KSTEP / 16; ++kk) {
                        const uint32_t off = kk * 32;
                        umma_bf16(d, sw64_desc(a0 + off), sw64_desc(b0 + off), idesc, (first && kk == 0) ? 0u : 1u);
                        umma_bf16(d, sw64_desc(a0 + off), sw64_desc(b1 + off), idesc, 1u);
                        umma_bf16(d, sw64_desc(a1 + off), sw64_desc(b0 + off), idesc, 1u);
                        umma_bf16(d, sw64_desc(a0 + off), sw64_desc(b2 + off), idesc, 1u);
                        umma_bf16(d, sw64_desc(a1 + off), sw64_desc(b1 + off), idesc, 1u);
                        umma_bf16(d, sw64_desc(a2 + off), sw64_desc(b0 + off), idesc, 1u);
                    }
                    umma_commit(&empty[s]);
                }
                if (ok) umma_commit(&acc_full[b]);
            }
            // no MMA of either issuer may still be running when TMEM is freed (also on the abort path)
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, abort_flag, a.status, CLEANUP_WAIT_LIMIT, false);
        }
    } else if (warp < SK_MMA2) {
        // ------------------------------------------------------ accumulator drain, epilogue
        const int q = warp & 3, hc = (warp - 2) >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        float part[SK_HALF];
#pragma unroll
        for (int i = 0; i < SK_HALF; ++i) part[i] = 0.0f;
        bool ok = true;
        for (int wd = 0; wd < nwin && ok; ++wd) {
            const int b = wd & 1;
            if (!(ok = warp_wait(&acc_full[b], (uint32_t)(wd >> 1) & 1u, abort_flag, a.status, a.wait_limit))) break;
            tc_fence_after();
            const uint32_t tb = tmem + lane_off + (uint32_t)(b * SK_N + hc * SK_HALF);
#pragma unroll
            for (int grp = 0; grp < SK_HALF / 16; ++grp) {
                uint32_t r[2][8];
                tmem_ld8(tb + (uint32_t)(grp * 16), r[0]);
                tmem_ld8(tb + (uint32_t)(grp * 16 + 8), r[1]);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int i = 0; i < 8; ++i) part[grp * 16 + u * 8 + i] += __uint_as_float(r[u][i]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drained[b]);
        }
        // ------------------------------------------------------------------ epilogue
        // a warp holds rows 32q .. 32q+31: lanes 2j and 2j+1 are the (Re K, Im K) rows of one
        // frequency; the even lane combines the first 16 pairs of the thread's 32, the odd lane
        // the last 16
        if (ok) {                                   // warp-uniform (the waits are warp-wide)
            const int row = q * 32 + lane;
            const int w = mt * (SK_M / 2) + (row >> 1);
            const bool odd = lane & 1;
#pragma unroll
            for (int xl = 0; xl < SK_HALF / 4; ++xl) {
                // even lane: pair xl of the thread's 32, odd lane: pair xl + 16; each sends the
                // partner the two values of its row that the partner's pair needs
                const int lo = 2 * xl, hi = 2 * (xl + SK_HALF / 4);
                const float s0 = odd ? part[lo] : part[hi], s1 = odd ? part[lo + 1] : part[hi + 1];
                const float r0 = __shfl_xor_sync(0xffffffffu, s0, 1), r1 = __shfl_xor_sync(0xffffffffu, s1, 1);
                const double Ar = odd ? r0 : part[lo], Cs = odd ? r1 : part[lo + 1];
                const double Dr = odd ? part[hi] : r0, Bi = odd ? part[hi + 1] : r1;
                const int xo = odd ? xl + SK_HALF / 4 : xl;
                const long long P = (long long)nt * (SK_N / 2) + hc * (SK_HALF / 2) + xo;
                const int p = (int)(P >> 10), X = (int)(P & 1023);
                const int2 pr = a.tp[p];
                const int G = pr.x * 32 + (X >> 5), H = pr.y * 32 + (X & 31);
                if (w >= a.nw || G >= a.ng || H >= a.ng) continue;
                double2* d = a.chi + ((size_t)w * a.ng + G) * a.ng + H;
                const double2 gh = make_double2(Ar - Bi, Cs + Dr);
                if (a.accumulate) {
                    d->x += gh.x;
                    d->y += gh.y;
                } else {
                    *d = gh;
                }
                if (pr.x != pr.y) {
                    double2* e = a.chi + ((size_t)w * a.ng + H) * a.ng + G;
                    const double2 hg = make_double2(Ar + Bi, Dr - Cs);
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
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * SK_N);
    }
}

// K table as three BF16 planes [rows][ld], row 2 w + r = (Re, Im) K(w, E_b) (FP64, rounded to
// FP32, split); zero for padded rows and for b >= nbin
__global__ void k_spec_ktab_split(int nw, int rows, long long ld, int nbin, const double* w, double E0, double step,
                                  double eta, __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2) {
    const long long n = (long long)rows * ld;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const int m = (int)(i / ld);
        const long long b = i - (long long)m * ld;
        const int iw = m >> 1;
        float v = 0.f;
        if (iw < nw && b < nbin) {
            const double E = E0 + step * (double)b;
            const double am = w[iw] - E, ap = w[iw] + E;
            const double d1 = 1.0 / (am * am + eta * eta), d2 = 1.0 / (ap * ap + eta * eta);
            v = (float)((m & 1) ? eta * (d2 - d1) : am * d1 - ap * d2);
        }
        const __nv_bfloat16 h0 = __float2bfloat16_rn(v);
        const float r1 = v - __bfloat162float(h0);
        const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
        p0[i] = h0;
        p1[i] = h1;
        p2[i] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
    }
}

// weights of one chunk [pair][point][32][32] (FP32 complex) -> three BF16 planes [2 x 1024 x pair][ld]
// (row 2 X + c, column = point in the chunk); zero for points >= nb.  Block (32, 8): a 32-point x
// 32-pair tile through shared memory.
__global__ void __launch_bounds__(256) k_spec_s_split(int nbc, int nb, long long ld, const float2* S,
                                                      __nv_bfloat16* p0, __nv_bfloat16* p1, __nv_bfloat16* p2) {
    __shared__ float2 t[32][33];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long X0 = (long long)blockIdx.x * 32;     // global pair index p 1024 + X
    const int b0 = blockIdx.y * 32;
    const long long p = X0 >> 10;
    const int xin = (int)(X0 & 1023);
    for (int j = ty; j < 32; j += 8) {
        const int b = b0 + j;
        float2 v = make_float2(0.f, 0.f);
        if (b < nb) v = S[((size_t)p * nbc + b) * 1024 + xin + tx];
        t[tx][j] = v;
    }
    __syncthreads();
    for (int j = ty; j < 32; j += 8) {
        const float2 v = t[j][tx];                       // pair X0 + j, point b0 + tx
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float x = c ? v.y : v.x;
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
            const float r1 = x - __bfloat162float(h0);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
            const size_t o = (size_t)(2 * (X0 + j) + c) * ld + b0 + tx;
            p0[o] = h0;
            p1[o] = h1;
            p2[o] = __float2bfloat16_rn(r1 - __bfloat162float(h1));
        }
    }
}

}  // namespace

size_t qcx_spec_tc_smem() { return 1024 + (size_t)SK_NSTAGE * SK_STAGE + (3 * SK_NSTAGE + 5) * 8 + 16; }

cudaError_t qcx_spec_tc_ktab(cudaStream_t st, int nw, int rows, long long ld, int nbin, const double* w, double E0,
                             double step, double eta, __nv_bfloat16* planes) {
    const long long n = (long long)rows * ld;
    k_spec_ktab_split<<<(int)std::min<long long>((n + 255) / 256, 16384), 256, 0, st>>>(
        nw, rows, ld, nbin, w, E0, step, eta, planes, planes + n, planes + 2 * n);
    return cudaGetLastError();
}

cudaError_t qcx_spec_tc_contract(cudaStream_t st, const CUtensorMap* kmaps, const CUtensorMap* smaps, int mtiles,
                                 int ntiles, int nw, int ng, int nbc, int nb, int kb0, long long sld, const float2* S,
                                 __nv_bfloat16* splanes, const int2* tp, int accumulate, double2* chi, int* status,
                                 long long wait_limit) {
    const long long n = (long long)ntiles * SK_N * sld;     // elements per weight plane
    dim3 sg((unsigned)((long long)ntiles * SK_N / 2 / 32), (unsigned)(sld / 32));
    k_spec_s_split<<<sg, dim3(32, 8), 0, st>>>(nbc, nb, sld, S, splanes, splanes + n, splanes + 2 * n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    SkArgs a;
    a.nw = nw;
    a.ng = ng;
    a.kstages = (nb + KSTEP - 1) / KSTEP;
    a.kb0 = kb0;
    a.tp = tp;
    a.accumulate = accumulate;
    a.chi = chi;
    a.status = status;
    a.wait_limit = wait_limit;
    const size_t smem = qcx_spec_tc_smem();
    e = cudaFuncSetAttribute((const void*)k_spec_kk_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_spec_kk_tc<<<dim3(mtiles, ntiles), SK_THREADS, smem, st>>>(kmaps[0], kmaps[1], kmaps[2], smaps[0], smaps[1],
                                                                   smaps[2], a);
    return cudaGetLastError();
}
