// Mixed-precision chi0 (Eq. (RPA)) on the tcgen05 tensor cores with the Dyson
// step fused in the epilogue.
//
// The complex contraction chi0_GG'(w) = pref sum_t W_t(w) conj(rho_t(G)) rho_t(G')
// is one real GEMM per q,
//   D[m][n] = sum_k A[m][k] B[n][k],   k = 2t + p (p = 0 real, 1 imaginary part),
//   n = G,  m = (G'-block, w, re|im, G' in block),
//   B[G][2t+p]           = (Re, Im) rho~_t(G)                                (operand read by TMA)
//   A[(w,re,G')][2t+p]   = (Re, Im) (W_t(w) rho~_t(G'))                     (generated in shared memory)
//   A[(w,im,G')][2t+p]   = (Im, -Re)(W_t(w) rho~_t(G')),
// so the re rows of D hold Re chi0_GG' and the im rows Im chi0_GG'.
//
// Precision.  B is rho~ = b0 + b1, the first two BF16 terms of the FP32 pair
// densities (16 significant bits), held exactly by the two planes; A is built
// from the same rho~ and split into three BF16 terms a = a0 + a1 + a2 (24 bits);
// D accumulates in FP32 the five products a0 b0 + a0 b1 + a1 b0 + a1 b1 + a2 b0
// (the one left out, a2 b1, is ~2^-24 of a b).  Because both sides carry the
// same rho~, the truncation of B is not an error of the contraction: the result
// is chi0 of the pair densities rho~ (a relative change of 2^-17 in each, which
// keeps the Hermitian part from Re W and the anti-Hermitian part from Im W
// apart).  Only the A side's 2^-24 and the dropped product are errors of the
// contraction, and those are what the inverse's condition number and the
// cancellation |Re W| |rho|^2 -> |Im W| |rho|^2 amplify.  (Truncating both sides to
// two terms with three or four products leaves 2^-17 on A and misses 1e-4 on
// the loss with local fields; two FP16 terms, scaled by powers of two, missed
// it too.)  W_t(w) = 1/(w - dE + i eta) - 1/(w + dE + i eta) is tabulated per q
// by k_weights with dE and w -+ dE in FP64 and fetched with each K stage.
//
// The tensor core's FP32 accumulation truncates, so long sums drift (about
// 2^-24 of the running value per MMA, always toward zero).  The accumulator
// is therefore restarted every PROMOTE K stages (20 MMAs; 40-MMA windows were 7 % faster
// but put the high-frequency heads of the uneven instances at 1e-4): TMEM holds two buffers used
// in turn, the finished buffer is drained into FP32 registers (round to
// nearest), and every FLUSH stages the register partials are added into an
// FP64 buffer owned by the CTA.  The Dyson step runs in FP64 from that
// buffer and eps is stored in FP64.
//
// CTA work item: one 64-row G' block, one frequency (a 128 x N accumulator:
// 64 re rows and 64 im rows), one N chunk of G.  Warp roles (five warpgroups):
// warp 0 issues TMA loads of the B tiles (and, when the G range is split, of the
// A-source rows); warp 1 owns TMEM; one thread of warp 1 issues the MMAs of the
// even accumulation windows and one thread of warp 2 those of the odd windows;
// warps 4-11 form W and the A tiles; warps 12-19 drain the accumulators and run
// the epilogue (eps = delta - v^1/2 chi0 v^1/2).  Every wait is bounded: on
// timeout the kernel records an error status, lets its own copies and MMAs
// finish, frees TMEM and returns.
#include "qcx_internal.h"
#include "tc_ptx.cuh"

#include <algorithm>

namespace {

// Five warpgroups.  WG0: warp 0 issues the TMA copies, warp 1 owns TMEM and with warp 2 issues
// the MMAs (alternate accumulation windows), warp 3 idles.  WG1-WG2 (warps 4-11) form W rho~
// and the A tiles.  WG3-WG4 (warps 12-19) drain the accumulators and run the epilogue.  A
// generation and the drain run in separate warps so that neither waits for the other; the
// drain warps hold 96 FP32 partial sums each, so the warpgroups trade registers (setmaxnreg):
// 40 for WG0, 64 for the A warps, 152 for the drain warps, 60416 in all of the 640 x 96
// the block is launched with (the launch is refused if the kernel was built with another count).
constexpr int NTHREADS = 640;
constexpr int LAUNCH_REGS = 96;              // 65536 / 640, rounded down to the allocation granule
constexpr int REG_CTRL = 40, REG_AGEN = 64, REG_DRAIN = 152;
static_assert(128 * REG_CTRL + 256 * REG_AGEN + 256 * REG_DRAIN <= NTHREADS * LAUNCH_REGS,
              "warpgroup register budgets exceed the launch allocation");
constexpr int MMA_WARP2 = 2;
constexpr int AGEN_WARP0 = 4;                // first A-generation warp (8 warps)
constexpr int DRAIN_WARP0 = 12;              // first drain/epilogue warp (8 warps)
constexpr int NSTAGE = 4;
constexpr int NPA = 3;                    // BF16 terms of the A operand (W rho~)
constexpr int NPB = 2;                    // BF16 terms of the B operand (rho~ = b0 + b1)
constexpr int ATILE = 128 * ROWB;         // one 128-row A piece
constexpr int GBLK = 64;                  // G' rows per half tile
constexpr int PROMOTE = 2;                // K stages accumulated in one TMEM buffer (20 MMAs)
constexpr int FLUSH = 128;                // stages between FP64 flushes of the register partials
constexpr int MAXHALF = 96;               // columns of the accumulator one thread drains (n_tile/2)
constexpr int SMEM_LIMIT = 232448;
constexpr int PREFETCH = 4;               // K stages between the L2 prefetch of a stage and its copy

struct TcArgs {
    int ng, nw, nv, nc;
    long long nt;
    int n_tile, n_gb, kstages, src_from_b;
    uint32_t acc_off, tmem_cols;      // second TMEM buffer column, columns allocated
    const float2* wtab;   // [nw][kp/2] W_t(w) in FP32 (tabulated with FP64 dE)
    long long wld;        // row length of wtab
    double pref;
    const double* vs;
    double* acc64;    // [grid][n_tile][128] FP64 partial sums, one region per CTA (column-major, so a
                      // warp's 32 accumulator rows are contiguous)
    double2* eps;     // [nw][ng][ng], eps^T: row G', column G (FP64)
    double2* chi;     // optional [nw][ng][ng], row G, column G'
    int* status;
    long long wait_limit;   // clock cycles before a pipeline wait gives up
    int withhold;           // fault injection: issue no copies
};

__global__ void __launch_bounds__(NTHREADS, 1)
    k_chi0_tc(const __grid_constant__ CUtensorMap mb0, const __grid_constant__ CUtensorMap mb1,
              const __grid_constant__ CUtensorMap ms0, const __grid_constant__ CUtensorMap ms1, TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gb = blockIdx.x / a.nw, iw = blockIdx.x % a.nw;
    const int n0 = blockIdx.y * a.n_tile;
    const uint32_t bbytes = (uint32_t)a.n_tile * ROWB;          // one B piece
    const uint32_t spiece = (uint32_t)GBLK * ROWB;              // one A-source piece
    const uint32_t sbytes = a.src_from_b ? 0u : NPB * spiece;
    const uint32_t aoff = NPB * bbytes + sbytes;                // A pieces start here in a stage
    const uint32_t stage_bytes = aoff + NPA * ATILE;
    constexpr int TPS = KSTEP / 2;                              // transitions per stage
    unsigned char* tail = base + NSTAGE * stage_bytes;
    float2* Wbuf = reinterpret_cast<float2*>(tail);             // [NSTAGE][TPS]
    // The copy and A-tile barriers of K stage it are number it mod 2 NSTAGE (ring slot it mod
    // NSTAGE): the previous phase of such a barrier lies at least two accumulation windows back
    // for an MMA issuer, so no wait can pass a phase early.
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail + NSTAGE * TPS * sizeof(float2));
    uint64_t* full_b = bars;                     // [2 NSTAGE] TMA landed
    uint64_t* full_a = bars + 2 * NSTAGE;        // [2 NSTAGE] A tiles written (8 warps)
    uint64_t* empty = bars + 4 * NSTAGE;         // [NSTAGE] MMAs of the slot done (smem reusable)
    uint64_t* acc_full = bars + 5 * NSTAGE;      // [2] TMEM buffer holds a finished window
    uint64_t* drained = acc_full + 2;        // [2] TMEM buffer read out (8 warps)
    uint64_t* mma_done = drained + 2;        // every issued MMA finished
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mma_done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

    if (threadIdx.x == 0) {
        for (int s = 0; s < NSTAGE; ++s) {
            mbar_init(&full_b[s], 1);
            mbar_init(&full_a[s], 8);
            mbar_init(&full_b[s + NSTAGE], 1);
            mbar_init(&full_a[s + NSTAGE], 8);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&drained[b], 8);
        }
        mbar_init(mma_done, 2);     // one commit per MMA issuer
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 1) tmem_alloc(tmem_slot, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nwin = (a.kstages + PROMOTE - 1) / PROMOTE;

    if (warp < AGEN_WARP0) {
        regs_dec<REG_CTRL>();
        if (warp == 0) {
            // ------------------------------------------------------ TMA producer
            if (lane == 0) {
                // a stage's lines are requested into L2 a few stages before its copy is issued
                auto prefetch = [&](int it) {
                    bulk_prefetch(a.wtab + (size_t)iw * a.wld + (size_t)it * TPS, TPS * sizeof(float2));
                    tma_prefetch_2d(&mb0, it * KSTEP, n0);
                    tma_prefetch_2d(&mb1, it * KSTEP, n0);
                    if (!a.src_from_b) {
                        tma_prefetch_2d(&ms0, it * KSTEP, gb * GBLK);
                        tma_prefetch_2d(&ms1, it * KSTEP, gb * GBLK);
                    }
                };
                for (int it = 0; it < PREFETCH && it < a.kstages; ++it) prefetch(it);
                int last = -1;
                // with copies withheld (fault injection for tests) nothing is issued, so the
                // consumers' first waits run out and the kernel reports a timeout
                for (int it = 0; it < (a.withhold ? 0 : a.kstages); ++it) {
                    const int s = it % NSTAGE;
                    const uint32_t ph = (uint32_t)(it / NSTAGE) & 1u;
                    if (it + PREFETCH < a.kstages) prefetch(it + PREFETCH);
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, a.status, a.wait_limit)) break;
                    uint64_t* fb = &full_b[it % (2 * NSTAGE)];
                    unsigned char* st = base + s * stage_bytes;
                    mbar_arrive_tx(fb, NPB * bbytes + sbytes + TPS * (uint32_t)sizeof(float2));
                    bulk_load(Wbuf + s * TPS, a.wtab + (size_t)iw * a.wld + (size_t)it * TPS, TPS * sizeof(float2),
                              fb);
                    tma_load_2d(st, &mb0, fb, it * KSTEP, n0);
                    tma_load_2d(st + bbytes, &mb1, fb, it * KSTEP, n0);
                    if (!a.src_from_b) {
                        unsigned char* sp = st + NPB * bbytes;
                        tma_load_2d(sp, &ms0, fb, it * KSTEP, gb * GBLK);
                        tma_load_2d(sp + spiece, &ms1, fb, it * KSTEP, gb * GBLK);
                    }
                    last = it;
                }
                // let every copy still in flight (at most the last NSTAGE stages) land before the CTA can exit
                for (int it = max(0, last - NSTAGE + 1); it <= last; ++it)
                    mbar_wait(&full_b[it % (2 * NSTAGE)], (uint32_t)(it / (2 * NSTAGE)) & 1u, abort_flag, a.status,
                              CLEANUP_WAIT_LIMIT, false);
            }
        } else if (warp == 1 || warp == MMA_WARP2) {
            // ------------------------------------------------------ MMA issuers
            // Issuing tcgen05.mma keeps the issuing thread busy for about as long as the
            // MMAs run, so one thread's barrier waits and bookkeeping would leave the
            // tensor pipe idle between stages.  Two issuers take alternate accumulation
            // windows (TMEM buffer 0 and 1), so one waits while the other's MMAs run.
            if (lane == 0) {
                const int par = warp == 1 ? 0 : 1;
                const uint32_t idesc = make_idesc(128, a.n_tile);
                bool ok = true;
                for (int win = par; win < nwin && ok; win += 2) {
                    const int b = win & 1;
                    if (win >= 2 &&
                        !mbar_wait(&drained[b], (uint32_t)((win - 2) >> 1) & 1u, abort_flag, a.status, a.wait_limit))
                        break;
                    const int it1 = min((win + 1) * PROMOTE, a.kstages);
                    for (int it = win * PROMOTE; it < it1; ++it) {
                        const int s = it % NSTAGE;
                        const bool first = it == win * PROMOTE;
                        // the A warps arrive only after they saw this stage's copies land
                        if (!mbar_wait(&full_a[it % (2 * NSTAGE)], (uint32_t)(it / (2 * NSTAGE)) & 1u, abort_flag,
                                       a.status, a.wait_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        unsigned char* st = base + s * stage_bytes;
                        const uint32_t b0 = smem_u32(st), b1 = b0 + bbytes;
                        const uint32_t d = tmem + (uint32_t)b * a.acc_off;
                        const uint32_t a0 = smem_u32(st + aoff), a1 = a0 + ATILE, a2 = a1 + ATILE;
#pragma unroll
                        for (int kk = 0; kk < KSTEP / 16; ++kk) {
                            const uint32_t off = kk * 32;
                            umma_bf16(d, sw64_desc(a0 + off), sw64_desc(b0 + off), idesc,
                                      (first && kk == 0) ? 0u : 1u);
                            umma_bf16(d, sw64_desc(a0 + off), sw64_desc(b1 + off), idesc, 1u);
                            umma_bf16(d, sw64_desc(a1 + off), sw64_desc(b0 + off), idesc, 1u);
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
        }
    } else if (warp < DRAIN_WARP0) {
        regs_dec<REG_AGEN>();
        // ------------------------------------------------------------ A generation
        const int g = threadIdx.x - 32 * AGEN_WARP0;   // 0..255
        const int j = g & 3;                           // 16-byte chunk = 4 transitions
        const int go = g >> 2;                         // G' offset in the block (0..63)
        const int Gp = gb * GBLK + go;
        for (int it = 0; it < a.kstages; ++it) {
            const int s = it % NSTAGE;
            const int s2 = it % (2 * NSTAGE);
            // the producer issued this stage's copies only after the MMAs of its previous use
            // finished, so a landed stage is also free to overwrite
            if (!warp_wait(&full_b[s2], (uint32_t)(it / (2 * NSTAGE)) & 1u, abort_flag, a.status, a.wait_limit))
                break;
            unsigned char* st = base + s * stage_bytes;
            const unsigned char* srcb = a.src_from_b ? st : st + NPB * bbytes;
            const uint32_t src_piece = a.src_from_b ? bbytes : spiece;
            uint32_t re0[4] = {0, 0, 0, 0}, re1[4] = {0, 0, 0, 0}, re2[4] = {0, 0, 0, 0};   // re row
            uint32_t im0[4] = {0, 0, 0, 0}, im1[4] = {0, 0, 0, 0}, im2[4] = {0, 0, 0, 0};   // im row
            if (Gp < a.ng) {
                const int srow = a.src_from_b ? Gp : go;
                const uint32_t coff = sw64_off(srow, j);
                const uint4 h0 = *reinterpret_cast<const uint4*>(srcb + coff);
                const uint4 h1 = *reinterpret_cast<const uint4*>(srcb + src_piece + coff);
                const uint32_t v0[4] = {h0.x, h0.y, h0.z, h0.w}, v1[4] = {h1.x, h1.y, h1.z, h1.w};
                const float4* Wv4 = reinterpret_cast<const float4*>(Wbuf + s * TPS + 4 * j);
                const float4 wa = Wv4[0], wb = Wv4[1];
                const float2 Wv[4] = {make_float2(wa.x, wa.y), make_float2(wa.z, wa.w), make_float2(wb.x, wb.y),
                                      make_float2(wb.z, wb.w)};
#pragma unroll
                for (int qq = 0; qq < 4; ++qq) {
                    // rho~ = b0 + b1 is exact in FP32 (16 significant bits)
                    const float2 f0 = bf2(v0[qq]), f1 = bf2(v1[qq]);
                    const float rr = f0.x + f1.x, ri = f0.y + f1.y;
                    const float2 wq = Wv[qq];
                    const float xr = wq.x * rr - wq.y * ri;
                    const float xi = wq.x * ri + wq.y * rr;
                    split3(xr, xi, re0[qq], re1[qq], re2[qq]);
                    // (xi, -xr) splits into the same terms as (xr, xi), swapped, the second negated
                    im0[qq] = perm_im(re0[qq]);
                    im1[qq] = perm_im(re1[qq]);
                    im2[qq] = perm_im(re2[qq]);
                }
            }
            unsigned char* ap = st + aoff;
            const uint32_t o_re = sw64_off(go, j), o_im = sw64_off(64 + go, j);
            *reinterpret_cast<uint4*>(ap + o_re) = make_uint4(re0[0], re0[1], re0[2], re0[3]);
            *reinterpret_cast<uint4*>(ap + ATILE + o_re) = make_uint4(re1[0], re1[1], re1[2], re1[3]);
            *reinterpret_cast<uint4*>(ap + 2 * ATILE + o_re) = make_uint4(re2[0], re2[1], re2[2], re2[3]);
            *reinterpret_cast<uint4*>(ap + o_im) = make_uint4(im0[0], im0[1], im0[2], im0[3]);
            *reinterpret_cast<uint4*>(ap + ATILE + o_im) = make_uint4(im1[0], im1[1], im1[2], im1[3]);
            *reinterpret_cast<uint4*>(ap + 2 * ATILE + o_im) = make_uint4(im2[0], im2[1], im2[2], im2[3]);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_a[s2]);
        }
    } else {
        regs_inc<REG_DRAIN>();
        // ---------------------------------------------- accumulator drain and epilogue
        const int wi = warp - DRAIN_WARP0;  // 0..7
        // TMEM lane quadrant q (a warp reads the lanes 32 (warp mod 4) ..), column half hc
        const int q = warp & 3, hc = wi >> 2;
        const int half = a.n_tile >> 1;
        const int nch16 = half >> 4;        // 16-column TMEM loads per thread (half is a multiple of 8)
        const bool tail8 = (half & 15) != 0;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int row = q * 32 + lane;      // accumulator row: 0..63 re, 64..127 im
        double* acc64 = a.acc64 + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * 128 * a.n_tile +
                        (size_t)(hc * half) * 128 + row;
        float part[MAXHALF];
#pragma unroll
        for (int i = 0; i < MAXHALF; ++i) part[i] = 0.0f;
        bool ok = true;
        int flushed = 0;                    // FP64 region initialised?
        for (int wd = 0; wd < nwin && ok; ++wd) {
            const int b = wd & 1;
            if (!(ok = warp_wait(&acc_full[b], (uint32_t)(wd >> 1) & 1u, abort_flag, a.status, a.wait_limit))) break;
            tc_fence_after();
            const uint32_t tb = tmem + lane_off + (uint32_t)b * a.acc_off + (uint32_t)(hc * half);
            // two 16-column loads in flight per wait (compile-time register indices)
#pragma unroll
            for (int grp = 0; grp < MAXHALF / 32; ++grp) {
                uint32_t r[2][16];
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (grp * 2 + u < nch16) tmem_ld16(tb + (uint32_t)((grp * 2 + u) * 16), r[u]);
                tmem_wait_ld();
#pragma unroll
                for (int u = 0; u < 2; ++u)
                    if (grp * 2 + u < nch16) {
#pragma unroll
                        for (int i = 0; i < 16; ++i) part[(grp * 2 + u) * 16 + i] += __uint_as_float(r[u][i]);
                    }
            }
            if (tail8) {                    // the last 8 columns of a half that is not a multiple of 16
                uint32_t r8[8];
                tmem_ld8(tb + (uint32_t)(nch16 * 16), r8);
                tmem_wait_ld();
#pragma unroll
                for (int c = 0; c < MAXHALF; c += 8)
                    if (c == nch16 * 16) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) part[c + i] += __uint_as_float(r8[i]);
                    }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&drained[b]);
            if (((wd + 1) * PROMOTE) % FLUSH == 0 || wd + 1 == nwin) {
#pragma unroll
                for (int c = 0; c < MAXHALF; ++c) {
                    if (c < half) {
                        acc64[(size_t)c * 128] = (flushed ? acc64[(size_t)c * 128] : 0.0) + (double)part[c];
                        part[c] = 0.0f;
                    }
                }
                flushed = 1;
            }
        }
        // -------------------------------------------------------------- epilogue
        if (ok) {
            const int cpart = row >> 6, gro = row & 63;
            const int Gr = gb * GBLK + gro;
            if (Gr < a.ng) {
                const double vsp = a.vs[Gr];
                const size_t rowoff = ((size_t)iw * a.ng + Gr) * a.ng;
                double* plane = reinterpret_cast<double*>(a.eps) + cpart;
                for (int col = 0; col < half; ++col) {
                    const int G = n0 + hc * half + col;
                    if (G < a.ng) {
                        const double ch = a.pref * acc64[(size_t)col * 128];
                        plane[2 * (rowoff + G)] = (cpart == 0 && G == Gr ? 1.0 : 0.0) - vsp * a.vs[G] * ch;
                        if (a.chi) {
                            double* dst = reinterpret_cast<double*>(a.chi + ((size_t)iw * a.ng + G) * a.ng + Gr);
                            dst[cpart] = ch;
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// W[w][t] = 1/(w - dE + i eta) - 1/(w + dE + i eta), dE = E_c(k+q) - E_v(k), with dE and
// w -+ dE formed in FP64; zero for padded t.
__global__ void k_weights(int nw, long long ld, long long nt, int nv, int nc, const double* Ek, const double* Ekq,
                          const double* w, double eta, float2* W) {
    const long long n = (long long)nw * ld;
    const int nvc = nv * nc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int iw = (int)(i / ld);
        const long long t = i - (long long)iw * ld;
        float2 v = make_float2(0.f, 0.f);
        if (t < nt) {
            const long long k = t / nvc;
            const int rem = (int)(t - k * nvc);
            const int vv = rem / nc, c = rem - vv * nc;
            const double dE = Ekq[k * nc + c] - Ek[k * nv + vv];
            const double x1 = w[iw] - dE, x2 = w[iw] + dE;
            const double n1 = x1 * x1 + eta * eta, n2 = x2 * x2 + eta * eta;
            const double r = 1.0 / (n1 * n2);         // one FP64 division for both denominators
            const double d1 = n2 * r, d2 = n1 * r;
            v = make_float2((float)(x1 * d1 - x2 * d2), (float)(eta * (d2 - d1)));
        }
        W[i] = v;
    }
}

// The diagonal of the mixed chi0 again, without the cancellation of the tensor-core GEMM:
// there Im chi0_GG is formed from products of size |Re W| |rho|^2 that cancel to
// |Im W| |rho|^2, so the split's 2^-24 is amplified by |w - dE|/eta far from resonance.
// Here chi0_GG(w) = pref sum_t W_t(w) |rho_t(G)|^2 with |rho|^2 formed first (FP32 rho as
// the sum of its three BF16 terms), FP32 sums over 256 transitions added in FP64.  The
// transitions are split into gridDim.z ranges of tps (a multiple of 256) so that the
// launch fills the GPU; each CTA (32 w x 32 G, thread 2 x 2, transitions staged 32 at a
// time) writes its range's FP64 sums to part[z][w][G], and k_diag_finish adds the ranges
// in a fixed order.
__global__ void __launch_bounds__(256) k_diag_chi(int nw, int ng, long long nt, long long tps, const float2* W,
                                                  long long wld, const __nv_bfloat162* p0,
                                                  const __nv_bfloat162* p1, const __nv_bfloat162* p2,
                                                  long long kp2, double2* part) {
    __shared__ float2 Ws[32][33];            // [t][w]
    __shared__ float Rs[32][33];             // [t][G]
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int G0 = blockIdx.x * 32, w0 = blockIdx.y * 32;
    const long long tb = (long long)blockIdx.z * tps, te = min(nt, tb + tps);
    float2 acc[2][2];
    double2 acc64[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            acc[i][j] = make_float2(0.f, 0.f);
            acc64[i][j] = make_double2(0.0, 0.0);
        }
    int chunk = 0;
    for (long long t0 = tb; t0 < te; t0 += 32) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int i = threadIdx.x + 256 * r;
            const int tt = i & 31, row = i >> 5;
            const long long t = t0 + tt;
            float2 wv = make_float2(0.f, 0.f);
            float rv = 0.f;
            if (t < te) {
                if (w0 + row < nw) wv = W[(long long)(w0 + row) * wld + t];
                if (G0 + row < ng) {
                    const long long o = (long long)(G0 + row) * kp2 + t;
                    const float2 a0 = __bfloat1622float2(p0[o]), a1 = __bfloat1622float2(p1[o]),
                                 a2 = __bfloat1622float2(p2[o]);
                    const float re = (a0.x + a1.x) + a2.x, im = (a0.y + a1.y) + a2.y;
                    rv = re * re + im * im;
                }
            }
            Ws[tt][row] = wv;
            Rs[tt][row] = rv;
        }
        __syncthreads();
#pragma unroll 8
        for (int tt = 0; tt < 32; ++tt) {
            const float2 wa = Ws[tt][ty], wb = Ws[tt][ty + 16];
            const float ra = Rs[tt][tx], rb = Rs[tt][tx + 16];
            acc[0][0].x = fmaf(wa.x, ra, acc[0][0].x);
            acc[0][0].y = fmaf(wa.y, ra, acc[0][0].y);
            acc[0][1].x = fmaf(wa.x, rb, acc[0][1].x);
            acc[0][1].y = fmaf(wa.y, rb, acc[0][1].y);
            acc[1][0].x = fmaf(wb.x, ra, acc[1][0].x);
            acc[1][0].y = fmaf(wb.y, ra, acc[1][0].y);
            acc[1][1].x = fmaf(wb.x, rb, acc[1][1].x);
            acc[1][1].y = fmaf(wb.y, rb, acc[1][1].y);
        }
        __syncthreads();
        if (++chunk == 8 || t0 + 32 >= te) {
            chunk = 0;
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    acc64[i][j].x += (double)acc[i][j].x;
                    acc64[i][j].y += (double)acc[i][j].y;
                    acc[i][j] = make_float2(0.f, 0.f);
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int w = w0 + ty + 16 * i, G = G0 + tx + 16 * j;
            if (w < nw && G < ng) part[((size_t)blockIdx.z * nw + w) * ng + G] = acc64[i][j];
        }
}

// eps_GG = 1 - v(G) chi0_GG from the ranges' sums (added in range order), and the chi0
// diagonal if it is kept; one thread per (w, G).
__global__ void k_diag_finish(int nw, int ng, int nsplit, const double2* part, double pref, const double* vs,
                              double2* eps, double2* chi) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nw * ng) return;
    const int w = i / ng, G = i - w * ng;
    double2 sum = make_double2(0.0, 0.0);
    for (int z = 0; z < nsplit; ++z) {
        const double2 v = part[(size_t)z * nw * ng + i];
        sum.x += v.x;
        sum.y += v.y;
    }
    const double2 ch = make_double2(pref * sum.x, pref * sum.y);
    const double vv = vs[G] * vs[G];
    const size_t o = ((size_t)w * ng + G) * ng + G;
    eps[o] = make_double2(1.0 - vv * ch.x, -vv * ch.y);
    if (chi) chi[o] = ch;
}

}  // namespace

typedef CUresult (*PFN_encodeTiled_t)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                      const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                      CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static PFN_encodeTiled_t get_encode() {
    static PFN_encodeTiled_t fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_encodeTiled_t>(p);
    }
    return fn;
}

// 2-D tensor map over one BF16 plane [rows][kp] (row length kp), box {box_k, box_rows} with the
// swizzle matching the row bytes of the box (32 or 64)
bool qcx_make_bf16_map(CUtensorMap* m, void* base, long long kp, int rows, int box_rows, int box_k) {
    PFN_encodeTiled_t enc = get_encode();
    if (!enc || (box_k != 16 && box_k != 32)) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
    const cuuint32_t box[2] = {(cuuint32_t)box_k, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               box_k == 16 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

cudaError_t qcx_launch_chi0_mixed(qcx_ctx* ctx, QSlot& s, int iq, double2* chi, int* d_status) {
    const int ng = s.ng;
    const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    TcArgs a{};
    a.ng = ng;
    a.nw = s.nw;
    a.nv = ctx->nv;
    a.nc = ctx->nc;
    a.nt = nt;
    int n_chunks;
    if (s.ngp <= 2 * MAXHALF) {
        n_chunks = 1;
        a.n_tile = s.ngp;
        a.src_from_b = 1;
    } else {
        n_chunks = (s.ngp + 2 * MAXHALF - 1) / (2 * MAXHALF);
        a.n_tile = ((s.ngp + n_chunks - 1) / n_chunks + 15) / 16 * 16;
        a.src_from_b = 0;
    }
    a.n_gb = (ng + GBLK - 1) / GBLK;
    a.kstages = (int)(s.kp / KSTEP);
    a.acc_off = a.n_tile <= 128 ? 128u : 256u;
    a.tmem_cols = 2u * a.acc_off;
    a.wld = s.kp / 2;
    const double* L = ctx->lattice;
    const double vol = fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                            L[2] * (L[3] * L[7] - L[4] * L[6]));
    a.pref = 2.0 / (ctx->nk * vol);
    a.vs = s.vs.as<double>();
    a.eps = s.eps.as<double2>();
    a.chi = chi;
    a.status = d_status;
    a.wait_limit = ctx->wait_limit;
    a.withhold = ctx->withhold_copies;
    if (a.n_tile > 2 * MAXHALF || a.n_tile < 16) return cudaErrorNotSupported;

    const uint32_t bbytes = (uint32_t)a.n_tile * ROWB;
    const uint32_t sbytes = a.src_from_b ? 0u : NPB * GBLK * ROWB;
    const size_t stage_bytes = NPB * bbytes + sbytes + NPA * ATILE;
    const size_t smem = 1024 + NSTAGE * stage_bytes + NSTAGE * (KSTEP / 2) * sizeof(float2) +
                        (5 * NSTAGE + 5) * sizeof(uint64_t) + 16;
    if (smem > SMEM_LIMIT) return cudaErrorNotSupported;

    // W table for this q (FP64 dE and w -+ dE, stored FP32)
    cudaError_t e = s.wtab.ensure((size_t)s.nw * (s.kp / 2) * sizeof(float2));
    if (e != cudaSuccess) return e;
    {
        const long long n = (long long)s.nw * (s.kp / 2);
        k_weights<<<(int)std::min<long long>((n + 255) / 256, 8192), 256, 0, ctx->stream>>>(
            s.nw, s.kp / 2, nt, ctx->nv, ctx->nc, ctx->d_Ek.as<double>(),
            ctx->d_Ekq.as<double>() + (size_t)iq * ctx->nk * ctx->nc, s.w.as<double>(), s.eta, s.wtab.as<float2>());
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    a.wtab = s.wtab.as<float2>();
    dim3 grid(a.n_gb * s.nw, n_chunks);
    // split of the transitions for the diagonal pass: enough CTAs to fill the GPU, each range a
    // multiple of 256 transitions; its partial sums reuse acc64 once k_chi0_tc has finished
    const dim3 dgrid((ng + 31) / 32, (s.nw + 31) / 32);
    const long long want = std::max<long long>(1, (8LL * 152 + dgrid.x * dgrid.y - 1) / (dgrid.x * dgrid.y));
    const long long tps = std::max<long long>(256, ((nt + want - 1) / want + 255) / 256 * 256);
    const int nsplit = (int)((nt + tps - 1) / tps);
    const size_t acc_bytes = std::max((size_t)grid.x * grid.y * 128 * a.n_tile * sizeof(double),
                                      (size_t)nsplit * s.nw * ng * sizeof(double2));
    e = s.acc64.ensure(acc_bytes);
    if (e != cudaSuccess) return e;
    a.acc64 = s.acc64.as<double>();

    unsigned char* p0 = reinterpret_cast<unsigned char*>(s.rho.p);
    const size_t plane = (size_t)s.ngp * s.kp * 2;
    CUtensorMap mb[NPB], ms[NPB];
    for (int i = 0; i < NPB; ++i)
        if (!qcx_make_bf16_map(&mb[i], p0 + i * plane, s.kp, s.ngp, a.n_tile, KSTEP) ||
            !qcx_make_bf16_map(&ms[i], p0 + i * plane, s.kp, s.ngp, GBLK, KSTEP))
            return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute((const void*)k_chi0_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    {
        // the warpgroups' register budgets assume this launch allocation; another one could leave a
        // setmaxnreg.inc waiting for registers that no warpgroup gives back
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, (const void*)k_chi0_tc);
        if (e != cudaSuccess) return e;
        if (fa.numRegs != LAUNCH_REGS) return cudaErrorNotSupported;
    }
    k_chi0_tc<<<grid, NTHREADS, smem, ctx->stream>>>(mb[0], mb[1], ms[0], ms[1], a);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const __nv_bfloat162* q0 = reinterpret_cast<const __nv_bfloat162*>(s.rho.p);
    const long long plane2 = (long long)s.ngp * (s.kp / 2);
    double2* part = s.acc64.as<double2>();
    k_diag_chi<<<dim3(dgrid.x, dgrid.y, nsplit), 256, 0, ctx->stream>>>(
        s.nw, ng, nt, tps, s.wtab.as<float2>(), s.kp / 2, q0, q0 + plane2, q0 + 2 * plane2, s.kp / 2, part);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_diag_finish<<<(s.nw * ng + 255) / 256, 256, 0, ctx->stream>>>(s.nw, ng, nsplit, part, a.pref,
                                                                     s.vs.as<double>(), s.eps.as<double2>(), chi);
    return cudaGetLastError();
}
