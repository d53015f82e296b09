// Persistent tensor-core chi0 (Eq. (RPA)) with the fused Dyson step over a
// list of uneven (q, w) instances, each with its own G set
// {G : |q+G| < G_max} of N_G = 15..339 vectors.
//
// The arithmetic per tile is that of the per-q kernel: one 64-row G' block
// of one instance at its frequency (a 128 x N accumulator: 64 re rows and 64
// im rows of chi0_GG'), one N chunk of its G list, the contraction over
// k' = 2t + p with B = rho~ = b0 + b1 (the first two BF16 terms of the FP32 pair
// densities) and A = W rho~ in three BF16 terms, the five products
// a0 b0 + a0 b1 + a1 b0 + a1 b1 + a2 b0 (both sides carry the same rho~, so only
// A's split and the dropped a2 b1 are errors of the contraction),
// FP32 accumulation restarted after 20 MMAs (two K stages) and promoted
// through FP32 registers into an FP64 buffer, and eps = delta - v^1/2 chi0 v^1/2
// written in FP64 (row G', column G).
//
// What changes is the scheduling (and, as in the per-q kernel, two MMA issuer
// warps take alternate accumulation windows).  One CTA per SM runs for the whole batch
// and walks a host-ordered tile list (largest N first, tile i to CTA
// i mod grid), so hundreds of small instances cost one launch.  The shared
// memory ring and the two TMEM accumulators keep their phases across tile
// boundaries, so the TMA producer already streams the next tile while the
// epilogue warps finish the current one.  Every instance of one q reads the
// same BF16 planes (the pair densities of the union of that q's G sets,
// sorted by |q+G| so that each instance's set is a prefix); the planes are
// addressed through one tensor map per q and piece, all passed by value.  B
// tiles of N <= 192 rows arrive as 64-row boxes.  Every wait is bounded.
#include "qcx_internal.h"
#include "tc_ptx.cuh"

#include <cstring>

namespace {

constexpr int NTHREADS = 384;             // warps: 0 TMA, 1 and 10 MMA, 2-9 A/drain/epilogue, 11 idle
constexpr int MMA_WARP2 = 10;
constexpr int NSTAGE = 4;
constexpr int NPA = 3;                    // BF16 terms of the A operand (W rho~)
constexpr int NPB = 2;                    // BF16 terms of the B operand (rho~ = b0 + b1)
constexpr int ATILE = 128 * ROWB;         // one 128-row A piece
constexpr int GBLK = 64;                  // G' rows per tile, rows per TMA box
constexpr int MAXHALF = 96;
constexpr int NMAX = 2 * MAXHALF;         // largest N of a tile
constexpr int BREG = NMAX * ROWB;         // one B piece region
constexpr int SPIECE = GBLK * ROWB;       // one A-source piece
constexpr int STAGE_BYTES = NPB * BREG + NPB * SPIECE + NPA * ATILE;
constexpr int TPS = KSTEP / 2;            // transitions per stage
constexpr uint32_t ACC_OFF = 256;         // second TMEM buffer
constexpr uint32_t TMEM_COLS = 512;
constexpr int SMEM_LIMIT = 232448;
constexpr size_t SMEM_BYTES =
    1024 + NSTAGE * (size_t)STAGE_BYTES + NSTAGE * TPS * sizeof(float2) + (5 * NSTAGE + 5) * sizeof(uint64_t) + 16;
static_assert(SMEM_BYTES <= (size_t)SMEM_LIMIT, "stage ring does not fit in shared memory");

struct MapSet {
    CUtensorMap m[QCX_BATCH_MAXQ][NPB];
};

struct BArgs {
    int ntile, kstages;
    int slot0;                // first slot of this launch's group (map index = slot - slot0)
    const int4* tiles;        // {inst, gb, n0, N | src_from_b << 16}
    const BatchInst* inst;
    const float2* wtab;       // [inst][wld] W_t(w_inst)
    long long wld;
    double pref;
    double* acc64;            // [grid][NMAX][128] (column-major: a warp's 32 rows are contiguous)
    double2* eps;
    int* status;
    long long wait_limit;     // clock cycles before a pipeline wait gives up
    int promote;              // K stages per accumulation window (20 MMAs)
    int flush;                // K stages between FP64 flushes (64 windows)
};

__global__ void __launch_bounds__(NTHREADS, 1) k_chi0_tc_batch(const __grid_constant__ MapSet maps, BArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* tail = base + NSTAGE * STAGE_BYTES;
    float2* Wbuf = reinterpret_cast<float2*>(tail);
    uint64_t* bars = reinterpret_cast<uint64_t*>(tail + NSTAGE * TPS * sizeof(float2));
    // copy and A-tile barriers of running stage gs: number gs mod 2 NSTAGE (ring slot gs mod NSTAGE),
    // so an issuer's wait never meets the previous phase of its barrier unfinished
    uint64_t* full_b = bars;                   // [2 NSTAGE]
    uint64_t* full_a = bars + 2 * NSTAGE;      // [2 NSTAGE]
    uint64_t* empty = bars + 4 * NSTAGE;       // [NSTAGE]
    uint64_t* acc_full = bars + 5 * NSTAGE;
    uint64_t* drained = acc_full + 2;
    uint64_t* mma_done = drained + 2;
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
    if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int nwin = (a.kstages + a.promote - 1) / a.promote;

    if (warp == 0) {
        // ---------------------------------------------------------- TMA producer
        if (lane == 0) {
            int gs = 0;
            int last = -1;
            bool ok = true;
            for (int ti = blockIdx.x; ti < a.ntile && ok; ti += gridDim.x) {
                const int4 tl = a.tiles[ti];
                const int nN = tl.w & 0xFFFF, src_b = tl.w >> 16;
                const int slot = a.inst[tl.x].slot - a.slot0;
                const int nbox = (nN + GBLK - 1) / GBLK;
                const uint32_t bytes = (uint32_t)(NPB * nbox * GBLK * ROWB + (src_b ? 0 : NPB * SPIECE) +
                                                  TPS * (int)sizeof(float2));
                const float2* wrow = a.wtab + (size_t)tl.x * a.wld;
                for (int it = 0; it < a.kstages; ++it, ++gs) {
                    const int s = (int)(gs % NSTAGE);
                    const uint32_t ph = (uint32_t)(gs / NSTAGE) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag, a.status, a.wait_limit)) {
                        ok = false;
                        break;
                    }
                    unsigned char* st = base + s * STAGE_BYTES;
                    uint64_t* fb = &full_b[gs % (2 * NSTAGE)];
                    mbar_arrive_tx(fb, bytes);
                    bulk_load(Wbuf + s * TPS, wrow + (size_t)it * TPS, TPS * sizeof(float2), fb);
                    for (int p = 0; p < NPB; ++p)
                        for (int r = 0; r < nbox; ++r)
                            tma_load_2d(st + p * BREG + r * SPIECE, &maps.m[slot][p], fb, it * KSTEP,
                                        tl.z + r * GBLK);
                    if (!src_b) {
                        unsigned char* sp = st + NPB * BREG;
                        for (int p = 0; p < NPB; ++p)
                            tma_load_2d(sp + p * SPIECE, &maps.m[slot][p], fb, it * KSTEP, tl.y * GBLK);
                    }
                    last = gs;
                }
            }
            // let every copy still in flight (at most the last NSTAGE stages) land before the CTA can exit
            for (int gs2 = max(0, last - NSTAGE + 1); gs2 <= last; ++gs2)
                mbar_wait(&full_b[gs2 % (2 * NSTAGE)], (uint32_t)(gs2 / (2 * NSTAGE)) & 1u, abort_flag, a.status,
                          CLEANUP_WAIT_LIMIT, false);
        }
    } else if (warp == 1 || warp == MMA_WARP2) {
        // ---------------------------------------------------------- MMA issuers
        // Two issuers take alternate accumulation windows (counted over the CTA's whole
        // tile sequence), so one waits while the other's MMAs run.
        if (lane == 0) {
            const int par = warp == 1 ? 0 : 1;
            bool ok = true;
            for (int lt = 0; blockIdx.x + lt * gridDim.x < a.ntile && ok; ++lt) {
                const int4 tl = a.tiles[blockIdx.x + lt * gridDim.x];
                const uint32_t idesc = make_idesc(128, tl.w & 0xFFFF);
                for (int wd = 0; wd < nwin && ok; ++wd) {
                    const int gw = lt * nwin + wd;
                    if ((gw & 1) != par) continue;
                    const int b = gw & 1;
                    if (gw >= 2 && !mbar_wait(&drained[b], (uint32_t)((gw - 2) >> 1) & 1u, abort_flag, a.status, a.wait_limit)) {
                        ok = false;
                        break;
                    }
                    const int it1 = min((wd + 1) * a.promote, a.kstages);
                    for (int it = wd * a.promote; it < it1; ++it) {
                        const int gs = lt * a.kstages + it;
                        const int s = gs % NSTAGE;
                        const bool first = it == wd * a.promote;
                        // the A warps arrive only after they saw this stage's copies land
                        if (!mbar_wait(&full_a[gs % (2 * NSTAGE)], (uint32_t)(gs / (2 * NSTAGE)) & 1u, abort_flag,
                                       a.status, a.wait_limit)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        unsigned char* st = base + s * STAGE_BYTES;
                        const uint32_t b0 = smem_u32(st), b1 = b0 + BREG;
                        const uint32_t d = tmem + (uint32_t)b * ACC_OFF;
                        const uint32_t a0 = smem_u32(st + NPB * BREG + NPB * SPIECE), a1 = a0 + ATILE,
                                       a2 = a1 + ATILE;
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
            }
            // no MMA of either issuer may still be running when TMEM is freed
            umma_commit(mma_done);
            mbar_wait(mma_done, 0, abort_flag, a.status, CLEANUP_WAIT_LIMIT, false);
        }
    } else if (warp < MMA_WARP2) {
        // ------------------------- A generation, accumulator drain, epilogue
        const int wi = warp - 2;
        const int g = threadIdx.x - 64;
        const int j = g & 3;
        const int go = g >> 2;
        const int q = warp & 3, hc = wi >> 2;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const int row = q * 32 + lane;
        float part[MAXHALF];
        bool ok = true;
        // all tiles have kstages stages and nwin windows, so the running stage and
        // window counters of this CTA follow from its local tile number lt
        for (int lt = 0; blockIdx.x + lt * gridDim.x < a.ntile && ok; ++lt) {
            int nch8, row0, lim;
            bool src_b;
            {
                const int4 tl = a.tiles[blockIdx.x + lt * gridDim.x];
                src_b = (tl.w >> 16) != 0;
                nch8 = (tl.w & 0xFFFF) >> 4;
                lim = a.inst[tl.x].ng - tl.y * GBLK;    // G' rows of this block inside the instance
                row0 = src_b ? tl.y * GBLK : 0;          // first source row in the staged tile
            }
            // register partials restart with every tile (dead across the epilogue)
#pragma unroll
            for (int i = 0; i < MAXHALF; ++i) part[i] = 0.0f;

            auto drain = [&](int wd) -> bool {
                const int gw = lt * nwin + wd;
                const int b = gw & 1;
                if (!warp_wait(&acc_full[b], (uint32_t)(gw >> 1) & 1u, abort_flag, a.status, a.wait_limit)) return false;
                tc_fence_after();
                const uint32_t tb = tmem + lane_off + (uint32_t)b * ACC_OFF + (uint32_t)(hc * nch8 * 8);
#pragma unroll
                for (int grp = 0; grp < MAXHALF / 16; ++grp) {
                    uint32_t r[2][8];
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if (grp * 2 + u < nch8) tmem_ld8(tb + (uint32_t)((grp * 2 + u) * 8), r[u]);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < 2; ++u)
                        if (grp * 2 + u < nch8) {
#pragma unroll
                            for (int i = 0; i < 8; ++i) part[(grp * 2 + u) * 8 + i] += __uint_as_float(r[u][i]);
                        }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&drained[b]);
                if (((wd + 1) * a.promote) % a.flush == 0 || wd + 1 == nwin) {
                    // the first flush of a tile starts the FP64 sums
                    const bool flushed = wd >= a.flush / a.promote;
                    double* acc64 = a.acc64 + (size_t)blockIdx.x * 128 * NMAX + (size_t)(hc * nch8 * 8) * 128 + row;
#pragma unroll
                    for (int c = 0; c < MAXHALF; ++c) {
                        if (c < nch8 * 8) {
                            acc64[(size_t)c * 128] = (flushed ? acc64[(size_t)c * 128] : 0.0) + (double)part[c];
                            part[c] = 0.0f;
                        }
                    }
                }
                return true;
            };

            for (int it = 0; it < a.kstages; ++it) {
                const int gs = lt * a.kstages + it;
                const int s = gs % NSTAGE;
                const int s2 = gs % (2 * NSTAGE);
                // the producer issued this stage's copies only after the MMAs of its previous
                // use finished, so a landed stage is also free to overwrite
                if (!(ok = warp_wait(&full_b[s2], (uint32_t)(gs / (2 * NSTAGE)) & 1u, abort_flag, a.status,
                                     a.wait_limit)))
                    break;
                unsigned char* st = base + s * STAGE_BYTES;
                const unsigned char* srcb = st + (src_b ? 0 : NPB * BREG);
                const uint32_t src_piece = src_b ? (uint32_t)BREG : (uint32_t)SPIECE;
                uint32_t re0[4] = {0, 0, 0, 0}, re1[4] = {0, 0, 0, 0}, re2[4] = {0, 0, 0, 0};
                uint32_t im0[4] = {0, 0, 0, 0}, im1[4] = {0, 0, 0, 0}, im2[4] = {0, 0, 0, 0};
                if (go < lim) {
                    const uint32_t coff = sw64_off(row0 + go, j);
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
                        split3(wq.x * rr - wq.y * ri, wq.x * ri + wq.y * rr, re0[qq], re1[qq], re2[qq]);
                        // (xi, -xr) splits into the terms of (xr, xi), swapped, the second negated
                        im0[qq] = perm_im(re0[qq]);
                        im1[qq] = perm_im(re1[qq]);
                        im2[qq] = perm_im(re2[qq]);
                    }
                }
                unsigned char* ap = st + NPB * BREG + NPB * SPIECE;
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
                // drain the previous window once this window's A tiles are queued; after the
                // last stage drain whatever is left (one call site keeps the code compact)
                int wd0 = nwin, wd1 = -1;
                if (it % a.promote == a.promote - 1 && it >= a.promote) wd0 = wd1 = it / a.promote - 1;
                if (it + 1 == a.kstages) {
                    wd0 = min(wd0, (it % a.promote == a.promote - 1 && it >= a.promote) ? it / a.promote - 1
                                                                                        : max(nwin - 2, 0));
                    wd1 = nwin - 1;
                }
                for (int wd = wd0; wd <= wd1 && ok; ++wd) ok = drain(wd);
                if (!ok) break;
            }
            if (!ok) break;
            // ------------------------------------------------------------ epilogue
            const int4 tl = a.tiles[blockIdx.x + lt * gridDim.x];
            const int gb = tl.y, n0 = tl.z, half = (tl.w & 0xFFFF) >> 1, ng = a.inst[tl.x].ng;
            const int cpart = row >> 6, gro = row & 63;
            const int Gr = gb * GBLK + gro;
            const double* acc64 = a.acc64 + (size_t)blockIdx.x * 128 * NMAX + (size_t)(hc * half) * 128 + row;
            if (Gr < ng) {
                const double* vs = a.inst[tl.x].vs;
                const double vsp = vs[Gr];
                double* plane = reinterpret_cast<double*>(a.eps + a.inst[tl.x].eps_off + (size_t)Gr * ng) + cpart;
                for (int col = 0; col < half; ++col) {
                    const int G = n0 + hc * half + col;
                    if (G < ng) {
                        const double ch = a.pref * acc64[(size_t)col * 128];
                        plane[2 * G] = (cpart == 0 && G == Gr ? 1.0 : 0.0) - vsp * vs[G] * ch;
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
}

}  // namespace

size_t qcx_chi0_tc_batch_acc_bytes(int grid) { return (size_t)grid * 128 * NMAX * sizeof(double); }

cudaError_t qcx_launch_chi0_tc_batch(cudaStream_t st, const CUtensorMap* maps, int slot0, int nslot, int ntile,
                                     const int4* d_tiles, int grid, const BatchInst* d_inst, const float2* wtab,
                                     long long wld, int kstages, double pref, double* acc64, double2* eps,
                                     int* status, long long wait_limit) {
    if (nslot < 1 || nslot > QCX_BATCH_MAXQ || ntile < 1 || grid < 1 || kstages < 1) return cudaErrorInvalidValue;
    MapSet ms;
    memset(&ms, 0, sizeof(ms));
    for (int s = 0; s < nslot; ++s)
        for (int p = 0; p < NPB; ++p) ms.m[s][p] = maps[3 * s + p];   // the first two of each slot's three planes
    BArgs a;
    a.ntile = ntile;
    a.kstages = kstages;
    a.slot0 = slot0;
    a.tiles = d_tiles;
    a.inst = d_inst;
    a.wtab = wtab;
    a.wld = wld;
    a.pref = pref;
    a.acc64 = acc64;
    a.eps = eps;
    a.status = status;
    a.wait_limit = wait_limit;
    a.promote = 2;                            // 20 MMAs per window: two K stages of ten
    a.flush = 64 * a.promote;
    cudaError_t e =
        cudaFuncSetAttribute((const void*)k_chi0_tc_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_BYTES);
    if (e != cudaSuccess) return e;
    k_chi0_tc_batch<<<grid, NTHREADS, SMEM_BYTES, st>>>(ms, a);
    return cudaGetLastError();
}
