// Batched solve of uneven (q, w) instances: each instance is one frequency
// of one q with the G set {G : |q+G| < G_max} (N_G = 15..339 in the uneven
// workload), and returns the heads L_LFE = -Im [eps^-1]_{00} and
// L_noLFE = -Im (1/eps_00) (Eqs. (RPA), (eps_LFE), (eps_noLFE)).
//
// Plan (host, once per distinct instance list):
//  * per distinct q, the union of its instances' G sets sorted by |q+G|
//    (ties by |G|^2 and the integer triple), so every instance's set is a
//    prefix of its q's list; pair densities are formed once per q on the
//    union list (the per-q pair-density kernel, unchanged);
//  * the mixed path cuts every instance into (64-row G' block, G chunk)
//    tiles for the persistent tensor-core kernel, largest first; the FP64
//    path into 32 x 32 tiles for a plain FP64 kernel;
//  * instance lists per CTA for the LU kernels by greedy longest-processing-
//    time over the cost N_G^3;
//  * the whole sequence (G set-up, pair densities, W table, chi0 + Dyson,
//    LU, FP64 residual and correction) is captured once in a CUDA graph and
//    replayed per call; only the frequencies are uploaded per call.
//  * Autotuner: the tile width (columns of G per tensor-core tile) has its own
//    cap per N_G class (65-128, 129-192, more than 192); on a new plan the
//    mixed path starts from caps of 192, then tries the narrower caps of one
//    class at a time (widest class first, the others at their best so far),
//    capturing a graph for each set and timing two replays with CUDA events,
//    and keeps the fastest.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <new>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

namespace {

constexpr int NREF = 2;            // FP64 refinement steps of the mixed solve
constexpr int MAX_NG = 512;        // largest instance the solve kernels take
constexpr int FT = 32, FK = 16;    // FP64 chi0 tile: 32 x 32 (G, G'), 16 transitions per stage
constexpr int TC_KSTEP = 32;       // BF16 K elements per tensor-core pipeline stage

// W[inst][t] = 1/(w - dE + i eta) - 1/(w + dE + i eta), dE = E_c(k+q) - E_v(k) in FP64; zero for padded t
__global__ void k_weights_batch(int ninst, long long ld, long long nt, int nv, int nc, int nk, const double* Ek,
                                const double* Ekq_all, const BatchInst* inst, double eta, float2* W) {
    const long long n = (long long)ninst * ld;
    const int nvc = nv * nc;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ii = (int)(i / ld);
        const long long t = i - (long long)ii * ld;
        float2 v = make_float2(0.f, 0.f);
        if (t < nt) {
            const long long k = t / nvc;
            const int rem = (int)(t - k * nvc);
            const int vv = rem / nc, c = rem - vv * nc;
            const double* Ekq = Ekq_all + (size_t)inst[ii].iq * nk * nc;
            const double dE = Ekq[k * nc + c] - Ek[k * nv + vv];
            const double w = inst[ii].w;
            const double x1 = w - dE, x2 = w + dE;
            const double d1 = 1.0 / (x1 * x1 + eta * eta), d2 = 1.0 / (x2 * x2 + eta * eta);
            v = make_float2((float)(x1 * d1 - x2 * d2), (float)(eta * (d2 - d1)));
        }
        W[i] = v;
    }
}

// Plain FP64 chi0 + Dyson step for one 32 x 32 (G, G') tile of one instance;
// eps row G, column G'.
__global__ void __launch_bounds__(256)
    k_chi0_fp64_batch(const int4* tiles, const BatchInst* inst, long long nt, int nv, int nc, int nk,
                      const double* Ek, const double* Ekq_all, double eta, double pref, double2* eps) {
    __shared__ double2 As[FK][FT + 1];
    __shared__ double2 Bs[FK][FT + 1];
    __shared__ double2 Ws[FK];
    const int4 tl = tiles[blockIdx.x];
    const BatchInst in = inst[tl.x];
    const int ng = in.ng, G0 = tl.y, H0 = tl.z;
    const double* Ekq = Ekq_all + (size_t)in.iq * nk * nc;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int nvc = nv * nc;
    double2 acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) acc[i][j] = make_double2(0.0, 0.0);
    for (long long t0 = 0; t0 < nt; t0 += FK) {
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            const int i = threadIdx.x + 256 * r;
            const int tt = i & (FK - 1), gg = i >> 4;
            const long long t = t0 + tt;
            double2 va = make_double2(0.0, 0.0), vb = make_double2(0.0, 0.0);
            if (t < nt) {
                if (G0 + gg < ng) va = in.rho64[(long long)(G0 + gg) * nt + t];
                if (H0 + gg < ng) vb = in.rho64[(long long)(H0 + gg) * nt + t];
            }
            As[tt][gg] = make_double2(va.x, -va.y);
            Bs[tt][gg] = vb;
        }
        if (threadIdx.x < FK) {
            const long long t = t0 + threadIdx.x;
            double2 wt = make_double2(0.0, 0.0);
            if (t < nt) {
                const long long k = t / nvc;
                const int rem = (int)(t - k * nvc);
                const int v = rem / nc, c = rem - v * nc;
                const double dE = Ekq[k * nc + c] - Ek[k * nv + v];
                const double x1 = in.w - dE, x2 = in.w + dE;
                const double d1 = 1.0 / (x1 * x1 + eta * eta), d2 = 1.0 / (x2 * x2 + eta * eta);
                wt = make_double2(x1 * d1 - x2 * d2, eta * (d2 - d1));
            }
            Ws[threadIdx.x] = wt;
        }
        __syncthreads();
#pragma unroll 4
        for (int tt = 0; tt < FK; ++tt) {
            const double2 w = Ws[tt];
            const double2 a0 = cmul(w, As[tt][ty]), a1 = cmul(w, As[tt][ty + 16]);
            const double2 b0 = Bs[tt][tx], b1 = Bs[tt][tx + 16];
            cfma(acc[0][0], a0, b0);
            cfma(acc[0][1], a0, b1);
            cfma(acc[1][0], a1, b0);
            cfma(acc[1][1], a1, b1);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const int G = G0 + ty + 16 * i;
        if (G >= ng) continue;
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int H = H0 + tx + 16 * j;
            if (H >= ng) continue;
            const double vv = in.vs[G] * in.vs[H] * pref;
            eps[in.eps_off + (long long)G * ng + H] =
                make_double2((G == H ? 1.0 : 0.0) - vv * acc[i][j].x, -vv * acc[i][j].y);
        }
    }
}

int sm_count(int device) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
        cudaGetLastError();
        n = 0;
    }
    return n > 0 ? n : 1;
}

}  // namespace

struct BatchPlan {
    unsigned long long gen = 0;
    int prec = 0;
    double eta = 0.0;
    std::vector<int> key_q;
    std::vector<double> key_gmax;

    int ninst = 0, nslot = 0, nmax = 0;
    long long nt = 0, kp = 0;
    double pref = 0.0;
    std::vector<int> slot_iq, slot_u, slot_gofs;
    std::vector<QSlot*> qs;
    std::vector<BatchInst> hinst;
    std::vector<int> h_ng;

    DevBuf d_G, d_inst, d_wtab, d_eps, d_work, d_rowmap, d_x, d_r, d_out, d_flags, d_status, d_acc;
    DevBuf d_tiles, d_cta, d_rtask;
    std::vector<CUtensorMap> maps;              // [nslot][3]: the three BF16 planes of each slot
    std::vector<int> grp_tile0, grp_ntile;      // tensor-core tiles per group of <= QCX_BATCH_MAXQ slots
    int tc_grid = 0, tile_cap = 0, ntile = 0;
    int caps[3] = {192, 192, 192};              // tile width cap per N_G class: (64, 128], (128, 192], > 192
    int lu_grid = 0, n_rtask = 0;
    int tuned = 0;
    double tune_ms = 0.0;
    int launches = 0;
    long long wait_limit = 0;                   // pipeline wait limit captured into the graph
    cudaGraphExec_t exec = nullptr;

    ~BatchPlan() {
        if (exec) cudaGraphExecDestroy(exec);
        for (auto* s : qs) delete s;
    }
};

void qcx_batch_destroy(BatchPlan* p) { delete p; }

namespace {

// reciprocal basis b_i (rows) = 2 pi inv(A)^T
void recip_basis(const double* A, double b[9]) {
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
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) b[3 * i + j] = 2.0 * M_PI * inv[3 * j + i];
}

struct GEntry {
    double k2, g2;
    int n[3];
};

// {G : |q+G| < gmax} sorted by |q+G|^2, then |G|^2, then the integer triple
std::vector<GEntry> g_union(const double* A, const double* q, double gmax) {
    double b[9];
    recip_basis(A, b);
    const double reach = gmax + std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    int m[3];
    for (int i = 0; i < 3; ++i) {
        const double al = std::sqrt(A[3 * i] * A[3 * i] + A[3 * i + 1] * A[3 * i + 1] + A[3 * i + 2] * A[3 * i + 2]);
        m[i] = (int)std::ceil(al * reach / (2.0 * M_PI)) + 1;
    }
    std::vector<GEntry> out;
    for (int n1 = -m[0]; n1 <= m[0]; ++n1)
        for (int n2 = -m[1]; n2 <= m[1]; ++n2)
            for (int n3 = -m[2]; n3 <= m[2]; ++n3) {
                double g[3], k[3];
                for (int c = 0; c < 3; ++c) {
                    g[c] = n1 * b[c] + n2 * b[3 + c] + n3 * b[6 + c];
                    k[c] = q[c] + g[c];
                }
                const double k2 = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
                if (k2 < gmax * gmax) out.push_back({k2, g[0] * g[0] + g[1] * g[1] + g[2] * g[2], {n1, n2, n3}});
            }
    std::sort(out.begin(), out.end(), [](const GEntry& x, const GEntry& y) {
        if (x.k2 != y.k2) return x.k2 < y.k2;
        if (x.g2 != y.g2) return x.g2 < y.g2;
        return std::lexicographical_compare(x.n, x.n + 3, y.n, y.n + 3);
    });
    return out;
}

// N_G class of an instance for the tile-width caps: -1 (at most 64, one tile whatever the cap),
// 0 (65-128), 1 (129-192), 2 (more than 192)
int ng_class(int ng) { return ng <= 64 ? -1 : (ng <= 128 ? 0 : (ng <= 192 ? 1 : 2)); }

// tensor-core tiles for the tile-width caps of the N_G classes, grouped by slot group, largest N
// first and, within one width, by q (slot), so the tiles that stream the same pair-density planes
// run side by side and find them in L2
void make_tc_tiles(const BatchPlan& p, const int (&caps)[3], std::vector<int4>& tiles, std::vector<int>& g0,
                   std::vector<int>& gn) {
    const int ngrp = (p.nslot + QCX_BATCH_MAXQ - 1) / QCX_BATCH_MAXQ;
    std::vector<std::vector<int4>> grp(ngrp);
    for (int i = 0; i < p.ninst; ++i) {
        const int ng = p.hinst[i].ng;
        const int cls = ng_class(ng);
        const int cap = cls < 0 ? 192 : caps[cls];
        const int chunks = ng <= cap ? 1 : (ng + cap - 1) / cap;
        const int nc = ((ng + chunks - 1) / chunks + 15) / 16 * 16;
        const int ngb = (ng + 63) / 64;
        for (int gb = 0; gb < ngb; ++gb)
            for (int c = 0; c < chunks; ++c) {
                const int n0 = c * nc;
                if (n0 >= ng) continue;
                const int N = (std::min(nc, ng - n0) + 15) / 16 * 16;
                grp[p.hinst[i].slot / QCX_BATCH_MAXQ].push_back(make_int4(i, gb, n0, N | ((chunks == 1) << 16)));
            }
    }
    tiles.clear();
    g0.clear();
    gn.clear();
    for (auto& v : grp) {
        std::stable_sort(v.begin(), v.end(), [&](const int4& x, const int4& y) {
            const int nx = x.w & 0xFFFF, ny = y.w & 0xFFFF;
            if (nx != ny) return nx > ny;
            return p.hinst[x.x].slot < p.hinst[y.x].slot;
        });
        g0.push_back((int)tiles.size());
        gn.push_back((int)v.size());
        tiles.insert(tiles.end(), v.begin(), v.end());
    }
}

// record the whole batch on the context stream (inside a capture)
cudaError_t record(qcx_ctx* ctx, BatchPlan& p) {
    cudaStream_t st = ctx->stream;
    const bool mixed = p.prec == QCX_MIXED;
    cudaError_t e;
    p.launches = 0;
    if ((e = cudaMemsetAsync(p.d_status.p, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.d_flags.p, 0, sizeof(int) * p.ninst, st)) != cudaSuccess) return e;
    for (int s = 0; s < p.nslot; ++s) {
        QSlot& q = *p.qs[s];
        const int iq = p.slot_iq[s];
        if ((e = qcx_launch_qsetup(ctx, q, p.d_G.as<int>() + 3 * p.slot_gofs[s], p.slot_u[s], &ctx->qpts[3 * iq])) !=
            cudaSuccess)
            return e;
        if ((e = qcx_launch_pair_density(ctx, q, iq, (qcx_precision)p.prec)) != cudaSuccess) return e;
        p.launches += 2;
    }
    const BatchInst* dinst = p.d_inst.as<BatchInst>();
    if (mixed) {
        const long long n = (long long)p.ninst * (p.kp / 2);
        k_weights_batch<<<(int)std::min<long long>((n + 255) / 256, 8192), 256, 0, st>>>(
            p.ninst, p.kp / 2, p.nt, ctx->nv, ctx->nc, ctx->nk, ctx->d_Ek.as<double>(), ctx->d_Ekq.as<double>(), dinst,
            p.eta, p.d_wtab.as<float2>());
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++p.launches;
        for (size_t g = 0; g < p.grp_tile0.size(); ++g) {
            if (!p.grp_ntile[g]) continue;
            const int s0 = (int)g * QCX_BATCH_MAXQ;
            const int ns = std::min(QCX_BATCH_MAXQ, p.nslot - s0);
            // slot indices inside a group are relative to its first slot
            e = qcx_launch_chi0_tc_batch(st, p.maps.data() + 3 * s0, s0, ns, p.grp_ntile[g],
                                         p.d_tiles.as<int4>() + p.grp_tile0[g], std::min(p.tc_grid, p.grp_ntile[g]),
                                         dinst, p.d_wtab.as<float2>(), p.kp / 2, (int)(p.kp / TC_KSTEP), p.pref,
                                         p.d_acc.as<double>(), p.d_eps.as<double2>(), p.d_status.as<int>(),
                                         p.wait_limit);
            if (e != cudaSuccess) return e;
            ++p.launches;
        }
    } else {
        k_chi0_fp64_batch<<<p.ntile, 256, 0, st>>>(p.d_tiles.as<int4>(), dinst, p.nt, ctx->nv, ctx->nc, ctx->nk,
                                                    ctx->d_Ek.as<double>(), ctx->d_Ekq.as<double>(), p.eta, p.pref,
                                                    p.d_eps.as<double2>());
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        ++p.launches;
    }
    BatchSolveArgs a;
    a.inst = dinst;
    a.cta_off = p.d_cta.as<int>();
    a.cta_ids = p.d_cta.as<int>() + p.lu_grid + 1;
    a.eps = p.d_eps.as<double2>();
    a.work = p.d_work.p;
    a.rowmap = p.d_rowmap.as<int>();
    a.x = p.d_x.as<double2>();
    a.r = p.d_r.as<double2>();
    a.out = p.d_out.as<double>();
    a.flags = p.d_flags.as<int>();
    a.ninst = p.ninst;
    if ((e = qcx_launch_lu_head(st, a, p.lu_grid, p.nmax, !mixed, mixed)) != cudaSuccess) return e;
    ++p.launches;
    if (mixed) {
        for (int it = 0; it < NREF; ++it) {
            if ((e = qcx_launch_resid(st, a, p.d_rtask.as<int2>(), p.n_rtask)) != cudaSuccess) return e;
            if ((e = qcx_launch_lu_correct(st, a, p.lu_grid, p.nmax, it == NREF - 1 ? 1 : 0)) != cudaSuccess)
                return e;
            p.launches += 2;
        }
    }
    return cudaSuccess;
}

cudaError_t capture(qcx_ctx* ctx, BatchPlan& p, cudaGraphExec_t* out) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return e;
    cudaError_t er = record(ctx, p);
    e = cudaStreamEndCapture(ctx->stream, &g);
    if (er != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return er;
    }
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(out, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace

namespace {

qcx_status build_plan(qcx_ctx* ctx, BatchPlan& p) {
    const bool mixed = p.prec == QCX_MIXED;
    const int ninst = p.ninst;
    p.nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    p.kp = (2 * p.nt + 63) / 64 * 64;
    const double* L = ctx->lattice;
    const double vol = std::fabs(L[0] * (L[4] * L[8] - L[5] * L[7]) - L[1] * (L[3] * L[8] - L[5] * L[6]) +
                                 L[2] * (L[3] * L[7] - L[4] * L[6]));
    p.pref = 2.0 / (ctx->nk * vol);

    // distinct q (in order of first appearance) and their union G lists
    std::vector<int> slot_of_q(ctx->nq, -1);
    for (int i = 0; i < ninst; ++i)
        if (slot_of_q[p.key_q[i]] < 0) {
            slot_of_q[p.key_q[i]] = (int)p.slot_iq.size();
            p.slot_iq.push_back(p.key_q[i]);
        }
    p.nslot = (int)p.slot_iq.size();
    std::vector<double> smax(p.nslot, 0.0);
    for (int i = 0; i < ninst; ++i) smax[slot_of_q[p.key_q[i]]] = std::max(smax[slot_of_q[p.key_q[i]]], p.key_gmax[i]);
    std::vector<std::vector<GEntry>> lists(p.nslot);
    std::vector<int> Gflat;
    for (int s = 0; s < p.nslot; ++s) {
        lists[s] = g_union(ctx->lattice, &ctx->qpts[3 * p.slot_iq[s]], smax[s]);
        p.slot_gofs.push_back((int)(Gflat.size() / 3));
        p.slot_u.push_back((int)lists[s].size());
        for (auto& ge : lists[s]) Gflat.insert(Gflat.end(), ge.n, ge.n + 3);
    }
    // instances
    p.hinst.resize(ninst);
    p.h_ng.resize(ninst);
    long long eps_off = 0, work_off = 0, vec_off = 0;
    p.nmax = 0;
    for (int i = 0; i < ninst; ++i) {
        const int s = slot_of_q[p.key_q[i]];
        const double g2 = p.key_gmax[i] * p.key_gmax[i];
        const auto& lst = lists[s];
        int ng = 0, head = -1;
        while (ng < (int)lst.size() && lst[ng].k2 < g2) {
            if (!lst[ng].n[0] && !lst[ng].n[1] && !lst[ng].n[2]) head = ng;
            ++ng;
        }
        if (head < 0) return ctx->fail(QCX_ERR_ARG, "solve_batch: instance " + std::to_string(i) +
                                                        " has G = 0 outside its cutoff (|q| >= G_max)");
        if (ng > MAX_NG)
            return ctx->fail(QCX_ERR_UNSUPPORTED, "solve_batch: instance " + std::to_string(i) + " has N_G = " +
                                                      std::to_string(ng) + " > " + std::to_string(MAX_NG));
        BatchInst& b = p.hinst[i];
        b.slot = s;
        b.ng = ng;
        b.head = head;
        b.iq = p.key_q[i];
        b.eps_off = eps_off;
        b.work_off = work_off;
        b.vs = nullptr;
        b.rho64 = nullptr;
        b.w = 0.0;
        b.vec_off = vec_off;
        eps_off += (long long)ng * ng;
        work_off += (long long)ng * (ng + 1);
        vec_off += ng;
        p.h_ng[i] = ng;
        p.nmax = std::max(p.nmax, ng);
    }
    // per-slot pair-density state
    for (int s = 0; s < p.nslot; ++s) {
        QSlot* q = new (std::nothrow) QSlot();
        if (!q) return ctx->fail(QCX_ERR_ALLOC, "solve_batch: slot");
        p.qs.push_back(q);
        const int U = p.slot_u[s];
        q->iq = p.slot_iq[s];
        q->ng = U;
        q->ngp = std::max(64, (U + 15) / 16 * 16);
        q->kp = p.kp;
        CUDA_OR_FAIL(q->kappa.ensure(3 * sizeof(double) * U), "alloc");
        CUDA_OR_FAIL(q->kappa32.ensure(3 * sizeof(float) * U), "alloc");
        CUDA_OR_FAIL(q->vs.ensure(sizeof(double) * U), "alloc");
        CUDA_OR_FAIL(q->vs32.ensure(sizeof(float) * U), "alloc");
        if (mixed) {
            const size_t bytes = 3 * (size_t)q->ngp * q->kp * sizeof(__nv_bfloat16);
            CUDA_OR_FAIL(q->rho.ensure(bytes), "alloc rho");
            CUDA_OR_FAIL(cudaMemsetAsync(q->rho.p, 0, bytes, ctx->stream), "clear rho");
        } else {
            CUDA_OR_FAIL(q->rho.ensure((size_t)U * p.nt * sizeof(double2)), "alloc rho");
        }
    }
    for (int i = 0; i < ninst; ++i) {
        QSlot& q = *p.qs[p.hinst[i].slot];
        p.hinst[i].vs = q.vs.as<double>();
        p.hinst[i].rho64 = mixed ? nullptr : q.rho.as<double2>();
    }
    // device buffers
    CUDA_OR_FAIL(p.d_G.ensure(sizeof(int) * Gflat.size()), "alloc");
    CUDA_OR_FAIL(cudaMemcpyAsync(p.d_G.p, Gflat.data(), sizeof(int) * Gflat.size(), cudaMemcpyHostToDevice,
                                 ctx->stream),
                 "copy G");
    if (mixed)   // tables of the FP32 pair densities per slot, planned before the graph is captured
        for (int s = 0; s < p.nslot; ++s)
            CUDA_OR_FAIL(qcx_pd_tab_prepare(ctx, *p.qs[s], Gflat.data() + 3 * p.slot_gofs[s], p.slot_u[s],
                                            p.slot_iq[s]),
                         "pair-density tables");
    CUDA_OR_FAIL(p.d_inst.ensure(sizeof(BatchInst) * ninst), "alloc");
    CUDA_OR_FAIL(p.d_eps.ensure(sizeof(double2) * eps_off), "alloc eps");
    CUDA_OR_FAIL(p.d_work.ensure((mixed ? sizeof(float2) : sizeof(double2)) * work_off), "alloc work");
    CUDA_OR_FAIL(p.d_rowmap.ensure(sizeof(int) * vec_off), "alloc");
    CUDA_OR_FAIL(p.d_x.ensure(sizeof(double2) * vec_off), "alloc");
    CUDA_OR_FAIL(p.d_r.ensure(sizeof(double2) * vec_off), "alloc");
    CUDA_OR_FAIL(p.d_out.ensure(sizeof(double) * 3 * ninst), "alloc");
    CUDA_OR_FAIL(p.d_flags.ensure(sizeof(int) * ninst), "alloc");
    CUDA_OR_FAIL(p.d_status.ensure(sizeof(int)), "alloc");
    const int nsm = sm_count(ctx->device);
    // LU instance lists: greedy LPT over cost n^3 + 64 n^2
    p.lu_grid = std::min(ninst, nsm);
    {
        std::vector<int> order(ninst);
        std::iota(order.begin(), order.end(), 0);
        auto cost = [&](int i) { const double n = p.h_ng[i]; return n * n * n + 64.0 * n * n; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
        typedef std::pair<double, int> LoadCta;
        std::priority_queue<LoadCta, std::vector<LoadCta>, std::greater<LoadCta>> pq;
        for (int c = 0; c < p.lu_grid; ++c) pq.push({0.0, c});
        std::vector<std::vector<int>> lists_c(p.lu_grid);
        for (int i : order) {
            LoadCta top = pq.top();
            pq.pop();
            lists_c[top.second].push_back(i);
            pq.push({top.first + cost(i), top.second});
        }
        std::vector<int> csr(p.lu_grid + 1 + ninst);
        int pos = 0;
        for (int c = 0; c < p.lu_grid; ++c) {
            csr[c] = pos;
            for (int i : lists_c[c]) csr[p.lu_grid + 1 + pos++] = i;
        }
        csr[p.lu_grid] = pos;
        CUDA_OR_FAIL(p.d_cta.ensure(sizeof(int) * csr.size()), "alloc");
        CUDA_OR_FAIL(cudaMemcpyAsync(p.d_cta.p, csr.data(), sizeof(int) * csr.size(), cudaMemcpyHostToDevice,
                                     ctx->stream),
                     "copy lists");
    }
    // residual tasks (32 rows each)
    {
        std::vector<int2> rt;
        for (int i = 0; i < ninst; ++i)
            for (int r0 = 0; r0 < p.h_ng[i]; r0 += 32) rt.push_back(make_int2(i, r0));
        p.n_rtask = (int)rt.size();
        CUDA_OR_FAIL(p.d_rtask.ensure(sizeof(int2) * rt.size()), "alloc");
        CUDA_OR_FAIL(cudaMemcpyAsync(p.d_rtask.p, rt.data(), sizeof(int2) * rt.size(), cudaMemcpyHostToDevice,
                                     ctx->stream),
                     "copy tasks");
    }
    if (mixed) {
        CUDA_OR_FAIL(p.d_wtab.ensure(sizeof(float2) * (size_t)ninst * (p.kp / 2)), "alloc W");
        p.maps.resize(3 * p.nslot);
        for (int s = 0; s < p.nslot; ++s) {
            QSlot& q = *p.qs[s];
            unsigned char* base = reinterpret_cast<unsigned char*>(q.rho.p);
            const size_t plane = (size_t)q.ngp * q.kp * 2;
            for (int pc = 0; pc < 3; ++pc)
                if (!qcx_make_bf16_map(&p.maps[3 * s + pc], base + pc * plane, q.kp, q.ngp, 64, 32))
                    return ctx->fail(QCX_ERR_CUDA, "solve_batch: tensor map");
        }
    } else {
        std::vector<int4> tiles;
        for (int i = 0; i < ninst; ++i) {
            const int ng = p.h_ng[i];
            for (int g0 = 0; g0 < ng; g0 += FT)
                for (int h0 = 0; h0 < ng; h0 += FT) tiles.push_back(make_int4(i, g0, h0, 0));
        }
        p.ntile = (int)tiles.size();
        CUDA_OR_FAIL(p.d_tiles.ensure(sizeof(int4) * tiles.size()), "alloc");
        CUDA_OR_FAIL(cudaMemcpyAsync(p.d_tiles.p, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                     ctx->stream),
                     "copy tiles");
    }
    return QCX_OK;
}

// set the tensor-core tiles for the caps of the N_G classes (uploads the list; no launch).  The
// tile and accumulator buffers are sized once for the narrowest caps before the first capture,
// so no captured graph ever sees them reallocated.
qcx_status set_tiles(qcx_ctx* ctx, BatchPlan& p, const int (&caps)[3]) {
    std::vector<int4> tiles;
    make_tc_tiles(p, caps, tiles, p.grp_tile0, p.grp_ntile);
    p.ntile = (int)tiles.size();
    for (int c = 0; c < 3; ++c) p.caps[c] = caps[c];
    p.tile_cap = caps[2];
    p.tc_grid = std::min(p.ntile, sm_count(ctx->device));
    if (p.d_tiles.bytes < sizeof(int4) * tiles.size() || p.d_acc.bytes < qcx_chi0_tc_batch_acc_bytes(p.tc_grid))
        return ctx->fail(QCX_ERR_STATE, "solve_batch: tile buffers not sized for this cap");
    CUDA_OR_FAIL(cudaMemcpyAsync(p.d_tiles.p, tiles.data(), sizeof(int4) * tiles.size(), cudaMemcpyHostToDevice,
                                 ctx->stream),
                 "copy tiles");
    return QCX_OK;
}

qcx_status upload_inst(qcx_ctx* ctx, BatchPlan& p, const std::vector<double>& w) {
    for (int i = 0; i < p.ninst; ++i) p.hinst[i].w = w[i];
    CUDA_OR_FAIL(cudaMemcpyAsync(p.d_inst.p, p.hinst.data(), sizeof(BatchInst) * p.ninst, cudaMemcpyHostToDevice,
                                 ctx->stream),
                 "copy instances");
    return QCX_OK;
}

qcx_status time_exec(qcx_ctx* ctx, cudaGraphExec_t ex, double* ms) {
    cudaEvent_t e0, e1;
    CUDA_OR_FAIL(cudaEventCreate(&e0), "event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return ctx->fail(QCX_ERR_CUDA, "event");
    }
    cudaError_t e = cudaGraphLaunch(ex, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    for (int r = 0; r < 2 && e == cudaSuccess; ++r) e = cudaGraphLaunch(ex, ctx->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CUDA_OR_FAIL(e, "autotune timing");
    *ms = t / 2.0;
    return QCX_OK;
}

qcx_status prepare(qcx_ctx* ctx, BatchPlan& p) {
    if (p.prec == QCX_FP64) {
        CUDA_OR_FAIL(capture(ctx, p, &p.exec), "capture batch graph");
        return QCX_OK;
    }
    const bool tune = ctx->batch_tune != 0;
    {
        // the narrowest caps give the most tiles: size the buffers for them once
        size_t most = 0;
        std::vector<int4> tiles;
        std::vector<int> g0, gn;
        const int narrow[3] = {64, 64, 64};
        make_tc_tiles(p, narrow, tiles, g0, gn);
        most = tiles.size();
        const int grid = (int)std::min<size_t>(most, (size_t)sm_count(ctx->device));
        CUDA_OR_FAIL(p.d_tiles.ensure(sizeof(int4) * most), "alloc tiles");
        CUDA_OR_FAIL(p.d_acc.ensure(qcx_chi0_tc_batch_acc_bytes(grid)), "alloc acc");
    }
    // classes present in this batch
    bool present[3] = {false, false, false};
    for (int i = 0; i < p.ninst; ++i) {
        const int c = ng_class(p.hinst[i].ng);
        if (c >= 0) present[c] = true;
    }
    cudaEvent_t t0, t1;
    CUDA_OR_FAIL(cudaEventCreate(&t0), "event");
    CUDA_OR_FAIL(cudaEventCreate(&t1), "event");
    cudaEventRecord(t0, ctx->stream);
    // capture and time one set of caps; keeps its graph when it is the fastest so far
    double best = 1e300;
    int best_caps[3] = {192, 192, 192};
    auto trial = [&](const int (&caps)[3]) -> qcx_status {
        qcx_status st = set_tiles(ctx, p, caps);
        if (st != QCX_OK) return st;
        cudaGraphExec_t ex = nullptr;
        CUDA_OR_FAIL(capture(ctx, p, &ex), "capture batch graph");
        if (!tune) {
            p.exec = ex;
            return QCX_OK;
        }
        double ms = 0.0;
        st = time_exec(ctx, ex, &ms);
        if (st != QCX_OK) {
            cudaGraphExecDestroy(ex);
            return st;
        }
        if (ms < best) {
            best = ms;
            for (int c = 0; c < 3; ++c) best_caps[c] = caps[c];
            if (p.exec) cudaGraphExecDestroy(p.exec);
            p.exec = ex;
        } else {
            cudaGraphExecDestroy(ex);
        }
        return QCX_OK;
    };
    {
        const int start[3] = {192, 192, 192};
        qcx_status st = trial(start);
        if (st != QCX_OK) return st;
    }
    if (tune) {
        // one pass of coordinate descent, widest class first: each class tries the narrower caps
        // with the others at their best so far (a 65-128 class has only one narrower cap that
        // changes its tiles)
        const int alt[3][2] = {{64, 0}, {128, 64}, {128, 64}};
        for (int c = 2; c >= 0; --c) {
            if (!present[c]) continue;
            for (int a = 0; a < 2 && alt[c][a]; ++a) {
                int caps[3] = {best_caps[0], best_caps[1], best_caps[2]};
                caps[c] = alt[c][a];
                qcx_status st = trial(caps);
                if (st != QCX_OK) return st;
            }
        }
    }
    cudaEventRecord(t1, ctx->stream);
    cudaEventSynchronize(t1);
    float tms = 0.f;
    cudaEventElapsedTime(&tms, t0, t1);
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    p.tune_ms = tms;
    p.tuned = tune ? 1 : 0;
    // the kept graph reads the tile list of its own caps
    return set_tiles(ctx, p, best_caps);
}

}  // namespace

extern "C" {

qcx_status qcx_solve_batch(qcx_ctx* ctx, int ninst, const int* inst_q, const double* inst_w,
                           const double* inst_gmax, double eta, qcx_precision prec, double* out_L_lfe_head,
                           double* out_L_nolfe_head, int* out_ng) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nq) return ctx->fail(QCX_ERR_STATE, "solve_batch: no states");
    if (ninst < 1 || ninst > (1 << 20) || !inst_q || !inst_w || !inst_gmax || !out_L_lfe_head ||
        !out_L_nolfe_head || (prec != QCX_FP64 && prec != QCX_MIXED) || !(eta > 0) || !std::isfinite(eta))
        return ctx->fail(QCX_ERR_ARG, "solve_batch: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<int> iq;
    std::vector<double> w, gm;
    CUDA_OR_FAIL(fetch(ctx, iq, inst_q, ninst), "solve_batch q list");
    CUDA_OR_FAIL(fetch(ctx, w, inst_w, ninst), "solve_batch w list");
    CUDA_OR_FAIL(fetch(ctx, gm, inst_gmax, ninst), "solve_batch cutoffs");
    for (int i = 0; i < ninst; ++i) {
        if (iq[i] < 0 || iq[i] >= ctx->nq) return ctx->fail(QCX_ERR_ARG, "solve_batch: q index out of range");
        if (!std::isfinite(w[i]) || !std::isfinite(gm[i]) || !(gm[i] > 0))
            return ctx->fail(QCX_ERR_ARG, "solve_batch: non-finite frequency or cutoff");
    }
    BatchPlan* p = ctx->batch;
    const bool same = p && p->gen == ctx->gen && p->prec == (int)prec && p->eta == eta && p->ninst == ninst &&
                      p->key_q == iq && p->key_gmax == gm && p->wait_limit == ctx->wait_limit;
    if (!same) {
        delete ctx->batch;
        ctx->batch = nullptr;
        p = new (std::nothrow) BatchPlan();
        if (!p) return ctx->fail(QCX_ERR_ALLOC, "solve_batch: plan");
        p->gen = ctx->gen;
        p->prec = prec;
        p->eta = eta;
        p->ninst = ninst;
        p->key_q = iq;
        p->key_gmax = gm;
        p->wait_limit = ctx->wait_limit;
        qcx_status st = build_plan(ctx, *p);
        if (st == QCX_OK) st = upload_inst(ctx, *p, w);
        if (st == QCX_OK) st = prepare(ctx, *p);
        if (st != QCX_OK) {
            delete p;
            return st;
        }
        ctx->batch = p;
    } else {
        qcx_status st = upload_inst(ctx, *p, w);
        if (st != QCX_OK) return st;
    }
    CUDA_OR_FAIL(cudaGraphLaunch(p->exec, ctx->stream), "launch batch graph");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L_lfe_head, p->d_out.p, sizeof(double) * ninst), "copy out");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L_nolfe_head, p->d_out.as<double>() + ninst, sizeof(double) * ninst),
                 "copy out");
    std::vector<int> flags(ninst);
    int status = 0;
    CUDA_OR_FAIL(cudaMemcpyAsync(flags.data(), p->d_flags.p, sizeof(int) * ninst, cudaMemcpyDeviceToHost, ctx->stream),
                 "flags");
    CUDA_OR_FAIL(cudaMemcpyAsync(&status, p->d_status.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    if (out_ng) {
        if (qcx_is_device_ptr(out_ng)) {
            CUDA_OR_FAIL(cudaMemcpyAsync(out_ng, p->h_ng.data(), sizeof(int) * ninst, cudaMemcpyHostToDevice,
                                         ctx->stream),
                         "copy out");
            CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
        } else {
            std::memcpy(out_ng, p->h_ng.data(), sizeof(int) * ninst);
        }
    }
    if (status) return ctx->fail(QCX_ERR_TIMEOUT, "solve_batch: a pipeline wait in the tensor-core kernel gave up");
    int sing = 0, nconv = 0;
    for (int f : flags) {
        sing += f == 1;
        nconv += f == 2;
    }
    if (sing) return ctx->fail(QCX_ERR_SINGULAR, "solve_batch: " + std::to_string(sing) + " singular instance(s)");
    if (nconv)
        return ctx->fail(QCX_ERR_NOT_CONVERGED,
                         "solve_batch: refinement did not converge for " + std::to_string(nconv) + " instance(s)");
    return QCX_OK;
}

qcx_status qcx_batch_info(const qcx_ctx* ctx, int n, long long* out) {
    if (!ctx || n < 1 || !out) return QCX_ERR_ARG;
    const BatchPlan* p = ctx->batch;
    long long v[13] = {0};
    if (p) {
        v[0] = p->tile_cap;
        v[1] = p->ntile;
        v[2] = p->tc_grid;
        v[3] = p->lu_grid;
        v[4] = p->launches;
        v[5] = p->tuned;
        v[6] = p->nslot;
        v[7] = p->nmax;
        v[8] = (long long)(p->tune_ms * 1000.0);
        v[9] = p->prec;
        for (int c = 0; c < 3; ++c) v[10 + c] = p->caps[c];
    }
    for (int i = 0; i < n; ++i) out[i] = i < 13 ? v[i] : 0;
    return p ? QCX_OK : QCX_ERR_STATE;
}

qcx_status qcx_batch_autotune(qcx_ctx* ctx, int enable) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->batch_tune = enable ? 1 : 0;
    return QCX_OK;
}

}  // extern "C"
