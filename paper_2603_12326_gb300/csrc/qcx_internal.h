// Internal declarations of libqcx (context, buffers, kernel launchers).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <cstring>
#include <string>
#include <vector>

#include "qcx.h"

// ----------------------------------------------------------------- helpers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    // grow-only; contents are not preserved
    cudaError_t ensure(size_t n) {
        if (n <= bytes && p) return cudaSuccess;
        release();
        cudaError_t e = cudaMalloc(&p, n ? n : 16);
        if (e == cudaSuccess) bytes = n;
        return e;
    }
    template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Tables of the FP32 pair densities for one q: the one-dimensional lattice sums per shell-group
// pair, axis, distinct k component and distinct (q+G) component, and the factor that depends on
// the pair and G only, so the per-(k, G) kernel reads them instead of forming them again.
struct PdTab {
    bool valid = false;
    int nkx[3] = {0, 0, 0}, nqx[3] = {0, 0, 0};   // distinct k and q+G components per axis
    int kofs[3] = {0, 0, 0}, qofs[3] = {0, 0, 0}; // first value of each axis in kval / qval
    long long tbase[4] = {0, 0, 0, 0};            // first entry of each axis (tbase[3] = entries)
    DevBuf kidx, gidx;         // [nk][3], [ng][3] int: class of each point's component
    DevBuf kval, qval;         // float values of the classes (axes concatenated)
    DevBuf tab;                // [entries][nchar][4] float2: E(0,0), E(1,0), E(0,1), E(1,1)
    DevBuf cmn;                // [npair][ng] float2
};

// Per-precision working set of one q.
struct QSlot {
    int iq = -1;               // q whose pair densities are stored here
    int ng = 0;
    int nw = 0;
    bool have_rho = false;
    bool have_eps = false;
    DevBuf kappa;              // [ng][3] double, q + G (bohr^-1)
    DevBuf kappa32;            // [ng][3] float
    DevBuf vs;                 // [ng] double, sqrt(4 pi)/|q+G|
    DevBuf vs32;               // [ng] float
    DevBuf rho;                // FP64: [ng][nt] double2 ; MIXED: three BF16 planes [ngp][kp]
    DevBuf eps;                // [nw][ng][ng] double2 (MIXED stores eps^T: row G', column G)
    DevBuf work;               // inverse work space
    DevBuf acc64;              // FP64 partial sums of the tensor-core chi0 (one region per CTA)
    DevBuf wtab;               // [nw][kp/2] float2 transition weights of the mixed path
    DevBuf kappa1;             // [nw] double condition estimates of the mixed inverse
    DevBuf w;                  // [nw] double
    DevBuf diag_inv;           // [nw][ng] double2
    DevBuf eps_diag;           // [nw][ng] double2
    DevBuf resid;              // [nw] double
    DevBuf flags;              // [nw] int (singular / error flags)
    int ngp = 0;               // padded G rows of the BF16 planes (multiple of 16)
    long long kp = 0;          // padded K' = 2 nt columns of the BF16 planes
    double eta = 0.0;
    PdTab pdt;                 // MIXED: tables of the pair-density kernel for this slot's q and G list
};

// Loss tables kept per q after qcx_invert_eps.
struct LossTab {
    bool valid = false;        // holds the tables of the current states; buffers are kept when invalidated
    int ng = 0, nw = 0;
    DevBuf L;                  // [2][nw][ng] double: LFE then noLFE
    DevBuf qmag;               // [ng] double |q+G|
    DevBuf eps;                // [2][nw][ng] double2: eps^LFE (from Re [eps^-1]_GG and -L_LFE), eps^noLFE = eps_GG
    DevBuf kvec;               // [ng][3] double q + G (bohr^-1)
    std::vector<double> w;     // frequency grid (host copy, to check consistency)
};

// Separable lattice-sum tables of the basis (host-built, device copies).
struct PairTables {
    int npair = 0;
    int nblk = 0;              // basis row blocks
    std::vector<int> blk_pair_start;   // [nblk+1]
    std::vector<int> blk_row0;         // [nblk+1] first basis row of each block
    DevBuf meta;               // int4 per pair: {sa, sb, off_dir0, packed counts}
    DevBuf dir_off;            // int per (pair, dir): table offset ; count in dir_cnt
    DevBuf dir_cnt;
    DevBuf dir_nlo;            // int per (pair, dir): first n
    DevBuf par64;              // double per pair: {p, alpha/p, beta/p, pref, P0x, P0y, P0z, pad}
    DevBuf par32;              // float version
    DevBuf tab64;              // double2 per term: {w_n, d_n}
    DevBuf tab32;              // float2
    int max_rows = 0;          // rows of the largest block
};

// One uneven instance of a batched solve (device copy, read by the batch kernels).
struct BatchInst {
    int slot;                  // distinct-q slot (pair densities on the union G list of that q)
    int ng;                    // N_G: the first ng entries of the slot's list
    int head;                  // position of G = 0 in the list
    int iq;                    // q index into the context's states
    long long eps_off;         // double2 offset of eps [ng][ng] in the batch eps buffer
    long long work_off;        // element offset of the LU work matrix [ng][ng+1]
    const double* vs;          // [>= ng] v^1/2(q+G) of the slot's list
    const double2* rho64;      // FP64 path: [U][nt] pair densities of the slot
    double w;                  // frequency (Hartree)
    long long vec_off;         // offset of the instance's vectors (pivot order, solution, residual)
};
#define QCX_BATCH_MAXQ 16      // distinct q per persistent tensor-core launch
struct BatchPlan;
void qcx_batch_destroy(BatchPlan* p);

// Optical limit: momentum matrix of the basis on the k grid (kept while basis and states are
// unchanged) and the momentum elements of the current call.
struct OpticalBufs {
    DevBuf pairs;              // shell pairs with their lattice boxes
    DevBuf P;                  // [nk][3][nb][nb] double2
    DevBuf p;                  // [nt][3] double2 <c k|grad|v k>
    DevBuf status;
    unsigned long long gen = ~0ull;
    int nk = 0;
};

// Work space of the spectral route to chi0 (one q at a time, either precision).
struct SpecBufs {
    DevBuf bin, x;             // [nt] grid point and hat weight of each transition
    DevBuf cnt, fill, off;     // per grid point: count, fill cursor, group offsets [nbin + 1]
    DevBuf perm0, perm;        // [nt] transitions grouped by grid point (then ascending t)
    DevBuf status, range;
    DevBuf rhos, xs;           // pair densities [ng][nt] and x [nt] in the grouped order
    DevBuf tp;                 // upper (G, G') tile pairs
    DevBuf ktab;               // [nw][ldk] K(w, E_b)
    DevBuf S;                  // spectral weights of one chunk of grid points
    DevBuf chi;                // [nw][ng][ng] double2 chi0 accumulated over the chunks
    DevBuf Sout;               // staging of exported weights
    DevBuf kplanes, splanes;   // mixed route on the tensor cores: K table and chunk weights as BF16 planes
    // stage times of the last call (CUDA events on the context's stream): grouping, gather and
    // K table, spectral weights, contraction, Dyson step (ms)
    std::vector<cudaEvent_t> ev;
    double ms[5] = {0, 0, 0, 0, 0};
    SpecBufs() = default;
    SpecBufs(const SpecBufs&) = delete;
    SpecBufs& operator=(const SpecBufs&) = delete;
    ~SpecBufs() {
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
    cudaError_t events(size_t n) {
        while (ev.size() < n) {
            cudaEvent_t e;
            cudaError_t r = cudaEventCreate(&e);
            if (r != cudaSuccess) return r;
            ev.push_back(e);
        }
        return cudaSuccess;
    }
};
struct MlpState;
void qcx_mlp_destroy(MlpState* m);

struct qcx_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::string err;

    // basis
    int natom = 0, nshell = 0, nb = 0;
    double lattice[9] = {0};
    double h = 0.0;            // orthogonal spacing with lattice subset of h Z^3
    int nchar = 0;             // index of the lattice in h Z^3
    double chars[4][3] = {{0}};// characters (fractions of 2 pi per unit step)
    std::vector<double> atom_xyz;
    std::vector<int> shell_atom, shell_l, shell_mu0;
    std::vector<double> shell_exp;
    DevBuf d_shell_l, d_shell_mu0;
    int ngrp = 0;                      // shell groups (same atom and exponent, s then p)
    std::vector<int> grp_mu0_h;        // [ngrp + 1] first basis function of each group
    DevBuf d_grp_mu0, d_grp_mask;
    PairTables pairs;

    // states
    int nk = 0, nv = 0, nc = 0, nq = 0;
    std::vector<double> qpts;  // host copy
    std::vector<double> kpts_h;    // host copy [nk][3]
    DevBuf d_kpts, d_kpts32;   // [nk][3]
    DevBuf d_Ck64, d_Ck32;     // [nk][nb][nv]
    DevBuf d_Ek;               // [nk][nv]
    DevBuf d_Ckq64, d_Ckq32;   // [nq][nk][nb][nc]
    DevBuf d_Ekq;              // [nq][nk][nc]

    QSlot slot[2];             // index = qcx_precision
    std::vector<LossTab*> loss;    // [nq]

    DevBuf scratch;            // host<->device staging for outputs
    DevBuf scratch2;

    unsigned long long gen = 0;    // bumped whenever basis or states change
    BatchPlan* batch = nullptr;    // cached plan (and captured graph) of the last batched solve
    int batch_tune = 1;            // autotune the batch tiling when a new plan is built
    double kappa_refine = 1.0e4;   // mixed inverse: FP64 diagonal correction above this kappa_1
    long long wait_limit = 4000000000LL;  // tensor-core kernels: clock cycles before a pipeline wait gives up
    int withhold_copies = 0;       // fault injection (tests): the per-q tensor-core kernel issues no copies
    MlpState* mlp = nullptr;       // surrogate network (parameters, Adam moments, work buffers)
    SpecBufs spec;                 // spectral route work space
    OpticalBufs optical;           // optical-limit work space
    int spec_chunk_bins = 0;       // grid points per chunk of the spectral route (0: from a 4 GiB budget)
    int spec_cuda_cores = 0;       // mixed spectral contraction on the CUDA cores (FP32) instead of tcgen05

    ~qcx_ctx();
    qcx_status fail(qcx_status s, const std::string& msg) {
        err = msg;
        return s;
    }
};

// ------------------------------------------------------------ small utils
// Return from a qcx_status function when a CUDA call fails: the last-error state is cleared
// and `what` is recorded with CUDA's message in the context.
#define CUDA_OR_FAIL(call, what)                                                                \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) {                                                                \
            cudaGetLastError();                                                                 \
            return ctx->fail(e_ == cudaErrorMemoryAllocation ? QCX_ERR_ALLOC : QCX_ERR_CUDA,    \
                             std::string(what) + ": " + cudaGetErrorString(e_));                \
        }                                                                                       \
    } while (0)

bool qcx_is_device_ptr(const void* p);

// Host copy of a small host-or-device array (device sources synchronise the stream).
template <typename T> cudaError_t fetch(qcx_ctx* ctx, std::vector<T>& out, const T* src, size_t n) {
    out.resize(n);
    if (!n) return cudaSuccess;
    if (qcx_is_device_ptr(src)) {
        cudaError_t e = cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream);
        if (e != cudaSuccess) return e;
        return cudaStreamSynchronize(ctx->stream);
    }
    std::memcpy(out.data(), src, n * sizeof(T));
    return cudaSuccess;
}

// copy `bytes` from a host-or-device source into device memory (stream-ordered)
cudaError_t qcx_copy_in(qcx_ctx* ctx, void* dst_dev, const void* src, size_t bytes);
// copy device memory to a host-or-device destination; host destinations synchronise
cudaError_t qcx_copy_out(qcx_ctx* ctx, void* dst, const void* src_dev, size_t bytes);

// ---------------------------------------------------------------- launchers
// pair densities (pair_density.cu)
cudaError_t qcx_launch_qsetup(qcx_ctx* ctx, QSlot& s, const int* d_G, int ng, const double* q);
cudaError_t qcx_launch_pair_density(qcx_ctx* ctx, QSlot& s, int iq, qcx_precision prec);
// Plan and upload the tables of the FP32 pair densities for q number iq and the host G list (outside
// any stream capture); leaves s.pdt invalid (the kernel then forms every term itself) when the
// tables would not save work or exceed their memory budget.
cudaError_t qcx_pd_tab_prepare(qcx_ctx* ctx, QSlot& s, const int* G_host, int ng, int iq);
cudaError_t qcx_launch_overlap(qcx_ctx* ctx, int nk, const double* d_kpts, double2* d_out);
cudaError_t qcx_pair_density_configure();

// optical limit (optical.cu): momentum elements and the G = 0 row rho~ = -i qhat.p/dE of the
// slot's pair densities, v^1/2 of that row set to sqrt(4 pi); d_status bit 1: a zero dE
cudaError_t qcx_launch_optical(qcx_ctx* ctx, QSlot& s, int iq, int g0, const double qhat[3], qcx_precision prec,
                               int* d_status);

// spectral route on the tensor cores (spectral_tc.cu): K table as three BF16 planes [rows][ld]
// (row 2 w + r); one chunk's weights [pair][point][32][32] split into three K-major planes and
// contracted with the K planes into chi (FP64, stored or added)
cudaError_t qcx_spec_tc_ktab(cudaStream_t st, int nw, int rows, long long ld, int nbin, const double* w, double E0,
                             double step, double eta, __nv_bfloat16* planes);
cudaError_t qcx_spec_tc_contract(cudaStream_t st, const CUtensorMap* kmaps, const CUtensorMap* smaps, int mtiles,
                                 int ntiles, int nw, int ng, int nbc, int nb, int kb0, long long sld, const float2* S,
                                 __nv_bfloat16* splanes, const int2* tp, int accumulate, double2* chi, int* status,
                                 long long wait_limit);

// chi0 (chi0_fp64.cu, chi0_tc.cu)
cudaError_t qcx_launch_chi0_fp64(qcx_ctx* ctx, QSlot& s, int iq, double2* d_chi0_out);
cudaError_t qcx_launch_chi0_mixed(qcx_ctx* ctx, QSlot& s, int iq, double2* d_chi0_out, int* d_status);
// 2-D tensor map over one BF16 plane [rows][kp], box {box_k, box_rows} (box_k 16: 32-byte
// swizzle, 32: 64-byte swizzle)
bool qcx_make_bf16_map(CUtensorMap* m, void* base, long long kp, int rows, int box_rows, int box_k);

// persistent tensor-core chi0 over a tile list of uneven instances (chi0_tc_batch.cu).
// maps: [nslot][3] tensor maps (box {32, 64}) of the BF16 planes of slots slot0 .. slot0 + nslot - 1;
// tiles: {inst, gb, n0, N | src<<16}, every tile's instance in that slot range.
cudaError_t qcx_launch_chi0_tc_batch(cudaStream_t st, const CUtensorMap* maps, int slot0, int nslot, int ntile,
                                     const int4* d_tiles, int grid, const BatchInst* d_inst, const float2* wtab,
                                     long long wld, int kstages, double pref, double* acc64, double2* eps,
                                     int* status, long long wait_limit);
size_t qcx_chi0_tc_batch_acc_bytes(int grid);

// batched solve for the heads of eps^-1 (batch_solve.cu)
struct BatchSolveArgs {
    const BatchInst* inst;
    const int* cta_off;        // [grid + 1] instance lists per CTA (CSR)
    const int* cta_ids;
    const double2* eps;        // FP64 eps of every instance
    void* work;                // LU factors ([ng][ng+1] per instance, FP32 or FP64 complex)
    int* rowmap;               // [sum ng] pivot order: logical row -> stored row
    double2* x;                // [sum ng] solution of A' x = e_last (refined in place)
    double2* r;                // [sum ng] FP64 residual
    double* out;               // [3][ninst]: L_LFE head, L_noLFE head, last relative correction
    int* flags;                // [ninst]: 0 ok, 1 zero pivot, 2 refinement not converged
    int ninst;
};
cudaError_t qcx_launch_lu_head(cudaStream_t st, const BatchSolveArgs& a, int grid, int nmax, bool fp64, bool want_x);
cudaError_t qcx_launch_resid(cudaStream_t st, const BatchSolveArgs& a, const int2* tasks, int ntask);
cudaError_t qcx_launch_lu_correct(cudaStream_t st, const BatchSolveArgs& a, int grid, int nmax, int last);

// inverse + loss (invert.cu)
cudaError_t qcx_launch_invert(qcx_ctx* ctx, QSlot& s, qcx_precision prec, double* d_loss_out);

// rate (rate.cu)
cudaError_t qcx_launch_bin(qcx_ctx* ctx, int nsel, const double* const* d_L, const double* const* d_qmag,
                           const int* d_ng, int nw, int which, int nbin, const double* d_edges,
                           double* d_out, double* d_cnt);
cudaError_t qcx_launch_rate(qcx_ctx* ctx, int nqbin, const double* d_q, int nw, const double* d_w,
                            const double* d_L, const qcx_halo_params& p, double* d_dRdw, int nQ,
                            double* d_dRQ);
cudaError_t qcx_launch_recoil(cudaStream_t st, int nw, const double* d_w, const double* d_dRdw, double wgap_eV,
                              double wpp_eV, int nQ, double* d_dRQ);
// rate_ext.cu: the per-q dielectric values kept for the 3-D binning (after qcx_launch_invert)
cudaError_t qcx_launch_store_eps(cudaStream_t st, int nw, int ng, const double2* diag_inv, const double2* eps_diag,
                                 const double* L_lfe, double2* out);

// 4 pi as used by v^1/2 = sqrt(4 pi)/|k|
#define QCX_SQRT_4PI 3.5449077018110318
