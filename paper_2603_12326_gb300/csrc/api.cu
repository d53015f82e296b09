// C ABI of libqcx: argument checks, device state, calls into the kernels.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <cmath>
#include <cstring>
#include <new>

qcx_status qcx_build_pair_tables(qcx_ctx* ctx);

namespace {

__global__ void k_to_float2(const double2* in, float2* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = make_float2((float)in[i].x, (float)in[i].y);
}
__global__ void k_to_float(const double* in, float* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}
// rho [ng][nt] (FP64) or the three BF16 planes [ngp][kp] -> [nt][ng] double2
__global__ void k_rho_export(int ng, long long nt, const double2* R64, const __nv_bfloat162* p0,
                             long long plane2, long long kp2, double2* out) {
    const long long n = nt * ng;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long t = i / ng;
        const int g = (int)(i - t * ng);
        if (R64) {
            out[i] = R64[(long long)g * nt + t];
        } else {
            const long long o = (long long)g * kp2 + t;
            const float2 a = __bfloat1622float2(p0[o]);
            const float2 b = __bfloat1622float2(p0[o + plane2]);
            const float2 c = __bfloat1622float2(p0[o + 2 * plane2]);
            out[i] = make_double2((double)a.x + (double)b.x + (double)c.x, (double)a.y + (double)b.y + (double)c.y);
        }
    }
}
__global__ void k_kmag(int ng, const double* kappa, double* out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g < ng) {
        const double x = kappa[3 * g], y = kappa[3 * g + 1], z = kappa[3 * g + 2];
        out[g] = sqrt(x * x + y * y + z * z);
    }
}

inline int nblocks(size_t n, int t = 256) {
    size_t b = (n + t - 1) / t;
    return (int)(b > 4096 ? 4096 : (b ? b : 1));
}

bool finite_all(const double* p, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

qcx_ctx::~qcx_ctx() {
    qcx_batch_destroy(batch);
    qcx_mlp_destroy(mlp);
    for (auto* l : loss) delete l;
    if (own_stream && stream) cudaStreamDestroy(stream);
}

bool qcx_is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

cudaError_t qcx_copy_in(qcx_ctx* ctx, void* dst_dev, const void* src, size_t bytes) {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(dst_dev, src, bytes, qcx_is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           ctx->stream);
}

cudaError_t qcx_copy_out(qcx_ctx* ctx, void* dst, const void* src_dev, size_t bytes) {
    if (!bytes || !dst) return cudaSuccess;
    if (qcx_is_device_ptr(dst))
        return cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDeviceToDevice, ctx->stream);
    cudaError_t e = cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(ctx->stream);
}

// ===================================================================== ABI
extern "C" {

qcx_status qcx_create(qcx_ctx** out, int device, void* cuda_stream) {
    if (!out) return QCX_ERR_ARG;
    *out = nullptr;
    qcx_ctx* ctx = new (std::nothrow) qcx_ctx();
    if (!ctx) return QCX_ERR_ALLOC;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        delete ctx;
        return QCX_ERR_CUDA;
    }
    cudaDeviceProp prop;
    if (cudaSetDevice(device) != cudaSuccess || cudaGetDeviceProperties(&prop, device) != cudaSuccess ||
        prop.major != 10 || prop.minor != 3) {
        cudaGetLastError();
        delete ctx;
        return QCX_ERR_CUDA;     // kernels are built for sm_103a only
    }
    // the kernels of this library must have been built for this device's architecture (10.3)
    cudaFuncAttributes fa;
    if (cudaFuncGetAttributes(&fa, (const void*)k_kmag) != cudaSuccess || fa.binaryVersion != 103) {
        cudaGetLastError();
        delete ctx;
        return QCX_ERR_CUDA;
    }
    ctx->device = device;
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return QCX_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return QCX_OK;
}

void qcx_destroy(qcx_ctx* ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    delete ctx;
}

const char* qcx_last_error(const qcx_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

qcx_status qcx_sync(qcx_ctx* ctx) {
    if (!ctx) return QCX_ERR_ARG;
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

int qcx_nbasis(const qcx_ctx* ctx) { return ctx ? ctx->nb : 0; }

qcx_status qcx_set_basis(qcx_ctx* ctx, const double* lattice, int natom, const double* atom_xyz, int nshell,
                         const int* shell_atom, const int* shell_l, const double* shell_exp) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!lattice || !atom_xyz || !shell_atom || !shell_l || !shell_exp || natom < 1 || nshell < 1 ||
        nshell > 4096)
        return ctx->fail(QCX_ERR_ARG, "set_basis: null array or bad size");
    cudaSetDevice(ctx->device);
    std::vector<double> lat, xyz, ex;
    std::vector<int> sa, sl;
    CUDA_OR_FAIL(fetch(ctx, lat, lattice, 9), "set_basis lattice");
    CUDA_OR_FAIL(fetch(ctx, xyz, atom_xyz, 3 * (size_t)natom), "set_basis atoms");
    CUDA_OR_FAIL(fetch(ctx, sa, shell_atom, nshell), "set_basis shells");
    CUDA_OR_FAIL(fetch(ctx, sl, shell_l, nshell), "set_basis shells");
    CUDA_OR_FAIL(fetch(ctx, ex, shell_exp, nshell), "set_basis shells");
    if (!finite_all(lat.data(), 9) || !finite_all(xyz.data(), xyz.size()))
        return ctx->fail(QCX_ERR_ARG, "set_basis: non-finite geometry");
    int nb = 0;
    std::vector<int> mu0(nshell);
    for (int s = 0; s < nshell; ++s) {
        if (sa[s] < 0 || sa[s] >= natom) return ctx->fail(QCX_ERR_ARG, "set_basis: shell_atom out of range");
        if (sl[s] != 0 && sl[s] != 1) return ctx->fail(QCX_ERR_UNSUPPORTED, "set_basis: only l = 0, 1 shells");
        if (!(ex[s] > 0) || !std::isfinite(ex[s])) return ctx->fail(QCX_ERR_ARG, "set_basis: exponent <= 0");
        mu0[s] = nb;
        nb += sl[s] ? 3 : 1;
    }
    // drop states that belonged to an earlier basis
    ++ctx->gen;
    ctx->nk = ctx->nv = ctx->nc = ctx->nq = 0;
    for (auto& s : ctx->slot) {
        s.iq = -1;
        s.have_rho = s.have_eps = false;
    }
    for (auto* l : ctx->loss) delete l;
    ctx->loss.clear();
    std::memcpy(ctx->lattice, lat.data(), sizeof(ctx->lattice));
    ctx->natom = natom;
    ctx->nshell = nshell;
    ctx->nb = nb;
    ctx->atom_xyz = xyz;
    ctx->shell_atom = sa;
    ctx->shell_l = sl;
    ctx->shell_exp = ex;
    ctx->shell_mu0 = mu0;
    qcx_status st = qcx_build_pair_tables(ctx);
    if (st != QCX_OK) {
        ctx->nb = 0;
        return st;
    }
    CUDA_OR_FAIL(ctx->d_shell_l.ensure(nshell * sizeof(int)), "alloc");
    CUDA_OR_FAIL(ctx->d_shell_mu0.ensure(nshell * sizeof(int)), "alloc");
    CUDA_OR_FAIL(cudaMemcpy(ctx->d_shell_l.p, sl.data(), nshell * sizeof(int), cudaMemcpyHostToDevice), "copy");
    CUDA_OR_FAIL(cudaMemcpy(ctx->d_shell_mu0.p, mu0.data(), nshell * sizeof(int), cudaMemcpyHostToDevice), "copy");
    return QCX_OK;
}

qcx_status qcx_overlap(qcx_ctx* ctx, int nk, const double* kpts, qcx_c64* out_S) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nb) return ctx->fail(QCX_ERR_STATE, "overlap: no basis");
    if (nk < 1 || !kpts || !out_S) return ctx->fail(QCX_ERR_ARG, "overlap: bad arguments");
    cudaSetDevice(ctx->device);
    const size_t nout = (size_t)nk * ctx->nb * ctx->nb * sizeof(double2);
    CUDA_OR_FAIL(ctx->scratch2.ensure(3 * sizeof(double) * nk), "alloc");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->scratch2.p, kpts, 3 * sizeof(double) * nk), "copy kpts");
    double2* dst = qcx_is_device_ptr(out_S) ? reinterpret_cast<double2*>(out_S) : nullptr;
    if (!dst) {
        CUDA_OR_FAIL(ctx->scratch.ensure(nout), "alloc");
        dst = ctx->scratch.as<double2>();
    }
    CUDA_OR_FAIL(qcx_launch_overlap(ctx, nk, ctx->scratch2.as<double>(), dst), "overlap kernel");
    if (dst != reinterpret_cast<double2*>(out_S)) CUDA_OR_FAIL(qcx_copy_out(ctx, out_S, dst, nout), "copy out");
    return QCX_OK;
}

qcx_status qcx_set_states(qcx_ctx* ctx, int nk, const double* kpts, int nv, const qcx_c64* C_k, const double* E_k,
                          int nq, const double* qpts, int nc, const qcx_c64* C_kq, const double* E_kq) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nb) return ctx->fail(QCX_ERR_STATE, "set_states: no basis");
    if (nk < 1 || nv < 1 || nc < 1 || nq < 1 || !kpts || !C_k || !E_k || !qpts || !C_kq || !E_kq)
        return ctx->fail(QCX_ERR_ARG, "set_states: bad arguments");
    if ((long long)nk * nv * nc > (1ll << 30)) return ctx->fail(QCX_ERR_ARG, "set_states: too many transitions");
    cudaSetDevice(ctx->device);
    std::vector<double> qh, kh;
    CUDA_OR_FAIL(fetch(ctx, qh, qpts, 3 * (size_t)nq), "set_states qpts");
    CUDA_OR_FAIL(fetch(ctx, kh, kpts, 3 * (size_t)nk), "set_states kpts");
    if (!finite_all(qh.data(), qh.size())) return ctx->fail(QCX_ERR_ARG, "set_states: non-finite q");
    const size_t nb = ctx->nb;
    const size_t nCk = (size_t)nk * nb * nv, nCkq = (size_t)nq * nk * nb * nc;
    CUDA_OR_FAIL(ctx->d_kpts.ensure(3 * sizeof(double) * nk), "alloc kpts");
    CUDA_OR_FAIL(ctx->d_kpts32.ensure(3 * sizeof(float) * nk), "alloc kpts");
    CUDA_OR_FAIL(ctx->d_Ck64.ensure(nCk * sizeof(double2)), "alloc C_k");
    CUDA_OR_FAIL(ctx->d_Ck32.ensure(nCk * sizeof(float2)), "alloc C_k");
    CUDA_OR_FAIL(ctx->d_Ek.ensure((size_t)nk * nv * sizeof(double)), "alloc E_k");
    CUDA_OR_FAIL(ctx->d_Ckq64.ensure(nCkq * sizeof(double2)), "alloc C_kq");
    CUDA_OR_FAIL(ctx->d_Ckq32.ensure(nCkq * sizeof(float2)), "alloc C_kq");
    CUDA_OR_FAIL(ctx->d_Ekq.ensure((size_t)nq * nk * nc * sizeof(double)), "alloc E_kq");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->d_kpts.p, kpts, 3 * sizeof(double) * nk), "copy kpts");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->d_Ck64.p, C_k, nCk * sizeof(double2)), "copy C_k");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->d_Ek.p, E_k, (size_t)nk * nv * sizeof(double)), "copy E_k");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->d_Ckq64.p, C_kq, nCkq * sizeof(double2)), "copy C_kq");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->d_Ekq.p, E_kq, (size_t)nq * nk * nc * sizeof(double)), "copy E_kq");
    k_to_float<<<nblocks(3 * nk), 256, 0, ctx->stream>>>(ctx->d_kpts.as<double>(), ctx->d_kpts32.as<float>(), 3 * nk);
    k_to_float2<<<nblocks(nCk), 256, 0, ctx->stream>>>(ctx->d_Ck64.as<double2>(), ctx->d_Ck32.as<float2>(), nCk);
    k_to_float2<<<nblocks(nCkq), 256, 0, ctx->stream>>>(ctx->d_Ckq64.as<double2>(), ctx->d_Ckq32.as<float2>(), nCkq);
    CUDA_OR_FAIL(cudaGetLastError(), "convert states");
    ++ctx->gen;
    ctx->kpts_h = kh;
    ctx->nk = nk;
    ctx->nv = nv;
    ctx->nc = nc;
    ctx->nq = nq;
    ctx->qpts = qh;
    for (auto& s : ctx->slot) {
        s.iq = -1;
        s.have_rho = s.have_eps = false;
    }
    // keep the tables' device buffers for the new states (no allocation in a steady loop)
    for (size_t i = nq; i < ctx->loss.size(); ++i) delete ctx->loss[i];
    ctx->loss.resize(nq, nullptr);
    for (auto* l : ctx->loss)
        if (l) l->valid = false;
    return QCX_OK;
}

qcx_status qcx_pair_density(qcx_ctx* ctx, int iq, int ng, const int* G_int, qcx_precision prec, qcx_c64* out_rho) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nq) return ctx->fail(QCX_ERR_STATE, "pair_density: no states");
    if (iq < 0 || iq >= ctx->nq || ng < 1 || ng > 4096 || !G_int || (prec != QCX_FP64 && prec != QCX_MIXED))
        return ctx->fail(QCX_ERR_ARG, "pair_density: bad arguments");
    cudaSetDevice(ctx->device);
    QSlot& s = ctx->slot[prec];
    const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
    s.iq = -1;
    s.have_rho = s.have_eps = false;
    s.ng = ng;
    s.ngp = (ng + 15) / 16 * 16;
    s.kp = (2 * nt + 63) / 64 * 64;   // K' = 2 nt padded to the 32-element stage (and 128-byte rows)
    CUDA_OR_FAIL(s.kappa.ensure(3 * sizeof(double) * ng), "alloc");
    CUDA_OR_FAIL(s.kappa32.ensure(3 * sizeof(float) * ng), "alloc");
    CUDA_OR_FAIL(s.vs.ensure(sizeof(double) * ng), "alloc");
    CUDA_OR_FAIL(s.vs32.ensure(sizeof(float) * ng), "alloc");
    CUDA_OR_FAIL(ctx->scratch2.ensure(3 * sizeof(int) * ng), "alloc");
    CUDA_OR_FAIL(qcx_copy_in(ctx, ctx->scratch2.p, G_int, 3 * sizeof(int) * ng), "copy G");
    CUDA_OR_FAIL(qcx_launch_qsetup(ctx, s, ctx->scratch2.as<int>(), ng, &ctx->qpts[3 * iq]), "q setup");
    if (prec == QCX_MIXED) {
        std::vector<int> Gh;
        CUDA_OR_FAIL(fetch(ctx, Gh, G_int, 3 * (size_t)ng), "G list");
        CUDA_OR_FAIL(qcx_pd_tab_prepare(ctx, s, Gh.data(), ng, iq), "pair-density tables");
    }
    if (prec == QCX_FP64) {
        CUDA_OR_FAIL(s.rho.ensure((size_t)ng * nt * sizeof(double2)), "alloc rho");
    } else {
        const size_t bytes = 3 * (size_t)s.ngp * s.kp * sizeof(__nv_bfloat16);
        CUDA_OR_FAIL(s.rho.ensure(bytes), "alloc rho");
        CUDA_OR_FAIL(cudaMemsetAsync(s.rho.p, 0, bytes, ctx->stream), "clear rho");
    }
    cudaError_t e = qcx_launch_pair_density(ctx, s, iq, prec);
    if (e == cudaErrorInvalidValue)
        return ctx->fail(QCX_ERR_UNSUPPORTED, "pair_density: basis too large for the shared-memory plan");
    CUDA_OR_FAIL(e, "pair density kernel");
    if (out_rho) {
        const size_t nout = (size_t)nt * ng * sizeof(double2);
        double2* dst = qcx_is_device_ptr(out_rho) ? reinterpret_cast<double2*>(out_rho) : nullptr;
        if (!dst) {
            CUDA_OR_FAIL(ctx->scratch.ensure(nout), "alloc");
            dst = ctx->scratch.as<double2>();
        }
        k_rho_export<<<nblocks((size_t)nt * ng), 256, 0, ctx->stream>>>(
            ng, nt, prec == QCX_FP64 ? s.rho.as<double2>() : nullptr,
            reinterpret_cast<const __nv_bfloat162*>(s.rho.p), (long long)s.ngp * (s.kp / 2), s.kp / 2, dst);
        CUDA_OR_FAIL(cudaGetLastError(), "export rho");
        if (dst != reinterpret_cast<double2*>(out_rho)) CUDA_OR_FAIL(qcx_copy_out(ctx, out_rho, dst, nout), "copy out");
    }
    s.iq = iq;
    s.have_rho = true;
    if (ctx->loss[iq]) ctx->loss[iq]->valid = false;
    return QCX_OK;
}

qcx_status qcx_pair_density_optical(qcx_ctx* ctx, int iq, int ng, const int* G_int, const double* qhat,
                                    qcx_precision prec, qcx_c64* out_rho) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (!ctx->nq) return ctx->fail(QCX_ERR_STATE, "pair_density_optical: no states");
    if (iq < 0 || iq >= ctx->nq || ng < 1 || ng > 4096 || !G_int || !qhat ||
        (prec != QCX_FP64 && prec != QCX_MIXED))
        return ctx->fail(QCX_ERR_ARG, "pair_density_optical: bad arguments");
    const double* q = &ctx->qpts[3 * iq];
    if (q[0] != 0.0 || q[1] != 0.0 || q[2] != 0.0)
        return ctx->fail(QCX_ERR_ARG, "pair_density_optical: q number iq must be zero");
    cudaSetDevice(ctx->device);
    std::vector<double> qh;
    CUDA_OR_FAIL(fetch(ctx, qh, qhat, 3), "optical direction");
    const double qn = std::sqrt(qh[0] * qh[0] + qh[1] * qh[1] + qh[2] * qh[2]);
    if (!(qn > 0.0) || !std::isfinite(qn)) return ctx->fail(QCX_ERR_ARG, "pair_density_optical: bad direction");
    const double dir[3] = {qh[0] / qn, qh[1] / qn, qh[2] / qn};
    std::vector<int> Gh;
    CUDA_OR_FAIL(fetch(ctx, Gh, G_int, 3 * (size_t)ng), "G list");
    int g0 = -1, n0 = 0;
    for (int g = 0; g < ng; ++g)
        if (Gh[3 * g] == 0 && Gh[3 * g + 1] == 0 && Gh[3 * g + 2] == 0) {
            g0 = g;
            ++n0;
        }
    if (n0 != 1) return ctx->fail(QCX_ERR_ARG, "pair_density_optical: the G list must hold G = 0 exactly once");
    qcx_status st = qcx_pair_density(ctx, iq, ng, G_int, prec, nullptr);
    if (st != QCX_OK) return st;
    QSlot& s = ctx->slot[prec];
    s.have_rho = false;                                 // until the G = 0 row is in place
    OpticalBufs& ob = ctx->optical;
    CUDA_OR_FAIL(ob.status.ensure(sizeof(int)), "alloc");
    CUDA_OR_FAIL(cudaMemsetAsync(ob.status.p, 0, sizeof(int), ctx->stream), "clear");
    cudaError_t e = qcx_launch_optical(ctx, s, iq, g0, dir, prec, ob.status.as<int>());
    if (e == cudaErrorInvalidValue)
        return ctx->fail(QCX_ERR_UNSUPPORTED, "pair_density_optical: basis x valence bands too large for shared memory");
    CUDA_OR_FAIL(e, "optical-limit kernels");
    int bad = 0;
    CUDA_OR_FAIL(cudaMemcpyAsync(&bad, ob.status.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    if (bad) return ctx->fail(QCX_ERR_ARG, "pair_density_optical: a transition with zero energy");
    if (out_rho) {
        const long long nt = (long long)ctx->nk * ctx->nv * ctx->nc;
        const size_t nout = (size_t)nt * ng * sizeof(double2);
        double2* dst = qcx_is_device_ptr(out_rho) ? reinterpret_cast<double2*>(out_rho) : nullptr;
        if (!dst) {
            CUDA_OR_FAIL(ctx->scratch.ensure(nout), "alloc");
            dst = ctx->scratch.as<double2>();
        }
        k_rho_export<<<nblocks((size_t)nt * ng), 256, 0, ctx->stream>>>(
            ng, nt, prec == QCX_FP64 ? s.rho.as<double2>() : nullptr,
            reinterpret_cast<const __nv_bfloat162*>(s.rho.p), (long long)s.ngp * (s.kp / 2), s.kp / 2, dst);
        CUDA_OR_FAIL(cudaGetLastError(), "export rho");
        if (dst != reinterpret_cast<double2*>(out_rho)) CUDA_OR_FAIL(qcx_copy_out(ctx, out_rho, dst, nout), "copy out");
    }
    s.have_rho = true;
    return QCX_OK;
}

qcx_status qcx_chi0(qcx_ctx* ctx, int iq, int nw, const double* w, double eta, qcx_precision prec,
                    qcx_c64* out_chi0) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (prec != QCX_FP64 && prec != QCX_MIXED) return ctx->fail(QCX_ERR_ARG, "chi0: bad precision");
    QSlot& s = ctx->slot[prec];
    if (!s.have_rho || s.iq != iq) return ctx->fail(QCX_ERR_STATE, "chi0: pair densities of this q not computed");
    if (nw < 1 || !w || !(eta > 0) || !std::isfinite(eta)) return ctx->fail(QCX_ERR_ARG, "chi0: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<double> wh;
    CUDA_OR_FAIL(fetch(ctx, wh, w, nw), "chi0 w");
    if (!finite_all(wh.data(), nw)) return ctx->fail(QCX_ERR_ARG, "chi0: non-finite frequency");
    s.nw = nw;
    s.eta = eta;
    s.have_eps = false;
    if (ctx->loss[iq]) ctx->loss[iq]->valid = false;     // the tables of iq belong to the previous chi0
    const int ng = s.ng;
    CUDA_OR_FAIL(s.w.ensure(sizeof(double) * nw), "alloc");
    CUDA_OR_FAIL(cudaMemcpyAsync(s.w.p, wh.data(), sizeof(double) * nw, cudaMemcpyHostToDevice, ctx->stream), "copy w");
    const size_t nmat = (size_t)nw * ng * ng;
    CUDA_OR_FAIL(s.eps.ensure(nmat * sizeof(double2)), "alloc eps");
    double2* chi = nullptr;
    if (out_chi0) {
        chi = qcx_is_device_ptr(out_chi0) ? reinterpret_cast<double2*>(out_chi0) : nullptr;
        if (!chi) {
            CUDA_OR_FAIL(ctx->scratch.ensure(nmat * sizeof(double2)), "alloc");
            chi = ctx->scratch.as<double2>();
        }
    }
    if (prec == QCX_FP64) {
        CUDA_OR_FAIL(qcx_launch_chi0_fp64(ctx, s, iq, chi), "chi0 fp64 kernel");
    } else {
        CUDA_OR_FAIL(s.flags.ensure(sizeof(int) * (nw > 4 ? nw : 4)), "alloc");
        CUDA_OR_FAIL(cudaMemsetAsync(s.flags.p, 0, sizeof(int), ctx->stream), "clear status");
        cudaError_t e = qcx_launch_chi0_mixed(ctx, s, iq, chi, s.flags.as<int>());
        if (e == cudaErrorNotSupported)
            return ctx->fail(QCX_ERR_UNSUPPORTED, "chi0: this G-set size is not handled by the tensor-core kernel");
        CUDA_OR_FAIL(e, "chi0 tensor-core kernel");
        int st = 0;
        CUDA_OR_FAIL(cudaMemcpyAsync(&st, s.flags.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream), "status");
        CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
        if (st) return ctx->fail(QCX_ERR_TIMEOUT, "chi0: a pipeline wait in the tensor-core kernel gave up");
    }
    if (out_chi0 && chi != reinterpret_cast<double2*>(out_chi0))
        CUDA_OR_FAIL(qcx_copy_out(ctx, out_chi0, chi, nmat * sizeof(double2)), "copy out");
    s.have_eps = true;
    return QCX_OK;
}

qcx_status qcx_invert_eps(qcx_ctx* ctx, int iq, qcx_precision prec, qcx_c64* out_diag_inv, qcx_c64* out_eps_diag,
                          double* out_resid) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (prec != QCX_FP64 && prec != QCX_MIXED) return ctx->fail(QCX_ERR_ARG, "invert: bad precision");
    QSlot& s = ctx->slot[prec];
    if (!s.have_eps || s.iq != iq) return ctx->fail(QCX_ERR_STATE, "invert: chi0 of this q not computed");
    cudaSetDevice(ctx->device);
    const int ng = s.ng, nw = s.nw;
    const size_t nmat = (size_t)nw * ng * ng;
    CUDA_OR_FAIL(s.work.ensure(nmat * (prec == QCX_FP64 ? sizeof(double2) : sizeof(float2))), "alloc work");
    CUDA_OR_FAIL(s.diag_inv.ensure((size_t)nw * ng * sizeof(double2)), "alloc");
    CUDA_OR_FAIL(s.eps_diag.ensure((size_t)nw * ng * sizeof(double2)), "alloc");
    CUDA_OR_FAIL(s.resid.ensure(nw * sizeof(double)), "alloc");
    CUDA_OR_FAIL(s.flags.ensure(nw * sizeof(int)), "alloc");
    LossTab* lt = ctx->loss[iq];
    if (!lt) {
        lt = new (std::nothrow) LossTab();
        if (!lt) return ctx->fail(QCX_ERR_ALLOC, "loss table");
        ctx->loss[iq] = lt;
    }
    lt->ng = ng;
    lt->nw = nw;
    CUDA_OR_FAIL(lt->L.ensure(2 * (size_t)nw * ng * sizeof(double)), "alloc loss");
    CUDA_OR_FAIL(lt->qmag.ensure(ng * sizeof(double)), "alloc");
    k_kmag<<<(ng + 127) / 128, 128, 0, ctx->stream>>>(ng, s.kappa.as<double>(), lt->qmag.as<double>());
    CUDA_OR_FAIL(qcx_launch_invert(ctx, s, prec, lt->L.as<double>()), "invert kernel");
    // the dielectric values of this q kept for the 3-D binning of the composite function
    CUDA_OR_FAIL(lt->eps.ensure(2 * (size_t)nw * ng * sizeof(double2)), "alloc eps table");
    CUDA_OR_FAIL(lt->kvec.ensure(3 * sizeof(double) * ng), "alloc");
    CUDA_OR_FAIL(qcx_launch_store_eps(ctx->stream, nw, ng, s.diag_inv.as<double2>(), s.eps_diag.as<double2>(),
                                      lt->L.as<double>(), lt->eps.as<double2>()),
                 "store eps");
    CUDA_OR_FAIL(cudaMemcpyAsync(lt->kvec.p, s.kappa.p, 3 * sizeof(double) * ng, cudaMemcpyDeviceToDevice,
                                 ctx->stream),
                 "copy q+G");
    lt->w.resize(nw);
    CUDA_OR_FAIL(cudaMemcpyAsync(lt->w.data(), s.w.p, nw * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream), "w");
    lt->valid = true;
    std::vector<int> flags(nw);
    CUDA_OR_FAIL(cudaMemcpyAsync(flags.data(), s.flags.p, nw * sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
                 "flags");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_diag_inv, s.diag_inv.p, (size_t)nw * ng * sizeof(double2)), "copy out");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_eps_diag, s.eps_diag.p, (size_t)nw * ng * sizeof(double2)), "copy out");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_resid, s.resid.p, nw * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    int bad = 0;
    for (int f : flags) bad += f != 0;
    if (bad) return ctx->fail(QCX_ERR_SINGULAR, "invert: " + std::to_string(bad) + " singular block(s)");
    return QCX_OK;
}

qcx_status qcx_set_wait_limit(qcx_ctx* ctx, long long cycles) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (cycles < 1) return ctx->fail(QCX_ERR_ARG, "set_wait_limit: cycles must be positive");
    ctx->wait_limit = cycles;
    return QCX_OK;
}

qcx_status qcx_set_fault_injection(qcx_ctx* ctx, int withhold_copies) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    ctx->withhold_copies = withhold_copies ? 1 : 0;
    return QCX_OK;
}

qcx_status qcx_loss_function(qcx_ctx* ctx, int iq, double* out_L_lfe, double* out_L_nolfe) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (iq < 0 || iq >= ctx->nq || !ctx->loss[iq] || !ctx->loss[iq]->valid)
        return ctx->fail(QCX_ERR_STATE, "loss: q not inverted");
    cudaSetDevice(ctx->device);
    LossTab* lt = ctx->loss[iq];
    const size_t n = (size_t)lt->nw * lt->ng * sizeof(double);
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L_lfe, lt->L.p, n), "copy out");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L_nolfe, lt->L.as<double>() + (size_t)lt->nw * lt->ng, n), "copy out");
    return QCX_OK;
}

qcx_status qcx_bin_loss(qcx_ctx* ctx, int nsel, const int* iq_list, int which, int nbin, const double* edges,
                        double* out_L, double* out_count) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (nsel < 1 || !iq_list || (which != 0 && which != 1) || nbin < 1 || !edges || !out_L)
        return ctx->fail(QCX_ERR_ARG, "bin_loss: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<int> iqs;
    std::vector<double> ed;
    CUDA_OR_FAIL(fetch(ctx, iqs, iq_list, nsel), "bin iq list");
    CUDA_OR_FAIL(fetch(ctx, ed, edges, nbin + 1), "bin edges");
    for (int i = 0; i < nbin; ++i)
        if (!(ed[i] < ed[i + 1])) return ctx->fail(QCX_ERR_ARG, "bin_loss: edges not ascending");
    std::vector<const double*> Lp(nsel), Qp(nsel);
    std::vector<int> ngs(nsel);
    int nw = -1;
    const std::vector<double>* wref = nullptr;
    for (int i = 0; i < nsel; ++i) {
        const int iq = iqs[i];
        if (iq < 0 || iq >= ctx->nq || !ctx->loss[iq] || !ctx->loss[iq]->valid)
            return ctx->fail(QCX_ERR_STATE, "bin_loss: q not inverted");
        LossTab* lt = ctx->loss[iq];
        if (nw < 0) {
            nw = lt->nw;
            wref = &lt->w;
        } else if (lt->nw != nw || lt->w != *wref) {
            return ctx->fail(QCX_ERR_ARG, "bin_loss: q tables use different frequency grids");
        }
        Lp[i] = lt->L.as<double>();
        Qp[i] = lt->qmag.as<double>();
        ngs[i] = lt->ng;
    }
    const size_t off_L = 0, off_Q = nsel * sizeof(void*), off_n = 2 * nsel * sizeof(void*);
    const size_t off_e = (off_n + nsel * sizeof(int) + 15) / 16 * 16;
    const size_t off_o = off_e + (nbin + 1) * sizeof(double);
    const size_t off_c = off_o + (size_t)nbin * nw * sizeof(double);
    const size_t total = off_c + nbin * sizeof(double);
    CUDA_OR_FAIL(ctx->scratch2.ensure(total), "alloc");
    char* base = ctx->scratch2.as<char>();
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_L, Lp.data(), nsel * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_Q, Qp.data(), nsel * sizeof(void*), cudaMemcpyHostToDevice, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_n, ngs.data(), nsel * sizeof(int), cudaMemcpyHostToDevice, ctx->stream), "copy");
    CUDA_OR_FAIL(cudaMemcpyAsync(base + off_e, ed.data(), (nbin + 1) * sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
                 "copy");
    CUDA_OR_FAIL(qcx_launch_bin(ctx, nsel, reinterpret_cast<const double* const*>(base + off_L),
                                reinterpret_cast<const double* const*>(base + off_Q),
                                reinterpret_cast<const int*>(base + off_n), nw, which, nbin,
                                reinterpret_cast<const double*>(base + off_e), reinterpret_cast<double*>(base + off_o),
                                reinterpret_cast<double*>(base + off_c)),
                 "bin kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_L, base + off_o, (size_t)nbin * nw * sizeof(double)), "copy out");
    if (out_count) CUDA_OR_FAIL(qcx_copy_out(ctx, out_count, base + off_c, nbin * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

qcx_status qcx_rate(qcx_ctx* ctx, int nqbin, const double* qbin, int nw, const double* w, const double* L,
                    const qcx_halo_params* params, double* out_dRdw, int nQ, double* out_dRQ) {
    if (!ctx) return QCX_ERR_ARG;
    ctx->err.clear();
    if (nqbin < 2 || nw < 2 || !qbin || !w || !L || !params || !out_dRdw || nQ < 0 || (nQ > 0 && !out_dRQ))
        return ctx->fail(QCX_ERR_ARG, "rate: bad arguments");
    const qcx_halo_params& p = *params;
    if (!(p.m_chi_eV > 0) || !(p.v0_kms > 0) || !(p.vesc_kms > 0) || !(p.vE_kms > 0) || !(p.rho_T_g_cm3 > 0) ||
        !(p.w_pp_eV > 0))
        return ctx->fail(QCX_ERR_ARG, "rate: non-physical halo parameters");
    cudaSetDevice(ctx->device);
    const size_t oq = 0, ow = nqbin * sizeof(double), oL = ow + nw * sizeof(double);
    const size_t oR = oL + (size_t)nqbin * nw * sizeof(double), oQ = oR + nw * sizeof(double);
    const size_t total = oQ + (nQ > 0 ? nQ : 1) * sizeof(double);
    CUDA_OR_FAIL(ctx->scratch2.ensure(total), "alloc");
    char* base = ctx->scratch2.as<char>();
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oq, qbin, nqbin * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + ow, w, nw * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_copy_in(ctx, base + oL, L, (size_t)nqbin * nw * sizeof(double)), "copy");
    CUDA_OR_FAIL(qcx_launch_rate(ctx, nqbin, reinterpret_cast<double*>(base + oq), nw,
                                 reinterpret_cast<double*>(base + ow), reinterpret_cast<double*>(base + oL), p,
                                 reinterpret_cast<double*>(base + oR), nQ, reinterpret_cast<double*>(base + oQ)),
                 "rate kernel");
    CUDA_OR_FAIL(qcx_copy_out(ctx, out_dRdw, base + oR, nw * sizeof(double)), "copy out");
    if (nQ > 0) CUDA_OR_FAIL(qcx_copy_out(ctx, out_dRQ, base + oQ, nQ * sizeof(double)), "copy out");
    CUDA_OR_FAIL(cudaStreamSynchronize(ctx->stream), "sync");
    return QCX_OK;
}

}  // extern "C"
