// Allocation-free inverse diagonal of caller-owned dielectric matrices.
//
// Some callers cannot allocate device memory when they need this result: a
// framework that owns the device allocator and forbids other libraries from
// calling cudaMalloc (cudaMalloc also synchronises the device, which a
// latency-sensitive or graph-replayed pipeline cannot afford), or a process
// that reserved its whole memory budget at start-up.  qcx_eps_inverse_diag_noalloc
// serves them: the caller passes device inputs and outputs, and the only
// scratch (the per-matrix work copies of the Gauss-Jordan elimination) lives in
// a file-scope device array of fixed size.  A device reserves it when it loads
// this file's code (with CUDA's lazy module loading: at the entry point's first
// call there) and keeps it until the process exits.
#include "qcx_internal.h"
#include "cplx.cuh"

#include <mutex>

namespace {

constexpr int NA_THREADS = 256;
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)16 << 20;   // 16 MiB
constexpr int MAX_DEVICES = 64;

// The scratch: in host code this name is only a stand-in, never a device
// address; host code uses the address resolved by cudaGetSymbolAddress.
static __device__ __align__(256) double2 g_noalloc_scratch[NOALLOC_SCRATCH_BYTES / sizeof(double2)];

std::mutex g_setup_mutex;
void* g_scratch_addr[MAX_DEVICES] = {nullptr};

// Gauss-Jordan with partial pivoting on a work copy in the scratch, FP64.
// Writes diag(eps^-1), -Im diag(eps^-1) and -Im(1/eps_GG) and a singular flag.
__global__ void __launch_bounds__(NA_THREADS)
    k_gj_noalloc(int n, const double2* eps, double2* scratch, double2* diag_inv, double* L_lfe, double* L_nolfe,
                 int* flags) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* rowk = reinterpret_cast<double2*>(smem_raw);
    double2* colk = rowk + n;
    int* piv = reinterpret_cast<int*>(colk + n);
    int* idx = piv + n;
    __shared__ double red_v[NA_THREADS / 32];
    __shared__ int red_i[NA_THREADS / 32];
    __shared__ int s_p, s_bad;
    const int b = blockIdx.x;
    const double2* A = eps + (size_t)b * n * n;
    double2* X = scratch + (size_t)b * n * n;
    // the work copy is fully overwritten here, so no part of the scratch needs clearing
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        const double2 z = A[e];
        X[e] = z;
        const int i = e / n;
        if (e == i * n + i && L_nolfe) L_nolfe[(size_t)b * n + i] = z.y / (z.x * z.x + z.y * z.y);
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        double best = -1.0;
        int bi = n;
        for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
            const double2 z = X[(size_t)i * n + k];
            const double v = z.x * z.x + z.y * z.y;
            if (v > best) {
                best = v;
                bi = i;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            const double ov = __shfl_down_sync(0xffffffffu, best, o);
            const int oi = __shfl_down_sync(0xffffffffu, bi, o);
            if (ov > best || (ov == best && oi < bi)) {
                best = ov;
                bi = oi;
            }
        }
        if ((threadIdx.x & 31) == 0) {
            red_v[threadIdx.x >> 5] = best;
            red_i[threadIdx.x >> 5] = bi;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double bv = red_v[0];
            int bix = red_i[0];
            for (int w = 1; w < NA_THREADS / 32; ++w)
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
        if (p != k) {
            for (int j = threadIdx.x; j < n; j += blockDim.x) {
                const double2 t = X[(size_t)k * n + j];
                X[(size_t)k * n + j] = X[(size_t)p * n + j];
                X[(size_t)p * n + j] = t;
            }
            __syncthreads();
        }
        const double2 pv = X[(size_t)k * n + k];
        const double d = 1.0 / (pv.x * pv.x + pv.y * pv.y);
        const double2 inv = make_double2(pv.x * d, -pv.y * d);
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const double2 v = (j == k) ? make_double2(1.0, 0.0) : X[(size_t)k * n + j];
            rowk[j] = cmul(v, inv);
            colk[j] = (j == k) ? make_double2(0.0, 0.0) : X[(size_t)j * n + k];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) X[(size_t)k * n + j] = rowk[j];
        for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
            const int i = e / n, j = e - i * n;
            if (i == k) continue;
            const double2 f = colk[i];
            double2 x = (j == k) ? make_double2(0.0, 0.0) : X[e];
            x.x -= f.x * rowk[j].x - f.y * rowk[j].y;
            x.y -= f.x * rowk[j].y + f.y * rowk[j].x;
            X[e] = x;
        }
        __syncthreads();
    }
    if (s_bad) {
        if (threadIdx.x == 0 && flags) flags[b] = 1;
        // every output of a singular matrix is zero (its diagonal may itself be zero, so the
        // no-LFE values written above are replaced as well)
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            diag_inv[(size_t)b * n + j] = make_double2(0.0, 0.0);
            if (L_lfe) L_lfe[(size_t)b * n + j] = 0.0;
            if (L_nolfe) L_nolfe[(size_t)b * n + j] = 0.0;
        }
        return;
    }
    if (threadIdx.x == 0) {
        if (flags) flags[b] = 0;
        for (int c = 0; c < n; ++c) idx[c] = c;
        for (int k = n - 1; k >= 0; --k) {
            const int t = idx[k];
            idx[k] = idx[piv[k]];
            idx[piv[k]] = t;
        }
    }
    __syncthreads();
    // diagonal of the inverse: its column j is the work copy's column idx[j]
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 z = X[(size_t)j * n + idx[j]];
        diag_inv[(size_t)b * n + j] = z;
        if (L_lfe) L_lfe[(size_t)b * n + j] = -z.y;
    }
}

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" qcx_status qcx_eps_inverse_diag_noalloc(const qcx_c64* eps, int nb, int n, qcx_c64* out_diag_inv,
                                                   double* out_L_lfe, double* out_L_nolfe, int* out_singular,
                                                   void* cuda_stream) {
    if (nb < 1 || n < 1 || n > 4096 || !eps || !out_diag_inv) return QCX_ERR_ARG;
    if ((size_t)nb * n * n * sizeof(double2) > NOALLOC_SCRATCH_BYTES) return QCX_ERR_ARG;   // over the fixed scratch
    if (!on_device(eps) || !on_device(out_diag_inv) || (out_L_lfe && !on_device(out_L_lfe)) ||
        (out_L_nolfe && !on_device(out_L_nolfe)) || (out_singular && !on_device(out_singular)))
        return QCX_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return QCX_ERR_CUDA;
    }
    void* scratch = nullptr;
    {
        // once per device, with that device current: resolve the device address of the array
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return QCX_ERR_CUDA;
            }
            g_scratch_addr[dev] = p;
        }
        scratch = g_scratch_addr[dev];
    }
    const size_t smem = (size_t)n * 2 * sizeof(double2) + (size_t)n * 2 * sizeof(int);
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute((const void*)k_gj_noalloc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
        cudaGetLastError();
        return QCX_ERR_CUDA;
    }
    k_gj_noalloc<<<nb, NA_THREADS, smem, (cudaStream_t)cuda_stream>>>(
        n, reinterpret_cast<const double2*>(eps), reinterpret_cast<double2*>(scratch),
        reinterpret_cast<double2*>(out_diag_inv), out_L_lfe, out_L_nolfe, out_singular);
    if (cudaGetLastError() != cudaSuccess) return QCX_ERR_CUDA;
    return QCX_OK;
}
