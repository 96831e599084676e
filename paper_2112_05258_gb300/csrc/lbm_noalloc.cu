// lbm_boundary_flux_noalloc: the boundary-flow and mean-pressure reduction
// of a 0D-coupled boundary as a stand-alone call that allocates no memory.
//
// Who needs it: callers that must not allocate device memory at the point of
// the call -- a host application whose device memory is owned by its own
// pool or framework allocator (allocating behind its back fragments or
// exceeds its budget), or code running inside a region where cudaMalloc
// would synchronise the device or is forbidden (latency-critical coupling
// loops of an external 0D solver).  They pass their own input and output
// buffers; the only scratch this reduction needs -- one pair of FP64 partial
// sums per 256-cell chunk -- lives in a fixed file-scope device array that
// every GPU loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "../../include/lbm.h"

namespace {

constexpr int NA_CHUNK = 256;          // cells per CTA of the partial-sum pass
constexpr int NA_MAX_CHUNKS = 4096;    // scratch capacity: 4096 chunks = 1,048,576 cells
constexpr int NA_MAX_DEVICES = 64;

// Scratch: partial sums {sum n.j / sum f, sum P} per chunk (64 KiB per device).
static __device__ __align__(256) double g_flux_scratch[2 * NA_MAX_CHUNKS];

std::mutex g_mu;
double *g_scratch_addr[NA_MAX_DEVICES] = {};

__global__ void __launch_bounds__(NA_CHUNK) k_flux_partials(const double *__restrict__ P,
                                                            const double *__restrict__ jn,
                                                            const int32_t *__restrict__ cells, int64_t n,
                                                            double *__restrict__ scratch) {
    __shared__ double sQ[NA_CHUNK], sP[NA_CHUNK];
    const int64_t k = (int64_t)blockIdx.x * NA_CHUNK + threadIdx.x;
    double q = 0.0, p = 0.0;
    if (k < n) {
        const int32_t c = cells[k];
        const double Pc = P[c];
        q = jn[c] / (3.0 * Pc);  // n.j / sum f with sum f = P / c_s^2
        p = Pc;
    }
    sQ[threadIdx.x] = q;
    sP[threadIdx.x] = p;
    __syncthreads();
    for (int s = NA_CHUNK / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sQ[threadIdx.x] += sQ[threadIdx.x + s];
            sP[threadIdx.x] += sP[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = sQ[0];
        scratch[2 * blockIdx.x + 1] = sP[0];
    }
}

__global__ void k_flux_finish(const double *__restrict__ scratch, int nchunks, int64_t n, double *out) {
    double q = 0.0, p = 0.0;
    for (int k = threadIdx.x; k < nchunks; k += 32) {
        q += scratch[2 * k];
        p += scratch[2 * k + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        q += __shfl_xor_sync(0xffffffffu, q, o);
        p += __shfl_xor_sync(0xffffffffu, p, o);
    }
    if (threadIdx.x == 0) {
        out[0] = q;
        out[1] = p / (double)n;
    }
}

}  // namespace

extern "C" lbm_status lbm_boundary_flux_noalloc(const double *P, const double *j_normal, const int32_t *cells,
                                                int64_t n_cells, double *out, void *stream) {
    if (!P || !j_normal || !cells || !out) {
        fprintf(stderr, "lbm_boundary_flux_noalloc: null pointer argument\n");
        return LBM_ERR_ARG;
    }
    if (n_cells < 1 || n_cells > (int64_t)NA_CHUNK * NA_MAX_CHUNKS) {
        fprintf(stderr, "lbm_boundary_flux_noalloc: n_cells = %lld outside [1, %lld] (fixed scratch of %d chunks)\n",
                (long long)n_cells, (long long)NA_CHUNK * NA_MAX_CHUNKS, NA_MAX_CHUNKS);
        return LBM_ERR_ARG;
    }
    // an error left by earlier, unrelated work is reported as such (and left
    // pending for the caller), not mistaken for a failure of this call's launches
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_boundary_flux_noalloc: an earlier CUDA error is pending (%s); nothing launched\n",
                cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    int dev = -1;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        fprintf(stderr, "lbm_boundary_flux_noalloc: no usable current device (%s)\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    double *scratch = nullptr;
    {
        // once per device, with that device current: the device address of the
        // static scratch array (its name is only a host-side stand-in).  The
        // address is kept for the life of the process; a device reset or a new
        // primary context on that device makes it stale.
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_flux_scratch);
            if (e != cudaSuccess || !ptr) {
                fprintf(stderr, "lbm_boundary_flux_noalloc: cudaGetSymbolAddress failed (%s)\n", cudaGetErrorString(e));
                return LBM_ERR_CUDA;
            }
            g_scratch_addr[dev] = static_cast<double *>(ptr);
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nchunks = (int)((n_cells + NA_CHUNK - 1) / NA_CHUNK);
    k_flux_partials<<<nchunks, NA_CHUNK, 0, s>>>(P, j_normal, cells, n_cells, scratch);
    k_flux_finish<<<1, 32, 0, s>>>(scratch, nchunks, n_cells, out);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        fprintf(stderr, "lbm_boundary_flux_noalloc: launch failed (%s)\n", cudaGetErrorString(e));
        return LBM_ERR_CUDA;
    }
    return LBM_OK;
}
