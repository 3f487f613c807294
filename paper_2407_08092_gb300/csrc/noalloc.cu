// lq_norm2_noalloc: the squared norm of a natural complex-double field, for
// callers that must not allocate device memory.
//
// It is the same two-stage deterministic reduction as lq_norm2 (per-block
// partial sums, then one block summing the partials in a fixed order), but its
// scratch is a file-scope static device array instead of memory owned by a
// context, and it needs no context at all.  Callers that cannot call
// cudaMalloc -- for instance code that runs inside a fixed device-memory budget
// handed out by another framework's pool, where an extra allocation could fail
// or implicitly synchronise the device at the wrong moment -- can use it with
// only their own input and output buffers.
//
// The paper has no counterpart of this entry point; it is a service of the
// library, not a step of the method.
#include <mutex>

#include "../../include/lqdd.h"
#include "lq_kernels.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 32;                                    // complex values per thread
constexpr long long NA_CHUNK = (long long)NA_THREADS * NA_PER_THREAD; // complex values per block
constexpr int NA_MAX_BLOCKS = 4096;                                  // 32 KiB of partial sums

static_assert((long long)NA_MAX_BLOCKS * NA_CHUNK / 12 == LQ_NORM2_NOALLOC_MAX_SITES,
              "header limit must match the scratch size");

}  // namespace

// The shared scratch: one partial sum per block.  Every GPU on which the
// library's module is loaded (under lazy module loading: by the first call on
// that device) holds these 32 KiB until the process exits.  In host code this name
// is only a host-side stand-in, so the host passes the device address obtained
// from cudaGetSymbolAddress instead.
static __device__ __align__(256) double lq_noalloc_scratch[NA_MAX_BLOCKS];

__global__ void __launch_bounds__(NA_THREADS) na_partial_kernel(const double2 *__restrict__ v, long long n,
                                                               double *partial)
{
    __shared__ double sh[NA_THREADS / 32];
    const long long base = blockIdx.x * NA_CHUNK;
    double acc = 0.0;
#pragma unroll 8
    for (int k = 0; k < NA_PER_THREAD; k++) {
        const long long i = base + (long long)k * NA_THREADS + threadIdx.x;
        if (i < n) {
            const double2 t = __ldg(v + i);
            acc += t.x * t.x + t.y * t.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < NA_THREADS / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = acc;   // every slot this call reads is written here
    }
}

__global__ void __launch_bounds__(NA_THREADS) na_finish_kernel(const double *__restrict__ partial, int nblocks,
                                                              double *out)
{
    __shared__ double sh[NA_THREADS / 32];
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) acc += partial[b];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = threadIdx.x < NA_THREADS / 32 ? sh[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *out = acc;
    }
}

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
double *na_scratch[NA_MAX_DEVICES] = {nullptr};

// Device address of the scratch array on the current device, looked up once
// per device (with that device current) and cached.
cudaError_t scratch_address(int dev, double **ptr)
{
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, lq_noalloc_scratch);
        if (e != cudaSuccess) return e;
        na_scratch[dev] = (double *)p;
    }
    *ptr = na_scratch[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lq_status lq_norm2_noalloc(const void *v, long long n_sites, double *out, void *stream)
{
    if (!out || n_sites < 0 || (n_sites > 0 && !v)) return LQ_ERR_ARG;
    if (n_sites > LQ_NORM2_NOALLOC_MAX_SITES) return LQ_ERR_ARG;
    // A launch error left on this host thread by earlier work would otherwise be
    // read (and cleared) by the check after our own launches: report it as
    // LQ_ERR_CUDA before launching anything, and leave it in place for its owner.
    if (cudaPeekAtLastError() != cudaSuccess) return LQ_ERR_CUDA;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return LQ_ERR_CUDA;
    }
    double *scratch = nullptr;
    if (scratch_address(dev, &scratch) != cudaSuccess) {
        cudaGetLastError();
        return LQ_ERR_CUDA;
    }
    const long long n = n_sites * 12;
    const int nblocks = (int)((n + NA_CHUNK - 1) / NA_CHUNK);
    cudaStream_t st = (cudaStream_t)stream;
    if (nblocks > 0) na_partial_kernel<<<nblocks, NA_THREADS, 0, st>>>((const double2 *)v, n, scratch);
    na_finish_kernel<<<1, NA_THREADS, 0, st>>>(scratch, nblocks, out);
    if (cudaGetLastError() != cudaSuccess) return LQ_ERR_CUDA;
    return LQ_OK;
}
