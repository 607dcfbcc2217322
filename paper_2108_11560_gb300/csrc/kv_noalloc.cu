// kv_sum_noalloc: the deterministic sum of kv_sum without any device allocation.
//
// kv_sum takes its per-block partial sums from a stream-ordered allocation on every call.  This
// variant keeps them in a file-scope device array instead, sized for KV_SUM_NOALLOC_MAX_N
// elements, so a call allocates nothing.  Every GPU that loads the library holds the array (128 KiB)
// until the process exits.  All calls on a device share it: calls whose work overlaps on the GPU
// (different streams without ordering between them) race on it and must be serialised by the
// caller.  The partial sums are fully overwritten by each call, so nothing needs clearing.
// The array's device address is looked up once per device and kept for the life of the process:
// a cudaDeviceReset, or anything else that destroys the device's primary context, invalidates it,
// so the entry point must not be used on a device after such a reset.
#include <cuda_runtime.h>

#include <mutex>

#include "kv_internal.h"

constexpr int kElemsPerPartial = 4096;
constexpr int kPartialsMax = KV_SUM_NOALLOC_MAX_N / kElemsPerPartial;

// The scratch: one double per kElemsPerPartial input elements (16384 doubles, 128 KiB).  In host
// code this name is only a stand-in; kernels get its device address from scratch_address().
static __device__ __align__(256) double g_sum_scratch[kPartialsMax];

namespace {

constexpr int kThreads = 256;
constexpr int kMaxDevices = 64;

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// The device address of the scratch array on the current device, looked up once per device.
int scratch_address(double** out)
{
    int dev = 0;
    KV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return KV_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        KV_CUDA_TRY(cudaGetSymbolAddress(&p, g_sum_scratch));
        g_scratch_ptr[dev] = (double*)p;
    }
    *out = g_scratch_ptr[dev];
    return KV_OK;
}

// partial_sums and final_sum repeat kv_sum's two kernels (kv_sum_partial and kv_sum_final in
// kv_core.cu) with the same block size, per-block stride and reduction order; with the same
// number of blocks (every n up to 4,194,304 elements, where kv_sum uses one block per 4096) the
// two entry points give the same bits.  A change to either pair must be made to both.
template <typename T>
__global__ void __launch_bounds__(kThreads) partial_sums(const T* a, int64_t n, double* part)
{
    // block b takes elements b*256 + t, then every (grid * 256)-th one after: about
    // kElemsPerPartial elements per block, interleaved for coalesced loads
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kThreads)
        acc += (double)a[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kThreads) final_sum(const double* part, int nb, double* out)
{
    __shared__ double sh[kThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

}  // namespace

extern "C" int kv_sum_noalloc(const void* a, int64_t n, int dtype, double* out, void* stream)
{
    if (dtype != KV_F64 && dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0 || n > KV_SUM_NOALLOC_MAX_N) return KV_ERR_SIZE;
    if (!out || (n > 0 && !a)) return KV_ERR_NULL;
    if (!kvh::aligned(out, 8) || (a && !kvh::aligned(a, kvh::elem_size(dtype)))) return KV_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    double* part = nullptr;
    int rc = scratch_address(&part);
    if (rc != KV_OK) return rc;
    if (n == 0) {
        final_sum<<<1, kThreads, 0, s>>>(part, 0, out);
        KV_LAUNCH_CHECK();
        return KV_OK;
    }
    const int nb = (int)((n + kElemsPerPartial - 1) / kElemsPerPartial);
    if (dtype == KV_F64)
        partial_sums<double><<<nb, kThreads, 0, s>>>((const double*)a, n, part);
    else
        partial_sums<float><<<nb, kThreads, 0, s>>>((const float*)a, n, part);
    KV_LAUNCH_CHECK();
    final_sum<<<1, kThreads, 0, s>>>(part, nb, out);
    KV_LAUNCH_CHECK();
    return KV_OK;
}
