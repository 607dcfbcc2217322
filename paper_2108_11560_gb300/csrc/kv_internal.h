// Shared host-side helpers of the library's translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/kv.h"

namespace kvh {

// Records a CUDA error string for kv_last_cuda_error() and returns KV_ERR_CUDA.
int cuda_fail(cudaError_t e);

// Number of SMs of the current device (cached per device).
int sm_count();

// Stream-ordered scratch memory (fallback lists, staging buffers, partial sums) from a pool of
// the library's own on the current device.  Its release threshold keeps freed memory reserved
// for the next call: a call that synchronizes (the host-buffer call) would otherwise see the
// default pool hand its memory back at every synchronization and map it again on the next call.
// kv_trim_memory() releases it.
cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s);
cudaError_t scratch_free(void* p, cudaStream_t s);
// The pool of the current device, or nullptr if none was created yet.
cudaError_t scratch_pool_get(cudaMemPool_t* pool);

inline bool aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline size_t elem_size(int dtype) { return dtype == KV_F64 ? 8 : 4; }

#define KV_CUDA_TRY(expr)                          \
    do {                                           \
        cudaError_t kv_e_ = (expr);                \
        if (kv_e_ != cudaSuccess) return kvh::cuda_fail(kv_e_); \
    } while (0)

// Counts one kernel launch (kv_launch_count) and checks it.
void note_launch();
#define KV_LAUNCH_CHECK()     \
    do {                      \
        kvh::note_launch();   \
        KV_CUDA_TRY(cudaGetLastError()); \
    } while (0)

// The learned-bracket network as the kernels see it (device pointers owned by the handle).
struct MlpView {
    const float* w1;            // [64][2]  FP32
    const float* b1;            // [64]
    const unsigned short* w2h;  // [64][64] BF16 bits (row = output unit)
    const float* b2;            // [64]
    const float* w3;            // [2][64]
    const float* b3;            // [2]
    float in_scale[4];          // a = asinh(v * in_scale[0]) * in_scale[1], b = log x * in_scale[2] + in_scale[3]
    float out_scale[4];         // log half-widths L_k = y_k * out_scale[2k] + out_scale[2k+1]
};

// Fills a view of the handle's inference weights; returns KV_OK or KV_ERR_HANDLE.
int mlp_view(const kv_mlp* h, MlpView* out);

// Launches the learned-bracket kernels (kv_mlp.cu).  Arguments are already validated.
// `scratch`: NULL, or device memory for n + 32 uint32 (the fallback list), reused across calls
// on the same stream; NULL allocates it on the stream for this call.
int launch_mlp_path(const kv_args* a, int bins, double log_eps, int max_iter, uint32_t* scratch);

// kv_fwd_bwd_ex with an optional preallocated learned-path scratch (see launch_mlp_path).
int fwd_bwd_ex(const kv_args* a, uint32_t* scratch);

}  // namespace kvh
