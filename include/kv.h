/*
 * kv.h -- batched log K_v(x), d/dv log K_v(x) and d/dx log K_v(x) on one GPU.
 *
 * The method is the fixed-bin integration of Takekawa, "Fast parallel calculation of modified
 * Bessel function of the second kind and its derivatives" (arXiv 2108.11560):
 *   K_v(x) = int_0^inf f(t) dt,  f(t) = cosh(vt) exp(-x cosh t)                 (Sec. 2, Eq. 1-2)
 * Each pair brackets the peak t_p of g = log f (Sec. 2.2, Algorithms 1-2), finds the range
 * [t0, t1] where f >= eps f(t_p) (Sec. 2.3), and sums a fixed number of trapezoid bins relative
 * to the peak (Sec. 2.4, Eq. int; Algorithm 3).  The derivatives integrate t sinh(vt) e^{-x cosh t}
 * and -cosh(t) cosh(vt) e^{-x cosh t} over the same bins (Sec. 4.1), each divided by the K sum.
 *
 * Conventions for every entry point below
 *   - Arrays are structure-of-arrays, n contiguous elements each, caller-owned DEVICE memory
 *     (except kv_fwd_bwd_host and kv_fwd_bwd_host_ex, which take host memory).  The library
 *     never keeps a pointer after the call's work on `stream` has finished.
 *   - Element type is set by `dtype`: KV_F64 -> double for inputs and outputs;
 *     KV_MIXED -> float for inputs and outputs.  Pointers must be aligned to the element size.
 *   - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *     asynchronous on that stream; argument errors are detected on the host before any launch.
 *   - n == 0 is a valid no-op.  Output pointers may alias nothing else.
 *   - Scratch device memory a call needs (the learned path's fallback list, 4 bytes per pair;
 *     the host call's staging buffers; partial sums) is allocated stream-ordered on `stream` from
 *     a memory pool of the library's own on the current device and freed to it before the call's
 *     work ends.  The pool keeps freed memory reserved for later calls (a synchronizing call would
 *     otherwise return it to the system and map it again each time); kv_trim_memory() releases it.
 *   - Return value: KV_OK (0) or a negative kv_status; kv_strerror() describes it.
 *
 * Per-pair domain results (no error code; Sec. 2 defines K for v real, x > 0):
 *   v < 0: uses |v| (K_{-v} = K_v) and negates d/dv.   v = 0: d/dv is exactly 0.
 *   x = 0: log K = +inf, d/dv = +-inf (0 if v = 0), d/dx = -inf.
 *   x = +inf: log K = -inf, d/dv = +-0, d/dx = -1.    |v| = inf, finite x > 0: +inf, +-inf, -inf.
 *   x < 0 or NaN in v or x: NaN in every output.
 */
#ifndef KV_H_
#define KV_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Arithmetic of the path (the `dtype` argument). */
enum kv_dtype {
    /* Everything in FP64: the paper's bracket (Algorithms 1-3) and the bins.  I/O double.
     * Default eps: 2^-52 (machine epsilon, Sec. 2.1).  Default bins: 128. */
    KV_F64 = 0,
    /* Peak and log-offset g(t_p) in extended precision, bins in FP32 relative to the peak,
     * with compensated sums.  I/O float.  Default eps: e^-20.  Default bins: 40 (32 suffice for
     * x >= 1e-3; the corner of small v and x < 1e-4 needs 40 for 2e-6 in d/dx). */
    KV_MIXED = 1
};

/* How the range [t0, t1] is found (kv_args.bracket). */
enum kv_bracket_mode {
    /* Algorithms 1-3 in FP64 (Sec. 2.2-2.3). */
    KV_BRACKET_PLAIN = 0,
    /* A 2-64-64-2 MLP on (v, log x) predicts (t0, t1); each pair checks g at both ends and falls
     * back to the plain bracket (in FP32, then FP64) when the check fails.  KV_MIXED only.
     * Needs kv_args.mlp. */
    KV_BRACKET_MLP = 1,
    /* Algorithms 1-3 in FP32 (the 32-bit variant of Sec. 4.2), with the range functions evaluated
     * as cancellation-free differences about a grid point next to the peak and the offset as a
     * float-float (no FP64 on the path); pairs whose FP32 range is not finite fall back to FP64.
     * KV_MIXED only. */
    KV_BRACKET_PLAIN_F32 = 2
};

/* Status codes. */
enum kv_status {
    KV_OK = 0,
    KV_ERR_NULL = -1,    /* a required pointer is NULL */
    KV_ERR_SIZE = -2,    /* n < 0, or a size limit exceeded */
    KV_ERR_BINS = -3,    /* bins < 1 or bins > KV_MAX_BINS */
    KV_ERR_DTYPE = -4,   /* unknown dtype, or a mode not available for this dtype */
    KV_ERR_ALIGN = -5,   /* a pointer is not aligned to its element size */
    KV_ERR_CUDA = -6,    /* a CUDA runtime call or launch failed (see kv_last_cuda_error) */
    KV_ERR_ARG = -7,     /* another argument is out of range (log_eps >= 0, max_iter < 1, ...) */
    KV_ERR_HANDLE = -8,  /* a NULL or invalid MLP handle */
    KV_ERR_IO = -9,      /* a checkpoint file could not be opened, read or written */
    KV_ERR_FORMAT = -10, /* a checkpoint file has the wrong magic, version or sizes */
    KV_ERR_NOMEM = -11   /* a device or host allocation failed */
};

#define KV_MAX_BINS 4096
/* FindZero iterations (Algorithm 2: max_iter = 10). */
#define KV_DEFAULT_MAX_ITER 10

/* ------------------------------------------------------------------ the four core calls */

/* log K_v(x) for n pairs (Algorithm 3 with Eq. int).  bins = the fixed n of Sec. 2.4. */
int kv_log(const void* v, const void* x, void* logk, int64_t n, int bins, int dtype, void* stream);

/* d/dv log K_v(x) (Sec. 4.1: integral of t sinh(vt) e^{-x cosh t} divided by K). */
int kv_log_dv(const void* v, const void* x, void* dlogk_dv, int64_t n, int bins, int dtype,
              void* stream);

/* d/dx log K_v(x) (Sec. 4.1: integral of -cosh(t) cosh(vt) e^{-x cosh t} divided by K). */
int kv_log_dx(const void* v, const void* x, void* dlogk_dx, int64_t n, int bins, int dtype,
              void* stream);

/* All three from one pass over the bins (one bracket per pair, reused by both derivatives). */
int kv_fwd_bwd(const void* v, const void* x, void* logk, void* dv, void* dx, int64_t n, int bins,
               int dtype, void* stream);

/* ------------------------------------------------------------------ the extended call */

typedef struct kv_mlp kv_mlp; /* opaque learned-bracket network, see below */

typedef struct kv_args {
    const void* v;        /* [n] orders */
    const void* x;        /* [n] arguments */
    void* logk;           /* [n] out, or NULL */
    void* dv;             /* [n] out, or NULL */
    void* dx;             /* [n] out, or NULL (at least one of logk, dv, dx is non-NULL) */
    const void* grad_out; /* [n] or NULL: if set, dv and dx are multiplied by it (fused backward) */
    int64_t n;
    int bins;             /* 0 = the dtype's default */
    int dtype;            /* enum kv_dtype */
    int bracket;          /* enum kv_bracket_mode */
    double log_eps;       /* log of the range's eps (< 0); 0 = the dtype's default */
    int max_iter;         /* FindZero iterations; 0 = KV_DEFAULT_MAX_ITER */
    int lanes;            /* lanes that share one pair's bins on the FP64-bracket paths (1, 2, 4, 8,
                           * 16, 32): every lane brackets its own pair, then groups of `lanes`
                           * lanes sum the pairs' bins in `lanes` rounds; 0 = automatic (1) */
    const kv_mlp* mlp;    /* network for KV_BRACKET_MLP, else ignored */
    uint8_t* status;      /* [n] or NULL: per-pair kv_pair_status bits */
    unsigned long long* fallback_count; /* device counter or NULL: += pairs that fell back */
    void* stream;
    /* Second derivatives of log K (Sec. 4.1, the integrands f^(n,m) with n + m = 2, over the same
     * bins and range): [n] outs or NULL, same element type as v and x.  d2v = d2/dv2,
     * dvx = d2/dv dx (odd in v, 0 at v = 0), d2x = d2/dx2.  When any is set, every pair runs one
     * per thread (lanes is ignored) and logk/dv/dx, if requested, come from the same sums;
     * grad_out does not scale them.  Edge pairs: x = +inf gives 0, the other edge inputs NaN. */
    void* d2v;
    void* dvx;
    void* d2x;
    int flags;            /* enum kv_flag bits; 0 = the paper's algorithms throughout */
} kv_args;

/* Options of kv_fwd_bwd_ex (kv_args.flags).  Unknown bits give KV_ERR_ARG. */
enum kv_flag {
    /* Not in the paper: the FP64 bracket's peak search (Sec. 2.2) skips Algorithm 1's doublings
     * and runs Algorithm 2 on the analytic bracket [0, asinh(v/x)] (g'(0) = 0, and
     * g'(asinh(v/x)) = v tanh(vt) - v < 0), falling back to the doublings where g' is not
     * negative there in rounded arithmetic.  Applies wherever the plain FP64 bracket runs
     * (KV_BRACKET_PLAIN, and the learned path's FP64 fallback); kv_bracket() always follows
     * Algorithms 1-3.  The peak then differs from Algorithms 1-2's within their convergence, which
     * moves the results only at the level of the method's own error. */
    KV_FLAG_PEAK_ANALYTIC_START = 1
};

/* Per-pair status bits written to kv_args.status. */
enum kv_pair_status {
    KV_PAIR_OK = 0,
    KV_PAIR_EDGE = 1,        /* the pair is a domain edge case (see the list at the top) */
    KV_PAIR_FALLBACK = 2,    /* the learned bracket failed its check; the plain one was used */
    KV_PAIR_RANGE_CAP = 4    /* FindRange hit its doubling cap (input far outside any use) */
};

/* The general form of kv_fwd_bwd: bracket mode, eps, iteration count, lanes per pair,
 * optional fused gradient epilogue, per-pair status and fallback counter. */
int kv_fwd_bwd_ex(const kv_args* a);

/* How kv_fwd_bwd_host_ex moves the data between host and device. */
enum kv_host_transfer {
    /* DIRECT when every buffer is device-addressable host memory (see DIRECT) and the device
     * reaches host memory over a coherent link (native host atomics or host page-table access,
     * as on NVLink-C2C Grace systems: kv_host_direct_supported() == 1), else STAGED. */
    KV_HOST_AUTO = 0,
    /* Copies through device buffers: chunks of up to 2^19 pairs pipelined over four buffer
     * slots (internal streams for the copies in, the copies out and each slot's kernels, ordered
     * by events and started after the work already on a->stream).  Device staging memory comes
     * from the library's scratch pool on a->stream.  Any host memory; pinned
     * (cudaHostAlloc) for full copy speed. */
    KV_HOST_STAGED = 1,
    /* No staging copies: the kernels read v and x from, and write the outputs to, the host
     * buffers themselves over the CPU-GPU link.  Every buffer must be page-locked host memory
     * mapped into the device's address space over its whole length (cudaHostAlloc /
     * cudaMallocHost under unified addressing, or cudaHostRegister with cudaHostRegisterMapped);
     * the call checks both ends of each buffer and returns KV_ERR_ARG otherwise, without
     * launching anything.  The fallback list of the learned path is device scratch memory on
     * a->stream. */
    KV_HOST_DIRECT = 2
};

/* kv_fwd_bwd_ex on HOST buffers: a->v, a->x, a->logk, a->dv and a->dx are host pointers; every
 * other field means what it means for kv_fwd_bwd_ex, except that grad_out, status,
 * fallback_count and the second-derivative outputs must be NULL (else KV_ERR_ARG), as must be a
 * `transfer` outside enum kv_host_transfer.  Returns when the host outputs are complete (the call
 * synchronizes a->stream). */
int kv_fwd_bwd_host_ex(const kv_args* a, int transfer);

/* kv_fwd_bwd_host_ex(a, KV_HOST_AUTO). */
int kv_fwd_bwd_host(const kv_args* a);

/* 1 if the current device reaches host memory over a coherent link (the condition under which
 * KV_HOST_AUTO picks DIRECT for device-addressable buffers), else 0. */
int kv_host_direct_supported(void);

/* ------------------------------------------------------------------ building blocks */

/* The plain bracket alone (Algorithms 1-3 through Sec. 2.3): per pair t0, t_p, t1 and the
 * offset g(t_p), all double, for any dtype of v and x.  Outputs may be NULL individually. */
int kv_bracket(const void* v, const void* x, double* t0, double* tp, double* t1, double* g_tp,
               int64_t n, int dtype, double log_eps, int max_iter, void* stream);

/* The backward epilogue on its own: grad_v = grad_out * dv, grad_x = grad_out * dx. */
int kv_grad(const void* grad_out, const void* dv, const void* dx, void* grad_v, void* grad_x,
            int64_t n, int dtype, void* stream);

/* The epilogue of the second backward pass (the backward of kv_grad's outputs
 * g_v = go * dv, g_x = go * dx with incoming gradients gg_v, gg_x):
 *   out_v  = go * (gg_v * d2v + gg_x * dvx)
 *   out_x  = go * (gg_v * dvx + gg_x * d2x)
 *   out_go = gg_v * dv + gg_x * dx
 * All pointers are [n] device arrays of the dtype's element type (gg_v or gg_x may be NULL for
 * zero); outputs may be NULL individually.  Errors as for kv_grad. */
int kv_grad2(const void* go, const void* gg_v, const void* gg_x, const void* dv, const void* dx,
             const void* d2v, const void* dvx, const void* d2x, void* out_v, void* out_x,
             void* out_go, int64_t n, int dtype, void* stream);

/* Deterministic sum of n elements (dtype's element type) into *out (one double, device memory).
 * Used for the log-likelihood sum_i log K(v_i, x_i).  Scratch memory for the per-block partial
 * sums comes from the library's scratch pool on `stream` (stream-ordered allocation). */
int kv_sum(const void* a, int64_t n, int dtype, double* out, void* stream);

/* The same deterministic sum for callers that cannot allocate device memory: applications whose
 * device memory is all reserved up front (a framework's caching allocator, or a fixed memory
 * budget), so that an allocation inside a library call would fail or would take memory the
 * caller has promised elsewhere.  The paper has no counterpart; this is a property of the
 * library, not of the method.
 *   - The partial sums live in a device array inside this library, sized for at most
 *     KV_SUM_NOALLOC_MAX_N elements (128 KiB, held on every GPU that loads the library until the
 *     process exits).  n > KV_SUM_NOALLOC_MAX_N returns KV_ERR_SIZE before any GPU work.
 *   - The call allocates and frees nothing.  Its first call on a device looks up the array's
 *     device address (cudaGetSymbolAddress), once per device; make that first call before any
 *     stream capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset (or anything else that destroys the device's primary context) this entry
 *     point must not be called on that device again.
 *   - All calls on a device share the array: calls whose work can overlap on the GPU (streams
 *     with no ordering between them) race on it, so the caller must order them.  Each call
 *     overwrites the partial sums it uses, so nothing needs clearing between calls.
 * Arguments, result and errors are otherwise those of kv_sum; for n up to 4,194,304 the
 * reduction order, and so the result, is the same as kv_sum's. */
#define KV_SUM_NOALLOC_MAX_N 67108864
int kv_sum_noalloc(const void* a, int64_t n, int dtype, double* out, void* stream);

/* ------------------------------------------------------------------ the learned bracket */
/* A 2-64-64-2 MLP on (v, log x) -> (t0, t1) with ReLU hidden units; FP32 master weights for
 * training, BF16 copies for inference with FP32 accumulation.  A handle owns its device memory. */

/* New network with seeded random weights on the current device. */
int kv_mlp_create(uint64_t seed, kv_mlp** out);
/* Releases the handle and its device memory (NULL is a no-op). */
int kv_mlp_free(kv_mlp* h);
/* Checkpoint file: little-endian header (magic "KVMLP1\0\0", version, layer sizes, input and
 * output scaling, Adam step) followed by FP32 weights and Adam moments. */
int kv_mlp_save(const kv_mlp* h, const char* path);
int kv_mlp_load(const char* path, kv_mlp** out);
/* Host copies of the FP32 parameters in the order W1[64][2], b1[64], W2[64][64], b2[64],
 * W3[2][64], b3[2] (4482 floats), and back. */
int kv_mlp_get_params(const kv_mlp* h, float* host_params, int64_t count);
int kv_mlp_set_params(kv_mlp* h, const float* host_params, int64_t count);
#define KV_MLP_NPARAMS 4482

typedef struct kv_train_args {
    const double* v;      /* [n] device: training orders */
    const double* x;      /* [n] device: training arguments */
    const double* t0;     /* [n] device: target lower ends (from kv_bracket) */
    const double* t1;     /* [n] device: target upper ends */
    int64_t n;
    int batch;            /* samples per Adam step */
    int steps;            /* Adam steps to run */
    float lr, beta1, beta2, adam_eps;
    uint64_t seed;        /* sample order */
    float* loss_out;      /* [steps] device or NULL: mean loss of each step's batch */
    void* stream;
} kv_train_args;

/* Runs Adam steps on the mean squared error of the network's outputs against the scaled
 * targets; forward, backward and the update are this library's kernels. */
int kv_mlp_train(kv_mlp* h, const kv_train_args* a);

/* Forward pass and gradient of one batch, without updating (for checks against a reference):
 * loss (device double) and grads (device float[KV_MLP_NPARAMS]). */
int kv_mlp_loss_grad(const kv_mlp* h, const double* v, const double* x, const double* t0,
                     const double* t1, int64_t n, double* loss, float* grads, void* stream);

/* Raw predictions (t0, t1) of the network, before any check. */
int kv_mlp_predict(const kv_mlp* h, const void* v, const void* x, void* t0, void* t1, int64_t n,
                   int dtype, void* stream);

/* ------------------------------------------------------------------ diagnostics */
/* Number of kernels this library has launched in this process (all threads, all devices). */
uint64_t kv_launch_count(void);

/* For tests of the failure path: sets the iteration limit of the learned fast path's bounded
 * wait for its tensor-core results (each iteration one mbarrier try-wait).  A CTA whose wait runs
 * out hands all its remaining pairs to the fallback pass (the plain bracket, FP32 then FP64; edge
 * inputs get their edge results there), so the results stay correct, only slower; the CTA still
 * waits, with the full default limit, for the tensor-core work in flight before it releases its
 * tensor memory.  iterations >= 0 sets the limit (0: the wait gives up at once); < 0 restores the
 * default (2^22).  Process-wide; returns the previous setting (-1 for the default). */
int kv_debug_set_wait_limit(int iterations);

/* For tests of the learned fast path's bins: with on = 0 the trapezoid terms of bin n (t = t1,
 * weight 1/2) are computed as one of the bins instead of being taken from the range check's
 * evaluation of the right end (which the path does by default from 4 bins up and while
 * log eps <= -12; the two agree to FP32 rounding).  Process-wide; returns the previous setting
 * (1 = on, the default). */
int kv_debug_set_end_terms(int on);

/* Releases the device memory the library's scratch pool on the current device keeps reserved
 * (cudaMemPoolTrimTo to 0; memory of calls still in flight stays).  KV_OK if there is no pool. */
int kv_trim_memory(void);

/* ------------------------------------------------------------------ errors */
const char* kv_strerror(int code);
/* The last CUDA error string seen by this thread's calls ("" if none). */
const char* kv_last_cuda_error(void);

#ifdef __cplusplus
}
#endif
#endif /* KV_H_ */
