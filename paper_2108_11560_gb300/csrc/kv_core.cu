// Core kernels and C-ABI entry points of the batched log K_v(x) library (see include/kv.h).
//
// A warp takes 32 / L consecutive (v, x) pairs per trip and gives each a group of L lanes.  The
// group runs its pair's bracket (Algorithms 1-3, FP64) together, its lanes evaluating several
// points of each search at once (kv_bracket.cuh), then shares the pair's bins (Sec. 2.4,
// Sec. 4.1) and reduces its partial sums by warp shuffles.  L = 1 (large batches) is one pair per
// lane throughout; small batches take L > 1 so that they still occupy several warps per SM:
// GB300's FP64 unit costs the same per warp instruction whatever the number of active lanes, and
// one warp uses one SM sub-partition's share of it.  Warps iterate over pair blocks in a
// grid-stride loop so that all lanes of a warp make the same number of trips (the shuffles need
// the whole group); pairs past the end are computed on dummy inputs and not stored.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "kv_bins.cuh"
#include "kv_bracket.cuh"
#include "kv_internal.h"

#include <atomic>
#include <mutex>

// The host-buffer entry point streams chunks of 2^KV_HOST_MIN_CHUNK_LOG2 up to
// 2^KV_HOST_CHUNK_LOG2 pairs through KV_HOST_SLOTS device buffer slots.
#ifndef KV_HOST_CHUNK_LOG2
#define KV_HOST_CHUNK_LOG2 19
#endif
#ifndef KV_HOST_MIN_CHUNK_LOG2
#define KV_HOST_MIN_CHUNK_LOG2 19
#endif
#ifndef KV_HOST_SLOTS
#define KV_HOST_SLOTS 4
#endif

namespace {
thread_local char g_last_cuda_error[256] = "";
std::atomic<uint64_t> g_launches{0};
}

namespace kvh {

int cuda_fail(cudaError_t e)
{
    snprintf(g_last_cuda_error, sizeof(g_last_cuda_error), "%s: %s", cudaGetErrorName(e),
             cudaGetErrorString(e));
    return KV_ERR_CUDA;
}

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[64];
}  // namespace

// The library's own stream-ordered pool on the current device, created on first use with a
// release threshold that keeps freed memory reserved.
static cudaError_t scratch_pool(cudaMemPool_t* out, bool create)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_pool_mu);
    if (!g_pool[dev] && create) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~(uint64_t)0;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

cudaError_t scratch_alloc(void** p, size_t bytes, cudaStream_t s)
{
    cudaMemPool_t pool = nullptr;
    cudaError_t e = scratch_pool(&pool, true);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

cudaError_t scratch_free(void* p, cudaStream_t s) { return cudaFreeAsync(p, s); }

cudaError_t scratch_pool_get(cudaMemPool_t* pool) { return scratch_pool(pool, false); }

int sm_count()
{
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = n > 0 ? n : 1;
    }
    return cache[dev];
}

}  // namespace kvh

namespace {

using namespace kvd;

constexpr int kBlock = 128;

struct KParams {
    const void* v;
    const void* x;
    void* logk;
    void* dv;
    void* dx;
    const void* go;
    uint8_t* status;
    void* d2v;  // second derivatives (may be NULL)
    void* dvx;
    void* d2x;
    int64_t n;
    int bins;
    double log_eps;
    int max_iter;
    int flags;
};

// Domain edge cases (the list at the top of kv.h).  Returns true and fills the outputs for an
// edge pair; false for a regular pair (finite v, finite x > 0).
__device__ __forceinline__ bool edge_pair(double v, double x, double& lk, double& dv, double& dx)
{
    if (isnan(v) || isnan(x) || x < 0.0) {
        lk = dv = dx = nan("");
        return true;
    }
    if (x == 0.0) {
        lk = INFINITY;
        dv = (v == 0.0) ? 0.0 : copysign(INFINITY, v);
        dx = -INFINITY;
        return true;
    }
    if (isinf(x)) {
        lk = -INFINITY;
        dv = copysign(0.0, v);
        dx = -1.0;
        return true;
    }
    if (isinf(v)) {
        lk = INFINITY;
        dv = copysign(INFINITY, v);
        dx = -INFINITY;
        return true;
    }
    return false;
}

__device__ __noinline__ BracketD bracket_call(double v, double x, double log_eps, int max_iter, int flags)
{
    return bracket_f64(v, x, log_eps, max_iter, (flags & KV_FLAG_PEAK_ANALYTIC_START) != 0);
}

// The bracket of this lane's pair: on the lane alone (L = 1), or on the L lanes of its group,
// which all hold the same pair (L >= 2).
template <int L>
__device__ __forceinline__ BracketD bracket_lanes(double v, double x, double log_eps, int max_iter, int flags)
{
    if constexpr (L == 1) {
        return bracket_call(v, x, log_eps, max_iter, flags);
    } else {
        const int lane = threadIdx.x & 31;
        LaneGroup G;
        G.first = lane & ~(L - 1);
        G.l = lane & (L - 1);
        G.mask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << G.first;
        return bracket_f64_group<L>(G, v, x, log_eps, max_iter, (flags & KV_FLAG_PEAK_ANALYTIC_START) != 0);
    }
}

template <typename T>
__device__ __forceinline__ void store_outputs(const KParams& p, int64_t i, double lk, double dv,
                                              double dx, uint8_t st)
{
    if (p.go) {
        double g = (double)((const T*)p.go)[i];
        dv *= g;
        dx *= g;
    }
    if (p.logk) ((T*)p.logk)[i] = (T)lk;
    if (p.dv) ((T*)p.dv)[i] = (T)dv;
    if (p.dx) ((T*)p.dx)[i] = (T)dx;
    if (p.status) p.status[i] = st;
}

// Second derivatives of an edge pair (x = +inf: all 0; other edge inputs: NaN).
__device__ __forceinline__ void edge_second(double x, double& d2v, double& dvx, double& d2x)
{
    d2v = dvx = d2x = (isinf(x) && x > 0.0) ? 0.0 : nan("");
}

template <typename T>
__device__ __forceinline__ void store_second(const KParams& p, int64_t i, double d2v, double dvx, double d2x)
{
    if (p.d2v) ((T*)p.d2v)[i] = (T)d2v;
    if (p.dvx) ((T*)p.dvx)[i] = (T)dvx;
    if (p.d2x) ((T*)p.d2x)[i] = (T)d2x;
}

// Per-pair state: bracket, bin constants and the inputs as given.
struct SlotD {
    BinsD b;
    double G;           // g(t_p)
    double vin, xin;    // the inputs as given (edge results and the sign of v)
    double ar, cr;      // t_p tanh(v t_p), cosh t_p (second derivatives)
    int flags;          // kSlot* bits
};
constexpr int kSlotActive = 1, kSlotEdge = 2, kSlotCapped = 4;

// Pair i of this lane's group: the domain edges, the bracket (Algorithms 1-3) and the FP64 bin
// constants (every lane of the group computes the same).
template <int L>
__device__ __forceinline__ SlotD bracket_slot_f64(const KParams& p, int64_t i)
{
    SlotD s;
    const bool active = i < p.n;
    s.vin = active ? ((const double*)p.v)[i] : 1.0;
    s.xin = active ? ((const double*)p.x)[i] : 1.0;
    double lk, dv, dx;
    const bool edge = edge_pair(s.vin, s.xin, lk, dv, dx);
    const double va = edge ? 1.0 : fabs(s.vin);
    const double xa = edge ? 1.0 : s.xin;
    BracketD br = bracket_lanes<L>(va, xa, p.log_eps, p.max_iter, p.flags);
    BinsD& b = s.b;
    b.v = va;
    b.x = xa;
    b.t0 = br.t0;
    b.h = (br.t1 - br.t0) / p.bins;
    b.tp = br.tp;
    b.s0 = br.t0 - br.tp;
    b.e2u = exp(-2.0 * va * br.tp);
    b.Lu = log1p(b.e2u);
    b.ep = exp(br.tp);
    b.em = 1.0 / b.ep;
    const double shp = sinh(br.tp);
    b.c1 = fma(-xa, shp, va);
    b.xch = xa * cosh(br.tp);
    b.xsh = xa * shp;
    b.shp = shp;
    b.n = p.bins;
    s.G = br.G;
    s.ar = br.tp * ((1.0 - b.e2u) / (1.0 + b.e2u));
    s.cr = cosh(br.tp);
    s.flags = (active ? kSlotActive : 0) | (edge ? kSlotEdge : 0) | (br.capped ? kSlotCapped : 0);
    return s;
}

// FP64 plain path: the paper's bracket and bins, all in double.  With D2 (L = 1 only) the bins
// also give the second derivatives (sums2_f64), and the first derivatives come from the same
// shifted sums.
template <int L, bool DERIV, bool D2 = false>
__global__ void __launch_bounds__(kBlock) kv_f64_kernel(KParams p)
{
    static_assert(!D2 || L == 1, "second derivatives run one pair per lane");
    constexpr int Q = 32 / L;  // pairs per warp trip (lane groups per warp)
    const int lane = threadIdx.x & 31;
    const int g = lane / L, l = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    for (int64_t base = warp * Q; base < p.n; base += nwarps * Q) {
        {
            const int64_t i = base + g;  // the pair this lane's group brackets and sums together
            const SlotD s = bracket_slot_f64<L>(p, i);
            const bool active = s.flags & kSlotActive;
            const bool edge = s.flags & kSlotEdge;
            const uint8_t st = edge ? KV_PAIR_EDGE : (s.flags & kSlotCapped) ? KV_PAIR_RANGE_CAP : KV_PAIR_OK;
            double lk, dv, dx;
            edge_pair(s.vin, s.xin, lk, dv, dx);
            if constexpr (D2) {
                const Sums2<double> m = sums2_f64<1>(s.b, 0);
                if (active) {
                    double d2v, dvx, d2x;
                    if (edge) {
                        edge_second(s.xin, d2v, dvx, d2x);
                    } else {
                        moments_finish<double>(m, s.ar, s.cr, dv, dx, d2v, dvx, d2x);
                        lk = s.G + log(s.b.h) + log(m.s0);
                        dv = s.vin == 0.0 ? 0.0 : copysign(dv, s.vin);
                        dvx = s.vin == 0.0 ? 0.0 : copysign(1.0, s.vin) * dvx;
                    }
                    store_outputs<double>(p, i, lk, dv, dx, st);
                    store_second<double>(p, i, d2v, dvx, d2x);
                }
            } else {
                double S0, S1, S2;
                sums_f64<L, DERIV>(s.b, l, S0, S1, S2);
                if (active && l == 0) {
                    if (!edge) {
                        lk = s.G + log(s.b.h) + log(S0);
                        dv = DERIV ? copysign(S1 / S0, s.vin) : 0.0;
                        if (s.vin == 0.0) dv = 0.0;
                        dx = DERIV ? -(S2 / S0) : 0.0;
                    }
                    store_outputs<double>(p, i, lk, dv, dx, st);
                }
            }
        }
    }
}

// Per-pair state of the mixed path with the FP64 bracket (FP32 bin constants, FP64 offset).
struct SlotF {
    BinsF b;
    double G;
    float vin, xin;
    float ar, cr;  // second derivatives
    int flags;
};

// Pair i of this lane's group on the mixed path: edges, the FP64 bracket, FP64 offset and
// constants rounded to the FP32 bins' form.
template <int L>
__device__ __forceinline__ SlotF bracket_slot_mixed(const KParams& p, int64_t i)
{
    SlotF s;
    const bool active = i < p.n;
    s.vin = active ? ((const float*)p.v)[i] : 1.0f;
    s.xin = active ? ((const float*)p.x)[i] : 1.0f;
    double lk, dv, dx;
    const bool edge = edge_pair((double)s.vin, (double)s.xin, lk, dv, dx);
    const double va = edge ? 1.0 : fabs((double)s.vin);
    const double xa = edge ? 1.0 : (double)s.xin;
    BracketD br = bracket_lanes<L>(va, xa, p.log_eps, p.max_iter, p.flags);
    const double ep = exp(br.tp), em = 1.0 / ep;
    const double u = va * br.tp;
    const double h = (br.t1 - br.t0) / p.bins;
    const double e2u = exp(-2.0 * u);
    BinsF& b = s.b;
    b.s0 = (float)(br.t0 - br.tp);
    b.h = (float)h;
    b.v = (float)va;
    b.u = (float)u;
    b.tp = (float)br.tp;
    b.c1 = (float)(va - xa * 0.5 * (ep - em));
    b.ap = (float)(xa * 0.5 * ep);
    b.am = (float)(xa * 0.5 * em);
    b.lu = (float)log1p(e2u);
    b.ep = (float)ep;
    b.em = (float)em;
    b.xch = (float)(xa * cosh(br.tp));
    b.xsh = (float)(xa * sinh(br.tp));
    b.e2u = (float)e2u;
    b.shp = (float)sinh(br.tp);
    b.n = p.bins;
    s.G = br.G;
    s.ar = (float)(br.tp * ((1.0 - e2u) / (1.0 + e2u)));
    s.cr = (float)cosh(br.tp);
    s.flags = (active ? kSlotActive : 0) | (edge ? kSlotEdge : 0) | (br.capped ? kSlotCapped : 0);
    return s;
}

// Mixed path with the plain FP64 bracket: FP64 peak, offset and per-pair constants, FP32 bins.
// D2 (L = 1 only): second derivatives from the shifted FP32 sums (sums2_f32).  Pairs per trip
// and lanes as in kv_f64_kernel.
template <int L, bool DERIV, bool D2 = false>
__global__ void __launch_bounds__(kBlock) kv_mixed_kernel(KParams p)
{
    static_assert(!D2 || L == 1, "second derivatives run one pair per lane");
    constexpr int Q = 32 / L;
    const int lane = threadIdx.x & 31;
    const int g = lane / L, l = lane % L;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) / 32;
    for (int64_t base = warp * Q; base < p.n; base += nwarps * Q) {
        {
            const int64_t i = base + g;
            const SlotF s = bracket_slot_mixed<L>(p, i);
            const bool active = s.flags & kSlotActive;
            const bool edge = s.flags & kSlotEdge;
            const uint8_t st = edge ? KV_PAIR_EDGE : (s.flags & kSlotCapped) ? KV_PAIR_RANGE_CAP : KV_PAIR_OK;
            const double v = (double)s.vin;
            double lk, dv, dx;
            edge_pair(v, (double)s.xin, lk, dv, dx);
            if constexpr (D2) {
                const Sums2<float> m = sums2_f32<1>(s.b, 0);
                if (active) {
                    double d2v, dvx, d2x;
                    if (edge) {
                        edge_second((double)s.xin, d2v, dvx, d2x);
                    } else {
                        float fdv, fdx, fd2v, fdvx, fd2x;
                        moments_finish<float>(m, s.ar, s.cr, fdv, fdx, fd2v, fdvx, fd2x);
                        lk = s.G + (double)logf(s.b.h * m.s0);
                        dv = v == 0.0 ? 0.0 : copysign((double)fdv, v);
                        dx = fdx;
                        d2v = fd2v;
                        dvx = v == 0.0 ? 0.0 : copysign(1.0, v) * (double)fdvx;
                        d2x = fd2x;
                    }
                    store_outputs<float>(p, i, lk, dv, dx, st);
                    store_second<float>(p, i, d2v, dvx, d2x);
                }
            } else {
                float S0, S1, S2;
                sums_f32<L, DERIV>(s.b, l, S0, S1, S2);
                if (active && l == 0) {
                    if (!edge) {
                        lk = s.G + (double)logf(s.b.h * S0);
                        float r = 1.0f / S0;
                        dv = DERIV ? copysign((double)(S1 * r), v) : 0.0;
                        if (v == 0.0) dv = 0.0;
                        dx = DERIV ? -(double)(S2 * r) : 0.0;
                    }
                    store_outputs<float>(p, i, lk, dv, dx, st);
                }
            }
        }
    }
}

// The bracket alone, for training targets and checks.
template <typename T>
__global__ void __launch_bounds__(kBlock) kv_bracket_kernel(const T* v, const T* x, double* t0,
                                                            double* tp, double* t1, double* gtp,
                                                            int64_t n, double log_eps, int max_iter)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double vv = fabs((double)v[i]), xx = (double)x[i];
        double lk, dv, dx;
        if (edge_pair((double)v[i], xx, lk, dv, dx)) {
            if (t0) t0[i] = nan("");
            if (tp) tp[i] = nan("");
            if (t1) t1[i] = nan("");
            if (gtp) gtp[i] = nan("");
            continue;
        }
        BracketD br = bracket_call(vv, xx, log_eps, max_iter, 0);
        if (t0) t0[i] = br.t0;
        if (tp) tp[i] = br.tp;
        if (t1) t1[i] = br.t1;
        if (gtp) gtp[i] = br.G;
    }
}

template <typename T>
__global__ void kv_grad_kernel(const T* go, const T* dv, const T* dx, T* gv, T* gx, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        T g = go[i];
        if (gv) gv[i] = g * dv[i];
        if (gx) gx[i] = g * dx[i];
    }
}

// The second backward pass's epilogue (the backward of g_v = go dv, g_x = go dx).
template <typename T>
struct Grad2Args {
    const T *go, *ggv, *ggx, *dv, *dx, *d2v, *dvx, *d2x;
    T *ov, *ox, *ogo;
    int64_t n;
};

template <typename T>
__global__ void kv_grad2_kernel(Grad2Args<T> a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const T gv = a.ggv ? a.ggv[i] : T(0), gx = a.ggx ? a.ggx[i] : T(0);
        if (a.ov || a.ox) {
            const T go = a.go[i], dvx = a.dvx[i];
            if (a.ov) a.ov[i] = go * (gv * a.d2v[i] + gx * dvx);
            if (a.ox) a.ox[i] = go * (gv * dvx + gx * a.d2x[i]);
        }
        if (a.ogo) a.ogo[i] = gv * a.dv[i] + gx * a.dx[i];
    }
}

// Deterministic two-stage sum: fixed grid for a given n, fixed reduction order.  kv_noalloc.cu
// repeats these two kernels for the sum without allocation (same order, same bits): a change
// here must be made there too.
constexpr int kSumBlock = 256;

template <typename T>
__global__ void __launch_bounds__(kSumBlock) kv_sum_partial(const T* a, int64_t n, double* part)
{
    __shared__ double sh[kSumBlock];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * kSumBlock + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSumBlock)
        acc += (double)a[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kSumBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(kSumBlock) kv_sum_final(const double* part, int nb, double* out)
{
    __shared__ double sh[kSumBlock];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += kSumBlock) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kSumBlock / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// ------------------------------------------------------------------ host side

template <typename K>
int launch_pairs(K kernel, const KParams& p, int pairs_per_warp, cudaStream_t s)
{
    // one block per kBlock / 32 warps' pairs (a block's four warps run on the SM's four
    // sub-partitions): the block scheduler hands each SM a new block as one finishes, where a
    // persistent grid with a fixed share per block ends with SMs running fewer and fewer blocks
    // (the blocks resident on one SM get unequal shares of its issue slots).  Beyond the largest
    // grid the kernels' grid-stride loops take the rest.
    const int64_t warps = (p.n + pairs_per_warp - 1) / pairs_per_warp;
    const int block = kBlock;
    const int64_t need = (warps * 32 + block - 1) / block;
    int grid = (int)(need < 0x7fffffffll ? need : 0x7fffffffll);
    if (grid < 1) grid = 1;
    kernel<<<grid, block, 0, s>>>(p);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

// Second derivatives: one pair per thread.
int dispatch_second(const KParams& p, int dtype, cudaStream_t s)
{
    if (dtype == KV_F64) return launch_pairs(kv_f64_kernel<1, true, true>, p, 32, s);
    return launch_pairs(kv_mixed_kernel<1, true, true>, p, 32, s);
}

template <int L>
int dispatch_deriv(const KParams& p, int dtype, bool deriv, cudaStream_t s)
{
    if (dtype == KV_F64)
        return deriv ? launch_pairs(kv_f64_kernel<L, true>, p, 32 / L, s)
                     : launch_pairs(kv_f64_kernel<L, false>, p, 32 / L, s);
    return deriv ? launch_pairs(kv_mixed_kernel<L, true>, p, 32 / L, s)
                 : launch_pairs(kv_mixed_kernel<L, false>, p, 32 / L, s);
}

int auto_lanes(int64_t n)
{
    // the most lanes per pair (fewest pairs per warp) for which the batch still needs no more
    // warps than the GPU has SM sub-partitions (four per SM): small batches then keep every
    // sub-partition's FP64 unit busy, large ones run one pair per lane
    const int64_t slots = 4 * (int64_t)kvh::sm_count();
    int L = 32;
    while (L > 1 && (n * L + 31) / 32 > slots) L /= 2;
    return L;
}

int validate(const kv_args* a, int* bins, double* log_eps, int* max_iter, int* lanes)
{
    if (!a) return KV_ERR_NULL;
    if (a->dtype != KV_F64 && a->dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (a->n < 0) return KV_ERR_SIZE;
    if (a->n > 0 && (!a->v || !a->x)) return KV_ERR_NULL;
    if (a->n > 0 && !a->logk && !a->dv && !a->dx && !a->d2v && !a->dvx && !a->d2x) return KV_ERR_NULL;
    *bins = a->bins == 0 ? (a->dtype == KV_F64 ? 128 : 40) : a->bins;
    if (*bins < 1 || *bins > KV_MAX_BINS) return KV_ERR_BINS;
    *log_eps = a->log_eps == 0.0 ? (a->dtype == KV_F64 ? -52.0 * kvd::LN2_D : -20.0) : a->log_eps;
    if (!(*log_eps < 0.0) || !isfinite(*log_eps)) return KV_ERR_ARG;
    *max_iter = a->max_iter == 0 ? KV_DEFAULT_MAX_ITER : a->max_iter;
    if (*max_iter < 1 || *max_iter > 64) return KV_ERR_ARG;
    int L = a->lanes == 0 ? auto_lanes(a->n) : a->lanes;
    if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16 && L != 32) return KV_ERR_ARG;
    *lanes = L;
    if (a->bracket != KV_BRACKET_PLAIN && a->bracket != KV_BRACKET_MLP && a->bracket != KV_BRACKET_PLAIN_F32)
        return KV_ERR_ARG;
    if (a->bracket != KV_BRACKET_PLAIN && a->dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (a->bracket == KV_BRACKET_MLP && !a->mlp) return KV_ERR_HANDLE;
    if (a->flags & ~KV_FLAG_PEAK_ANALYTIC_START) return KV_ERR_ARG;
    size_t es = kvh::elem_size(a->dtype);
    const void* ptrs[9] = {a->v, a->x, a->logk, a->dv, a->dx, a->grad_out, a->d2v, a->dvx, a->d2x};
    for (const void* q : ptrs)
        if (q && !kvh::aligned(q, es)) return KV_ERR_ALIGN;
    return KV_OK;
}

}  // namespace

extern "C" {

int kv_fwd_bwd_ex(const kv_args* a) { return kvh::fwd_bwd_ex(a, nullptr); }

}  // extern "C"

int kvh::fwd_bwd_ex(const kv_args* a, uint32_t* scratch)
{
    int bins, max_iter, lanes;
    double log_eps;
    int rc = validate(a, &bins, &log_eps, &max_iter, &lanes);
    if (rc != KV_OK) return rc;
    if (a->n == 0) return KV_OK;
    if (a->bracket != KV_BRACKET_PLAIN) return kvh::launch_mlp_path(a, bins, log_eps, max_iter, scratch);
    KParams p;
    p.v = a->v;
    p.x = a->x;
    p.logk = a->logk;
    p.dv = a->dv;
    p.dx = a->dx;
    p.go = a->grad_out;
    p.status = a->status;
    p.d2v = a->d2v;
    p.dvx = a->dvx;
    p.d2x = a->d2x;
    p.n = a->n;
    p.bins = bins;
    p.log_eps = log_eps;
    p.max_iter = max_iter;
    p.flags = a->flags;
    const bool deriv = a->dv || a->dx;
    cudaStream_t s = (cudaStream_t)a->stream;
    if (a->d2v || a->dvx || a->d2x) return dispatch_second(p, a->dtype, s);
    switch (lanes) {
        case 1: return dispatch_deriv<1>(p, a->dtype, deriv, s);
        case 2: return dispatch_deriv<2>(p, a->dtype, deriv, s);
        case 4: return dispatch_deriv<4>(p, a->dtype, deriv, s);
        case 8: return dispatch_deriv<8>(p, a->dtype, deriv, s);
        case 16: return dispatch_deriv<16>(p, a->dtype, deriv, s);
        default: return dispatch_deriv<32>(p, a->dtype, deriv, s);
    }
}

extern "C" {

static int core_call(const void* v, const void* x, void* logk, void* dv, void* dx, int64_t n,
                     int bins, int dtype, void* stream)
{
    if (bins == 0) return KV_ERR_BINS;  // the four core calls take an explicit bin count
    kv_args a;
    memset(&a, 0, sizeof(a));
    a.v = v;
    a.x = x;
    a.logk = logk;
    a.dv = dv;
    a.dx = dx;
    a.n = n;
    a.bins = bins;
    a.dtype = dtype;
    a.stream = stream;
    return kv_fwd_bwd_ex(&a);
}

int kv_log(const void* v, const void* x, void* logk, int64_t n, int bins, int dtype, void* stream)
{
    if (n > 0 && !logk) return KV_ERR_NULL;
    return core_call(v, x, logk, nullptr, nullptr, n, bins, dtype, stream);
}

int kv_log_dv(const void* v, const void* x, void* dlogk_dv, int64_t n, int bins, int dtype,
              void* stream)
{
    if (n > 0 && !dlogk_dv) return KV_ERR_NULL;
    return core_call(v, x, nullptr, dlogk_dv, nullptr, n, bins, dtype, stream);
}

int kv_log_dx(const void* v, const void* x, void* dlogk_dx, int64_t n, int bins, int dtype,
              void* stream)
{
    if (n > 0 && !dlogk_dx) return KV_ERR_NULL;
    return core_call(v, x, nullptr, nullptr, dlogk_dx, n, bins, dtype, stream);
}

int kv_fwd_bwd(const void* v, const void* x, void* logk, void* dv, void* dx, int64_t n, int bins,
               int dtype, void* stream)
{
    if (n > 0 && (!logk || !dv || !dx)) return KV_ERR_NULL;
    return core_call(v, x, logk, dv, dx, n, bins, dtype, stream);
}

int kv_bracket(const void* v, const void* x, double* t0, double* tp, double* t1, double* g_tp,
               int64_t n, int dtype, double log_eps, int max_iter, void* stream)
{
    if (dtype != KV_F64 && dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0) return KV_ERR_SIZE;
    if (n == 0) return KV_OK;
    if (!v || !x) return KV_ERR_NULL;
    if (!t0 && !tp && !t1 && !g_tp) return KV_ERR_NULL;
    if (log_eps == 0.0) log_eps = dtype == KV_F64 ? -52.0 * kvd::LN2_D : -20.0;
    if (!(log_eps < 0.0) || !isfinite(log_eps)) return KV_ERR_ARG;
    if (max_iter == 0) max_iter = KV_DEFAULT_MAX_ITER;
    if (max_iter < 1 || max_iter > 64) return KV_ERR_ARG;
    size_t es = kvh::elem_size(dtype);
    if (!kvh::aligned(v, es) || !kvh::aligned(x, es)) return KV_ERR_ALIGN;
    const void* outs[4] = {t0, tp, t1, g_tp};
    for (const void* q : outs)
        if (q && !kvh::aligned(q, 8)) return KV_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t need = (n + kBlock - 1) / kBlock;
    int64_t cap = (int64_t)kvh::sm_count() * 8;
    int grid = (int)(need < cap ? need : cap);
    if (dtype == KV_F64)
        kv_bracket_kernel<double><<<grid, kBlock, 0, s>>>((const double*)v, (const double*)x, t0, tp,
                                                          t1, g_tp, n, log_eps, max_iter);
    else
        kv_bracket_kernel<float><<<grid, kBlock, 0, s>>>((const float*)v, (const float*)x, t0, tp,
                                                         t1, g_tp, n, log_eps, max_iter);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

int kv_grad(const void* grad_out, const void* dv, const void* dx, void* grad_v, void* grad_x,
            int64_t n, int dtype, void* stream)
{
    if (dtype != KV_F64 && dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0) return KV_ERR_SIZE;
    if (n == 0) return KV_OK;
    if (!grad_out || (!grad_v && !grad_x)) return KV_ERR_NULL;
    if ((grad_v && !dv) || (grad_x && !dx)) return KV_ERR_NULL;
    size_t es = kvh::elem_size(dtype);
    const void* ptrs[5] = {grad_out, dv, dx, grad_v, grad_x};
    for (const void* q : ptrs)
        if (q && !kvh::aligned(q, es)) return KV_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t need = (n + 255) / 256;
    int64_t cap = (int64_t)kvh::sm_count() * 16;
    int grid = (int)(need < cap ? need : cap);
    if (dtype == KV_F64)
        kv_grad_kernel<double><<<grid, 256, 0, s>>>((const double*)grad_out, (const double*)dv,
                                                    (const double*)dx, (double*)grad_v,
                                                    (double*)grad_x, n);
    else
        kv_grad_kernel<float><<<grid, 256, 0, s>>>((const float*)grad_out, (const float*)dv,
                                                   (const float*)dx, (float*)grad_v, (float*)grad_x,
                                                   n);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

}  // extern "C"

template <typename T>
static void launch_grad2(const void* go, const void* ggv, const void* ggx, const void* dv,
                         const void* dx, const void* d2v, const void* dvx, const void* d2x,
                         void* ov, void* ox, void* ogo, int64_t n, int grid, cudaStream_t s)
{
    Grad2Args<T> a{(const T*)go, (const T*)ggv, (const T*)ggx, (const T*)dv, (const T*)dx,
                   (const T*)d2v, (const T*)dvx, (const T*)d2x, (T*)ov, (T*)ox, (T*)ogo, n};
    kv_grad2_kernel<T><<<grid, 256, 0, s>>>(a);
}

extern "C" {

int kv_grad2(const void* go, const void* gg_v, const void* gg_x, const void* dv, const void* dx,
             const void* d2v, const void* dvx, const void* d2x, void* out_v, void* out_x,
             void* out_go, int64_t n, int dtype, void* stream)
{
    if (dtype != KV_F64 && dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0) return KV_ERR_SIZE;
    if (n == 0) return KV_OK;
    if (!out_v && !out_x && !out_go) return KV_ERR_NULL;
    if ((out_v || out_x) && (!go || !d2v || !dvx || !d2x)) return KV_ERR_NULL;
    if (out_go && (!dv || !dx)) return KV_ERR_NULL;
    size_t es = kvh::elem_size(dtype);
    const void* ptrs[11] = {go, gg_v, gg_x, dv, dx, d2v, dvx, d2x, out_v, out_x, out_go};
    for (const void* q : ptrs)
        if (q && !kvh::aligned(q, es)) return KV_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t need = (n + 255) / 256;
    int64_t cap = (int64_t)kvh::sm_count() * 16;
    int grid = (int)(need < cap ? need : cap);
    if (dtype == KV_F64)
        launch_grad2<double>(go, gg_v, gg_x, dv, dx, d2v, dvx, d2x, out_v, out_x, out_go, n, grid, s);
    else
        launch_grad2<float>(go, gg_v, gg_x, dv, dx, d2v, dvx, d2x, out_v, out_x, out_go, n, grid, s);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

// Number of partial sums for n elements: a function of n only, so results are reproducible.
static int sum_blocks(int64_t n)
{
    int64_t b = (n + 4095) / 4096;
    if (b < 1) b = 1;
    if (b > 1024) b = 1024;
    return (int)b;
}

int kv_sum(const void* a, int64_t n, int dtype, double* out, void* stream)
{
    if (dtype != KV_F64 && dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0) return KV_ERR_SIZE;
    if (!out || (n > 0 && !a)) return KV_ERR_NULL;
    if (!kvh::aligned(out, 8) || (a && !kvh::aligned(a, kvh::elem_size(dtype)))) return KV_ERR_ALIGN;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {
        KV_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double), s));
        return KV_OK;
    }
    int nb = sum_blocks(n);
    double* part = nullptr;
    KV_CUDA_TRY(kvh::scratch_alloc((void**)&part, sizeof(double) * nb, s));
    if (dtype == KV_F64)
        kv_sum_partial<double><<<nb, kSumBlock, 0, s>>>((const double*)a, n, part);
    else
        kv_sum_partial<float><<<nb, kSumBlock, 0, s>>>((const float*)a, n, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        kvh::note_launch();
        kv_sum_final<<<1, kSumBlock, 0, s>>>(part, nb, out);
        kvh::note_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = kvh::scratch_free(part, s);
    if (e != cudaSuccess) return kvh::cuda_fail(e);
    if (e2 != cudaSuccess) return kvh::cuda_fail(e2);
    return KV_OK;
}

}  // extern "C"

namespace {

// The device address of host buffer [p, p + bytes) when the whole range is page-locked host
// memory mapped into the device's address space (both ends are checked, and they must map
// contiguously), else nullptr.  Never leaves a CUDA error behind.
void* host_device_alias(const void* p, size_t bytes)
{
    if (!p || bytes == 0) return nullptr;
    cudaPointerAttributes a0, a1;
    const char* last = (const char*)p + (bytes - 1);
    const bool ok = cudaPointerGetAttributes(&a0, p) == cudaSuccess &&
                    cudaPointerGetAttributes(&a1, last) == cudaSuccess && a0.type == cudaMemoryTypeHost &&
                    a1.type == cudaMemoryTypeHost && a0.devicePointer && a1.devicePointer &&
                    (const char*)a1.devicePointer == (const char*)a0.devicePointer + (bytes - 1);
    cudaGetLastError();
    return ok ? a0.devicePointer : nullptr;
}

// Whether the current device reaches host memory over a coherent link (native host atomics or
// access through the host's page tables, as on NVLink-C2C systems), where kernels reading and
// writing host buffers directly keep up with the fused kernel.
bool coherent_host_link()
{
    static int cache[64];
    static bool known[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return false;
    }
    if (!known[dev]) {
        int atomics = 0, host_tables = 0;
        cudaDeviceGetAttribute(&atomics, cudaDevAttrHostNativeAtomicSupported, dev);
        cudaDeviceGetAttribute(&host_tables, cudaDevAttrPageableMemoryAccessUsesHostPageTables, dev);
        cudaGetLastError();
        cache[dev] = (atomics == 1 || host_tables == 1) ? 1 : 0;
        known[dev] = true;
    }
    return cache[dev] == 1;
}

// DIRECT transfer: one launch of the path on the host buffers' device aliases, on the caller's
// stream; the fallback list is device memory allocated on the stream.
int host_direct(const kv_args* h, void* const alias[5])
{
    kv_args d = *h;
    d.v = alias[0];
    d.x = alias[1];
    d.logk = alias[2];
    d.dv = alias[3];
    d.dx = alias[4];
    int rc = kvh::fwd_bwd_ex(&d, nullptr);
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)h->stream);
    if (rc != KV_OK) return rc;
    if (e != cudaSuccess) return kvh::cuda_fail(e);
    return KV_OK;
}

int host_staged(const kv_args* h);

}  // namespace

extern "C" {

int kv_host_direct_supported(void) { return coherent_host_link() ? 1 : 0; }

int kv_fwd_bwd_host_ex(const kv_args* h, int transfer)
{
    if (!h) return KV_ERR_NULL;
    if (h->grad_out || h->status || h->fallback_count || h->d2v || h->dvx || h->d2x) return KV_ERR_ARG;
    if (transfer != KV_HOST_AUTO && transfer != KV_HOST_STAGED && transfer != KV_HOST_DIRECT) return KV_ERR_ARG;
    int bins_, max_iter_, lanes_;
    double log_eps_;
    int rc = validate(h, &bins_, &log_eps_, &max_iter_, &lanes_);
    if (rc != KV_OK) return rc;
    if (h->n == 0) return KV_OK;
    if (transfer != KV_HOST_STAGED) {
        const size_t bytes = kvh::elem_size(h->dtype) * (size_t)h->n;
        const void* host[5] = {h->v, h->x, h->logk, h->dv, h->dx};
        void* alias[5] = {};
        bool all = true;
        for (int k = 0; k < 5; ++k)
            if (host[k] && !(alias[k] = host_device_alias(host[k], bytes))) all = false;
        if (transfer == KV_HOST_DIRECT && !all) return KV_ERR_ARG;
        if (all && (transfer == KV_HOST_DIRECT || coherent_host_link())) return host_direct(h, alias);
    }
    return host_staged(h);
}

int kv_fwd_bwd_host(const kv_args* h) { return kv_fwd_bwd_host_ex(h, KV_HOST_AUTO); }

}  // extern "C"

namespace {

// STAGED transfer: chunks rotate over KV_HOST_SLOTS device buffer slots; one internal stream
// copies inputs in, one copies outputs out and one per slot runs the kernels, ordered by events,
// so one chunk's input copy, other chunks' kernels and another's output copy run at the same
// time.  Device buffers (and the learned path's fallback lists) are allocated once per call.
int host_staged(const kv_args* h)
{
    int rc = KV_OK;
    const int64_t n = h->n;
    const size_t es = kvh::elem_size(h->dtype);
    // chunk sizes: doubling from the minimum at the start and halving towards the end (short
    // fill and drain of the pipeline), the maximum in between (few launches)
    const int64_t cmax = (int64_t)1 << KV_HOST_CHUNK_LOG2, cmin = (int64_t)1 << KV_HOST_MIN_CHUNK_LOG2;
    const int64_t chunk = n < cmax ? n : cmax;  // the slot size
    auto chunk_size = [&](int64_t c, int64_t left) {
        int64_t sz = cmin << (c < 20 ? c : 20);
        if (sz > left / 2) sz = left / 2;
        if (sz < cmin) sz = cmin;
        if (sz > chunk) sz = chunk;
        return sz < left ? sz : left;
    };
    int64_t nchunks = 0;
    for (int64_t off = 0; off < n; ++nchunks) off += chunk_size(nchunks, n - off);
    const int nslots = nchunks < KV_HOST_SLOTS ? (int)nchunks : KV_HOST_SLOTS;
    const bool mlp = h->bracket != KV_BRACKET_PLAIN;  // the paths with a fallback list
    // a slot: inputs (2 arrays) and outputs (3 arrays) with separate lifetimes, and the fallback
    // list of the learned path
    const size_t in_bytes = 2 * es * chunk, out_bytes = 3 * es * chunk;
    const size_t slot_bytes = in_bytes + out_bytes + (mlp ? sizeof(uint32_t) * (chunk + 32) : 0);
    // streams: one for host-to-device copies, one for device-to-host copies, one per slot for
    // the kernels; events order them.  An input slot is refilled as soon as its kernel has read
    // it, an output slot as soon as its copy-out is done, so the copy engines never wait for a
    // whole slot cycle.
    cudaStream_t caller = (cudaStream_t)h->stream;
    cudaStream_t sin = nullptr, sout = nullptr, sk[KV_HOST_SLOTS] = {};
    cudaEvent_t start = nullptr, in_ready[KV_HOST_SLOTS] = {}, done[KV_HOST_SLOTS] = {},
                out_free[KV_HOST_SLOTS] = {};
    bool used_in[KV_HOST_SLOTS] = {}, used_out[KV_HOST_SLOTS] = {};
    cudaError_t e = cudaStreamCreateWithFlags(&sin, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sout, cudaStreamNonBlocking);
    for (int k = 0; k < nslots && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&sk[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&start, cudaEventDisableTiming);
    for (int k = 0; k < nslots && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&in_ready[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&out_free[k], cudaEventDisableTiming);
    }
    char* buf = nullptr;
    if (e == cudaSuccess) e = kvh::scratch_alloc((void**)&buf, slot_bytes * nslots, caller);
    // everything starts after the caller's stream has reached this call (and the allocation)
    if (e == cudaSuccess) e = cudaEventRecord(start, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sin, start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, start, 0);
    for (int k = 0; k < nslots && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(sk[k], start, 0);
    int64_t off = 0;
    for (int64_t c = 0; e == cudaSuccess && rc == KV_OK && c < nchunks; ++c) {
        const int k = (int)(c % nslots);
        const int64_t m = chunk_size(c, n - off);
        char* base = buf + slot_bytes * k;
        char* dvin = base;
        char* dxin = base + es * chunk;
        char* dl = base + in_bytes;
        char* ddv = dl + es * chunk;
        char* ddx = ddv + es * chunk;
        uint32_t* scratch = mlp ? (uint32_t*)(base + in_bytes + out_bytes) : nullptr;
        // copy in once the slot's previous kernel has read its inputs
        if (used_in[k]) e = cudaStreamWaitEvent(sin, done[k], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dvin, (const char*)h->v + es * off, es * m, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dxin, (const char*)h->x + es * off, es * m, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess) e = cudaEventRecord(in_ready[k], sin);
        used_in[k] = true;
        // compute once the inputs are in and the slot's previous outputs have been copied out
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sk[k], in_ready[k], 0);
        if (e == cudaSuccess && used_out[k]) e = cudaStreamWaitEvent(sk[k], out_free[k], 0);
        if (e != cudaSuccess) break;
        kv_args d = *h;
        d.v = dvin;
        d.x = dxin;
        d.logk = h->logk ? dl : nullptr;
        d.dv = h->dv ? ddv : nullptr;
        d.dx = h->dx ? ddx : nullptr;
        d.n = m;
        d.stream = sk[k];
        rc = kvh::fwd_bwd_ex(&d, scratch);
        if (rc != KV_OK) break;
        e = cudaEventRecord(done[k], sk[k]);
        // copy out once the kernel is done
        if (e == cudaSuccess) e = cudaStreamWaitEvent(sout, done[k], 0);
        if (e == cudaSuccess && h->logk)
            e = cudaMemcpyAsync((char*)h->logk + es * off, dl, es * m, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess && h->dv)
            e = cudaMemcpyAsync((char*)h->dv + es * off, ddv, es * m, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess && h->dx)
            e = cudaMemcpyAsync((char*)h->dx + es * off, ddx, es * m, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess) e = cudaEventRecord(out_free[k], sout);
        used_out[k] = true;
        off += m;
    }
    // join every internal stream into the caller's before the buffer goes
    cudaStream_t all[KV_HOST_SLOTS + 2] = {sin, sout};
    for (int k = 0; k < nslots; ++k) all[2 + k] = sk[k];
    for (int k = 0; k < nslots + 2; ++k) {
        if (!all[k] || !start) continue;
        cudaError_t e2 = cudaEventRecord(start, all[k]);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(caller, start, 0);
        if (e == cudaSuccess) e = e2;
    }
    if (buf) {
        cudaError_t e2 = kvh::scratch_free(buf, caller);
        if (e == cudaSuccess) e = e2;
    }
    cudaError_t e3 = cudaStreamSynchronize(caller);
    if (e == cudaSuccess) e = e3;
    for (int k = 0; k < nslots; ++k) {
        if (in_ready[k]) cudaEventDestroy(in_ready[k]);
        if (done[k]) cudaEventDestroy(done[k]);
        if (out_free[k]) cudaEventDestroy(out_free[k]);
        if (sk[k]) cudaStreamDestroy(sk[k]);
    }
    if (start) cudaEventDestroy(start);
    if (sin) cudaStreamDestroy(sin);
    if (sout) cudaStreamDestroy(sout);
    if (rc != KV_OK) return rc;
    if (e != cudaSuccess) return kvh::cuda_fail(e);
    return KV_OK;
}

}  // namespace

extern "C" {

const char* kv_strerror(int code)
{
    switch (code) {
        case KV_OK: return "ok";
        case KV_ERR_NULL: return "a required pointer is NULL";
        case KV_ERR_SIZE: return "n < 0 or a size limit exceeded";
        case KV_ERR_BINS: return "bins out of range [1, KV_MAX_BINS]";
        case KV_ERR_DTYPE: return "unknown dtype or mode not available for this dtype";
        case KV_ERR_ALIGN: return "a pointer is not aligned to its element size";
        case KV_ERR_CUDA: return "a CUDA call failed (see kv_last_cuda_error)";
        case KV_ERR_ARG: return "an argument is out of range";
        case KV_ERR_HANDLE: return "NULL or invalid MLP handle";
        case KV_ERR_IO: return "checkpoint file could not be opened, read or written";
        case KV_ERR_FORMAT: return "checkpoint file has the wrong magic, version or sizes";
        case KV_ERR_NOMEM: return "allocation failed";
        default: return "unknown status";
    }
}

const char* kv_last_cuda_error(void) { return g_last_cuda_error; }

uint64_t kv_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int kv_trim_memory(void)
{
    cudaMemPool_t pool = nullptr;
    cudaError_t e = kvh::scratch_pool_get(&pool);
    if (e == cudaSuccess && pool) e = cudaMemPoolTrimTo(pool, 0);
    if (e != cudaSuccess) return kvh::cuda_fail(e);
    return KV_OK;
}

}  // extern "C"
