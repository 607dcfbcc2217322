// The learned bracket: a 2-64-64-2 MLP on (v, log x) that predicts the range [t0, t1] of
// Sec. 2.3, replacing Algorithms 1-3 on the hot path, with a per-pair check of g at the ends and
// a fallback to the plain FP64 bracket.
//
// Network (all parameters FP32 masters; inference reads W2 and h1 as BF16, FP32 accumulation):
//   a = asinh(v * in[0]) * in[1],  b = ln x * in[2] + in[3]
//   h1 = relu(W1 [a b] + b1),  h2 = relu(W2 h1 + b2),  y = W3 h2 + b3
//   L_k = y_k * out[2k] + out[2k+1];  t0 = max(t_ref - max(e^{L_0} - DELTA, 0), 0),
//   t1 = t_ref + max(e^{L_1} - DELTA, 0), with t_ref the peak of g.
// The network predicts log half-widths of the range about the peak; the peak itself comes from
// two FP32 Newton steps on g' from asinh(v/x) (g' is concave and <= 0 there, so the iterates
// fall monotonically onto the zero).
//
// Fast path per pair (kv_mlp_tc_kernel): MLP (hidden layer on the tensor cores) -> peak ->
// float-float offset g(t_ref) and constants -> check that g - g(t_ref) at both ends lies in
// [log eps - W, log eps] (the range is neither too narrow nor too wide), with a few FP32 Newton
// corrections of an end that misses -> FP32 bins.  Pairs that still fail are appended to a list
// and recomputed by a second kernel with the plain FP64 bracket, so one failing lane does not
// stall its warp on the slow path.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <vector>

#include "kv_bins.cuh"
#include "kv_bracket.cuh"
#include "kv_bracket_f32.cuh"
#include "kv_dfloat.cuh"
#include "kv_internal.h"

namespace {

constexpr int H = 64;
constexpr int NP = KV_MLP_NPARAMS;  // 4482
// offsets of W1[64][2], b1[64], W2[64][64], b2[64], W3[2][64], b3[2] in the parameter vector
constexpr int OFF_W1 = 0, OFF_B1 = 2 * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H,
              OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + 2 * H;
static_assert(OFF_B3 + 2 == NP, "parameter layout");
constexpr float DELTA = 1e-3f;
constexpr uint32_t kMagic = 0x4b564d4cu;  // handle tag
constexpr double kWindow = 12.0;          // nats of allowed over-width at each end

}  // namespace

struct kv_mlp {
    uint32_t magic;
    int device;
    float* params;           // [NP] FP32 masters
    float* adam_m;           // [NP]
    float* adam_s;           // [NP]
    unsigned short* w2h;     // [H*H] BF16 copy of W2
    int64_t step;            // Adam steps taken
    float in_scale[4];
    float out_scale[4];
    float* host;             // [NP] host copy of params (for the kernel-parameter weights)
    bool host_ok;            // host matches params (false after training until refreshed)
};

namespace {

using namespace kvd;

bool valid(const kv_mlp* h) { return h && h->magic == kMagic && h->params; }

uint64_t mix64(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t mix64_d(uint64_t z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

unsigned short bf16_bits_host(float f)
{
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7fffffffu) > 0x7f800000u) return (unsigned short)((u >> 16) | 0x40);  // NaN
    u += 0x7fffu + ((u >> 16) & 1u);  // round to nearest even
    return (unsigned short)(u >> 16);
}

int upload(kv_mlp* h, const float* host)
{
    KV_CUDA_TRY(cudaMemcpy(h->params, host, sizeof(float) * NP, cudaMemcpyHostToDevice));
    memcpy(h->host, host, sizeof(float) * NP);
    h->host_ok = true;
    std::vector<unsigned short> w2(H * H);
    for (int k = 0; k < H * H; ++k) w2[k] = bf16_bits_host(host[OFF_W2 + k]);
    KV_CUDA_TRY(cudaMemcpy(h->w2h, w2.data(), sizeof(unsigned short) * H * H, cudaMemcpyHostToDevice));
    return KV_OK;
}

int alloc_handle(kv_mlp** out)
{
    kv_mlp* h = new kv_mlp;
    memset(h, 0, sizeof(*h));
    h->magic = kMagic;
    cudaGetDevice(&h->device);
    cudaError_t e = cudaMalloc((void**)&h->params, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->adam_m, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->adam_s, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMalloc((void**)&h->w2h, sizeof(unsigned short) * H * H);
    if (e == cudaSuccess) e = cudaMemset(h->adam_m, 0, sizeof(float) * NP);
    if (e == cudaSuccess) e = cudaMemset(h->adam_s, 0, sizeof(float) * NP);
    h->host = new (std::nothrow) float[NP];
    if (e != cudaSuccess || !h->host) {
        cudaFree(h->params);
        cudaFree(h->adam_m);
        cudaFree(h->adam_s);
        cudaFree(h->w2h);
        delete[] h->host;
        delete h;
        return e != cudaSuccess ? kvh::cuda_fail(e) : KV_ERR_NOMEM;
    }
    // feature and output scaling: a = asinh(2 v) / asinh(400) * 2 spreads small orders (v < 1)
    // over a useful share of [0, 2] for v in [0, 200]; log10 x in [-4, 4] maps to [-1, 1]
    h->in_scale[0] = 2.0f;
    h->in_scale[1] = (float)(2.0 / asinh(400.0));
    h->in_scale[2] = (float)(1.0 / (4.0 * log(10.0)));
    h->in_scale[3] = 0.0f;
    h->out_scale[0] = 3.0f;
    h->out_scale[1] = -3.0f;
    h->out_scale[2] = 2.0f;
    h->out_scale[3] = -1.0f;
    *out = h;
    return KV_OK;
}

// ------------------------------------------------------------------ device pieces

// asinh(z) for z >= 0 as ln(z + sqrt(z^2 + 1)) with the approximate logarithm and reciprocal
// square root: absolute error a few 1e-7 (relative error grows as z -> 0, where the result is
// tiny).  Used for the network's order feature and the start of the peak search, neither of which
// needs more.
__device__ __forceinline__ float fast_asinh(float z)
{
    if (z > 1e18f) return __logf(2.0f * z);
    const float q = fmaf(z, z, 1.0f);
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q));
    return __logf(fmaf(q, r, z));
}

// The peak of g by STEPS FP32 Newton steps from the least of three upper bounds (0 when
// v^2 <= x).  On the fast path (one step: a second changed neither the fallback rate, 0 on the
// hard band and 3.7e-4 on the extreme range, nor the accuracy) its accuracy does not enter the
// results: the bins are exact relative to any reference point near the peak, and the range check
// tests the predicted ends themselves.  The training targets and the raw predictions, which are
// measured from the peak, take eight.  The steps use the approximate exponential, reciprocal and
// division.  The start is nudged up so that it stays on the side of the zero where g' <= 0
// despite the approximate asinh.
template <int STEPS>
__device__ __forceinline__ float peak_f32(float v, float x)
{
    if (!(v * v > x)) return 0.0f;
    const float q = __fdividef(v, x);
    const float a = fast_asinh(q);
    float t = a;
    // Where v a >= 1 both other bounds lie at or above a (at t = a, v^2 t / x >= q = sinh t), so
    // they are computed only where v a < 1 (each lane by its own test, so a pair's result does
    // not depend on the other pairs of its warp).
    if (v * a < 1.0f) {
        const float f = fast_asinh(fminf(q, v * q * a));
        const float d = fmaf(v, v, -x) * rcp_approx(30.0f * x);  // (r - 1)/30, v^2 - x rounded once
        const float e = d + 1.0f / 36.0f;
        float rs;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rs) : "f"(e));
        const float z = 60.0f * d * rcp_approx(fmaf(e, rs, 1.0f / 6.0f));
        float rz;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(rz) : "f"(z));
        t = fminf(fminf(a, f), z * rz);
    }
    t *= 1.0f + 0x1.0p-16f;
#pragma unroll
    for (int k = 0; k < STEPS; ++k) {
        float e2 = ex2_approx(-2.0f * LOG2E_F * v * t);
        float r = rcp_approx(1.0f + e2);
        float th = (1.0f - e2) * r;
        float sech2 = 4.0f * e2 * r * r;
        float et = ex2_approx(t * LOG2E_F);
        float eti = rcp_approx(et);
        float g1 = v * th - 0.5f * x * (et - eti);
        float g2 = v * v * sech2 - 0.5f * x * (et + eti);
        float tn = t - __fdividef(g1, g2);
        if (isfinite(tn)) t = fminf(fmaxf(tn, 0.0f), t);
    }
    return t;
}

struct MlpSmem {
    float w1[2 * H], b1[H], w2[H * H], b2[H], w3[2 * H], b3[2];
    float in_scale[4], out_scale[4];
};

// Forward pass of one pair on the CUDA cores: log half-widths (L0, L1).  W2 holds the BF16
// weights widened to FP32; h1 is rounded to BF16 as the tensor-core form sees it (b2, which the
// tensor-core form splits into two BF16 parts, stays FP32 here).
__device__ __forceinline__ void mlp_forward(const MlpSmem& s, float v, float x, float& L0, float& L1)
{
    const float a = fast_asinh(v * s.in_scale[0]) * s.in_scale[1];
    const float b = fmaf(__logf(x), s.in_scale[2], s.in_scale[3]);
    float h1[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
        float z = fmaf(s.w1[2 * i], a, fmaf(s.w1[2 * i + 1], b, s.b1[i]));
        h1[i] = __bfloat162float(__float2bfloat16_rn(fmaxf(z, 0.0f)));
    }
    float y0 = s.b3[0], y1 = s.b3[1];
    for (int j = 0; j < H; ++j) {
        const float4* row = reinterpret_cast<const float4*>(&s.w2[j * H]);
        float acc = s.b2[j];
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            float4 w = row[q];
            acc = fmaf(w.x, h1[4 * q], acc);
            acc = fmaf(w.y, h1[4 * q + 1], acc);
            acc = fmaf(w.z, h1[4 * q + 2], acc);
            acc = fmaf(w.w, h1[4 * q + 3], acc);
        }
        const float h2 = fmaxf(acc, 0.0f);
        y0 = fmaf(s.w3[j], h2, y0);
        y1 = fmaf(s.w3[H + j], h2, y1);
    }
    L0 = fmaf(y0, s.out_scale[0], s.out_scale[1]);
    L1 = fmaf(y1, s.out_scale[2], s.out_scale[3]);
}

__device__ void load_mlp_smem(MlpSmem& s, const kvh::MlpView& m)
{
    for (int k = threadIdx.x; k < 2 * H; k += blockDim.x) {
        s.w1[k] = m.w1[k];
        s.w3[k] = m.w3[k];
    }
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        s.b1[k] = m.b1[k];
        s.b2[k] = m.b2[k];
    }
    for (int k = threadIdx.x; k < H * H; k += blockDim.x)
        s.w2[k] = __uint_as_float(((uint32_t)m.w2h[k]) << 16);
    if (threadIdx.x < 2) s.b3[threadIdx.x] = m.b3[threadIdx.x];
    if (threadIdx.x < 4) {
        s.in_scale[threadIdx.x] = m.in_scale[threadIdx.x];
        s.out_scale[threadIdx.x] = m.out_scale[threadIdx.x];
    }
}

// The reference point of the bins: t_r = j ln2/128, the grid point nearest the peak estimate.
// On this grid e^{+-t_r} = 2^{+-(j >> 7)} 2^{+-(j & 127)/128} come exactly (as float-floats) from
// a 128-entry table, so the constants whose inputs cancel need no extended-precision exponential.
// |t_r - t_p| <= ln2/256 = 0.0027, and the bins are exact relative to any reference point.
constexpr int kGridBits = 7;
constexpr float kGridInv = 184.6649652337873f;         // 128 / ln2
constexpr float kGridStepHi = 5.415212363e-03f;        // ln2 / 128 rounded
constexpr float kGridStepLo = -1.488011103e-11f;       // ln2 / 128 - kGridStepHi

struct ExpTable {
    float4 e[1 << kGridBits];  // {hi, lo} of 2^{i/128}, then {hi, lo} of 2^{-i/128}
};

// The table on each device (read through the L1 cache), filled once per device.
__device__ float4 g_exp_tab[1 << kGridBits];

const ExpTable& exp_table()
{
    static const ExpTable t = [] {
        ExpTable r;
        for (int i = 0; i < (1 << kGridBits); ++i) {
            const double p = exp2((double)i / (1 << kGridBits)), m = exp2(-(double)i / (1 << kGridBits));
            const float ph = (float)p, mh = (float)m;
            r.e[i] = make_float4(ph, (float)(p - ph), mh, (float)(m - mh));
        }
        return r;
    }();
    return t;
}

int ensure_exp_table()
{
    static std::mutex mu;
    static bool ready[64];
    int dev = 0;
    KV_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return KV_ERR_ARG;
    std::lock_guard<std::mutex> lock(mu);
    if (!ready[dev]) {
        KV_CUDA_TRY(cudaMemcpyToSymbol(g_exp_tab, exp_table().e, sizeof(ExpTable)));
        ready[dev] = true;
    }
    return KV_OK;
}

// 2^k for |k| <= 126 (exact); larger |k| saturates (inf or the smallest normal).
__device__ __forceinline__ float pow2i(int k)
{
    return __int_as_float(min(max(k + 127, 1), 254) << 23);
}

// Per-pair constants of the FP32 bins at the reference point t_r, with the offset g(t_r) as a
// float-float (no FP64): G = v t_r + log1p(e^{-2 v t_r}) - ln 2 - x cosh t_r.
struct PeakConst {
    df G;
    BinsF b;
};

__device__ __forceinline__ PeakConst peak_constants(float v, float x, float tp, const float4* tab)
{
    PeakConst c;
    const float j = rintf(tp * kGridInv);
    const int ji = (int)j;
    const float4 T = __ldg(&tab[ji & ((1 << kGridBits) - 1)]);
    const float p2 = pow2i(ji >> kGridBits), p2i = pow2i(-(ji >> kGridBits));
    const df E{T.x * p2, T.y * p2}, Ei{T.z * p2i, T.w * p2i};  // e^{t_r}, e^{-t_r}
    df tr = two_prod(j, kGridStepHi);
    tr = fast_two_sum(tr.hi, fmaf(j, kGridStepLo, tr.lo));
    df u = two_prod(v, tr.hi);
    u = fast_two_sum(u.hi, fmaf(v, tr.lo, u.lo));
    // log1p(e^{-2u}) in [0, ln 2] from the approximate 2^x and log2 (absolute error ~2e-7)
    const float e2u = ex2_approx(-2.0f * LOG2E_F * u.hi);
    const float lu = lg2_approx(1.0f + e2u) * LN2_F;
    // e^{t_r} >= e^{-t_r}, so their high parts add and subtract exactly by FastTwoSum
    const df shr = df_sub_ordered(E, Ei);                  // 2 sinh t_r
    c.b.shp = 0.5f * (shr.hi + shr.lo);
    const df ch = df_mul_f(df_add_ordered(E, Ei), 0.5f * x);  // x cosh t_r
    const df sh = df_mul_f(shr, 0.5f * x);                 // x sinh t_r
    // G = (u - x cosh t_r) + (lu - ln 2): the two large terms cancel, so their high parts are
    // subtracted exactly (TwoSum) and everything else, at most a few units in size, is added
    // in FP32 (absolute error a few 1e-8, below lu's own).  The pair is not normalised: the
    // finish adds it to log(h S0) in that order (offset_plus).
    const df d = two_sum(u.hi, -ch.hi);
    c.G = df{d.hi, ((u.lo - ch.lo) + d.lo) + (lu - LN2_F)};
    c.b.v = v;
    c.b.u = u.hi;
    c.b.tp = tr.hi;
    // v - x sinh t_r: where the two are within a factor 2 of each other the first difference is
    // exact, elsewhere there is no cancellation; either way one rounding of the result
    c.b.c1 = (v - sh.hi) - sh.lo;
    c.b.ap = 0.5f * x * E.hi;
    c.b.am = 0.5f * x * Ei.hi;
    c.b.lu = lu;
    c.b.ep = E.hi;
    c.b.em = Ei.hi;
    c.b.e2u = e2u;
    c.b.xch = ch.hi + ch.lo;
    c.b.xsh = sh.hi + sh.lo;
    return c;
}

// log K = G + log(h S0) from the offset pair of peak_constants and y = log(h S0) in FP32: the
// high part and y are added exactly (TwoSum), then the small rest, so the result is rounded once
// (and carries y's own error, about 1e-7).
__device__ __forceinline__ float offset_plus(const df& G, float y)
{
    const df s = two_sum(G.hi, y);
    return s.hi + (s.lo + G.lo);
}

// The small per-unit weights of layers 1 and 3, passed by value with the launch so that the
// kernel reads them from the constant bank (operands of its FMAs) instead of shared memory.
struct MlpConst {
    float2 w1a[H / 2], w1b[H / 2], b1[H / 2];  // by unit pairs: {W1[u][0], W1[u+1][0]}, ...
    float2 w3[H];                              // {W3[0][j], W3[1][j]}
    float b3[2];
    float in_scale[4], out_scale[4];
};

struct MlpPathParams {
    const float* v;
    const float* x;
    float* logk;
    float* dv;
    float* dx;
    const float* go;
    uint8_t* status;
    float* d2v;  // second derivatives (may be NULL)
    float* dvx;
    float* d2x;
    int64_t n;
    int bins;
    float inv_bins;  // 1 / bins
    float log_eps;
    uint32_t* fb_list;
    uint32_t* fb_count;
    uint32_t* tile_ctr;  // tiles claimed beyond each CTA's first (zero at launch)
    kvh::MlpView mlp;
    MlpConst wc;
    int wait_limit;  // iterations of the per-tile wait for the tensor-core results
    int end_terms;   // bin n's terms from the range check (see pair_tail)
};

constexpr int kMlpBlock = 128;

__device__ __forceinline__ bool float_edge(float v, float x, float& lk, float& dv, float& dx)
{
    if (isnan(v) || isnan(x) || x < 0.0f) {
        lk = dv = dx = nanf("");
        return true;
    }
    if (x == 0.0f) {
        lk = INFINITY;
        dv = (v == 0.0f) ? 0.0f : copysignf(INFINITY, v);
        dx = -INFINITY;
        return true;
    }
    if (isinf(x)) {
        lk = -INFINITY;
        dv = copysignf(0.0f, v);
        dx = -1.0f;
        return true;
    }
    if (isinf(v)) {
        lk = INFINITY;
        dv = copysignf(INFINITY, v);
        dx = -INFINITY;
        return true;
    }
    return false;
}

// The check of a learned range: g - g(tr) at each end within [le - W, le] (le = log eps).  Both
// ends are evaluated together (paired instructions).  The left one is taken at t = 0 when the
// prediction puts it within the last kLeftZeroFrac of [0, t_r] (where the network cannot tell a
// range that starts at 0 from one that nearly does): a range may start at 0 with the integrand
// there anywhere above le - W (not too wide is all that is asked); otherwise the predicted end
// must lie inside the window, and then g(0) is below it too, since g rises on [0, t_p].  Only
// the pairs that miss take the slow part: a right end outside the window gets up to
// kNewtonSteps FP32 Newton steps towards the middle of the window (the slope of the same
// cancellation-free difference); a left end that missed starts at 0 if the integrand there is
// above le - W, else gets the same Newton steps from the predicted end.  Returns false when the
// pair must fall back to the plain bracket.  `end` receives the trapezoid terms of bin n
// (t = t1, weight 1/2) from the right end's last evaluation, in the units of the bins' sums:
// w = e^{g(t1) - g(t_r)} / 2, w t1 tanh(v t1) and -w x cosh(t1) log2 e.  At a passing end
// w <= e^{le} / 2, so the coarse evaluation's absolute error of about 1e-3 in the exponent
// changes S0 by less than 1e-3 e^{le} of its peak term.
constexpr float kLeftZeroFrac = 0.9f;
constexpr int kNewtonSteps = 3;
struct EndTerms {
    float w, w1, w2;
};

__device__ __forceinline__ bool check_range(const BinsF& b, float tr, float w0, float w1, float le,
                                            float lo, float& t0, float& t1, EndTerms& end)
{
    const float mid = le - 0.5f * (float)kWindow;
    auto in_window = [&](float d) { return d <= le && d >= lo; };
    float s1 = w1;
    const float s0p = -fminf(w0, tr);                     // the predicted left end
    const bool at0 = w0 >= kLeftZeroFrac * tr;            // take the left end at t = 0
    float s0 = at0 ? -tr : s0p;
    float2 e2p, esp, emsp;
    const float2 dp = delta_g_coarse2(b, make_float2(s1, s0), e2p, esp, emsp);
    float d1 = dp.x, e21 = e2p.x, es1 = esp.x, ems1 = emsp.x;
    const bool ok0 = at0 ? dp.y >= lo : in_window(dp.y);
    bool ok = in_window(d1) && ok0;
    if (!ok) {
        for (int k = 0; k < kNewtonSteps && !in_window(d1); ++k) {
            const float slope = delta_g_slope_f32(b, e21, es1, ems1);
            float sn = s1 - __fdividef(d1 - mid, slope);
            if (!(slope < 0.0f) || !isfinite(sn)) sn = d1 > le ? 2.0f * s1 : 0.5f * s1;
            s1 = fminf(fmaxf(sn, 0.25f * s1), 4.0f * s1);
            d1 = delta_g_coarse(b, s1, e21, es1, ems1);
        }
        bool okl = ok0;
        if (!ok0) {
            float e2, es, ems;
            const float dz = at0 ? dp.y : delta_g_coarse(b, -tr, e2, es, ems);
            if (dz >= lo) {
                s0 = -tr;  // the range starts at 0, where the integrand is not too small
                okl = true;
            } else if (s0p > -tr) {
                s0 = s0p;
                float d0 = delta_g_coarse(b, s0, e2, es, ems);  // again, for the slope's inputs
                for (int k = 0; k < kNewtonSteps && !in_window(d0) && s0 > -tr; ++k) {
                    const float slope = delta_g_slope_f32(b, e2, es, ems);
                    float sn = s0 - __fdividef(d0 - mid, slope);
                    if (!(slope > 0.0f) || !isfinite(sn)) sn = d0 > le ? 2.0f * s0 : 0.5f * s0;
                    s0 = fmaxf(fminf(sn, 0.25f * s0), 4.0f * s0);
                    if (s0 <= -tr) {
                        s0 = -tr;
                        d0 = dz;
                    } else {
                        d0 = delta_g_coarse(b, s0, e2, es, ems);
                    }
                }
                okl = in_window(d0) || (s0 <= -tr && d0 >= lo);
            }
        }
        ok = in_window(d1) && okl;
    }
    t1 = tr + s1;
    t0 = fmaxf(tr + s0, 0.0f);
    const float we = 0.5f * ex2_approx(d1 * LOG2E_F);
    end.w = we;
    end.w1 = we * (t1 * ((1.0f - e21) * rcp_approx(1.0f + e21)));
    end.w2 = (we * -LOG2E_F) * fmaf(b.ap, es1, b.am * ems1);
    return ok;
}

// ------------------------------------------------------------------ tensor-core hidden layer

// Shared-memory matrix descriptor of the tcgen05 MMA for a K-major tile without swizzling:
// 8-row x 16-byte core matrices stored contiguously (128 B); `lbo` = bytes between core
// matrices along K, `sbo` = bytes between 8-row groups; bits 46-48 hold the fixed value 0b001.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (row r, k) in a K-major tile of 64 columns: 8 core matrices per 8-row
// group (LBO = 128 B, SBO = 1024 B).
__device__ __forceinline__ int tile_off(int r, int k) { return (r >> 3) * 1024 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

// Offset of element (row r, k) in a K-major slice of 16 columns (two core matrices per 8-row
// group: LBO = 128 B, SBO = 256 B).
__device__ __forceinline__ int slice_off(int r, int k) { return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

struct TcSmem {
    unsigned char a[128 * H * 2];    // h1, then h2, of the CTA's 128 pairs (BF16, K-major)
    unsigned char b[H * H * 2];      // W2 (BF16): row = output unit, K = input unit
    unsigned char bb[H * 16 * 2];    // B of layer 2's extra K slice: k = 0, 1 hold b2 split hi + lo
    unsigned char ones[8 * 16 * 2];  // A of that slice, one 8-row group read by every group: 1, 1, 0...
    uint64_t mbar;
    uint32_t next_tile;  // the tile thread 0 claimed for the CTA's next trip
    uint32_t tmem;
};

__device__ __forceinline__ unsigned short bf16_bits(float f) { return __bfloat16_as_ushort(__float2bfloat16_rn(f)); }
__device__ __forceinline__ float bf16_value(unsigned short h) { return __uint_as_float(((uint32_t)h) << 16); }

// One tcgen05.mma (BF16 inputs, FP32 accumulators in TMEM); acc = 0 overwrites the accumulators.
__device__ __forceinline__ void mma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(bar)));
}

// Waits (bounded) for the mbarrier phase `phase` to complete; false if the limit ran out.
constexpr int kWaitLimit = 1 << 22;
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t phase, int limit = kWaitLimit)
{
    uint32_t done = 0;
    for (int it = 0; it < limit && !done; ++it)
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(phase));
    return done != 0;
}

__device__ __forceinline__ void tmem_ld16(uint32_t addr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
}

// Makes this thread's shared-memory tile writes visible to the tensor cores and orders them
// (and earlier TMEM reads) before the MMA that one thread issues after the barrier.
__device__ __forceinline__ void sync_for_mma()
{
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
}

constexpr uint32_t kTmemCols = 64;

// The rest of a pair once its range is known (or not: ok = false), shared by the fast path and
// the FP32 plain-bracket path.  A regular pair whose range failed goes to the fallback list and
// runs the bins on a placeholder range (results discarded), so that every lane of the warp runs
// the same straight-line code into the bins.  Then FP32 bins, the finish with the float-float
// offset, and the stores.  An edge pair's results are taken from (v, x) again after the bins, so
// that they hold no registers during them.
// `end`: bin n's terms from the range check (check_range), used while log eps <= kEndTermLogEps
// and n >= kEndTermMinBins, where their coarse exponent cannot matter (with four or more bins one
// of them lies within two widths of the peak, so S0 >= e^-2 while the end term is below e^le / 2);
// otherwise bin n is one of the bins.  kv_debug_set_end_terms(0) turns them off (tests).
constexpr float kEndTermLogEps = -12.0f;
constexpr int kEndTermMinBins = 4;

template <bool DERIV, bool D2, bool COMP = true>
__device__ __forceinline__ void pair_tail(const MlpPathParams& p, int64_t i, bool active, bool edge, bool ok,
                                          float v, float x, PeakConst& c, float t0, float t1,
                                          uint8_t ok_status = KV_PAIR_OK, const EndTerms* end = nullptr)
{
    const float tr = c.b.tp;
    const bool regular = active && !edge;
    if (regular && !ok) {
        uint32_t k = atomicAdd(p.fb_count, 1u);
        p.fb_list[k] = (uint32_t)i;
    }
    if (!ok) {  // keep the bins of a failed lane finite; its results are not stored
        t0 = fmaxf(tr - 1.0f, 0.0f);
        t1 = tr + 1.0f;
    }
    __syncwarp();
    c.b.s0 = t0 - c.b.tp;
    c.b.h = (t1 - t0) * p.inv_bins;
    c.b.n = p.bins;
    float S0, S1, S2;
    float d2v = 0.0f, dvx = 0.0f, d2x = 0.0f;
    if constexpr (D2) {
        // second derivatives (and the first ones) from the shifted sums
        const Sums2<float> m = sums2_f32<1, true>(c.b, 0);
        S0 = m.s0;
        const float ar = tr * (c.b.u < TANH_SERIES_MAX ? tanh_small(c.b.u)
                                                        : (1.0f - c.b.e2u) / (1.0f + c.b.e2u));
        float fdv, fdx;
        moments_finish<float>(m, ar, 0.5f * (c.b.ep + c.b.em), fdv, fdx, d2v, dvx, d2x);
        S1 = fdv * S0;
        S2 = -fdx * S0;
        if (v == 0.0f) dvx = 0.0f;
        if (v < 0.0f) dvx = -dvx;
        if (edge) d2v = dvx = d2x = (isinf(x) && x > 0.0f) ? 0.0f : nanf("");
    } else {
        if (end)
            sums_f32<1, DERIV, true, COMP>(c.b, 0, S0, S1, S2,
                                           p.end_terms && p.log_eps <= kEndTermLogEps && p.bins >= kEndTermMinBins,
                                           end->w, end->w1, end->w2);
        else
            sums_f32<1, DERIV, true, COMP>(c.b, 0, S0, S1, S2);
    }
    float lk = 0.0f, dv = 0.0f, dx = 0.0f;
    if (regular && ok) {
        // log(h S0) from the approximate log2 (absolute error about 1e-7)
        lk = offset_plus(c.G, lg2_approx(c.b.h * S0) * LN2_F);
        const float r = rcp_approx(S0);
        dv = DERIV ? copysignf(S1 * r, v) : 0.0f;
        if (v == 0.0f) dv = 0.0f;
        dx = DERIV ? -(S2 * r) : 0.0f;
    }
    if (__any_sync(0xffffffffu, edge)) {  // edge pairs are rare: only their warps take this
        float le, de, xe;
        if (float_edge(v, x, le, de, xe)) {
            lk = le;
            dv = de;
            dx = xe;
        }
    }
    if (active && (edge || ok)) {
        if (p.go) {
            dv *= p.go[i];
            dx *= p.go[i];
        }
        if (p.logk) p.logk[i] = lk;
        if (p.dv) p.dv[i] = dv;
        if (p.dx) p.dx[i] = dx;
        if (p.status) p.status[i] = edge ? KV_PAIR_EDGE : ok_status;
        if constexpr (D2) {
            if (p.d2v) p.d2v[i] = d2v;
            if (p.dvx) p.dvx[i] = dvx;
            if (p.d2x) p.d2x[i] = d2x;
        }
    }
}

// The plain bracket in FP32 (Algorithms 1-3, kv_bracket_f32.cuh) followed by the fast path's
// offset at a grid point, bins and finish: the paper's 32-bit variant of the whole path, one pair
// per thread.  Pairs whose FP32 range is not a finite range go to the FP64 fallback.  COMP: the
// bins' block sums compensated (more than kPlainSumsMaxBins bins) or plain.
template <bool DERIV, bool D2 = false, bool COMP = true>
__global__ void __launch_bounds__(kMlpBlock) kv_plain_f32_kernel(MlpPathParams p, int max_iter)
{
    const int t = threadIdx.x;
    for (int64_t base = (int64_t)blockIdx.x * kMlpBlock; base < p.n; base += (int64_t)gridDim.x * kMlpBlock) {
        const int64_t i = base + t;
        const bool active = i < p.n;
        const float v = active ? p.v[i] : 1.0f;
        const float x = active ? p.x[i] : 1.0f;
        float lk, dv, dx;
        const bool edge = float_edge(v, x, lk, dv, dx);
        const float va = edge ? 1.0f : fabsf(v);
        const float xa = edge ? 1.0f : x;
        bool capped = false;
        const float tp = peak_alg12_f32(va, xa, max_iter, capped);
        PeakConst c = peak_constants(va, xa, tp, g_exp_tab);
        float t0, t1;
        const bool ok = range_alg12_f32(c.b, tp, p.log_eps, max_iter, t0, t1, capped);
        pair_tail<DERIV, D2, COMP>(p, i, active, edge, ok, v, x, c, t0, t1, capped ? KV_PAIR_RANGE_CAP : KV_PAIR_OK);
    }
}

// The fast path with the hidden layer on the tensor cores.  Each CTA of 128 threads takes a tile
// of 128 pairs per trip (one per thread; the tiles after the first claimed from a global
// counter): layer 1 on the CUDA cores writes h1 as BF16 into a K-major shared tile; one
// elected thread issues five tcgen05.mma (M = 128, N = 64, K = 16; the fifth multiplies a column
// of ones by b2 split into two BF16 parts, so the bias comes out of the tensor cores too) into 64
// TMEM columns and commits them to an mbarrier; after the wait, warp w reads TMEM lanes
// 32w..32w+31 (its own pairs' rows) and finishes layer 3 in registers.  (Layer 3 on the tensor
// cores as well measured slower, also with its MMAs overlapped with the previous tile's bins: the
// second round trip and barrier per tile cost about what the 128 FMAs save.)  A wait that does not
// finish within its limit sends the CTA's remaining pairs and every tile still unclaimed to the
// fallback list (correct, slower) instead of hanging.  COMP: the bins' block sums compensated
// (more than kPlainSumsMaxBins bins) or plain.
template <bool DERIV, bool D2 = false, bool COMP = true>
__global__ void __launch_bounds__(kMlpBlock, D2 ? 6 : 8) kv_mlp_tc_kernel(MlpPathParams p)
{
    __shared__ __align__(1024) TcSmem sm;
    const int t = threadIdx.x;
    const int warp = t >> 5;
    // W2 into its K-major tile, eight BF16 (one 16-byte core-matrix row) per load and store
    for (int q = t; q < H * H / 8; q += kMlpBlock) {
        const int k = 8 * q;
        *reinterpret_cast<uint4*>(sm.b + tile_off(k / H, k % H)) = __ldg(reinterpret_cast<const uint4*>(p.mlp.w2h) + q);
    }
    if (t < H) {  // row t of the bias slice: b2 = hi + lo in BF16 at k = 0, 1, zeros elsewhere
        const float b2 = p.mlp.b2[t];
        const unsigned short hi = bf16_bits(b2);
        const unsigned short lo = bf16_bits(b2 - bf16_value(hi));
        *reinterpret_cast<uint4*>(sm.bb + slice_off(t, 0)) = make_uint4((uint32_t)hi | ((uint32_t)lo << 16), 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(sm.bb + slice_off(t, 8)) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (t < 8 * 16)
        *reinterpret_cast<unsigned short*>(sm.ones + slice_off(t >> 4, t & 15)) = (t & 15) < 2 ? 0x3F80 : 0;
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem;
    // instruction descriptor: FP32 accumulators, BF16 A and B, both K-major, M = 128, N = 64
    const uint32_t idesc2 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(H >> 3) << 17) | ((128u >> 4) << 24);
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);  // this warp's TMEM lanes
    const float lo_ok = p.log_eps - (float)kWindow;
    uint32_t phase = 0;
    bool aborted = false;
    // Tiles are handed out dynamically: each CTA starts with tile blockIdx.x and claims every
    // further tile from a global counter, one trip ahead (thread 0, published to the CTA at the
    // tile's first barrier).  The CTAs resident on one SM get unequal shares of its issue slots,
    // so a fixed share of tiles per CTA leaves the SM with fewer and fewer CTAs towards the end.
    // (tile indices fit 32 bits: the path takes at most 2^32 pairs)
    const uint32_t ntiles = (uint32_t)((p.n + kMlpBlock - 1) / kMlpBlock);
    uint32_t tile = blockIdx.x;
    uint32_t next = ntiles;
    // this thread's inputs of the next tile are loaded one tile ahead, so their DRAM latency
    // overlaps the current tile's work
    float v_next = (int64_t)tile * kMlpBlock + t < p.n ? __ldcs(p.v + (int64_t)tile * kMlpBlock + t) : 1.0f;
    float x_next = (int64_t)tile * kMlpBlock + t < p.n ? __ldcs(p.x + (int64_t)tile * kMlpBlock + t) : 1.0f;
    for (; tile < ntiles; tile = next) {
        const int64_t i = (int64_t)tile * kMlpBlock + t;
        const bool active = i < p.n;
        const float v = v_next;
        const float x = x_next;
        uint32_t claimed = 0;
        if (t == 0) claimed = atomicAdd(p.tile_ctr, 1u);
        float lk, dv, dx;
        const bool edge = float_edge(v, x, lk, dv, dx);
        const float va = edge ? 1.0f : fabsf(v);
        const float xa = edge ? 1.0f : x;
        // layer 1 -> BF16 row t of the A tile
        {
            const float a = fast_asinh(va * p.wc.in_scale[0]) * p.wc.in_scale[1];
            const float b = fmaf(__logf(xa), p.wc.in_scale[2], p.wc.in_scale[3]);
#pragma unroll
            for (int c = 0; c < H / 8; ++c) {
                uint32_t packed[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int u = 4 * c + q;  // units 2u, 2u + 1
                    const float2 z = fma2(p.wc.w1a[u], f2(a), fma2(p.wc.w1b[u], f2(b), p.wc.b1[u]));
                    // relu and round to BF16 in one conversion (unit 2u in the low half)
                    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(packed[q]) : "f"(z.y), "f"(z.x));
                }
                *reinterpret_cast<uint4*>(sm.a + tile_off(t, 8 * c)) = make_uint4(packed[0], packed[1], packed[2], packed[3]);
            }
        }
        if (t == 0) sm.next_tile = min(gridDim.x + claimed, ntiles);
        sync_for_mma();
        next = sm.next_tile;
        if ((int64_t)next * kMlpBlock + t < p.n) {
            v_next = __ldcs(p.v + (int64_t)next * kMlpBlock + t);
            x_next = __ldcs(p.x + (int64_t)next * kMlpBlock + t);
        }
        if (t == 0) {  // layer 2: h1 W2^T + 1 (b2 hi + b2 lo)
#pragma unroll
            for (int kk = 0; kk < H / 16; ++kk)
                mma_bf16(tmem, umma_desc(smem_addr(sm.a) + kk * 256, 128, 1024),
                         umma_desc(smem_addr(sm.b) + kk * 256, 128, 1024), idesc2, kk > 0);
            mma_bf16(tmem, umma_desc(smem_addr(sm.ones), 128, 0), umma_desc(smem_addr(sm.bb), 128, 256), idesc2, 1);
            mma_commit(&sm.mbar);
        }
        if (__syncthreads_or(!mbar_wait(&sm.mbar, phase, p.wait_limit))) {
            aborted = true;
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        // layer 3 from this thread's row of the layer 2 accumulators (TMEM lane t)
        float2 y = make_float2(p.wc.b3[0], p.wc.b3[1]);
#pragma unroll
        for (int c = 0; c < H; c += 16) {
            uint32_t r[16];
            tmem_ld16(lane_base + (uint32_t)c, r);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
            for (int j = 0; j < 16; ++j) y = fma2(p.wc.w3[c + j], f2(fmaxf(__uint_as_float(r[j]), 0.0f)), y);
        }
        const float y0 = y.x, y1 = y.y;
        asm volatile("tcgen05.fence::before_thread_sync;");
        // Every lane runs the same straight-line code from here (edge and inactive lanes on
        // their placeholder inputs), so the warp is converged when it enters the bins:
        // otherwise lanes that took a different path through the check would run the bins
        // separately, once per group.
        const float L0 = fmaf(y0, p.wc.out_scale[0], p.wc.out_scale[1]);
        const float L1 = fmaf(y1, p.wc.out_scale[2], p.wc.out_scale[3]);
        const float tp = peak_f32<1>(va, xa);
        PeakConst c = peak_constants(va, xa, tp, g_exp_tab);
        const float tr = c.b.tp;  // the grid point next to tp: the bins' reference
        // the predicted range [tp - w0, tp + w1] as distances below and above tr
        const float w0 = fmaxf(fmaxf(__expf(L0) - DELTA, 0.0f) - (tp - tr), 0.0f);
        const float w1 = fmaxf(fmaxf(__expf(L1) - DELTA, 0.0f) + (tp - tr), 1e-6f * (1.0f + tr));
        float t0, t1;
        EndTerms et;
        const bool ok = check_range(c.b, tr, w0, w1, p.log_eps, lo_ok, t0, t1, et);
        pair_tail<DERIV, D2, COMP>(p, i, active, edge, ok, v, x, c, t0, t1, KV_PAIR_OK, D2 ? nullptr : &et);
    }
    if (aborted) {
        // a tensor-core wait ran out: this tile, the one claimed for the next trip and every tile
        // still unclaimed go to the fallback pass
        for (;;) {
            const int64_t i = (int64_t)tile * kMlpBlock + t;
            if (i < p.n) {
                uint32_t k = atomicAdd(p.fb_count, 1u);
                p.fb_list[k] = (uint32_t)i;
            }
            tile = next;
            if (tile >= ntiles) break;
            __syncthreads();
            if (t == 0) sm.next_tile = min(gridDim.x + atomicAdd(p.tile_ctr, 1u), ntiles);
            __syncthreads();
            next = sm.next_tile;
        }
        mbar_wait(&sm.mbar, phase);  // let the MMA in flight finish before its TMEM goes (full bound)
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// Resident CTAs per SM for a tensor-core kernel, capped at 8 (512 TMEM columns / 64).  The
// kernel prefers the largest shared-memory carve-out; the occupancy query then sees the
// configuration the launch gets (with the default preference it reported one CTA per SM).
template <typename K>
int tc_blocks_per_sm(K kernel)
{
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                         (int)cudaSharedmemCarveoutMaxShared);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kMlpBlock, 0) != cudaSuccess)
        per_sm = 0;
    if (per_sm < 2) {
        // from the kernel's registers and shared memory against the SM's budgets
        cudaFuncAttributes fa;
        int regs_sm = 65536, smem_sm = 0;
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        if (cudaFuncGetAttributes(&fa, kernel) == cudaSuccess) {
            const int regs = ((fa.numRegs + 7) / 8) * 8 * kMlpBlock;
            const int by_regs = regs > 0 ? regs_sm / regs : 1;
            const int by_smem = smem_sm / (int)(fa.sharedSizeBytes + 1024);
            per_sm = by_regs < by_smem ? by_regs : by_smem;
        }
    }
    cudaGetLastError();  // the queries must not leave an error behind for the launch check
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    if (dev >= 0 && dev < 64) cache[dev] = per_sm;
    return per_sm;
}

struct FallbackParams {
    MlpPathParams p;
    double log_eps;
    int max_iter;
    int flags;    // kv_args.flags (the FP64 bracket's peak start)
    int try_f32;  // first try the plain bracket in FP32 (the learned path's failures)
    unsigned long long* fallback_total;
};

// The pairs whose learned bracket failed its check: the plain bracket in FP32 first (Algorithms
// 1-3, kv_bracket_f32.cuh, with the fast path's offset and bins), and where that does not give a
// finite range (or for the FP32 path's own failures), the plain FP64 bracket and FP64 constants,
// then the same FP32 bins.
template <bool DERIV, bool D2 = false>
__global__ void __launch_bounds__(kMlpBlock) kv_fallback_kernel(FallbackParams f)
{
    const MlpPathParams& p = f.p;
    const uint32_t cnt = *p.fb_count;
    if (blockIdx.x == 0 && threadIdx.x == 0 && f.fallback_total)
        atomicAdd(f.fallback_total, (unsigned long long)cnt);
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        const int64_t i = p.fb_list[k];
        {
            // an edge pair is on the list only when a fast-path CTA gave up its tensor-core wait
            // and handed over all its remaining pairs
            float lk, dv, dx;
            const float ve = p.v[i], xe = p.x[i];
            if (float_edge(ve, xe, lk, dv, dx)) {
                if (p.go) {
                    dv *= p.go[i];
                    dx *= p.go[i];
                }
                if (p.logk) p.logk[i] = lk;
                if (p.dv) p.dv[i] = dv;
                if (p.dx) p.dx[i] = dx;
                if (p.status) p.status[i] = KV_PAIR_EDGE;
                if constexpr (D2) {
                    const float e = (isinf(xe) && xe > 0.0f) ? 0.0f : nanf("");
                    if (p.d2v) p.d2v[i] = e;
                    if (p.dvx) p.dvx[i] = e;
                    if (p.d2x) p.d2x[i] = e;
                }
                continue;
            }
        }
        if (f.try_f32) {
            const float vf = p.v[i], xf = p.x[i];
            const float va = fabsf(vf);
            bool capped = false;
            const float tp = peak_alg12_f32(va, xf, f.max_iter, capped);
            PeakConst c = peak_constants(va, xf, tp, g_exp_tab);
            float t0, t1;
            if (range_alg12_f32(c.b, tp, p.log_eps, f.max_iter, t0, t1, capped)) {
                c.b.s0 = t0 - c.b.tp;
                c.b.h = (t1 - t0) * p.inv_bins;
                c.b.n = p.bins;
                float S0, S1, S2, d2v = 0.0f, dvx = 0.0f, d2x = 0.0f;
                if constexpr (D2) {
                    const Sums2<float> m = sums2_f32<1>(c.b, 0);
                    S0 = m.s0;
                    const float tr = c.b.tp;
                    const float ar = tr * (c.b.u < TANH_SERIES_MAX ? tanh_small(c.b.u)
                                                                    : (1.0f - c.b.e2u) / (1.0f + c.b.e2u));
                    float fdv, fdx;
                    moments_finish<float>(m, ar, 0.5f * (c.b.ep + c.b.em), fdv, fdx, d2v, dvx, d2x);
                    S1 = fdv * S0;
                    S2 = -fdx * S0;
                    if (vf == 0.0f) dvx = 0.0f;
                    if (vf < 0.0f) dvx = -dvx;
                } else {
                    sums_f32<1, DERIV>(c.b, 0, S0, S1, S2);
                }
                const float lkf = offset_plus(c.G, lg2_approx(c.b.h * S0) * LN2_F);
                const float r = rcp_approx(S0);
                float dv = DERIV ? copysignf(S1 * r, vf) : 0.0f;
                if (vf == 0.0f) dv = 0.0f;
                float dx = DERIV ? -(S2 * r) : 0.0f;
                if (p.go) {
                    dv *= p.go[i];
                    dx *= p.go[i];
                }
                if (p.logk) p.logk[i] = lkf;
                if (p.dv) p.dv[i] = dv;
                if (p.dx) p.dx[i] = dx;
                if (p.status) p.status[i] = KV_PAIR_FALLBACK | (capped ? KV_PAIR_RANGE_CAP : 0);
                if constexpr (D2) {
                    if (p.d2v) p.d2v[i] = d2v;
                    if (p.dvx) p.dvx[i] = dvx;
                    if (p.d2x) p.d2x[i] = d2x;
                }
                continue;
            }
        }
        const double v = (double)p.v[i], x = (double)p.x[i];
        const double va = fabs(v);
        BracketD br = bracket_f64(va, x, f.log_eps, f.max_iter, (f.flags & KV_FLAG_PEAK_ANALYTIC_START) != 0);
        const double ep = exp(br.tp), em = 1.0 / ep;
        const double u = va * br.tp;
        const double h = (br.t1 - br.t0) / p.bins;
        BinsF b;
        b.s0 = (float)(br.t0 - br.tp);
        b.h = (float)h;
        b.v = (float)va;
        b.u = (float)u;
        b.tp = (float)br.tp;
        b.c1 = (float)(va - x * 0.5 * (ep - em));
        b.ap = (float)(x * 0.5 * ep);
        b.am = (float)(x * 0.5 * em);
        b.lu = (float)log1p(exp(-2.0 * u));
        b.ep = (float)ep;
        b.em = (float)em;
        b.xch = (float)(x * cosh(br.tp));
        b.xsh = (float)(x * sinh(br.tp));
        b.n = p.bins;
        float S0, S1, S2;
        if constexpr (D2) {
            const double e2u = exp(-2.0 * u);
            b.e2u = (float)e2u;
            b.shp = (float)sinh(br.tp);
            const Sums2<float> m = sums2_f32<1>(b, 0);
            float fdv, fdx, d2v, dvx, d2x;
            moments_finish<float>(m, (float)(br.tp * ((1.0 - e2u) / (1.0 + e2u))), (float)cosh(br.tp), fdv,
                                  fdx, d2v, dvx, d2x);
            S0 = m.s0;
            S1 = fdv * S0;
            S2 = -fdx * S0;
            if (v == 0.0) dvx = 0.0f;
            if (v < 0.0) dvx = -dvx;
            if (p.d2v) p.d2v[i] = d2v;
            if (p.dvx) p.dvx[i] = dvx;
            if (p.d2x) p.d2x[i] = d2x;
        } else {
            sums_f32<1, DERIV>(b, 0, S0, S1, S2);
        }
        double lk = br.G + (double)logf(b.h * S0);
        float r = 1.0f / S0;
        double dv = DERIV ? copysign((double)(S1 * r), v) : 0.0;
        if (v == 0.0) dv = 0.0;
        double dx = DERIV ? -(double)(S2 * r) : 0.0;
        if (p.go) {
            dv *= (double)p.go[i];
            dx *= (double)p.go[i];
        }
        if (p.logk) p.logk[i] = (float)lk;
        if (p.dv) p.dv[i] = (float)dv;
        if (p.dx) p.dx[i] = (float)dx;
        if (p.status) p.status[i] = KV_PAIR_FALLBACK | (br.capped ? KV_PAIR_RANGE_CAP : 0);
    }
}

// ------------------------------------------------------------------ raw predictions

__global__ void __launch_bounds__(kMlpBlock) kv_predict_kernel(kvh::MlpView m, const float* v,
                                                               const float* x, float* t0,
                                                               float* t1, int64_t n)
{
    __shared__ MlpSmem sm;
    load_mlp_smem(sm, m);
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float va = fabsf(v[i]);
        float L0, L1;
        mlp_forward(sm, va, x[i], L0, L1);
        const float tr = peak_f32<8>(va, x[i]);
        t0[i] = fmaxf(tr - fmaxf(__expf(L0) - DELTA, 0.0f), 0.0f);
        t1[i] = tr + fmaxf(__expf(L1) - DELTA, 0.0f);
    }
}

// ------------------------------------------------------------------ training

constexpr int kTrainBlock = 128;  // samples per block

struct GradArgs {
    const float* params;
    const double* v;
    const double* x;
    const double* t0;
    const double* t1;
    int64_t n;
    int batch;
    int64_t step;
    uint64_t seed;
    int sequential;  // 1: sample k of the batch is element k (no shuffling)
    float* partial;  // [gridDim.x][NP + 1]
    float in_scale[4];
    float out_scale[4];
};

// Per-block forward and backward of 128 samples, then the block's share of the parameter
// gradients (and of the loss) as sums over its samples, written to partial[block].
__global__ void __launch_bounds__(kTrainBlock) mlp_grad_kernel(GradArgs g)
{
    // per-sample vectors are stored unit-major with a padded stride (X[i * kPad + sample]), so
    // that both the per-sample loops and the per-parameter sums over samples are conflict-free
    constexpr int kPad = kTrainBlock + 1;
    extern __shared__ float sh[];
    float* W = sh;                              // [NP]
    float* F = W + NP + 2;                      // [128][2] features
    float* DY = F + 2 * kTrainBlock;            // [128][2]
    float* LS = DY + 2 * kTrainBlock;           // [128] per-sample loss
    float* H1 = LS + kTrainBlock;               // [64][kPad]
    float* H2 = H1 + H * kPad;                  // [64][kPad]
    float* DZ2 = H2 + H * kPad;                 // [64][kPad]
    float* DZ1 = DZ2 + H * kPad;                // [64][kPad]
    for (int k = threadIdx.x; k < NP; k += blockDim.x) W[k] = g.params[k];
    __syncthreads();
    const int s = threadIdx.x;
    const int64_t kb = (int64_t)blockIdx.x * kTrainBlock + s;
    const bool active = kb < g.batch;
    struct Col {
        float* p;
        __device__ float& operator[](int i) const { return p[i * kPad]; }
    };
    Col h1{H1 + s}, h2{H2 + s}, dz2{DZ2 + s}, dz1{DZ1 + s};
    if (active) {
        const int64_t idx = g.sequential ? kb : (int64_t)(mix64_d(g.seed + (uint64_t)g.step * g.batch + kb) % (uint64_t)g.n);
        const double vd = fabs(g.v[idx]), xd = g.x[idx];
        const float a = (float)(asinh(vd * g.in_scale[0]) * g.in_scale[1]);
        const float b = (float)(log(xd) * g.in_scale[2] + g.in_scale[3]);
        F[2 * s] = a;
        F[2 * s + 1] = b;
        for (int i = 0; i < H; ++i)
            h1[i] = fmaxf(fmaf(W[OFF_W1 + 2 * i], a, fmaf(W[OFF_W1 + 2 * i + 1], b, W[OFF_B1 + i])), 0.0f);
        float y0 = W[OFF_B3], y1 = W[OFF_B3 + 1];
        for (int j = 0; j < H; ++j) {
            float acc = W[OFF_B2 + j];
            for (int i = 0; i < H; ++i) acc = fmaf(W[OFF_W2 + j * H + i], h1[i], acc);
            float z = fmaxf(acc, 0.0f);
            h2[j] = z;
            y0 = fmaf(W[OFF_W3 + j], z, y0);
            y1 = fmaf(W[OFF_W3 + H + j], z, y1);
        }
        // targets: log half-widths about the peak
        const float tr = peak_f32<8>((float)vd, (float)xd);
        const double T0 = (log(fmax((double)tr - g.t0[idx], 0.0) + (double)DELTA) - g.out_scale[1]) / g.out_scale[0];
        const double T1 = (log(fmax(g.t1[idx] - (double)tr, 0.0) + (double)DELTA) - g.out_scale[3]) / g.out_scale[2];
        const float r0 = y0 - (float)T0, r1 = y1 - (float)T1;
        LS[s] = 0.5f * (r0 * r0 + r1 * r1);
        const float dy0 = r0 / (float)g.batch, dy1 = r1 / (float)g.batch;
        DY[2 * s] = dy0;
        DY[2 * s + 1] = dy1;
        for (int j = 0; j < H; ++j)
            dz2[j] = h2[j] > 0.0f ? fmaf(W[OFF_W3 + j], dy0, W[OFF_W3 + H + j] * dy1) : 0.0f;
        for (int i = 0; i < H; ++i) {
            float acc = 0.0f;
            for (int j = 0; j < H; ++j) acc = fmaf(W[OFF_W2 + j * H + i], dz2[j], acc);
            dz1[i] = h1[i] > 0.0f ? acc : 0.0f;
        }
    } else {
        F[2 * s] = F[2 * s + 1] = 0.0f;
        DY[2 * s] = DY[2 * s + 1] = 0.0f;
        LS[s] = 0.0f;
        for (int i = 0; i < H; ++i) h1[i] = h2[i] = dz2[i] = dz1[i] = 0.0f;
    }
    __syncthreads();
    float* out = g.partial + (int64_t)blockIdx.x * (NP + 1);
    for (int q = threadIdx.x; q <= NP; q += blockDim.x) {
        float acc = 0.0f;
        if (q < OFF_B1) {                       // W1[i][c]
            const int i = q / 2, c = q % 2;
            for (int t = 0; t < kTrainBlock; ++t) acc = fmaf(DZ1[i * kPad + t], F[2 * t + c], acc);
        } else if (q < OFF_W2) {                // b1[i]
            const int i = q - OFF_B1;
            for (int t = 0; t < kTrainBlock; ++t) acc += DZ1[i * kPad + t];
        } else if (q < OFF_B2) {                // W2[j][i]
            const int j = (q - OFF_W2) / H, i = (q - OFF_W2) % H;
            for (int t = 0; t < kTrainBlock; ++t) acc = fmaf(DZ2[j * kPad + t], H1[i * kPad + t], acc);
        } else if (q < OFF_W3) {                // b2[j]
            const int j = q - OFF_B2;
            for (int t = 0; t < kTrainBlock; ++t) acc += DZ2[j * kPad + t];
        } else if (q < OFF_B3) {                // W3[k][j]
            const int k = (q - OFF_W3) / H, j = (q - OFF_W3) % H;
            for (int t = 0; t < kTrainBlock; ++t) acc = fmaf(DY[2 * t + k], H2[j * kPad + t], acc);
        } else if (q < NP) {                    // b3[k]
            const int k = q - OFF_B3;
            for (int t = 0; t < kTrainBlock; ++t) acc += DY[2 * t + k];
        } else {                                // loss share
            for (int t = 0; t < kTrainBlock; ++t) acc += LS[t];
            acc /= (float)g.batch;
        }
        out[q] = acc;
    }
}

struct ReduceArgs {
    const float* partial;
    int nblocks;
    float* params;
    float* m;
    float* s;
    unsigned short* w2h;
    int update;
    float lr, beta1, beta2, eps;
    float bc1, bc2;          // 1 - beta^t
    float* loss_out;         // [1] slot for this step, or NULL
    double* loss_d;          // or NULL
    float* grads_out;        // [NP] or NULL
};

// Sum of the block partials (fixed order) and, optionally, the Adam update of every parameter.
__global__ void mlp_reduce_kernel(ReduceArgs r)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q > NP) return;
    double acc = 0.0;
    for (int b = 0; b < r.nblocks; ++b) acc += (double)r.partial[(int64_t)b * (NP + 1) + q];
    const float gq = (float)acc;
    if (q == NP) {
        if (r.loss_out) *r.loss_out = gq;
        if (r.loss_d) *r.loss_d = acc;
        return;
    }
    if (r.grads_out) r.grads_out[q] = gq;
    if (!r.update) return;
    const float m = r.beta1 * r.m[q] + (1.0f - r.beta1) * gq;
    const float s = r.beta2 * r.s[q] + (1.0f - r.beta2) * gq * gq;
    r.m[q] = m;
    r.s[q] = s;
    const float w = r.params[q] - r.lr * (m / r.bc1) / (sqrtf(s / r.bc2) + r.eps);
    r.params[q] = w;
    if (q >= OFF_W2 && q < OFF_B2) r.w2h[q - OFF_W2] = __bfloat16_as_ushort(__float2bfloat16_rn(w));
}

size_t grad_smem_bytes() { return sizeof(float) * (NP + 2 + 5 * kTrainBlock + 4 * H * (kTrainBlock + 1)); }

int run_grad(const kv_mlp* h, const double* v, const double* x, const double* t0,
             const double* t1, int64_t n, int batch, int64_t step, uint64_t seed, int sequential,
             float* partial, cudaStream_t s)
{
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        KV_CUDA_TRY(cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)grad_smem_bytes()));
        attr_set[dev] = true;
    }
    GradArgs g;
    g.params = h->params;
    g.v = v;
    g.x = x;
    g.t0 = t0;
    g.t1 = t1;
    g.n = n;
    g.batch = batch;
    g.step = step;
    g.seed = seed;
    g.sequential = sequential;
    g.partial = partial;
    memcpy(g.in_scale, h->in_scale, sizeof(g.in_scale));
    memcpy(g.out_scale, h->out_scale, sizeof(g.out_scale));
    const int nb = (batch + kTrainBlock - 1) / kTrainBlock;
    mlp_grad_kernel<<<nb, kTrainBlock, grad_smem_bytes(), s>>>(g);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

}  // namespace

// ------------------------------------------------------------------ library-internal hooks

namespace kvh {

int mlp_view(const kv_mlp* h, MlpView* out)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    out->w1 = h->params + OFF_W1;
    out->b1 = h->params + OFF_B1;
    out->w2h = h->w2h;
    out->b2 = h->params + OFF_B2;
    out->w3 = h->params + OFF_W3;
    out->b3 = h->params + OFF_B3;
    memcpy(out->in_scale, h->in_scale, sizeof(out->in_scale));
    memcpy(out->out_scale, h->out_scale, sizeof(out->out_scale));
    return KV_OK;
}

// The kernel-parameter weights from the handle's host copy, refreshed from the device (ordered on
// `s`) after training moved the parameters on.
int fill_mlp_const(const kv_mlp* hc, cudaStream_t s, MlpConst* c)
{
    static std::mutex refresh;
    kv_mlp* h = const_cast<kv_mlp*>(hc);
    {
        std::lock_guard<std::mutex> lock(refresh);
        if (!h->host_ok) {
            KV_CUDA_TRY(cudaMemcpyAsync(h->host, h->params, sizeof(float) * NP, cudaMemcpyDeviceToHost, s));
            KV_CUDA_TRY(cudaStreamSynchronize(s));
            h->host_ok = true;
        }
    }
    const float* w = h->host;
    for (int k = 0; k < H / 2; ++k) {
        c->w1a[k] = make_float2(w[OFF_W1 + 4 * k], w[OFF_W1 + 4 * k + 2]);
        c->w1b[k] = make_float2(w[OFF_W1 + 4 * k + 1], w[OFF_W1 + 4 * k + 3]);
        c->b1[k] = make_float2(w[OFF_B1 + 2 * k], w[OFF_B1 + 2 * k + 1]);
    }
    for (int k = 0; k < H; ++k) c->w3[k] = make_float2(w[OFF_W3 + k], w[OFF_W3 + H + k]);
    c->b3[0] = w[OFF_B3];
    c->b3[1] = w[OFF_B3 + 1];
    memcpy(c->in_scale, h->in_scale, sizeof(c->in_scale));
    memcpy(c->out_scale, h->out_scale, sizeof(c->out_scale));
    return KV_OK;
}

std::atomic<int> g_wait_limit{-1};  // < 0: kWaitLimit
std::atomic<int> g_end_terms{1};

int launch_mlp_path(const kv_args* a, int bins, double log_eps, int max_iter, uint32_t* scratch_in)
{
    if (a->n > (int64_t)0xffffffffll) return KV_ERR_SIZE;
    const bool f32_plain = a->bracket == KV_BRACKET_PLAIN_F32;
    MlpPathParams p;
    memset(&p, 0, sizeof(p));
    int rc = f32_plain ? KV_OK : mlp_view(a->mlp, &p.mlp);
    if (rc != KV_OK) return rc;
    p.v = (const float*)a->v;
    p.x = (const float*)a->x;
    p.logk = (float*)a->logk;
    p.dv = (float*)a->dv;
    p.dx = (float*)a->dx;
    p.go = (const float*)a->grad_out;
    p.status = a->status;
    p.d2v = (float*)a->d2v;
    p.dvx = (float*)a->dvx;
    p.d2x = (float*)a->d2x;
    p.n = a->n;
    rc = f32_plain ? KV_OK : fill_mlp_const(a->mlp, (cudaStream_t)a->stream, &p.wc);
    if (rc != KV_OK) return rc;
    p.bins = bins;
    p.inv_bins = 1.0f / (float)bins;
    p.log_eps = (float)log_eps;
    const int wl = g_wait_limit.load(std::memory_order_relaxed);
    p.wait_limit = wl < 0 ? kWaitLimit : wl;
    p.end_terms = g_end_terms.load(std::memory_order_relaxed);
    rc = ensure_exp_table();
    if (rc != KV_OK) return rc;
    cudaStream_t s = (cudaStream_t)a->stream;
    // scratch: the fallback list and its counter (the caller's, or allocated on the stream)
    uint32_t* scratch = scratch_in;
    if (!scratch) KV_CUDA_TRY(scratch_alloc((void**)&scratch, sizeof(uint32_t) * (a->n + 32), s));
    p.fb_count = scratch;
    p.tile_ctr = scratch + 1;
    p.fb_list = scratch + 32;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 2 * sizeof(uint32_t), s);
    const bool second = a->d2v || a->dvx || a->d2x;
    const bool deriv = a->dv || a->dx || second;
    const bool plain = bins <= kPlainSumsMaxBins;  // few enough bins per lane for plain block sums
    if (e == cudaSuccess && f32_plain) {
        // one CTA per tile: the block scheduler balances the SMs as CTAs finish
        int grid = (int)((a->n + kMlpBlock - 1) / kMlpBlock);
        if (second) kv_plain_f32_kernel<true, true><<<grid, kMlpBlock, 0, s>>>(p, max_iter);
        else if (deriv && plain) kv_plain_f32_kernel<true, false, false><<<grid, kMlpBlock, 0, s>>>(p, max_iter);
        else if (deriv) kv_plain_f32_kernel<true><<<grid, kMlpBlock, 0, s>>>(p, max_iter);
        else if (plain) kv_plain_f32_kernel<false, false, false><<<grid, kMlpBlock, 0, s>>>(p, max_iter);
        else kv_plain_f32_kernel<false><<<grid, kMlpBlock, 0, s>>>(p, max_iter);
        note_launch();
        e = cudaGetLastError();
    } else if (e == cudaSuccess) {
        // persistent grid; at most 8 CTAs per SM so that their 64 TMEM columns each fit in 512
        const int per_sm = second  ? tc_blocks_per_sm(kv_mlp_tc_kernel<true, true>)
                           : deriv ? tc_blocks_per_sm(kv_mlp_tc_kernel<true>)
                                   : tc_blocks_per_sm(kv_mlp_tc_kernel<false>);
        int64_t need = (a->n + kMlpBlock - 1) / kMlpBlock;
        int64_t cap = (int64_t)sm_count() * per_sm;
        int grid = (int)(need < cap ? need : cap);
        if (second) kv_mlp_tc_kernel<true, true><<<grid, kMlpBlock, 0, s>>>(p);
        else if (deriv && plain) kv_mlp_tc_kernel<true, false, false><<<grid, kMlpBlock, 0, s>>>(p);
        else if (deriv) kv_mlp_tc_kernel<true><<<grid, kMlpBlock, 0, s>>>(p);
        else if (plain) kv_mlp_tc_kernel<false, false, false><<<grid, kMlpBlock, 0, s>>>(p);
        else kv_mlp_tc_kernel<false><<<grid, kMlpBlock, 0, s>>>(p);
        note_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        FallbackParams f;
        f.p = p;
        f.log_eps = log_eps;
        f.max_iter = max_iter;
        f.flags = a->flags;
        f.try_f32 = f32_plain ? 0 : 1;
        f.fallback_total = a->fallback_count;
        // grid-stride over the list (most calls have none), no more CTAs than the list can fill
        const int64_t most = (a->n + kMlpBlock - 1) / kMlpBlock;
        int grid = sm_count();
        if (most < grid) grid = (int)most;
        if (second) kv_fallback_kernel<true, true><<<grid, kMlpBlock, 0, s>>>(f);
        else if (deriv) kv_fallback_kernel<true><<<grid, kMlpBlock, 0, s>>>(f);
        else kv_fallback_kernel<false><<<grid, kMlpBlock, 0, s>>>(f);
        note_launch();
        e = cudaGetLastError();
    }
    cudaError_t e2 = scratch_in ? cudaSuccess : scratch_free(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e);
    if (e2 != cudaSuccess) return cuda_fail(e2);
    return KV_OK;
}

}  // namespace kvh

// ------------------------------------------------------------------ C ABI

extern "C" {

int kv_mlp_create(uint64_t seed, kv_mlp** out)
{
    if (!out) return KV_ERR_NULL;
    kv_mlp* h = nullptr;
    int rc = alloc_handle(&h);
    if (rc != KV_OK) return rc;
    // He-uniform weights U(-sqrt(6/fan_in), sqrt(6/fan_in)) from SplitMix64, zero biases
    std::vector<float> w(NP, 0.0f);
    auto uni = [&](uint64_t k) { return (double)(mix64(seed * 0x100000001B3ull + k) >> 11) * 0x1.0p-53; };
    for (int k = 0; k < 2 * H; ++k) w[OFF_W1 + k] = (float)((2 * uni(k) - 1) * sqrt(6.0 / 2.0));
    for (int k = 0; k < H * H; ++k) w[OFF_W2 + k] = (float)((2 * uni(1000 + k) - 1) * sqrt(6.0 / H));
    for (int k = 0; k < 2 * H; ++k) w[OFF_W3 + k] = (float)((2 * uni(10000 + k) - 1) * sqrt(6.0 / H));
    rc = upload(h, w.data());
    if (rc != KV_OK) {
        kv_mlp_free(h);
        return rc;
    }
    *out = h;
    return KV_OK;
}

int kv_mlp_free(kv_mlp* h)
{
    if (!h) return KV_OK;
    if (h->magic != kMagic) return KV_ERR_HANDLE;
    cudaFree(h->params);
    cudaFree(h->adam_m);
    cudaFree(h->adam_s);
    cudaFree(h->w2h);
    delete[] h->host;
    h->magic = 0;
    delete h;
    return KV_OK;
}

struct FileHeader {
    char magic[8];
    uint32_t version, hidden, nparams, reserved;
    float in_scale[4], out_scale[4];
    int64_t step;
};

int kv_mlp_save(const kv_mlp* h, const char* path)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (!path) return KV_ERR_NULL;
    std::vector<float> buf(3 * NP);
    KV_CUDA_TRY(cudaMemcpy(buf.data(), h->params, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    KV_CUDA_TRY(cudaMemcpy(buf.data() + NP, h->adam_m, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    KV_CUDA_TRY(cudaMemcpy(buf.data() + 2 * NP, h->adam_s, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    FileHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "KVMLP1\0\0", 8);
    hd.version = 1;
    hd.hidden = H;
    hd.nparams = NP;
    memcpy(hd.in_scale, h->in_scale, sizeof(hd.in_scale));
    memcpy(hd.out_scale, h->out_scale, sizeof(hd.out_scale));
    hd.step = h->step;
    FILE* f = fopen(path, "wb");
    if (!f) return KV_ERR_IO;
    bool ok = fwrite(&hd, sizeof(hd), 1, f) == 1 && fwrite(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    ok = (fclose(f) == 0) && ok;
    return ok ? KV_OK : KV_ERR_IO;
}

int kv_mlp_load(const char* path, kv_mlp** out)
{
    if (!path || !out) return KV_ERR_NULL;
    FILE* f = fopen(path, "rb");
    if (!f) return KV_ERR_IO;
    FileHeader hd;
    std::vector<float> buf(3 * NP);
    bool ok = fread(&hd, sizeof(hd), 1, f) == 1;
    if (ok && (memcmp(hd.magic, "KVMLP1\0\0", 8) != 0 || hd.version != 1 || hd.hidden != H ||
               hd.nparams != NP)) {
        fclose(f);
        return KV_ERR_FORMAT;
    }
    ok = ok && fread(buf.data(), sizeof(float), buf.size(), f) == buf.size();
    fclose(f);
    if (!ok) return KV_ERR_FORMAT;
    kv_mlp* h = nullptr;
    int rc = alloc_handle(&h);
    if (rc != KV_OK) return rc;
    memcpy(h->in_scale, hd.in_scale, sizeof(hd.in_scale));
    memcpy(h->out_scale, hd.out_scale, sizeof(hd.out_scale));
    h->step = hd.step;
    rc = upload(h, buf.data());
    cudaError_t e = cudaSuccess;
    if (rc == KV_OK) e = cudaMemcpy(h->adam_m, buf.data() + NP, sizeof(float) * NP, cudaMemcpyHostToDevice);
    if (rc == KV_OK && e == cudaSuccess)
        e = cudaMemcpy(h->adam_s, buf.data() + 2 * NP, sizeof(float) * NP, cudaMemcpyHostToDevice);
    if (rc == KV_OK && e != cudaSuccess) rc = kvh::cuda_fail(e);
    if (rc != KV_OK) {
        kv_mlp_free(h);
        return rc;
    }
    *out = h;
    return KV_OK;
}

int kv_mlp_get_params(const kv_mlp* h, float* host_params, int64_t count)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (!host_params) return KV_ERR_NULL;
    if (count != NP) return KV_ERR_SIZE;
    KV_CUDA_TRY(cudaMemcpy(host_params, h->params, sizeof(float) * NP, cudaMemcpyDeviceToHost));
    return KV_OK;
}

int kv_mlp_set_params(kv_mlp* h, const float* host_params, int64_t count)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (!host_params) return KV_ERR_NULL;
    if (count != NP) return KV_ERR_SIZE;
    KV_CUDA_TRY(cudaMemset(h->adam_m, 0, sizeof(float) * NP));
    KV_CUDA_TRY(cudaMemset(h->adam_s, 0, sizeof(float) * NP));
    h->step = 0;
    return upload(h, host_params);
}

int kv_mlp_loss_grad(const kv_mlp* h, const double* v, const double* x, const double* t0,
                     const double* t1, int64_t n, double* loss, float* grads, void* stream)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (n < 1 || n > (1 << 24)) return KV_ERR_SIZE;
    if (!v || !x || !t0 || !t1 || !loss || !grads) return KV_ERR_NULL;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n + kTrainBlock - 1) / kTrainBlock);
    float* partial = nullptr;
    KV_CUDA_TRY(kvh::scratch_alloc((void**)&partial, sizeof(float) * (size_t)nb * (NP + 1), s));
    int rc = run_grad(h, v, x, t0, t1, n, (int)n, 0, 0, 1, partial, s);
    if (rc == KV_OK) {
        ReduceArgs r;
        memset(&r, 0, sizeof(r));
        r.partial = partial;
        r.nblocks = nb;
        r.update = 0;
        r.loss_d = loss;
        r.grads_out = grads;
        mlp_reduce_kernel<<<(NP + 1 + 127) / 128, 128, 0, s>>>(r);
        kvh::note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = kvh::cuda_fail(e);
    }
    cudaError_t e2 = kvh::scratch_free(partial, s);
    if (rc == KV_OK && e2 != cudaSuccess) rc = kvh::cuda_fail(e2);
    return rc;
}

int kv_mlp_train(kv_mlp* h, const kv_train_args* a)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (!a) return KV_ERR_NULL;
    if (!a->v || !a->x || !a->t0 || !a->t1) return KV_ERR_NULL;
    if (a->n < 1 || a->n > (int64_t)0xffffffffll) return KV_ERR_SIZE;
    if (a->batch < 1 || a->batch > (1 << 20) || a->steps < 0) return KV_ERR_ARG;
    if (!(a->lr > 0.0f) || !(a->beta1 >= 0.0f && a->beta1 < 1.0f) ||
        !(a->beta2 >= 0.0f && a->beta2 < 1.0f) || !(a->adam_eps > 0.0f))
        return KV_ERR_ARG;
    cudaStream_t s = (cudaStream_t)a->stream;
    const int nb = (a->batch + kTrainBlock - 1) / kTrainBlock;
    float* partial = nullptr;
    KV_CUDA_TRY(kvh::scratch_alloc((void**)&partial, sizeof(float) * (size_t)nb * (NP + 1), s));
    int rc = KV_OK;
    if (a->steps > 0) h->host_ok = false;  // the device copy moves on; refreshed at the next use
    for (int j = 0; j < a->steps && rc == KV_OK; ++j) {
        const int64_t t = h->step + 1;
        rc = run_grad(h, a->v, a->x, a->t0, a->t1, a->n, a->batch, h->step, a->seed, 0, partial, s);
        if (rc != KV_OK) break;
        ReduceArgs r;
        memset(&r, 0, sizeof(r));
        r.partial = partial;
        r.nblocks = nb;
        r.params = h->params;
        r.m = h->adam_m;
        r.s = h->adam_s;
        r.w2h = h->w2h;
        r.update = 1;
        r.lr = a->lr;
        r.beta1 = a->beta1;
        r.beta2 = a->beta2;
        r.eps = a->adam_eps;
        r.bc1 = (float)(1.0 - pow((double)a->beta1, (double)t));
        r.bc2 = (float)(1.0 - pow((double)a->beta2, (double)t));
        r.loss_out = a->loss_out ? a->loss_out + j : nullptr;
        mlp_reduce_kernel<<<(NP + 1 + 127) / 128, 128, 0, s>>>(r);
        kvh::note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) rc = kvh::cuda_fail(e);
        h->step = t;
    }
    cudaError_t e2 = kvh::scratch_free(partial, s);
    if (rc == KV_OK && e2 != cudaSuccess) rc = kvh::cuda_fail(e2);
    return rc;
}

int kv_mlp_predict(const kv_mlp* h, const void* v, const void* x, void* t0, void* t1, int64_t n,
                   int dtype, void* stream)
{
    if (!valid(h)) return KV_ERR_HANDLE;
    if (dtype != KV_MIXED) return KV_ERR_DTYPE;
    if (n < 0) return KV_ERR_SIZE;
    if (n == 0) return KV_OK;
    if (!v || !x || !t0 || !t1) return KV_ERR_NULL;
    kvh::MlpView m;
    int rc = kvh::mlp_view(h, &m);
    if (rc != KV_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int64_t need = (n + kMlpBlock - 1) / kMlpBlock;
    int64_t cap = (int64_t)kvh::sm_count() * 8;
    int grid = (int)(need < cap ? need : cap);
    kv_predict_kernel<<<grid, kMlpBlock, 0, s>>>(m, (const float*)v, (const float*)x, (float*)t0,
                                                 (float*)t1, n);
    KV_LAUNCH_CHECK();
    return KV_OK;
}

int kv_debug_set_wait_limit(int iterations)
{
    return kvh::g_wait_limit.exchange(iterations < 0 ? -1 : iterations, std::memory_order_relaxed);
}

int kv_debug_set_end_terms(int on)
{
    return kvh::g_end_terms.exchange(on ? 1 : 0, std::memory_order_relaxed);
}

}  // extern "C"
