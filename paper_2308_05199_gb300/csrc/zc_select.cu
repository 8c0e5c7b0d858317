// zc_select.cu -- the per-chunk codec selector: chunk statistics, the
// 16-64-64-4 MLP (forward, loss gradient, momentum SGD) and the selection of
// block size or raw storage, written into a batched-compression plan.
//
// The statistics, the network and the cost model are defined in the header
// comment of zc.h (zc_batch_chunk_stats .. zc_batch_select).  Everything runs
// on the device; nothing is read back, so a whole select-then-compress
// sequence can be captured in one CUDA graph.
#include <cstddef>
#include <cstring>

#include "zc_launch.h"

namespace zc {

constexpr int N_STATS = ZC_STATS;
constexpr unsigned FULL_MASK_ALL = 0xffffffffu;
constexpr int ST_SPANS = 16;
constexpr int ST_SPAN = 128;

constexpr int NI = ZC_MLP_IN, NH = ZC_MLP_HIDDEN, NO = ZC_MLP_OUT;
constexpr int NPARAM = ZC_MLP_PARAMS;
constexpr int OFF_B1 = NH * NI, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH;
constexpr int OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NO * NH;
static_assert(OFF_B3 + NO == NPARAM, "parameter layout");
constexpr int NPAD = 5512;  // per-CTA partial gradient stride (NPARAM + loss, rounded)
constexpr int TB = 64;      // samples per CTA
constexpr int MT = 256;     // threads per MLP CTA

__device__ __forceinline__ int bitlen_u(unsigned v) { return 32 - __clz(v); }

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// ---- chunk statistics: one warp per item ----------------------------------------
// Lane l holds elements 4l .. 4l + 3 of a 128-element span (one 16-byte load
// of FP32, one 8-byte load of BF16, when the chunk is aligned for it), so
// three of every four differences are taken within the lane and a block of
// L elements is L / 4 consecutive lanes: its largest |delta| is one segmented
// warp reduction.  Per-lane sums stay 32-bit (64 sampled elements per lane at
// most: |q| < 2^23, |d| < 2^24, |d2| < 2^25) and are widened for the warp sum.
struct StatAcc {
    unsigned b16 = 0, b32 = 0, b64 = 0, b128 = 0;  // codec block bits per L (block-first lanes)
    unsigned sum_ad = 0, sum_aq = 0, sum_ad2 = 0;
    unsigned max_ad = 0, nz_d = 0, nz_q = 0, n_sc = 0, head_bits = 0;
    int qmin = 0x7fffffff, qmax = -0x7fffffff - 1;
    int bad = 0;
};

// The four elements of this lane in span [s0, s0 + cnt) (zero beyond cnt).
__device__ __forceinline__ void load_span4(const Item& it, bool vec, unsigned long long s0, int cnt,
                                           float v[4])
{
    const int lane = threadIdx.x & 31;
    const int i0 = 4 * lane;
    if (it.x_dtype == ZC_F32) {
        const float* p = (const float*)it.x + s0 + i0;
        if (vec && i0 + 4 <= cnt) {
            const float4 w = __ldg((const float4*)p);
            v[0] = w.x; v[1] = w.y; v[2] = w.z; v[3] = w.w;
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = i0 + m < cnt ? __ldg(p + m) : 0.0f;
        }
    } else {
        const unsigned short* p = (const unsigned short*)it.x + s0 + i0;
        if (vec && i0 + 4 <= cnt) {
            const uint2 w = __ldg((const uint2*)p);
            v[0] = __uint_as_float(w.x << 16);
            v[1] = __uint_as_float(w.x & 0xffff0000u);
            v[2] = __uint_as_float(w.y << 16);
            v[3] = __uint_as_float(w.y & 0xffff0000u);
        } else {
#pragma unroll
            for (int m = 0; m < 4; ++m) v[m] = i0 + m < cnt ? bf16_to_f32(__ldg(p + m)) : 0.0f;
        }
    }
}

// Largest block |delta| of the lane's block at blocks of G lanes (L = 4G):
// the block's first lane contributes |q| of its first element (the head is
// predicted from 0), every other lane |d| of its first element.
// (xor shuffles within aligned groups of G lanes: every lane takes part with
// the full mask, so no group waits for another)
template <int G>
__device__ __forceinline__ unsigned block_max(unsigned rest, unsigned e0q, unsigned e0d)
{
    const int lane = threadIdx.x & 31;
    unsigned v = max(rest, (lane & (G - 1)) == 0 ? e0q : e0d);
    if (G == 32) return __reduce_max_sync(FULL, v);
#pragma unroll
    for (int off = G / 2; off; off >>= 1) v = max(v, __shfl_xor_sync(FULL, v, off));
    return v;
}

// One span of cnt elements (v: this lane's four); returns the span's L = 32
// block bits (the same in every lane).  FULL: cnt == 128.  Branch-free:
// elements outside the span, and the differences that do not exist at the
// span's start, are masked out.
template <bool FULL>
__device__ __forceinline__ unsigned stat_span(const float v[4], int cnt, const Item& it,
                                              StatAcc& A)
{
    const int lane = threadIdx.x & 31;
    const int i0 = 4 * lane;
    int q[4];
    bool ok[4];
    // the exact quantizer: fast rounding for all four, the exact slow path
    // only when some lane's fast result may be off (one vote)
    bool slow = false;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        ok[m] = FULL || i0 + m < cnt;
        slow |= !quantize_fast(ok[m] ? v[m] : 0.0f, it.inv, q[m]);
    }
    if (__any_sync(FULL_MASK_ALL, slow)) {
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            int qq = 0;
            if (ok[m] && quantize(v[m], it.eb, it.two_eb, it.inv, qq) != 0) {
                A.bad = 1;
                qq = 0;
            }
            q[m] = qq;
        }
    }
    // first differences d (element i >= 1) and the previous one pd (i >= 2)
    int d[4], pd[4];
    d[0] = q[0] - __shfl_up_sync(FULL_MASK_ALL, q[3], 1);
#pragma unroll
    for (int m = 1; m < 4; ++m) d[m] = q[m] - q[m - 1];
    pd[0] = __shfl_up_sync(FULL_MASK_ALL, d[3], 1);
#pragma unroll
    for (int m = 1; m < 4; ++m) pd[m] = d[m - 1];
    unsigned rest = 0;  // largest |d| of elements 1..3 of the lane
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const bool v0 = ok[m];
        const bool v1 = v0 && (m > 0 || lane > 0);   // element i >= 1
        const bool v2 = v0 && (m > 1 || lane > 0);   // element i >= 2
        const unsigned aq = v0 ? (unsigned)abs(q[m]) : 0u;
        const unsigned ad = v1 ? (unsigned)abs(d[m]) : 0u;
        const unsigned ad2 = v2 ? (unsigned)abs(d[m] - pd[m]) : 0u;
        A.nz_q += (v0 && q[m] == 0) ? 1u : 0u;
        A.sum_aq += aq;
        A.qmin = min(A.qmin, v0 ? q[m] : 0x7fffffff);
        A.qmax = max(A.qmax, v0 ? q[m] : -0x7fffffff - 1);
        A.sum_ad += ad;
        A.max_ad = max(A.max_ad, ad);
        A.nz_d += (v1 && d[m] == 0) ? 1u : 0u;
        if (m > 0) rest = max(rest, ad);
        A.sum_ad2 += ad2;
        const bool sc = (d[m] > 0 && pd[m] < 0) || (d[m] < 0 && pd[m] > 0);
        A.n_sc += (v2 && sc) ? 1u : 0u;
    }
    const unsigned e0q = ok[0] ? (unsigned)abs(q[0]) : 0u;
    const unsigned e0d = (ok[0] && i0 >= 1) ? (unsigned)abs(d[0]) : 0u;
    const unsigned m16 = block_max<4>(rest, e0q, e0d);
    const unsigned m32 = block_max<8>(rest, e0q, e0d);
    const unsigned m64 = block_max<16>(rest, e0q, e0d);
    const unsigned m128 = block_max<32>(rest, e0q, e0d);
    const unsigned b32 = ((lane & 7) == 0 && m32) ? (bitlen_u(m32) + 1) * 32 : 0u;
    A.b16 += ((lane & 3) == 0 && m16) ? (bitlen_u(m16) + 1) * 16 : 0u;
    A.b64 += ((lane & 15) == 0 && m64) ? (bitlen_u(m64) + 1) * 64 : 0u;
    A.b128 += (lane == 0 && m128) ? (bitlen_u(m128) + 1) * 128 : 0u;
    A.b32 += b32;
    A.head_bits += ((lane & 7) == 0 && ok[0]) ? bitlen_u(e0q) : 0u;
    return __reduce_add_sync(FULL_MASK_ALL, b32);
}

__global__ void __launch_bounds__(256, 4) k_chunk_stats(const Item* items, unsigned n_items,
                                                     float* feat)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned idx = blockIdx.x * 8 + warp;
    if (idx >= n_items) return;  // warp-uniform; only warp-level sync below
    const Item it = items[idx];
    float* out = feat + (size_t)idx * N_STATS;
    const unsigned long long n = it.n;
    if (n == 0 || it.x == nullptr || !(it.two_eb > 0.0f)) {
        if (lane < N_STATS) out[lane] = __int_as_float(0x7fc00000);  // NaN row
        return;
    }
    const unsigned long long m = n / ST_SPAN;
    const int S = m == 0 ? 1 : (int)(m < ST_SPANS ? m : ST_SPANS);
    const int cnt = m == 0 ? (int)n : ST_SPAN;  // elements of every sampled span
    // spans start at multiples of 128 elements: aligned loads when the chunk is
    const bool vec = ((uintptr_t)it.x & (it.x_dtype == ZC_F32 ? 15u : 7u)) == 0u;
    // span j starts at 128 floor(j (m - 1) / (S - 1)): stepped without a
    // division per span (quotient and remainder of (m - 1) / (S - 1) once)
    const unsigned long long den = S > 1 ? (unsigned long long)(S - 1) : 1ull;
    const unsigned long long num = m > 0 ? m - 1 : 0ull;
    const unsigned long long qa = num / den, ra = num % den;
    unsigned long long sq = 0ull, sr = 0ull;  // floor(j num / den) and its remainder, next span
    auto next_span0 = [&]() -> unsigned long long {
        const unsigned long long v = (unsigned long long)ST_SPAN * sq;
        sq += qa;
        sr += ra;
        if (sr >= den) {
            sr -= den;
            sq += 1ull;
        }
        return v;
    };
    StatAcc A;
    // sum over the spans of their L = 32 bits, and of its squares (warp-uniform;
    // a span holds at most 128 x 25 bits, so both fit 32 bits over 16 spans)
    unsigned span_b1 = 0u, span_b2 = 0u;
    auto add_span = [&](unsigned b) {
        span_b1 += b;
        span_b2 += b * b;
    };
    if (cnt == ST_SPAN) {
        // full spans: two loaded ahead of the one being summarised
        float xa[4], xb[4], xc[4];
        load_span4(it, vec, next_span0(), cnt, xa);
        if (S > 1) load_span4(it, vec, next_span0(), cnt, xb);
#pragma unroll 1
        for (int j = 0; j < S; ++j) {
            if (j + 2 < S) load_span4(it, vec, next_span0(), cnt, xc);
            add_span(stat_span<true>(xa, cnt, it, A));
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                xa[k] = xb[k];
                xb[k] = xc[k];
            }
        }
    } else {
        float xa[4];
        load_span4(it, vec, 0ull, cnt, xa);
        add_span(stat_span<false>(xa, cnt, it, A));
    }
    const unsigned long long B16 = warp_sum_u64(A.b16), B32 = warp_sum_u64(A.b32);
    const unsigned long long B64 = warp_sum_u64(A.b64), B128 = warp_sum_u64(A.b128);
    const unsigned long long SAD = warp_sum_u64(A.sum_ad), SAQ = warp_sum_u64(A.sum_aq);
    const unsigned long long SAD2 = warp_sum_u64(A.sum_ad2);
    const unsigned long long NZD = __reduce_add_sync(FULL, A.nz_d);
    const unsigned long long NZQ = __reduce_add_sync(FULL, A.nz_q);
    const unsigned long long NSC = __reduce_add_sync(FULL, A.n_sc);
    const unsigned long long HB = __reduce_add_sync(FULL, A.head_bits);
    const unsigned MAD = __reduce_max_sync(FULL, A.max_ad);
    const int QMN = __reduce_min_sync(FULL, A.qmin), QMX = __reduce_max_sync(FULL, A.qmax);
    const int BAD = __any_sync(FULL, A.bad);
    if (lane != 0) return;
    if (BAD) {
        for (int k = 0; k < N_STATS; ++k) out[k] = __int_as_float(0x7fc00000);
        return;
    }
    const unsigned long long bits[4] = {B16, B32, B64, B128};
    // The features in FP32 (this GPU's FP64 rate is a small fraction of its
    // FP32 rate): counts are exact integers below 2^24, each quotient is one
    // correctly rounded division, each logarithm CUDA's log2f.
    const float tot = (float)(S * cnt), fn = (float)n;
    const float nd = (float)(S * (cnt - 1));
    const float nd2 = cnt >= 2 ? (float)(S * (cnt - 2)) : 0.0f;
    const float nheads = (float)(S * ((cnt + 31) / 32));
    const float hdr = __fdiv_rn(256.0f, fn);
    float f[N_STATS];
    f[0] = __fadd_rn(__fadd_rn(__fdiv_rn((float)bits[0], tot), 0.5f), hdr);
    f[1] = __fadd_rn(__fadd_rn(__fdiv_rn((float)bits[1], tot), 0.25f), hdr);
    f[2] = __fadd_rn(__fadd_rn(__fdiv_rn((float)bits[2], tot), 0.125f), hdr);
    f[3] = __fadd_rn(__fadd_rn(__fdiv_rn((float)bits[3], tot), 0.0625f), hdr);
    f[4] = log2f(1.0f + (float)((long long)QMX - (long long)QMN));
    f[5] = nd > 0.0f ? log2f(1.0f + __fdiv_rn((float)SAD, nd)) : 0.0f;
    f[6] = nd > 0.0f ? log2f(1.0f + (float)MAD) : 0.0f;
    f[7] = nd > 0.0f ? __fdiv_rn((float)NZD, nd) : 0.0f;
    f[8] = __fdiv_rn((float)NZQ, tot);
    f[9] = log2f(1.0f + __fdiv_rn((float)SAQ, tot));
    f[10] = nd2 > 0.0f ? log2f(1.0f + __fdiv_rn((float)SAD2, nd2)) : 0.0f;
    f[11] = nd2 > 0.0f ? __fdiv_rn((float)NSC, nd2) : 0.0f;
    f[12] = __fdiv_rn(__fdiv_rn((float)HB, nheads), 24.0f);
    // population spread of the spans' bits per element b_j / cnt, from exact
    // integer moments: S^2 cnt^2 var = S sum b_j^2 - (sum b_j)^2
    const long long dvar = (long long)S * (long long)span_b2 - (long long)span_b1 * (long long)span_b1;
    const float sc2 = (float)S * (float)cnt;
    f[13] = sqrtf(__fdiv_rn((float)dvar, __fmul_rn(sc2, sc2)));
    f[14] = it.x_dtype == ZC_F32 ? 1.0f : 0.5f;
    f[15] = __fdiv_rn(log2f(fn), 16.0f);
#pragma unroll
    for (int k = 0; k < N_STATS; ++k) out[k] = f[k];
}

// ---- MLP ------------------------------------------------------------------------------
// Shared memory of an MLP CTA (floats): the parameters with padded row
// strides (no bank conflicts), the normalised inputs, both layers'
// activations (after the ReLU), one 64 x 64 gradient buffer and the outputs.
// Rows that the forward pass reads four at a time (W2, W3, X, A1, A2) have
// strides of a multiple of 4 floats: 16-byte loads, and at stride 68 the 8
// rows of a quarter warp fall in distinct bank groups.
constexpr int NHP = NH + 4, NIP = NI + 4;
struct MlpSmem {
    float W1[NH][NI + 1], b1[NH];
    alignas(16) float W2[NH][NHP];
    float b2[NH];
    alignas(16) float W3[NO][NHP];
    float b3[NO];
    alignas(16) float X[TB][NIP];
    alignas(16) float A1[TB][NHP];
    alignas(16) float A2[TB][NHP];  // later: dA1
    float D[TB][NH + 1];            // dA2
    float Y[TB][NO];                // outputs, later dY
    float red[MT / 32];
};
static_assert(offsetof(MlpSmem, W2) % 16 == 0 && offsetof(MlpSmem, W3) % 16 == 0 &&
                  offsetof(MlpSmem, X) % 16 == 0 && offsetof(MlpSmem, A1) % 16 == 0 &&
                  offsetof(MlpSmem, A2) % 16 == 0,
              "16-byte rows");

__device__ __forceinline__ float relu(float v) { return v > 0.0f ? v : 0.0f; }

// Loads the parameters into shared memory (no barrier).
__device__ __forceinline__ void mlp_load_params(MlpSmem& sm, const float* P)
{
    const int t = threadIdx.x;
    for (int p = t; p < NH * NI; p += MT) sm.W1[p / NI][p % NI] = P[p];
    for (int p = t; p < NH * NH; p += MT) sm.W2[p / NH][p % NH] = P[OFF_W2 + p];
    for (int p = t; p < NO * NH; p += MT) sm.W3[p / NH][p % NH] = P[OFF_W3 + p];
    if (t < NH) {
        sm.b1[t] = P[OFF_B1 + t];
        sm.b2[t] = P[OFF_B2 + t];
    }
    if (t < NO) sm.b3[t] = P[OFF_B3 + t];
}

// Loads the tile's rows (normalised) into shared memory; rows past B are
// zero (no barrier).
__device__ __forceinline__ void mlp_load_rows(MlpSmem& sm, const float* norm, const float* X,
                                              const int* idx, int B, int row0)
{
    const int t = threadIdx.x;
    for (int p = t; p < TB * NI; p += MT) {
        const int s = p / NI, k = p % NI, r = row0 + s;
        float v = 0.0f;
        if (r < B) {
            const long long row = idx != nullptr ? (long long)idx[r] : (long long)r;
            v = __fmul_rn(__fsub_rn(X[row * NI + k], norm[k]), norm[NI + k]);
        }
        sm.X[s][k] = v;
    }
}

// Loads the parameters and the tile's rows.
__device__ __forceinline__ void mlp_load(MlpSmem& sm, const float* P, const float* norm,
                                         const float* X, const int* idx, int B, int row0)
{
    mlp_load_params(sm, P);
    mlp_load_rows(sm, norm, X, idx, B, row0);
    __syncthreads();
}

// H1 = relu(X W1^T + b1), H2 = relu(H1 W2^T + b2), Y = H2 W3^T + b3, each
// sum accumulated by FMAs in input order.  sm.A1 and sm.A2 hold the
// activations after the ReLU: the gradient's ReLU derivative only asks
// whether the pre-activation was positive, which H > 0 answers alike.
__device__ __forceinline__ void mlp_forward_tile(MlpSmem& sm)
{
    const int t = threadIdx.x, j = t & (NH - 1), g = t >> 6;
    {
        float w[NI];
#pragma unroll
        for (int k = 0; k < NI; ++k) w[k] = sm.W1[j][k];
        for (int i = 0; i < TB / 4; ++i) {
            const int s = g * (TB / 4) + i;
            float a = sm.b1[j];
#pragma unroll
            for (int k = 0; k < NI; k += 4) {
                const float4 x = *reinterpret_cast<const float4*>(&sm.X[s][k]);
                a = __fmaf_rn(w[k], x.x, a);
                a = __fmaf_rn(w[k + 1], x.y, a);
                a = __fmaf_rn(w[k + 2], x.z, a);
                a = __fmaf_rn(w[k + 3], x.w, a);
            }
            sm.A1[s][j] = relu(a);
        }
    }
    __syncthreads();
    {
        float acc[TB / 4];
#pragma unroll
        for (int i = 0; i < TB / 4; ++i) acc[i] = sm.b2[j];
#pragma unroll 2
        for (int k = 0; k < NH; k += 4) {
            const float4 w = *reinterpret_cast<const float4*>(&sm.W2[j][k]);
#pragma unroll
            for (int i = 0; i < TB / 4; ++i) {
                const float4 a = *reinterpret_cast<const float4*>(&sm.A1[g * (TB / 4) + i][k]);
                acc[i] = __fmaf_rn(w.x, a.x, acc[i]);
                acc[i] = __fmaf_rn(w.y, a.y, acc[i]);
                acc[i] = __fmaf_rn(w.z, a.z, acc[i]);
                acc[i] = __fmaf_rn(w.w, a.w, acc[i]);
            }
        }
#pragma unroll
        for (int i = 0; i < TB / 4; ++i) sm.A2[g * (TB / 4) + i][j] = relu(acc[i]);
    }
    __syncthreads();
    {
        const int s = t >> 2, o = t & 3;
        float y = sm.b3[o];
#pragma unroll 4
        for (int k = 0; k < NH; k += 4) {
            const float4 w = *reinterpret_cast<const float4*>(&sm.W3[o][k]);
            const float4 a = *reinterpret_cast<const float4*>(&sm.A2[s][k]);
            y = __fmaf_rn(w.x, a.x, y);
            y = __fmaf_rn(w.y, a.y, y);
            y = __fmaf_rn(w.z, a.z, y);
            y = __fmaf_rn(w.w, a.w, y);
        }
        sm.Y[s][o] = y;
    }
    __syncthreads();
}

// Persistent over row tiles: the parameters are loaded once per CTA, then
// the CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ... (every row's
// arithmetic is the same as with one tile per CTA).
__global__ void __launch_bounds__(MT) k_mlp_forward(const float* P, const float* norm,
                                                    const float* X, int B, float* Yout)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem& sm = *reinterpret_cast<MlpSmem*>(raw);
    const int ntiles = (B + TB - 1) / TB;
    mlp_load_params(sm, P);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int row0 = tile * TB;
        mlp_load_rows(sm, norm, X, nullptr, B, row0);
        __syncthreads();
        mlp_forward_tile(sm);  // ends with a barrier: sm.Y is complete
        const int t = threadIdx.x, s = t >> 2, o = t & 3;
        if (row0 + s < B) Yout[(long long)(row0 + s) * NO + o] = sm.Y[s][o];
    }
}

// Per-CTA partial gradient of sum((Y - T)^2) / (B * NO) over its rows, and
// the partial sum of squared residuals, at partial + blockIdx.x * NPAD.
__global__ void __launch_bounds__(MT) k_mlp_grad(const float* P, const float* norm,
                                                 const float* X, const float* T, const int* idx,
                                                 int B, float* partial)
{
    extern __shared__ __align__(16) uint8_t raw[];
    MlpSmem& sm = *reinterpret_cast<MlpSmem*>(raw);
    const int row0 = blockIdx.x * TB;
    mlp_load(sm, P, norm, X, idx, B, row0);
    mlp_forward_tile(sm);
    const int t = threadIdx.x, j = t & (NH - 1), g = t >> 6;
    float* G = partial + (size_t)blockIdx.x * NPAD;
    const float scale = 2.0f / (float)(B * NO);
    // dY and the squared residuals
    {
        const int s = t >> 2, o = t & 3, r = row0 + s;
        float sq = 0.0f, dy = 0.0f;
        if (r < B) {
            const long long row = idx != nullptr ? (long long)idx[r] : (long long)r;
            const float res = __fsub_rn(sm.Y[s][o], T[row * NO + o]);
            sq = __fmul_rn(res, res);
            dy = __fmul_rn(scale, res);
        }
        __syncthreads();  // every Y read before it becomes dY
        sm.Y[s][o] = dy;
#pragma unroll
        for (int off = 16; off; off >>= 1) sq = __fadd_rn(sq, __shfl_xor_sync(FULL, sq, off));
        if ((t & 31) == 0) sm.red[t >> 5] = sq;
    }
    __syncthreads();
    if (t == 0) {
        float l = 0.0f;
        for (int w = 0; w < MT / 32; ++w) l = __fadd_rn(l, sm.red[w]);
        G[NPARAM] = l;
    }
    // dW3[o][k] = sum_s dY[s][o] H2[s][k]; db3
    {
        const int o = t >> 6, k = t & 63;
        float acc = 0.0f;
        for (int s = 0; s < TB; ++s) acc = __fadd_rn(acc, __fmul_rn(sm.Y[s][o], sm.A2[s][k]));
        G[OFF_W3 + o * NH + k] = acc;
        if (t < NO) {
            float b = 0.0f;
            for (int s = 0; s < TB; ++s) b = __fadd_rn(b, sm.Y[s][t]);
            G[OFF_B3 + t] = b;
        }
    }
    // dA2[s][j] = (sum_o dY[s][o] W3[o][j]) [H2 > 0]
    for (int i = 0; i < TB / 4; ++i) {
        const int s = g * (TB / 4) + i;
        float a = 0.0f;
#pragma unroll
        for (int o = 0; o < NO; ++o) a = __fadd_rn(a, __fmul_rn(sm.Y[s][o], sm.W3[o][j]));
        sm.D[s][j] = sm.A2[s][j] > 0.0f ? a : 0.0f;
    }
    __syncthreads();
    // dW2[j][k] = sum_s dA2[s][j] H1[s][k] for k in this thread's 16; db2
    {
        float acc[NH / 4];
#pragma unroll
        for (int kk = 0; kk < NH / 4; ++kk) acc[kk] = 0.0f;
        float b = 0.0f;
        for (int s = 0; s < TB; ++s) {
            const float a = sm.D[s][j];
            b = __fadd_rn(b, a);
#pragma unroll
            for (int kk = 0; kk < NH / 4; ++kk)
                acc[kk] = __fadd_rn(acc[kk], __fmul_rn(a, sm.A1[s][g * (NH / 4) + kk]));
        }
#pragma unroll
        for (int kk = 0; kk < NH / 4; ++kk) G[OFF_W2 + j * NH + g * (NH / 4) + kk] = acc[kk];
        if (g == 0) G[OFF_B2 + j] = b;
    }
    // dA1[s][k] = (sum_j dA2[s][j] W2[j][k]) [H1 > 0], into A2's storage (k = this thread's j)
    {
        float acc[TB / 4];
#pragma unroll
        for (int i = 0; i < TB / 4; ++i) acc[i] = 0.0f;
        for (int jj = 0; jj < NH; ++jj) {
            const float w = sm.W2[jj][j];
#pragma unroll
            for (int i = 0; i < TB / 4; ++i)
                acc[i] = __fadd_rn(acc[i], __fmul_rn(sm.D[g * (TB / 4) + i][jj], w));
        }
        __syncthreads();  // A2 (read above for dA2) is dead from here on
#pragma unroll
        for (int i = 0; i < TB / 4; ++i) {
            const int s = g * (TB / 4) + i;
            sm.A2[s][j] = sm.A1[s][j] > 0.0f ? acc[i] : 0.0f;
        }
    }
    __syncthreads();
    // dW1[j][k] = sum_s dA1[s][j] X[s][k] for k in this thread's 4; db1
    {
        float acc[NI / 4];
#pragma unroll
        for (int kk = 0; kk < NI / 4; ++kk) acc[kk] = 0.0f;
        float b = 0.0f;
        for (int s = 0; s < TB; ++s) {
            const float a = sm.A2[s][j];
            b = __fadd_rn(b, a);
#pragma unroll
            for (int kk = 0; kk < NI / 4; ++kk)
                acc[kk] = __fadd_rn(acc[kk], __fmul_rn(a, sm.X[s][g * (NI / 4) + kk]));
        }
#pragma unroll
        for (int kk = 0; kk < NI / 4; ++kk) G[j * NI + g * (NI / 4) + kk] = acc[kk];
        if (g == 0) G[OFF_B1 + j] = b;
    }
}

// Sums the CTAs' partial gradients in CTA order (deterministic).
__global__ void k_mlp_reduce(const float* partial, int nct, int B, float* grad, float* loss)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > NPARAM) return;
    float acc = 0.0f;
    for (int c = 0; c < nct; ++c) acc = __fadd_rn(acc, partial[(size_t)c * NPAD + p]);
    if (p < NPARAM) grad[p] = acc;
    else if (loss != nullptr) *loss = acc / (float)(B * NO);
}

// v <- momentum v + g; p <- p - lr v.
__global__ void k_mlp_sgd(float* P, float* V, const float* G, float lr, float momentum)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= NPARAM) return;
    const float v = __fadd_rn(__fmul_rn(momentum, V[p]), G[p]);
    V[p] = v;
    P[p] = __fsub_rn(P[p], __fmul_rn(lr, v));
}

// ---- selection: one thread per item -------------------------------------------------
struct SelectArgs {
    float link, c[4], c_raw, judge, judge_time;
};

// With `pred_time`, a message's coded cost at L_k takes its own predicted ns
// per input byte, 2^pred_time[k], where that prediction is finite and within
// judge_time (log2) of the batch-wide rate c[k]; elsewhere c[k] stays.
__global__ void k_select(Item* items, unsigned n_items, const float* feat, const float* pred,
                         const float* pred_time, SelectArgs a, int* choice, unsigned* counts)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_items) return;
    Item& it = items[i];
    const float nf = (float)it.n;
    const float bytes_in = nf * (it.x_dtype == ZC_F32 ? 4.0f : 2.0f);
    const float* f = feat + (size_t)i * N_STATS;
    const float cost_raw = __fadd_rn(__fmul_rn(bytes_in, a.c_raw), __fdiv_rn(__fadd_rn(32.0f, bytes_in), a.link));
    // the heuristic: L = 32 unless the sampled estimate says coding does not pay
    int h = 0;
    if (isfinite(f[1])) {
        const float c32 = __fadd_rn(__fmul_rn(bytes_in, a.c[1]),
                                    __fdiv_rn(__fdiv_rn(__fmul_rn(nf, f[1]), 8.0f), a.link));
        h = c32 < cost_raw ? 32 : 0;
    }
    int c = h;
    bool fell_back = false;
    if (pred != nullptr) {
        const float* y = pred + (size_t)i * NO;
        bool ok = true;
        for (int k = 0; k < 4; ++k) ok = ok && isfinite(y[k]) && isfinite(f[k]);
        if (ok) {
            int kb = 0;
            float best = 0.0f;
            for (int k = 0; k < 4; ++k) {
                const float bits = exp2f(y[k]);
                float rate = a.c[k];
                if (pred_time != nullptr) {
                    const float t = pred_time[(size_t)i * NO + k];
                    if (isfinite(t) && fabsf(__fsub_rn(t, log2f(a.c[k]))) <= a.judge_time)
                        rate = exp2f(t);
                }
                const float ck = __fadd_rn(__fmul_rn(bytes_in, rate),
                                           __fdiv_rn(__fdiv_rn(__fmul_rn(nf, bits), 8.0f), a.link));
                if (k == 0 || ck < best) {
                    best = ck;
                    kb = k;
                }
            }
            if (fabsf(__fsub_rn(y[kb], log2f(f[kb]))) > a.judge) fell_back = true;
            else c = best < cost_raw ? (16 << kb) : 0;
        } else {
            fell_back = true;
        }
    }
    if (!(it.two_eb > 0.0f)) c = 0;  // planned without a bound: raw only
    it.log2L = c == 16 ? 4 : c == 32 ? 5 : c == 64 ? 6 : c == 128 ? 7 : -1;
    if (choice != nullptr) choice[i] = c;
    if (counts != nullptr) {
        if (fell_back) atomicAdd(counts, 1u);
        if (c == 0) atomicAdd(counts + 1, 1u);
    }
}

}  // namespace zc

using namespace zc;

extern "C" {

int zc_batch_chunk_stats(const zc_batch* plan, float* d_feat, zc_stream_t s)
{
    if (plan == nullptr || plan->d_table == nullptr || plan->n_msgs < 1 || plan->decompress != 0 ||
        d_feat == nullptr || (reinterpret_cast<uintptr_t>(d_feat) & 3) != 0)
        return ZC_ERR_ARG;
    const unsigned n = (unsigned)plan->n_msgs;
    k_chunk_stats<<<(n + 7) / 8, 256, 0, (cudaStream_t)s>>>((const Item*)plan->d_table, n, d_feat);
    return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

static cudaError_t mlp_prepare()
{
    const cudaError_t e1 = smem_limit<k_mlp_forward>((int)sizeof(MlpSmem));
    const cudaError_t e2 = smem_limit<k_mlp_grad>((int)sizeof(MlpSmem));
    return e1 != cudaSuccess ? e1 : e2;
}

int zc_mlp_forward(const float* d_params, const float* d_norm, const float* d_x, int B,
                   float* d_y, zc_stream_t s)
{
    if (d_params == nullptr || d_norm == nullptr || B < 0 || (B > 0 && (d_x == nullptr || d_y == nullptr)))
        return ZC_ERR_ARG;
    if (B == 0) return ZC_OK;
    if (mlp_prepare() != cudaSuccess) return ZC_ERR_CUDA;
    // two CTAs per SM fit (shared memory), each looping over row tiles
    int dev = 0, n_sm = 152;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return ZC_ERR_CUDA;
    const int ntiles = (B + TB - 1) / TB;
    const int grid = ntiles < 2 * n_sm ? ntiles : 2 * n_sm;
    k_mlp_forward<<<grid, MT, sizeof(MlpSmem), (cudaStream_t)s>>>(d_params, d_norm, d_x, B, d_y);
    return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

size_t zc_mlp_scratch_bytes(int B)
{
    if (B < 1) return 0;
    return (size_t)((B + TB - 1) / TB) * NPAD * sizeof(float);
}

int zc_mlp_grad(const float* d_params, const float* d_norm, const float* d_x, const float* d_t,
                const int* d_idx, int B, float* d_grad, float* d_loss, void* d_scratch,
                size_t scratch_bytes, zc_stream_t s)
{
    if (d_params == nullptr || d_norm == nullptr || d_x == nullptr || d_t == nullptr || B < 1 ||
        d_grad == nullptr || d_scratch == nullptr || scratch_bytes < zc_mlp_scratch_bytes(B) ||
        (reinterpret_cast<uintptr_t>(d_scratch) & 3) != 0)
        return ZC_ERR_ARG;
    if (mlp_prepare() != cudaSuccess) return ZC_ERR_CUDA;
    const int nct = (B + TB - 1) / TB;
    k_mlp_grad<<<nct, MT, sizeof(MlpSmem), (cudaStream_t)s>>>(d_params, d_norm, d_x, d_t, d_idx, B,
                                                             (float*)d_scratch);
    if (cudaGetLastError() != cudaSuccess) return ZC_ERR_CUDA;
    k_mlp_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, (cudaStream_t)s>>>((const float*)d_scratch, nct,
                                                                       B, d_grad, d_loss);
    return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

int zc_mlp_sgd(float* d_params, float* d_vel, const float* d_grad, float lr, float momentum,
               zc_stream_t s)
{
    if (d_params == nullptr || d_vel == nullptr || d_grad == nullptr) return ZC_ERR_ARG;
    k_mlp_sgd<<<(NPARAM + 255) / 256, 256, 0, (cudaStream_t)s>>>(d_params, d_vel, d_grad, lr,
                                                                 momentum);
    return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

int zc_batch_select_timed(const zc_batch* plan, const float* d_feat, const float* d_pred,
                          const float* d_pred_time, const zc_select_cfg* cfg, int* d_choice,
                          unsigned* d_counts, zc_stream_t s)
{
    if (plan == nullptr || plan->d_table == nullptr || plan->n_msgs < 1 || plan->decompress != 0 ||
        d_feat == nullptr || cfg == nullptr || !(cfg->link_gbs > 0.0f) || !(cfg->judge_log2 >= 0.0f))
        return ZC_ERR_ARG;
    if (d_pred_time != nullptr && (d_pred == nullptr || !(cfg->judge_time_log2 >= 0.0f)))
        return ZC_ERR_ARG;
    SelectArgs a;
    a.link = cfg->link_gbs;
    for (int k = 0; k < 4; ++k) a.c[k] = cfg->ns_per_byte[k];
    a.c_raw = cfg->raw_ns_per_byte;
    a.judge = cfg->judge_log2;
    a.judge_time = d_pred_time != nullptr ? cfg->judge_time_log2 : 0.0f;
    if (d_counts != nullptr &&
        cudaMemsetAsync(d_counts, 0, 2 * sizeof(unsigned), (cudaStream_t)s) != cudaSuccess)
        return ZC_ERR_CUDA;
    const unsigned n = (unsigned)plan->n_msgs;
    k_select<<<(n + 255) / 256, 256, 0, (cudaStream_t)s>>>((Item*)plan->d_table, n, d_feat, d_pred,
                                                           d_pred_time, a, d_choice, d_counts);
    return cudaGetLastError() == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

int zc_batch_select(const zc_batch* plan, const float* d_feat, const float* d_pred,
                    const zc_select_cfg* cfg, int* d_choice, unsigned* d_counts, zc_stream_t s)
{
    return zc_batch_select_timed(plan, d_feat, d_pred, nullptr, cfg, d_choice, d_counts, s);
}

}  // extern "C"
