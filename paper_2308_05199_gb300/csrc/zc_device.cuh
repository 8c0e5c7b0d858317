// zc_device.cuh -- device building blocks of the codec kernels.
//
// Control block, status word, memory-ordering helpers, the bounded
// decoupled look-back that turns per-tile byte counts into stream offsets in
// one pass, the warp bit-matrix transpose that builds bit planes, and the
// exact prequantizer.  Everything here is sm_103a CUDA; nothing is shared with
// the CPU oracle.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "zc.h"

namespace zc {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NWARPS = 8;                  // warps per CTA
constexpr int NTHREADS = NWARPS * 32;      // threads per CTA
constexpr int MIN_ROWS = 4;                // smallest rows-per-warp: tile = 1024 elements
constexpr unsigned WS_MAGIC = 0x5a435753u; // "ZCWS"
constexpr int RANGE_SLOTS = 4096;          // partial min/max slots of the range kernel
constexpr uint64_t WS_CTL_BYTES = 256;
constexpr uint64_t WS_RANGE_BYTES = RANGE_SLOTS * 8;
constexpr int QMAX = 1 << 22;              // largest |q|

// Workspace control block (first 256 bytes of the workspace).
struct Ctl {
    unsigned status;          // first data error, 0 = none
    unsigned magic;           // WS_MAGIC once zc_workspace_init ran
    unsigned long long detail;
    unsigned ticket;          // tile ticket; wraps to 0 at the end of every launch
    unsigned done;            // finished CTAs; wraps to 0 at the end of every launch
    unsigned epoch;           // launch generation stamped on look-back flags
    unsigned range_done;      // finished CTAs of the range kernel
    float eb, two_eb, inv;    // bound resolved on the device (relative mode)
    float mn, mx;             // extremes seen by the range kernel
    unsigned eb_ok;           // 1 when eb/two_eb/inv above are usable
};
static_assert(sizeof(Ctl) <= WS_CTL_BYTES, "control block too large");

// ---- memory-ordering helpers -------------------------------------------

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
// Acquire fence: a relaxed load that observed a value written by a release
// store, followed by this fence, sees everything written before that store.
// Polling with relaxed loads and fencing once after the last one keeps the
// (costly) acquire out of the polling loops.
__device__ __forceinline__ void fence_acquire_gpu()
{
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ unsigned ld_volatile_u32(const unsigned* p)
{
    return *(const volatile unsigned*)p;
}
__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First error wins; `detail` records where it was seen.
__device__ __forceinline__ void fail(Ctl* c, unsigned code, unsigned long long detail)
{
    if (atomicCAS(&c->status, 0u, code) == 0u) c->detail = detail;
}

// Bounds-checked builds (compiled with -DZC_DEBUG): a checked access is
// tested against its buffer first; a failed check records ZC_ERR_BOUNDS with
// the offending offset (first error wins) and the caller skips the access.
// Release builds compile every check to `true`.
#ifdef ZC_DEBUG
constexpr bool DEBUG_BUILD = true;
__device__ __forceinline__ bool dcheck(Ctl* c, bool ok, unsigned long long detail)
{
    if (!ok) fail(c, ZC_ERR_BOUNDS, detail);
    return ok;
}
#else
constexpr bool DEBUG_BUILD = false;
__device__ __forceinline__ bool dcheck(Ctl*, bool, unsigned long long) { return true; }
#endif

// Normal (not zero, subnormal, infinite or NaN) FP32 value.
__device__ __forceinline__ bool is_normal(float f)
{
    const unsigned e = (__float_as_uint(f) >> 23) & 0xffu;
    return e != 0u && e != 0xffu;
}

__device__ __forceinline__ unsigned long long ceil16(unsigned long long v)
{
    return (v + 15ull) & ~15ull;
}

// ---- warp bit-matrix transpose -----------------------------------------
// Lane i holds word u_i; afterwards lane k holds the word whose bit i is bit k
// of u_i.  Five butterfly stages exchange the off-diagonal sub-blocks of the
// current block size through one shuffle each: the two byte-granular stages
// (16- and 8-bit blocks) merge with one byte permute, the three sub-byte
// stages with one funnel rotate and one bit-select.  The per-lane selectors,
// rotate counts and masks are computed once per kernel (TpC).  The transpose
// is its own inverse.  If every u_i < 2^16, packing two rows as
// u_a | u_b << 16 transposes both at once: lanes 0..15 get the planes of a,
// lanes 16..31 those of b.
struct TpC {
    uint32_t s16, s8, r4, r2, r1, k4, k2, k1;
};
__device__ __forceinline__ TpC tp_consts(int lane)
{
    TpC c;
    c.s16 = (lane & 16) ? 0x3276u : 0x5410u;
    c.s8 = (lane & 8) ? 0x3715u : 0x6240u;
    c.r4 = (lane & 4) ? 28u : 4u;
    c.k4 = (lane & 4) ? 0xf0f0f0f0u : 0x0f0f0f0fu;
    c.r2 = (lane & 2) ? 30u : 2u;
    c.k2 = (lane & 2) ? 0xccccccccu : 0x33333333u;
    c.r1 = (lane & 1) ? 31u : 1u;
    c.k1 = (lane & 1) ? 0xaaaaaaaau : 0x55555555u;
    return c;
}
__device__ __forceinline__ uint32_t tpose(uint32_t u, const TpC& c)
{
    uint32_t p = __shfl_xor_sync(FULL, u, 16);
    u = __byte_perm(u, p, c.s16);
    p = __shfl_xor_sync(FULL, u, 8);
    u = __byte_perm(u, p, c.s8);
    p = __shfl_xor_sync(FULL, u, 4);
    u = (u & c.k4) | (__funnelshift_l(p, p, c.r4) & ~c.k4);
    p = __shfl_xor_sync(FULL, u, 2);
    u = (u & c.k2) | (__funnelshift_l(p, p, c.r2) & ~c.k2);
    p = __shfl_xor_sync(FULL, u, 1);
    u = (u & c.k1) | (__funnelshift_l(p, p, c.r1) & ~c.k1);
    return u;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while the kernel before it on the stream still
// runs; grid_dep_wait() blocks until that kernel has completed and its memory
// operations are visible (it returns at once in a kernel launched without
// the attribute).  grid_dep_launch() lets the dependent kernel start early.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Inclusive prefix sum over segments of W lanes, using the in-range predicate
// of shfl.up so each step is one shuffle and one predicated add.
template <int W>
__device__ __forceinline__ int scan_incl(int v)
{
#pragma unroll
    for (int off = 1; off < W; off <<= 1) {
        asm("{\n\t.reg .s32 t;\n\t.reg .pred p;\n\t"
            "shfl.sync.up.b32 t|p, %0, %1, %2, -1;\n\t"
            "@p add.s32 %0, %0, t;\n\t}"
            : "+r"(v)
            : "r"(off), "r"((32 - W) << 8));
    }
    return v;
}

// ---- prequantization ------------------------------------------------------
// q = the integer nearest to x / two_eb, ties to even, exactly.
// Fast path: v = x * inv rounds (at most two roundings) to within |v| 2^-22.9
// of the exact quotient; if v is farther than |v| 2^-22 from a half-integer,
// rint(v) is the exact answer.  The test f + |v| 2^-22 < 0.5 (f = |v - rint v|,
// exact) is rounded once; its rounding error (at most 2^-26 near 0.5) stays
// inside the factor-two margin for |v| > 1/8, and for |v| <= 1/8 both v and
// the quotient round to 0.  rint uses the 1.5 * 2^23 magic add (exact for
// |v| < 2^22; the fast test already fails for |v| >= 2^21).
// Slow path (near a tie, large |v|, non-finite): q0 = rint(v), then the
// residual r = x - q0 * two_eb, rounded once by an FMA, decides exactly
// whether q0 or its neighbour is nearest (the residual is a multiple of
// ulp(eb) near |r| = eb, so rounding cannot move it across eb).
// Returns 0 or a zc_status code.
// Branch-free fast path of quantize(): q = rint(x * inv); returns false when
// that may differ from the exact rounding (near a tie, |v| >= 2^21, NaN/Inf).
__device__ __forceinline__ bool quantize_fast(float x, float inv, int& q)
{
    const float v = __fmul_rn(x, inv);
    const float t = __fadd_rn(v, 12582912.0f);
    const float r = __fsub_rn(t, 12582912.0f);
    const float f = fabsf(__fsub_rn(v, r));
    q = __float_as_int(t) - 0x4b400000;
    return __fmaf_rn(fabsf(v), 2.384185791015625e-07f, f) < 0.5f;  // |v| * 2^-22
}

// The same, returning the bit pattern of the rounded float (q + QBIAS):
// differences of two such values are differences of q, so an encoder that
// only needs deltas skips the offset.
constexpr int QBIAS = 0x4b400000;  // the bits of 1.5 * 2^23, the rounding constant
__device__ __forceinline__ bool quantize_fast_bits(float x, float inv, int& qb)
{
    const float v = __fmul_rn(x, inv);
    const float t = __fadd_rn(v, 12582912.0f);
    const float r = __fsub_rn(t, 12582912.0f);
    const float f = fabsf(__fsub_rn(v, r));
    qb = __float_as_int(t);
    return __fmaf_rn(fabsf(v), 2.384185791015625e-07f, f) < 0.5f;  // |v| * 2^-22
}

__device__ __forceinline__ int quantize(float x, float eb, float two_eb, float inv, int& q)
{
    const float v = __fmul_rn(x, inv);
    const float t = __fadd_rn(v, 12582912.0f);
    const float r = __fsub_rn(t, 12582912.0f);
    const float f = fabsf(__fsub_rn(v, r));
    if (__fmaf_rn(fabsf(v), 2.384185791015625e-07f, f) < 0.5f) {  // |v| * 2^-22
        q = __float_as_int(t) - 0x4b400000;
        return 0;
    }
    q = 0;
    if (!isfinite(x)) return ZC_ERR_NONFINITE;
    if (!(fabsf(v) <= 4194308.0f)) return ZC_ERR_RANGE;
    int q0 = __float2int_rn(v);
    const float res = __fmaf_rn(-__int2float_rn(q0), two_eb, x);
    const float ares = fabsf(res);
    const int step = res > 0.0f ? 1 : -1;
    if (ares > eb) q0 += step;
    else if (ares == eb && (q0 & 1)) q0 += step;
    if (q0 > QMAX || q0 < -QMAX) return ZC_ERR_RANGE;
    q = q0;
    return 0;
}

// ---- decoupled look-back over tile byte counts ---------------------------
// A chain of tiles computes, in one pass, the byte position where each tile's
// payload starts.  Tile t contributes a transform X -> X + a, or, when it ends
// a stream (h), X -> ceil16(X + a) + b (the stream is padded to 16 bytes).
// Transforms compose associatively, so a tile sums its predecessors'
// published aggregates until it meets a published inclusive prefix.
struct Xf {
    unsigned long long a, b;
    bool h;
};
__device__ __forceinline__ Xf xf_id() { return Xf{0ull, 0ull, false}; }
// apply f first, then s
__device__ __forceinline__ Xf xf_compose(const Xf& f, const Xf& s)
{
    Xf r;
    if (!s.h) {
        r.h = f.h;
        r.a = f.h ? f.a : f.a + s.a;
        r.b = f.h ? f.b + s.a : 0ull;
    } else if (!f.h) {
        r.h = true;
        r.a = f.a + s.a;
        r.b = s.b;
    } else {
        r.h = true;
        r.a = f.a;
        r.b = ceil16(f.b + s.a) + s.b;
    }
    return r;
}
__device__ __forceinline__ unsigned long long xf_apply(const Xf& f, unsigned long long x)
{
    return f.h ? ceil16(x + f.a) + f.b : x + f.a;
}
__device__ __forceinline__ Xf xf_shfl_up(const Xf& f, int off)
{
    Xf o;
    o.a = __shfl_up_sync(FULL, f.a, off);
    o.b = __shfl_up_sync(FULL, f.b, off);
    o.h = __shfl_up_sync(FULL, (int)f.h, off) != 0;
    return o;
}
__device__ __forceinline__ Xf xf_shfl(const Xf& f, int src)
{
    Xf o;
    o.a = __shfl_sync(FULL, f.a, src);
    o.b = __shfl_sync(FULL, f.b, src);
    o.h = __shfl_sync(FULL, (int)f.h, src) != 0;
    return o;
}

// Look-back record of a tile: 16 bytes, written by one 16-byte store and
// read by one 16-byte load, so the state and its value travel together and
// no fence orders them.  x: [63:32] launch generation E, [31:30] state,
// [29] h (the tile ends a stream).  y: [63:40] the low 24 bits of E again, a
// check that the value belongs to the same store as the state, [39:0] the
// value: the tile's aggregate (state AGG) or inclusive prefix (PREFIX).
// Values are byte counts below 2^40.
constexpr unsigned ST_AGG = 1u, ST_PREFIX = 2u;
constexpr int REC_VAL_BITS = 40;
constexpr unsigned long long REC_VAL_MASK = (1ull << REC_VAL_BITS) - 1ull;

struct Chain {
    ulonglong2* rec;  // per tile (16-byte aligned)
};

__device__ __forceinline__ void rec_store(ulonglong2* p, unsigned E, unsigned st, bool h,
                                          unsigned long long v)
{
    const unsigned long long x = ((unsigned long long)E << 32) | ((unsigned long long)st << 30) |
                                 ((unsigned long long)h << 29);
    const unsigned long long y = ((unsigned long long)(E & 0xffffffu) << REC_VAL_BITS) |
                                 (v & REC_VAL_MASK);
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(x), "l"(y)
                 : "memory");
}
__device__ __forceinline__ ulonglong2 rec_load(const ulonglong2* p)
{
    ulonglong2 r;
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];"
                 : "=l"(r.x), "=l"(r.y)
                 : "l"(p)
                 : "memory");
    return r;
}
__device__ __forceinline__ bool rec_valid(const ulonglong2& r, unsigned E)
{
    return (unsigned)(r.x >> 32) == E && ((r.x >> 30) & 3u) != 0u &&
           (unsigned)(r.y >> REC_VAL_BITS) == (E & 0xffffffu);
}
__device__ __forceinline__ unsigned rec_state(const ulonglong2& r) { return (unsigned)(r.x >> 30) & 3u; }
__device__ __forceinline__ bool rec_h(const ulonglong2& r) { return ((r.x >> 29) & 1ull) != 0ull; }
__device__ __forceinline__ unsigned long long rec_val(const ulonglong2& r) { return r.y & REC_VAL_MASK; }

struct WaitCfg {
    unsigned long long limit_ns;
    long long withhold;  // tile that never publishes (test hook), -1 = none
};

// Scratch of the look-back.
struct LbSmem {
    unsigned long long excl;
    int timed_out;
};

constexpr int LB_PER_LANE = 4;                 // predecessors inspected per lane
constexpr int LB_WINDOW = 32 * LB_PER_LANE;    // predecessors per look-back round

// Run by one whole warp.  g: this tile's slot; g0: first slot of its chain
// (whose exclusive value is 0).  Publishes g's aggregate (unless the caller
// already has: agg_out), then inspects the LB_WINDOW preceding slots
// (LB_PER_LANE consecutive slots per lane), waits until all of them have
// published, composes the aggregates after the nearest inclusive prefix, and
// repeats further back if there is none.  Publishes g's inclusive prefix and
// returns g's exclusive value (the same in every lane).  If the wait runs
// out, records ZC_ERR_TIMEOUT, sets `expired` and returns 0 (the prefix is
// still published, so the chain moves on; the status word already marks the
// result unusable).
__device__ __forceinline__ unsigned long long lookback_warp(const Chain& ch, unsigned g,
                                                            unsigned g0, unsigned long long agg,
                                                            bool h, unsigned E, const WaitCfg& wc,
                                                            Ctl* ctl, bool& expired,
                                                            bool agg_out = false)
{
    const int lane = threadIdx.x & 31;
    const bool publish = (long long)g != wc.withhold;
    const Xf self{agg, 0ull, h};
    expired = false;
    if (g == g0) {
        if (lane == 0 && publish) rec_store(ch.rec + g, E, ST_PREFIX, h, xf_apply(self, 0ull));
        return 0ull;
    }
    if (lane == 0 && publish && !agg_out) rec_store(ch.rec + g, E, ST_AGG, h, agg);
    Xf acc = xf_id();
    long long hi = (long long)g - 1;
    unsigned long long excl = 0ull;
    const unsigned long long t0 = globaltimer();
    while (true) {
        // slots j0 .. j0 + LB_PER_LANE - 1 of this lane, oldest first
        const long long j0 = hi - (LB_WINDOW - 1) + (long long)lane * LB_PER_LANE;
        ulonglong2 f[LB_PER_LANE];
        unsigned valid = 0;
#pragma unroll
        for (int i = 0; i < LB_PER_LANE; ++i) {
            const long long j = j0 + i;
            if (j < (long long)g0) {
                f[i] = make_ulonglong2(0ull, 0ull);
                valid |= 1u << i;
            } else {
                f[i] = rec_load(ch.rec + j);
                if (rec_valid(f[i], E)) valid |= 1u << i;
            }
        }
        unsigned ns = 32;
        while (!__all_sync(FULL, valid == (1u << LB_PER_LANE) - 1u)) {
            expired = __any_sync(FULL, globaltimer() - t0 > wc.limit_ns);
            if (expired) break;
            __nanosleep(ns);
            ns = ns < 256 ? ns * 2 : ns;
#pragma unroll
            for (int i = 0; i < LB_PER_LANE; ++i) {
                if (!((valid >> i) & 1u)) {
                    f[i] = rec_load(ch.rec + (j0 + i));
                    if (rec_valid(f[i], E)) valid |= 1u << i;
                }
            }
        }
        if (expired) {
            if (lane == 0) fail(ctl, ZC_ERR_TIMEOUT, g);
            excl = 0ull;
            break;
        }
        // this lane's newest prefix slot (virtual slots before g0 count as prefix 0)
        int pi = -1;
#pragma unroll
        for (int i = 0; i < LB_PER_LANE; ++i) {
            const bool is_pref = (j0 + i < (long long)g0) || rec_state(f[i]) == ST_PREFIX;
            if (is_pref) pi = i;
        }
        const unsigned pm = __ballot_sync(FULL, pi >= 0);
        const int pl = pm ? 31 - __clz(pm) : -1;  // lane holding the newest prefix
        // this lane's composed transform of its slots after the newest prefix
        Xf t = xf_id();
        if (lane >= pl) {
#pragma unroll
            for (int i = 0; i < LB_PER_LANE; ++i) {
                const long long j = j0 + i;
                if (j >= (long long)g0 && (lane > pl || i > pi)) {
                    Xf x;
                    x.h = rec_h(f[i]);
                    x.a = rec_val(f[i]);
                    x.b = 0ull;
                    t = xf_compose(t, x);
                }
            }
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const Xf o = xf_shfl_up(t, off);
            if (lane >= off) t = xf_compose(o, t);
        }
        acc = xf_compose(xf_shfl(t, 31), acc);
        if (pl >= 0) {
            unsigned long long pv = 0ull;
#pragma unroll
            for (int i = 0; i < LB_PER_LANE; ++i)
                if (lane == pl && i == pi && j0 + pi >= (long long)g0) pv = rec_val(f[i]);
            pv = __shfl_sync(FULL, pv, pl);
            excl = xf_apply(acc, pv);
            break;
        }
        hi -= LB_WINDOW;
    }
    if (lane == 0 && publish)
        rec_store(ch.rec + g, E, ST_PREFIX, h, xf_apply(self, expired ? 0ull : excl));
    return excl;
}

// The same for a whole CTA: warp 0 runs the look-back while the other warps
// wait at a barrier; every thread gets the exclusive value.
__device__ __forceinline__ unsigned long long lookback_cta(const Chain& ch, unsigned g,
                                                           unsigned g0, unsigned long long agg,
                                                           bool h, unsigned E, const WaitCfg& wc,
                                                           Ctl* ctl, bool& timed_out, LbSmem& ls)
{
    if (threadIdx.x < 32) {
        bool expired = false;
        const unsigned long long ex = lookback_warp(ch, g, g0, agg, h, E, wc, ctl, expired);
        if (threadIdx.x == 0) {
            ls.excl = ex;
            ls.timed_out = expired;
        }
    }
    __syncthreads();
    timed_out = ls.timed_out != 0;
    const unsigned long long ex = ls.excl;
    __syncthreads();  // ls may be reused right after
    return ex;
}

// Named barriers (ids 1..15) shared by a subset of a CTA's warps: `n`
// threads (whole warps) take part.  bar.arrive does not wait; both order the
// caller's earlier memory accesses before the barrier completes.
__device__ __forceinline__ void bar_sync_n(unsigned id, unsigned n)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(unsigned id, unsigned n)
{
    asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bounded wait for a record published with rec_store (generation E, any
// state); returns false if the wait ran out, else its value in `v`.
__device__ __forceinline__ bool wait_rec(const ulonglong2* p, unsigned E,
                                         unsigned long long limit_ns, unsigned long long& v)
{
    unsigned long long t0 = 0ull;
    unsigned ns = 32;
    while (true) {
        const ulonglong2 r = rec_load(p);
        if (rec_valid(r, E)) {
            v = rec_val(r);
            return true;
        }
        const unsigned long long now = globaltimer();
        if (t0 == 0ull) t0 = now;
        else if (now - t0 > limit_ns) return false;
        __nanosleep(ns);
        ns = ns < 2048 ? ns * 2 : ns;
    }
}

// ---- element access -------------------------------------------------------

__device__ __forceinline__ float bf16_to_f32(uint16_t b)
{
    return __uint_as_float((uint32_t)b << 16);
}
// Round to nearest even; the reconstruction is finite.
__device__ __forceinline__ uint16_t f32_to_bf16(float f)
{
    uint32_t u = __float_as_uint(f);
    if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)((u >> 16) | ((u & 0x7fffffu) ? 0x40u : 0u));
    u += 0x7fffu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

}  // namespace zc
