// zc_codec.cuh -- the tile kernels: compress, decompress, the fused ring step
// (decompress -> add -> recompress) and the scatter pack.
//
// Geometry.  A CTA is 8 warps.  A sub-tile is 2048 consecutive elements: each
// warp owns R = 8 rows of 32, lane i holding element i of a row.  A block of
// L elements is L/32 rows (L >= 32) or half a row (L = 16); blocks never
// straddle warps.
//
// Encoding a row: exact quantization, Lorenzo delta against the previous
// element of the block (the block head against 0), the magnitude shifted left
// with the sign in bit 0, then one warp bit-matrix transpose: lane k then
// holds bit plane k-1 (lane 0: the sign plane) of the row, so a block with
// w-bit deltas is exactly lanes 0 .. w of its rows.  Decoding runs the same
// steps backwards with an inclusive warp scan in place of the delta.
//
// Encoder offsets.  An encoder tile is S sub-tiles.  Every warp appends its
// blocks' planes to its own shared-memory segment of each sub-tile (the
// running offset is warp-uniform: no scan), so nothing waits until the whole
// tile is encoded.  Then one CTA scan over the 8 S segment sizes, one
// CTA-wide decoupled look-back for the tile's position in the stream, and a
// coalesced copy of every segment to its place.  The first tile of a stream
// also counts the 32-byte header and the padded width bytes; the last one
// rounds the stream up to 16 bytes; in packed mode (the scatter pack) one
// chain runs through all streams.
//
// Decoder offsets.  k_wscan reads only the width bytes of a stream and
// writes the payload offset of every 2048-element decode tile (a chain over
// 256-tile chunks); decoding then needs no look-back and no barrier.
#pragma once

#include <type_traits>

#include "zc_device.cuh"

namespace zc {

constexpr int GR = 8;                  // rows held in registers at a time
constexpr int WSCAN = NTHREADS;        // warp units per width-scan chunk
constexpr int DEC_U = 64;              // rows per warp unit of the decompressor
// Batched decompression: items of at most this many decode tiles get no
// width-scan chunks; their decoder CTAs find the unit offsets themselves.
constexpr unsigned DEC_LOCAL_TILES = 4;

// Rows per warp unit of an encoder tile of `chunks` 2048-element chunks.
__host__ __device__ constexpr int unit_rows(int chunks) { return chunks * 8; }
// Largest payload of one warp unit of U rows: 32 U elements x 25 planes / 8.
__host__ __device__ constexpr int seg_bytes(int U) { return U * 100; }

struct Item {
    const void* x;            // raw input (compress) or local chunk (ring step), or null
    const uint8_t* cin;       // received stream, or null
    uint8_t* out;             // output stream (non-packed) / packed buffer base, or null
    void* raw_out;            // decoded values / FP32 sum, or null
    unsigned long long* out_bytes;
    unsigned long long n, cin_cap, out_cap;
    float eb, two_eb, inv;    // encoding bound
    unsigned tile_begin, ntiles;    // tiles of this launch's geometry
    unsigned chunk_begin, nchunks;  // width-scan chunks
    int x_dtype, out_dtype;
    int log2L;                // batched compression: block size, or -1 for a raw stream
};

struct Launch {
    Ctl* ctl;
    Chain chB;                        // encoder tiles
    Chain chC;                        // width-scan chunks
    unsigned long long* offs;         // payload offset of every decode tile (global slot)
    ulonglong2* seg_rec;              // packed mode: stream start published per item
    unsigned long long* seg_off;      // packed mode: P + 1 stream offsets (caller's)
    const Item* items;                // device items, or null for `one`
    Item one;
    unsigned n_items, total_tiles;    // total_tiles: tiles (or chunks for k_wscan)
    int urows;                        // rows per warp unit (decode slot = tile * NWARPS + warp)
    int eb_from_ctl;                  // relative bound resolved into ctl
    int packed;
    WaitCfg wc;
    // batched decompression: item i's stream sits at in_base + in_off[i] (in_off
    // written by an earlier launch; in_cap bytes at in_base)
    const uint8_t* in_base;
    const unsigned long long* in_off;
    unsigned long long in_cap;
    // item of every tile (written by k_tile_map before the launch), or null:
    // then the item is found by a binary search over tile_begin
    const unsigned* tile_map;
    // encoder launches: the CTAs' tile rings (ring_cta_bytes each, in CTA order)
    uint8_t* ring;
    unsigned long long ring_bytes;
    unsigned long long ws_cap;  // entries of every workspace array (bounds-checked builds)
    // grouped batch (packed mode): the streams lie in ticket order, not item
    // order, so seg_off[i] is only item i's start and seg_off[n_items] the
    // packed total; a decoder bounds a stream by seg_off[n_items]
    int grouped;
    // encoder launches: launched dependent on the kernel just before on the
    // stream (programmatic serialisation), whose results the CTAs wait for
    // in their prologue (a relative bound, eb_from_ctl, implies it)
    int dep;
};

struct Smem {
    LbSmem lb;
    unsigned long long base, start, end;
    unsigned ticket, item, E;
    int abort, hdr_lg;
    float eb, two_eb, inv;
};

// Encoder CTAs: NWARPS encoder warps plus one resolver warp, enc_slots(U)
// tiles in flight.  Every tile slot has, per encoder warp, a payload segment
// of seg_bytes(U) in the CTA's ring (global memory) and U * 2 width bytes in
// shared memory.  Three slots give the resolver two tiles' time; the largest
// tiles take two, which keeps the rings of all CTAs inside L2.
__host__ __device__ constexpr int enc_slots(int U) { return U >= 128 ? 2 : 3; }
constexpr int ENC_SLOTS_MAX = 3;
constexpr int ENC_THREADS = NTHREADS + 32;
constexpr int ENC_CTAS_PER_SM = 4;            // resident encoder CTAs per SM (registers)
constexpr unsigned BAR_ENCW = 1;              // named barrier: the encoder warps
constexpr unsigned BAR_ENC = 2;               // + slot: tile encoded (resolver waits)
constexpr unsigned BAR_RES = BAR_ENC + ENC_SLOTS_MAX;  // + slot: tile resolved (encoders wait)
static_assert(BAR_RES + ENC_SLOTS_MAX <= 16, "named barriers per CTA");
__host__ __device__ constexpr unsigned long long ring_cta_bytes(int U)
{
    return (unsigned long long)enc_slots(U) * NWARPS * seg_bytes(U);
}
// Rows of a warp unit staged in shared memory before a copy to the ring: the
// whole unit up to 64 rows for the single-stream kernels (compress, scatter
// pack), 32 rows at a time otherwise (16-chunk tiles, the batch kernel with
// its many code paths, the fused ring step whose decoder metadata also takes
// shared memory), so that 4 CTAs fit an SM; the stage holds their worst case
// plus the carried partial 16 bytes.
__host__ __device__ constexpr int stage_rows(int U, bool single) { return (single && U <= 64) ? U : 32; }
__host__ __device__ constexpr int stage_bytes(int rows) { return seg_bytes(rows) + 16; }
// Dynamic shared memory of an encoder CTA: width bytes of every slot and
// warp, then every encoder warp's stage.
__host__ __device__ constexpr int enc_wb_bytes(int U) { return enc_slots(U) * NWARPS * U * 2; }
// (The single-stream kernels take their stages in dynamic shared memory;
// the others in a static array of 32-row stages, which leaves the driver
// free to give the rest of the SM's memory to L1.)
__host__ __device__ constexpr int enc_smem_bytes(int U, bool single = false)
{
    return enc_wb_bytes(U) + (single ? NWARPS * stage_bytes(stage_rows(U, true)) : 0);
}

template <typename T>
__device__ __forceinline__ float load_x(const T* p, int i);
template <>
__device__ __forceinline__ float load_x<float>(const float* p, int i)
{
    return __ldcs(p + i);  // read once: evict first, the tile rings stay in L2
}
template <>
__device__ __forceinline__ float load_x<uint16_t>(const uint16_t* p, int i)
{
    return bf16_to_f32(__ldcs((const unsigned short*)p + i));
}

__device__ __forceinline__ void store_raw(void* p, int dtype, unsigned long long i, float v)
{
    if (dtype == ZC_F32) ((float*)p)[i] = v;
    else ((uint16_t*)p)[i] = f32_to_bf16(v);
}

__device__ __forceinline__ int warp_excl_scan(int v, int lane, int& total)
{
    int s = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int o = __shfl_up_sync(FULL, s, off);
        if (lane >= off) s += o;
    }
    total = __shfl_sync(FULL, s, 31);
    return s - v;
}

__device__ __forceinline__ int warp_sum(int v)
{
#pragma unroll
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(FULL, v, off);
    return v;
}

// Reads and checks an input stream header for `it`; returns its log2 L (plus
// 8 when its block heads are stored apart), -1 for a format error (reported
// when `report`), -2 / -3 for a raw FP32 / BF16 stream.  A caller that names
// the block size it expects (the fused ring step) takes plain streams only.
__device__ __forceinline__ int check_header(const Item& it, Ctl* ctl, unsigned item_idx,
                                            int expect_log2L, float& eb_in, bool report)
{
    const uint8_t* s = it.cin;
    if (it.cin_cap < 32) {
        if (report) fail(ctl, ZC_ERR_FORMAT, item_idx);
        return -1;
    }
    const uint32_t w0 = __ldg((const unsigned*)s);
    const uint32_t w1 = __ldg((const unsigned*)s + 1);
    const unsigned long long n = __ldg((const unsigned long long*)s + 1);
    eb_in = __uint_as_float(__ldg((const unsigned*)s + 4));
    const uint32_t nb = __ldg((const unsigned*)s + 5);
    const unsigned long long payload = __ldg((const unsigned long long*)s + 3);
    const int dtype = w1 & 0xff, lg = (w1 >> 8) & 0xff, flags = (w1 >> 16) & 0xff;
    bool ok = w0 == 0x3176435au && (w1 >> 24) == 0u && (dtype == 0 || dtype == 1) &&
              (flags & ~3) == 0 && flags != 3 && n == it.n;
    int ret = lg;
    if (ok && (flags & 1)) {
        const unsigned long long es = dtype == 0 ? 4ull : 2ull;
        ok = nb == 0u && payload == n * es && 32ull + ceil16(payload) <= it.cin_cap &&
             expect_log2L < 0;
        ret = -2 - dtype;
    } else if (ok) {
        const bool heads = (flags & 2) != 0;
        ok = lg >= 4 && lg <= 7 && (expect_log2L < 0 || (lg == expect_log2L && !heads)) &&
             (unsigned long long)nb == ((n + (1ull << lg) - 1) >> lg) &&
             32ull + ceil16(nb) + (heads ? ceil16(3ull * nb) : 0ull) + ceil16(payload) <=
                 it.cin_cap;
        if (ok && nb > 0) ok = is_normal(eb_in) && eb_in > 0.0f && isfinite(eb_in + eb_in);
        if (heads) ret = lg + 8;
    }
    if (!ok) {
        if (report) fail(ctl, ZC_ERR_FORMAT, item_idx);
        return -1;
    }
    return ret;
}

__device__ __forceinline__ int planes_of(int w) { return w ? w + 1 : 0; }


__device__ __forceinline__ uint8_t width_byte(int np) { return (uint8_t)(np ? np - 1 : 0); }

// width_byte of four blocks at once, from their plane counts packed one per
// byte (each at most 32).  Adding 0x7f to a byte sets its top bit exactly when
// its count is nonzero and carries into no neighbour, so subtracting those
// bits, shifted down to bit 0, borrows across no byte.
__device__ __forceinline__ uint32_t width_bytes4(uint32_t c)
{
    return c - (((c + 0x7f7f7f7fu) & 0x80808080u) >> 7);
}

// Inclusive prefix sum of exact FP32 integers over 32 lanes (FMA pipe).
__device__ __forceinline__ float scan_incl_f(float v)
{
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        asm("{\n\t.reg .f32 t;\n\t.reg .pred p;\n\t"
            "shfl.sync.up.b32 t|p, %0, %1, 0, -1;\n\t"
            "@p add.rn.f32 %0, %0, t;\n\t}"
            : "+f"(v)
            : "r"(off));
    }
    return v;
}
// The same over segments of 16 lanes.
__device__ __forceinline__ float scan_incl_f16(float v)
{
#pragma unroll
    for (int off = 1; off < 16; off <<= 1) {
        asm("{\n\t.reg .f32 t;\n\t.reg .pred p;\n\t"
            "shfl.sync.up.b32 t|p, %0, %1, 4096, -1;\n\t"
            "@p add.rn.f32 %0, %0, t;\n\t}"
            : "+f"(v)
            : "r"(off));
    }
    return v;
}

// ---- decoding ------------------------------------------------------------------
// Two rows' sign-magnitude words u_a | u_b << 16 (each below 2^11: |d| <=
// 1023) -> d_a + B | (d_b + B) << 16 with B = 1024: both halves in [1, 2047],
// so an integer prefix sum over 32 lanes (at most 65504 per half) carries
// nothing from one half into the other and two rows scan with one shuffle per
// step.  Sum at lane j: q_j - q_-1 + (j + 1) B, q_-1 the value before the row.
constexpr uint32_t PAIR_B = 1024u;
constexpr int PAIR_MAX_PLANES = 11;
__device__ __forceinline__ uint32_t biased_pair(uint32_t t)
{
    const uint32_t m2 = (t >> 1) & 0x7fff7fffu;                  // magnitudes
    const uint32_t plus = (PAIR_B | PAIR_B << 16) + m2;
    const uint32_t minus = (PAIR_B | PAIR_B << 16) - m2;         // no borrow: each half >= 1
    const uint32_t neg = (t & 0x00010001u) * 0xffffu;            // all-ones halves where d < 0
    return (plus & ~neg) | (minus & neg);
}
// Exact FP32 of a half of a biased pair scan: (half + kbits) holds the float
// bits of q + 1.5 * 2^23 (|q| < 2^22), kbits = 0x4b400000 - (j + 1) B (+ the
// value before the row when it is nonzero, added by the caller in FP32).
__device__ __forceinline__ float pair_half_f(uint32_t half, uint32_t kbits)
{
    return __fsub_rn(__uint_as_float(half + kbits), 12582912.0f);
}

// Block planes and payload offsets of one warp unit of an input stream:
// meta[b] = (planes, byte offset from the unit's payload start) for the
// unit's blocks.  Returns the unit's payload start in the stream; a unit whose
// planes would lie beyond cin_cap is reported and gets zero planes.
// off_local >= 0: the unit's payload offset found by the caller (a small
// item's decoder CTA), in place of the width scan's P.offs[slot].
template <int LOG2L, int U, bool HEADS = false>
__device__ __forceinline__ unsigned long long unit_meta(const Launch& P, const Item& it,
                                                        unsigned slot, unsigned long long ue0,
                                                        int2* meta, bool& narrow, bool& narrow11,
                                                        long long off_local = -1)
{
    constexpr int L = 1 << LOG2L;
    constexpr int PB = L / 8;
    constexpr int BU = U * 32 / L;                // blocks per unit
    constexpr int BPL = BU >= 32 ? BU / 32 : 1;   // blocks per lane
    const int lane = threadIdx.x & 31;
    const unsigned long long nb = (it.n + L - 1) >> LOG2L;
    const unsigned long long b0 = (ue0 >> LOG2L) + (unsigned long long)lane * BPL;
    static_assert(BPL == 1 || BPL == 2 || BPL == 4 || BPL == 8, "width bytes per lane");
    const bool mine = BU >= 32 || lane < BU;
    uint32_t wv[2] = {0u, 0u};  // this lane's BPL width bytes, little-endian
    if (mine && b0 < ceil16(nb)) {
        // b0 is a multiple of BPL and the width bytes are zero padded to 16:
        // the BPL bytes from b0 are inside the stream and naturally aligned
        const uint8_t* wp = it.cin + 32 + b0;
        if (BPL == 8) {
            const uint2 v = __ldg((const uint2*)wp);
            wv[0] = v.x;
            wv[1] = v.y;
        } else if (BPL == 4) {
            wv[0] = __ldg((const unsigned*)wp);
        } else if (BPL == 2) {
            wv[0] = __ldg((const unsigned short*)wp);
        } else {
            wv[0] = __ldg(wp);
        }
    }
    int np[BPL];
    int sum = 0;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < BPL; ++i) {
        int w = (wv[i >> 2] >> (8 * (i & 3))) & 0xff;
        if (w > ZC_MAX_WIDTH) {
            bad = true;
            w = 0;
        }
        np[i] = planes_of(w);
        sum += np[i] * PB;
    }
    if (bad) fail(P.ctl, ZC_ERR_FORMAT, b0);
    {
        int npmax = 0;
#pragma unroll
        for (int i = 0; i < BPL; ++i) npmax = max(npmax, np[i]);
        narrow = __all_sync(FULL, npmax <= 16);
        narrow11 = !HEADS && __all_sync(FULL, npmax <= PAIR_MAX_PLANES);
    }
    int tot;
    int off = warp_excl_scan(sum, lane, tot);
    const bool slot_ok = off_local >= 0 || dcheck(P.ctl, slot < P.ws_cap, slot);
    const unsigned long long uoff =
        off_local >= 0 ? (unsigned long long)off_local : (slot_ok ? P.offs[slot] : 0ull);
    const unsigned long long base = 32ull + ceil16(nb) + (HEADS ? ceil16(3ull * nb) : 0ull) + uoff;
    const bool ok = slot_ok && base + (unsigned long long)tot <= it.cin_cap;
    if (!ok && lane == 0) fail(P.ctl, ZC_ERR_FORMAT, slot);
    if (DEBUG_BUILD && mine && lane == (BU >= 32 ? 31 : BU - 1))
        dcheck(P.ctl, off + sum == tot, slot);  // the last block's planes end at the unit's
    __syncwarp();  // earlier readers of meta are done
    if (mine) {
#pragma unroll
        for (int i = 0; i < BPL; ++i) {
            meta[lane * BPL + i] = make_int2(ok ? np[i] : 0, off);
            off += np[i] * PB;
        }
    }
    __syncwarp();
    // the whole unit payload is requested into L2 at once (one bulk prefetch,
    // 16-byte aligned inner range); the per-group plane loads then hit L2
    if (ok && lane == 0 && tot > 0) {
        const uintptr_t a0 = (uintptr_t)(it.cin + base), a1 = a0 + (uintptr_t)tot;
        const uintptr_t s0 = (a0 + 15) & ~(uintptr_t)15, s1 = a1 & ~(uintptr_t)15;
        if (s1 > s0)
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s0),
                         "r"((unsigned)(s1 - s0))
                         : "memory");
    }
    return ok ? base : 0ull;
}

// Sign-magnitude word of one element -> its delta as an exact FP32 value
// (|d| < 2^23), the sign injected into the float's sign bit.
__device__ __forceinline__ float delta_f(uint32_t u)
{
    const float mag = __fsub_rn(__int_as_float((u >> 1) | 0x4b000000u), 8388608.0f);
    return __int_as_float(__float_as_int(mag) ^ (u << 31));
}

// Decodes rows [g GR, g GR + GR) of a warp unit into acc[] (x^ = q * 2eb).
// `src` points at the unit's payload, `meta` at its block metadata.  All of
// the group's plane words are requested before the first transpose so their
// loads overlap.  A pair of rows whose blocks have at most 16 planes shares
// one transpose and is scanned in FP32 (every partial sum is an integer below
// 2^22: exact); wider rows are scanned in integers.
// Block head of the heads-apart format: 24-bit two's complement, little-endian.
__device__ __forceinline__ int load_head(const uint8_t* p)
{
    const unsigned v = (unsigned)__ldg(p) | ((unsigned)__ldg(p + 1) << 8) |
                       ((unsigned)__ldg(p + 2) << 16);
    return (int)v - ((v & 0x800000u) ? (1 << 24) : 0);
}

template <int LOG2L, bool NARROW, bool HEADS = false, bool BIASED = false>
__device__ __forceinline__ void decode_group(const uint8_t* src, const int2* meta, int g,
                                             float two_eb, float acc[GR], const TpC& tc,
                                             const uint8_t* hsrc = nullptr)
{
    constexpr int L = 1 << LOG2L;
    constexpr int RPB = L >= 32 ? L / 32 : 1;
    constexpr int NR = L == 128 ? 4 : 2;  // rows per step (pair, or quad at L = 128)
    constexpr int NS = GR / NR;           // steps per group
    const int lane = threadIdx.x & 31;
    const int k = lane & 15;
    const bool hi = lane >= 16;
    const int fb = L >= 32 ? g * GR / RPB : g * GR * 2;  // first block of the group
    const int2* mt = meta + fb;
    // ---- phase 1: metadata, plane loads (and block heads) of every step ----
    int hv[GR];  // heads apart: the head of this lane's block where this lane is one
    if (HEADS) {
#pragma unroll
        for (int r = 0; r < GR; ++r) {
            hv[r] = 0;
            int b = -1;  // block of the unit whose head this lane holds in row r
            if (L == 16 && k == 0) b = 2 * (g * GR + r) + (hi ? 1 : 0);
            else if (L == 32 && lane == 0) b = g * GR + r;
            else if (L >= 64 && lane == 0 && (r % RPB) == 0) b = (g * GR + r) / RPB;
            if (b >= 0) hv[r] = load_head(hsrc + 3 * b);
        }
    }
    uint32_t wv[NS][NR];
    unsigned paired = 0;  // bit s: step s has at most 16 planes per block
    static_assert(!BIASED || (NARROW && !HEADS), "the biased pair scan: narrow plain units");
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        const int r = st * NR;
        if (L == 32) {
            const int4 m = *(const int4*)&mt[r];
            if (NARROW || (m.x <= 16 && m.z <= 16)) {
                paired |= 1u << st;
                const int np = hi ? m.z : m.x, off = hi ? m.w : m.y;
                wv[st][0] = k < np ? __ldg((const unsigned*)src + (((unsigned)off >> 2) + k)) : 0u;
            } else {
                wv[st][0] = lane < m.x ? __ldg((const unsigned*)(src + m.y) + lane) : 0u;
                wv[st][1] = lane < m.z ? __ldg((const unsigned*)(src + m.w) + lane) : 0u;
            }
        } else if (L == 16) {
            const int4 m0 = *(const int4*)&mt[2 * r];
            const int4 m1 = *(const int4*)&mt[2 * r + 2];
            if (NARROW || max(max(m0.x, m0.z), max(m1.x, m1.z)) <= 16) {
                paired |= 1u << st;
                const int npL = hi ? m1.x : m0.x, offL = hi ? m1.y : m0.y;
                const int npH = hi ? m1.z : m0.z, offH = hi ? m1.w : m0.w;
                const uint32_t wl = k < npL ? __ldg((const unsigned short*)(src + offL) + k) : 0u;
                const uint32_t wh = k < npH ? __ldg((const unsigned short*)(src + offH) + k) : 0u;
                wv[st][0] = wl | (wh << 16);
            } else {
                uint32_t wl = lane < m0.x ? __ldg((const unsigned short*)(src + m0.y) + lane) : 0u;
                uint32_t wh = lane < m0.z ? __ldg((const unsigned short*)(src + m0.w) + lane) : 0u;
                wv[st][0] = wl | (wh << 16);
                wl = lane < m1.x ? __ldg((const unsigned short*)(src + m1.y) + lane) : 0u;
                wh = lane < m1.z ? __ldg((const unsigned short*)(src + m1.w) + lane) : 0u;
                wv[st][1] = wl | (wh << 16);
            }
        } else if (L == 64) {
            const int2 m = mt[r / 2];
            if (NARROW || m.x <= 16) {
                paired |= 1u << st;
                wv[st][0] =
                    k < m.x ? __ldg((const unsigned*)(src + m.y + 8 * k + (hi ? 4 : 0))) : 0u;
            } else {
                uint2 v = make_uint2(0u, 0u);
                if (lane < m.x) v = __ldg((const uint2*)(src + m.y) + lane);
                wv[st][0] = v.x;
                wv[st][1] = v.y;
            }
        } else {
            const int2 m = mt[r / 4];
            if (NARROW || m.x <= 16) {
                paired |= 1u << st;
                const uint8_t* pp = src + m.y + 16 * k + (hi ? 4 : 0);
                wv[st][0] = k < m.x ? __ldg((const unsigned*)pp) : 0u;
                wv[st][1] = k < m.x ? __ldg((const unsigned*)(pp + 8)) : 0u;
            } else {
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (lane < m.x) v = __ldg((const uint4*)(src + m.y) + lane);
                wv[st][0] = v.x;
                wv[st][1] = v.y;
                wv[st][2 % NR] = v.z;
                wv[st][3 % NR] = v.w;
            }
        }
    }
    // ---- phase 2: transposes, prefix sums, reconstruction ----
#pragma unroll
    for (int st = 0; st < NS; ++st) {
        const int r = st * NR;
        if (BIASED) {
            // lane position within its block row
            const uint32_t kbits = 0x4b400000u - ((uint32_t)(L == 16 ? k : lane) + 1u) * PAIR_B;
            // two rows per integer scan: (q + (j + 1) B) of both rows in one word
            float carry = 0.0f;
#pragma unroll
            for (int h2 = 0; h2 < NR; h2 += 2) {
                uint32_t v = biased_pair(tpose(wv[st][h2 / 2], tc));
                v = (uint32_t)(L == 16 ? scan_incl<16>((int)v) : scan_incl<32>((int)v));
                float fa = pair_half_f(v & 0xffffu, kbits);
                float fb = pair_half_f(v >> 16, kbits);
                if (L >= 64) {
                    // rows of one block: each continues from the last value of the row before
                    if (((r + h2) % RPB) != 0) fa = __fadd_rn(fa, carry);
                    fb = __fadd_rn(fb, __shfl_sync(FULL, fa, 31));
                    if (((r + h2 + 1) % RPB) != RPB - 1) carry = __shfl_sync(FULL, fb, 31);
                }
                acc[r + h2] = __fmul_rn(fa, two_eb);
                acc[r + h2 + 1] = __fmul_rn(fb, two_eb);
            }
            continue;
        }
        uint32_t u[4];
        const bool pr = NARROW || ((paired >> st) & 1u);
        if (pr) {
            const uint32_t t0 = tpose(wv[st][0], tc);
            u[0] = t0 & 0xffffu;
            u[1] = t0 >> 16;
            if (NR == 4) {
                const uint32_t t1 = tpose(wv[st][1 % NR], tc);
                u[2] = t1 & 0xffffu;
                u[3] = t1 >> 16;
            }
        } else {
#pragma unroll
            for (int h = 0; h < NR; ++h) u[h] = tpose(wv[st][h], tc);
        }
        if (pr) {
            float carry = 0.0f;
#pragma unroll
            for (int h = 0; h < NR; ++h) {
                float dv = delta_f(u[h]);
                if (HEADS) dv = __fadd_rn(dv, __int2float_rn(hv[r + h]));  // the head's delta is 0
                float v = L == 16 ? scan_incl_f16(dv) : scan_incl_f(dv);
                if (L >= 64 && ((r + h) % RPB) != 0) v = __fadd_rn(v, carry);
                if (L >= 64 && ((r + h) % RPB) != RPB - 1) carry = __shfl_sync(FULL, v, 31);
                acc[r + h] = __fmul_rn(v, two_eb);
            }
        } else {
            int carry = 0;
#pragma unroll
            for (int h = 0; h < NR; ++h) {
                const int mag = (int)(u[h] >> 1);
                int dv = (u[h] & 1u) ? -mag : mag;
                if (HEADS) dv += hv[r + h];
                int v = L == 16 ? scan_incl<16>(dv) : scan_incl<32>(dv);
                if (L >= 64 && ((r + h) % RPB) != 0) v += carry;
                if (L >= 64 && ((r + h) % RPB) != RPB - 1) carry = __shfl_sync(FULL, v, 31);
                acc[r + h] = __fmul_rn(__int2float_rn(v), two_eb);
            }
        }
    }
}

// ---- encoding ------------------------------------------------------------------
// Predicated stores without a branch: the store happens when a < b.  `p` is
// a shared-memory address (the warp's staging buffer).
__device__ __forceinline__ void sts_u32_if(unsigned p, uint32_t v, int a, int b)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %2, %3;\n\t@q st.shared.u32 [%0], %1;\n\t}"
                 ::"r"(p), "r"(v), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void sts_u16_if(unsigned p, uint32_t v, int a, int b)
{
    asm volatile("{\n\t.reg .pred q;\n\t.reg .b16 h;\n\tcvt.u16.u32 h, %1;\n\t"
                 "setp.lt.s32 q, %2, %3;\n\t@q st.shared.u16 [%0], h;\n\t}"
                 ::"r"(p), "r"(v), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void sts_u64_if(unsigned p, uint32_t v0, uint32_t v1, int a, int b)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %3, %4;\n\t@q st.shared.v2.u32 [%0], {%1, %2};\n\t}"
                 ::"r"(p), "r"(v0), "r"(v1), "r"(a), "r"(b) : "memory");
}
__device__ __forceinline__ void sts_u128_if(unsigned p, uint32_t v0, uint32_t v1, uint32_t v2,
                                            uint32_t v3, int a, int b)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.lt.s32 q, %5, %6;\n\t"
                 "@q st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n\t}"
                 ::"r"(p), "r"(v0), "r"(v1), "r"(v2), "r"(v3), "r"(a), "r"(b) : "memory");
}
// Stores when m != 0 (a lane's bit of a mask); `p` is a shared-memory address.
__device__ __forceinline__ void sts_u32_m(unsigned p, uint32_t v, uint32_t m)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t@q st.shared.u32 [%0], %1;\n\t}"
                 ::"r"(p), "r"(v), "r"(m) : "memory");
}
__device__ __forceinline__ void sts_u8_m(unsigned p, uint32_t v, uint32_t m)
{
    asm volatile("{\n\t.reg .pred q;\n\t.reg .b16 h;\n\tcvt.u16.u32 h, %1;\n\t"
                 "setp.ne.u32 q, %2, 0;\n\t@q st.shared.u8 [%0], h;\n\t}"
                 ::"r"(p), "r"(v), "r"(m) : "memory");
}
__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
// Predicated shared-memory stores of width bytes (`p` in shared memory).
__device__ __forceinline__ void sts_if(uint8_t* p, uint4 v, bool c)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %5, 0;\n\t@q st.shared.v4.u32 [%0], {%1, %2, %3, %4};\n\t}"
                 ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"((int)c) : "memory");
}
__device__ __forceinline__ void sts_if(uint8_t* p, uint2 v, bool c)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %3, 0;\n\t@q st.shared.v2.u32 [%0], {%1, %2};\n\t}"
                 ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v.x), "r"(v.y), "r"((int)c) : "memory");
}
__device__ __forceinline__ void sts_if(uint8_t* p, uint32_t v, bool c)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %2, 0;\n\t@q st.shared.u32 [%0], %1;\n\t}"
                 ::"r"((unsigned)__cvta_generic_to_shared(p)), "r"(v), "r"((int)c) : "memory");
}
__device__ __forceinline__ void sts_if(uint8_t* p, unsigned short v, bool c)
{
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.s32 q, %2, 0;\n\t@q st.shared.u16 [%0], %1;\n\t}"
                 ::"r"((unsigned)__cvta_generic_to_shared(p)), "h"(v), "r"((int)c) : "memory");
}

// The previous lane's q within segments of W lanes; the first lane of a
// segment gets `fill` (uses the in-range predicate of shfl.up).
template <int W>
__device__ __forceinline__ int prev_lane(int q, int fill)
{
    int p;
    asm("{\n\t.reg .pred ok;\n\t"
        "shfl.sync.up.b32 %0|ok, %1, 1, %2, -1;\n\t"
        "@!ok mov.b32 %0, %3;\n\t}"
        : "=r"(p)
        : "r"(q), "r"((32 - W) << 8), "r"(fill));
    return p;
}

// Quantizes, delta-codes and bit-plane packs GR rows (the first `nrem`
// elements are valid, all of them when ALL; the rest are padding with zero
// deltas), appends the planes of their blocks at byte `lo` of the unit's
// payload (shared-memory address seg + lo: the warp's staging buffer), writes
// their width bytes to `wb` (shared memory, one store per group), ORs any
// quantizer error into `err`, and returns the new `lo`.  Two rows whose
// values fit 16 bits share one transpose.
template <int LOG2L, bool ALL, bool HEADS = false>
__device__ __forceinline__ int encode_group(const float acc[GR], int nrem, float eb, float two_eb,
                                            float inv, unsigned seg, int lo, uint8_t* wb, int& err,
                                            const TpC& tc, uint8_t* hout = nullptr)
{
    constexpr int L = 1 << LOG2L;
    constexpr int RPB = L >= 32 ? L / 32 : 1;
    const int lane = threadIdx.x & 31;
    const int k = lane & 15;
    const bool hi = lane >= 16;
    // quantize: the exactness of the fast rounding is voted once per group.
    // q holds q + QBIAS (the rounded float's bits): the deltas are the same
    int q[GR];
    {
        bool slow = false;
#pragma unroll
        for (int r = 0; r < GR; ++r) slow |= !quantize_fast_bits(acc[r], inv, q[r]);
        if (__any_sync(FULL, slow)) {
#pragma unroll
            for (int r = 0; r < GR; ++r) {
                int qq = 0;
                if (ALL || r * 32 + lane < nrem) err |= quantize(acc[r], eb, two_eb, inv, qq);
                q[r] = qq + QBIAS;
            }
        }
    }
    uint32_t u[GR];
    uint32_t wide = 0;
    int carry = 0;
#pragma unroll
    for (int r = 0; r < GR; ++r) {
        const int fill = (L >= 64 && (r % RPB) != 0) ? carry : QBIAS;  // a block starts from q = 0
        const int prev = prev_lane<L == 16 ? 16 : 32>(q[r], fill);
        if (L >= 64 && (r % RPB) != RPB - 1) carry = __shfl_sync(FULL, q[r], 31);
        int d = q[r] - prev;
        if (!ALL && r * 32 + lane >= nrem) d = 0;
        if (HEADS) {
            // heads apart: the block head goes to its 3-byte field (in the
            // output, at block position), its own delta is 0
            int b = -1;
            if (L == 16 && k == 0) b = 2 * r + (hi ? 1 : 0);
            else if (L == 32 && lane == 0) b = r;
            else if (L >= 64 && lane == 0 && (r % RPB) == 0) b = r / RPB;
            if (b >= 0) {
                if (ALL || r * 32 + lane < nrem) {
                    const int head = q[r] - QBIAS;
                    uint8_t* p = hout + 3 * b;
                    p[0] = (uint8_t)head;
                    p[1] = (uint8_t)(head >> 8);
                    p[2] = (uint8_t)(head >> 16);
                }
                d = 0;
            }
        }
        const uint32_t ad = (uint32_t)(d < 0 ? -d : d);
        u[r] = __funnelshift_l((uint32_t)d, ad, 1);  // |d| << 1 | sign
        wide |= u[r];
    }
    // one vote: does any value of the group need more than 16 planes?
    const bool any_wide = __any_sync(FULL, (wide >> 16) != 0u);
    const uint32_t hmask = hi ? 0xffffffffu : 0u;
    // the group's width bytes, gathered in registers and stored once (GR * 32 / L bytes)
    uint32_t wacc[4] = {0u, 0u, 0u, 0u};
    uint32_t pk[GR / 2];  // L = 32: plane counts of the row pairs
    // Every value of the group within 8 planes (the common case at moderate
    // bounds; L >= 32): four rows share a transpose, and lane 8m + j then
    // holds plane j of row m.  M is the ballot of nonzero planes.
    //   L = 32 (a block per row): smearing every byte of M downwards gives F,
    //   whose byte m has the low np_m bits set; a lane stores its plane if
    //   its bit of F is set, at 4 popc(F & lanes below) bytes past the quad's
    //   start, and the quad takes 4 popc(F) bytes.  The lane at a row's top
    //   plane (j = np - 1), or lane j = 0 of a row without planes, writes the
    //   row's width byte, j, itself.
    //   L = 64 (rows 0-1 and 2-3 are blocks): the block masks are bytes 0 | 1
    //   and 2 | 3 of M; plane j of a block is 8 bytes, its two rows' words.
    //   L = 128 (one block): the block mask is the OR of M's bytes; plane j
    //   is 16 bytes, the four rows' words.
    const bool quad = L >= 32 && !any_wide && !__any_sync(FULL, (wide >> 8) != 0u);
    if (quad) {
        const int j = lane & 7, m4 = lane >> 3;
        const uint32_t lt = lanemask_lt(), eq = 1u << lane;
        const unsigned wrow = (unsigned)__cvta_generic_to_shared(wb) + (unsigned)m4;
#pragma unroll
        for (int r = 0; r < GR; r += 4) {
            const uint32_t w = __byte_perm(__byte_perm(u[r], u[r + 1], 0x0040),
                                           __byte_perm(u[r + 2], u[r + 3], 0x0040), 0x5410);
            const uint32_t t = tpose(w, tc);
            const uint32_t M = __ballot_sync(FULL, t != 0u);
            if (L == 32) {
                uint32_t F = M | ((M >> 1) & 0x7f7f7f7fu);
                F |= (F >> 2) & 0x3f3f3f3fu;
                F |= (F >> 4) & 0x0f0f0f0fu;
                sts_u32_m(seg + lo + 4u * (unsigned)__popc(F & lt), t, F & eq);
                const uint32_t top = (F & ~((F >> 1) & 0x7f7f7f7fu)) | (~F & 0x01010101u);
                sts_u8_m(wrow + r, (uint32_t)j, top & eq);
                lo += 4 * __popc(F);
            } else if (L == 64) {
                const uint32_t X = M | (M >> 8);
                const int npA = 32 - __clz(X & 0xffu), npB = 32 - __clz((X >> 16) & 0xffu);
                sts_u32_if(seg + lo + 8 * j + 4 * (m4 & 1) + (hmask & (8 * npA)), t, j,
                           hi ? npB : npA);
                wacc[0] |= ((uint32_t)width_byte(npA) | ((uint32_t)width_byte(npB) << 8)) << (8 * (r / 2));
                lo += 8 * (npA + npB);
            } else {
                const uint32_t X = M | (M >> 16);
                const int np = 32 - __clz((X | (X >> 8)) & 0xffu);
                sts_u32_if(seg + lo + 16 * j + 4 * m4, t, j, np);
                wacc[0] |= (uint32_t)width_byte(np) << (8 * (r / 4));
                lo += 16 * np;
            }
        }
    } else if (!any_wide) {
        // every value of the group fits 16 bits (the common case): paired (or
        // quadrupled) rows share a transpose, with no per-pair votes
#pragma unroll
        for (int r = 0; r < GR; r += (L == 128 ? 4 : 2)) {
            if (L == 32) {
                const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                const unsigned m = __ballot_sync(FULL, t != 0u);
                const int na = 32 - __clz(m & 0xffffu), nb = 32 - __clz(m >> 16);
                sts_u32_if(seg + 4 * k + lo + (hmask & (4 * na)), t, k, hi ? nb : na);
                // the pair's plane counts as bytes [na, nb, 0, 0]
                pk[r / 2] = __byte_perm((uint32_t)na, (uint32_t)nb, 0x1140);
                lo += 4 * (na + nb);
            } else if (L == 16) {
                const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                const unsigned m0 = __ballot_sync(FULL, (t & 0xffffu) != 0u);
                const unsigned m1 = __ballot_sync(FULL, (t >> 16) != 0u);
                const int npA = 32 - __clz(m0 & 0xffffu), npB = 32 - __clz(m1 & 0xffffu);
                const int npC = 32 - __clz(m0 >> 16), npD = 32 - __clz(m1 >> 16);
                const int oA = lo, oB = oA + 2 * npA, oC = oB + 2 * npB, oD = oC + 2 * npC;
                sts_u16_if(seg + (hi ? oC : oA) + 2 * k, t & 0xffffu, k, hi ? npC : npA);
                sts_u16_if(seg + (hi ? oD : oB) + 2 * k, t >> 16, k, hi ? npD : npB);
                wacc[r / 2] = (uint32_t)width_byte(npA) | ((uint32_t)width_byte(npB) << 8) |
                              ((uint32_t)width_byte(npC) << 16) | ((uint32_t)width_byte(npD) << 24);
                lo += 2 * (npA + npB + npC + npD);
            } else if (L == 64) {
                const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                const unsigned m = __ballot_sync(FULL, t != 0u);
                const int np = 32 - __clz((m & 0xffffu) | (m >> 16));
                sts_u32_if(seg + lo + 8 * k + (hmask & 4), t, k, np);
                wacc[0] |= (uint32_t)width_byte(np) << (8 * (r / 2));
                lo += 8 * np;
            } else {
                const uint32_t t0 = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                const uint32_t t1 = tpose(__byte_perm(u[r + 2], u[r + 3], 0x5410), tc);
                const unsigned m = __ballot_sync(FULL, (t0 | t1) != 0u);
                const int np = 32 - __clz((m & 0xffffu) | (m >> 16));
                const unsigned pp = seg + lo + 16 * k + (hmask & 4);
                sts_u32_if(pp, t0, k, np);
                sts_u32_if(pp + 8, t1, k, np);
                wacc[0] |= (uint32_t)width_byte(np) << (8 * (r / 4));
                lo += 16 * np;
            }
        }
        if (L == 32) {
            // the width bytes of two pairs at a time
#pragma unroll
            for (int w = 0; w < GR / 4; ++w)
                wacc[w] = width_bytes4(__byte_perm(pk[2 * w], pk[2 * w + 1], 0x5410));
        }
    } else {
    #pragma unroll
        for (int r = 0; r < GR; r += (L == 128 ? 4 : 2)) {
            if (L == 32) {
                int fa, fb;  // highest nonzero plane of blocks r, r + 1 (-1: none)
                if (!any_wide || !__any_sync(FULL, ((u[r] | u[r + 1]) >> 16) != 0u)) {
                    const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                    const unsigned m = __ballot_sync(FULL, t != 0u);
                    fa = 31 - __clz(m & 0xffffu);
                    fb = 31 - __clz(m >> 16);
                    const int npm = hi ? fb + 1 : fa + 1;
                    sts_u32_if(seg + lo + (hmask & (4 * fa + 4)) + 4 * k, t, k, npm);
                } else {
                    const uint32_t ta = tpose(u[r], tc), tb = tpose(u[r + 1], tc);
                    fa = 31 - __clz(__ballot_sync(FULL, ta != 0u));
                    fb = 31 - __clz(__ballot_sync(FULL, tb != 0u));
                    sts_u32_if(seg + lo + 4 * lane, ta, lane, fa + 1);
                    sts_u32_if(seg + lo + 4 * fa + 4 + 4 * lane, tb, lane, fb + 1);
                }
                wacc[r / 4] |= ((uint32_t)max(fa, 0) | ((uint32_t)max(fb, 0) << 8)) << (8 * (r % 4));
                lo += 4 * (fa + fb + 2);
            } else if (L == 16) {
                int npA, npB, npC, npD;
                if (!any_wide || !__any_sync(FULL, ((u[r] | u[r + 1]) >> 16) != 0u)) {
                    const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                    const unsigned m0 = __ballot_sync(FULL, (t & 0xffffu) != 0u);
                    const unsigned m1 = __ballot_sync(FULL, (t >> 16) != 0u);
                    npA = 32 - __clz(m0 & 0xffffu);
                    npB = 32 - __clz(m1 & 0xffffu);
                    npC = 32 - __clz(m0 >> 16);
                    npD = 32 - __clz(m1 >> 16);
                    const int oA = lo, oB = oA + 2 * npA, oC = oB + 2 * npB, oD = oC + 2 * npC;
                    const int npL = hi ? npC : npA, npH = hi ? npD : npB;
                    const int offL = hi ? oC : oA, offH = hi ? oD : oB;
                    sts_u16_if(seg + offL + 2 * k, t & 0xffffu, k, npL);
                    sts_u16_if(seg + offH + 2 * k, t >> 16, k, npH);
                } else {
                    const uint32_t ta = tpose(u[r], tc), tb = tpose(u[r + 1], tc);
                    npA = 32 - __clz(__ballot_sync(FULL, (ta & 0xffffu) != 0u));
                    npB = 32 - __clz(__ballot_sync(FULL, (ta >> 16) != 0u));
                    npC = 32 - __clz(__ballot_sync(FULL, (tb & 0xffffu) != 0u));
                    npD = 32 - __clz(__ballot_sync(FULL, (tb >> 16) != 0u));
                    const int oA = lo, oB = oA + 2 * npA, oC = oB + 2 * npB, oD = oC + 2 * npC;
                    sts_u16_if(seg + oA + 2 * lane, ta & 0xffffu, lane, npA);
                    sts_u16_if(seg + oB + 2 * lane, ta >> 16, lane, npB);
                    sts_u16_if(seg + oC + 2 * lane, tb & 0xffffu, lane, npC);
                    sts_u16_if(seg + oD + 2 * lane, tb >> 16, lane, npD);
                }
                wacc[r / 2] = (uint32_t)width_byte(npA) | ((uint32_t)width_byte(npB) << 8) |
                              ((uint32_t)width_byte(npC) << 16) | ((uint32_t)width_byte(npD) << 24);
                lo += 2 * (npA + npB + npC + npD);
            } else if (L == 64) {
                int np;
                if (!any_wide || !__any_sync(FULL, ((u[r] | u[r + 1]) >> 16) != 0u)) {
                    const uint32_t t = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                    const unsigned m = __ballot_sync(FULL, t != 0u);
                    np = 32 - __clz((m & 0xffffu) | (m >> 16));
                    sts_u32_if(seg + lo + 8 * k + (hmask & 4), t, k, np);
                } else {
                    const uint32_t ta = tpose(u[r], tc), tb = tpose(u[r + 1], tc);
                    np = 32 - __clz(__ballot_sync(FULL, (ta | tb) != 0u));
                    sts_u64_if(seg + lo + 8 * lane, ta, tb, lane, np);
                }
                wacc[0] |= (uint32_t)width_byte(np) << (8 * (r / 2));
                lo += 8 * np;
            } else {
                int np;
                if (!any_wide ||
                    !__any_sync(FULL, ((u[r] | u[r + 1] | u[r + 2] | u[r + 3]) >> 16) != 0u)) {
                    const uint32_t t0 = tpose(__byte_perm(u[r], u[r + 1], 0x5410), tc);
                    const uint32_t t1 = tpose(__byte_perm(u[r + 2], u[r + 3], 0x5410), tc);
                    const unsigned m = __ballot_sync(FULL, (t0 | t1) != 0u);
                    np = 32 - __clz((m & 0xffffu) | (m >> 16));
                    const unsigned pp = seg + lo + 16 * k + (hmask & 4);
                    sts_u32_if(pp, t0, k, np);
                    sts_u32_if(pp + 8, t1, k, np);
                } else {
                    const uint32_t t0 = tpose(u[r], tc), t1 = tpose(u[r + 1], tc);
                    const uint32_t t2 = tpose(u[r + 2], tc), t3 = tpose(u[r + 3], tc);
                    np = 32 - __clz(__ballot_sync(FULL, (t0 | t1 | t2 | t3) != 0u));
                    sts_u128_if(seg + lo + 16 * lane, t0, t1, t2, t3, lane, np);
                }
                wacc[0] |= (uint32_t)width_byte(np) << (8 * (r / 4));
                lo += 16 * np;
            }
        }
    }
    // one store of the group's width bytes (wb is 16-byte aligned per group
    // at L = 16, 8 at L = 32, 4 at L = 64, 2 at L = 128)
    if (L == 16) sts_if(wb, make_uint4(wacc[0], wacc[1], wacc[2], wacc[3]), lane == 0);
    else if (L == 32) sts_if(wb, make_uint2(wacc[0], wacc[1]), lane == 0 && !quad);
    else if (L == 64) sts_if(wb, wacc[0], lane == 0);
    else sts_if(wb, (unsigned short)wacc[0], lane == 0);
    return lo;
}

// ---- encoder tiles -------------------------------------------------------------
// An encoder CTA runs two kinds of warps.  Its NWARPS encoder warps take tiles
// in ticket order and encode each of the tile's warp units into the CTA's ring
// (global memory, enc_slots(U) tiles deep) and its width bytes into shared
// memory.  Its resolver warp takes every encoded tile, sums the units' sizes,
// runs the tile's look-back (and, for packed streams, the stream-start wait)
// and hands the tile's place in the output back.  enc_slots(U) - 1 tiles later
// the encoder warps copy the tile from the ring to the stream.  So the encoder
// warps never stop for a look-back: the wait for the tiles before this one
// overlaps the encoding of the tiles after it.

// Copies `len` bytes (a multiple of UNIT) from the ring (16-byte aligned) to
// `dst` (UNIT-aligned) with one warp; four loads per lane are in flight.  The
// staged bytes are dead afterwards: their L2 lines (the segment owns whole
// 128-byte lines) are dropped without a write-back, so the ring costs no DRAM
// traffic as long as a tile's lines stay in L2 until it is stored.
template <int UNIT>
__device__ __forceinline__ void ring_copy(uint8_t* dst, const uint8_t* src, int len)
{
    const int lane = threadIdx.x & 31;
    using T = typename std::conditional<
        UNIT == 16, uint4,
        typename std::conditional<UNIT == 8, uint2,
                                  typename std::conditional<UNIT == 4, unsigned,
                                                            unsigned short>::type>::type>::type;
    const int cnt = len / UNIT;
    for (int b = 0; b < cnt; b += 32 * 4) {
        T v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = b + k * 32 + lane;
            if (i < cnt) v[k] = __ldcs((const T*)src + i);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int i = b + k * 32 + lane;
            if (i < cnt) __stcs((T*)dst + i, v[k]);
        }
    }
    __syncwarp();
    for (int l = lane; l < (len + 127) >> 7; l += 32)
        asm volatile("discard.global.L2 [%0], 128;" ::"l"(__cvta_generic_to_global(src + 128 * l))
                     : "memory");
}

// Packed mode (one chain through many streams): the first tile of a stream
// publishes where the stream starts (its exclusive value ex), the stream's
// other tiles wait for that.  Outside packed mode a stream starts at 0.
// Returns false (status set) when the wait runs out.  Run by one warp.
__device__ __forceinline__ bool packed_start_warp(const Launch& P, bool first, unsigned item_idx,
                                                  unsigned long long ex, unsigned g, unsigned E,
                                                  unsigned long long& start)
{
    const int lane = threadIdx.x & 31;
    start = 0ull;
    if (!P.packed) return true;
    if (first) {
        start = ex;
        if (lane == 0) {
            P.seg_off[item_idx] = ex;
            rec_store(P.seg_rec + item_idx, E, ST_PREFIX, false, ex);
        }
        return true;
    }
    int ok = 1;
    unsigned long long v = 0ull;
    if (lane == 0) {
        ok = wait_rec(P.seg_rec + item_idx, E, P.wc.limit_ns, v);
        if (!ok) fail(P.ctl, ZC_ERR_TIMEOUT, g);
    }
    ok = __shfl_sync(FULL, ok, 0);
    start = __shfl_sync(FULL, v, 0);
    return ok != 0;
}

// One tile in flight.  The encoder warps fill it (thread 0 the scalars, lane
// 0 of every warp its unit's size), the resolver warp adds ex, start and ok.
struct TileSlot {
    unsigned g, item, tile;       // ticket, item, tile within the item
    int valid;                    // g is a tile of this launch
    int pub;                      // the tile takes part in the chain
    int first, last;              // first / last tile of its stream
    unsigned long long head;      // bytes of the tile besides its units' payload
    int segsz[NWARPS];            // payload bytes of every warp unit
    unsigned long long ex, start; // place in the chain, start of its stream
    int ok;                       // ex and start are usable: store the tile
    int nfin;                     // encoder warps done with the tile
};

struct EncShared {
    unsigned E;    // launch generation
    int abort;     // 1: unusable workspace (the CTA does nothing), 2: no usable bound
    int hdr_bad;   // fused ring step: the tile's input stream failed its check
    float eb_in;   // its bound
};

// Encoder warp `warp`'s unit of one tile: quantize, delta-code and bit-plane
// pack its U rows, through its shared-memory `stage` (SR rows at a time),
// into its ring segment `seg`, and its width bytes into `wb`; returns the
// segment's size.  HAS_CIN: decode `it.cin` first (same block size, unit
// offsets from k_wscan) and add the local chunk; the FP32 sum then goes to
// `it.raw_out` when that is set.  Null pointers switch a step off.  HEADS
// (block heads stored apart, single unpacked streams) writes the heads
// straight to their fixed place in the output.  Thread 0 fills the slot's
// scalars.
template <int LOG2L, int U, bool HAS_CIN, typename TX, bool HEADS = false, int SR = 32>
__device__ __forceinline__ int enc_tile(const Launch& P, const Item& it, unsigned item_idx,
                                        unsigned tile_in_item, uint8_t* seg, uint8_t* wb,
                                        uint8_t* stage, TileSlot& S, EncShared& es)
{
    static_assert(!HEADS || !HAS_CIN, "heads apart: compression only");
    constexpr int L = 1 << LOG2L;
    constexpr int BU = U * 32 / L;  // blocks per warp unit
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    Ctl* ctl = P.ctl;
    const unsigned long long n = it.n;
    const unsigned long long ue0 = (unsigned long long)tile_in_item * (NWARPS * U * 32) +
                                   (unsigned long long)warp * U * 32;
    const unsigned long long nb = (n + L - 1) >> LOG2L;
    const unsigned long long wbytes = ceil16(nb);
    const bool first = tile_in_item == 0;
    const bool do_cin = HAS_CIN && it.cin != nullptr;
    const bool do_enc = it.out != nullptr;
    if (tid == 0) {
        S.first = first;
        S.last = tile_in_item + 1 == it.ntiles;
        S.head = first ? 32ull + wbytes + (HEADS ? ceil16(3ull * nb) : 0ull) : 0ull;
        S.pub = do_enc;
    }
    float two_eb_in = 0.0f;
    if (do_cin) {
        if (tid == 0) {
            float eb_in;
            const int lg = check_header(it, ctl, item_idx, LOG2L, eb_in, first);
            es.hdr_bad = lg != LOG2L;
            es.eb_in = eb_in;
            if (es.hdr_bad) S.pub = 0;
        }
        bar_sync_n(BAR_ENCW, NTHREADS);
        if (es.hdr_bad) return 0;
        two_eb_in = __fadd_rn(es.eb_in, es.eb_in);
    }
    float eb = it.eb, two_eb = it.two_eb, inv = it.inv;
    if (P.eb_from_ctl) {
        eb = ctl->eb;
        two_eb = ctl->two_eb;
        inv = ctl->inv;
    }

    const TpC tc = tp_consts(lane);
    int err = 0;
    int lo = 0;
    // The unit's payload is staged in shared memory (`stage`, this warp's
    // stage_bytes(SR)), SR rows at a time, and flushed to its ring segment
    // `seg` with 16-byte copies.  The
    // stage holds ring bytes [sbase, lo) (sbase 16-byte aligned); a flush
    // copies them and keeps the partial last 16 bytes at the stage start.
    static_assert(SR % GR == 0 && U % SR == 0, "stage geometry");
    __shared__ __align__(16) int2 meta_all[HAS_CIN ? NWARPS : 1][HAS_CIN ? BU : 1];
    const unsigned stage_s = (unsigned)__cvta_generic_to_shared(stage);
    int sbase = 0;
    auto flush = [&](int lo_end) {
        int n16 = (lo_end - sbase + 15) >> 4;
        if (!dcheck(ctl, sbase + 16 * n16 <= seg_bytes(U), ue0)) n16 = 0;
        for (int i = lane; i < n16; i += 32)
            ((uint4*)(seg + sbase))[i] = ((const uint4*)stage)[i];
        const int nbase = lo_end & ~15;
        __syncwarp();
        if (lane == 0 && nbase != sbase && (lo_end & 15) != 0)
            ((uint4*)stage)[0] = ((const uint4*)stage)[(nbase - sbase) >> 4];
        __syncwarp();
        sbase = nbase;
    };
    if (do_enc && it.x != nullptr && ue0 + U * 32 <= n) {
        // a whole unit (every unit but the last of a stream): no tails, and
        // few live values, so the group loop stays in registers
        const TX* const xb = (const TX*)it.x + ue0 + lane;
        if (lane == 0) {
            // the whole unit's input into L2 at once (16-byte aligned inner range)
            const uintptr_t a0 = (uintptr_t)((const TX*)it.x + ue0), a1 = a0 + U * 32 * sizeof(TX);
            const uintptr_t s0 = (a0 + 15) & ~(uintptr_t)15, s1 = a1 & ~(uintptr_t)15;
            if (s1 > s0)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(s0),
                             "r"((unsigned)(s1 - s0))
                             : "memory");
        }
        const uint8_t* src = nullptr;
        int2* meta = nullptr;
        bool narrow = false, narrow11 = false;
        if constexpr (HAS_CIN) {
            meta = meta_all[warp];
            if (do_cin)
                src = it.cin + unit_meta<LOG2L, U>(P, it, S.g * NWARPS + warp, ue0, meta, narrow,
                                                   narrow11);
        }
#pragma unroll 1
        for (int gi = 0; gi < U / GR; ++gi) {
            float acc[GR];
#pragma unroll
            for (int r = 0; r < GR; ++r) acc[r] = load_x<TX>(xb, gi * GR * 32 + r * 32);
            if constexpr (HAS_CIN) {
                if (do_cin) {
                    float dv[GR];
                    if (narrow11) decode_group<LOG2L, true, false, true>(src, meta, gi, two_eb_in, dv, tc);
                    else if (narrow) decode_group<LOG2L, true>(src, meta, gi, two_eb_in, dv, tc);
                    else decode_group<LOG2L, false>(src, meta, gi, two_eb_in, dv, tc);
#pragma unroll
                    for (int r = 0; r < GR; ++r) acc[r] = __fadd_rn(dv[r], acc[r]);
                }
                if (it.raw_out != nullptr) {
                    float* op = (float*)it.raw_out + ue0 + gi * GR * 32 + lane;
#pragma unroll
                    for (int r = 0; r < GR; ++r) op[r * 32] = acc[r];
                }
            }
            const int b0 = L >= 32 ? gi * GR / (L / 32) : gi * GR * 2;
            uint8_t* hout = nullptr;
            if (HEADS) hout = it.out + 32 + wbytes + 3ull * ((ue0 >> LOG2L) + b0);
            if (HEADS && DEBUG_BUILD)
                dcheck(ctl, 32 + wbytes + 3ull * ((ue0 >> LOG2L) + b0 + GR * 32 / L) <= it.out_cap,
                       ue0);
            if (dcheck(ctl, lo - sbase + seg_bytes(GR) <= stage_bytes(SR), ue0))
                lo = encode_group<LOG2L, true, HEADS>(acc, GR * 32, eb, two_eb, inv, stage_s - sbase,
                                                      lo, wb + b0, err, tc, hout);
            if ((gi + 1) % (SR / GR) == 0) flush(lo);
        }
    } else if (ue0 < n) {
        const uint8_t* src = nullptr;
        int2* meta = nullptr;
        bool narrow = false, narrow11 = false;
        if constexpr (HAS_CIN) {
            meta = meta_all[warp];
            if (do_cin)
                src = it.cin + unit_meta<LOG2L, U>(P, it, S.g * NWARPS + warp, ue0, meta, narrow,
                                                   narrow11);
        }
        // the next group's input is loaded while the current one is encoded
        float xn[GR];
        const TX* const xbase = it.x != nullptr ? (const TX*)it.x + ue0 + lane : nullptr;
        {
            const int nrem0 = (int)min(n - ue0, (unsigned long long)(GR * 32));
#pragma unroll
            for (int r = 0; r < GR; ++r)
                xn[r] = (xbase != nullptr && r * 32 + lane < nrem0) ? load_x<TX>(xbase, r * 32) : 0.0f;
        }
#pragma unroll 1
        for (int gi = 0; gi < U / GR; ++gi) {
            const unsigned long long e0 = ue0 + (unsigned long long)gi * GR * 32;
            if (e0 >= n) break;
            const int nrem = (int)min(n - e0, (unsigned long long)(GR * 32));
            float acc[GR];
#pragma unroll
            for (int r = 0; r < GR; ++r) acc[r] = xn[r];
            if (gi + 1 < U / GR && e0 + GR * 32 < n) {
                const TX* xp = xbase + (gi + 1) * GR * 32;
                if (xbase != nullptr && e0 + 2 * GR * 32 <= n) {
#pragma unroll
                    for (int r = 0; r < GR; ++r) xn[r] = load_x<TX>(xp, r * 32);
                } else {
                    const int nrem1 = (int)min(n - e0 - GR * 32, (unsigned long long)(GR * 32));
#pragma unroll
                    for (int r = 0; r < GR; ++r)
                        xn[r] = (xbase != nullptr && r * 32 + lane < nrem1) ? load_x<TX>(xp, r * 32)
                                                                             : 0.0f;
                }
            }
            if constexpr (HAS_CIN) {
                if (do_cin) {
                    float dv[GR];
                    if (narrow11) decode_group<LOG2L, true, false, true>(src, meta, gi, two_eb_in, dv, tc);
                    else if (narrow) decode_group<LOG2L, true>(src, meta, gi, two_eb_in, dv, tc);
                    else decode_group<LOG2L, false>(src, meta, gi, two_eb_in, dv, tc);
#pragma unroll
                    for (int r = 0; r < GR; ++r) acc[r] = __fadd_rn(dv[r], acc[r]);
                }
            }
            if (HAS_CIN && it.raw_out != nullptr) {
                float* op = (float*)it.raw_out + e0 + lane;
                const bool check = do_cin && !do_enc;
#pragma unroll
                for (int r = 0; r < GR; ++r) {
                    if (r * 32 + lane < nrem) {
                        op[r * 32] = acc[r];
                        if (check && !isfinite(acc[r])) err |= ZC_ERR_NONFINITE;
                    }
                }
            }
            if (do_enc) {
                const int b0 = L >= 32 ? gi * GR / (L / 32) : gi * GR * 2;
                uint8_t* hout = nullptr;
                if (HEADS) hout = it.out + 32 + wbytes + 3ull * ((ue0 >> LOG2L) + b0);
                if (!dcheck(ctl, lo - sbase + seg_bytes(GR) <= stage_bytes(SR), e0))
                    ;
                else if (nrem == GR * 32)
                    lo = encode_group<LOG2L, true, HEADS>(acc, nrem, eb, two_eb, inv,
                                                          stage_s - sbase, lo, wb + b0, err, tc,
                                                          hout);
                else
                    lo = encode_group<LOG2L, false, HEADS>(acc, nrem, eb, two_eb, inv,
                                                           stage_s - sbase, lo, wb + b0, err, tc,
                                                           hout);
                if ((gi + 1) % (SR / GR) == 0) flush(lo);
            }
        }
        if (do_enc) flush(lo);
    }
    {
        const unsigned bad = __ballot_sync(FULL, err != 0);
        if (bad && lane == __ffs(bad) - 1) fail(ctl, (unsigned)err, ue0);
    }
    return do_enc ? lo : 0;
}

// Stores of one encoded tile once its place is known: every encoder warp
// copies its unit's segment from the ring and its width bytes; the last tile
// of a stream zero-pads the width array (and the heads) and the payload and
// writes the header.
template <int LOG2L, int U, bool HAS_CIN, bool HEADS = false>
__device__ __forceinline__ void fin_tile(const Launch& P, const Item& it, unsigned item_idx,
                                         unsigned tile_in_item, unsigned g, const TileSlot& S,
                                         const uint8_t* seg, const uint8_t* wb)
{
    constexpr int L = 1 << LOG2L;
    constexpr int PB = L / 8;
    constexpr int BU = U * 32 / L;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const unsigned long long n = it.n;
    const unsigned long long ue0 = (unsigned long long)tile_in_item * (NWARPS * U * 32) +
                                   (unsigned long long)warp * U * 32;
    const unsigned long long nb = (n + L - 1) >> LOG2L;
    const unsigned long long wbytes = ceil16(nb);
    const unsigned long long hbytes = HEADS ? ceil16(3ull * nb) : 0ull;
    int segoff = 0, payload_i = 0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) {
        if (w < warp) segoff += S.segsz[w];
        payload_i += S.segsz[w];
    }
    const unsigned long long payload = (unsigned long long)payload_i;
    const unsigned long long ex = S.ex, start = S.start;
    const unsigned long long base = ex + S.head;
    const unsigned long long cap = it.out_cap;
    uint8_t* const out = it.out;
    const unsigned long long end = base + payload;  // unpadded end of this tile's payload
    if (base + payload <= cap) {
        if (dcheck(P.ctl, S.segsz[warp] <= seg_bytes(U), g))
            ring_copy<PB>(out + base + segoff, seg, S.segsz[warp]);
    } else if (tid == 0) {
        fail(P.ctl, ZC_ERR_CAPACITY, g);
    }
    {
        const unsigned long long b0 = ue0 >> LOG2L;
        const unsigned long long pos0 = start + 32 + b0;  // 16-byte aligned when BU is
        if (BU % 16 == 0 && b0 + BU <= nb && pos0 + BU <= cap) {
            if (lane < BU / 16) ((uint4*)(out + pos0))[lane] = ((const uint4*)wb)[lane];
        } else {
            for (int i = lane; i < BU; i += 32) {
                const unsigned long long b = b0 + i;
                const unsigned long long pos = pos0 + i;
                if (b < nb && pos < cap) out[pos] = wb[i];
            }
        }
    }
    if (S.last) {
        const unsigned long long total = ceil16(end);
        const unsigned long long pl = end - start - 32 - wbytes - hbytes;
        for (unsigned long long p = start + 32 + nb + tid; p < start + 32 + wbytes; p += NTHREADS)
            if (p < cap) out[p] = 0;
        if (HEADS)
            for (unsigned long long p = start + 32 + wbytes + 3 * nb + tid;
                 p < start + 32 + wbytes + hbytes; p += NTHREADS)
                if (p < cap) out[p] = 0;
        for (unsigned long long p = end + tid; p < total; p += NTHREADS)
            if (p < cap) out[p] = 0;
        if (tid < 8 && start + 32 <= cap) {
            uint32_t v = 0;
            const int xdt = HAS_CIN ? ZC_F32 : it.x_dtype;
            switch (tid) {
            case 0: v = 0x3176435au; break;  // "ZCv1"
            case 1: v = (uint32_t)xdt | ((uint32_t)LOG2L << 8) | (HEADS ? (2u << 16) : 0u); break;
            case 2: v = (uint32_t)n; break;
            case 3: v = (uint32_t)(n >> 32); break;
            case 4: v = __float_as_uint(P.eb_from_ctl ? P.ctl->eb : it.eb); break;
            case 5: v = (uint32_t)nb; break;
            case 6: v = (uint32_t)pl; break;
            default: v = (uint32_t)(pl >> 32); break;
            }
            ((uint32_t*)(out + start))[tid] = v;
        }
        if (tid == 0) {
            if (it.out_bytes) *it.out_bytes = total - start;
            if (P.packed && !P.grouped) P.seg_off[item_idx + 1] = total;
            else if (P.packed && g + 1 == P.total_tiles) P.seg_off[P.n_items] = total;
        }
    }
}

// One tile of a raw (verbatim) stream: the item's elements of this tile go
// unchanged after the 32-byte header (flag bit 0 set, no width bytes).  Same
// tile geometry, look-back and stream-start protocol as an encoded tile, so
// raw and encoded streams mix in one packed launch.  Nothing is staged: the
// tile's size is known from its element count.
template <int U>
__device__ __forceinline__ int enc_raw(const Item& it, unsigned tile_in_item, TileSlot& S)
{
    if (threadIdx.x == 0) {
        constexpr unsigned long long TE = (unsigned long long)NWARPS * U * 32;
        const unsigned long long es = it.x_dtype == ZC_F32 ? 4ull : 2ull;
        const unsigned long long te0 = (unsigned long long)tile_in_item * TE;
        const unsigned long long cnt = te0 < it.n ? min(it.n - te0, TE) : 0ull;
        S.first = tile_in_item == 0;
        S.last = tile_in_item + 1 == it.ntiles;
        S.head = cnt * es + (tile_in_item == 0 ? 32ull : 0ull);
        S.pub = it.out != nullptr;
    }
    return 0;
}

template <int U>
__device__ __forceinline__ void fin_raw(const Launch& P, const Item& it, unsigned item_idx,
                                        unsigned tile_in_item, unsigned g, const TileSlot& S)
{
    constexpr unsigned long long TE = (unsigned long long)NWARPS * U * 32;
    const int tid = threadIdx.x;
    const unsigned long long n = it.n;
    const unsigned long long es = it.x_dtype == ZC_F32 ? 4ull : 2ull;
    const unsigned long long te0 = (unsigned long long)tile_in_item * TE;
    const unsigned long long cnt = te0 < n ? min(n - te0, TE) : 0ull;
    const unsigned long long bytes = cnt * es;
    const unsigned long long ex = S.ex, start = S.start;
    const unsigned long long base = ex + (S.first ? 32ull : 0ull);  // 16-byte aligned
    const unsigned long long cap = it.out_cap;
    uint8_t* const out = it.out;
    if (base + bytes <= cap) {
        const uint8_t* src = (const uint8_t*)it.x + te0 * es;
        if (((uintptr_t)src & 15u) == 0) {
            const unsigned long long nv = bytes / 16;
            for (unsigned long long i = tid; i < nv; i += NTHREADS)
                ((uint4*)(out + base))[i] = __ldg((const uint4*)src + i);
            for (unsigned long long i = nv * 16 + tid * 2; i < bytes; i += 2 * NTHREADS)
                *(uint16_t*)(out + base + i) = __ldg((const unsigned short*)(src + i));
        } else {
            // the input is only element-aligned: 2-byte copies
            for (unsigned long long i = (unsigned long long)tid * 2; i < bytes; i += 2 * NTHREADS)
                *(uint16_t*)(out + base + i) = __ldg((const unsigned short*)(src + i));
        }
    } else if (tid == 0) {
        fail(P.ctl, ZC_ERR_CAPACITY, g);
    }
    if (S.last) {
        const unsigned long long end = ex + S.head;
        const unsigned long long total = ceil16(end);
        const unsigned long long pl = n * es;
        for (unsigned long long p = end + tid; p < total; p += NTHREADS)
            if (p < cap) out[p] = 0;
        if (tid < 8 && start + 32 <= cap) {
            uint32_t v = 0;
            switch (tid) {
            case 0: v = 0x3176435au; break;  // "ZCv1"
            case 1: v = (uint32_t)it.x_dtype | (5u << 8) | (1u << 16); break;  // raw flag
            case 2: v = (uint32_t)n; break;
            case 3: v = (uint32_t)(n >> 32); break;
            case 4: v = 0u; break;  // eb: none
            case 5: v = 0u; break;  // no blocks
            case 6: v = (uint32_t)pl; break;
            default: v = (uint32_t)(pl >> 32); break;
            }
            ((uint32_t*)(out + start))[tid] = v;
        }
        if (tid == 0) {
            if (it.out_bytes) *it.out_bytes = total - start;
            if (P.packed && !P.grouped) P.seg_off[item_idx + 1] = total;
            else if (P.packed && g + 1 == P.total_tiles) P.seg_off[P.n_items] = total;
        }
    }
}

// ---- item sources ------------------------------------------------------------

struct ItemsSrc {
    const Launch& P;
    __device__ unsigned find(unsigned g) const
    {
        if (P.items == nullptr) return 0u;
        if (P.tile_map != nullptr) return P.tile_map[g];
        unsigned lo = 0, hi = P.n_items;
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (P.items[mid].tile_begin <= g) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    __device__ Item get(unsigned i) const { return P.items != nullptr ? P.items[i] : P.one; }
};

// Scatter pack: segments of one input, described by value in the kernel
// parameters (so a call needs no descriptor upload).
constexpr int SCATTER_MAX = 1024;
struct ScatterParams {
    unsigned tile_begin[SCATTER_MAX + 1];
    unsigned long long displ[SCATTER_MAX];
    unsigned long long count[SCATTER_MAX];
};
struct ScatterSrc {
    const Launch& P;
    const ScatterParams& S;
    __device__ unsigned find(unsigned g) const
    {
        unsigned lo = 0, hi = P.n_items;
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (S.tile_begin[mid] <= g) lo = mid;
            else hi = mid;
        }
        return lo;
    }
    __device__ Item get(unsigned i) const
    {
        Item it = P.one;  // shared fields: out, out_cap, eb, dtype
        const unsigned long long es = it.x_dtype == ZC_F32 ? 4ull : 2ull;
        it.x = (const uint8_t*)P.one.x + S.displ[i] * es;
        it.n = S.count[i];
        it.tile_begin = S.tile_begin[i];
        it.ntiles = S.tile_begin[i + 1] - S.tile_begin[i];
        it.out_bytes = nullptr;
        return it;
    }
};

// Published by the last encoder warp to finish a tile: the tile's aggregate
// (its byte count), so that the look-backs of the tiles after it need not wait
// until this CTA's resolver warp reaches it (the resolver handles its tiles in
// order, and a tile it is still waiting on would hold back this one's
// aggregate).  The resolver then publishes the tile's inclusive prefix.  A
// chain's first tile publishes its prefix at once (resolver), and a withheld
// tile (test hook) publishes nothing.
__device__ __forceinline__ void publish_aggregate(const Launch& P, const TileSlot& S, unsigned E)
{
    if (!S.valid || !S.pub) return;
    const unsigned g0 = P.packed ? 0u : S.g - S.tile;
    if (S.g == g0 || (long long)S.g == P.wc.withhold || S.g >= P.ws_cap) return;
    unsigned long long agg = S.head;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) agg += (unsigned long long)S.segsz[w];
    rec_store(P.chB.rec + S.g, E, ST_AGG, S.last != 0, agg);
}

// Resolver warp: the tile's place in the chain (look-back over the tiles
// before it) and, in packed mode, its stream's start.
__device__ __forceinline__ void resolve_slot(const Launch& P, TileSlot& S, unsigned E)
{
    int ok = 0;
    unsigned long long ex = 0ull, start = 0ull;
    if (S.pub && dcheck(P.ctl, S.g < P.ws_cap && S.item < max(P.n_items, 1u), S.g)) {
        unsigned long long agg = S.head;
#pragma unroll
        for (int w = 0; w < NWARPS; ++w) agg += (unsigned long long)S.segsz[w];
        const unsigned g0 = P.packed ? 0u : S.g - S.tile;
        bool expired = false;
        // the encoder warps published the aggregate already (publish_aggregate)
        ex = lookback_warp(P.chB, S.g, g0, agg, S.last != 0, E, P.wc, P.ctl, expired, true);
        ok = !expired && packed_start_warp(P, S.first != 0, S.item, ex, S.g, E, start);
    }
    if ((threadIdx.x & 31) == 0) {
        S.ex = ex;
        S.start = start;
        S.ok = ok;
    }
}

// The encoder CTA.  Tickets are taken in order, so a tile only ever waits for
// tiles taken earlier by CTAs that are running or done; every resolver
// publishes its tiles in ticket order, so the chain always advances.  The
// last CTA to finish advances the launch generation.
//   enc(item, index, tile in item, segment, width bytes, stage, slot, shared) -> unit size
//   fin(item, index, tile in item, ticket, slot, segment, width bytes)
// Barrier protocol per tile in slot s: the encoder warps arrive on BAR_ENC + s
// after encoding it, the resolver waits there, resolves it and arrives on
// BAR_RES + s, where the encoder warps wait NS - 1 tiles later before
// storing it.  A slot's barriers are used again only after both sides have
// passed them, and every path through the loops meets every barrier.
template <int U, bool SINGLE, typename Src, typename Enc, typename Fin>
__device__ __forceinline__ void enc_pipeline(const Launch& P, const Src& src, Enc enc, Fin fin)
{
    constexpr int NS = enc_slots(U);  // tiles in flight
    constexpr int D = NS - 1;         // tiles between a tile's encoding and its stores
    __shared__ TileSlot slots[NS];
    __shared__ EncShared es;
    extern __shared__ __align__(16) uint8_t dsm[];  // width bytes [slot][warp][2U] (, stages)
    __shared__ __align__(16) uint8_t stage_static[SINGLE ? 1 : NWARPS][SINGLE ? 16 : stage_bytes(32)];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a relative bound comes from the range kernel launched just before, the
    // fused ring step's offsets and tile map from the kernels before it: an
    // encoder launched dependent on them waits here for them to complete
    // (every thread: their results are read below and in every tile)
    if (P.eb_from_ctl || P.dep) grid_dep_wait();
    if (tid == 0) {
        es.E = ld_volatile_u32(&P.ctl->epoch) + 1u;
        int a = ld_volatile_u32(&P.ctl->magic) != WS_MAGIC;
        if (a) {
            fail(P.ctl, ZC_ERR_WORKSPACE, 0);
        } else if ((unsigned long long)gridDim.x * ring_cta_bytes(U) > P.ring_bytes) {
            a = 1;  // more CTAs than rings: the whole launch does nothing
            if (blockIdx.x == 0) fail(P.ctl, ZC_ERR_WORKSPACE, 1);
        } else if (P.eb_from_ctl && ld_volatile_u32(&P.ctl->eb_ok) != 1u) {
            a = 2;
        }
        es.abort = a;
    }
    __syncthreads();
    if (es.abort == 1) return;
    const bool no_eb = es.abort == 2;
    const unsigned E = es.E;
    const unsigned modulus = P.total_tiles + gridDim.x - 1u;
    uint8_t* const ring = P.ring + (unsigned long long)blockIdx.x * ring_cta_bytes(U);
    if (warp < NWARPS) {
        auto seg_of = [&](int s) { return ring + (unsigned long long)(s * NWARPS + warp) * seg_bytes(U); };
        auto wb_of = [&](int s) { return dsm + (s * NWARPS + warp) * (U * 2); };
        auto stage_of = [&]() -> uint8_t* {
            if constexpr (SINGLE) return dsm + enc_wb_bytes(U) + warp * stage_bytes(stage_rows(U, true));
            else return stage_static[warp];
        };
        auto store = [&](int q) {
            bar_sync_n(BAR_RES + q, ENC_THREADS);
            const TileSlot& Q = slots[q];
            if (Q.ok) {
                const Item it = src.get(Q.item);
                fin(it, Q.item, Q.tile, Q.g, Q, seg_of(q), wb_of(q));
            }
        };
        int s = 0;
        for (int i = 0;; ++i) {
            bar_sync_n(BAR_ENCW, NTHREADS);  // slot s's previous tile is stored
            if (tid == 0) {
                TileSlot& S = slots[s];
                const unsigned g = atomicInc(&P.ctl->ticket, modulus);
                S.g = g;
                S.valid = g < P.total_tiles;
                S.item = g < P.total_tiles ? src.find(g) : 0u;
                S.pub = 0;
                S.nfin = 0;
            }
            bar_sync_n(BAR_ENCW, NTHREADS);
            TileSlot& S = slots[s];
            const bool valid = S.valid != 0;
            int lo = 0;
            if (valid && !no_eb) {
                const Item it = src.get(S.item);
                const unsigned t = S.g - it.tile_begin;
                if (tid == 0) S.tile = t;
                lo = enc(it, S.item, t, seg_of(s), wb_of(s), stage_of(), S, es);
            }
            if (lane == 0) {
                S.segsz[warp] = lo;
                __threadfence_block();
                if (atomicAdd(&S.nfin, 1) == NWARPS - 1) {  // the tile's last encoder warp
                    __threadfence_block();
                    publish_aggregate(P, S, E);
                }
            }
            bar_arrive_n(BAR_ENC + s, ENC_THREADS);
            if (!valid) {
                // the tiles still waiting for their stores, oldest first
                for (int k = (i < D ? i : D) - 1; k >= 0; --k) store((s + NS - 1 - k) % NS);
                break;
            }
            if (i >= D) store((s + 1) % NS);
            s = s + 1 == NS ? 0 : s + 1;
        }
    } else {
        int s = 0;
        while (true) {
            bar_sync_n(BAR_ENC + s, ENC_THREADS);
            TileSlot& S = slots[s];
            if (!S.valid) break;
            resolve_slot(P, S, E);
            __syncwarp();
            bar_arrive_n(BAR_RES + s, ENC_THREADS);
            s = s + 1 == NS ? 0 : s + 1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        if (atomicInc(&P.ctl->done, gridDim.x - 1u) == gridDim.x - 1u) {
            P.ctl->epoch = E;
            __threadfence();
        }
    }
}

template <int LOG2L, int U, typename TX, bool HEADS = false>
__global__ void __launch_bounds__(ENC_THREADS, ENC_CTAS_PER_SM) k_compress(const Launch P)
{
    enc_pipeline<U, true>(
        P, ItemsSrc{P},
        [&](const Item& it, unsigned idx, unsigned t, uint8_t* seg, uint8_t* wb, uint8_t* stage,
            TileSlot& S, EncShared& es) {
            return enc_tile<LOG2L, U, false, TX, HEADS, stage_rows(U, true)>(P, it, idx, t, seg, wb,
                                                                          stage, S, es);
        },
        [&](const Item& it, unsigned idx, unsigned t, unsigned g, const TileSlot& S,
            const uint8_t* seg, const uint8_t* wb) { fin_tile<LOG2L, U, false, HEADS>(P, it, idx, t, g, S, seg, wb); });
}

template <int LOG2L, int U, typename TX>
__global__ void __launch_bounds__(ENC_THREADS, ENC_CTAS_PER_SM) k_scatter(const Launch P,
                                                                          const ScatterParams SP)
{
    enc_pipeline<U, true>(
        P, ScatterSrc{P, SP},
        [&](const Item& it, unsigned idx, unsigned t, uint8_t* seg, uint8_t* wb, uint8_t* stage,
            TileSlot& S, EncShared& es) {
            return enc_tile<LOG2L, U, false, TX, false, stage_rows(U, true)>(P, it, idx, t, seg, wb,
                                                                          stage, S, es);
        },
        [&](const Item& it, unsigned idx, unsigned t, unsigned g, const TileSlot& S,
            const uint8_t* seg, const uint8_t* wb) { fin_tile<LOG2L, U, false>(P, it, idx, t, g, S, seg, wb); });
}

template <int LOG2L, int U>
__global__ void __launch_bounds__(ENC_THREADS, ENC_CTAS_PER_SM) k_reduce(const Launch P)
{
    enc_pipeline<U, false>(
        P, ItemsSrc{P},
        [&](const Item& it, unsigned idx, unsigned t, uint8_t* seg, uint8_t* wb, uint8_t* stage,
            TileSlot& S, EncShared& es) {
            return enc_tile<LOG2L, U, true, float>(P, it, idx, t, seg, wb, stage, S, es);
        },
        [&](const Item& it, unsigned idx, unsigned t, unsigned g, const TileSlot& S,
            const uint8_t* seg, const uint8_t* wb) { fin_tile<LOG2L, U, true>(P, it, idx, t, g, S, seg, wb); });
}

// ---- batched compression -----------------------------------------------------
// Every item is a stream of its own block size and input type (or raw), all
// packed back to back by one chain; the CTAs take tiles of all items from one
// ticket counter, so one launch of a few CTAs per SM covers any mix of
// message sizes.
template <int U>
__global__ void __launch_bounds__(ENC_THREADS, ENC_CTAS_PER_SM) k_batch(const Launch P)
{
    enc_pipeline<U, false>(
        P, ItemsSrc{P},
        [&](const Item& it, unsigned idx, unsigned t, uint8_t* seg, uint8_t* wb, uint8_t* stage,
            TileSlot& S, EncShared& es) -> int {
            const bool f32 = it.x_dtype == ZC_F32;
            switch (it.log2L) {
            case 4:
                return f32 ? enc_tile<4, U, false, float>(P, it, idx, t, seg, wb, stage, S, es)
                           : enc_tile<4, U, false, uint16_t>(P, it, idx, t, seg, wb, stage, S, es);
            case 5:
                return f32 ? enc_tile<5, U, false, float>(P, it, idx, t, seg, wb, stage, S, es)
                           : enc_tile<5, U, false, uint16_t>(P, it, idx, t, seg, wb, stage, S, es);
            case 6:
                return f32 ? enc_tile<6, U, false, float>(P, it, idx, t, seg, wb, stage, S, es)
                           : enc_tile<6, U, false, uint16_t>(P, it, idx, t, seg, wb, stage, S, es);
            case 7:
                return f32 ? enc_tile<7, U, false, float>(P, it, idx, t, seg, wb, stage, S, es)
                           : enc_tile<7, U, false, uint16_t>(P, it, idx, t, seg, wb, stage, S, es);
            default: return enc_raw<U>(it, t, S);
            }
        },
        [&](const Item& it, unsigned idx, unsigned t, unsigned g, const TileSlot& S,
            const uint8_t* seg, const uint8_t* wb) {
            switch (it.log2L) {
            case 4: fin_tile<4, U, false>(P, it, idx, t, g, S, seg, wb); break;
            case 5: fin_tile<5, U, false>(P, it, idx, t, g, S, seg, wb); break;
            case 6: fin_tile<6, U, false>(P, it, idx, t, g, S, seg, wb); break;
            case 7: fin_tile<7, U, false>(P, it, idx, t, g, S, seg, wb); break;
            default: fin_raw<U>(P, it, idx, t, g, S); break;
            }
        });
}

// Batched decompression: item idx's stream, from a packed buffer written by an
// earlier launch.  A start or an end outside the buffer, or a start that is
// not 16-byte aligned, leaves a stream too short for its header (reported as
// a format error by the decoder).
__device__ __forceinline__ void resolve_packed(const Launch& P, Item& it, unsigned idx)
{
    if (P.in_off == nullptr) return;
    const unsigned long long a = P.in_off[idx];
    const unsigned long long b = P.in_off[P.grouped ? P.n_items : idx + 1];
    const bool ok = (a & 15ull) == 0 && a <= b && b <= P.in_cap;
    it.cin = P.in_base + (ok ? a : 0ull);
    it.cin_cap = ok ? b - a : 0ull;
}

#ifdef ZC_DECODE_KERNELS  // defined by the one translation unit that launches them

// Item of every encoder tile (by_chunk: of every width-scan chunk) of a
// multi-item launch, so that a CTA finds its ticket's item with one load
// instead of a binary search of dependent loads.
// Launched dependent on a width scan (the fused ring step), the map is
// built while the scan runs; the kernel then waits for the scan, so that it
// never completes before it (the step launched dependent on the map reads
// the scan's offsets too).  Thread 0 always reaches the wait.
__global__ void __launch_bounds__(NTHREADS) k_tile_map(const Item* items, unsigned n_items,
                                                      unsigned total_tiles, unsigned* map,
                                                      int by_chunk)
{
    grid_dep_launch();
    const unsigned g = blockIdx.x * NTHREADS + threadIdx.x;
    if (g >= total_tiles) return;
    unsigned lo = 0, hi = n_items;
    while (hi - lo > 1) {
        const unsigned mid = (lo + hi) >> 1;
        const unsigned b = by_chunk ? __ldg(&items[mid].chunk_begin) : __ldg(&items[mid].tile_begin);
        if (b <= g) lo = mid;
        else hi = mid;
    }
    map[g] = lo;
    grid_dep_wait();
}

// ---- grouped batches ------------------------------------------------------------
// The tiles of all messages of one block size (classes: raw, 16, 32, 64, 128)
// take consecutive tickets, so the CTAs running at any time mostly run one
// encoder variant.  Within a class, messages keep their order.  Three small
// launches over GROUP_T messages per CTA: per-CTA tile sums of every class;
// one CTA turns them into every CTA's first ticket per class; each CTA then
// gives its messages their first tickets and fills the ticket -> item map.
constexpr int GROUP_T = 256;
constexpr int GROUP_CLASSES = 5;
__device__ __forceinline__ int group_class(int log2L) { return log2L < 4 ? 0 : log2L - 3; }

__global__ void __launch_bounds__(GROUP_T) k_group_count(const Item* items, unsigned n_items,
                                                         unsigned* part)
{
    __shared__ unsigned red[GROUP_CLASSES][GROUP_T / 32];
    const unsigned i = blockIdx.x * GROUP_T + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c = -1;
    unsigned t = 0;
    if (i < n_items) {
        c = group_class(__ldg(&items[i].log2L));
        t = __ldg(&items[i].ntiles);
    }
#pragma unroll
    for (int k = 0; k < GROUP_CLASSES; ++k) {
        const unsigned v = __reduce_add_sync(FULL, c == k ? t : 0u);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < GROUP_CLASSES) {
        unsigned v = 0;
        for (int w = 0; w < GROUP_T / 32; ++w) v += red[threadIdx.x][w];
        part[(size_t)blockIdx.x * GROUP_CLASSES + threadIdx.x] = v;
    }
}

// One CTA of 1024 threads: part[b][c] (tiles of class c in CTA b's messages)
// becomes the first ticket of class c in CTA b: the class's base (the tiles
// of all smaller classes) plus the class's tiles in CTAs before b.
__global__ void __launch_bounds__(1024) k_group_scan(unsigned* part, unsigned nblk)
{
    __shared__ unsigned wsum[32];
    __shared__ unsigned carry[GROUP_CLASSES];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid < GROUP_CLASSES) carry[tid] = 0;
    __syncthreads();
    // pass over the classes: exclusive scans within each class
    for (int c = 0; c < GROUP_CLASSES; ++c) {
        for (unsigned b0 = 0; b0 < nblk; b0 += 1024) {
            const unsigned b = b0 + tid;
            const unsigned v = b < nblk ? part[(size_t)b * GROUP_CLASSES + c] : 0u;
            unsigned s = v;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned o = __shfl_up_sync(FULL, s, off);
                if (lane >= off) s += o;
            }
            if (lane == 31) wsum[warp] = s;
            __syncthreads();
            if (warp == 0) {
                unsigned w = wsum[lane];
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const unsigned o = __shfl_up_sync(FULL, w, off);
                    if (lane >= off) w += o;
                }
                wsum[lane] = w;  // inclusive over warps
            }
            __syncthreads();
            const unsigned excl = carry[c] + (warp ? wsum[warp - 1] : 0u) + s - v;
            if (b < nblk) part[(size_t)b * GROUP_CLASSES + c] = excl;
            __syncthreads();
            if (tid == 0) carry[c] += wsum[31];
            __syncthreads();
        }
    }
    // class bases: the tiles of the smaller classes
    unsigned base = 0;
    for (int c = 0; c < GROUP_CLASSES; ++c) {
        const unsigned tot = carry[c];
        for (unsigned b = tid; b < nblk; b += 1024) part[(size_t)b * GROUP_CLASSES + c] += base;
        base += tot;
    }
}

__global__ void __launch_bounds__(GROUP_T) k_group_place(Item* items, unsigned n_items,
                                                         const unsigned* part, unsigned* map)
{
    __shared__ unsigned wsum[GROUP_CLASSES][GROUP_T / 32];
    const unsigned i = blockIdx.x * GROUP_T + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int c = -1;
    unsigned t = 0;
    if (i < n_items) {
        c = group_class(items[i].log2L);
        t = items[i].ntiles;
    }
    unsigned mine = 0;  // exclusive sum of this class's tiles before message i within the warp
#pragma unroll
    for (int k = 0; k < GROUP_CLASSES; ++k) {
        const unsigned v = c == k ? t : 0u;
        unsigned s = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned o = __shfl_up_sync(FULL, s, off);
            if (lane >= off) s += o;
        }
        if (lane == 31) wsum[k][warp] = s;
        if (c == k) mine = s - v;
    }
    __syncthreads();
    if (i >= n_items) return;
    unsigned first = part[(size_t)blockIdx.x * GROUP_CLASSES + c] + mine;
    for (int w = 0; w < warp; ++w) first += wsum[c][w];
    items[i].tile_begin = first;
    for (unsigned k = 0; k < t; ++k) map[first + k] = i;
}

// ---- width scan: payload offset of every decode tile --------------------------
// One CTA per chunk of WSCAN warp units of one item; thread i sums the plane
// bytes of unit i from its width bytes; a CTA scan and a look-back over the
// item's chunks give every unit's payload offset (global decode slot = item
// tile slot * NWARPS + unit in tile).  A multi-item launch finds a chunk's
// item in P.tile_map, here the chunk -> item map (k_tile_map by chunk).
__global__ void __launch_bounds__(NTHREADS) k_wscan(const Launch P)
{
    __shared__ Smem sm;
    __shared__ int wsum[NWARPS];
    grid_dep_launch();  // the decoder after it may be launched now (it waits for the offsets)
    if (threadIdx.x == 0) {
        sm.E = ld_volatile_u32(&P.ctl->epoch) + 1u;
        sm.abort = ld_volatile_u32(&P.ctl->magic) != WS_MAGIC;
        if (sm.abort) fail(P.ctl, ZC_ERR_WORKSPACE, 0);
    }
    __syncthreads();
    if (sm.abort) return;
    const unsigned modulus = P.total_tiles + gridDim.x - 1u;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    while (true) {
        __syncthreads();
        if (tid == 0) {
            sm.ticket = atomicInc(&P.ctl->ticket, modulus);
            unsigned it = 0;
            if (P.items != nullptr && sm.ticket < P.total_tiles) {
                if (P.tile_map != nullptr) {
                    it = P.tile_map[sm.ticket];  // the chunk map of this launch
                } else {
                    unsigned lo = 0, hi = P.n_items;
                    while (hi - lo > 1) {
                        const unsigned mid = (lo + hi) >> 1;
                        if (P.items[mid].chunk_begin <= sm.ticket) lo = mid;
                        else hi = mid;
                    }
                    it = lo;
                }
            }
            sm.item = it;
        }
        __syncthreads();
        const unsigned c = sm.ticket;
        if (c >= P.total_tiles) break;
        Item it = P.items != nullptr ? P.items[sm.item] : P.one;
        resolve_packed(P, it, sm.item);
        if (it.cin == nullptr) continue;  // nothing received: no offsets needed
        const unsigned chunk = c - it.chunk_begin;
        float eb_in;
        const int lg = check_header(it, P.ctl, sm.item, -1, eb_in, false);
        if (lg < 4) continue;  // raw or malformed: the decoder reports it
        const int lgb = lg & 7;  // block size (heads apart or not: same widths)
        const unsigned long long L = 1ull << lgb;
        const unsigned long long nb = (it.n + L - 1) >> lgb;
        const int PB = (int)(L / 8);
        const unsigned long long ntile = (unsigned long long)it.ntiles * NWARPS;  // units
        const unsigned long long k = (unsigned long long)chunk * WSCAN + tid;    // unit in item
        const int bpt = (P.urows * 32) >> lgb;                                   // blocks per unit
        int sum = 0;
        if (k < ntile) {
            const unsigned long long b0 = k * bpt;
            const uint8_t* w = it.cin + 32;
            // bpt is 8 (32-row units at L = 128) or a multiple of 16
            const int step = bpt < 16 ? 8 : 16;
            for (int i = 0; i < bpt; i += step) {
                if (b0 + i >= ceil16(nb)) break;
                unsigned ws[4] = {0u, 0u, 0u, 0u};
                if (step == 16) {
                    const uint4 v = __ldg((const uint4*)(w + b0 + i));
                    ws[0] = v.x;
                    ws[1] = v.y;
                    ws[2] = v.z;
                    ws[3] = v.w;
                } else {
                    const uint2 v = __ldg((const uint2*)(w + b0 + i));
                    ws[0] = v.x;
                    ws[1] = v.y;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int wv = (ws[q] >> (8 * b)) & 0xff;
                        if (wv > ZC_MAX_WIDTH) fail(P.ctl, ZC_ERR_FORMAT, b0 + i + 4 * q + b);
                        else sum += planes_of(wv) * PB;
                    }
            }
        }
        int tot;
        const int ex = warp_excl_scan(sum, lane, tot);
        if (lane == 0) wsum[warp] = tot;
        __syncthreads();
        unsigned long long wbase = 0, cagg = 0;
        for (int w = 0; w < NWARPS; ++w) {
            if (w < warp) wbase += wsum[w];
            cagg += wsum[w];
        }
        bool to = false;
        if (DEBUG_BUILD && tid == 0) dcheck(P.ctl, c < P.ws_cap, c);
        const unsigned long long cex =
            lookback_cta(P.chC, c, it.chunk_begin, cagg, false, sm.E, P.wc, P.ctl, to, sm.lb);
        if (to) continue;
        const unsigned long long oslot = (unsigned long long)it.tile_begin * NWARPS + k;
        if (k < ntile && dcheck(P.ctl, oslot < P.ws_cap, oslot)) P.offs[oslot] = cex + wbase + ex;
        if (chunk + 1 == it.nchunks && tid == 0) {
            const unsigned long long payload = __ldg((const unsigned long long*)it.cin + 3);
            if (cex + cagg != payload) fail(P.ctl, ZC_ERR_FORMAT, sm.item);
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicInc(&P.ctl->done, gridDim.x - 1u) == gridDim.x - 1u) {
            P.ctl->epoch = sm.E;
            __threadfence();
        }
    }
}

// ---- decompression -------------------------------------------------------------

// Raw streams: copy (and convert) the elements of this warp unit.
__device__ __forceinline__ void unit_raw_copy(const Item& it, int src_dtype, unsigned long long ue0)
{
    const uint8_t* src = it.cin + 32;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < DEC_U; ++r) {
        const unsigned long long e = ue0 + (unsigned long long)r * 32 + lane;
        if (e < it.n) {
            const float v = src_dtype == ZC_F32 ? __ldg((const float*)src + e)
                                                : bf16_to_f32(__ldg((const unsigned short*)src + e));
            store_raw(it.raw_out, it.out_dtype, e, v);
        }
    }
}

template <int LOG2L, typename TO, bool HEADS = false>
__device__ __forceinline__ void unit_decode(const Launch& P, const Item& it, unsigned slot,
                                            unsigned long long ue0, float two_eb, int2* meta,
                                            long long off_local)
{
    const int lane = threadIdx.x & 31;
    const TpC tc = tp_consts(lane);
    bool narrow;
    bool narrow11;
    const uint8_t* src = it.cin + unit_meta<LOG2L, DEC_U, HEADS>(P, it, slot, ue0, meta, narrow,
                                                                 narrow11, off_local);
    const uint8_t* hsrc = nullptr;  // heads apart: the heads of this unit's blocks
    if (HEADS) {
        const unsigned long long nb = (it.n + (1ull << LOG2L) - 1) >> LOG2L;
        hsrc = it.cin + 32 + ceil16(nb) + 3ull * (ue0 >> LOG2L);
    }
#pragma unroll 1
    for (int gi = 0; gi < DEC_U / GR; ++gi) {
        const unsigned long long e0 = ue0 + (unsigned long long)gi * GR * 32;
        if (e0 >= it.n) break;
        const int nrem = (int)min(it.n - e0, (unsigned long long)(GR * 32));
        float acc[GR];
        if (!HEADS && narrow11) decode_group<LOG2L, true, false, true>(src, meta, gi, two_eb, acc, tc);
        else if (narrow) decode_group<LOG2L, true, HEADS>(src, meta, gi, two_eb, acc, tc, hsrc);
        else decode_group<LOG2L, false, HEADS>(src, meta, gi, two_eb, acc, tc, hsrc);
        TO* op = (TO*)it.raw_out + e0 + lane;
        if (nrem == GR * 32) {
#pragma unroll
            for (int r = 0; r < GR; ++r) {
                if (sizeof(TO) == 4) ((float*)op)[r * 32] = acc[r];
                else ((uint16_t*)op)[r * 32] = f32_to_bf16(acc[r]);
            }
        } else {
#pragma unroll
            for (int r = 0; r < GR; ++r) {
                if (r * 32 + lane < nrem) {
                    if (sizeof(TO) == 4) ((float*)op)[r * 32] = acc[r];
                    else ((uint16_t*)op)[r * 32] = f32_to_bf16(acc[r]);
                }
            }
        }
    }
}

// Items of at most DEC_LOCAL_TILES decode tiles (planned with no width-scan
// chunks) need no width scan: the decoder CTA of tile t sums the plane bytes
// of the item's blocks before its tile itself (at most DEC_LOCAL_TILES - 1
// tiles' width bytes) and its warps' units (one value per warp), which gives
// every warp its unit's payload offset; the item's last tile checks the total
// against the header's payload size, as the width scan does.  Called by every
// thread of the CTA (coded streams only: lg >= 4).
__device__ __forceinline__ unsigned long long local_unit_offset(const Item& it, int lg, unsigned t,
                                                                Ctl* ctl, unsigned item_idx)
{
    __shared__ unsigned long long s_pre[NWARPS], s_own[NWARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int lgb = lg & 7;
    const unsigned long long PB = (1ull << lgb) / 8;
    const unsigned long long nb = (it.n + (1ull << lgb) - 1) >> lgb;
    const unsigned long long bpu = (unsigned long long)(DEC_U * 32) >> lgb;  // blocks per unit
    const uint8_t* w = it.cin + 32;
    auto bytes_of = [&](unsigned long long b) -> unsigned long long {
        const int wv = __ldg(w + b);
        return wv > ZC_MAX_WIDTH ? 0ull : (unsigned long long)planes_of(wv) * PB;
    };
    const unsigned long long pre_end = min((unsigned long long)t * NWARPS * bpu, nb);
    unsigned long long pre = 0ull;
    for (unsigned long long b = tid; b < pre_end; b += NTHREADS) pre += bytes_of(b);
    const unsigned long long u_lo = ((unsigned long long)t * NWARPS + warp) * bpu;
    const unsigned long long u_hi = min(u_lo + bpu, nb);
    unsigned long long own = 0ull;
    for (unsigned long long b = u_lo + lane; b < u_hi; b += 32) own += bytes_of(b);
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        pre += __shfl_xor_sync(FULL, pre, o);
        own += __shfl_xor_sync(FULL, own, o);
    }
    if (lane == 0) {
        s_pre[warp] = pre;
        s_own[warp] = own;
    }
    __syncthreads();
    unsigned long long off = 0ull, total = 0ull;
#pragma unroll
    for (int v = 0; v < NWARPS; ++v) {
        off += s_pre[v] + (v < warp ? s_own[v] : 0ull);
        total += s_pre[v] + s_own[v];
    }
    if (t + 1 == it.ntiles && tid == 0 &&
        total != __ldg((const unsigned long long*)it.cin + 3))
        fail(ctl, ZC_ERR_FORMAT, item_idx);
    return off;
}

// NWARPS warp units per CTA, one per warp, independent of each other; the
// block size comes from the stream's header.
// 5 CTAs per SM (48 registers): the decoder waits on its plane loads, and the
// extra warps hide more of that than the few spilled values cost (measured on
// the 512^3 field: 0.166 ms at 5 CTAs per SM, 0.175 ms at 4, 0.168 ms at 6)
// BATCH: a multi-item launch (items may find their own unit offsets); the
// single-stream decoder is compiled without that path, which would cost it
// registers.
template <bool BATCH>
__device__ __forceinline__ void decompress_tile(const Launch& P)
{
    __shared__ __align__(16) int2 meta[NWARPS][DEC_U * 2];
    const unsigned tile = blockIdx.x;
    unsigned idx = 0;
    if (P.tile_map != nullptr) {
        idx = P.tile_map[tile];
    } else if (P.items != nullptr) {
        unsigned lo = 0, hi = P.n_items;
        while (hi - lo > 1) {
            const unsigned mid = (lo + hi) >> 1;
            if (P.items[mid].tile_begin <= tile) lo = mid;
            else hi = mid;
        }
        idx = lo;
    }
    Item it = P.items != nullptr ? P.items[idx] : P.one;
    resolve_packed(P, it, idx);
    const unsigned t = tile - it.tile_begin;
    const int warp = threadIdx.x >> 5;
    const unsigned long long ue0 = ((unsigned long long)t * NWARPS + warp) * (DEC_U * 32);
    const unsigned slot = tile * NWARPS + warp;
    float eb_in;
    const int lg = check_header(it, P.ctl, idx, -1, eb_in, threadIdx.x == 0 && t == 0);
    long long loff = -1;  // the unit's payload offset, when this CTA finds it
    if (BATCH && it.nchunks == 0 && lg >= 4)  // uniform in the CTA
        loff = (long long)local_unit_offset(it, lg, t, P.ctl, idx);
    // the width scan's offsets are read from here on: a single-stream decoder
    // launched dependent on the scan has looked up its tile and checked the
    // header while the scan ran, and waits for it now.  Every thread passes
    // this wait, so the decoder never completes before the scan (later
    // launches on the stream find the scan finished).
    if (!BATCH) grid_dep_wait();
    if (ue0 >= it.n) return;
    const float two = __fadd_rn(eb_in, eb_in);
    if (it.out_dtype == ZC_F32) {
        switch (lg) {
        case 4: unit_decode<4, float>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 5: unit_decode<5, float>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 6: unit_decode<6, float>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 7: unit_decode<7, float>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 12: unit_decode<4, float, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 13: unit_decode<5, float, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 14: unit_decode<6, float, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 15: unit_decode<7, float, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        default: break;
        }
    } else {
        switch (lg) {
        case 4: unit_decode<4, uint16_t>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 5: unit_decode<5, uint16_t>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 6: unit_decode<6, uint16_t>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 7: unit_decode<7, uint16_t>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 12: unit_decode<4, uint16_t, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 13: unit_decode<5, uint16_t, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 14: unit_decode<6, uint16_t, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        case 15: unit_decode<7, uint16_t, true>(P, it, slot, ue0, two, meta[warp], loff); return;
        default: break;
        }
    }
    if (lg == -2) unit_raw_copy(it, ZC_F32, ue0);
    else if (lg == -3) unit_raw_copy(it, ZC_BF16, ue0);
}

template <bool BATCH>
__global__ void __launch_bounds__(NTHREADS, 5) k_decompress(const Launch P)
{
    decompress_tile<BATCH>(P);
}

#endif  // ZC_DECODE_KERNELS

}  // namespace zc
