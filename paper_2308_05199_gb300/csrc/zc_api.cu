// zc_api.cu -- the C ABI declared in include/zc.h: argument checks, workspace
// carving, tile planning and kernel launches.  No call allocates memory, reads
// device memory back (except zc_get_device_status and the setup-time plan
// builder) or synchronises the stream.
#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "zc_launch.h"

using namespace zc;

namespace {

int g_chunks = 0;  // sub-tiles of 2048 elements per encoder tile; 0: chosen per launch
unsigned long long g_wait_ns = 1000000000ull;
long long g_withhold = -1;

inline uint64_t pad16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

int log2_block(int block)
{
    switch (block) {
    case 16: return 4;
    case 32: return 5;
    case 64: return 6;
    case 128: return 7;
    default: return -1;
    }
}

inline bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }
inline bool dtype_ok(int t) { return t == ZC_F32 || t == ZC_BF16; }
// An encoder tile is NWARPS warp units of `rows` rows of 32 elements (tile
// size knob: chunks of 2048 elements, rows = 8 chunks); the decompressor's
// tile is NWARPS units of DEC_U rows.
inline uint64_t tiles_for(uint64_t n, int rows)
{
    const uint64_t te = (uint64_t)NWARPS * rows * 32;
    const uint64_t t = (n + te - 1) / te;
    return t ? t : 1;
}
// Width-scan chunks for `ntiles` tiles (one thread per warp unit).
inline uint64_t chunks_for(uint64_t ntiles)
{
    return (ntiles * NWARPS + WSCAN - 1) / WSCAN;
}

// Host copy of the FP32 bound: eb, 2 eb and the rounded reciprocal of 2 eb.
int qparams(double eb_abs, float* eb, float* two, float* inv)
{
    if (!(eb_abs > 0.0) || !std::isfinite(eb_abs)) return ZC_ERR_ARG;
    const float e = (float)eb_abs;
    if (!std::isnormal(e) || e <= 0.0f) return ZC_ERR_ARG;
    volatile float t = e;
    t = t + e;
    if (!std::isfinite((float)t)) return ZC_ERR_ARG;
    *eb = e;
    *two = t;
    *inv = (float)(0.5 / (double)e);
    return ZC_OK;
}

// Workspace: control block, range partials, then 9 arrays of `cap` u64:
// decode-tile offsets, encoder look-back (flag, wide aggregate, prefix),
// width-scan look-back (same three), per-item stream-start flags, and the
// tile-to-item map of multi-item encoder launches (u32 entries); then the
// encoder CTAs' tile rings: ring_ctas(cap) rings of the largest tile size.
constexpr uint64_t WS_ARRAYS = 9;
constexpr uint64_t RING_CTAS_MAX = 152 * ENC_CTAS_PER_SM;  // every resident encoder CTA
constexpr uint64_t RING_UNIT = ring_cta_bytes(unit_rows(16));  // the largest ring of any tile size
static_assert(RING_UNIT >= ring_cta_bytes(unit_rows(8)) && RING_UNIT >= ring_cta_bytes(unit_rows(4)), "ring unit");

// Rings (of the largest tile size) for a workspace of `cap` array entries:
// one per 16 entries (a tile of 8 chunks needs 16 entries of decode slots),
// at least one.
inline uint64_t ring_ctas(uint64_t cap)
{
    const uint64_t r = (cap + 15) / 16;
    return r < 1 ? 1 : (r > RING_CTAS_MAX ? RING_CTAS_MAX : r);
}
inline uint64_t ring_offset(uint64_t cap)
{
    return (WS_CTL_BYTES + WS_RANGE_BYTES + cap * WS_ARRAYS * 8 + 255) & ~(uint64_t)255;
}
inline uint64_t ws_total(uint64_t cap) { return ring_offset(cap) + ring_ctas(cap) * RING_UNIT; }

struct WsView {
    Ctl* ctl;
    float2* partial;
    unsigned long long* offs;
    Chain chB, chC;
    ulonglong2* seg_rec;
    unsigned* tile_map;
    uint64_t cap;  // decode tiles (and tiles, chunks, items) the workspace can hold
    uint8_t* ring;
    uint64_t ring_bytes;
    uint64_t ring_off;
};

// The arrays at `ws` with `cap` entries, the rings given apart.
void ws_carve(void* ws, uint64_t cap, uint8_t* ring, uint64_t ring_bytes, WsView& v)
{
    const uint64_t fixed = WS_CTL_BYTES + WS_RANGE_BYTES;
    unsigned long long* base = (unsigned long long*)((char*)ws + fixed);
    v.ctl = (Ctl*)ws;
    v.partial = (float2*)((char*)ws + WS_CTL_BYTES);
    v.offs = base;
    // look-back records (16 bytes per slot; cap is even, so they are 16-byte
    // aligned): encoder tiles in [cap, 3 cap), width-scan chunks in
    // [4 cap, 6 cap), stream starts of packed items in [7 cap, 8 cap)
    v.chB = Chain{(ulonglong2*)(base + cap)};
    v.chC = Chain{(ulonglong2*)(base + 4 * cap)};
    v.seg_rec = (ulonglong2*)(base + 7 * cap);
    v.tile_map = (unsigned*)(base + 8 * cap);
    v.cap = cap;
    v.ring = ring;
    v.ring_bytes = ring_bytes;
    v.ring_off = ring_offset(cap);
}

// The layout of a workspace of `bytes`: the largest cap whose arrays and
// rings fit (ws_total grows with cap, so a bisection finds it).
int ws_view(void* ws, size_t bytes, WsView& v)
{
    if (ws == nullptr || !aligned(ws, 16)) return ZC_ERR_ARG;
    if (bytes < ws_total(4)) return ZC_ERR_WORKSPACE;
    uint64_t lo = 4, hi = bytes / (WS_ARRAYS * 8) + 1;  // ws_total(lo) <= bytes < ws_total(hi)
    while (hi - lo > 1) {
        const uint64_t mid = lo + (hi - lo) / 2;
        if (ws_total(mid) <= bytes) lo = mid;
        else hi = mid;
    }
    lo &= ~1ull;  // even: the look-back records stay 16-byte aligned (ws_total(lo) still fits)
    ws_carve(ws, lo, (uint8_t*)ws + ring_offset(lo), ring_ctas(lo) * RING_UNIT, v);
    return ZC_OK;
}

// Width scans over at least this many items find a chunk's item in a map
// (one extra launch); fewer items are searched (at most 8 dependent loads).
constexpr int CHUNK_MAP_ITEMS = 256;

// SM count of the current device (queried once per device).
int sm_count()
{
    static std::atomic<int> sms[64];  // SM count per device, 0 until queried
    int dev = 0;
    int n_sm = 152;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        int c = sms[dev].load(std::memory_order_relaxed);
        if (c == 0 && cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            c > 0)
            sms[dev].store(c, std::memory_order_relaxed);
        if (c > 0) n_sm = c;
    }
    return n_sm;
}

// Tile size of a launch over `total` elements in items of `per_item`
// elements on average, unless zc_set_tile_chunks fixed one: the largest of 16
// and 8 chunks that is no larger than the mean item and still gives about 5/3
// tiles per resident encoder CTA, else 4.  Larger tiles cost fewer look-backs
// and per-tile steps, smaller ones keep every CTA busy (compression of the
// 512^3 field's first 2^20 .. 2^27 elements was fastest at 4 chunks up to
// 2^23 elements, 8 at 2^24 and 16 from 2^25 on).
int tile_chunks_for(uint64_t total, uint64_t per_item)
{
    if (g_chunks) return g_chunks;
    const uint64_t want = (uint64_t)sm_count() * ENC_CTAS_PER_SM * 5 / 3;
    for (int C = 16; C >= 8; C /= 2) {
        const uint64_t te = (uint64_t)NWARPS * unit_rows(C) * 32;
        if (te <= per_item && (total + te - 1) / te >= want) return C;
    }
    return 4;
}

// Encoder CTAs for a launch that wants `want` (its tile count or a chosen
// grid): at most one per ring and the resident CTAs of this GPU.
uint64_t enc_grid(uint64_t want, int U, const WsView& w)
{
    const int n_sm = sm_count();
    uint64_t g = want;
    const uint64_t rings = w.ring_bytes / ring_cta_bytes(U);
    const uint64_t resident = (uint64_t)n_sm * ENC_CTAS_PER_SM;
    if (g > rings) g = rings;
    if (g > resident) g = resident;
    return g;
}

Launch base_launch(const WsView& w)
{
    Launch P;
    std::memset(&P, 0, sizeof(P));
    P.ctl = w.ctl;
    P.chB = w.chB;
    P.chC = w.chC;
    P.offs = w.offs;
    P.seg_rec = w.seg_rec;
    P.urows = DEC_U;
    P.ring = w.ring;
    P.ring_bytes = w.ring_bytes;
    P.ws_cap = w.cap;
    P.wc.limit_ns = g_wait_ns;
    P.wc.withhold = g_withhold;
    return P;
}

int cuda_status(cudaError_t e) { return e == cudaSuccess ? ZC_OK : ZC_ERR_CUDA; }

unsigned range_grid(uint64_t n)
{
    uint64_t g = (n + 256 * 32 - 1) / (256 * 32);
    if (g < 1) g = 1;
    const uint64_t cap = (uint64_t)sm_count() * 4;  // 4 CTAs of 256 per SM: the fastest measured
    if (g > cap) g = cap;
    return (unsigned)g;
}

cudaError_t launch_compress_any(int lg, int S, int dt, const Launch& P, unsigned grid,
                                cudaStream_t s)
{
    switch (lg) {
    case 4: return launch_compress_lg<4>(S, dt, P, grid, s);
    case 5: return launch_compress_lg<5>(S, dt, P, grid, s);
    case 6: return launch_compress_lg<6>(S, dt, P, grid, s);
    default: return launch_compress_lg<7>(S, dt, P, grid, s);
    }
}

cudaError_t launch_reduce_any(int lg, int S, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (lg) {
    case 4: return launch_reduce_lg<4>(S, P, grid, s);
    case 5: return launch_reduce_lg<5>(S, P, grid, s);
    case 6: return launch_reduce_lg<6>(S, P, grid, s);
    default: return launch_reduce_lg<7>(S, P, grid, s);
    }
}

cudaError_t launch_scatter_any(int lg, int C, int dt, const Launch& P, const ScatterParams& S,
                               unsigned grid, cudaStream_t s)
{
    switch (lg) {
    case 4: return launch_scatter_lg<4>(C, dt, P, S, grid, s);
    case 5: return launch_scatter_lg<5>(C, dt, P, S, grid, s);
    case 6: return launch_scatter_lg<6>(C, dt, P, S, grid, s);
    default: return launch_scatter_lg<7>(C, dt, P, S, grid, s);
    }
}

cudaError_t launch_batch(int C, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (C) {
    case 4: return launch_batch_u<32>(P, grid, s);
    case 8: return launch_batch_u<64>(P, grid, s);
    default: return launch_batch_u<128>(P, grid, s);
    }
}

inline uint64_t elem_bytes(int dtype) { return dtype == ZC_F32 ? 4 : 2; }

}  // namespace

extern "C" {

#ifdef ZC_DEBUG
const char* zc_version(void) { return "zc 0.1 (sm_103a, bounds-checked)"; }
#else
const char* zc_version(void) { return "zc 0.1 (sm_103a)"; }
#endif

size_t zc_max_compressed_bytes(uint64_t n, int block)
{
    const int lg = log2_block(block);
    if (lg < 0) return 0;
    const uint64_t L = 1ull << lg;
    const uint64_t nb = (n + L - 1) / L;
    return 32 + pad16(nb) + pad16(nb * (ZC_MAX_WIDTH + 1) * (L / 8));
}

size_t zc_raw_stream_bytes(uint64_t n, int dtype)
{
    if (!dtype_ok(dtype)) return 0;
    return 32 + pad16(n * (dtype == ZC_F32 ? 4 : 2));
}

size_t zc_workspace_bytes(uint64_t n_total, int n_items)
{
    if (n_items < 1) n_items = 1;
    // decode slots: one per warp unit of at least 32 rows (1024 elements),
    // plus the partial tiles of every item
    const uint64_t cap = (n_total / 1024 + 16ull * (uint64_t)n_items + 3) & ~1ull;  // even
    return ws_total(cap);
}

int zc_workspace_init(void* d_ws, size_t ws_bytes, zc_stream_t s)
{
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    // the rings need no initial contents
    if (cudaMemsetAsync(d_ws, 0, w.ring_off, (cudaStream_t)s) != cudaSuccess) return ZC_ERR_CUDA;
    return cuda_status(launch_ws_init(w.ctl, (cudaStream_t)s));
}

int zc_minmax(const void* d_in, uint64_t n, int dtype, float* d_minmax, void* d_ws,
              size_t ws_bytes, zc_stream_t s)
{
    if ((n > 0 && d_in == nullptr) || !dtype_ok(dtype) || d_minmax == nullptr) return ZC_ERR_ARG;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    RangeLaunch R;
    std::memset(&R, 0, sizeof(R));
    R.ctl = w.ctl;
    R.partial = w.partial;
    R.minmax_out = d_minmax;
    R.one = RangeSeg{d_in, n};
    R.total = n;
    R.rel = 0.0;
    R.dtype = dtype;
    return cuda_status(launch_range(R, range_grid(n), (cudaStream_t)s));
}

}  // extern "C"

namespace {

cudaError_t launch_compress_heads_any(int lg, int dt, const Launch& P, unsigned grid,
                                      cudaStream_t s)
{
    switch (lg) {
    case 4: return launch_compress_heads_lg<4>(dt, P, grid, s);
    case 5: return launch_compress_heads_lg<5>(dt, P, grid, s);
    case 6: return launch_compress_heads_lg<6>(dt, P, grid, s);
    default: return launch_compress_heads_lg<7>(dt, P, grid, s);
    }
}

int compress_impl(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value,
                  int block, void* d_out, size_t out_cap, uint64_t* d_out_bytes, void* d_ws,
                  size_t ws_bytes, zc_stream_t s, bool heads)
{
    const int lg = log2_block(block);
    if (lg < 0 || !dtype_ok(dtype) || (n > 0 && d_in == nullptr) || d_out == nullptr ||
        !aligned(d_out, 16) || d_out_bytes == nullptr || !aligned(d_in, dtype == ZC_F32 ? 4 : 2))
        return ZC_ERR_ARG;
    if (eb_mode != ZC_EB_ABS && eb_mode != ZC_EB_REL) return ZC_ERR_ARG;
    if (!(eb_value > 0.0) || !std::isfinite(eb_value)) return ZC_ERR_ARG;
    const uint64_t nb = (n + (1ull << lg) - 1) >> lg;
    if (nb > 0xffffffffull) return ZC_ERR_ARG;
    // the heads (stored apart) are written straight to their place: all of
    // their area must fit
    if (out_cap < 32 + pad16(nb) + (heads ? pad16(3 * nb) : 0)) return ZC_ERR_CAPACITY;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    const int C = heads ? 8 : tile_chunks_for(n, n);
    const uint64_t tiles = tiles_for(n, unit_rows(C));
    if (tiles > w.cap || tiles > 0x7fffffffull) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    Item& it = P.one;
    it.x = d_in;
    it.out = (uint8_t*)d_out;
    it.out_bytes = (unsigned long long*)d_out_bytes;
    it.n = n;
    it.out_cap = out_cap;
    it.ntiles = (unsigned)tiles;
    it.x_dtype = dtype;
    it.out_dtype = dtype;
    if (eb_mode == ZC_EB_ABS) {
        st = qparams(eb_value, &it.eb, &it.two_eb, &it.inv);
        if (st) return st;
    } else {
        RangeLaunch R;
        std::memset(&R, 0, sizeof(R));
        R.ctl = w.ctl;
        R.partial = w.partial;
        R.one = RangeSeg{d_in, n};
        R.total = n;
        R.rel = eb_value;
        R.dtype = dtype;
        if (launch_range(R, range_grid(n), (cudaStream_t)s) != cudaSuccess) return ZC_ERR_CUDA;
        P.eb_from_ctl = 1;
    }
    P.n_items = 1;
    P.total_tiles = (unsigned)tiles;
    P.urows = unit_rows(C);
    if (heads) {
        const uint64_t grid = enc_grid(tiles, unit_rows(8), w);
        if (grid == 0) return ZC_ERR_WORKSPACE;
        return cuda_status(launch_compress_heads_any(lg, dtype, P, (unsigned)grid, (cudaStream_t)s));
    }
    const uint64_t grid = enc_grid(tiles, unit_rows(C), w);
    if (grid == 0) return ZC_ERR_WORKSPACE;
    return cuda_status(launch_compress_any(lg, C, dtype, P, (unsigned)grid, (cudaStream_t)s));
}

}  // namespace

extern "C" {

int zc_compress(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value, int block,
                void* d_out, size_t out_cap, uint64_t* d_out_bytes, void* d_ws, size_t ws_bytes,
                zc_stream_t s)
{
    return compress_impl(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes,
                         d_ws, ws_bytes, s, false);
}

int zc_compress_heads(const void* d_in, uint64_t n, int dtype, int eb_mode, double eb_value,
                      int block, void* d_out, size_t out_cap, uint64_t* d_out_bytes, void* d_ws,
                      size_t ws_bytes, zc_stream_t s)
{
    return compress_impl(d_in, n, dtype, eb_mode, eb_value, block, d_out, out_cap, d_out_bytes,
                         d_ws, ws_bytes, s, true);
}

size_t zc_max_compressed_bytes_heads(uint64_t n, int block)
{
    const int lg = log2_block(block);
    if (lg < 0) return 0;
    const uint64_t nb = (n + (1ull << lg) - 1) >> lg;
    return zc_max_compressed_bytes(n, block) + pad16(3 * nb);
}

int zc_decompress(const void* d_cmp, size_t cmp_cap, void* d_out, uint64_t n, int out_dtype,
                  void* d_ws, size_t ws_bytes, zc_stream_t s)
{
    if (d_cmp == nullptr || !aligned(d_cmp, 16) || cmp_cap < 32 || (n > 0 && d_out == nullptr) ||
        !dtype_ok(out_dtype) || !aligned(d_out, out_dtype == ZC_F32 ? 4 : 2))
        return ZC_ERR_ARG;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    const uint64_t tiles = tiles_for(n, DEC_U);
    const uint64_t chunks = chunks_for(tiles);
    if (tiles * NWARPS > w.cap || tiles > 0x7fffffffull) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    Item& it = P.one;
    it.cin = (const uint8_t*)d_cmp;
    it.cin_cap = cmp_cap;
    it.raw_out = d_out;
    it.n = n;
    it.ntiles = (unsigned)tiles;
    it.nchunks = (unsigned)chunks;
    it.out_dtype = out_dtype;
    P.n_items = 1;
    P.urows = DEC_U;
    P.total_tiles = (unsigned)chunks;
    if (launch_wscan(P, (unsigned)chunks, (cudaStream_t)s) != cudaSuccess) return ZC_ERR_CUDA;
    P.total_tiles = (unsigned)tiles;
    return cuda_status(launch_decompress(P, (unsigned)tiles, (cudaStream_t)s, true));
}

int zc_reduce_step(const void* d_cmp_in, size_t cmp_in_cap, const float* d_local, uint64_t n,
                   double eb_abs, int block, void* d_cmp_out, size_t out_cap,
                   uint64_t* d_out_bytes, float* d_sum_out, void* d_ws, size_t ws_bytes,
                   zc_stream_t s)
{
    const int lg = log2_block(block);
    if (lg < 0 || (n > 0 && d_local == nullptr) || !aligned(d_local, 4)) return ZC_ERR_ARG;
    if (d_cmp_out == nullptr && d_sum_out == nullptr) return ZC_ERR_ARG;
    if (d_cmp_in != nullptr && (!aligned(d_cmp_in, 16) || cmp_in_cap < 32)) return ZC_ERR_ARG;
    if (d_cmp_out != nullptr && (!aligned(d_cmp_out, 16) || d_out_bytes == nullptr))
        return ZC_ERR_ARG;
    if (!aligned(d_sum_out, 4)) return ZC_ERR_ARG;
    const uint64_t nb = (n + (1ull << lg) - 1) >> lg;
    if (d_cmp_out != nullptr && out_cap < 32 + pad16(nb)) return ZC_ERR_CAPACITY;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    const int C = tile_chunks_for(n, n);
    const uint64_t tiles = tiles_for(n, unit_rows(C));
    const uint64_t chunks = chunks_for(tiles);
    if (tiles * NWARPS > w.cap || tiles > 0x7fffffffull) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    Item& it = P.one;
    st = qparams(eb_abs, &it.eb, &it.two_eb, &it.inv);
    if (st) return st;
    it.x = d_local;
    it.cin = (const uint8_t*)d_cmp_in;
    it.cin_cap = cmp_in_cap;
    it.out = (uint8_t*)d_cmp_out;
    it.out_cap = out_cap;
    it.out_bytes = (unsigned long long*)d_out_bytes;
    it.raw_out = d_sum_out;
    it.n = n;
    it.ntiles = (unsigned)tiles;
    it.nchunks = (unsigned)chunks;
    it.x_dtype = ZC_F32;
    it.out_dtype = ZC_F32;
    P.n_items = 1;
    P.urows = unit_rows(C);
    if (d_cmp_in != nullptr) {
        P.total_tiles = (unsigned)chunks;
        if (launch_wscan(P, (unsigned)chunks, (cudaStream_t)s) != cudaSuccess) return ZC_ERR_CUDA;
    }
    P.total_tiles = (unsigned)tiles;
    const uint64_t grid = enc_grid(tiles, unit_rows(C), w);
    if (grid == 0) return ZC_ERR_WORKSPACE;
    return cuda_status(launch_reduce_any(lg, C, P, (unsigned)grid, (cudaStream_t)s));
}

size_t zc_plan_table_bytes(int n_items)
{
    return n_items > 0 ? sizeof(Item) * (size_t)n_items : 0;
}

int zc_plan_reduce(zc_plan* plan, int P, const zc_reduce_item* h_items, double eb_abs, int block,
                   void* d_table, size_t table_bytes)
{
    const int lg = log2_block(block);
    if (plan == nullptr || P < 1 || h_items == nullptr || lg < 0 || d_table == nullptr ||
        !aligned(d_table, 16) || table_bytes < zc_plan_table_bytes(P))
        return ZC_ERR_ARG;
    float eb, two, inv;
    int st = qparams(eb_abs, &eb, &two, &inv);
    if (st) return st;
    uint64_t total_n = 0;
    for (int r = 0; r < P; ++r) total_n += h_items[r].n;
    const int C = tile_chunks_for(total_n, total_n / (uint64_t)P);
    std::vector<Item> items((size_t)P);
    uint64_t tile = 0, chunk = 0;
    int has_cin = 0;
    for (int r = 0; r < P; ++r) {
        const zc_reduce_item& h = h_items[r];
        const uint64_t nb = (h.n + (1ull << lg) - 1) >> lg;
        if ((h.n > 0 && h.local == nullptr) || (h.cmp_out == nullptr && h.sum_out == nullptr))
            return ZC_ERR_ARG;
        if (h.cmp_in != nullptr && (!aligned(h.cmp_in, 16) || h.cmp_in_cap < 32)) return ZC_ERR_ARG;
        if (h.cmp_out != nullptr && (!aligned(h.cmp_out, 16) || h.out_bytes == nullptr))
            return ZC_ERR_ARG;
        if (h.cmp_out != nullptr && h.out_cap < 32 + pad16(nb)) return ZC_ERR_CAPACITY;
        if (!aligned(h.local, 4) || !aligned(h.sum_out, 4)) return ZC_ERR_ARG;
        Item& it = items[r];
        std::memset(&it, 0, sizeof(it));
        it.x = h.local;
        it.cin = (const uint8_t*)h.cmp_in;
        it.cin_cap = h.cmp_in_cap;
        it.out = (uint8_t*)h.cmp_out;
        it.out_cap = h.out_cap;
        it.out_bytes = (unsigned long long*)h.out_bytes;
        it.raw_out = h.sum_out;
        it.n = h.n;
        it.eb = eb;
        it.two_eb = two;
        it.inv = inv;
        it.tile_begin = (unsigned)tile;
        it.ntiles = (unsigned)tiles_for(h.n, unit_rows(C));
        it.chunk_begin = (unsigned)chunk;
        it.nchunks = (unsigned)chunks_for(it.ntiles);
        it.x_dtype = ZC_F32;
        it.out_dtype = ZC_F32;
        tile += it.ntiles;
        chunk += it.nchunks;
        has_cin |= h.cmp_in != nullptr;
    }
    if (tile > 0x7fffffffull) return ZC_ERR_ARG;
    if (cudaMemcpy(d_table, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return ZC_ERR_CUDA;
    plan->n_items = P;
    plan->tile_chunks = C;
    plan->block = block;
    plan->has_input = has_cin;
    plan->total_tiles = tile;
    plan->total_chunks = chunk;
    plan->d_table = d_table;
    return ZC_OK;
}

int zc_reduce_step_batch(const zc_plan* plan, void* d_ws, size_t ws_bytes, zc_stream_t s)
{
    if (plan == nullptr || plan->d_table == nullptr || plan->n_items < 1) return ZC_ERR_ARG;
    const int lg = log2_block(plan->block);
    if (lg < 0) return ZC_ERR_ARG;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    const int C = plan->tile_chunks;
    if (plan->total_tiles * NWARPS > w.cap || plan->total_chunks > w.cap) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    P.items = (const Item*)plan->d_table;
    P.n_items = (unsigned)plan->n_items;
    P.urows = unit_rows(C);
    if (plan->has_input) {
        P.total_tiles = (unsigned)plan->total_chunks;
        if (plan->n_items >= CHUNK_MAP_ITEMS) {
            // chunk -> item map for the width scan (the tile map below reuses its space)
            if (launch_tile_map(P.items, P.n_items, P.total_tiles, w.tile_map, (cudaStream_t)s,
                                true) != cudaSuccess)
                return ZC_ERR_CUDA;
            P.tile_map = w.tile_map;
        }
        if (launch_wscan(P, (unsigned)plan->total_chunks, (cudaStream_t)s) != cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = nullptr;
    }
    P.total_tiles = (unsigned)plan->total_tiles;
    const uint64_t grid = enc_grid(plan->total_tiles, unit_rows(C), w);
    if (grid == 0) return ZC_ERR_WORKSPACE;
    // each launch of the step is dependent on the one before it: the tile
    // map is built while the width scan runs, the fused kernel's CTAs become
    // resident while the map finishes (both wait for their inputs)
    if (plan->n_items > 1) {
        if (launch_tile_map(P.items, P.n_items, P.total_tiles, w.tile_map, (cudaStream_t)s,
                            false, plan->has_input != 0) != cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = w.tile_map;
        P.dep = 1;
    } else {
        P.dep = plan->has_input != 0;
    }
    return cuda_status(launch_reduce_any(lg, C, P, (unsigned)grid, (cudaStream_t)s));
}

int zc_scatter_pack(const void* d_in, int dtype, int P, const uint64_t* h_counts,
                    const uint64_t* h_displs, int eb_mode, double eb_value, int block,
                    void* d_out, size_t out_cap, uint64_t* d_seg_off, void* d_ws,
                    size_t ws_bytes, zc_stream_t s)
{
    const int lg = log2_block(block);
    if (lg < 0 || !dtype_ok(dtype) || P < 1 || P > SCATTER_MAX || h_counts == nullptr ||
        h_displs == nullptr || d_out == nullptr || !aligned(d_out, 16) || d_seg_off == nullptr ||
        !aligned(d_in, dtype == ZC_F32 ? 4 : 2))
        return ZC_ERR_ARG;
    if (eb_mode != ZC_EB_ABS && eb_mode != ZC_EB_REL) return ZC_ERR_ARG;
    if (!(eb_value > 0.0) || !std::isfinite(eb_value)) return ZC_ERR_ARG;
    WsView w;
    int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    uint64_t all_n = 0;
    for (int p = 0; p < P; ++p) all_n += h_counts[p];
    const int C = tile_chunks_for(all_n, all_n / (uint64_t)P);
    thread_local static ScatterParams SP;  // host staging of the by-value parameter block
    uint64_t tile = 0, total_n = 0, min_cap = 0;
    std::vector<const void*> ptrs((size_t)P);
    std::vector<unsigned long long> cnts((size_t)P);
    const uint64_t es = dtype == ZC_F32 ? 4 : 2;
    for (int p = 0; p < P; ++p) {
        if (h_counts[p] > 0 && d_in == nullptr) return ZC_ERR_ARG;
        const uint64_t nb = (h_counts[p] + (1ull << lg) - 1) >> lg;
        if (nb > 0xffffffffull) return ZC_ERR_ARG;
        SP.tile_begin[p] = (unsigned)tile;
        SP.displ[p] = h_displs[p];
        SP.count[p] = h_counts[p];
        tile += tiles_for(h_counts[p], unit_rows(C));
        total_n += h_counts[p];
        min_cap += 32 + pad16(nb);
        ptrs[p] = (const uint8_t*)d_in + h_displs[p] * es;
        cnts[p] = h_counts[p];
    }
    SP.tile_begin[P] = (unsigned)tile;
    if (out_cap < min_cap) return ZC_ERR_CAPACITY;
    if (tile > w.cap || (uint64_t)P + 1 > w.cap || tile > 0x7fffffffull) return ZC_ERR_WORKSPACE;
    Launch L = base_launch(w);
    Item& it = L.one;
    it.x = d_in;
    it.out = (uint8_t*)d_out;
    it.out_cap = out_cap;
    it.x_dtype = dtype;
    it.out_dtype = dtype;
    if (eb_mode == ZC_EB_ABS) {
        st = qparams(eb_value, &it.eb, &it.two_eb, &it.inv);
        if (st) return st;
    } else {
        RangeLaunch R;
        std::memset(&R, 0, sizeof(R));
        R.ctl = w.ctl;
        R.partial = w.partial;
        R.total = total_n;
        R.rel = eb_value;
        R.dtype = dtype;
        if (launch_range_multi(R, ptrs.data(), cnts.data(), (unsigned)P, range_grid(total_n),
                               (cudaStream_t)s) != cudaSuccess)
            return ZC_ERR_CUDA;
        L.eb_from_ctl = 1;
    }
    L.packed = 1;
    L.seg_off = (unsigned long long*)d_seg_off;
    L.n_items = (unsigned)P;
    L.total_tiles = (unsigned)tile;
    L.urows = unit_rows(C);
    const uint64_t grid = enc_grid(tile, unit_rows(C), w);
    if (grid == 0) return ZC_ERR_WORKSPACE;
    return cuda_status(launch_scatter_any(lg, C, dtype, L, SP, (unsigned)grid, (cudaStream_t)s));
}

size_t zc_batch_table_bytes(int n_msgs)
{
    return n_msgs > 0 ? sizeof(Item) * (size_t)n_msgs : 0;
}

size_t zc_batch_max_bytes(int n_msgs, const zc_message* h_msgs)
{
    if (n_msgs < 1 || h_msgs == nullptr) return 0;
    size_t total = 0;
    for (int i = 0; i < n_msgs; ++i) {
        const zc_message& m = h_msgs[i];
        const size_t b = m.block == ZC_RAW ? zc_raw_stream_bytes(m.n, m.dtype)
                                           : zc_max_compressed_bytes(m.n, m.block);
        if (b == 0) return 0;
        total += b;
    }
    return total;
}

int zc_plan_compress_batch(zc_batch* plan, int n_msgs, const zc_message* h_msgs, int tile_chunks,
                           int grid, void* d_packed, size_t packed_cap, uint64_t* d_msg_off,
                           void* d_table, size_t table_bytes)
{
    if (plan == nullptr || n_msgs < 1 || h_msgs == nullptr || grid < 0 || d_packed == nullptr ||
        !aligned(d_packed, 16) || d_msg_off == nullptr || !aligned(d_msg_off, 8) ||
        d_table == nullptr || !aligned(d_table, 16) || table_bytes < zc_batch_table_bytes(n_msgs))
        return ZC_ERR_ARG;
    uint64_t all_n = 0;
    for (int i = 0; i < n_msgs; ++i) all_n += h_msgs[i].n;
    const int C = tile_chunks ? tile_chunks : tile_chunks_for(all_n, all_n / (uint64_t)n_msgs);
    if (C != 4 && C != 8 && C != 16) return ZC_ERR_ARG;
    std::vector<Item> items((size_t)n_msgs);
    uint64_t tile = 0, min_cap = 0;
    for (int i = 0; i < n_msgs; ++i) {
        const zc_message& m = h_msgs[i];
        if (!dtype_ok(m.dtype) || (m.n > 0 && m.in == nullptr) || !aligned(m.in, elem_bytes(m.dtype)))
            return ZC_ERR_ARG;
        Item& it = items[(size_t)i];
        std::memset(&it, 0, sizeof(it));
        if (m.block == ZC_RAW) {
            it.log2L = -1;
            min_cap += 32 + pad16(m.n * elem_bytes(m.dtype));
        } else {
            it.log2L = log2_block(m.block);
            if (it.log2L < 0) return ZC_ERR_ARG;
            const uint64_t nb = (m.n + (1ull << it.log2L) - 1) >> it.log2L;
            if (nb > 0xffffffffull) return ZC_ERR_ARG;
            const int st = qparams(m.eb_abs, &it.eb, &it.two_eb, &it.inv);
            if (st) return st;
            min_cap += 32 + pad16(nb);
        }
        it.x = m.in;
        it.out = (uint8_t*)d_packed;
        it.out_cap = packed_cap;
        it.n = m.n;
        it.tile_begin = (unsigned)tile;
        it.ntiles = (unsigned)tiles_for(m.n, unit_rows(C));
        it.x_dtype = m.dtype;
        it.out_dtype = m.dtype;
        tile += it.ntiles;
        if (tile > 0x7fffffffull) return ZC_ERR_ARG;
    }
    if (packed_cap < min_cap) return ZC_ERR_CAPACITY;
    if (cudaMemcpy(d_table, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return ZC_ERR_CUDA;
    std::memset(plan, 0, sizeof(*plan));
    plan->n_msgs = n_msgs;
    plan->tile_chunks = C;
    plan->grid = grid;
    plan->decompress = 0;
    plan->total_tiles = tile;
    plan->d_table = d_table;
    plan->d_packed = d_packed;
    plan->packed_cap = packed_cap;
    plan->d_msg_off = d_msg_off;
    return ZC_OK;
}

int zc_compress_batch(const zc_batch* plan, void* d_ws, size_t ws_bytes, zc_stream_t s)
{
    if (plan == nullptr || plan->d_table == nullptr || plan->n_msgs < 1 || plan->decompress != 0)
        return ZC_ERR_ARG;
    const int C = plan->tile_chunks;
    if (C != 4 && C != 8 && C != 16) return ZC_ERR_ARG;
    WsView w;
    const int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    if (plan->total_tiles > w.cap || (uint64_t)plan->n_msgs + 1 > w.cap) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    P.items = (const Item*)plan->d_table;
    P.n_items = (unsigned)plan->n_msgs;
    P.packed = 1;
    P.seg_off = (unsigned long long*)plan->d_msg_off;
    P.urows = unit_rows(C);
    P.total_tiles = (unsigned)plan->total_tiles;
    uint64_t grid = plan->grid > 0 ? (uint64_t)plan->grid : plan->total_tiles;
    if (grid > plan->total_tiles) grid = plan->total_tiles;
    grid = enc_grid(grid, unit_rows(C), w);
    if (grid == 0) return ZC_ERR_WORKSPACE;
    if (plan->grouped) {
        // first tickets by block size, rewritten on the device from the table's
        // current block sizes (a selection made earlier on this stream included);
        // the per-CTA class sums use the decoder offsets' array, idle here
        if ((uint64_t)((plan->n_msgs + 255) / 256) * 5 > 2 * w.cap) return ZC_ERR_WORKSPACE;
        if (launch_group((Item*)plan->d_table, P.n_items, (unsigned*)w.offs, w.tile_map,
                         (cudaStream_t)s) != cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = w.tile_map;
        P.grouped = 1;
    } else if (plan->n_msgs > 1) {
        if (launch_tile_map(P.items, P.n_items, P.total_tiles, w.tile_map, (cudaStream_t)s) !=
            cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = w.tile_map;
    }
    return cuda_status(launch_batch(C, P, (unsigned)grid, (cudaStream_t)s));
}

int zc_plan_decompress_batch(zc_batch* plan, int n_msgs, const zc_message* h_msgs,
                             const void* d_packed, size_t packed_cap, const uint64_t* d_msg_off,
                             void* d_table, size_t table_bytes)
{
    if (plan == nullptr || n_msgs < 1 || h_msgs == nullptr || d_packed == nullptr ||
        !aligned(d_packed, 16) || d_msg_off == nullptr || !aligned(d_msg_off, 8) ||
        d_table == nullptr || !aligned(d_table, 16) || table_bytes < zc_batch_table_bytes(n_msgs))
        return ZC_ERR_ARG;
    std::vector<Item> items((size_t)n_msgs);
    uint64_t tile = 0, chunk = 0;
    for (int i = 0; i < n_msgs; ++i) {
        const zc_message& m = h_msgs[i];
        if (!dtype_ok(m.dtype) || (m.n > 0 && m.out == nullptr) ||
            !aligned(m.out, elem_bytes(m.dtype)))
            return ZC_ERR_ARG;
        Item& it = items[(size_t)i];
        std::memset(&it, 0, sizeof(it));
        it.cin = (const uint8_t*)d_packed;  // the kernels read the stream's start from d_msg_off
        it.raw_out = m.out;
        it.n = m.n;
        it.tile_begin = (unsigned)tile;
        it.ntiles = (unsigned)tiles_for(m.n, DEC_U);
        it.chunk_begin = (unsigned)chunk;
        it.nchunks = it.ntiles <= DEC_LOCAL_TILES ? 0u : (unsigned)chunks_for(it.ntiles);
        it.x_dtype = m.dtype;
        it.out_dtype = m.dtype;
        tile += it.ntiles;
        chunk += it.nchunks;
        if (tile > 0x7fffffffull) return ZC_ERR_ARG;
    }
    if (cudaMemcpy(d_table, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return ZC_ERR_CUDA;
    std::memset(plan, 0, sizeof(*plan));
    plan->n_msgs = n_msgs;
    plan->tile_chunks = 0;
    plan->grid = 0;
    plan->decompress = 1;
    plan->total_tiles = tile;
    plan->total_chunks = chunk;
    plan->d_table = d_table;
    plan->d_packed = const_cast<void*>(d_packed);
    plan->packed_cap = packed_cap;
    plan->d_msg_off = const_cast<uint64_t*>(d_msg_off);
    return ZC_OK;
}

int zc_plan_decompress_streams(zc_batch* plan, int n_msgs, const void* const* h_streams,
                               const uint64_t* h_caps, const zc_message* h_msgs, void* d_table,
                               size_t table_bytes)
{
    if (plan == nullptr || n_msgs < 1 || h_streams == nullptr || h_caps == nullptr ||
        h_msgs == nullptr || d_table == nullptr || !aligned(d_table, 16) ||
        table_bytes < zc_batch_table_bytes(n_msgs))
        return ZC_ERR_ARG;
    std::vector<Item> items((size_t)n_msgs);
    uint64_t tile = 0, chunk = 0;
    for (int i = 0; i < n_msgs; ++i) {
        const zc_message& m = h_msgs[i];
        if (!dtype_ok(m.dtype) || (m.n > 0 && m.out == nullptr) ||
            !aligned(m.out, elem_bytes(m.dtype)) || h_streams[i] == nullptr ||
            !aligned(h_streams[i], 16) || h_caps[i] < 32)
            return ZC_ERR_ARG;
        Item& it = items[(size_t)i];
        std::memset(&it, 0, sizeof(it));
        it.cin = (const uint8_t*)h_streams[i];
        it.cin_cap = h_caps[i];
        it.raw_out = m.out;
        it.n = m.n;
        it.tile_begin = (unsigned)tile;
        it.ntiles = (unsigned)tiles_for(m.n, DEC_U);
        it.chunk_begin = (unsigned)chunk;
        it.nchunks = it.ntiles <= DEC_LOCAL_TILES ? 0u : (unsigned)chunks_for(it.ntiles);
        it.x_dtype = m.dtype;
        it.out_dtype = m.dtype;
        tile += it.ntiles;
        chunk += it.nchunks;
        if (tile > 0x7fffffffull) return ZC_ERR_ARG;
    }
    if (cudaMemcpy(d_table, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice) !=
        cudaSuccess)
        return ZC_ERR_CUDA;
    std::memset(plan, 0, sizeof(*plan));
    plan->n_msgs = n_msgs;
    plan->decompress = 1;
    plan->total_tiles = tile;
    plan->total_chunks = chunk;
    plan->d_table = d_table;
    return ZC_OK;
}

int zc_decompress_batch(const zc_batch* plan, void* d_ws, size_t ws_bytes, zc_stream_t s)
{
    if (plan == nullptr || plan->d_table == nullptr || plan->n_msgs < 1 || plan->decompress != 1)
        return ZC_ERR_ARG;
    WsView w;
    const int st = ws_view(d_ws, ws_bytes, w);
    if (st) return st;
    if (plan->total_tiles * NWARPS > w.cap || plan->total_chunks > w.cap) return ZC_ERR_WORKSPACE;
    Launch P = base_launch(w);
    P.items = (const Item*)plan->d_table;
    P.n_items = (unsigned)plan->n_msgs;
    P.urows = DEC_U;
    P.in_base = (const uint8_t*)plan->d_packed;
    P.in_off = (const unsigned long long*)plan->d_msg_off;
    P.in_cap = plan->packed_cap;
    P.grouped = plan->grouped;
    P.total_tiles = (unsigned)plan->total_chunks;
    if (plan->total_chunks > 0) {  // none when every item is small (offsets found by the decoder)
        if (plan->n_msgs >= CHUNK_MAP_ITEMS) {
            // chunk -> item map for the width scan (the tile map below reuses its space)
            if (launch_tile_map(P.items, P.n_items, P.total_tiles, w.tile_map, (cudaStream_t)s,
                                true) != cudaSuccess)
                return ZC_ERR_CUDA;
            P.tile_map = w.tile_map;
        }
        if (launch_wscan(P, (unsigned)plan->total_chunks, (cudaStream_t)s) != cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = nullptr;
    }
    P.total_tiles = (unsigned)plan->total_tiles;
    if (plan->n_msgs > 1) {
        if (launch_tile_map(P.items, P.n_items, P.total_tiles, w.tile_map, (cudaStream_t)s) !=
            cudaSuccess)
            return ZC_ERR_CUDA;
        P.tile_map = w.tile_map;
    }
    return cuda_status(launch_decompress(P, (unsigned)plan->total_tiles, (cudaStream_t)s));
}

int zc_batch_set_grouped(zc_batch* plan, int grouped)
{
    if (plan == nullptr || (grouped != 0 && grouped != 1)) return ZC_ERR_ARG;
    if (grouped && plan->decompress == 1 && plan->d_msg_off == nullptr) return ZC_ERR_ARG;
    plan->grouped = grouped;
    return ZC_OK;
}

int zc_get_device_status(const void* d_ws, zc_stream_t s, int* status, uint64_t* detail)
{
    if (d_ws == nullptr || status == nullptr) return ZC_ERR_ARG;
    Ctl c;
    if (cudaMemcpyAsync(&c, d_ws, sizeof(Ctl), cudaMemcpyDeviceToHost, (cudaStream_t)s) != cudaSuccess)
        return ZC_ERR_CUDA;
    if (cudaStreamSynchronize((cudaStream_t)s) != cudaSuccess) return ZC_ERR_CUDA;
    *status = (int)c.status;
    if (detail) *detail = c.detail;
    return ZC_OK;
}

int zc_clear_device_status(void* d_ws, zc_stream_t s)
{
    if (d_ws == nullptr) return ZC_ERR_ARG;
    return cudaMemsetAsync(d_ws, 0, 4, (cudaStream_t)s) == cudaSuccess ? ZC_OK : ZC_ERR_CUDA;
}

void zc_set_wait_limit_ns(uint64_t ns) { g_wait_ns = ns ? ns : 1; }

void zc_debug_withhold_tile(int64_t tile) { g_withhold = tile; }

int zc_set_tile_chunks(int chunks)
{
    if (chunks != 0 && chunks != 4 && chunks != 8 && chunks != 16) return ZC_ERR_ARG;
    g_chunks = chunks;
    return ZC_OK;
}

}  // extern "C"
