// zc_launch.h -- host-side launch entry points of the kernel translation units.
#pragma once

#include <atomic>

#include "zc_codec.cuh"

namespace zc {

// Raises kernel K's dynamic shared-memory limit to `bytes` on the current
// device, once per device: the attribute belongs to the device's context, so
// a process that drives several GPUs sets it on each of them.
template <auto K>
inline cudaError_t smem_limit(int bytes)
{
    static std::atomic<unsigned long long> done{0ull};  // bit d: set on device d
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = (dev >= 0 && dev < 64) ? 1ull << dev : 0ull;
    if (bit != 0ull && (done.load(std::memory_order_acquire) & bit) != 0ull) return cudaSuccess;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
    return e;
}

// Launchers of the encoder kernels at block size 2^LG; each is defined and
// explicitly instantiated by the object of zc_kenc.cu built for that LG.
// `chunks` is the tile size in 2048-element chunks (4, 8 or 16); these pick
// the kernel instantiation at run time.
template <int LG>
cudaError_t launch_compress_lg(int chunks, int x_dtype, const Launch& P, unsigned grid,
                               cudaStream_t s);
template <int LG>
cudaError_t launch_compress_heads_lg(int x_dtype, const Launch& P, unsigned grid, cudaStream_t s);
template <int LG>
cudaError_t launch_reduce_lg(int chunks, const Launch& P, unsigned grid, cudaStream_t s);
template <int LG>
cudaError_t launch_scatter_lg(int chunks, int x_dtype, const Launch& P, const ScatterParams& SP,
                              unsigned grid, cudaStream_t s);
// Batched compression with warp units of U rows (defined per U by zc_kbatch.cu).
template <int U>
cudaError_t launch_batch_u(const Launch& P, unsigned grid, cudaStream_t s);

cudaError_t launch_wscan(const Launch& P, unsigned grid, cudaStream_t s);
// after_wscan (single streams): the width scan was the launch just before on
// `s`; the decoder is launched dependent on it (programmatic serialisation).
cudaError_t launch_decompress(const Launch& P, unsigned grid, cudaStream_t s,
                              bool after_wscan = false);
// Item of every tile (by_chunk: of every width-scan chunk) of a multi-item
// launch; `dependent`: launched dependent on the width scan just before it.
cudaError_t launch_tile_map(const Item* items, unsigned n_items, unsigned total_tiles,
                            unsigned* map, cudaStream_t s, bool by_chunk = false,
                            bool dependent = false);
// Grouped batches: first tickets of every item by block size (rewrites the
// items' tile_begin) and the ticket -> item map; `part` holds 5 u32 per 256 items.
cudaError_t launch_group(Item* items, unsigned n_items, unsigned* part, unsigned* map,
                         cudaStream_t s);

// Range: extremes of the listed segments, then (rel > 0) the bound they imply.
struct RangeSeg {
    const void* x;
    unsigned long long n;
};
constexpr int RANGE_MAX_SEGS = 1024;
struct RangeLaunch {
    Ctl* ctl;
    float2* partial;        // RANGE_SLOTS slots
    float* minmax_out;      // optional: device float[2]
    RangeSeg one;           // the input (single-segment launches)
    unsigned n_segs;
    unsigned long long total;
    double rel;             // > 0: resolve eb = rel * range into ctl
    int dtype;
};
cudaError_t launch_range(const RangeLaunch& R, unsigned grid, cudaStream_t s);
cudaError_t launch_range_multi(const RangeLaunch& R, const void* const* ptrs,
                               const unsigned long long* counts, unsigned nseg, unsigned grid,
                               cudaStream_t s);
cudaError_t launch_ws_init(Ctl* ctl, cudaStream_t s);

}  // namespace zc
