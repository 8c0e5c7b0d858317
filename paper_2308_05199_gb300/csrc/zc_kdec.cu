// zc_kdec.cu -- width scan (decode-tile offsets) and decompression kernels.
#define ZC_DECODE_KERNELS
#include "zc_launch.h"

namespace zc {

cudaError_t launch_wscan(const Launch& P, unsigned grid, cudaStream_t s)
{
    k_wscan<<<grid, NTHREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_tile_map(const Item* items, unsigned n_items, unsigned total_tiles,
                            unsigned* map, cudaStream_t s, bool by_chunk, bool dependent)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((total_tiles + NTHREADS - 1) / NTHREADS);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = dependent ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k_tile_map, items, n_items, total_tiles, map,
                              by_chunk ? 1 : 0);
}

cudaError_t launch_group(Item* items, unsigned n_items, unsigned* part, unsigned* map,
                         cudaStream_t s)
{
    const unsigned nblk = (n_items + GROUP_T - 1) / GROUP_T;
    k_group_count<<<nblk, GROUP_T, 0, s>>>(items, n_items, part);
    k_group_scan<<<1, 1024, 0, s>>>(part, nblk);
    k_group_place<<<nblk, GROUP_T, 0, s>>>(items, n_items, part, map);
    return cudaGetLastError();
}

cudaError_t launch_decompress(const Launch& P, unsigned grid, cudaStream_t s, bool after_wscan)
{
    if (P.items != nullptr) {
        k_decompress<true><<<grid, NTHREADS, 0, s>>>(P);
        return cudaGetLastError();
    }
    if (!after_wscan) {
        k_decompress<false><<<grid, NTHREADS, 0, s>>>(P);
        return cudaGetLastError();
    }
    // launched dependent on the width scan just before it on the stream: its
    // CTAs read their headers and width bytes while the scan still runs
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(NTHREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_decompress<false>, P);
}

}  // namespace zc
