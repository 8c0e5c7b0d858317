// zc_kbatch.cu -- launcher of the batched compression kernel at one tile
// size.  The build compiles this file once per warp-unit size with
// -DZC_BATCH_U=32, 64 or 128 (tiles of 4, 8 or 16 chunks of 2048 elements),
// so the three instantiations compile in parallel.
#include "zc_launch.h"

#ifndef ZC_BATCH_U
#error "zc_kbatch.cu is compiled once per tile size, with -DZC_BATCH_U=32, 64 or 128"
#endif

namespace zc {

template <int U>
cudaError_t launch_batch_u(const Launch& P, unsigned grid, cudaStream_t s)
{
    const cudaError_t e = smem_limit<k_batch<U>>(enc_smem_bytes(U));
    if (e != cudaSuccess) return e;
    k_batch<U><<<grid, ENC_THREADS, enc_smem_bytes(U), s>>>(P);
    return cudaGetLastError();
}

template cudaError_t launch_batch_u<ZC_BATCH_U>(const Launch&, unsigned, cudaStream_t);

}  // namespace zc
