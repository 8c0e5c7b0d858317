// zc_kdec.cu -- decompression kernels (block size read from each stream).
#include "zc_launch.h"

namespace zc {

cudaError_t launch_decompress(int rows, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (rows) {
    case 4: k_decompress<4><<<grid, NTHREADS, 0, s>>>(P); break;
    case 8: k_decompress<8><<<grid, NTHREADS, 0, s>>>(P); break;
    case 16: k_decompress<16><<<grid, NTHREADS, 0, s>>>(P); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace zc
