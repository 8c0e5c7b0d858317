// zc_k32.cu -- compress and ring-step kernels at block size L = 32.
#include "zc_launch.h"

namespace zc {

template <int R>
static cudaError_t compress_rows(int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    if (x_dtype == ZC_F32) k_compress<5, R, float><<<grid, NTHREADS, 0, s>>>(P);
    else k_compress<5, R, uint16_t><<<grid, NTHREADS, 0, s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_compress_l32(int rows, int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (rows) {
    case 4: return compress_rows<4>(x_dtype, P, grid, s);
    case 8: return compress_rows<8>(x_dtype, P, grid, s);
    case 16: return compress_rows<16>(x_dtype, P, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_reduce_l32(int rows, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (rows) {
    case 4: k_reduce<5, 4><<<grid, NTHREADS, 0, s>>>(P); break;
    case 8: k_reduce<5, 8><<<grid, NTHREADS, 0, s>>>(P); break;
    case 16: k_reduce<5, 16><<<grid, NTHREADS, 0, s>>>(P); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int R>
static cudaError_t scatter_rows(int x_dtype, const Launch& P, const ScatterParams& S, unsigned grid,
                                cudaStream_t s)
{
    if (x_dtype == ZC_F32) k_scatter<5, R, float><<<grid, NTHREADS, 0, s>>>(P, S);
    else k_scatter<5, R, uint16_t><<<grid, NTHREADS, 0, s>>>(P, S);
    return cudaGetLastError();
}

cudaError_t launch_scatter_l32(int rows, int x_dtype, const Launch& P, const ScatterParams& S,
                               unsigned grid, cudaStream_t s)
{
    switch (rows) {
    case 4: return scatter_rows<4>(x_dtype, P, S, grid, s);
    case 8: return scatter_rows<8>(x_dtype, P, S, grid, s);
    case 16: return scatter_rows<16>(x_dtype, P, S, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace zc
