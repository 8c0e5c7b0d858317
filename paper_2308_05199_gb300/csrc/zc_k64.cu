// zc_k64.cu -- encoder kernels (compress, scatter pack, ring step) at L = 64.
#include "zc_launch.h"

namespace zc {

template <int U>
static cudaError_t compress_u(int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    const cudaError_t e32 = smem_limit<k_compress<6, U, float>>(enc_smem_bytes(U, true));
    const cudaError_t e16 = smem_limit<k_compress<6, U, uint16_t>>(enc_smem_bytes(U, true));
    if (e32 != cudaSuccess || e16 != cudaSuccess) return e32 != cudaSuccess ? e32 : e16;
    if (x_dtype == ZC_F32) k_compress<6, U, float><<<grid, ENC_THREADS, enc_smem_bytes(U, true), s>>>(P);
    else k_compress<6, U, uint16_t><<<grid, ENC_THREADS, enc_smem_bytes(U, true), s>>>(P);
    return cudaGetLastError();
}

// Block heads stored apart: 8-chunk tiles (64-row warp units) only.
cudaError_t launch_compress_heads_l64(int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    const cudaError_t e32 = smem_limit<k_compress<6, 64, float, true>>(enc_smem_bytes(64, true));
    const cudaError_t e16 = smem_limit<k_compress<6, 64, uint16_t, true>>(enc_smem_bytes(64, true));
    if (e32 != cudaSuccess || e16 != cudaSuccess) return e32 != cudaSuccess ? e32 : e16;
    if (x_dtype == ZC_F32)
        k_compress<6, 64, float, true><<<grid, ENC_THREADS, enc_smem_bytes(64, true), s>>>(P);
    else
        k_compress<6, 64, uint16_t, true><<<grid, ENC_THREADS, enc_smem_bytes(64, true), s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_compress_l64(int chunks, int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (chunks) {
    case 4: return compress_u<32>(x_dtype, P, grid, s);
    case 8: return compress_u<64>(x_dtype, P, grid, s);
    case 16: return compress_u<128>(x_dtype, P, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int U>
static cudaError_t scatter_u(int x_dtype, const Launch& P, const ScatterParams& SP, unsigned grid,
                             cudaStream_t s)
{
    const cudaError_t e32 = smem_limit<k_scatter<6, U, float>>(enc_smem_bytes(U, true));
    const cudaError_t e16 = smem_limit<k_scatter<6, U, uint16_t>>(enc_smem_bytes(U, true));
    if (e32 != cudaSuccess || e16 != cudaSuccess) return e32 != cudaSuccess ? e32 : e16;
    if (x_dtype == ZC_F32) k_scatter<6, U, float><<<grid, ENC_THREADS, enc_smem_bytes(U, true), s>>>(P, SP);
    else k_scatter<6, U, uint16_t><<<grid, ENC_THREADS, enc_smem_bytes(U, true), s>>>(P, SP);
    return cudaGetLastError();
}

cudaError_t launch_scatter_l64(int chunks, int x_dtype, const Launch& P, const ScatterParams& SP,
                               unsigned grid, cudaStream_t s)
{
    switch (chunks) {
    case 4: return scatter_u<32>(x_dtype, P, SP, grid, s);
    case 8: return scatter_u<64>(x_dtype, P, SP, grid, s);
    case 16: return scatter_u<128>(x_dtype, P, SP, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int U>
static cudaError_t reduce_u(const Launch& P, unsigned grid, cudaStream_t s)
{
    const cudaError_t e = smem_limit<k_reduce<6, U>>(enc_smem_bytes(U));
    if (e != cudaSuccess) return e;
    k_reduce<6, U><<<grid, ENC_THREADS, enc_smem_bytes(U), s>>>(P);
    return cudaGetLastError();
}

cudaError_t launch_reduce_l64(int chunks, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (chunks) {
    case 4: return reduce_u<32>(P, grid, s);
    case 8: return reduce_u<64>(P, grid, s);
    case 16: return reduce_u<128>(P, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace zc
