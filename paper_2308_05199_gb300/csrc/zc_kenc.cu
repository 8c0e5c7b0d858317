// zc_kenc.cu -- launchers of the encoder kernels (compress, heads-apart
// compress, scatter pack, fused ring step) at one block size.  The build
// compiles this file once per block size with -DZC_LOG2L=4..7, so the four
// heavy kernel sets compile in parallel; each object explicitly instantiates
// the launchers of its block size.
#include "zc_launch.h"

#ifndef ZC_LOG2L
#error "zc_kenc.cu is compiled once per block size, with -DZC_LOG2L=4, 5, 6 or 7"
#endif

namespace zc {

// One encoder launch; `after_range`: the kernel this one waits for (the range
// kernel of a relative bound, the fused step's width scan or tile map) was
// the launch just before on `s`, and this one is launched dependent on it
// (programmatic serialisation): its CTAs become resident while that kernel
// finishes and wait for it in their prologue.
template <typename... A>
static cudaError_t launch_enc(void (*k)(A...), unsigned grid, int smem, cudaStream_t s,
                              bool after_range, const A&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(ENC_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = after_range ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <auto K, auto K16>
static cudaError_t launch_typed(int x_dtype, int smem, unsigned grid, cudaStream_t s,
                                const Launch& P)
{
    const cudaError_t e32 = smem_limit<K>(smem);
    const cudaError_t e16 = smem_limit<K16>(smem);
    if (e32 != cudaSuccess || e16 != cudaSuccess) return e32 != cudaSuccess ? e32 : e16;
    const bool after_range = P.eb_from_ctl != 0 || P.dep != 0;
    return x_dtype == ZC_F32 ? launch_enc(K, grid, smem, s, after_range, P)
                             : launch_enc(K16, grid, smem, s, after_range, P);
}

template <int LG>
cudaError_t launch_compress_lg(int chunks, int x_dtype, const Launch& P, unsigned grid,
                               cudaStream_t s)
{
    switch (chunks) {
    case 4:
        return launch_typed<k_compress<LG, 32, float>, k_compress<LG, 32, uint16_t>>(
            x_dtype, enc_smem_bytes(32, true), grid, s, P);
    case 8:
        return launch_typed<k_compress<LG, 64, float>, k_compress<LG, 64, uint16_t>>(
            x_dtype, enc_smem_bytes(64, true), grid, s, P);
    case 16:
        return launch_typed<k_compress<LG, 128, float>, k_compress<LG, 128, uint16_t>>(
            x_dtype, enc_smem_bytes(128, true), grid, s, P);
    default: return cudaErrorInvalidValue;
    }
}

// Block heads stored apart: 8-chunk tiles (64-row warp units) only.
template <int LG>
cudaError_t launch_compress_heads_lg(int x_dtype, const Launch& P, unsigned grid, cudaStream_t s)
{
    return launch_typed<k_compress<LG, 64, float, true>, k_compress<LG, 64, uint16_t, true>>(
        x_dtype, enc_smem_bytes(64, true), grid, s, P);
}

template <int LG, int U>
static cudaError_t scatter_u(int x_dtype, const Launch& P, const ScatterParams& SP, unsigned grid,
                             cudaStream_t s)
{
    const int smem = enc_smem_bytes(U, true);
    const cudaError_t e32 = smem_limit<k_scatter<LG, U, float>>(smem);
    const cudaError_t e16 = smem_limit<k_scatter<LG, U, uint16_t>>(smem);
    if (e32 != cudaSuccess || e16 != cudaSuccess) return e32 != cudaSuccess ? e32 : e16;
    const bool after_range = P.eb_from_ctl != 0 || P.dep != 0;
    return x_dtype == ZC_F32
               ? launch_enc(k_scatter<LG, U, float>, grid, smem, s, after_range, P, SP)
               : launch_enc(k_scatter<LG, U, uint16_t>, grid, smem, s, after_range, P, SP);
}

template <int LG>
cudaError_t launch_scatter_lg(int chunks, int x_dtype, const Launch& P, const ScatterParams& SP,
                              unsigned grid, cudaStream_t s)
{
    switch (chunks) {
    case 4: return scatter_u<LG, 32>(x_dtype, P, SP, grid, s);
    case 8: return scatter_u<LG, 64>(x_dtype, P, SP, grid, s);
    case 16: return scatter_u<LG, 128>(x_dtype, P, SP, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template <int LG, int U>
static cudaError_t reduce_u(const Launch& P, unsigned grid, cudaStream_t s)
{
    const cudaError_t e = smem_limit<k_reduce<LG, U>>(enc_smem_bytes(U));
    if (e != cudaSuccess) return e;
    return launch_enc(k_reduce<LG, U>, grid, enc_smem_bytes(U), s, P.dep != 0, P);
}

template <int LG>
cudaError_t launch_reduce_lg(int chunks, const Launch& P, unsigned grid, cudaStream_t s)
{
    switch (chunks) {
    case 4: return reduce_u<LG, 32>(P, grid, s);
    case 8: return reduce_u<LG, 64>(P, grid, s);
    case 16: return reduce_u<LG, 128>(P, grid, s);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_compress_lg<ZC_LOG2L>(int, int, const Launch&, unsigned, cudaStream_t);
template cudaError_t launch_compress_heads_lg<ZC_LOG2L>(int, const Launch&, unsigned, cudaStream_t);
template cudaError_t launch_scatter_lg<ZC_LOG2L>(int, int, const Launch&, const ScatterParams&,
                                                 unsigned, cudaStream_t);
template cudaError_t launch_reduce_lg<ZC_LOG2L>(int, const Launch&, unsigned, cudaStream_t);

}  // namespace zc
