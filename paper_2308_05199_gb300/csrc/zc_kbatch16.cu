// zc_kbatch16.cu -- batched compression kernel, tiles of 16 chunks (128-row warp units).
#include "zc_launch.h"

namespace zc {

cudaError_t launch_batch_c16(const Launch& P, unsigned grid, cudaStream_t s)
{
    return launch_batch_u<128>(P, grid, s);
}

}  // namespace zc
