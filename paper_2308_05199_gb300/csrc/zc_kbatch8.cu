// zc_kbatch8.cu -- batched compression kernel, tiles of 8 chunks (64-row warp units).
#include "zc_launch.h"

namespace zc {

cudaError_t launch_batch_c8(const Launch& P, unsigned grid, cudaStream_t s)
{
    return launch_batch_u<64>(P, grid, s);
}

}  // namespace zc
