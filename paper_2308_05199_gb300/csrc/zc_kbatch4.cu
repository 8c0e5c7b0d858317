// zc_kbatch4.cu -- batched compression kernel, tiles of 4 chunks (32-row warp units).
#include "zc_launch.h"

namespace zc {

cudaError_t launch_batch_c4(const Launch& P, unsigned grid, cudaStream_t s)
{
    return launch_batch_u<32>(P, grid, s);
}

}  // namespace zc
