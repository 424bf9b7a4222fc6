// L2 read-bandwidth probe: the measured denominator for the L2 side of the
// ray cast's roofline (its node and triangle fetches are mostly L2 hits).
#include <cuda_runtime.h>
#include <stdint.h>

#include "sonar_host.h"

namespace sonar {
namespace {

// Grid-stride passes over the buffer with L2-cached, L1-bypassing 16-byte
// loads, four in flight per thread; the block's sum of everything it read is
// written out, so no load can be dropped and a test can check the count.
__global__ void __launch_bounds__(512) k_l2_read(const float4* __restrict__ buf, int64_t n, int passes,
                                                 float* block_sums) {
    __shared__ float red[16];
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    for (int p = 0; p < passes; ++p) {
        int64_t i = t0;
        for (; i + 3 * stride < n; i += 4 * stride) {
            const float4 v0 = __ldcg(buf + i), v1 = __ldcg(buf + i + stride);
            const float4 v2 = __ldcg(buf + i + 2 * stride), v3 = __ldcg(buf + i + 3 * stride);
            a0 += (v0.x + v0.y) + (v0.z + v0.w);
            a1 += (v1.x + v1.y) + (v1.z + v1.w);
            a2 += (v2.x + v2.y) + (v2.z + v2.w);
            a3 += (v3.x + v3.y) + (v3.z + v3.w);
        }
        for (; i < n; i += stride) {
            const float4 v = __ldcg(buf + i);
            a0 += (v.x + v.y) + (v.z + v.w);
        }
    }
    float s = (a0 + a1) + (a2 + a3);
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0f;
        for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = s;
    }
}

}  // namespace

cudaError_t launch_l2_read(const void* buf, int64_t bytes, int passes, float* block_sums, int n_blocks,
                           cudaStream_t st) {
    k_l2_read<<<n_blocks, 512, 0, st>>>(static_cast<const float4*>(buf), bytes / 16, passes, block_sums);
    return cudaGetLastError();
}

}  // namespace sonar
