// Underwater image formation (OceanSim, arXiv 2503.01074, Sec. III-A-1, Eq. 1).
//
// k_uw_image   per pixel and colour channel c:
//                I_c = J_c exp(-beta_attn,c d) + B_inf,c (1 - exp(-beta_bs,c d)),
//              J the in-air image (pixel-major RGB, f32), d the depth (f32, m).
//              A streaming kernel: 12 B of J and 4 B of depth in, 12 B out per
//              pixel; each thread takes 4 pixels as 16-byte loads and stores
//              (three float4 of RGB, one float4 of depth) when the arrays are
//              16-byte aligned, and single pixels otherwise and for the tail.
//              The grid is one resident wave, and each thread's grid-stride
//              loop is unrolled four times so that 16 loads are in flight.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sonar_host.h"
#include "sonar_internal.cuh"

namespace sonar {
namespace {

// exp(-beta d); a zero coefficient attenuates nothing, also at d = +inf
__device__ __forceinline__ float transmission(float beta, float d) {
    return beta == 0.0f ? 1.0f : expf(-beta * d);
}

__device__ __forceinline__ float uw_value(float j, float d, const UwCoef& k, int c) {
    return fmaf(j, transmission(k.b_attn[c], d), k.b_inf[c] * (1.0f - transmission(k.b_bs[c], d)));
}

// I may alias J: a thread reads its pixels before writing them, and no thread
// touches another's pixels (so plain loads, not the read-only path).
__global__ void __launch_bounds__(256) k_uw_image(const float* J, const float* depth, int64_t n, UwCoef k,
                                                  float* I, int vec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (vec) {
        const int64_t quads = n >> 2;
        const float4* J4 = reinterpret_cast<const float4*>(J);
        const float4* d4 = reinterpret_cast<const float4*>(depth);
        float4* I4 = reinterpret_cast<float4*>(I);
#pragma unroll 4
        for (int64_t q = t0; q < quads; q += stride) {
            const float4 a = J4[3 * q], b = J4[3 * q + 1], c = J4[3 * q + 2];
            const float4 d = d4[q];
            // the four pixels' channels: a = (p0r p0g p0b p1r), b = (p1g p1b p2r p2g), c = (p2b p3r p3g p3b)
            I4[3 * q] = make_float4(uw_value(a.x, d.x, k, 0), uw_value(a.y, d.x, k, 1), uw_value(a.z, d.x, k, 2),
                                    uw_value(a.w, d.y, k, 0));
            I4[3 * q + 1] = make_float4(uw_value(b.x, d.y, k, 1), uw_value(b.y, d.y, k, 2), uw_value(b.z, d.z, k, 0),
                                        uw_value(b.w, d.z, k, 1));
            I4[3 * q + 2] = make_float4(uw_value(c.x, d.z, k, 2), uw_value(c.y, d.w, k, 0), uw_value(c.z, d.w, k, 1),
                                        uw_value(c.w, d.w, k, 2));
        }
        done = quads << 2;
    }
    for (int64_t p = done + t0; p < n; p += stride) {
        const float d = depth[p];
        const float j0 = J[3 * p], j1 = J[3 * p + 1], j2 = J[3 * p + 2];
        I[3 * p] = uw_value(j0, d, k, 0);
        I[3 * p + 1] = uw_value(j1, d, k, 1);
        I[3 * p + 2] = uw_value(j2, d, k, 2);
    }
}

}  // namespace

cudaError_t launch_uw_image(const float* J, const float* depth, int64_t n, const UwCoef& k, float* I, int sm_count,
                            cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    const bool vec = ((reinterpret_cast<uintptr_t>(J) | reinterpret_cast<uintptr_t>(depth) |
                       reinterpret_cast<uintptr_t>(I)) & 15u) == 0;
    // one resident wave: every SM streams from start to end, with no partly
    // occupied second round of the grid-stride loop
    int per_sm = 0;   // a host-side calculation, no device work
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_uw_image, 256, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t work = vec ? (n + 3) / 4 : n;
    const int64_t want = (work + 255) / 256;
    const int64_t cap = (int64_t)sm_count * per_sm;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min(want, cap));
    k_uw_image<<<blocks, 256, 0, st>>>(J, depth, n, k, I, vec ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace sonar
