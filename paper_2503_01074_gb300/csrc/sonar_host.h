// Host-side internal declarations shared by the libsonar translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "sonar_internal.cuh"

namespace sonar {

// A built scene: packed hierarchies (4-wide and 8-wide) and triangles (owned
// by the context).  n_pairs counts 4-wide nodes, n_nodes8 8-wide ones.
struct SceneStore {
    float4* nodes = nullptr;
    float4* nodes8 = nullptr;
    float4* tris = nullptr;
    int32_t* mat_orig = nullptr;
    int32_t root = kEmpty;
    int64_t n_tris = 0, n_pairs = 0, n_nodes8 = 0;
    int32_t height = 0;
    int32_t max_mat = -1;
    size_t bytes = 0;
};

sonar_status build_scene(const float* verts, int64_t nv, const int32_t* tris, const int32_t* mat,
                         int64_t nt, cudaStream_t st, SceneStore* out, std::string* msg);
void free_scene(SceneStore* s);

inline SceneDev scene_dev(const SceneStore& s) {
    return SceneDev{s.nodes, s.tris, s.mat_orig, s.root, (int32_t)s.n_tris, s.nodes8};
}

// Kernel launchers (trace.cu: ray cast and counters; render.cu: binning, noise,
// normalisation, fan and adjoint; image.cu: Eq. 1 camera; dvl.cu: DVL;
// probe.cu: L2 read-bandwidth probe).
void set_kernel_attributes();
cudaError_t launch_trig(const SensorDev* sensors, const SensorDev& one, int n_sensors, int max_angles,
                        cudaStream_t st);
cudaError_t launch_trace(const TraceArgs& a, int blocks, int occupancy, cudaStream_t st);
cudaError_t launch_bin(const BinArgs& a, int det, int grid, int block, size_t smem, cudaStream_t st);
int bin_blocks_per_sm(int det, int block, size_t smem);
constexpr size_t kMaxDynSmem = 200 * 1024;
cudaError_t launch_philox(const void* ctr, int64_t n, uint32_t k0, uint32_t k1, void* out, cudaStream_t st);
cudaError_t launch_norm(const NormArgs& a, cudaStream_t st);
cudaError_t launch_fan_tiles(const FanArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_fan_lut(const FanLutArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_fan_group(const FanGroupArgs& a, int blocks, cudaStream_t st);
cudaError_t launch_adj_rows(const SensorDev* sensors, const int32_t* row_map, const SensorDev& one, int n_sensors,
                            int64_t total_groups, int normalise, const float* noised,
                            const float* grad, RowInfo* info, int32_t* zero_word, cudaStream_t st);
cudaError_t launch_adjoint(const AdjArgs& a, int grid, int block, size_t smem, float* dtheta, cudaStream_t st);
int adjoint_blocks_per_sm(int block, size_t smem);
cudaError_t launch_stats(const SensorDev& s, const SceneDev& sc, const sonar_params& p,
                         const TraceCounters& tc, uint32_t* err, cudaStream_t st);
cudaError_t launch_uw_image(const float* J, const float* depth, int64_t n, const UwCoef& k, float* I, int sm_count,
                            cudaStream_t st);
cudaError_t launch_dvl(const DvlArgs& a, cudaStream_t st);
cudaError_t launch_dvl_schedule(const float* period, int64_t n_veh, int64_t n_steps, float dt, int32_t* emit,
                                cudaStream_t st);
cudaError_t launch_popcount(const uint32_t* bits, int64_t words, unsigned long long* out,
                            cudaStream_t st);
cudaError_t launch_l2_read(const void* buf, int64_t bytes, int passes, float* block_sums, int n_blocks,
                           cudaStream_t st);

}  // namespace sonar
