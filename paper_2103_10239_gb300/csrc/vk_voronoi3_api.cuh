// vk_voronoi3_api.cuh -- launchers of the 3D Voronoi rule (vk_voronoi3.cu).
#pragma once
#include "vk_internal.cuh"

namespace vk {

// search + update of every particle: warp = 0 one thread per cell, 1 one warp
// per cell (same results); the overflow kernel finishes the cells that
// outgrow the main kernel's
cudaError_t launch_voronoi3_step(const Geometry& g, const Buffers& b, const StepParams& P, int warp,
                                 cudaStream_t st);
// pass 0: deg[id] = neighbor count; pass 1: the ids of row id at out_off[id], sorted by id
cudaError_t launch_voronoi3_export(const Geometry& g, const Buffers& b, int rep, int n, int pass, int32_t* deg,
                                   const int64_t* out_off, int32_t* out_ids, cudaStream_t st);

}  // namespace vk
