// wg_fused_cfg3.cu -- instantiations of the fused kernel for tile configuration 3
// (one translation unit per configuration so that they compile in parallel).
#include "wg_fused.cuh"

namespace wg {

cudaError_t fused_launch_cfg3(const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    return launch_mode<Cfg3>(args, grid, mode, stream);
}

cudaError_t fused_occupancy_cfg3(int *blocks) { return occupancy_cfg<Cfg3>(blocks); }

int fused_tile_points_cfg3() { return Cfg3::kT; }

int fused_warps_cfg3() { return Cfg3::kW; }

size_t fused_smem_bytes_cfg3() { return Cfg3::kBytes; }

}  // namespace wg
