// wg_fused_cfg2.cu -- instantiations of the fused kernel for tile configuration 2
// (one translation unit per configuration so that they compile in parallel).
#include "wg_fused.cuh"

namespace wg {

cudaError_t fused_launch_cfg2(const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    return launch_mode<Cfg2>(args, grid, mode, stream);
}

cudaError_t fused_occupancy_cfg2(int *blocks) { return occupancy_cfg<Cfg2>(blocks); }

int fused_tile_points_cfg2() { return Cfg2::kT; }

int fused_warps_cfg2() { return Cfg2::kW; }

size_t fused_smem_bytes_cfg2() { return Cfg2::kBytes; }

}  // namespace wg
