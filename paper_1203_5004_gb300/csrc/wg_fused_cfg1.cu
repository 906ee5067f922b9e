// wg_fused_cfg1.cu -- instantiations of the fused kernel for tile configuration 1
// (one translation unit per configuration so that they compile in parallel).
#include "wg_fused.cuh"

namespace wg {

cudaError_t fused_launch_cfg1(const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    return launch_mode<Cfg1>(args, grid, mode, stream);
}

cudaError_t fused_occupancy_cfg1(int *blocks) { return occupancy_cfg<Cfg1>(blocks); }

int fused_tile_points_cfg1() { return Cfg1::kT; }

int fused_warps_cfg1() { return Cfg1::kW; }

size_t fused_smem_bytes_cfg1() { return Cfg1::kBytes; }

}  // namespace wg
