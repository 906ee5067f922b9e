// wg_fused_cfg4.cu -- instantiations of the fused kernel for tile configuration 4
// (one translation unit per configuration so that they compile in parallel).
#include "wg_fused.cuh"

namespace wg {

cudaError_t fused_launch_cfg4(const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    return launch_mode<Cfg4>(args, grid, mode, stream);
}

cudaError_t fused_occupancy_cfg4(int *blocks) { return occupancy_cfg<Cfg4>(blocks); }

int fused_tile_points_cfg4() { return Cfg4::kT; }

int fused_warps_cfg4() { return Cfg4::kW; }

size_t fused_smem_bytes_cfg4() { return Cfg4::kBytes; }

}  // namespace wg
