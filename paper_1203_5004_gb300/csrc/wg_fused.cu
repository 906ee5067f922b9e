// wg_fused.cu -- dispatch over the tile configurations of the fused kernel
// (the kernel itself is in wg_fused.cuh, instantiated in wg_fused_cfg*.cu).
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wg {

#define WG_DECL_CFG(i)                                                                        \
    cudaError_t fused_launch_cfg##i(const FusedArgs &args, int grid, int mode, cudaStream_t s); \
    cudaError_t fused_occupancy_cfg##i(int *blocks);                                          \
    int fused_tile_points_cfg##i();                                                           \
    int fused_warps_cfg##i();                                                                 \
    size_t fused_smem_bytes_cfg##i();
WG_DECL_CFG(1)
WG_DECL_CFG(2)
WG_DECL_CFG(3)
WG_DECL_CFG(4)
#undef WG_DECL_CFG

cudaError_t fused_launch(int cfg, const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    switch (cfg) {
    case 1: return fused_launch_cfg1(args, grid, mode, stream);
    case 2: return fused_launch_cfg2(args, grid, mode, stream);
    case 3: return fused_launch_cfg3(args, grid, mode, stream);
    default: return fused_launch_cfg4(args, grid, mode, stream);
    }
}

cudaError_t fused_occupancy(int cfg, int *blocks)
{
    switch (cfg) {
    case 1: return fused_occupancy_cfg1(blocks);
    case 2: return fused_occupancy_cfg2(blocks);
    case 3: return fused_occupancy_cfg3(blocks);
    default: return fused_occupancy_cfg4(blocks);
    }
}

int fused_tile_points(int cfg)
{
    switch (cfg) {
    case 1: return fused_tile_points_cfg1();
    case 2: return fused_tile_points_cfg2();
    case 3: return fused_tile_points_cfg3();
    default: return fused_tile_points_cfg4();
    }
}

int fused_warps(int cfg)
{
    switch (cfg) {
    case 1: return fused_warps_cfg1();
    case 2: return fused_warps_cfg2();
    case 3: return fused_warps_cfg3();
    default: return fused_warps_cfg4();
    }
}

size_t fused_smem_bytes(int cfg)
{
    switch (cfg) {
    case 1: return fused_smem_bytes_cfg1();
    case 2: return fused_smem_bytes_cfg2();
    case 3: return fused_smem_bytes_cfg3();
    default: return fused_smem_bytes_cfg4();
    }
}

}  // namespace wg
