// wg_sort.h -- the device sort (wg_sort.cu), for the host entry points.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace wg {

// Device sort of up to kSortMaxN grid points by (x, y), stable: sorted points
// and the permutation (perm[i] = input index of sorted point i).
constexpr long long kSortMaxN = 1LL << 30;
size_t sort_workspace_bytes(long long n);
cudaError_t sort_launch(const float *points, long long n, float *sorted, int32_t *perm, void *ws, cudaStream_t s);
// out[i] = perm[out[i]] for i < *count (corners of the sorted points mapped back).
cudaError_t sort_map_launch(int32_t *out, const int32_t *count, const int32_t *perm, long long n, cudaStream_t s);

}  // namespace wg
