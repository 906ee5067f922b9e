// wg_hull.cu -- the convex hull (the paper's title problem; Section 2
// computes its upper half, the upper hood) from two upper-hood calls.
//
// The lower hood of the points is the upper hood of the points turned by 180
// degrees: (x, y) -> (c - x, c - y) with c = 1 - 2^-24, read in reverse
// order. The turned points are again grid points in [0, 1) (c - k 2^-24 =
// (2^24 - 1 - k) 2^-24 exactly) and again sorted, so the fused upper-hood
// kernel computes the lower hood unchanged; its corners run from the last
// point back to the first. The hull is the upper hood followed by that chain
// without its two ends. A repeated point keeps its first occurrence: the
// turned order meets the last copy first, which the stitch maps back to the
// first copy (a binary search over the sorted input).
#include <cuda_runtime.h>

#include <cstdint>

#include "wg.h"
#include "wg_internal.h"

namespace wg {

// rot[k] = turned point n - 1 - k
__global__ void hull_turn_kernel(const float2 *__restrict__ p, float2 *__restrict__ rot, long long n)
{
    const float c = 0x1.fffffep-1f;  // 1 - 2^-24
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (long long)gridDim.x * blockDim.x) {
        const float2 v = p[n - 1 - k];
        rot[k] = make_float2(__fsub_rn(c, v.x), __fsub_rn(c, v.y));
    }
}

__device__ __forceinline__ bool lex_less(float2 a, float2 b) { return a.x < b.x || (a.x == b.x && a.y < b.y); }

// out[hu + j - 1] = first copy of the input point behind turned corner
// lidx[j], for 1 <= j < hl - 1; *count = hu + max(hl - 2, 0).
__global__ void hull_stitch_kernel(const float2 *__restrict__ p, long long n, const int32_t *__restrict__ lidx,
                                   const int32_t *__restrict__ lcount, int32_t *__restrict__ out,
                                   int32_t *__restrict__ count)
{
    const int hu = *count;  // the upper hood's count, written by the first call
    const int hl = *lcount;
    const int m = hl - 2;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const long long i = n - 1 - lidx[j + 1];
        const float2 v = p[i];
        // first index f <= i with p[f] == v (copies are consecutive)
        long long lo = 0, hi = i;
        while (lo < hi) {
            const long long mid = (lo + hi) >> 1;
            if (lex_less(p[mid], v))
                lo = mid + 1;
            else
                hi = mid;
        }
        out[hu + j] = (int32_t)lo;
    }
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = hu + (m > 0 ? m : 0);
}

cudaError_t hull_turn(const float *points, float *rot, long long n, int sms, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    const long long blocks = (n + 255) / 256;
    const int grid = (int)(blocks < 8LL * sms ? blocks : 8LL * sms);
    hull_turn_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<const float2 *>(points), reinterpret_cast<float2 *>(rot),
                                           n);
    return cudaGetLastError();
}

cudaError_t hull_stitch(const float *points, long long n, const int32_t *lidx, const int32_t *lcount, int32_t *out,
                        int32_t *count, int sms, cudaStream_t st)
{
    // one block: the stitch must read the upper count before any block
    // writes the total
    (void)sms;
    hull_stitch_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<const float2 *>(points), n, lidx, lcount, out, count);
    return cudaGetLastError();
}

}  // namespace wg
