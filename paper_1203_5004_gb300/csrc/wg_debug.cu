// wg_debug.cu -- small kernels behind the wg_debug_* entry points, so that the
// predicate, the bridge search and the in-register stages can be compared
// with the CPU oracle on their own.
#include <cuda_runtime.h>
#include <cstdint>

#include "wg_device.cuh"

namespace wg {

template <int MODE>
__global__ void dbg_orient_kernel(const float2 *p, long long ntri, int8_t *signs,
                                  unsigned long long *fallbacks)
{
    PredCount pc;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < ntri;
         t += (long long)gridDim.x * blockDim.x)
        signs[t] = (int8_t)orient<MODE | kModeCount>(pc, p[3 * t], p[3 * t + 1], p[3 * t + 2]);
    unsigned long long f = pc.fallbacks;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) f += __shfl_xor_sync(kFull, f, o);
    if ((threadIdx.x & 31) == 0 && f) atomicAdd(fallbacks, f);
}

template <int MODE>
__global__ void dbg_bridge_kernel(const float2 *P, int hp, const float2 *Q, int hq, int *out)
{
    PredCount pc;
    int2 pq = bridge_warp<MODE>(pc, PtrHood{P}, hp, PtrHood{Q}, hq);
    {
        // the search that probes the end of P first must give the same bridge
        const int2 r = bridge_tail<MODE>(pc, PtrHood{P}, hp, PtrHood{Q}, hq);
        if (r.x != pq.x || r.y != pq.y) pq = make_int2(-1, -1);
    }
    if (hp <= 32 && hq <= 32) {
        // the small-hood search must give the same bridge
        const int2 r = bridge_small<MODE>(pc, PtrHood{P}, hp, PtrHood{Q}, hq);
        if (r.x != pq.x || r.y != pq.y) pq = make_int2(-1, -1);
    }
    if (threadIdx.x == 0) {
        out[0] = pq.x;
        out[1] = pq.y;
    }
}

template <int MODE>
__global__ void dbg_bridge_cta_kernel(const float2 *P, int hp, const float2 *Q, int hq, int *out)
{
    __shared__ int sh[2 * 32 + 2];
    PredCount pc;
    const int2 pq = bridge_cta<MODE>(pc, PtrHood{P}, hp, PtrHood{Q}, hq, sh);
    if (threadIdx.x == 0) {
        out[0] = pq.x;
        out[1] = pq.y;
    }
}

template <int MODE>
__global__ void dbg_warp_hood_kernel(const float2 *pts, int m, int *out, int *count)
{
    PredCount pc;
    const int lane = threadIdx.x;
    float2 pt = make_float2(0.f, 0.f);
    int id = lane;
    if (lane < m) pt = pts[lane];
    const int h = warp_hood_regs<MODE>(pc, pt, id, m);
    if (lane < h) out[lane] = id;
    if (lane == 0) *count = h;
}

cudaError_t debug_orient(const float *p, long long ntri, int8_t *signs, unsigned long long *fb,
                         int fp64, cudaStream_t st)
{
    if (ntri == 0) return cudaSuccess;
    const long long blocks = (ntri + 255) / 256;
    const int grid = (int)(blocks < 4096 ? blocks : 4096);
    const float2 *pp = reinterpret_cast<const float2 *>(p);
    if (fp64)
        dbg_orient_kernel<kModeFp64Only><<<grid, 256, 0, st>>>(pp, ntri, signs, fb);
    else
        dbg_orient_kernel<0><<<grid, 256, 0, st>>>(pp, ntri, signs, fb);
    return cudaGetLastError();
}

cudaError_t debug_bridge_cta(const float *P, int hp, const float *Q, int hq, int *out, int fp64, cudaStream_t st)
{
    const float2 *p = reinterpret_cast<const float2 *>(P), *q = reinterpret_cast<const float2 *>(Q);
    if (fp64)
        dbg_bridge_cta_kernel<kModeFp64Only><<<1, 256, 0, st>>>(p, hp, q, hq, out);
    else
        dbg_bridge_cta_kernel<0><<<1, 256, 0, st>>>(p, hp, q, hq, out);
    return cudaGetLastError();
}

cudaError_t debug_bridge(const float *P, int hp, const float *Q, int hq, int *out, int fp64,
                         cudaStream_t st)
{
    const float2 *pp = reinterpret_cast<const float2 *>(P);
    const float2 *qq = reinterpret_cast<const float2 *>(Q);
    if (fp64)
        dbg_bridge_kernel<kModeFp64Only><<<1, 32, 0, st>>>(pp, hp, qq, hq, out);
    else
        dbg_bridge_kernel<0><<<1, 32, 0, st>>>(pp, hp, qq, hq, out);
    return cudaGetLastError();
}

cudaError_t debug_warp_hood(const float *pts, int m, int *out, int *count, int fp64, cudaStream_t st)
{
    const float2 *pp = reinterpret_cast<const float2 *>(pts);
    if (fp64)
        dbg_warp_hood_kernel<kModeFp64Only><<<1, 32, 0, st>>>(pp, m, out, count);
    else
        dbg_warp_hood_kernel<0><<<1, 32, 0, st>>>(pp, m, out, count);
    return cudaGetLastError();
}

}  // namespace wg
