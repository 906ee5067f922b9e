// wg_batched.cu -- many independent sets in one persistent launch.
//
// A planning kernel reads the CSR offsets on the device and turns every
// non-empty set into work items for the fused kernel: one item (a whole set on
// one CTA) for sets of up to kMaxTilesPerSeg tiles, several segments for
// larger sets, whose segment hoods the last-arriving CTA merges. Items are
// binned by size (large sets first) so the dynamic queue of the persistent
// kernel finishes with the short items.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "wg_internal.h"

namespace wg {

cudaError_t fused_launch(int cfg, const FusedArgs &args, int grid, int mode, cudaStream_t stream);
cudaError_t fused_occupancy(int cfg, int *blocks);
int fused_tile_points(int cfg);

constexpr int kMaxTilesPerSeg = 128;
constexpr int kMaxSegPerSet = 2048;  // the final merge keeps 2 ints per segment in one tile buffer
constexpr int kPlanThreads = 1024;
constexpr int kBins = 3;

struct BatchLayout {
    size_t arrivals, seg_count, seg_ymax, items, stage_xy, stage_sidx, stage_live, stage_pair, stage_bridge, ctl, total;
    long long max_items, max_stage;
};

static size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// header | arrivals (per set) | per item: count, max y, the item itself |
// per stage slot (segments of multi-segment sets take one each): staged hood
// coordinates, final-merge scratch | control words.
static BatchLayout batch_layout(int num_sets, long long max_items, long long max_stage)
{
    BatchLayout L;
    size_t o = 256;
    L.arrivals = o;
    o = align256(o + (size_t)std::max(num_sets, 1) * 4);
    L.seg_count = o;
    o = align256(o + (size_t)std::max<long long>(max_items, 1) * 4);
    L.seg_ymax = o;
    o = align256(o + (size_t)std::max<long long>(max_items, 1) * 4);
    L.items = o;
    o = align256(o + (size_t)std::max<long long>(max_items, 1) * sizeof(SegItem));
    L.stage_xy = o;
    o = align256(o + (size_t)std::max<long long>(max_stage, 1) * 8 * kStageCorners);
    L.stage_sidx = o;
    o = align256(o + (size_t)std::max<long long>(max_stage, 1) * 4 * kStageCorners);
    L.stage_live = o;
    o = align256(o + (size_t)std::max<long long>(max_stage, 1) * 64);
    L.stage_pair = o;
    o = align256(o + (size_t)std::max<long long>(max_stage, 1) * 4);
    L.stage_bridge = o;
    o = align256(o + (size_t)std::max<long long>(max_stage, 1) * 8);
    L.ctl = o;  // num_items, queue, done, bounds
    o = align256(o + 64);
    L.total = o;
    L.max_items = max_items;
    L.max_stage = max_stage;
    return L;
}

static int min_tile_points()
{
    int t = 1 << 30;
    for (int c = 1; c <= kNumTileCfgs; ++c) t = std::min(t, 32 * kTileCfgs[c - 1].k);
    return t;
}

size_t batched_workspace_bytes(const int64_t *h_offsets, int num_sets)
{
    const int T = min_tile_points();
    long long items = 0;
    for (int s = 0; s < num_sets; ++s) {
        const long long n = h_offsets[s + 1] - h_offsets[s];
        if (n <= 0) continue;
        const long long tiles = (n + T - 1) / T;
        const long long ns = std::min<long long>((tiles + kMaxTilesPerSeg - 1) / kMaxTilesPerSeg, kMaxSegPerSet);
        items += ns;
    }
    return batch_layout(num_sets, items, items).total;
}

__device__ __forceinline__ int bin_of(long long tiles) { return tiles >= 8 ? 0 : (tiles >= 2 ? 1 : 2); }

__global__ void __launch_bounds__(kPlanThreads)
    batch_plan_kernel(const int64_t *off, int num_sets, int T, SegItem *items, long long max_items,
                      long long max_stage, int *ctl, int32_t *out_counts, int *status)
{
    __shared__ int s_bin[kBins];
    __shared__ int s_cur[kBins];
    __shared__ int s_stage;
    const int tid = threadIdx.x;
    if (tid < kBins) s_bin[tid] = 0;
    if (tid == 0) s_stage = 0;
    __syncthreads();
    for (int s = tid; s < num_sets; s += kPlanThreads) {
        const long long n = off[s + 1] - off[s];
        if (n <= 0) {
            out_counts[s] = 0;
            continue;
        }
        const long long tiles = (n + T - 1) / T;
        const int nseg = (int)min((tiles + kMaxTilesPerSeg - 1) / kMaxTilesPerSeg, (long long)kMaxSegPerSet);
        atomicAdd(&s_bin[bin_of(tiles)], nseg);
    }
    __syncthreads();
    if (tid == 0) {
        int acc = 0;
        for (int b = 0; b < kBins; ++b) {
            s_cur[b] = acc;
            acc += s_bin[b];
        }
        if (acc > max_items) {
            atomicCAS(status, 0, 2);
            acc = 0;
        }
        ctl[0] = acc;  // number of items
        ctl[1] = 0;    // queue
        ctl[2] = 0;    // done
    }
    __syncthreads();
    if (ctl[0] == 0) return;
    for (int s = tid; s < num_sets; s += kPlanThreads) {
        const long long a0 = off[s], n = off[s + 1] - a0;
        if (n <= 0) continue;
        const long long tiles = (n + T - 1) / T;
        const int nseg = (int)min((tiles + kMaxTilesPerSeg - 1) / kMaxTilesPerSeg, (long long)kMaxSegPerSet);
        const int base = atomicAdd(&s_cur[bin_of(tiles)], nseg);
        int stage = 0;
        if (nseg > 1) {
            stage = atomicAdd(&s_stage, nseg);
            if (stage + nseg > max_stage) {
                atomicCAS(status, 0, 2);
                stage = 0;
            }
        }
        for (int c = 0; c < nseg; ++c) {
            SegItem it;
            const long long lo = (long long)c * tiles / nseg, hi = (long long)(c + 1) * tiles / nseg;
            it.set_base = a0;
            it.a = lo * T;
            it.b = hi * T < n ? hi * T : n;
            it.set = s;
            it.c = c;
            it.nseg = nseg;
            it.slot = base + c;
            it.slot0 = base;
            it.pad = stage + c;
            items[base + c] = it;
        }
    }
}

cudaError_t batched_launch(const float *points, const int64_t *offsets, int num_sets, int32_t *out_idx,
                           int32_t *out_counts, void *ws, size_t ws_bytes, int cfg, int mode, int validate,
                           cudaStream_t st)
{
    // The item bound of the workspace, recovered from its size (every item
    // has a stage slot, so one bound sizes everything).
    long long lo = 0, hi = 1;
    while (batch_layout(num_sets, hi, hi).total <= ws_bytes && hi < (1ll << 40)) hi *= 2;
    while (lo + 1 < hi) {
        const long long mid = (lo + hi) / 2;
        if (batch_layout(num_sets, mid, mid).total <= ws_bytes) lo = mid; else hi = mid;
    }
    if (lo < 1 || batch_layout(num_sets, lo, lo).total > ws_bytes) return cudaErrorInvalidValue;
    const BatchLayout L = batch_layout(num_sets, lo, lo);
    char *w = static_cast<char *>(ws);
    WsHeader *hdr = reinterpret_cast<WsHeader *>(w);
    int *ctl = reinterpret_cast<int *>(w + L.ctl);
    SegItem *items = reinterpret_cast<SegItem *>(w + L.items);
    const int T = fused_tile_points(cfg);
    batch_plan_kernel<<<1, kPlanThreads, 0, st>>>(offsets, num_sets, T, items, L.max_items, L.max_stage, ctl,
                                                  out_counts, &hdr->status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    int blocks = 0;
    if ((e = fused_occupancy(cfg, &blocks)) != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    FusedArgs a;
    std::memset(&a, 0, sizeof(a));
    a.points = points;
    a.out_idx = out_idx;
    a.out_count = out_counts;
    a.items = items;
    a.num_items = 0;
    a.num_items_dev = ctl;
    a.queue = reinterpret_cast<unsigned *>(ctl + 1);
    a.done = reinterpret_cast<unsigned *>(ctl + 2);
    a.validate = validate;
    a.hdr = hdr;
    a.seg_count = reinterpret_cast<int *>(w + L.seg_count);
    a.seg_ymax = reinterpret_cast<float *>(w + L.seg_ymax);
    a.seg_xy = reinterpret_cast<float *>(w + L.stage_xy);
    a.seg_live = reinterpret_cast<int *>(w + L.stage_live);
    a.seg_sidx = reinterpret_cast<int *>(w + L.stage_sidx);
    a.seg_pair = reinterpret_cast<unsigned *>(w + L.stage_pair);
    a.seg_bridge = reinterpret_cast<unsigned long long *>(w + L.stage_bridge);
    a.arrivals = reinterpret_cast<unsigned *>(w + L.arrivals);
    const int grid = std::max(1, blocks) * sms;
    return fused_launch(cfg, a, grid, mode, st);
}

}  // namespace wg
