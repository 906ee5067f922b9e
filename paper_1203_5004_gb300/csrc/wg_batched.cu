// wg_batched.cu -- many independent sets in one persistent launch.
//
// Two planning passes read the CSR offsets on the device and turn every
// non-empty set into work items for the fused kernel: one item (a whole set on
// one warp) for sets of up to `cap` tiles, several segments for larger sets
// (claimed by different warps; the warp that completes the set merges the
// segment hoods). Items are binned by size (large sets first) so that the
// dynamic queue of the persistent kernel finishes with the short items. The
// segment cap is a launch parameter (the batched autotuner chooses it).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "wg_internal.h"

namespace wg {

cudaError_t fused_launch(int cfg, const FusedArgs &args, int grid, int mode, cudaStream_t stream);
cudaError_t fused_occupancy(int cfg, int *blocks);
int fused_tile_points(int cfg);

constexpr int kDefaultSegTiles = 128;  // tiles per segment of a large set (default cap)
constexpr int kMinSegTiles = 8;        // the smallest cap a call may use (sizes the workspace)
constexpr int kMaxSegPerSet = 2048;
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
    L.ctl = o;  // items, queue, done, items per bin, bin cursors, stage cursor
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
        const long long ns = std::min<long long>((tiles + kMinSegTiles - 1) / kMinSegTiles, kMaxSegPerSet);
        items += ns;
    }
    return batch_layout(num_sets, items, items).total;
}

__device__ __forceinline__ int bin_of(long long tiles) { return tiles >= 8 ? 0 : (tiles >= 2 ? 1 : 2); }

// Segments of a set of n points: one per `cap` tiles (at most
// kMaxSegPerSet), and its size bin.
__device__ __forceinline__ int set_segments(long long n, int T, int cap, int &bin)
{
    const long long tiles = (n + T - 1) / T;
    bin = bin_of(tiles);
    return (int)min((tiles + cap - 1) / cap, (long long)kMaxSegPerSet);
}

// Planning, in two grid-wide passes. ctl: [0] items, [1] queue, [2] done,
// [3..5] items per bin, [6..8] bin cursors, [9] stage-slot cursor (3..9
// cleared before the first pass).
// Pass 1: items per size bin (one global add per bin and block).
__global__ void __launch_bounds__(kPlanThreads)
    batch_count_kernel(const int64_t *off, int num_sets, int T, int cap, int *ctl, int32_t *out_counts)
{
    __shared__ int s_bin[kBins];
    const int tid = threadIdx.x;
    if (tid < kBins) s_bin[tid] = 0;
    __syncthreads();
    for (int s = blockIdx.x * kPlanThreads + tid; s < num_sets; s += gridDim.x * kPlanThreads) {
        const long long n = off[s + 1] - off[s];
        if (n <= 0) {
            out_counts[s] = 0;
            continue;
        }
        int bin;
        const int nseg = set_segments(n, T, cap, bin);
        atomicAdd(&s_bin[bin], nseg);
    }
    __syncthreads();
    if (tid < kBins && s_bin[tid]) atomicAdd(ctl + 3 + tid, s_bin[tid]);
}

// Pass 2: every set's items, written at its bin's offset (larger sets
// first), with stage slots for sets of several segments. A block reserves
// its ranges with one global add per bin, then places its own sets.
__global__ void __launch_bounds__(kPlanThreads)
    batch_assign_kernel(const int64_t *off, int num_sets, int T, int cap, SegItem *items, long long max_items,
                        long long max_stage, int *ctl, int *status)
{
    __shared__ int s_bin[kBins];
    __shared__ int s_cur[kBins];
    __shared__ int s_stage, s_stage_cur;
    const int tid = threadIdx.x;
    int base[kBins];
    long long acc = 0;
#pragma unroll
    for (int b = 0; b < kBins; ++b) {
        base[b] = (int)acc;
        acc += ctl[3 + b];
    }
    const bool over = acc > max_items;
    if (blockIdx.x == 0 && tid == 0) {
        ctl[0] = over ? 0 : (int)acc;  // number of items
        ctl[1] = 0;                    // queue
        ctl[2] = 0;                    // done
        if (over) atomicCAS(status, 0, 2);
    }
    if (over || acc == 0) return;
    if (tid < kBins) s_bin[tid] = 0;
    if (tid == 0) s_stage = 0;
    __syncthreads();
    for (int s = blockIdx.x * kPlanThreads + tid; s < num_sets; s += gridDim.x * kPlanThreads) {
        const long long n = off[s + 1] - off[s];
        if (n <= 0) continue;
        int bin;
        const int nseg = set_segments(n, T, cap, bin);
        atomicAdd(&s_bin[bin], nseg);
        if (nseg > 1) atomicAdd(&s_stage, nseg);
    }
    __syncthreads();
    if (tid < kBins) s_cur[tid] = base[tid] + (s_bin[tid] ? atomicAdd(ctl + 6 + tid, s_bin[tid]) : 0);
    if (tid == 0) s_stage_cur = s_stage ? atomicAdd(ctl + 9, s_stage) : 0;
    __syncthreads();
    for (int s = blockIdx.x * kPlanThreads + tid; s < num_sets; s += gridDim.x * kPlanThreads) {
        const long long a0 = off[s], n = off[s + 1] - a0;
        if (n <= 0) continue;
        int bin;
        const int nseg = set_segments(n, T, cap, bin);
        const long long tiles = (n + T - 1) / T;
        const int slot0 = atomicAdd(&s_cur[bin], nseg);
        int stage = 0;
        if (nseg > 1) {
            stage = atomicAdd(&s_stage_cur, nseg);
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
            it.slot = slot0 + c;
            it.slot0 = slot0;
            it.pad = stage + c;
            items[slot0 + c] = it;
        }
    }
}

cudaError_t batched_launch(const float *points, const int64_t *offsets, int num_sets, int32_t *out_idx,
                           int32_t *out_counts, void *ws, size_t ws_bytes, int cfg, int cap, int mode, int validate,
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
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int plan_blocks =
        (int)std::max(1LL, std::min<long long>((num_sets + kPlanThreads - 1) / kPlanThreads, 4LL * std::max(1, sms)));
    cudaError_t e = cudaMemsetAsync(ctl + 3, 0, 7 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (cap < kMinSegTiles) cap = kDefaultSegTiles;
    batch_count_kernel<<<plan_blocks, kPlanThreads, 0, st>>>(offsets, num_sets, T, cap, ctl, out_counts);
    batch_assign_kernel<<<plan_blocks, kPlanThreads, 0, st>>>(offsets, num_sets, T, cap, items, L.max_items,
                                                              L.max_stage, ctl, &hdr->status);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;

    int blocks = 0;
    if ((e = fused_occupancy(cfg, &blocks)) != cudaSuccess) return e;
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
