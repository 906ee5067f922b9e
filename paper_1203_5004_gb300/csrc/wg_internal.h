// wg_internal.h -- structures shared by the host launch code and the kernels.
#pragma once

#include <cstddef>
#include <cstdint>

namespace wg {

// Workspace header (first 256 bytes of every workspace).
struct WsHeader {
    int status;                    // first device-side error (wg_status code), sticky
    int stall_test_ns;             // test hook: > 0 makes each CTA run one bounded wait on an
                                   // mbarrier that nothing completes, for this many ns
    unsigned long long tests;      // orientation tests (count_predicates = 1)
    unsigned long long fallbacks;  // float64 recomputations (count_predicates = 1)
    unsigned long long pad[28];
    unsigned epoch;                // calls completed on this workspace (tags of this call: epoch + 1)
    unsigned done_ctas;            // CTAs of the running call that have finished
};
static_assert(sizeof(WsHeader) == 256, "header is 256 bytes");

// One work item of the fused kernel: a contiguous range of one set.
struct SegItem {
    long long set_base;  // absolute index of the set's first point
    long long a, b;      // set-relative point range [a, b)
    int set;             // set index (out_counts / arrivals slot)
    int c;               // segment index within the set
    int nseg;            // segments of this set
    int slot;            // index of this segment's count in seg_count
    int slot0;           // slot of segment 0 of this set
    int pad;             // stage slot (segments of multi-segment sets)
};

struct FusedArgs {
    const float *points;     // (x, y) pairs
    int32_t *out_idx;
    int32_t *out_count;      // per set
    // single-set plan (items == nullptr): segments of `tiles_per_seg`-ish tiles
    long long n;
    int tiles;
    int nseg;
    // explicit items (batched), else nullptr
    const SegItem *items;
    int num_items;
    const int *num_items_dev;  // batched: item count written by the planning kernel
    unsigned *queue;           // batched: dynamic item queue (reset by the last CTA)
    unsigned *done;            // batched: CTAs finished
    int validate;
    WsHeader *hdr;
    int *seg_count;          // one per segment slot (negative: coordinates not staged)
    float *seg_ymax;         // one per segment slot: max y of the segment
    float *seg_xy;           // per stage slot: kStageCorners float2 (segment hood coordinates)
    int *seg_sidx;           // per stage slot: kStageCorners ints (segment hood indices, set-relative)
    int *seg_live;           // per stage slot: 16 ints of final-merge scratch
    unsigned *seg_pair;      // per stage slot: tag of the call whose segment hood (this or the next
                             // segment) was published first, for the pair (this, next)
    unsigned long long *seg_bridge;  // per stage slot: bridge of the pair (this, next): tag << 32 | p << 16 | q
    unsigned *arrivals;      // one per set
};

// Corners of a segment hood whose coordinates are staged for the final merge
// (the running window of every tile configuration has this size).
constexpr int kStageCorners = 128;

// Tile configurations (warps per CTA, points per lane (odd), tile buffers
// per warp, running window). Index 1..kNumTileCfgs as exposed in the ABI.
struct TileCfgDesc {
    int warps, k, stages, rcap;
};
constexpr int kNumTileCfgs = 4;
constexpr TileCfgDesc kTileCfgs[kNumTileCfgs] = {
    {8, 23, 4, 128},
    {12, 15, 4, 128},
    {8, 31, 3, 128},
    {6, 31, 4, 128},
};

// Plain full-stage path.
struct PlainArgs {
    const float *points;
    long long n;
    // hood arrays of the stage input (dense) and output
    const float *in_xy;      // float2 per corner
    const int32_t *in_idx;
    const int32_t *in_off;   // hood h occupies [in_off[h], in_off[h+1])
    int in_hoods;
    float *out_xy;
    int32_t *out_idx;
    int32_t *out_off;        // out_off[0..out_hoods]
    int out_hoods;
    unsigned long long *lookback;  // one status word per block of this stage
    unsigned *ticket;              // block ticket counter of this stage
    int32_t *final_idx;            // last stage: write corners here ...
    int32_t *final_count;          // ... and the count here
    WsHeader *hdr;
};

}  // namespace wg
