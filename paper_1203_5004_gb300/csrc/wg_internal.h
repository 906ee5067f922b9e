// wg_internal.h -- structures shared by the host launch code and the kernels.
#pragma once

#include <cuda_runtime.h>

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
    unsigned long long pad[24];
    // single-set schedule and final merge (reset within every call)
    unsigned claim;                // segments claimed by warps (reset by the last CTA)
    unsigned phase1;               // tag of the call whose hood list is ready
    unsigned phase2;               // tag of the call whose output plan is ready
    unsigned pair_work;            // pair bridges taken
    unsigned pair_done;            // pair bridges finished
    unsigned nlist;                // hoods left after the staircase
    unsigned nplan;                // plan entries (kept hoods)
    unsigned spare;
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
    // single-set plan (items == nullptr): segments claimed dynamically by
    // warps; segment c covers tiles [tile0(c), tile0(c + 1)) with
    // sch_n1 segments of sch_l1 tiles, then sch_n2 of sch_l2, then single tiles
    long long n;
    int tiles;
    int nseg;
    int sch_n1, sch_l1, sch_n2, sch_l2;
    int *list_lid;            // single set: hoods left after the staircase (segment ids)
    int *list_bp;             // ... bridge of the pair (i, i + 1): corner of hood i
    int *list_bq;             // ... and of hood i + 1
    int4 *plan;               // single set: kept hoods (stage slot, first corner, length, destination)
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

// Most segments of one single-set call (the final merge keeps per-segment
// arrays of this size in one CTA's shared memory).
constexpr int kMaxSegSingle = 4096;

// Small sets (wg_small.cu): one CTA holds the whole set, up to this many points.
constexpr long long kSmallMaxN = 8192;
// Upper hood of points[0, n), 1 <= n <= kSmallMaxN, in one launch; hdr is the
// workspace header (status and counters).
cudaError_t small_launch(const float *points, long long n, int32_t *out_idx, int32_t *out_count, void *hdr,
                         int mode, int validate, cudaStream_t stream);

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

// Single-set schedule: the first n1 segments (one per warp) have l1 tiles,
// the next n2 have l2 tiles, the rest one tile each, so that segments get
// shorter towards the end of the input and the warps that claim them last
// finish close together. At most max_seg segments.
struct Schedule {
    int n1, l1, n2, l2, nseg;
};

// balanced = true: one segment per warp instead, the tiles split as evenly
// as possible (the first tiles % warps segments one tile longer).
inline Schedule make_schedule(long long tiles, long long warps, int max_seg, bool balanced = false)
{
    Schedule s{0, 1, 0, 1, 0};
    if (balanced) {
        long long n = warps < max_seg ? warps : max_seg;
        if (n > tiles) n = tiles;
        if (n < 1) n = 1;
        const long long q = tiles / n, r = tiles % n;
        s.n1 = (int)r;
        s.l1 = (int)(q + 1);
        s.n2 = (int)(n - r);
        s.l2 = (int)q;
        s.nseg = (int)n;
        return s;
    }
    if (tiles <= max_seg) {
        s.n1 = (int)tiles;
        s.nseg = (int)tiles;
        return s;
    }
    long long n1 = warps < max_seg / 2 ? warps : max_seg / 2;
    if (n1 < 1) n1 = 1;
    long long l1 = (long long)(0.78 * (double)tiles / (double)n1);
    if (l1 < 1) l1 = 1;
    if (n1 * l1 > tiles) l1 = tiles / n1;
    const long long rem = tiles - n1 * l1;
    long long n3 = n1 / 4 < rem ? n1 / 4 : rem;
    const long long r2 = rem - n3;
    const long long room = max_seg - n1 - n3;
    long long l2 = room > 0 ? (r2 + room - 1) / room : r2;
    if (l2 < 1) l2 = 1;
    // the last partial group of l2 tiles becomes single tiles: grow l2 until
    // every segment fits
    long long n2 = r2 / l2;
    while (n1 + n2 + (rem - n2 * l2) > max_seg) {
        ++l2;
        n2 = r2 / l2;
    }
    n3 = rem - n2 * l2;
    s.n1 = (int)n1;
    s.l1 = (int)l1;
    s.n2 = (int)n2;
    s.l2 = (int)l2;
    s.nseg = (int)(n1 + n2 + n3);
    return s;
}

// First tile of segment c under a schedule (c may equal nseg: returns tiles).
__host__ __device__ inline long long schedule_tile0(int n1, int l1, int n2, int l2, long long tiles, int c)
{
    long long t;
    if (c <= n1)
        t = (long long)c * l1;
    else if (c <= n1 + n2)
        t = (long long)n1 * l1 + (long long)(c - n1) * l2;
    else
        t = (long long)n1 * l1 + (long long)n2 * l2 + (c - n1 - n2);
    return t < tiles ? t : tiles;
}

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
