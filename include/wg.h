/*
 * wg.h -- C ABI of libwagener: the upper hood (upper convex hull) of sorted
 * planar points on one GB300 GPU, by the merge schedule of Wagener's PRAM
 * algorithm as implemented in C. O Dunlaing, "CUDA implementation of
 * Wagener's 2D convex hull PRAM algorithm" (arXiv:1203.5004).
 *
 * The problem (paper Section 2): n points presented left to right; return the
 * corners of their upper hood, left to right. Every stage of the paper's
 * schedule merges adjacent pairs of hoods: it finds the bridge (upper common
 * tangent) of each pair with the paper's g/f tests and LOW/EQUAL/HIGH votes
 * (Section 2, match_and_merge, phases mam 1 to mam 5) and keeps
 * P[0..p] ++ Q[q..] (mam 6).
 *
 * Input contract shared by every entry point
 *   - points: float32 pairs (x, y), interleaved, 8-byte aligned; x and y are
 *     integers times 2^-24 in [0, 1) (the "grid"); sorted lexicographically by
 *     (x, y), except for wg_sort_points and wg_upper_hood_unsorted, which take
 *     them in any order. Grid coordinates make every coordinate difference exact in
 *     float32, which the orientation predicate relies on (see wg_options).
 *     Off-grid or unsorted input gives unspecified (but memory-safe) output
 *     unless validation is enabled.
 *   - Readings fixed where the paper is silent: equal x values are allowed
 *     (order is lexicographic); a point equal to an earlier point is never a
 *     corner (first occurrence wins); collinear points are not corners (each
 *     corner is a strict right turn); any n >= 0 is accepted.
 *   - Output of the upper-hood calls: the input indices of the corners, left
 *     to right (strictly increasing for sorted input), and their count. n = 0
 *     gives count 0; otherwise the first point is always the first corner.
 *     wg_convex_hull and wg_upper_hood_unsorted state their own order.
 *
 * Ownership and asynchrony
 *   - The caller owns every buffer. The library never allocates device memory
 *     inside a call. Device pointers must stay valid until the stream work
 *     completes.
 *   - Calls enqueue work on `stream` (NULL = legacy default stream) and return
 *     without synchronising, unless stated otherwise. The return code covers
 *     argument checks and launch errors. Errors found on the device (a bounded
 *     wait that gave up, invalid input in validation mode) are recorded in a
 *     status word inside the workspace; read it with wg_get_device_status.
 *   - A workspace must be zero-filled once before its first use (cudaMemset);
 *     every call leaves it ready for the next, and replays of a captured
 *     CUDA graph are calls like any other. After a call that recorded a
 *     device error (wg_get_device_status != WG_OK), zero-fill it again.
 *     Calls that share one workspace must not overlap on the GPU (use one
 *     stream, or one workspace each).
 */
#ifndef WG_H_
#define WG_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st *wg_stream_t; /* same type as cudaStream_t */

typedef enum wg_status {
    WG_OK = 0,
    WG_ERR_INVALID_VALUE = 1, /* null pointer, negative size, misaligned pointer, bad option */
    WG_ERR_WORKSPACE = 2,     /* workspace null or smaller than the size query returns */
    WG_ERR_UNSORTED = 3,      /* validation: points not sorted by (x, y) */
    WG_ERR_OFF_GRID = 4,      /* validation: a coordinate not k * 2^-24 in [0, 1) */
    WG_ERR_TIMEOUT = 5,       /* a bounded device wait gave up; output is not valid */
    WG_ERR_CUDA = 6,          /* a CUDA runtime call failed (launch, copy, attribute) */
    WG_ERR_UNSUPPORTED = 7    /* no usable sm_103 device, or a size beyond the limits */
} wg_status;

/* Orientation predicate precision (the only arithmetic on the path).
 * WG_PRED_FILTERED: det(a - o, b - o) in float32 from exact differences;
 *   the sign is accepted when |det| > 2^-22 (|t1| + |t2|), t1 and t2 being the
 *   two rounded products, which bounds the rounding error; otherwise the
 *   determinant is recomputed exactly in float64 (products of 24-bit
 *   differences are exact there).
 * WG_PRED_FP64: always the exact float64 evaluation. */
typedef enum wg_pred_mode { WG_PRED_FILTERED = 0, WG_PRED_FP64 = 1 } wg_pred_mode;

typedef struct wg_options {
    int32_t pred_mode;       /* wg_pred_mode */
    int32_t count_predicates;/* 1: count orientation tests and float64 fallbacks (slower) */
    int32_t validate;        /* 1: check grid membership and order; report WG_ERR_* on device */
    int32_t tile_config;     /* 0 = library choice (single set: autotuned if wg_autotune ran, else 1;
                                batched: 3); else 1..WG_NUM_TILE_CONFIGS */
    int32_t segments_per_cta;/* 0 = library choice; else the schedule plans its first, long segments
                                for this many times the resident warps (1..8) */
    int32_t schedule;        /* single set: 0 = library choice; 1 = balanced (one segment per warp,
                                equal shares); 2 = guided (long segments first, then shorter ones
                                claimed by warps as they become free); 3 = one CTA (balanced over
                                the warps of a single CTA); 4 = small (n <= WG_SMALL_MAX_N: one CTA
                                holds the set in registers and prunes the survivors in shared
                                memory, no tiles and no merge; the default up to that size) */
    int32_t batch_seg_tiles; /* batched: 0 = library choice (autotuned if wg_autotune_batched ran,
                                else 128); else 8..4096 tiles per segment of a large set (larger
                                sets are split over several warps) */
    int32_t reserved[1];
} wg_options;

#define WG_NUM_TILE_CONFIGS 4
#define WG_SCHEDULE_BALANCED 1
#define WG_SCHEDULE_GUIDED 2
#define WG_SCHEDULE_ONE_CTA 3
#define WG_SCHEDULE_SMALL 4
#define WG_SMALL_MAX_N 8192

/* Fills *opts with the defaults (filtered predicate, no counters, no
 * validation, library-chosen tiling). */
void wg_options_default(wg_options *opts);

/* ------------------------------------------------------------------------
 * Single set, fused schedule (the fast path).
 * Stages 1..log2(T) of the paper's schedule run inside one CTA per tile of T
 * points (Section 2, stage loop of main, fused; Section 3, strips); each CTA
 * merges its consecutive tile hoods into one segment hood; the last CTA to
 * finish merges the segment hoods. One kernel launch.
 *
 * points    device, n (x, y) pairs as above
 * n         0 <= n <= 2^31 - 1
 * out_idx   device int32[max(n, 1)]: corners at out_idx[0..count). The
 *           whole array is used as scratch during the call.
 * out_count device int32[1]
 * workspace device, >= wg_upper_hood_workspace_size(n) bytes, 256-B aligned
 * Returns WG_OK or an argument/launch error.
 * ---------------------------------------------------------------------- */
size_t wg_upper_hood_workspace_size(int64_t n);
wg_status wg_upper_hood(const float *points, int64_t n, int32_t *out_idx,
                        int32_t *out_count, void *workspace, size_t ws_bytes,
                        wg_stream_t stream);
wg_status wg_upper_hood_ex(const float *points, int64_t n, int32_t *out_idx,
                           int32_t *out_count, void *workspace, size_t ws_bytes,
                           const wg_options *opts, wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Single set, plain full-stage schedule: the paper's stage loop (Section 2,
 * main) kept on the device, one kernel launch per stage d = 1, 2, 4, ... Each
 * launch merges every adjacent pair of hoods (bridge by the sampled LOW/EQUAL/
 * HIGH search, mam 1-5) and packs the merged hoods densely with a single-pass
 * decoupled look-back scan (mam 6 with explicit lengths instead of REMOTE
 * padding). Same output as wg_upper_hood; slower; kept as the unfused form.
 * workspace >= wg_upper_hood_plain_workspace_size(n) bytes.
 * ---------------------------------------------------------------------- */
size_t wg_upper_hood_plain_workspace_size(int64_t n);
wg_status wg_upper_hood_plain(const float *points, int64_t n, int32_t *out_idx,
                              int32_t *out_count, void *workspace,
                              size_t ws_bytes, const wg_options *opts,
                              wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Convex hull: the paper's title problem, of which Section 2 computes the
 * upper half. The corners clockwise from the first point: the upper hood
 * from the first point to the last, then the lower hood back to the first,
 * without its two ends. The lower hood is the upper hood of the points turned
 * by 180 degrees ((x, y) -> (1 - 2^-24 - x, 1 - 2^-24 - y), still grid points,
 * in reverse order, still sorted), so the call runs the fused upper-hood
 * kernel twice with a turning pass between and a stitch after. Same input
 * contract and readings (strict corners; a repeated point counts once, by its
 * first occurrence).
 * out_idx   device int32[max(n, 1)]: corners at out_idx[0..count)
 * workspace >= wg_convex_hull_workspace_size(n) bytes, zero-filled once
 * ---------------------------------------------------------------------- */
size_t wg_convex_hull_workspace_size(int64_t n);
wg_status wg_convex_hull(const float *points, int64_t n, int32_t *out_idx,
                         int32_t *out_count, void *workspace, size_t ws_bytes,
                         const wg_options *opts, wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Unsorted input. Section 2 takes its points sorted left to right; these
 * calls supply that order on the device.
 *
 * wg_sort_points: sorts n grid points (each coordinate k * 2^-24 in [0, 1),
 * any order) by (x, y): sorted_points[i] is the input point perm[i]. The sort
 * is stable, so the copies of a repeated point keep their input order.
 * points, sorted_points: device float[2n], 8-byte aligned, not overlapping;
 * perm: device int32[n]; n <= 2^30 (WG_ERR_UNSUPPORTED beyond). The workspace
 * (>= wg_sort_points_workspace_size(n) bytes, 256-byte aligned) needs no
 * initialisation. A point inside [0, 1)^2 but off the grid is sorted by its
 * coordinates rounded down to the grid; coordinates outside [0, 1) are not
 * supported (their order is unspecified, nothing is written out of range).
 *
 * wg_upper_hood_unsorted: the upper hood of points given in any order: the
 * sort, wg_upper_hood_ex on the sorted points, and the corners mapped back
 * to input indices. A repeated point counts by its first copy in the input.
 * The workspace (>= wg_upper_hood_unsorted_workspace_size(n) bytes) is
 * zero-filled once, as for wg_upper_hood.
 * ---------------------------------------------------------------------- */
size_t wg_sort_points_workspace_size(int64_t n);
wg_status wg_sort_points(const float *points, int64_t n, float *sorted_points,
                         int32_t *perm, void *workspace, size_t ws_bytes,
                         wg_stream_t stream);
size_t wg_upper_hood_unsorted_workspace_size(int64_t n);
wg_status wg_upper_hood_unsorted(const float *points, int64_t n,
                                 int32_t *out_idx, int32_t *out_count,
                                 void *workspace, size_t ws_bytes,
                                 const wg_options *opts, wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Many independent sets in one persistent launch. Set s is
 * points[offsets[s] .. offsets[s+1]) (each set sorted on its own); its
 * corners, as indices local to the set, go to out_idx[offsets[s] ...] and
 * their count to out_counts[s]. Sets are binned by size on the device and
 * taken from a queue by warps, largest first: a set of up to batch_seg_tiles
 * tiles is one warp's item; a larger set is split into segments taken by
 * several warps, and the warp that completes it merges their hoods.
 * offsets   device int64[num_sets + 1], non-decreasing, offsets[0] >= 0
 * h_offsets host copy of the same offsets (only read by the size query)
 * out_idx   device int32[max(offsets[num_sets], 1)], CSR-aligned with points
 * out_counts device int32[max(num_sets, 1)]
 * num_sets  >= 0; empty sets are allowed (count 0)
 * ---------------------------------------------------------------------- */
size_t wg_upper_hood_batched_workspace_size(const int64_t *h_offsets,
                                            int32_t num_sets);
wg_status wg_upper_hood_batched(const float *points, const int64_t *offsets,
                                int32_t num_sets, int32_t *out_idx,
                                int32_t *out_counts, void *workspace,
                                size_t ws_bytes, const wg_options *opts,
                                wg_stream_t stream);

/* ------------------------------------------------------------------------
 * End to end from host memory: copies points (host, ideally pinned) to the
 * caller's device buffer d_points, runs wg_upper_hood_ex, and copies the count
 * and the corners back to h_out_idx / h_out_count. Synchronises `stream`.
 * d_out_idx: device int32[max(n,1)]; d_out_count: device int32[1].
 * If the device recorded an error in the workspace (see wg_get_device_status)
 * that status is returned (and left in the workspace) instead of WG_OK, and
 * the host outputs are not valid.
 * ---------------------------------------------------------------------- */
wg_status wg_upper_hood_from_host(const float *h_points, int64_t n,
                                  int32_t *h_out_idx, int32_t *h_out_count,
                                  float *d_points, int32_t *d_out_idx,
                                  int32_t *d_out_count, void *workspace,
                                  size_t ws_bytes, const wg_options *opts,
                                  wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Diagnostics.
 * wg_get_device_status: synchronises `stream`, returns the first error the
 * device recorded in `workspace` since the last read (WG_OK if none) and
 * clears it.
 * wg_read_counters: synchronises `stream`; returns the orientation tests and
 * float64 fallbacks counted by calls made with count_predicates = 1 since the
 * last read, and clears them.
 * ---------------------------------------------------------------------- */
wg_status wg_get_device_status(void *workspace, wg_stream_t stream);
wg_status wg_read_counters(void *workspace, uint64_t *tests,
                           uint64_t *fallbacks, wg_stream_t stream);
const char *wg_status_string(wg_status status);

/* ------------------------------------------------------------------------
 * Autotuner: times every tile configuration and segment count on the
 * caller's input (which must be a valid input for wg_upper_hood), keeps the
 * fastest for this device and the size bucket of n, and writes it to *best.
 * Later calls with tile_config = 0 use the kept choice for that bucket.
 * Synchronises `stream`; runs each candidate a few times.
 * ---------------------------------------------------------------------- */
wg_status wg_autotune(const float *points, int64_t n, int32_t *out_idx,
                      int32_t *out_count, void *workspace, size_t ws_bytes,
                      wg_options *best, wg_stream_t stream);

/* Autotuner of the batched form: times every tile configuration and the
 * segment caps 16, 32 and 128 tiles on the caller's sets (a valid input for
 * wg_upper_hood_batched, with its workspace), keeps the fastest for this
 * device and writes it to *best. Later batched calls with tile_config = 0
 * and batch_seg_tiles = 0 use the kept choice. Synchronises `stream`. The
 * paper has no counterpart (tuning). */
wg_status wg_autotune_batched(const float *points, const int64_t *offsets,
                              int32_t num_sets, int32_t *out_idx,
                              int32_t *out_counts, void *workspace,
                              size_t ws_bytes, wg_options *best,
                              wg_stream_t stream);

/* ------------------------------------------------------------------------
 * Unit entry points for tests (small sizes; one warp or one CTA).
 * wg_debug_orient: signs[t] = sign(det(p[3t+1] - p[3t], p[3t+2] - p[3t]))
 *   for t < ntri (points device float pairs, signs device int8), plus the
 *   number of float64 fallbacks taken, added to *d_fallbacks (device uint64).
 *   The paper's left_of (Section 2) is signs[t] > 0.
 * wg_debug_bridge: the bridge of two hoods P (hp corners) and Q (hq corners),
 *   P entirely left of Q, each a strictly convex upper chain: writes
 *   d_pq[0] = p, d_pq[1] = q with H(P u Q) = P[0..p] ++ Q[q..] (Section 2,
 *   mam 1-5). hp, hq >= 1. The search that probes the end of P first runs
 *   as well, and so does the small-hood search (one corner per lane) when
 *   hp, hq <= 32; if either disagrees, d_pq = (-1, -1).
 * wg_debug_warp_hood: the hood of m <= 32 sorted distinct points computed by
 *   one warp in registers (stages d = 1..16 of the schedule); writes the
 *   corner positions to d_out[0..h) and h to d_out_count.
 * ---------------------------------------------------------------------- */
wg_status wg_debug_orient(const float *points, int64_t ntri, int8_t *signs,
                          uint64_t *d_fallbacks, int32_t pred_mode,
                          wg_stream_t stream);
wg_status wg_debug_bridge(const float *P, int32_t hp, const float *Q,
                          int32_t hq, int32_t *d_pq, int32_t pred_mode,
                          wg_stream_t stream);
/* wg_debug_bridge_cta: the same bridge by one CTA of 256 threads with the
 *   multi-level bracketing search (the paper's closing section: samples of P
 *   at decreasing intervals, here one corner per warp per round, each with a
 *   32-way search of its tangent corner on Q), for hoods of many thousands of
 *   corners. d_pq[0] = p, d_pq[1] = q. */
wg_status wg_debug_bridge_cta(const float *P, int32_t hp, const float *Q,
                              int32_t hq, int32_t *d_pq, int32_t pred_mode,
                              wg_stream_t stream);
wg_status wg_debug_warp_hood(const float *points, int32_t m, int32_t *d_out,
                             int32_t *d_out_count, int32_t pred_mode,
                             wg_stream_t stream);

/* Test hook for the bounded device waits: with stall_ns > 0, every CTA of
 * later fused calls on this workspace first waits at most stall_ns
 * nanoseconds on a barrier that nothing completes, records WG_ERR_TIMEOUT and
 * exits (no output is written). 0 turns the hook off. Synchronises `stream`.
 * The paper has no counterpart; it exists so that the timeout path can be
 * tested without hanging or faulting a GPU. */
wg_status wg_debug_set_stall(void *workspace, int32_t stall_ns, wg_stream_t stream);

/* ------------------------------------------------------------------------
 * wg_upper_hood_noalloc: the same result as wg_upper_hood, for callers that
 * must not allocate device memory. The paper has no counterpart; it exists
 * for callers such as a plugin that runs inside another program's fixed
 * device-memory budget, a real-time loop that may never block in the
 * allocator, or code that has nowhere to keep a workspace between calls.
 *
 * The caller passes only the input and the outputs (as for wg_upper_hood).
 * The bookkeeping lives in one fixed array (about 3.3 MB) in this library's
 * own device memory, which every GPU that loads the library holds until the
 * process exits. It covers at most 2048 segments, and the call never plans
 * more, so every n from 0 to 2^31 - 1 fits; a larger n is rejected with
 * WG_ERR_UNSUPPORTED, a negative n with WG_ERR_INVALID_VALUE.
 *
 * - The first call on a device looks up the array's device address (with
 *   that device current) and keeps it; make that first call before any
 *   stream capture. The kept address belongs to the device's context: do
 *   not use this entry point after cudaDeviceReset on that device.
 * - Nothing is allocated: no cudaMalloc, cudaFree or allocating library
 *   routine. Each call clears the part of the array that must start at zero
 *   with a cudaMemsetAsync on `stream`, then launches the fused kernel.
 * - All calls in the process share the array. Calls whose GPU work overlaps
 *   (on different streams, or from different threads) race on it and give
 *   wrong results; serialise them.
 * - Only argument and launch errors are returned. The count is set to -1
 *   before the launch, so a call whose device work gave up (a bounded wait
 *   that timed out) leaves a negative count; wg_upper_hood_ex with a
 *   workspace reports such errors by name.
 * ---------------------------------------------------------------------- */
wg_status wg_upper_hood_noalloc(const float *points, int64_t n, int32_t *out_idx,
                                int32_t *out_count, wg_stream_t stream);

/* Library version string. */
const char *wg_version(void);

#ifdef __cplusplus
}
#endif
#endif /* WG_H_ */
