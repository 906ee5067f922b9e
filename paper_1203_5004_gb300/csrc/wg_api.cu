// wg_api.cu -- the extern "C" entry points declared in include/wg.h: argument
// checks, workspace layout, launch planning, the autotuner and diagnostics.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <atomic>
#include <mutex>
#include <vector>

#include "wg.h"
#include "wg_internal.h"
#include "wg_sort.h"

namespace wg {
cudaError_t fused_launch(int cfg, const FusedArgs &args, int grid, int mode, cudaStream_t stream);
cudaError_t fused_occupancy(int cfg, int *blocks);
int fused_tile_points(int cfg);
int fused_warps(int cfg);
size_t fused_smem_bytes(int cfg);
cudaError_t plain_stage_launch(const PlainArgs &a, bool first, int mode, cudaStream_t st);
long long plain_blocks(long long hoods);
cudaError_t batched_launch(const float *points, const int64_t *offsets, int num_sets,
                           int32_t *out_idx, int32_t *out_counts, void *ws, size_t ws_bytes,
                           int cfg, int cap, int mode, int validate, cudaStream_t st);
size_t batched_workspace_bytes(const int64_t *h_offsets, int num_sets);
cudaError_t debug_orient(const float *p, long long ntri, int8_t *signs, unsigned long long *fb,
                         int fp64, cudaStream_t st);
cudaError_t debug_bridge(const float *P, int hp, const float *Q, int hq, int *out, int fp64,
                         cudaStream_t st);
cudaError_t debug_warp_hood(const float *pts, int m, int *out, int *count, int fp64, cudaStream_t st);
cudaError_t debug_bridge_cta(const float *P, int hp, const float *Q, int hq, int *out, int fp64, cudaStream_t st);
cudaError_t hull_turn(const float *points, float *rot, long long n, int sms, cudaStream_t st);
cudaError_t hull_stitch(const float *points, long long n, const int32_t *lidx, const int32_t *lcount, int32_t *out,
                        int32_t *count, int sms, cudaStream_t st);
}  // namespace wg

using namespace wg;

namespace {

// Single-set workspace: header | arrivals | per segment: count, max y,
// final-merge scratch (16 ints), staged hood coordinates and indices
// (kStageCorners), pair word, pair bridge, hood list, list bridges (two
// ints) and output plan (four ints).
constexpr int kMaxSeg = kMaxSegSingle;  // segments of one fused call
constexpr size_t kOffArrivals = 256;
constexpr size_t kOffSegCount = 512;
constexpr size_t kOffSegYmax = kOffSegCount + 4 * kMaxSeg;
constexpr size_t kOffSegLive = kOffSegYmax + 4 * kMaxSeg;
constexpr size_t kOffSegXy = kOffSegLive + 64 * kMaxSeg;
constexpr size_t kOffSegSidx = kOffSegXy + 8 * (size_t)kStageCorners * kMaxSeg;
constexpr size_t kOffSegPair = kOffSegSidx + 4 * (size_t)kStageCorners * kMaxSeg;
constexpr size_t kOffSegBridge = kOffSegPair + 4 * (size_t)kMaxSeg;
constexpr size_t kOffListLid = kOffSegBridge + 8 * (size_t)kMaxSeg;
constexpr size_t kOffListBp = kOffListLid + 4 * (size_t)kMaxSeg;
constexpr size_t kOffListBq = kOffListBp + 4 * (size_t)kMaxSeg;
constexpr size_t kOffPlan = kOffListBq + 4 * (size_t)kMaxSeg;
constexpr size_t kSingleWsBytes = kOffPlan + 16 * (size_t)kMaxSeg;
constexpr int kDefaultCfg = 1;         // single set, before any autotuning (best for small n)
constexpr int64_t kOneCtaMaxN = 1 << 15;  // untuned: one CTA up to this many points
constexpr int kBatchedDefaultCfg = 3;  // batched form, before any autotuning
constexpr int kBatchedDefaultSegTiles = 128;  // batched: tiles per segment of a large set, untuned

struct DevInfo {
    std::atomic<bool> ready{false};  // set (release) once the fields below are filled
    bool init = false;
    bool ok = false;
    int sms = 0;
    int occ[kNumTileCfgs + 1] = {0};
};

std::mutex g_mu;
DevInfo g_dev[64];

// Autotuned choice per device and size bucket floor(log2 n).
// Autotuned choice per device and size bucket, packed in one word so that
// calls read it without a lock: cfg | spc << 8 | sched << 16 (0: not tuned).
std::atomic<int> g_tuned[64][33];
// Batched form, per device: cfg | segment cap << 8 (0: not tuned).
std::atomic<int> g_tuned_batched[64];

inline cudaStream_t S(wg_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

// Device facts, looked up once per device (the first call takes the lock;
// later calls read them without it). *dev_out receives the device number.
wg_status dev_info(DevInfo **out, int *dev_out = nullptr)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WG_ERR_CUDA;
    if (dev_out) *dev_out = dev;
    DevInfo &d = g_dev[dev];
    if (d.ready.load(std::memory_order_acquire)) {
        if (!d.ok) return WG_ERR_UNSUPPORTED;
        *out = &d;
        return WG_OK;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (!d.init) {
        d.init = true;
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return WG_ERR_CUDA;
        d.ok = (prop.major == 10 && prop.minor == 3);
        d.sms = prop.multiProcessorCount;
        for (int c = 1; c <= kNumTileCfgs; ++c) {
            int b = 0;
            if (fused_occupancy(c, &b) != cudaSuccess) {
                cudaGetLastError();
                d.ok = false;
            }
            d.occ[c] = b;
        }
        d.ready.store(true, std::memory_order_release);
    }
    if (!d.ok) return WG_ERR_UNSUPPORTED;
    *out = &d;
    return WG_OK;
}

int bucket(int64_t n)
{
    int b = 0;
    while (b < 32 && (int64_t(1) << (b + 1)) <= n) ++b;
    return b;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

wg_status check_common(const float *points, int64_t n, const void *out_idx, const void *out_count,
                       const void *ws, size_t ws_bytes, size_t need)
{
    if (n < 0) return WG_ERR_INVALID_VALUE;
    if (n > INT32_MAX) return WG_ERR_UNSUPPORTED;
    if (n > 0 && (!points || (reinterpret_cast<uintptr_t>(points) & 7u))) return WG_ERR_INVALID_VALUE;
    if (!out_idx || !out_count) return WG_ERR_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(out_idx) & 3u) || (reinterpret_cast<uintptr_t>(out_count) & 3u))
        return WG_ERR_INVALID_VALUE;
    if (!ws || ws_bytes < need) return WG_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(ws) & 255u) return WG_ERR_INVALID_VALUE;
    return WG_OK;
}

int pred_mode_bits(const wg_options &o)
{
    return (o.pred_mode == WG_PRED_FP64 ? 1 : 0) | (o.count_predicates ? 2 : 0);
}

wg_status check_opts(const wg_options &o)
{
    if (o.pred_mode != WG_PRED_FILTERED && o.pred_mode != WG_PRED_FP64) return WG_ERR_INVALID_VALUE;
    if (o.tile_config < 0 || o.tile_config > kNumTileCfgs) return WG_ERR_INVALID_VALUE;
    if (o.segments_per_cta < 0 || o.segments_per_cta > 8) return WG_ERR_INVALID_VALUE;
    if (o.schedule < 0 || o.schedule > WG_SCHEDULE_SMALL) return WG_ERR_INVALID_VALUE;
    if (o.batch_seg_tiles != 0 && (o.batch_seg_tiles < 8 || o.batch_seg_tiles > 4096)) return WG_ERR_INVALID_VALUE;
    return WG_OK;
}

}  // namespace

extern "C" {

void wg_options_default(wg_options *opts)
{
    if (!opts) return;
    std::memset(opts, 0, sizeof(*opts));
    opts->pred_mode = WG_PRED_FILTERED;
}

const char *wg_version(void) { return "libwagener 0.1 (sm_103a)"; }

const char *wg_status_string(wg_status s)
{
    switch (s) {
    case WG_OK: return "ok";
    case WG_ERR_INVALID_VALUE: return "invalid argument";
    case WG_ERR_WORKSPACE: return "workspace missing or too small";
    case WG_ERR_UNSORTED: return "input not sorted by (x, y)";
    case WG_ERR_OFF_GRID: return "coordinate not on the 2^-24 grid in [0, 1)";
    case WG_ERR_TIMEOUT: return "a bounded device wait timed out";
    case WG_ERR_CUDA: return "CUDA runtime error";
    case WG_ERR_UNSUPPORTED: return "unsupported device or size";
    }
    return "unknown status";
}

size_t wg_upper_hood_workspace_size(int64_t n)
{
    (void)n;
    return kSingleWsBytes;
}

wg_status wg_upper_hood_ex(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                           void *workspace, size_t ws_bytes, const wg_options *opts,
                           wg_stream_t stream)
{
    wg_options o;
    if (opts) o = *opts; else wg_options_default(&o);
    wg_status st = check_opts(o);
    if (st != WG_OK) return st;
    st = check_common(points, n, out_idx, out_count, workspace, ws_bytes, wg_upper_hood_workspace_size(n));
    if (st != WG_OK) return st;
    if (o.schedule == WG_SCHEDULE_SMALL && n > kSmallMaxN) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    int dev = 0;
    st = dev_info(&d, &dev);
    if (st != WG_OK) return st;
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), S(stream)) == cudaSuccess ? WG_OK : WG_ERR_CUDA;

    int cfg = o.tile_config, spc = o.segments_per_cta, sched = o.schedule;
    {
        const int t = g_tuned[dev][bucket(n)].load(std::memory_order_relaxed);
        if (cfg == 0) cfg = (t & 0xff) ? (t & 0xff) : kDefaultCfg;
        if (spc == 0) spc = ((t >> 8) & 0xff) ? ((t >> 8) & 0xff) : 1;
        if (sched == 0) sched = ((t >> 16) & 0xff) ? ((t >> 16) & 0xff)
                                : (n <= kSmallMaxN ? WG_SCHEDULE_SMALL
                                                   : (n <= kOneCtaMaxN ? WG_SCHEDULE_ONE_CTA : WG_SCHEDULE_BALANCED));
        // a tuned choice of the small path covers its bucket only up to the limit
        if (sched == WG_SCHEDULE_SMALL && n > kSmallMaxN) sched = WG_SCHEDULE_BALANCED;
    }
    if (sched == WG_SCHEDULE_SMALL) {
        return small_launch(points, n, out_idx, out_count, workspace, pred_mode_bits(o), o.validate ? 1 : 0,
                            S(stream)) == cudaSuccess
                   ? WG_OK
                   : WG_ERR_CUDA;
    }
    // Segments are claimed dynamically by the warps of one resident wave of
    // CTAs; segments_per_cta scales the number of warps the schedule plans
    // its first, long segments for (more, shorter segments when > 1).
    const int T = fused_tile_points(cfg);
    const int W = fused_warps(cfg);
    const long long tiles = (n + T - 1) / T;
    const int resident = sched == WG_SCHEDULE_ONE_CTA ? 1 : std::max(1, d->occ[cfg]) * d->sms;
    const Schedule sch =
        make_schedule(tiles, (long long)resident * W * spc, kMaxSeg, sched != WG_SCHEDULE_GUIDED);
    const int grid = (int)std::min<long long>(resident, (sch.nseg + W - 1) / W);

    FusedArgs a;
    std::memset(&a, 0, sizeof(a));
    a.points = points;
    a.out_idx = out_idx;
    a.out_count = out_count;
    a.n = n;
    a.tiles = (int)tiles;
    a.nseg = sch.nseg;
    a.sch_n1 = sch.n1;
    a.sch_l1 = sch.l1;
    a.sch_n2 = sch.n2;
    a.sch_l2 = sch.l2;
    a.items = nullptr;
    a.validate = o.validate ? 1 : 0;
    a.hdr = reinterpret_cast<WsHeader *>(workspace);
    a.arrivals = reinterpret_cast<unsigned *>(static_cast<char *>(workspace) + kOffArrivals);
    a.seg_count = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffSegCount);
    a.seg_ymax = reinterpret_cast<float *>(static_cast<char *>(workspace) + kOffSegYmax);
    a.seg_live = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffSegLive);
    a.seg_xy = reinterpret_cast<float *>(static_cast<char *>(workspace) + kOffSegXy);
    a.seg_sidx = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffSegSidx);
    a.seg_pair = reinterpret_cast<unsigned *>(static_cast<char *>(workspace) + kOffSegPair);
    a.seg_bridge = reinterpret_cast<unsigned long long *>(static_cast<char *>(workspace) + kOffSegBridge);
    a.list_lid = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffListLid);
    a.list_bp = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffListBp);
    a.list_bq = reinterpret_cast<int *>(static_cast<char *>(workspace) + kOffListBq);
    a.plan = reinterpret_cast<int4 *>(static_cast<char *>(workspace) + kOffPlan);
    if (fused_launch(cfg, a, grid, pred_mode_bits(o), S(stream)) != cudaSuccess) return WG_ERR_CUDA;
    return WG_OK;
}

wg_status wg_upper_hood(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                        void *workspace, size_t ws_bytes, wg_stream_t stream)
{
    return wg_upper_hood_ex(points, n, out_idx, out_count, workspace, ws_bytes, nullptr, stream);
}

// ------------------------------------------------------------------ convex hull
// Workspace: the single-set workspace | turned points (8n) | lower corners
// (4n) | lower count.
static void hull_layout(int64_t n, size_t *off_rot, size_t *off_lidx, size_t *off_lcnt, size_t *total)
{
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    size_t o = align_up(kSingleWsBytes, 256);
    *off_rot = o;
    o = align_up(o + nn * 8, 256);
    *off_lidx = o;
    o = align_up(o + nn * 4, 256);
    *off_lcnt = o;
    o = align_up(o + 4, 256);
    *total = o;
}

size_t wg_convex_hull_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    size_t a, b, c, t;
    hull_layout(n, &a, &b, &c, &t);
    return t;
}

wg_status wg_convex_hull(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count, void *workspace,
                         size_t ws_bytes, const wg_options *opts, wg_stream_t stream)
{
    if (n < 0) return WG_ERR_INVALID_VALUE;
    wg_status st = check_common(points, n, out_idx, out_count, workspace, ws_bytes, wg_convex_hull_workspace_size(n));
    if (st != WG_OK) return st;
    DevInfo *d = nullptr;
    st = dev_info(&d);
    if (st != WG_OK) return st;
    cudaStream_t s = S(stream);
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
    size_t orot, olidx, olcnt, total;
    hull_layout(n, &orot, &olidx, &olcnt, &total);
    char *w = static_cast<char *>(workspace);
    float *rot = reinterpret_cast<float *>(w + orot);
    int32_t *lidx = reinterpret_cast<int32_t *>(w + olidx);
    int32_t *lcnt = reinterpret_cast<int32_t *>(w + olcnt);
    // upper hood into the caller's output, then the lower hood of the turned
    // points into the workspace (both calls share the single-set workspace)
    if ((st = wg_upper_hood_ex(points, n, out_idx, out_count, workspace, kSingleWsBytes, opts, stream)) != WG_OK)
        return st;
    if (hull_turn(points, rot, n, d->sms, s) != cudaSuccess) return WG_ERR_CUDA;
    if ((st = wg_upper_hood_ex(rot, n, lidx, lcnt, workspace, kSingleWsBytes, opts, stream)) != WG_OK) return st;
    return hull_stitch(points, n, lidx, lcnt, out_idx, out_count, d->sms, s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
}

// ------------------------------------------------------------------ unsorted input
size_t wg_sort_points_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    return sort_workspace_bytes(n);
}

wg_status wg_sort_points(const float *points, int64_t n, float *sorted_points, int32_t *perm, void *workspace,
                         size_t ws_bytes, wg_stream_t stream)
{
    if (n < 0 || n > kSortMaxN) return n < 0 ? WG_ERR_INVALID_VALUE : WG_ERR_UNSUPPORTED;
    if (n == 0) return WG_OK;
    if (!points || !sorted_points || !perm) return WG_ERR_INVALID_VALUE;
    if ((reinterpret_cast<uintptr_t>(points) | reinterpret_cast<uintptr_t>(sorted_points)) & 7u)
        return WG_ERR_INVALID_VALUE;
    if (!workspace || ws_bytes < sort_workspace_bytes(n)) return WG_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    wg_status st = dev_info(&d);
    if (st != WG_OK) return st;
    return sort_launch(points, n, sorted_points, perm, workspace, S(stream)) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
}

// Workspace: the single-set workspace | sorted points (8n) | permutation (4n)
// | the sort's own workspace.
static void unsorted_layout(int64_t n, size_t *off_pts, size_t *off_perm, size_t *off_sort, size_t *total)
{
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    size_t o = align_up(kSingleWsBytes, 256);
    *off_pts = o;
    o = align_up(o + 8 * nn, 256);
    *off_perm = o;
    o = align_up(o + 4 * nn, 256);
    *off_sort = o;
    *total = o + sort_workspace_bytes(n);
}

size_t wg_upper_hood_unsorted_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    size_t a, b, c, t;
    unsorted_layout(n, &a, &b, &c, &t);
    return t;
}

wg_status wg_upper_hood_unsorted(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                                 void *workspace, size_t ws_bytes, const wg_options *opts, wg_stream_t stream)
{
    if (n < 0 || n > kSortMaxN) return n < 0 ? WG_ERR_INVALID_VALUE : WG_ERR_UNSUPPORTED;
    wg_status st =
        check_common(points, n, out_idx, out_count, workspace, ws_bytes, wg_upper_hood_unsorted_workspace_size(n));
    if (st != WG_OK) return st;
    cudaStream_t s = S(stream);
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
    size_t opts_off, operm, osort, total;
    unsorted_layout(n, &opts_off, &operm, &osort, &total);
    char *w = static_cast<char *>(workspace);
    float *sorted = reinterpret_cast<float *>(w + opts_off);
    int32_t *perm = reinterpret_cast<int32_t *>(w + operm);
    if ((st = wg_sort_points(points, n, sorted, perm, w + osort, total - osort, stream)) != WG_OK) return st;
    // corners of the sorted points, then mapped back to input indices
    if ((st = wg_upper_hood_ex(sorted, n, out_idx, out_count, workspace, kSingleWsBytes, opts, stream)) != WG_OK)
        return st;
    return sort_map_launch(out_idx, out_count, perm, n, s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
}

// ------------------------------------------------------------------ plain path
// Workspace: header | two hood buffers (xy, idx) of n corners | two offset
// arrays | look-back words of every stage | tickets of every stage.
static void plain_layout(int64_t n, size_t *off_xy0, size_t *off_xy1, size_t *off_id0, size_t *off_id1,
                         size_t *off_o0, size_t *off_o1, size_t *off_lb, size_t *off_tk, size_t *total,
                         int *stages, long long *lb_words)
{
    int s = 0;
    long long words = 0, h = n;
    while (true) {
        const long long out = (h + 1) / 2;
        words += plain_blocks(out);
        ++s;
        h = out;
        if (h <= 1) break;
    }
    size_t o = 256;
    const size_t nn = (size_t)std::max<int64_t>(n, 1);
    *off_xy0 = o; o = align_up(o + nn * 8, 256);
    *off_xy1 = o; o = align_up(o + nn * 8, 256);
    *off_id0 = o; o = align_up(o + nn * 4, 256);
    *off_id1 = o; o = align_up(o + nn * 4, 256);
    *off_o0 = o; o = align_up(o + (nn / 2 + 2) * 4, 256);
    *off_o1 = o; o = align_up(o + (nn / 2 + 2) * 4, 256);
    *off_lb = o; o = align_up(o + (size_t)words * 8, 256);
    *off_tk = o; o = align_up(o + (size_t)(s + 1) * 4, 256);
    *total = o;
    *stages = s;
    *lb_words = words;
}

size_t wg_upper_hood_plain_workspace_size(int64_t n)
{
    if (n < 0) return 0;
    size_t a, b, c, d, e, f, g, h, t;
    int s;
    long long w;
    plain_layout(n, &a, &b, &c, &d, &e, &f, &g, &h, &t, &s, &w);
    return t;
}

wg_status wg_upper_hood_plain(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                              void *workspace, size_t ws_bytes, const wg_options *opts,
                              wg_stream_t stream)
{
    wg_options o;
    if (opts) o = *opts; else wg_options_default(&o);
    wg_status st = check_opts(o);
    if (st != WG_OK) return st;
    st = check_common(points, n, out_idx, out_count, workspace, ws_bytes,
                      n >= 0 ? wg_upper_hood_plain_workspace_size(n) : 0);
    if (st != WG_OK) return st;
    DevInfo *d = nullptr;
    st = dev_info(&d);
    if (st != WG_OK) return st;
    cudaStream_t s = S(stream);
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;

    size_t oxy[2], oid[2], oo[2], olb, otk, total;
    int stages;
    long long words;
    plain_layout(n, &oxy[0], &oxy[1], &oid[0], &oid[1], &oo[0], &oo[1], &olb, &otk, &total, &stages, &words);
    char *w = static_cast<char *>(workspace);
    if (cudaMemsetAsync(w + olb, 0, (otk - olb) + (size_t)(stages + 1) * 4, s) != cudaSuccess) return WG_ERR_CUDA;

    PlainArgs a;
    std::memset(&a, 0, sizeof(a));
    a.points = points;
    a.n = n;
    a.hdr = reinterpret_cast<WsHeader *>(w);
    long long hoods = n, lb_off = 0;
    int cur = 0;
    for (int stage = 0; stage < stages; ++stage) {
        const long long out = (hoods + 1) / 2;
        a.in_xy = reinterpret_cast<const float *>(w + oxy[cur]);
        a.in_idx = reinterpret_cast<const int32_t *>(w + oid[cur]);
        a.in_off = reinterpret_cast<const int32_t *>(w + oo[cur]);
        a.in_hoods = (int)hoods;
        a.out_xy = reinterpret_cast<float *>(w + oxy[1 - cur]);
        a.out_idx = reinterpret_cast<int32_t *>(w + oid[1 - cur]);
        a.out_off = reinterpret_cast<int32_t *>(w + oo[1 - cur]);
        a.out_hoods = (int)out;
        a.lookback = reinterpret_cast<unsigned long long *>(w + olb) + lb_off;
        a.ticket = reinterpret_cast<unsigned *>(w + otk) + stage;
        a.final_idx = (out == 1) ? out_idx : nullptr;
        a.final_count = (out == 1) ? out_count : nullptr;
        if (plain_stage_launch(a, stage == 0, pred_mode_bits(o), s) != cudaSuccess) return WG_ERR_CUDA;
        lb_off += plain_blocks(out);
        hoods = out;
        cur = 1 - cur;
    }
    return WG_OK;
}

// ------------------------------------------------------------------ batched
size_t wg_upper_hood_batched_workspace_size(const int64_t *h_offsets, int32_t num_sets)
{
    if (num_sets < 0 || (num_sets > 0 && !h_offsets)) return 0;
    return batched_workspace_bytes(h_offsets, num_sets);
}

wg_status wg_upper_hood_batched(const float *points, const int64_t *offsets, int32_t num_sets,
                                int32_t *out_idx, int32_t *out_counts, void *workspace,
                                size_t ws_bytes, const wg_options *opts, wg_stream_t stream)
{
    wg_options o;
    if (opts) o = *opts; else wg_options_default(&o);
    wg_status st = check_opts(o);
    if (st != WG_OK) return st;
    if (num_sets < 0 || (num_sets > 0 && (!offsets || !out_idx || !out_counts))) return WG_ERR_INVALID_VALUE;
    if (points && (reinterpret_cast<uintptr_t>(points) & 7u)) return WG_ERR_INVALID_VALUE;
    if (reinterpret_cast<uintptr_t>(offsets) & 7u) return WG_ERR_INVALID_VALUE;
    if (!workspace) return WG_ERR_WORKSPACE;
    if (reinterpret_cast<uintptr_t>(workspace) & 255u) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    st = dev_info(&d);
    if (st != WG_OK) return st;
    if (num_sets == 0) return WG_OK;
    int dev = 0;
    cudaGetDevice(&dev);
    const int tuned = dev >= 0 && dev < 64 ? g_tuned_batched[dev].load(std::memory_order_relaxed) : 0;
    const int cfg = o.tile_config ? o.tile_config : ((tuned & 0xff) ? (tuned & 0xff) : kBatchedDefaultCfg);
    const int cap = o.batch_seg_tiles ? o.batch_seg_tiles : ((tuned >> 8) ? (tuned >> 8) : kBatchedDefaultSegTiles);
    const cudaError_t e = batched_launch(points, offsets, num_sets, out_idx, out_counts, workspace,
                                         ws_bytes, cfg, cap, pred_mode_bits(o), o.validate, S(stream));
    if (e == cudaErrorInvalidValue) return WG_ERR_WORKSPACE;
    return e == cudaSuccess ? WG_OK : WG_ERR_CUDA;
}

// ------------------------------------------------------------------ host e2e
wg_status wg_upper_hood_from_host(const float *h_points, int64_t n, int32_t *h_out_idx,
                                  int32_t *h_out_count, float *d_points, int32_t *d_out_idx,
                                  int32_t *d_out_count, void *workspace, size_t ws_bytes,
                                  const wg_options *opts, wg_stream_t stream)
{
    if (n < 0 || (n > 0 && (!h_points || !d_points)) || !h_out_idx || !h_out_count)
        return WG_ERR_INVALID_VALUE;
    cudaStream_t s = S(stream);
    if (n > 0 && cudaMemcpyAsync(d_points, h_points, (size_t)n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return WG_ERR_CUDA;
    wg_status st = wg_upper_hood_ex(d_points, n, d_out_idx, d_out_count, workspace, ws_bytes, opts, stream);
    if (st != WG_OK) return st;
    if (cudaMemcpyAsync(h_out_count, d_out_count, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return WG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return WG_ERR_CUDA;
    // an error recorded on the device (a bounded wait that timed out) means
    // the count and corners are not valid: report it instead
    {
        int dst = 0;
        const WsHeader *hh = reinterpret_cast<const WsHeader *>(workspace);
        if (cudaMemcpy(&dst, &hh->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WG_ERR_CUDA;
        if (dst != 0) return static_cast<wg_status>(dst);
    }
    const int32_t h = *h_out_count;
    if (h < 0 || h > std::max<int64_t>(n, 1)) return WG_ERR_CUDA;
    if (h > 0 && cudaMemcpyAsync(h_out_idx, d_out_idx, (size_t)h * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return WG_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return WG_ERR_CUDA;
    return WG_OK;
}

// ------------------------------------------------------------------ diagnostics
wg_status wg_get_device_status(void *workspace, wg_stream_t stream)
{
    if (!workspace) return WG_ERR_INVALID_VALUE;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return WG_ERR_CUDA;
    int v = 0;
    WsHeader *h = reinterpret_cast<WsHeader *>(workspace);
    if (cudaMemcpy(&v, &h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return WG_ERR_CUDA;
    if (v != 0 && cudaMemset(&h->status, 0, sizeof(int)) != cudaSuccess) return WG_ERR_CUDA;
    return static_cast<wg_status>(v);
}

wg_status wg_read_counters(void *workspace, uint64_t *tests, uint64_t *fallbacks, wg_stream_t stream)
{
    if (!workspace || !tests || !fallbacks) return WG_ERR_INVALID_VALUE;
    if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return WG_ERR_CUDA;
    WsHeader *h = reinterpret_cast<WsHeader *>(workspace);
    unsigned long long v[2];
    if (cudaMemcpy(v, &h->tests, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return WG_ERR_CUDA;
    if (cudaMemset(&h->tests, 0, sizeof(v)) != cudaSuccess) return WG_ERR_CUDA;
    *tests = v[0];
    *fallbacks = v[1];
    return WG_OK;
}

wg_status wg_debug_set_stall(void *workspace, int32_t stall_ns, wg_stream_t stream)
{
    if (!workspace || stall_ns < 0) return WG_ERR_INVALID_VALUE;
    WsHeader *h = reinterpret_cast<WsHeader *>(workspace);
    return cudaMemcpyAsync(&h->stall_test_ns, &stall_ns, sizeof(int), cudaMemcpyHostToDevice, S(stream)) ==
                   cudaSuccess && cudaStreamSynchronize(S(stream)) == cudaSuccess
               ? WG_OK
               : WG_ERR_CUDA;
}

wg_status wg_autotune(const float *points, int64_t n, int32_t *out_idx, int32_t *out_count,
                      void *workspace, size_t ws_bytes, wg_options *best, wg_stream_t stream)
{
    if (!best) return WG_ERR_INVALID_VALUE;
    wg_options o;
    wg_options_default(&o);
    wg_status st = check_common(points, n, out_idx, out_count, workspace, ws_bytes,
                                wg_upper_hood_workspace_size(n));
    if (st != WG_OK) return st;
    DevInfo *d = nullptr;
    st = dev_info(&d);
    if (st != WG_OK) return st;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaStream_t s = S(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WG_ERR_CUDA;
    float best_ms = 1e30f;
    int best_cfg = kDefaultCfg, best_spc = 1, best_sched = WG_SCHEDULE_GUIDED;
    const int variants[][2] = {{WG_SCHEDULE_BALANCED, 1}, {WG_SCHEDULE_BALANCED, 2}, {WG_SCHEDULE_GUIDED, 1},
                               {WG_SCHEDULE_ONE_CTA, 1}, {WG_SCHEDULE_SMALL, 1}};
    for (int cfg = 1; cfg <= kNumTileCfgs; ++cfg) {
        for (const auto &var : variants) {
            if (var[0] == WG_SCHEDULE_ONE_CTA && n > (int64_t(1) << 21)) continue;
            // the small path has no tiles: timed once, with the first configuration
            if (var[0] == WG_SCHEDULE_SMALL && (n > kSmallMaxN || cfg != 1)) continue;
            const int spc = var[1];
            o.tile_config = cfg;
            o.segments_per_cta = spc;
            o.schedule = var[0];
            if ((st = wg_upper_hood_ex(points, n, out_idx, out_count, workspace, ws_bytes, &o, stream)) != WG_OK)
                break;
            const int reps = 5;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r)
                wg_upper_hood_ex(points, n, out_idx, out_count, workspace, ws_bytes, &o, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = WG_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best_ms) {
                best_ms = ms;
                best_cfg = cfg;
                best_spc = spc;
                best_sched = var[0];
            }
        }
        if (st != WG_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WG_OK) return st;
    g_tuned[dev][bucket(n)].store(best_cfg | best_spc << 8 | best_sched << 16, std::memory_order_relaxed);
    wg_options_default(best);
    best->tile_config = best_cfg;
    best->segments_per_cta = best_spc;
    best->schedule = best_sched;
    return WG_OK;
}

wg_status wg_autotune_batched(const float *points, const int64_t *offsets, int32_t num_sets, int32_t *out_idx,
                              int32_t *out_counts, void *workspace, size_t ws_bytes, wg_options *best,
                              wg_stream_t stream)
{
    if (!best) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    int dev = 0;
    wg_status st = dev_info(&d, &dev);
    if (st != WG_OK) return st;
    cudaStream_t s = S(stream);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WG_ERR_CUDA;
    wg_options o;
    wg_options_default(&o);
    float best_ms = 1e30f;
    int best_cfg = kBatchedDefaultCfg, best_cap = kBatchedDefaultSegTiles;
    const int caps[] = {16, 32, 128};
    for (int cfg = 1; cfg <= kNumTileCfgs && st == WG_OK; ++cfg) {
        for (int cap : caps) {
            o.tile_config = cfg;
            o.batch_seg_tiles = cap;
            if ((st = wg_upper_hood_batched(points, offsets, num_sets, out_idx, out_counts, workspace, ws_bytes, &o,
                                            stream)) != WG_OK)
                break;
            const int reps = 2;
            cudaEventRecord(e0, s);
            for (int r = 0; r < reps; ++r)
                wg_upper_hood_batched(points, offsets, num_sets, out_idx, out_counts, workspace, ws_bytes, &o, stream);
            cudaEventRecord(e1, s);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                st = WG_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= reps;
            if (ms < best_ms) {
                best_ms = ms;
                best_cfg = cfg;
                best_cap = cap;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WG_OK) return st;
    g_tuned_batched[dev].store(best_cfg | best_cap << 8, std::memory_order_relaxed);
    wg_options_default(best);
    best->tile_config = best_cfg;
    best->batch_seg_tiles = best_cap;
    return WG_OK;
}

// ------------------------------------------------------------------ debug
wg_status wg_debug_orient(const float *points, int64_t ntri, int8_t *signs, uint64_t *d_fallbacks,
                          int32_t pred_mode, wg_stream_t stream)
{
    if (ntri < 0 || (ntri > 0 && (!points || !signs)) || !d_fallbacks) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    wg_status st = dev_info(&d);
    if (st != WG_OK) return st;
    return debug_orient(points, ntri, signs, reinterpret_cast<unsigned long long *>(d_fallbacks),
                        pred_mode == WG_PRED_FP64, S(stream)) == cudaSuccess
               ? WG_OK
               : WG_ERR_CUDA;
}

wg_status wg_debug_bridge(const float *P, int32_t hp, const float *Q, int32_t hq, int32_t *d_pq,
                          int32_t pred_mode, wg_stream_t stream)
{
    if (!P || !Q || !d_pq || hp < 1 || hq < 1) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    wg_status st = dev_info(&d);
    if (st != WG_OK) return st;
    return debug_bridge(P, hp, Q, hq, d_pq, pred_mode == WG_PRED_FP64, S(stream)) == cudaSuccess
               ? WG_OK
               : WG_ERR_CUDA;
}

wg_status wg_debug_bridge_cta(const float *P, int32_t hp, const float *Q, int32_t hq, int32_t *d_pq,
                              int32_t pred_mode, wg_stream_t stream)
{
    if (!P || !Q || !d_pq || hp < 1 || hq < 1) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    wg_status st = dev_info(&d);
    if (st != WG_OK) return st;
    return debug_bridge_cta(P, hp, Q, hq, d_pq, pred_mode == WG_PRED_FP64, S(stream)) == cudaSuccess ? WG_OK
                                                                                                   : WG_ERR_CUDA;
}

wg_status wg_debug_warp_hood(const float *points, int32_t m, int32_t *d_out, int32_t *d_out_count,
                             int32_t pred_mode, wg_stream_t stream)
{
    if (m < 0 || m > 32 || (m > 0 && !points) || !d_out || !d_out_count) return WG_ERR_INVALID_VALUE;
    DevInfo *d = nullptr;
    wg_status st = dev_info(&d);
    if (st != WG_OK) return st;
    return debug_warp_hood(points, m, d_out, d_out_count, pred_mode == WG_PRED_FP64, S(stream)) == cudaSuccess
               ? WG_OK
               : WG_ERR_CUDA;
}

}  // extern "C"
