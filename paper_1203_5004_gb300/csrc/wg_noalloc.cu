// wg_noalloc.cu -- wg_upper_hood_noalloc: the fused upper-hood call for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs under a fixed device
// memory budget handed out by someone else (a plugin inside a host
// application, a real-time loop that must never block in the allocator, a
// process whose memory pool is owned and capped by its host), or code that
// simply has no way to keep a workspace alive between calls. This entry
// point needs nothing but the caller's input and output buffers: its
// bookkeeping lives in one fixed array in the library's own device memory,
// sized once for the largest plan the fused kernel makes (at most
// kNoAllocSegments segments).
//
// The array is a file-scope __device__ variable. On the host its name only
// stands for the symbol; the device address is obtained once per device with
// cudaGetSymbolAddress (on the first call that runs on that device, with that
// device current) and passed to the kernel like any other pointer.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "wg.h"
#include "wg_internal.h"

namespace wg {
cudaError_t fused_launch(int cfg, const FusedArgs &args, int grid, int mode, cudaStream_t stream);
cudaError_t fused_occupancy(int cfg, int *blocks);
int fused_tile_points(int cfg);
int fused_warps(int cfg);
}  // namespace wg

using namespace wg;

namespace {

// Layout of the fixed workspace: header (the set's arrival count sits in its
// spare words) | per segment: count, max y, merge scratch (16 ints), staged
// hood coordinates and indices (kStageCorners), pair word, pair bridge.
constexpr int kNoAllocSegments = 2048;
static_assert(kNoAllocSegments <= kMaxSegSingle, "the final merge holds at most kMaxSegSingle segments");
constexpr size_t kNaOffArrivals = offsetof(WsHeader, pad);
constexpr size_t kNaOffCount = 256;
constexpr size_t kNaOffYmax = kNaOffCount + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffLive = kNaOffYmax + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffXy = kNaOffLive + 64 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffSidx = kNaOffXy + 8 * (size_t)kStageCorners * kNoAllocSegments;
constexpr size_t kNaOffPair = kNaOffSidx + 4 * (size_t)kStageCorners * kNoAllocSegments;
constexpr size_t kNaOffBridge = kNaOffPair + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffLid = kNaOffBridge + 8 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffBp = kNaOffLid + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffBq = kNaOffBp + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaOffPlan = kNaOffBq + 4 * (size_t)kNoAllocSegments;
constexpr size_t kNaBytes = kNaOffPlan + 16 * (size_t)kNoAllocSegments;  // about 3.4 MB
// Bytes that every call must see as zero: the status word, the counters and
// the arrival count of the last-segment merge. The call counter after them
// (and the pair words it tags) must survive from call to call.
constexpr size_t kNaZeroBytes = offsetof(WsHeader, epoch);
static_assert(kNaOffArrivals + 4 <= kNaZeroBytes, "arrival count inside the cleared header words");
constexpr int kNaTileCfg = 3;

static __device__ __align__(256) unsigned char g_noalloc_ws[kNaBytes];

static_assert(kNaBytes == kNaOffPlan + 16 * (size_t)kNoAllocSegments, "the fixed layout ends at kNaBytes");
static_assert(16 * kNoAllocSegments >= 13 * kNoAllocSegments + 106,
              "the merge scratch holds the batched merge's arrays for every segment");

// Per device, filled once with that device current: the array's device
// address, the SM count and the resident CTAs per SM.
struct NaDevice {
    void *ws = nullptr;
    int sms = 0;
    int blocks = 0;
    bool ok = false;
};
std::mutex g_na_mu;
NaDevice g_na_dev[64];

inline cudaStream_t S(wg_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

extern "C" wg_status wg_upper_hood_noalloc(const float *points, int64_t n, int32_t *out_idx,
                                           int32_t *out_count, wg_stream_t stream)
{
    if (n < 0) return WG_ERR_INVALID_VALUE;
    if (n > INT32_MAX) return WG_ERR_UNSUPPORTED;
    if (n > 0 && (!points || (reinterpret_cast<uintptr_t>(points) & 7u))) return WG_ERR_INVALID_VALUE;
    if (!out_idx || !out_count || (reinterpret_cast<uintptr_t>(out_idx) & 3u) ||
        (reinterpret_cast<uintptr_t>(out_count) & 3u))
        return WG_ERR_INVALID_VALUE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WG_ERR_CUDA;

    // Set-up, once per device, with that device current: the device address
    // of the fixed array (in host code its name is only a stand-in for the
    // symbol), the device's SM count and the kernel's occupancy.
    NaDevice nd;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        NaDevice &d = g_na_dev[dev];
        if (!d.ws) {
            int major = 0, minor = 0, sms = 0, blocks = 0;
            if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                return WG_ERR_CUDA;
            if (!(major == 10 && minor == 3)) return WG_ERR_UNSUPPORTED;
            if (fused_occupancy(kNaTileCfg, &blocks) != cudaSuccess) return WG_ERR_CUDA;
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_ws) != cudaSuccess || !p) return WG_ERR_CUDA;
            d.sms = sms;
            d.blocks = std::max(1, blocks);
            d.ok = true;
            d.ws = p;
        }
        nd = d;
    }
    void *ws = nd.ws;

    cudaStream_t s = S(stream);
    if (n == 0) return cudaMemsetAsync(out_count, 0, sizeof(int32_t), s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;

    // The array keeps the previous call's contents: clear the part that must
    // start at zero. The count starts at -1, so that a call whose device work
    // gave up (a bounded wait that timed out) leaves a negative count.
    if (cudaMemsetAsync(ws, 0, kNaZeroBytes, s) != cudaSuccess) return WG_ERR_CUDA;
    if (cudaMemsetAsync(out_count, 0xff, sizeof(int32_t), s) != cudaSuccess) return WG_ERR_CUDA;

    const int T = fused_tile_points(kNaTileCfg);
    const int W = fused_warps(kNaTileCfg);
    const long long tiles = (n + T - 1) / T;
    const long long resident = (long long)nd.blocks * nd.sms;
    const Schedule sch = make_schedule(tiles, resident * W, kNoAllocSegments, true);
    const int grid = (int)std::min<long long>(resident, (sch.nseg + W - 1) / W);

    char *w = static_cast<char *>(ws);
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
    a.list_lid = reinterpret_cast<int *>(w + kNaOffLid);
    a.list_bp = reinterpret_cast<int *>(w + kNaOffBp);
    a.list_bq = reinterpret_cast<int *>(w + kNaOffBq);
    a.plan = reinterpret_cast<int4 *>(w + kNaOffPlan);
    a.hdr = reinterpret_cast<WsHeader *>(w);
    a.arrivals = reinterpret_cast<unsigned *>(w + kNaOffArrivals);
    a.seg_count = reinterpret_cast<int *>(w + kNaOffCount);
    a.seg_ymax = reinterpret_cast<float *>(w + kNaOffYmax);
    a.seg_live = reinterpret_cast<int *>(w + kNaOffLive);
    a.seg_xy = reinterpret_cast<float *>(w + kNaOffXy);
    a.seg_sidx = reinterpret_cast<int *>(w + kNaOffSidx);
    a.seg_pair = reinterpret_cast<unsigned *>(w + kNaOffPair);
    a.seg_bridge = reinterpret_cast<unsigned long long *>(w + kNaOffBridge);
    return fused_launch(kNaTileCfg, a, grid, 0, s) == cudaSuccess ? WG_OK : WG_ERR_CUDA;
}
