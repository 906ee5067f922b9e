// wg_small.cu -- the upper hood of a small set (n <= 8192 points) in one
// CTA and one launch, with no wait on any other CTA and no tiles.
//
// The fused kernel's final merge (the grid's hoods joined after a grid-wide
// hand-off) costs a fixed ~15 us of latency whatever n is, which dominates
// small sets. Here one CTA of 512 threads holds the whole set, 16 contiguous
// points per thread in registers, and keeps:
//  1. by height (the rule of the fused kernel's strips): a point goes when
//     every earlier point is at least as high and some later point is
//     strictly higher (it then lies on or below a segment between two input
//     points);
//  2. by the point rules: a repeat of the previous input point goes (first
//     occurrence wins), and so does a point with a strictly higher point
//     directly above it when the point below it is in the same column or it
//     is not in the set's first column;
//  3. rounds of neighbour pruning over the remaining list (shared memory), in
//     input order: an entry p with orient(a, p, b) >= 0 for its list
//     neighbours a and b lies on or below the segment ab between two input
//     points and goes; all of a round's deletions rest on input points, so
//     they are made at once. When a round deletes nothing every interior
//     entry is a strict right turn: the list is a convex chain, the hood.
//     (After kSmRounds rounds the monotone chain finishes the list instead.)
// Results are the same index list as every other path.
#include <cuda_runtime.h>

#include <cstdint>

#include "wg.h"
#include "wg_device.cuh"
#include "wg_internal.h"

namespace wg {

namespace {

constexpr int kSmThreads = 512;
constexpr int kSmWarps = kSmThreads / 32;
constexpr int kSmPPT = 16;  // points per thread
constexpr int kSmRounds = 64;
static_assert((long long)kSmThreads * kSmPPT == kSmallMaxN, "one point slot per input point");

// shared memory: two lists (point, index) of kSmallMaxN entries, a keep
// flag per entry, each thread's first and last point, the block scratch
constexpr size_t kSmCap = (size_t)kSmallMaxN;
constexpr size_t kSmOffXy0 = 0;
constexpr size_t kSmOffXy1 = kSmOffXy0 + 8 * kSmCap;
constexpr size_t kSmOffId0 = kSmOffXy1 + 8 * kSmCap;
constexpr size_t kSmOffId1 = kSmOffId0 + 4 * kSmCap;
constexpr size_t kSmOffFlag = kSmOffId1 + 4 * kSmCap;
constexpr size_t kSmOffFirst = kSmOffFlag + kSmCap;
constexpr size_t kSmOffLast = kSmOffFirst + 8 * (size_t)kSmThreads;
constexpr size_t kSmOffScratch = kSmOffLast + 8 * (size_t)kSmThreads;
constexpr size_t kSmBytes = kSmOffScratch + 4 * (3 * kSmWarps + 8);
static_assert(kSmBytes <= 227 * 1024, "shared memory of one CTA");

struct SmallArgs {
    const float2 *points;
    int n;
    int32_t *out_idx;
    int32_t *out_count;
    WsHeader *hdr;
    int validate;
};

__device__ __forceinline__ float sm_neg_inf() { return __int_as_float(0xff800000); }

// Block-wide exclusive max before and after thread t of v.
__device__ __forceinline__ void block_pre_suf_max(float v, float *wpre, float *wsuf, float &pre, float &suf)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const float ip = warp_incl_prefix_max(v), is = warp_incl_suffix_max(v);
    if (lane == 31) wpre[w] = ip;
    if (lane == 0) wsuf[w] = is;
    __syncthreads();
    float p = __shfl_up_sync(kFull, ip, 1), s = __shfl_down_sync(kFull, is, 1);
    if (lane == 0) p = sm_neg_inf();
    if (lane == 31) s = sm_neg_inf();
    for (int k = 0; k < kSmWarps; ++k) {
        if (k < w) p = fmaxf(p, wpre[k]);
        if (k > w) s = fmaxf(s, wsuf[k]);
    }
    pre = p;
    suf = s;
    __syncthreads();
}

// Block-wide exclusive sum of v before thread t, and the total.
__device__ __forceinline__ int block_excl_sum(int v, int *wsum, int &tot)
{
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int incl = warp_incl_sum(v);
    if (lane == 31) wsum[w] = incl;
    __syncthreads();
    int before = incl - v, all = 0;
    for (int k = 0; k < kSmWarps; ++k) {
        const int a = wsum[k];
        if (k < w) before += a;
        all += a;
    }
    tot = all;
    __syncthreads();
    return before;
}

// Thread t's contiguous share [e0, e1) of m entries.
__device__ __forceinline__ void share(int m, int &e0, int &e1)
{
    const int per = (m + kSmThreads - 1) / kSmThreads;
    e0 = min(m, (int)threadIdx.x * per);
    e1 = min(m, e0 + per);
}

template <int MODE>
__global__ void __launch_bounds__(kSmThreads, 1) small_kernel(SmallArgs a)
{
    extern __shared__ __align__(16) unsigned char smem[];
    float2 *xy[2] = {reinterpret_cast<float2 *>(smem + kSmOffXy0), reinterpret_cast<float2 *>(smem + kSmOffXy1)};
    int *id[2] = {reinterpret_cast<int *>(smem + kSmOffId0), reinterpret_cast<int *>(smem + kSmOffId1)};
    unsigned char *flag = smem + kSmOffFlag;
    float2 *first = reinterpret_cast<float2 *>(smem + kSmOffFirst);
    float2 *last = reinterpret_cast<float2 *>(smem + kSmOffLast);
    float *wpre = reinterpret_cast<float *>(smem + kSmOffScratch);
    float *wsuf = wpre + kSmWarps;
    int *wsum = reinterpret_cast<int *>(wsuf + kSmWarps);

    const int t = threadIdx.x;
    const float2 *P = a.points;
    const int n = a.n;
    const float xfirst = P[0].x;
    PredCount pc;

    // 1. the points, 16 per thread (16-byte loads when the array allows)
    const int i0 = t * kSmPPT;
    const int nv = max(0, min(kSmPPT, n - i0));
    float2 v[kSmPPT];
    if ((reinterpret_cast<uintptr_t>(P) & 15u) == 0 && nv == kSmPPT) {
        const float4 *q = reinterpret_cast<const float4 *>(P + i0);
#pragma unroll
        for (int j = 0; j < kSmPPT / 2; ++j) {
            const float4 f = __ldg(q + j);
            v[2 * j] = make_float2(f.x, f.y);
            v[2 * j + 1] = make_float2(f.z, f.w);
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSmPPT; ++j) v[j] = j < nv ? __ldg(P + i0 + j) : make_float2(0.f, 0.f);
    }
    float tm = sm_neg_inf();
#pragma unroll
    for (int j = 0; j < kSmPPT; ++j)
        if (j < nv) tm = fmaxf(tm, v[j].y);
    if (nv > 0) {
        first[t] = v[0];
        last[t] = v[nv - 1];
    }
    float bpre, bsuf;
    block_pre_suf_max(tm, wpre, wsuf, bpre, bsuf);  // (its barrier also publishes first / last)

    // 2. height rule and point rules
    unsigned keep = 0;
    if (nv > 0) {
        unsigned later_high = 0;  // something strictly higher after the point
        float s = bsuf;
#pragma unroll
        for (int j = kSmPPT - 1; j >= 0; --j) {
            if (j < nv) {
                if (v[j].y < s) later_high |= 1u << j;
                s = fmaxf(s, v[j].y);
            }
        }
        float run = bpre;
        const float2 pv0 = t > 0 ? last[t - 1] : v[0];
        const bool nx_next = i0 + nv < n;  // thread t + 1 holds the next point
        const float2 nxl = nx_next ? first[t + 1] : v[nv - 1];
        int bad = 0;
#pragma unroll
        for (int j = 0; j < kSmPPT; ++j) {
            if (j < nv) {
                const float2 p = v[j];
                const bool hp = i0 + j > 0;
                const float2 pv = j > 0 ? v[j - 1] : pv0;
                const bool hn = j + 1 < nv || nx_next;
                const float2 nx = j + 1 < nv ? v[j + 1] : nxl;
                bool d = !(p.y > run) && ((later_high >> j) & 1u);
                d = d || (hp && same_point(pv, p));
                d = d || (hn && nx.x == p.x && nx.y > p.y && ((hp && pv.x == p.x) || p.x > xfirst));
                keep |= (d ? 0u : 1u) << j;
                run = fmaxf(run, p.y);
                if (a.validate) {
                    const float sx = p.x * 16777216.f, sy = p.y * 16777216.f;
                    if (!(p.x >= 0.f && p.x < 1.f && p.y >= 0.f && p.y < 1.f && sx == truncf(sx) &&
                          sy == truncf(sy)))
                        bad = kStOffGrid;
                    if (hp && (pv.x > p.x || (pv.x == p.x && pv.y > p.y))) bad = bad ? bad : kStUnsorted;
                }
            }
        }
        if (bad) record_status(&a.hdr->status, bad);
    }
    int m;
    {
        int r = block_excl_sum(__popc(keep), wsum, m);
#pragma unroll
        for (int j = 0; j < kSmPPT; ++j) {
            if ((keep >> j) & 1u) {
                xy[0][r] = v[j];
                id[0][r] = i0 + j;
                ++r;
            }
        }
    }
    __syncthreads();

    // 3. pruning rounds, list s -> list 1 - s
    int s = 0;
    bool convex = false;
    for (int round = 0; round < kSmRounds; ++round) {
        int e0, e1;
        share(m, e0, e1);
        const float2 *L = xy[s];
        int cnt = 0;
        if (e0 < e1) {
            float2 pa = e0 > 0 ? L[e0 - 1] : make_float2(0.f, 0.f);
            float2 cu = L[e0];
            for (int e = e0; e < e1; ++e) {
                const bool hn = e + 1 < m;
                const float2 nb = hn ? L[e + 1] : cu;
                const bool drop = e > 0 && hn && orient<MODE>(pc, pa, cu, nb) >= 0;
                flag[e] = drop ? 0 : 1;
                cnt += drop ? 0 : 1;
                pa = cu;
                cu = nb;
            }
        }
        int tot;
        int r = block_excl_sum(cnt, wsum, tot);
        if (tot == m) {
            convex = true;
            break;
        }
        for (int e = e0; e < e1; ++e) {
            if (flag[e]) {
                xy[1 - s][r] = L[e];
                id[1 - s][r] = id[s][e];
                ++r;
            }
        }
        __syncthreads();
        s = 1 - s;
        m = tot;
    }
    if (!convex) {
        // the monotone chain over what is left (one thread)
        if (t == 0) {
            const float2 *L = xy[s];
            const int *Li = id[s];
            float2 *H = xy[1 - s];
            int *Hi = id[1 - s];
            int h = 0;
            for (int e = 0; e < m; ++e) {
                const float2 p = L[e];
                while (h >= 2 && orient<MODE>(pc, H[h - 2], H[h - 1], p) >= 0) --h;
                H[h] = p;
                Hi[h] = Li[e];
                ++h;
            }
            wsum[0] = h;
        }
        __syncthreads();
        m = wsum[0];
        s = 1 - s;
    }

    // output
    for (int e = t; e < m; e += kSmThreads) a.out_idx[e] = id[s][e];
    if (t == 0) a.out_count[0] = m;
    if (MODE & kModeCount) {
        unsigned long long tt = pc.tests, ff = pc.fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            tt += __shfl_xor_sync(kFull, tt, o);
            ff += __shfl_xor_sync(kFull, ff, o);
        }
        if ((t & 31) == 0) {
            atomicAdd(&a.hdr->tests, tt);
            atomicAdd(&a.hdr->fallbacks, ff);
        }
    }
}

template <int MODE>
cudaError_t small_launch_mode(const SmallArgs &a, cudaStream_t stream)
{
    static bool attr = false;  // set once per mode (same value every time, so a race is harmless)
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(small_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmBytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    small_kernel<MODE><<<1, kSmThreads, kSmBytes, stream>>>(a);
    return cudaGetLastError();
}

}  // namespace

cudaError_t small_launch(const float *points, long long n, int32_t *out_idx, int32_t *out_count, void *hdr,
                         int mode, int validate, cudaStream_t stream)
{
    SmallArgs a;
    a.points = reinterpret_cast<const float2 *>(points);
    a.n = (int)n;
    a.out_idx = out_idx;
    a.out_count = out_count;
    a.hdr = static_cast<WsHeader *>(hdr);
    a.validate = validate;
    switch (mode) {
    case 0: return small_launch_mode<0>(a, stream);
    case 1: return small_launch_mode<1>(a, stream);
    case 2: return small_launch_mode<2>(a, stream);
    default: return small_launch_mode<3>(a, stream);
    }
}

}  // namespace wg
