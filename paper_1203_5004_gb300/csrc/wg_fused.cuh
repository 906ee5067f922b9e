// wg_fused.cuh -- the fused upper-hood kernel (one launch per call).
//
// The paper's stage loop (Section 2, main) merges hoods of size d into hoods
// of size 2d for d = 1, 2, 4, ... with one launch per stage and the hood array
// copied to the host and back every stage. Here the whole schedule runs in one
// persistent launch of warp streams:
//
//  * Every warp owns segments: contiguous ranges of one set, each a whole
//    number of tiles (32 * K points). It streams them through its own
//    shared-memory ring of S tiles, filled by 1-D bulk copies (TMA) and
//    tracked by its own mbarriers, so warps never wait for each other.
//  * Per tile, exact elimination: a point p goes when some earlier point is
//    at least as high and some later point (this tile, or the next tile,
//    already resident) is strictly higher; p then lies on or below a segment
//    between two input points and cannot be a corner. A lane whose whole
//    strip of K points goes learns it from the strip maximum alone. Where
//    many strips survive (points along a sloped curve) the same test runs in
//    the frame sheared by the tile's chord slope, each height an interval
//    that bounds its rounding. A tile inside one column takes the column
//    rule alone. Then the point rules: a repeat of the previous input point
//    goes (first occurrence wins), and so does a point with a strictly
//    higher point directly above it and a point below it in its column or
//    to its left.
//  * The survivors are appended, in input order, to the warp's pending list
//    (several tiles' worth). A full list is flushed: rounds of neighbour
//    pruning (each deletion rests on two input points) until the list is a
//    convex chain, its hood, which one bridge (mam 1-5, probing the running
//    hood's end first) and mam 6 merge into the warp's running segment hood
//    (a shared-memory window of its right end; older corners spill to the
//    output array).
//  * Single set: at the end of a segment the warp publishes the segment hood
//    (indices in the output array; coordinates and indices staged in the
//    workspace when they fit one window), its count and the segment's
//    maximum y. The CTA whose warp finishes last leads the final merge: a
//    staircase of the segment maxima drops whole segments (the same exact
//    rule); the bridges of adjacent listed hoods are found in its shared
//    memory, or by every warp of the grid when the hoods do not fit; hoods
//    that contribute nothing are dropped round by round; the kept ranges are
//    copied to the output.
//  * Batched: warps take items (sets, or segments of large sets) from a
//    queue; the second publisher of two neighbouring segments bridges them,
//    and the warp that publishes a set's last segment merges the set.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "wg_device.cuh"
#include "wg_internal.h"

namespace wg {

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s bound on any device wait
__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

constexpr int kShearLanes = 3;         // more surviving strips than this: shear the tile
constexpr int kShearBackoffLanes = 8;  // after failed trials, skip trials only up to this many
constexpr int kPruneRounds = 16;       // neighbour-pruning rounds of a pending flush before the chain

// The frame in which a tile's points are compared by height: y itself, or
// the sheared y' = (y - y0) - s (x - x0). Shearing keeps every orientation.
// x - x0 and y - y0 are exact for points on the grid; the two other roundings
// are bounded per point, so lo = y' - e <= exact y' <= hi = y' + e with
// e = 2^-22 (|s (x - x0)| + |y'|). With s = 0 all of it is exact and e = 0.
struct Frame {
    float x0, y0, s, ec;
    __device__ __forceinline__ void bounds(float2 v, float &lo, float &hi) const
    {
        const float t = __fmul_rn(s, __fsub_rn(v.x, x0));
        const float yp = __fsub_rn(__fsub_rn(v.y, y0), t);
        const float e = __fmul_rn(__fadd_rn(fabsf(t), fabsf(yp)), ec);
        lo = __fsub_rn(yp, e);
        hi = __fadd_rn(yp, e);
    }
};

// A tile decided in the frame sheared by its chord slope (from its first to
// its last point), for tiles where the plain height test leaves many strips:
// points along a sloped curve. Heights are intervals (see Frame): a strip goes
// when the lows before it reach its high and a low after it exceeds its high;
// inside a strip each point is tested the same way. The frame is kept only if
// fewer strips survive than the plain test's `live_plain`. Returns the lane's
// mask of remaining points in the low 32 bits and 1 in bit 32 when the frame
// is kept (warp-uniform), 0 otherwise. The strip's bounds are computed once
// and kept in registers for the three passes. Any slope gives an exact test
// (the bounds cover the roundings for the slope actually used), so the chord
// slope is taken from a fast division.
template <int K>
__device__ __forceinline__ unsigned long long sheared_tile(const float2 *tb, int cnt, int nvalid, int live_plain,
                                                          float2 prev_pt, bool has_prev)
{
    const int lane = threadIdx.x & 31;
    const int sbase = lane * K;
    const float2 f0 = tb[0], f1 = tb[cnt - 1];
    float sl = f1.x > f0.x ? __fdividef(f1.y - f0.y, f1.x - f0.x) : 0.f;
    if (!(fabsf(sl) < 1e6f)) sl = 0.f;
    const Frame f{f0.x, f0.y, sl, sl != 0.f ? 0x1p-22f : 0.f};
    float lo[K], hi[K];
    float mlo = neg_inf(), mhi = neg_inf();
#pragma unroll
    for (int j = 0; j < K; ++j) {
        lo[j] = neg_inf();
        hi[j] = neg_inf();
        if (j < nvalid) {
            f.bounds(tb[sbase + j], lo[j], hi[j]);
            mlo = fmaxf(mlo, lo[j]);
            mhi = fmaxf(mhi, hi[j]);
        }
    }
    float carry = neg_inf();
    if (has_prev) {
        float h;
        f.bounds(prev_pt, carry, h);
    }
    const float jpre = warp_incl_prefix_max(mlo);
    const float jsuf = warp_incl_suffix_max(mlo);
    float pre = __shfl_up_sync(kFull, jpre, 1);
    float suf = __shfl_down_sync(kFull, jsuf, 1);
    if (lane == 0) pre = neg_inf();
    if (lane == 31) suf = neg_inf();
    const float pm0 = fmaxf(carry, pre);
    const bool dead = !(mhi > pm0) && mhi < suf;
    const unsigned live = __ballot_sync(kFull, !dead && nvalid > 0);
    if (__popc(live) >= live_plain) return 0ull;
    unsigned surv = 0;
    if (!dead && nvalid > 0) {
        unsigned kpre = 0;
        float pm = pm0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            kpre |= (hi[j] <= pm ? 1u : 0u) << j;
            pm = fmaxf(pm, lo[j]);
        }
        float smx = suf;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            if (!(((kpre >> j) & 1u) && hi[j] < smx)) surv |= 1u << j;
            smx = fmaxf(smx, lo[j]);
        }
        surv &= nvalid >= K ? (K == 32 ? kFull : ((1u << K) - 1u)) : ((1u << nvalid) - 1u);
    }
    return (1ull << 32) | surv;
}


template <int W, int K, int S, int RCAP, int PCAP>
struct Cfg {
    static constexpr int kW = W, kNT = W * 32, kK = K, kT = 32 * K, kS = S;
    static constexpr int kRCap = RCAP, kPCap = PCAP;
    static constexpr int kBuf = kT + 2;  // points per tile buffer (+2: alignment shift)
    // per-warp region
    static constexpr size_t kOffTiles = 0;
    static constexpr size_t kOffPxy = kOffTiles + size_t(S) * kBuf * 8;
    static constexpr size_t kOffPidx = kOffPxy + size_t(PCAP) * 8;
    static constexpr size_t kOffRxy = kOffPidx + size_t(PCAP) * 4;
    static constexpr size_t kOffRidx = kOffRxy + size_t(RCAP) * 8;
    static constexpr size_t kOffMeta = kOffRidx + size_t(RCAP) * 4;  // per ring slot: tile start, count, flags
    static constexpr size_t kOffBar = kOffMeta + size_t(S) * 16;
    static constexpr size_t kWarpBytes = ((kOffBar + 8 * (S + 1)) + 127) / 128 * 128;
    // after the warp regions: one CTA word (the item whose merge this CTA runs)
    static constexpr size_t kBytes = kWarpBytes * W + 128;
    static_assert(K % 2 == 1 && K < 32, "K must be odd (bank-conflict-free strips) and < 32");
    static_assert(S >= 3, "three tile buffers: current, look-ahead, in flight");
    static_assert(RCAP % 64 == 0 && PCAP % 32 == 0 && PCAP >= 64 && PCAP <= 256, "window / list sizes");
    static_assert(kT % 2 == 0, "even tile");
    static_assert(RCAP == kStageCorners, "staged segment hoods hold one window");
};

// Running hood: corners [0, g) live in the output array (indices only), corners
// [g, g + w) in the shared window (coordinates and indices).
struct RState {
    int g, w;
    int32_t *gout;
    const float2 *pts;
};

struct RunAcc {
    const float2 *wxy;
    int g;
    const int32_t *gidx;
    const float2 *pts;
    __device__ __forceinline__ float2 pt(int i) const
    {
        if (i >= g) return wxy[i - g];
        return pts[gidx[i]];
    }
};

// Workspace pointers of the fused kernel.
struct SegStore {
    int *count;      // per slot: corners of the segment hood
    float *ymax;     // per slot: max y over the segment's points
    float2 *xy;      // per stage slot: coordinates of the hood (RCAP each), if it fit the window
    int *sidx;       // per stage slot: indices of the hood (RCAP each), staged with xy
    int *live;       // per stage slot: scratch of the final merge (16 ints each)
    unsigned *pair;  // per stage slot: publication tag of the pair (this, next)
    unsigned long long *bridge;  // per stage slot: bridge of the pair (this, next), tagged
};

// Tags of one call: the workspace's call counter + 1, mixed with a constant
// so that no other word of any workspace layout can equal a tag.
constexpr unsigned kTagMix = 0x9E3779B9u;

template <class C, int MODE>
struct Warp {
    const FusedArgs &args;
    unsigned char *base;  // this warp's region
    PredCount pc;
    int lane;
    int pn;               // corners in the pending list
    float xfirst;         // x of the set's first point (column rule)
    int sh_skip, sh_fail;  // sheared-frame trials: tiles to skip, failures in a row
    unsigned tag;          // this call's tag (pair words, pair bridges)

    __device__ Warp(const FusedArgs &a, unsigned char *b) : args(a), base(b), pn(0) { lane = threadIdx.x & 31; }

    __device__ float2 *buf(int b) const { return reinterpret_cast<float2 *>(base + C::kOffTiles) + size_t(b) * C::kBuf; }
    __device__ float2 *pxy() const { return reinterpret_cast<float2 *>(base + C::kOffPxy); }
    __device__ int *pidx() const { return reinterpret_cast<int *>(base + C::kOffPidx); }
    __device__ float2 *rxy() const { return reinterpret_cast<float2 *>(base + C::kOffRxy); }
    __device__ int *ridx() const { return reinterpret_cast<int *>(base + C::kOffRidx); }
    __device__ uint64_t *bars() const { return reinterpret_cast<uint64_t *>(base + C::kOffBar); }
    __device__ int4 *meta() const { return reinterpret_cast<int4 *>(base + C::kOffMeta); }

    // ------------------------------------------------------------------ items
    __device__ SegItem item(int i) const
    {
        if (args.items) return args.items[i];
        SegItem it;
        it.set_base = 0;
        it.a = seg_a(i);
        it.b = seg_b(i);
        it.set = 0;
        it.c = i;
        it.nseg = args.nseg;
        it.slot = i;
        it.slot0 = 0;
        it.pad = i;  // stage slot
        return it;
    }

    // Single set: point range [seg_a(c), seg_b(c)) of segment c.
    __device__ long long seg_a(int c) const
    {
        return schedule_tile0(args.sch_n1, args.sch_l1, args.sch_n2, args.sch_l2, args.tiles, c) * C::kT;
    }
    __device__ long long seg_b(int c) const
    {
        const long long e = seg_a(c + 1);
        return e < args.n ? e : args.n;
    }

    __device__ SegStore store() const
    {
        SegStore s;
        s.count = args.seg_count;
        s.ymax = args.seg_ymax;
        s.xy = reinterpret_cast<float2 *>(args.seg_xy);
        s.sidx = args.seg_sidx;
        s.live = args.seg_live;
        s.pair = args.seg_pair;
        s.bridge = args.seg_bridge;
        return s;
    }

    // ------------------------------------------------------- tile staging
    // Tile k of segment [a, b) of set points P goes to buffer (seq % S). The
    // 16-byte-aligned interior is one bulk copy; at most one point at each end
    // (when the tile start or end is not 16-byte aligned) is a plain load,
    // made visible by the release semantics of the mbarrier arrive. Lane 0.
    __device__ void issue(const float2 *P, long long a, long long b, int k, unsigned seq) const
    {
        const int bi = seq % C::kS;
        uint64_t *bar = bars() + bi;
        const long long start = a + (long long)k * C::kT;
        const long long rem = b - start;
        const int cnt = rem < C::kT ? (int)rem : C::kT;
        const float2 *src = P + start;
        const int shift = (int)((reinterpret_cast<uintptr_t>(src) >> 3) & 1);
        float2 *dst = buf(bi);
        const int nint = cnt > shift ? ((cnt - shift) & ~1) : 0;
        if (shift && cnt > 0) dst[1] = src[0];
        const int tail = shift + nint;
        if (tail < cnt) dst[shift + tail] = src[tail];
        if (nint > 0) {
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(bar, (unsigned)nint * 8u);
            bulk_g2s_hint(dst + 2 * shift, src + shift, (unsigned)nint * 8u, bar, l2_evict_first_policy());
        } else {
            mbar_arrive(bar);
        }
    }

    __device__ static int tile_shift(const float2 *P, long long start)
    {
        return (int)((reinterpret_cast<uintptr_t>(P + start) >> 3) & 1);
    }

    // ------------------------------------------------------- running hood
    __device__ __forceinline__ void r_flush_half(RState &R) const
    {
        constexpr int F = C::kRCap / 2;
        int *ri = ridx();
        float2 *rx = rxy();
        for (int k = lane; k < F; k += 32) R.gout[R.g + k] = ri[k];
        __syncwarp();
        const int rest = R.w - F;
        for (int b0 = 0; b0 < rest; b0 += 32) {
            const int k = b0 + lane;
            float2 v = make_float2(0.f, 0.f);
            int id = 0;
            if (k < rest) {
                v = rx[F + k];
                id = ri[F + k];
            }
            __syncwarp();
            if (k < rest) {
                rx[k] = v;
                ri[k] = id;
            }
            __syncwarp();
        }
        R.g += F;
        R.w = rest;
    }

    // Corner i of the running hood.
    __device__ __forceinline__ float2 r_pt(const RState &R, int i) const
    {
        return i >= R.g ? rxy()[i - R.g] : R.pts[R.gout[i]];
    }

    // Brings the last spilled corners back into the window (when pops have
    // nearly emptied it): indices from the output array, coordinates from
    // the input.
    __device__ void r_refill(RState &R) const
    {
        const int k = min(R.g, C::kRCap / 2);
        float2 v = make_float2(0.f, 0.f);
        int id = 0;
        if (lane < R.w) {
            v = rxy()[lane];
            id = ridx()[lane];
        }
        __syncwarp();
        if (lane < R.w) {
            rxy()[k + lane] = v;
            ridx()[k + lane] = id;
        }
        for (int t = lane; t < k; t += 32) {
            const int gi = R.gout[R.g - k + t];
            ridx()[t] = gi;
            rxy()[t] = R.pts[gi];
        }
        __syncwarp();
        R.g -= k;
        R.w += k;
    }

    // Append H[from..to) (coordinates and indices) to the running hood.
    __device__ void r_append(RState &R, const float2 *hxy, const int *hid, int from, int to) const
    {
        int done = from;
        while (done < to) {
            if (R.w == C::kRCap) r_flush_half(R);
            const int n = min(to - done, C::kRCap - R.w);
            for (int k = lane; k < n; k += 32) {
                rxy()[R.w + k] = hxy[done + k];
                ridx()[R.w + k] = hid[done + k];
            }
            R.w += n;
            done += n;
            __syncwarp();
        }
    }

    // Merge hood H (h >= 1 corners, all right of the running hood) into it:
    // the bridge (p, q) of the two hoods (mam 1-5, probing the running
    // hood's last corners first), then R = R[0..p] ++ H[q..h) (mam 6).
    __device__ void r_merge(RState &R, const float2 *hxy, const int *hid, int h)
    {
        if (R.g + R.w == 0) {
            r_append(R, hxy, hid, 0, h);
            return;
        }
        const RunAcc ra{rxy(), R.g, R.gout, R.pts};
        const int2 pq = bridge_tail<MODE>(pc, ra, R.g + R.w, PtrHood{hxy}, h);
        if (pq.x < R.g) {
            R.g = pq.x + 1;
            R.w = 0;
        } else {
            R.w = pq.x + 1 - R.g;
        }
        __syncwarp();
        r_append(R, hxy, hid, pq.y, h);
    }

    // Monotone-chain pushes of the listed points (in input order) onto the
    // running hood: before a point b is pushed, the top corner a (with o
    // below it) is popped while orient(o, a, b) >= 0, i.e. while a is not a
    // strict right turn. Every lane runs the same steps and stores the same
    // values, so the window needs no synchronisation between them.
    __device__ void r_push(RState &R, const float2 *L, const int *Lid, int m)
    {
        int h = R.g + R.w;
        float2 A = make_float2(0.f, 0.f), B = A;
        if (h >= 1) B = r_pt(R, h - 1);
        if (h >= 2) A = r_pt(R, h - 2);
        for (int e = 0; e < m; ++e) {
            const float2 p = L[e];
            while (h >= 2 && orient<MODE>(pc, A, B, p) >= 0) {
                --h;
                if (R.w > 0) --R.w; else --R.g;
                B = A;
                if (h >= 2) {
                    if (R.w < 2 && R.g > 0) r_refill(R);
                    A = r_pt(R, h - 2);
                }
            }
            if (R.w == C::kRCap) r_flush_half(R);
            rxy()[R.w] = p;
            ridx()[R.w] = Lid[e];
            ++R.w;
            ++h;
            A = B;
            B = p;
        }
        __syncwarp();
    }

    // --------------------------------------------- merge of the pending list
    // The pending list holds candidate points in input order, all distinct.
    // Rounds of neighbour pruning, in parallel: a live entry p whose nearest
    // live neighbours a (before; the running hood's last corner for the
    // first entry) and b (after) satisfy orient(a, p, b) >= 0 lies on or
    // below the segment between two input points a <lex p <lex b, so it is
    // not a corner. Every deletion rests on input points, so a round's
    // deletions may all be made at once. When a round deletes nothing, every
    // live entry is a strict right turn between its neighbours: the live
    // entries form a convex chain, the hood of the list (the paper's stages
    // over these points, reached by local tests), and it is merged into the
    // running hood by one bridge (mam 1-5) and mam 6. The survivors are
    // packed after every round, so that an entry's live neighbours are the
    // adjacent entries (a shuffle each) and later rounds touch only the
    // groups of 32 still occupied. If the rounds run out first, the
    // survivors are pushed one by one by the monotone chain instead.
    __device__ __forceinline__ void flush_pending(RState &R)
    {
        constexpr int Q = C::kPCap / 32;
        int m = pn;
        pn = 0;
        if (m == 0) return;
        float2 *L = pxy();
        int *Lid = pidx();
        const int h0 = R.g + R.w;
        const bool anchor = h0 >= 1;
        const float2 Bv = anchor ? r_pt(R, h0 - 1) : make_float2(0.f, 0.f);
        bool convex = false;
        for (int round = 0; round < kPruneRounds; ++round) {
            // the live entries are L[0, m), packed: entry e's neighbours are
            // e - 1 (the running hood's last corner for e = 0) and e + 1
            const int nq = (m + 31) >> 5;
            float2 mine[Q];
            int mid[Q];
            unsigned keep[Q];
            unsigned any = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                keep[q] = 0;
                if (q < nq) {
                    const int e = q * 32 + lane;
                    const bool in = e < m;
                    mine[q] = in ? L[e] : make_float2(0.f, 0.f);
                    mid[q] = in ? Lid[e] : 0;
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (q < nq) {
                    const int e = q * 32 + lane;
                    const bool in = e < m;
                    float2 a = shfl2(mine[q], (lane + 31) & 31);
                    const float2 aw = q > 0 ? shfl2(mine[q > 0 ? q - 1 : 0], 31) : Bv;
                    if (lane == 0) a = aw;
                    float2 b = shfl2(mine[q], (lane + 1) & 31);
                    const float2 bw = q + 1 < nq ? shfl2(mine[q + 1 < Q ? q + 1 : q], 0) : b;
                    if (lane == 31) b = bw;
                    const bool d = in && (e > 0 || anchor) && e + 1 < m && orient<MODE>(pc, a, mine[q], b) >= 0;
                    const unsigned dead = __ballot_sync(kFull, d);
                    any |= dead;
                    keep[q] = __ballot_sync(kFull, in) & ~dead;
                }
            }
            if (!any) {
                convex = true;
                break;
            }
            // pack the survivors to the front of the list, in order
            __syncwarp();
            int base = 0;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                if (q < nq) {
                    if ((keep[q] >> lane) & 1u) {
                        const int r = base + __popc(keep[q] & ((1u << lane) - 1u));
                        L[r] = mine[q];
                        Lid[r] = mid[q];
                    }
                    base += __popc(keep[q]);
                }
            }
            __syncwarp();
            m = base;
        }
        if (convex && m > 1)
            r_merge(R, L, Lid, m);
        else
            r_push(R, L, Lid, m);
    }

    // Per-point elimination in one strip (not all dropped), by height: a
    // point goes when everything before it reaches its height and something
    // after it is strictly higher. pm0 / sm0: max height before / after the
    // strip. Returns the mask of the strip's points that remain.
    __device__ __forceinline__ unsigned elim_plain(const float2 *tb, int sbase, int nvalid, float pm0,
                                                   float sm0) const
    {
        constexpr int K = C::kK;
        float py[K];
#pragma unroll
        for (int j = 0; j < K; ++j) py[j] = j < nvalid ? tb[sbase + j].y : neg_inf();
        unsigned kpre = 0;
        float pm = pm0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            kpre |= (py[j] <= pm ? 1u : 0u) << j;
            pm = fmaxf(pm, py[j]);
        }
        unsigned surv = 0;
        float smx = sm0;
#pragma unroll
        for (int j = K - 1; j >= 0; --j) {
            if (!(((kpre >> j) & 1u) && py[j] < smx)) surv |= 1u << j;
            smx = fmaxf(smx, py[j]);
        }
        surv &= nvalid >= K ? ((1u << K) - 1u) : ((1u << nvalid) - 1u);
        return surv;
    }

    // First occurrence and the column rule on the strip's remaining points
    // (surv): a repeat of the previous input point goes (first occurrence
    // wins), and so does a point with a strictly higher point directly above
    // it when the point below it is in the same column (three collinear
    // points) or some point lies further left (it is then strictly below the
    // segment from the set's first point to the point above).
    __device__ __forceinline__ unsigned point_rules(const float2 *tb, int sbase, int nvalid, unsigned surv,
                                                    float2 prev_pt, bool has_prev) const
    {
        unsigned out = surv;
        while (surv) {
            const int j = __ffs(surv) - 1;
            surv &= surv - 1;
            const float2 Pj = tb[sbase + j];
            float2 pv = prev_pt;
            bool hv = has_prev;
            if (sbase + j > 0) {
                pv = tb[sbase + j - 1];
                hv = true;
            }
            bool drop = hv && same_point(pv, Pj);
            if (!drop && j + 1 < nvalid) {
                const float2 nx = tb[sbase + j + 1];
                drop = nx.x == Pj.x && nx.y > Pj.y && ((hv && pv.x == Pj.x) || Pj.x > xfirst);
            }
            if (drop) out &= ~(1u << j);
        }
        return out;
    }

    // The rules of point_rules for a strip of a tile that lies in one column
    // (every x equal), over the whole strip in one unrolled pass on the y's:
    // a repeat of the previous point goes, and so does a point with a higher
    // point next (in the tile) when its previous point is in the column too or
    // the column is not the set's first. The height rule is not applied: in
    // the set's first column every point is a new height maximum, and the
    // column rule leaves about one point per tile.
    __device__ __forceinline__ unsigned column_rules(const float2 *tb, int sbase, int nvalid, float2 prev_pt,
                                                     bool has_prev) const
    {
        constexpr int K = C::kK;
        const float x = tb[sbase].x;
        const float2 p0 = sbase > 0 ? tb[sbase - 1] : prev_pt;
        bool same_col = (sbase > 0 || has_prev) && p0.x == x;
        float yp = p0.y;
        float yc = tb[sbase].y;
        const bool later_col = x > xfirst;
        unsigned out = 0;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (j < nvalid) {
                const bool hn = j + 1 < nvalid;
                const float yn = hn ? tb[sbase + j + 1].y : yc;
                const bool repeat = same_col && yp == yc;
                const bool up = hn && yn > yc;
                if (!(repeat || (up && (same_col || later_col)))) out |= 1u << j;
                same_col = true;
                yp = yc;
                yc = yn;
            }
        }
        return out;
    }

    __device__ __forceinline__ void validate_strip(const float2 *tb, int sbase, int nvalid, float2 prev_pt,
                                                bool has_prev) const
    {
        int bad = 0;
        for (int j = 0; j < nvalid && j < C::kK; ++j) {
            const float2 v = tb[sbase + j];
            const float sx = v.x * 16777216.f, sy = v.y * 16777216.f;
            if (!(v.x >= 0.f && v.x < 1.f && v.y >= 0.f && v.y < 1.f && sx == truncf(sx) && sy == truncf(sy)))
                bad = kStOffGrid;
            float2 pv = prev_pt;
            bool hv = has_prev;
            if (sbase + j > 0) {
                pv = tb[sbase + j - 1];
                hv = true;
            }
            if (hv && (pv.x > v.x || (pv.x == v.x && pv.y > v.y))) bad = bad ? bad : kStUnsorted;
        }
        if (bad) record_status(&args.hdr->status, bad);
    }

    // Max y over this lane's strip of a tile.
    __device__ __forceinline__ float strip_max(const float2 *tb, int cnt) const
    {
        const int sbase = lane * C::kK;
        float ym = neg_inf();
        if (sbase + C::kK <= cnt) {
            float m0 = neg_inf(), m1 = neg_inf();
#pragma unroll
            for (int j = 0; j + 1 < C::kK; j += 2) {
                m0 = fmaxf(m0, tb[sbase + j].y);
                m1 = fmaxf(m1, tb[sbase + j + 1].y);
            }
            ym = fmaxf(fmaxf(m0, m1), tb[sbase + C::kK - 1].y);
        } else {
            for (int j = 0; sbase + j < cnt; ++j) ym = fmaxf(ym, tb[sbase + j].y);
        }
        return ym;
    }

    // ------------------------------------------------ one tile, decided
    // Tile at tb (cnt points, the first at set-relative index `start`);
    // ymax_mine = max y of this lane's strip, tmax = max y of the tile, ynext
    // = max y of the look-ahead tile (or -inf). Survivor corners go to the
    // pending list.
    __device__ __forceinline__ void decide(const float2 *tb, int cnt, long long start, float ymax_mine, float tmax,
                                           float ynext, float &pm_carry, float2 &prev_pt, bool &has_prev,
                                           RState &R)
    {
        constexpr int K = C::kK;
        const int sbase = lane * K;
        const int nvalid = cnt - sbase;
        // Whole strip dropped: everything before it is at least as high as its
        // maximum (pm0), and something after it is strictly higher (sm0).
        float pm0, sm0;
        if (tmax <= pm_carry) {
            // the tile's own earlier strips add nothing to pm_carry
            pm0 = pm_carry;
            if (tmax < ynext) {
                sm0 = ynext;
            } else {
                const float isuf = warp_incl_suffix_max(ymax_mine);
                float esuf = __shfl_down_sync(kFull, isuf, 1);
                if (lane == 31) esuf = neg_inf();
                sm0 = fmaxf(esuf, ynext);
            }
        } else {
            const float ipre = warp_incl_prefix_max(ymax_mine);
            const float isuf = warp_incl_suffix_max(ymax_mine);
            float epre = __shfl_up_sync(kFull, ipre, 1);
            float esuf = __shfl_down_sync(kFull, isuf, 1);
            if (lane == 0) epre = neg_inf();
            if (lane == 31) esuf = neg_inf();
            pm0 = fmaxf(pm_carry, epre);
            sm0 = fmaxf(esuf, ynext);
        }
        const bool dead = !(ymax_mine > pm0) && ymax_mine < sm0;
        const unsigned live = __ballot_sync(kFull, !dead && nvalid > 0);
        unsigned surv = 0;
        if (live && __popc(live) > 1 && tb[0].x == tb[cnt - 1].x) {
            // The tile lies in one column.
            if (!dead && nvalid > 0) surv = column_rules(tb, sbase, nvalid, prev_pt, has_prev);
        } else if (live) {
            bool sheared = false;
            if (sh_skip > 0 && __popc(live) <= kShearBackoffLanes) {
                --sh_skip;
            } else if (__popc(live) > kShearLanes) {
                // Many strips survive: try the sheared frame. After a trial
                // that does not pay, skip the next 2, 4, ... 64 tiles' trials
                // that leave at most kShearBackoffLanes strips.
                const unsigned long long r = sheared_tile<K>(tb, cnt, nvalid, __popc(live), prev_pt, has_prev);
                if (r >> 32) {
                    sheared = true;
                    surv = (unsigned)r;
                    sh_fail = 0;
                } else {
                    sh_fail = min(sh_fail + 1, 6);
                    sh_skip = 1 << sh_fail;
                }
            }
            if (!sheared && __popc(live) == 1) {
                // One strip survives: the whole warp tests its points, one per lane.
                const int L = __ffs(live) - 1;
                const unsigned S = strip_survivors_warp(tb, cnt, L, __shfl_sync(kFull, pm0, L),
                                                        __shfl_sync(kFull, sm0, L), prev_pt, has_prev);
                if (lane == L) surv = S;
            } else {
                if (!sheared && !dead && nvalid > 0) surv = elim_plain(tb, sbase, nvalid, pm0, sm0);
                if (surv) surv = point_rules(tb, sbase, nvalid, surv, prev_pt, has_prev);
            }
        }
        if (args.validate && nvalid > 0) validate_strip(tb, sbase, nvalid, prev_pt, has_prev);

        pm_carry = fmaxf(pm_carry, tmax);
        prev_pt = tb[cnt - 1];
        has_prev = true;

        // The remaining points go to the pending list, in input order.
        const unsigned with = __ballot_sync(kFull, surv != 0);
        if (!with) return;
        const int hc = __popc(surv);
        const int incl = warp_incl_sum(hc);
        const int m = __shfl_sync(kFull, incl, 31);
        const int rank0 = incl - hc;
        for (int r0 = 0; r0 < m;) {
            if (pn == C::kPCap) flush_pending(R);
            const int take = min(C::kPCap - pn, m - r0);
            if (surv && rank0 < r0 + take && rank0 + hc > r0) {
                int r = rank0;
                unsigned bits = surv;
                while (bits) {
                    const int j = __ffs(bits) - 1;
                    bits &= bits - 1;
                    if (r >= r0 && r < r0 + take) {
                        pxy()[pn + r - r0] = tb[sbase + j];
                        pidx()[pn + r - r0] = (int)(start + sbase + j);
                    }
                    ++r;
                }
            }
            __syncwarp();
            pn += take;
            r0 += take;
        }
    }

    // Survivors of strip L of a tile (the only strip not dropped whole),
    // tested by the whole warp, lane j holding the strip's point j: the
    // height rule (pm0 / sm0: max height before / after the strip), first
    // occurrence and the column rule, as elim_plain and point_rules apply
    // them. Returns the mask of the strip's remaining points (all lanes).
    __device__ __forceinline__ unsigned strip_survivors_warp(const float2 *tb, int cnt, int L, float pm0,
                                                             float sm0, float2 prev_pt, bool has_prev) const
    {
        constexpr int K = C::kK;
        const float nan = __int_as_float(0x7fffffff);
        const int sb = L * K;
        const int nv = min(K, cnt - sb);
        const bool mine = lane < nv;
        const float2 q = mine ? tb[sb + lane] : make_float2(nan, neg_inf());
        float2 qp = shfl2(q, (lane + 31) & 31);
        bool hvp = lane > 0;
        if (lane == 0 && (sb > 0 || has_prev)) {
            qp = sb > 0 ? tb[sb - 1] : prev_pt;
            hvp = true;
        }
        float2 qn = shfl2(q, (lane + 1) & 31);
        if (lane == nv - 1) qn = sb + nv < cnt ? tb[sb + nv] : make_float2(nan, neg_inf());
        const float ip = warp_incl_prefix_max(q.y), is = warp_incl_suffix_max(q.y);
        float ep = __shfl_up_sync(kFull, ip, 1), es = __shfl_down_sync(kFull, is, 1);
        if (lane == 0) ep = neg_inf();
        if (lane == 31) es = neg_inf();
        ep = fmaxf(ep, pm0);
        es = fmaxf(es, sm0);
        bool keep = mine && !(q.y <= ep && q.y < es);
        keep = keep && !(hvp && same_point(qp, q));
        const bool up = qn.x == q.x && qn.y > q.y;
        const bool left = (hvp && qp.x == q.x) || q.x > xfirst;
        keep = keep && !(up && left);
        return __ballot_sync(kFull, keep);
    }

    // Wait (bounded) for tiles [from, to) after a timeout, so that no bulk
    // copy is still writing when the warp exits.
    __device__ void drain(unsigned from, unsigned to) const
    {
        if (lane != 0) return;
        for (unsigned s = from; s < to; ++s)
            mbar_wait_bounded(bars() + (s % C::kS), (s / C::kS) & 1u, kWaitNs / 10);
    }

    __device__ void write_r(RState &R) const
    {
        for (int k = lane; k < R.w; k += 32) R.gout[R.g + k] = ridx()[k];
    }

    // ------------------------------------------------------- one segment
    __device__ bool run_segment(int item_index, unsigned &seq)
    {
        const SegItem it = item(item_index);
        const float2 *P = reinterpret_cast<const float2 *>(args.points) + it.set_base;
        int32_t *out = args.out_idx + it.set_base;
        const long long a = it.a, b = it.b;
        const int M = (int)((b - a + C::kT - 1) / C::kT);
        RState R{0, 0, out + a, P};
        pn = 0;
        xfirst = P[0].x;
        sh_skip = 0;
        sh_fail = 0;
        float pm_carry = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        if (a > 0) {
            prev_pt = P[a - 1];
            has_prev = true;
        }
        const int npre = M < C::kS ? M : C::kS;
        // The tile buffers may hold generic writes of an earlier merge: order
        // them before the bulk copies that reuse the buffers.
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0)
            for (int k = 0; k < npre; ++k) issue(P, a, b, k, seq + k);
        unsigned issued = seq + npre;
        __syncwarp();

        float ymax_prev = neg_inf(), tmax_prev = neg_inf();
        for (int i = 0; i <= M; ++i) {
            float ymax_cur = neg_inf(), ynext = neg_inf();
            if (i < M) {
                const unsigned s = seq + i;
                const int bi = s % C::kS;
                const bool ok = mbar_wait_bounded(bars() + bi, (s / C::kS) & 1u, kWaitNs);
                if (!__all_sync(kFull, ok)) {
                    record_status(&args.hdr->status, kStTimeout);
                    drain(s, issued);
                    return false;
                }
                const long long st = a + (long long)i * C::kT;
                const int cnt = (int)((b - st) < C::kT ? (b - st) : C::kT);
                ymax_cur = strip_max(buf(bi) + tile_shift(P, st), cnt);
                ynext = warp_max(ymax_cur);
            }
            if (i >= 1) {
                const unsigned s = seq + i - 1;
                const long long st = a + (long long)(i - 1) * C::kT;
                const int cnt = (int)((b - st) < C::kT ? (b - st) : C::kT);
                decide(buf(s % C::kS) + tile_shift(P, st), cnt, st, ymax_prev, tmax_prev, ynext, pm_carry,
                       prev_pt, has_prev, R);
                __syncwarp();
                if (i - 1 + C::kS < M) {
                    if (lane == 0) {
                        fence_proxy_async_smem();
                        issue(P, a, b, i - 1 + C::kS, seq + i - 1 + C::kS);
                    }
                    ++issued;
                }
            }
            ymax_prev = ymax_cur;
            tmax_prev = ynext;
        }
        seq += M;
        flush_pending(R);
        write_r(R);
        const int count = R.g + R.w;
        if (it.nseg == 1) {
            if (lane == 0) args.out_count[it.set] = count;
            return true;
        }
        bool last = false;
        publish(it, item_index, R, pm_carry, last);
        // Batched: the second publisher of each neighbouring pair bridges it;
        // the warp that completes the set merges alone (the other warps are
        // busy with other sets).
        if (!last && R.g == 0) pair_bridges(it, item_index, count);
        if (last) merge_set(it, item_index, 1, 0);
        return true;
    }

    // ------------------------------------------- single set: tile stream
    struct Stream {
        unsigned issued;  // ring sequence number of the next tile to issue
        int sI, kI, MI;   // segment being issued, its next tile, its tile count
        long long aI, bI; // its point range
        int next;         // lane 0: the next segment, claimed when this one's last tile was issued
        bool dry;         // no segment left to claim
    };

    // Issue tiles until `limit` (exclusive ring sequence) or the input runs
    // out, claiming segments as the previous one is fully issued. Slot
    // metadata: tile start, point count, segment | first << 30 | last << 31.
    __device__ void fill(Stream &st, unsigned limit, const float2 *P)
    {
        while (st.issued < limit) {
            if (st.kI == st.MI) {
                if (st.dry) break;
                const int c = __shfl_sync(kFull, st.next, 0);
                if (c >= args.nseg) {
                    st.dry = true;
                    break;
                }
                st.sI = c;
                st.aI = seg_a(c);
                st.bI = seg_b(c);
                st.MI = (int)((st.bI - st.aI + C::kT - 1) / C::kT);
                st.kI = 0;
                if (st.MI == 0) {  // (segments are never empty)
                    st.dry = true;
                    break;
                }
            }
            if (lane == 0) {
                const long long start = st.aI + (long long)st.kI * C::kT;
                const int cnt = (int)(st.bI - start < C::kT ? st.bI - start : C::kT);
                issue(P, st.aI, st.bI, st.kI, st.issued);
                const unsigned fl = (st.kI == 0 ? 1u << 30 : 0u) | (st.kI == st.MI - 1 ? 1u << 31 : 0u);
                meta()[st.issued % C::kS] = make_int4((int)start, cnt, (int)((unsigned)st.sI | fl), 0);
                // the segment's last tile is issued: claim the next segment
                // now; the atomic completes while this warp works through the
                // tiles in its ring, and its result is read at the next fill
                if (st.kI == st.MI - 1)
                    st.next = min(args.nseg, (int)gridDim.x * C::kW) + (int)atomicAdd(&args.hdr->claim, 1u);
            }
            ++st.kI;
            ++st.issued;
        }
        __syncwarp();
    }

    // Single set: the warp streams the tiles of the segments it claims, in
    // claim order (which is input order), through its ring; the look-ahead
    // tile may belong to the next claimed segment (its points are later input
    // points, so they are valid witnesses for the elimination rule), and so
    // may the running maximum of earlier points. Each segment gets its own
    // running hood, published at its end.
    __device__ bool run_stream(unsigned &seq)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points);
        int32_t *out = args.out_idx;
        xfirst = P[0].x;
        sh_skip = 0;
        sh_fail = 0;
        Stream st;
        st.issued = seq;
        st.sI = -1;
        st.kI = 0;
        st.MI = 0;
        st.aI = st.bI = 0;
        // The first segments go one per warp in warp order; the rest are
        // claimed from the call's counter as warps become free.
        const int nstatic = min(args.nseg, (int)gridDim.x * C::kW);
        const int gwarp = blockIdx.x * C::kW + (threadIdx.x >> 5);
        st.next = gwarp;
        if (gwarp >= nstatic && lane == 0) st.next = nstatic + (int)atomicAdd(&args.hdr->claim, 1u);
        st.dry = false;
        const unsigned base = seq;
        fence_proxy_async_smem();
        __syncwarp();
        fill(st, base + C::kS, P);
        if (st.issued == base) {
            warp_done();
            return true;
        }

        RState R{0, 0, out, P};
        float pm_carry = neg_inf(), seg_max = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        long long last_end = -1;
        float ymax_prev = neg_inf(), tmax_prev = neg_inf();
        for (unsigned i = base;; ++i) {
            const bool have = i < st.issued;
            float ymax_cur = neg_inf(), ynext = neg_inf();
            if (have) {
                const int bi = i % C::kS;
                const bool ok = mbar_wait_bounded(bars() + bi, (i / C::kS) & 1u, kWaitNs);
                if (!__all_sync(kFull, ok)) {
                    record_status(&args.hdr->status, kStTimeout);
                    drain(i, st.issued);
                    seq = st.issued;
                    return false;
                }
                const int4 mt = meta()[bi];
                ymax_cur = strip_max(buf(bi) + tile_shift(P, mt.x), mt.y);
                ynext = warp_max(ymax_cur);
            }
            if (i > base) {
                const int4 md = meta()[(i - 1) % C::kS];
                const long long start = md.x;
                const int cnt = md.y;
                const unsigned fl = (unsigned)md.z;
                if (fl & (1u << 30)) {
                    // first tile of a segment: a new running hood
                    R = RState{0, 0, out + start, P};
                    pn = 0;
                    seg_max = neg_inf();
                    if (start != last_end) {
                        has_prev = start > 0;
                        prev_pt = start > 0 ? P[start - 1] : make_float2(0.f, 0.f);
                    }
                }
                decide(buf((i - 1) % C::kS) + tile_shift(P, start), cnt, start, ymax_prev, tmax_prev, ynext,
                       pm_carry, prev_pt, has_prev, R);
                seg_max = fmaxf(seg_max, tmax_prev);
                last_end = start + cnt;
                __syncwarp();
                if (fl & (1u << 31)) end_segment_single((int)(fl & 0x3fffffffu), R, seg_max);
                fill(st, i + C::kS, P);
            }
            if (!have) break;
            ymax_prev = ymax_cur;
            tmax_prev = ynext;
        }
        seq = st.issued;
        warp_done();
        return true;
    }

    // A warp whose stream has ended (every segment it claimed is published)
    // counts itself; the last of all the grid's warps marks its CTA as the
    // one that leads the final merge (every segment is published by then).
    __device__ void warp_done()
    {
        if (args.nseg <= 1) return;
        __threadfence();
        __syncwarp();
        unsigned old = 0;
        if (lane == 0) old = atomicAdd(args.arrivals, 1u);
        old = __shfl_sync(kFull, old, 0);
        if (old == gridDim.x * (unsigned)C::kW - 1u) {
            __threadfence();
            if (lane == 0) *cta_flag() = 1;
        }
    }

    // End of segment c of the single set: its hood is the running hood.
    // With one segment it is the answer; otherwise it is published (indices
    // in the output array; coordinates and indices also staged in the
    // workspace when it fits one window), with its count and the segment's
    // maximum y. They become visible to the merge through warp_done's fence.
    __device__ void end_segment_single(int c, RState &R, float seg_max)
    {
        flush_pending(R);
        write_r(R);
        const int count = R.g + R.w;
        if (args.nseg == 1) {
            if (lane == 0) args.out_count[0] = count;
            return;
        }
        const SegStore ss = store();
        if (R.g == 0) {
            float2 *dst = ss.xy + (size_t)c * C::kRCap;
            int *dsti = ss.sidx + (size_t)c * C::kRCap;
            for (int k = lane; k < R.w; k += 32) {
                dst[k] = rxy()[k];
                dsti[k] = ridx()[k];
            }
        }
        if (lane == 0) {
            ss.count[c] = R.g == 0 ? count : -count - 1;  // negative: coordinates not staged
            ss.ymax[c] = seg_max;
        }
        __syncwarp();
    }

    // ------------------------------------------- single set: final merge
    // Bounded wait, by one thread of the CTA, until *word == tag; the CTA's
    // other threads wait at the barrier. Polls back off (up to ~1 us) so that
    // a grid of waiting CTAs does not crowd the line in L2. Returns false
    // (in every thread) if the wait timed out or another part of the call
    // recorded an error.
    __device__ bool cta_wait_tag(const unsigned *word, unsigned want) const
    {
        __shared__ int s_ok;
        if (threadIdx.x == 0) {
            int ok = 1;
            const uint64_t t0 = global_ns();
            unsigned nap = 32;
            for (uint32_t it = 0;; ++it) {
                unsigned v;
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(word) : "memory");
                if (v == want) break;
                if (*reinterpret_cast<volatile int *>(&args.hdr->status) != 0 || global_ns() - t0 > kWaitNs) {
                    ok = 0;
                    break;
                }
                __nanosleep(nap);
                if (nap < 1024) nap <<= 1;
            }
            s_ok = ok;
        }
        __syncthreads();
        return s_ok != 0;
    }

    __device__ void release_tag(unsigned *word) const
    {
        __threadfence();
        asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(word), "r"(tag) : "memory");
    }

    // Bridges of adjacent hoods of the list, spread over every warp of the
    // grid: pair k is (list[k], list[k + 1]). Each warp counts its pairs
    // once they are stored.
    __device__ void pair_work(float2 *stg)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points);
        const SegStore ss = store();
        WsHeader *hdr = args.hdr;
        const int nl = (int)__ldcg(&hdr->nlist);
        const int gwarp = blockIdx.x * C::kW + (threadIdx.x >> 5), nwarps = gridDim.x * C::kW;
        int done = 0;
        for (int k0 = gwarp; k0 < nl - 1; k0 += 32 * nwarps) {
            // this warp's next 32 pairs, one per lane: their hoods and sizes
            // in two rounds of loads
            const int kl = k0 + lane * nwarps;
            const bool valid = kl < nl - 1;
            const int c = valid ? __ldcg(args.list_lid + kl) : 0, d = valid ? __ldcg(args.list_lid + kl + 1) : 0;
            const int rc = valid ? __ldcg(ss.count + c) : 0, rd = valid ? __ldcg(ss.count + d) : 0;
            const int m = min(32, (nl - 1 - k0 + nwarps - 1) / nwarps);
            for (int e = 0; e < m; ++e) {
                const int ce = __shfl_sync(kFull, c, e), de = __shfl_sync(kFull, d, e);
                const int rce = __shfl_sync(kFull, rc, e), rde = __shfl_sync(kFull, rd, e);
                const int2 pq = bridge_hoods(ss, P, args.out_idx, 0, ce, rce, seg_a(ce), de, rde, seg_a(de), stg);
                if (lane == 0) {
                    __stcg(args.list_bp + k0 + e * nwarps, pq.x);
                    __stcg(args.list_bq + k0 + e * nwarps, pq.y);
                }
                ++done;
            }
        }
        if (done && lane == 0) {
            __threadfence();
            atomicAdd(&hdr->pair_done, (unsigned)done);
        }
        __syncwarp();
    }

    // Copy of the kept hood ranges listed in the plan, from the staged
    // indices to their places in the output; entries spread over all warps.
    __device__ void copy_plan()
    {
        const SegStore ss = store();
        const int np = (int)__ldcg(&args.hdr->nplan);
        const int gwarp = blockIdx.x * C::kW + (threadIdx.x >> 5), nwarps = gridDim.x * C::kW;
        for (int k0 = gwarp; k0 < np; k0 += 32 * nwarps) {
            // this warp's next 32 entries, one per lane, in one round of loads
            const int kl = k0 + lane * nwarps;
            const int4 mine = kl < np ? __ldcg(args.plan + kl) : make_int4(0, 0, 0, 0);
            const int m = min(32, (np - k0 + nwarps - 1) / nwarps);
            for (int e = 0; e < m; e += 4) {
                // four entries' loads in flight before their stores
                int v[4][C::kRCap / 32];
                int4 pe[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    pe[q] = make_int4(__shfl_sync(kFull, mine.x, (e + q) & 31), __shfl_sync(kFull, mine.y, (e + q) & 31),
                                      __shfl_sync(kFull, mine.z, (e + q) & 31), __shfl_sync(kFull, mine.w, (e + q) & 31));
                    if (e + q >= m) pe[q].z = 0;
                    const int *src = ss.sidx + (size_t)pe[q].x * C::kRCap + pe[q].y;
#pragma unroll
                    for (int u = 0; u < C::kRCap / 32; ++u)
                        if (lane + 32 * u < pe[q].z) v[q][u] = __ldcg(src + lane + 32 * u);
                }
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int u = 0; u < C::kRCap / 32; ++u)
                        if (lane + 32 * u < pe[q].z) args.out_idx[pe[q].w + lane + 32 * u] = v[q][u];
            }
        }
    }

    // The warps of a CTA that does not lead the merge (every warp of it calls
    // this): help with the pair bridges once the hood list is out, then with
    // the copy once the plan is.
    __device__ void merge_help()
    {
        if (!cta_wait_tag(&args.hdr->phase1, tag)) return;
        pair_work(buf(0));
        if (!cta_wait_tag(&args.hdr->phase2, tag)) return;
        copy_plan();
    }

    // Loads n ints from global memory (L2) into shared memory, every thread
    // keeping U loads in flight (consecutive threads, consecutive words).
    template <int U>
    __device__ __forceinline__ static void cta_load(int *dst, const int *src, int n, int t, int nthreads)
    {
        for (int b0 = 0; b0 < n; b0 += nthreads * U) {
            int v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = b0 + u * nthreads + t;
                if (i < n) v[u] = __ldcg(src + i);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = b0 + u * nthreads + t;
                if (i < n) dst[i] = v[u];
            }
        }
    }

    // Block-wide exclusive prefix sums over entries 0..n-1 (n <=
    // kMaxSegSingle) in order: thread t holds the contiguous entries
    // [t m, t m + m) in registers, m = ceil(n / threads) (so that a short
    // list is spread over the threads too). f(i) is entry i's value;
    // g(i, before) receives its exclusive prefix. Returns the total. Every
    // thread of the CTA calls it.
    template <class F, class G>
    __device__ int cta_scan(int n, int t, int gw, int *xsum, F f, G g) const
    {
        constexpr int nw = C::kW, nthreads = nw * 32;
        constexpr int M = (kMaxSegSingle + nthreads - 1) / nthreads;
        const int m = (n + nthreads - 1) / nthreads;
        const int c0 = t * m;
        int v[M];
        int sum = 0;
#pragma unroll
        for (int j = 0; j < M; ++j) {
            v[j] = j < m && c0 + j < n ? f(c0 + j) : 0;
            sum += v[j];
        }
        const int incl = warp_incl_sum(sum);
        if (lane == 31) xsum[gw] = incl;
        __syncthreads();
        int before = incl - sum, total = 0;
        for (int w = 0; w < nw; ++w) {
            const int x = xsum[w];
            if (w < gw) before += x;
            total += x;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < M; ++j) {
            if (j < m && c0 + j < n) g(c0 + j, before);
            before += v[j];
        }
        return total;
    }

    // The CTA whose warp finished last leads the merge of the segment hoods
    // (every warp of it calls this; gw = its warp index):
    //  1. hood staircase over all segments: a segment is dropped whole when
    //     its max y is at most the max of all earlier segments and below the
    //     max of some later one (its points lie on or below a segment between
    //     two input points); the others form the hood list;
    //  2. the bridges of all adjacent hoods of the list (mam 1-5): when the
    //     listed hoods fit in shared memory this CTA computes them there;
    //     otherwise the list is published and every warp of the grid
    //     bridges its share of the pairs;
    //  3. hood i keeps its corners from the left bridge's corner s_i to the
    //     right bridge's corner e_i; if s_i > e_i, or s_i == e_i and that
    //     corner is not a strict right turn between the two bridges, hood i
    //     lies on or below the segment joining its neighbours' bridge corners
    //     and is dropped; its live neighbours become adjacent (links skip the
    //     dropped hoods) and are bridged, and so on;
    //  4. the kept ranges are laid out in order (mam 6): this CTA copies
    //     them when the result is small; otherwise it publishes a plan and
    //     every warp of the grid copies planned ranges (ranges of hoods too
    //     large to be staged are moved within the output array first, here).
    __device__ __noinline__ void merge_lead(int gw)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points);
        int32_t *out = args.out_idx;
        const SegStore ss = store();
        WsHeader *hdr = args.hdr;
        const int nh = args.nseg;
        constexpr int nw = C::kW;
        constexpr int nthreads = nw * 32;
        constexpr int M = (kMaxSegSingle + nthreads - 1) / nthreads;
        const int t = gw * 32 + lane;
        unsigned char *cta_base = base - C::kWarpBytes * gw;
        constexpr size_t kStg = 2 * C::kRCap * sizeof(float2);
        constexpr size_t kCtaBytes = C::kWarpBytes * C::kW;
        constexpr size_t kScratch = kCtaBytes - nw * kStg;
        float2 *stg = reinterpret_cast<float2 *>(cta_base + kCtaBytes - (size_t)(gw + 1) * kStg);
        // control words and cross-warp slots at the start of shared memory
        int *ctl = reinterpret_cast<int *>(cta_base);  // [0] smem hoods, [1] pairs ok, [2] copied here
        float *xpre = reinterpret_cast<float *>(ctl + 8);
        float *xsuf = xpre + 32;
        int *xsum = reinterpret_cast<int *>(xsuf + 32);
        int *sm = xsum + 32;  // scratch ints
        const size_t sm_ints = (kScratch - (size_t)(8 + 96) * 4) / 4;
        static_assert((size_t)11 * kMaxSegSingle + 1 <= (kScratch - (size_t)(8 + 96) * 4) / 4,
                      "the merge's arrays fit in shared memory");

        // 1. staircase: thread t takes segments [t M, t M + M) in registers
        int *rv = sm;  // segment counts (to the end)
        int *lid = sm + nh;  // the hood list
        int nl = 0;
        {
            const int c0 = t * M;
            float y[M];
            int r[M];
#pragma unroll
            for (int j = 0; j < M; ++j) {
                y[j] = neg_inf();
                r[j] = 0;
                if (c0 + j < nh) {
                    y[j] = __ldcg(ss.ymax + c0 + j);
                    r[j] = __ldcg(ss.count + c0 + j);
                }
            }
            float bm = neg_inf();
#pragma unroll
            for (int j = 0; j < M; ++j) {
                bm = fmaxf(bm, y[j]);
                if (c0 + j < nh) rv[c0 + j] = r[j];
            }
            const float ip = warp_incl_prefix_max(bm), is = warp_incl_suffix_max(bm);
            if (lane == 31) xpre[gw] = ip;
            if (lane == 0) xsuf[gw] = is;
            __syncthreads();
            float before = __shfl_up_sync(kFull, ip, 1), later = __shfl_down_sync(kFull, is, 1);
            if (lane == 0) before = neg_inf();
            if (lane == 31) later = neg_inf();
            for (int w = 0; w < gw; ++w) before = fmaxf(before, xpre[w]);
            for (int w = gw + 1; w < nw; ++w) later = fmaxf(later, xsuf[w]);
            float lat[M];
#pragma unroll
            for (int j = M - 1; j >= 0; --j) {
                lat[j] = later;
                later = fmaxf(later, y[j]);
            }
            unsigned keep = 0;
#pragma unroll
            for (int j = 0; j < M; ++j) {
                const int cn = r[j] < 0 ? -r[j] - 1 : r[j];
                if (cn > 0 && !(!(y[j] > before) && y[j] < lat[j])) keep |= 1u << j;
                before = fmaxf(before, y[j]);
            }
            const int nk = __popc(keep);
            const int incl = warp_incl_sum(nk);
            if (lane == 31) xsum[gw] = incl;
            __syncthreads();
            int k = incl - nk;
            for (int w = 0; w < nw; ++w) {
                if (w < gw) k += xsum[w];
                nl += xsum[w];
            }
            __syncthreads();
            while (keep) {
                const int j = __ffs(keep) - 1;
                keep &= keep - 1;
                lid[k++] = c0 + j;
            }
        }
        // list arrays after the list: 9 nl + 1 ints; then the listed hoods'
        // corners when they fit
        int *bp = lid + nl, *bq = bp + nl, *pv = bq + nl, *dead = pv + nl, *kill = dead + nl;
        int *nxt = kill + nl, *prv = nxt + nl, *hb = prv + nl, *pos = hb + nl;  // pos: nl + 1
        const size_t arr_end = (size_t)nh + 10 * (size_t)nl + 1;
        const size_t hs_off = (arr_end + 3) & ~(size_t)3;
        float2 *hstore = reinterpret_cast<float2 *>(sm + hs_off);
        const long long store_cap = hs_off + 4 <= sm_ints ? (long long)(sm_ints - hs_off) / 2 : 0;
        __syncthreads();
        {
            int hs = 0;
            bool unstaged = false;
            for (int i = t; i < nl; i += nthreads) {
                const int r = rv[lid[i]];
                hs += r < 0 ? -r - 1 : r;
                unstaged |= r < 0;
                nxt[i] = i + 1 < nl ? i + 1 : -1;
                prv[i] = i - 1;
                dead[i] = 0;
            }
            const bool any_unstaged = __syncthreads_or(unstaged);
            hs = __reduce_add_sync(kFull, (unsigned)hs);
            if (lane == 0) xsum[gw] = hs;
            __syncthreads();
            if (t == 0) {
                long long htot = 0;
                for (int w = 0; w < nw; ++w) htot += xsum[w];
                ctl[0] = htot <= store_cap;
                // the result (at most htot corners) will be copied here
                ctl[2] = ctl[0] && !any_unstaged && htot <= 8 * nthreads;
            }
            __syncthreads();
        }
        const bool smem = ctl[0] != 0;

        if (smem) {
            // 2 (in this CTA). The listed hoods' corners, copied in by warps
            // (one hood per warp at a time); the pairs are bridged below.
            auto hsize = [&](int i) {
                const int r = rv[lid[i]];
                return r < 0 ? -r - 1 : r;
            };
            cta_scan(nl, t, gw, xsum, hsize, [&](int i, int before) { hb[i] = before; });
            __syncthreads();
            for (int i = gw; i < nl; i += nw) {
                const int c = lid[i];
                const int r = rv[c];
                if (r >= 0) {
                    // staged: the coordinates themselves
                    const float2 *src = ss.xy + (size_t)c * C::kRCap;
                    float2 v[C::kRCap / 32];
#pragma unroll
                    for (int u = 0; u < C::kRCap / 32; ++u)
                        if (lane + 32 * u < r) v[u] = __ldcg(src + lane + 32 * u);
#pragma unroll
                    for (int u = 0; u < C::kRCap / 32; ++u)
                        if (lane + 32 * u < r) hstore[hb[i] + lane + 32 * u] = v[u];
                } else {
                    // not staged: gathered through the indices in the output array
                    const int h = -r - 1;
                    const int32_t *idx = out + seg_a(c);
                    for (int k0 = 0; k0 < h; k0 += 128) {
                        int id[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (k0 + lane + 32 * u < h) id[u] = __ldcg(idx + k0 + lane + 32 * u);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (k0 + lane + 32 * u < h) hstore[hb[i] + k0 + lane + 32 * u] = P[id[u]];
                    }
                }
            }
            for (int i = t; i < nl; i += nthreads) pv[i] = 0;
            if (t == 0) {
                hdr->nlist = 0;  // nothing for the other warps to bridge
                hdr->pair_done = 0;
                if (ctl[2]) {
                    // nor to copy: they may leave now
                    hdr->nplan = 0;
                    *args.arrivals = 0;
                }
            }
            __syncthreads();
            if (t == 0) {
                release_tag(&hdr->phase1);
                if (ctl[2]) release_tag(&hdr->phase2);
            }
        } else {
            // 2 (with the grid). Publish the list; every warp bridges its
            // share of the pairs.
            for (int i = t; i < nl; i += nthreads) __stcg(args.list_lid + i, lid[i]);
            if (t == 0) {
                hdr->nlist = (unsigned)nl;
                hdr->pair_done = 0;
            }
            __syncthreads();
            if (t == 0) release_tag(&hdr->phase1);
            pair_work(stg);
            if (t == 0) {
                int ok = 1;
                if (nl > 1) {
                    const uint64_t t0 = global_ns();
                    for (uint32_t it = 0;; ++it) {
                        unsigned v;
                        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];"
                                     : "=r"(v)
                                     : "l"(&hdr->pair_done)
                                     : "memory");
                        if ((int)v >= nl - 1) break;
                        if ((it & 63u) == 63u &&
                            (*reinterpret_cast<volatile int *>(&hdr->status) != 0 || global_ns() - t0 > kWaitNs)) {
                            record_status(&hdr->status, kStTimeout);
                            ok = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
                ctl[1] = ok;
            }
            __syncthreads();
            if (!ctl[1]) return;
            cta_load<16>(bp, args.list_bp, nl - 1, t, nthreads);
            cta_load<16>(bq, args.list_bq, nl - 1, t, nthreads);
            for (int i = t; i < nl; i += nthreads) pv[i] = i + 1 < nl;
            __syncthreads();
        }

        // 3. drop rounds over the linked list
        auto corner = [&](int i, int j) -> float2 {
            if (smem) return hstore[hb[i] + j];
            const int c = lid[i];
            return seg_hood(ss, P, out, 0, c, seg_a(c), rv[c]).pt(j);
        };
        for (int round = 0; round < nh + 1; ++round) {
            // live hoods whose pair with the next live hood has no bridge:
            // warp gw takes hoods gw + nw (32 j + l), found 32 at a time
            for (int j0 = 0; gw + nw * j0 < nl; j0 += 32) {
                const int i1 = gw + nw * (j0 + lane);
                unsigned need = __ballot_sync(kFull, i1 < nl && !dead[i1] && nxt[i1] >= 0 && !pv[i1]);
                while (need) {
                    const int i = gw + nw * (j0 + __ffs(need) - 1);
                    need &= need - 1;
                    const int k = nxt[i];
                    const int c = lid[i], d = lid[k];
                    int2 pq;
                    const int hc = rv[c] < 0 ? -rv[c] - 1 : rv[c], hd = rv[d] < 0 ? -rv[d] - 1 : rv[d];
                    if (smem && hc <= 32 && hd <= 32)
                        pq = bridge_small<MODE>(pc, FlatHood{hstore + hb[i]}, hc, FlatHood{hstore + hb[k]}, hd);
                    else if (smem)
                        pq = bridge_warp<MODE>(pc, FlatHood{hstore + hb[i]}, hc, FlatHood{hstore + hb[k]}, hd);
                    else
                        pq = bridge_hoods(ss, P, out, 0, c, rv[c], seg_a(c), d, rv[d], seg_a(d), stg);
                    if (lane == 0) {
                        bp[i] = pq.x;
                        bq[i] = pq.y;
                        pv[i] = 1;
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            int drop = 0;
            for (int i = t; i < nl; i += nthreads) {
                int dd = 0;
                const int p = prv[i], k = nxt[i];
                if (!dead[i] && p >= 0 && k >= 0) {
                    const int si = bq[p], ei = bp[i];
                    if (si > ei) {
                        dd = 1;
                    } else if (si == ei) {
                        const float2 A = corner(p, bp[p]);
                        const float2 Bc = corner(i, si);
                        const float2 Cc = corner(k, bq[i]);
                        dd = orient<MODE>(pc, A, Bc, Cc) >= 0;
                    }
                }
                kill[i] = dd;
                drop |= dd;
            }
            if (!__syncthreads_or(drop)) break;
            for (int i = t; i < nl; i += nthreads) dead[i] |= kill[i];
            __syncthreads();
            // relink the live hoods past the dropped ones (the links of
            // dropped hoods stay as they were, so the chains end at live hoods)
            for (int i = t; i < nl; i += nthreads) {
                if (dead[i]) continue;
                int k = nxt[i];
                while (k >= 0 && dead[k]) k = nxt[k];
                int p = prv[i];
                while (p >= 0 && dead[p]) p = prv[p];
                kill[i] = k;  // kill[] reused: the new next
                pos[i] = p;   // pos[] reused: the new previous
            }
            __syncthreads();
            for (int i = t; i < nl; i += nthreads) {
                if (dead[i]) continue;
                if (kill[i] != nxt[i]) pv[i] = 0;
                nxt[i] = kill[i];
                prv[i] = pos[i];
            }
            __syncthreads();
        }

        // 4. kept range [s_i, e_i] of live hood i and its place in the output
        bool unstaged = false;
        for (int i = t; i < nl; i += nthreads) unstaged |= !dead[i] && rv[lid[i]] < 0;
        const bool any_unstaged = __syncthreads_or(unstaged);
        auto s_of = [&](int i) { return prv[i] >= 0 ? bq[prv[i]] : 0; };
        auto range_len = [&](int i) {
            if (dead[i]) return 0;
            const int r = rv[lid[i]];
            const int hi = r < 0 ? -r - 1 : r;
            const int ei = nxt[i] >= 0 ? bp[i] : hi - 1;
            return ei - s_of(i) + 1;
        };
        const int total_out = cta_scan(nl, t, gw, xsum, range_len, [&](int i, int before) { pos[i] = before; });
        if (t == 0) pos[nl] = total_out;
        __syncthreads();
        const bool here = !any_unstaged && total_out <= 8 * nthreads;
        if (here) {
            // small result: copied by this CTA from the staged indices, a
            // hood per warp at a time
            for (int i = gw; i < nl; i += nw) {
                if (dead[i]) continue;
                const int len = pos[i + 1] - pos[i];
                const int *src = ss.sidx + (size_t)lid[i] * C::kRCap + s_of(i);
                for (int k = lane; k < len; k += 32) out[pos[i] + k] = __ldcg(src + k);
            }
        } else {
            // plan entries (staged live hoods), copied by every warp after the release
            for (int i = t; i < nl; i += nthreads) {
                const int len = dead[i] || rv[lid[i]] < 0 ? 0 : pos[i + 1] - pos[i];
                __stcg(args.plan + i, make_int4(lid[i], dead[i] ? 0 : s_of(i), len, pos[i]));
            }
            if (any_unstaged) {
                // hoods whose indices are only in the output array: moved in
                // place, in batches whose destinations all lie below every
                // source in the batch (destinations never exceed sources)
                int i0 = 0;
                while (i0 < nl && dead[i0]) ++i0;
                while (i0 < nl) {
                    const long long a0 = seg_a(lid[i0]) + s_of(i0);
                    int i1 = i0 + 1;
                    while (i1 < nl && (long long)pos[i1 + 1] <= a0) ++i1;
                    for (int i = i0 + gw; i < i1; i += nw) {
                        if (dead[i]) continue;
                        const int c = lid[i];
                        if (rv[c] >= 0) continue;
                        const long long ac = seg_a(c);
                        const int si = s_of(i);
                        const int len = pos[i + 1] - pos[i], dst = pos[i];
                        if ((long long)dst == ac + si) continue;  // already in place
                        for (int b0 = 0; b0 < len; b0 += 32) {
                            const int k = b0 + lane;
                            int v = 0;
                            if (k < len) v = __ldcg(out + ac + si + k);
                            __syncwarp();
                            if (k < len) out[dst + k] = v;
                            __syncwarp();
                        }
                    }
                    __threadfence_block();
                    __syncthreads();
                    i0 = i1;
                    while (i0 < nl && dead[i0]) ++i0;
                }
            }
        }
        if (t == 0) args.out_count[0] = total_out;
        if (ctl[2]) return;  // phase 2 is out already
        if (t == 0) {
            hdr->nplan = here ? 0u : (unsigned)nl;
            *args.arrivals = 0;
        }
        __syncthreads();
        if (t == 0) release_tag(&hdr->phase2);
        if (!here) copy_plan();
    }

    // End of a segment of a multi-segment set: publish the segment hood (its
    // indices are already in the output array; its coordinates and indices
    // are also staged in the workspace when it fits one window), its count
    // and its max y. `last` is set in the warp that completed the set's last
    // segment.
    __device__ void publish(const SegItem &it, int item_index, RState &R, float segmax, bool &last)
    {
        const SegStore ss = store();
        const int count = R.g + R.w;
        const int stage0 = args.items ? args.items[item_index - it.c].pad : 0;
        if (R.g == 0) {
            float2 *dst = ss.xy + (size_t)(stage0 + it.c) * C::kRCap;
            int *dsti = ss.sidx + (size_t)(stage0 + it.c) * C::kRCap;
            for (int k = lane; k < R.w; k += 32) {
                dst[k] = rxy()[k];
                dsti[k] = ridx()[k];
            }
        }
        if (lane == 0) {
            ss.count[it.slot] = R.g == 0 ? count : -count - 1;  // negative: coordinates not staged
            ss.ymax[it.slot] = segmax;
        }
        __threadfence();
        __syncwarp();
        unsigned old = 0;
        if (lane == 0) {
            __threadfence();
            old = atomicAdd(args.arrivals + it.set, 1u);
        }
        old = __shfl_sync(kFull, old, 0);
        last = old == (unsigned)(it.nseg - 1);
        if (last) __threadfence();
    }

    // After publishing segment hood c (staged, `count` corners): for each
    // neighbour pair (c - 1, c) and (c, c + 1), the second of its two
    // segments to be published computes the pair's bridge and stores it,
    // tagged with this call, for the final merge (which computes any pair
    // bridge it does not find).
    __device__ __noinline__ void pair_bridges(const SegItem &it, int item_index, int count)
    {
        const SegStore ss = store();
        const float2 *P = reinterpret_cast<const float2 *>(args.points) + it.set_base;
        const int32_t *out = args.out_idx + it.set_base;
        const int stage0 = args.items ? args.items[item_index - it.c].pad : 0;
        for (int side = 0; side < 2; ++side) {
            const int l = it.c - 1 + side;  // the pair (l, l + 1)
            if (l < 0 || l + 1 >= it.nseg) continue;
            unsigned old = 0;
            if (lane == 0) old = atomicExch(ss.pair + stage0 + l, tag);
            old = __shfl_sync(kFull, old, 0);
            if (old != tag) continue;  // the other hood comes later; its warp bridges the pair
            __threadfence();
            const int o = side == 0 ? l : l + 1;
            const int ro = __ldcg(ss.count + it.slot0 + o);
            if (ro < 0) continue;  // the other hood is not staged
            const int rl = side == 0 ? ro : count, rr = side == 0 ? count : ro;
            const int2 pq = bridge_hoods(ss, P, out, stage0, l, rl, seg_start(it, item_index, l), l + 1, rr,
                                         seg_start(it, item_index, l + 1), buf(0));
            if (lane == 0)
                __stcg(ss.bridge + stage0 + l,
                       ((unsigned long long)tag << 32) | ((unsigned long long)pq.x << 16) | (unsigned)pq.y);
        }
    }

    // ------------------------------------------------------- final merge
    // Corners of published segment hood c: staged coordinates when present,
    // else gathered through the indices in the output array.
    struct SegHood {
        const float2 *xy;
        const int32_t *idx;
        const float2 *P;
        __device__ __forceinline__ float2 pt(int j) const { return xy ? __ldcg(xy + j) : P[__ldcg(idx + j)]; }
    };

    // Staged corners read from global memory (L2).
    struct CgHood {
        const float2 *xy;
        __device__ __forceinline__ float2 pt(int j) const { return __ldcg(xy + j); }
    };

    // Corners copied into shared memory.
    struct FlatHood {
        const float2 *xy;
        __device__ __forceinline__ float2 pt(int j) const { return xy[j]; }
    };

    // Bridge of published hoods c (left) and d (right). When both have their
    // coordinates staged, they are first copied into shared memory at stg
    // (2 RCAP corners; one round of global loads) and searched there.
    __device__ int2 bridge_hoods(const SegStore &ss, const float2 *P, const int32_t *out, int stage0, int c,
                                 int rc, long long a_c, int d, int rd, long long a_d, float2 *stg)
    {
        const int hc = rc < 0 ? -rc - 1 : rc, hd = rd < 0 ? -rd - 1 : rd;
        if (rc >= 0 && rd >= 0 && hc <= 32 && hd <= 32)
            return bridge_small<MODE>(pc, CgHood{ss.xy + (size_t)(stage0 + c) * C::kRCap}, hc,
                                      CgHood{ss.xy + (size_t)(stage0 + d) * C::kRCap}, hd);
        if (rc >= 0 && rd >= 0) {
            const float2 *xa = ss.xy + (size_t)(stage0 + c) * C::kRCap;
            const float2 *xb = ss.xy + (size_t)(stage0 + d) * C::kRCap;
            constexpr int U = C::kRCap / 32;
            float2 va[U], vb[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = lane + 32 * u;
                if (k < hc) va[u] = __ldcg(xa + k);
                if (k < hd) vb[u] = __ldcg(xb + k);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int k = lane + 32 * u;
                if (k < hc) stg[k] = va[u];
                if (k < hd) stg[C::kRCap + k] = vb[u];
            }
            __syncwarp();
            const int2 pq = bridge_warp<MODE>(pc, FlatHood{stg}, hc, FlatHood{stg + C::kRCap}, hd);
            __syncwarp();
            return pq;
        }
        const SegHood A = seg_hood(ss, P, out, stage0, c, a_c, rc);
        const SegHood B = seg_hood(ss, P, out, stage0, d, a_d, rd);
        return bridge_warp<MODE>(pc, A, hc, B, hd);
    }

    __device__ SegHood seg_hood(const SegStore &ss, const float2 *P, const int32_t *out, int stage0, int c,
                                long long a_c, int raw) const
    {
        SegHood h;
        h.xy = raw >= 0 ? ss.xy + (size_t)(stage0 + c) * C::kRCap : nullptr;
        h.idx = out + a_c;
        h.P = P;
        return h;
    }

    __device__ long long seg_start(const SegItem &it, int item_index, int c) const
    {
        if (args.items) return args.items[item_index - it.c + c].a;
        return seg_a(c);
    }

    // Merge the published segment hoods of a set into its output, with nw
    // warps (this one is number gw; nw == 1: this warp alone, else the whole
    // CTA). Stages of the paper over the whole list at once:
    //  1. hood staircase: a segment is dropped whole when its max y is at most
    //     the max over all earlier segments and below the max over some later
    //     one (its points then lie on or below a segment between two input
    //     points);
    //  2. the bridge (bridge_warp) of every adjacent pair of remaining hoods,
    //     the pairs spread over the warps (pairs of neighbouring segments may
    //     come bridged from publication);
    //  3. hood i keeps its corners from the left bridge's corner s_i to the
    //     right bridge's corner e_i. If s_i > e_i, or s_i == e_i and that
    //     corner is not a strict right turn between the two bridges, every
    //     corner of hood i lies on or below the segment joining its
    //     neighbours' bridge corners: hood i is dropped and the new adjacent
    //     pairs are bridged; repeat until nothing is dropped;
    //  4. the kept ranges are compacted into the output (mam 6).
    // The resulting chain is strictly convex, runs from the first point to the
    // last and has every input point on or below it: it is the upper hood.
    // With the whole CTA, the remaining hoods' coordinates are copied into
    // shared memory once when they fit, and stages 2-3 run there.
    __device__ __noinline__ void merge_set(const SegItem &it, int item_index, int nw, int gw)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points) + it.set_base;
        int32_t *out = args.out_idx + it.set_base;
        const SegStore ss = store();
        const int nh = it.nseg;
        const int stage0 = args.items ? args.items[item_index - it.c].pad : 0;
        const int slot0 = it.slot0;
        const bool cta = nw > 1;
        const int nthreads = nw * 32, t = gw * 32 + lane;
        auto sync = [&]() {
            if (cta) __syncthreads(); else __syncwarp();
        };
        // staging of bridge operands: 2 RCAP corners per warp, at the end of
        // the CTA's warp regions (CTA) or in tile buffer 0 (one warp)
        unsigned char *cta_base = base - C::kWarpBytes * (threadIdx.x >> 5);
        constexpr size_t kStg = 2 * C::kRCap * sizeof(float2);
        constexpr size_t kCtaBytes = C::kWarpBytes * C::kW;
        float2 *stg = cta ? reinterpret_cast<float2 *>(cta_base + kCtaBytes - (size_t)(gw + 1) * kStg) : buf(0);
        // scratch: 13 nh + 2 ints, 3 x 32 cross-warp words, 8 control words
        int *sm;
        const size_t need = (size_t)(13 * nh + 2 + 96 + 8) * 4;
        if (cta && need + C::kW * kStg <= kCtaBytes) sm = reinterpret_cast<int *>(cta_base);
        else if (!cta && need <= (size_t)(C::kS - 2) * C::kBuf * 8) sm = reinterpret_cast<int *>(buf(2));
        else sm = ss.live + (size_t)stage0 * 16;  // 16 ints per segment: >= 13 nh + 106 once nh >= 36,
                                                   // and smaller sets always fit the shared scratch
        float *yv = reinterpret_cast<float *>(sm);
        int *rv = sm + nh;
        int *lidA = sm + 2 * nh, *bpA = sm + 3 * nh, *bqA = sm + 4 * nh, *pvA = sm + 5 * nh;
        int *lidB = sm + 6 * nh, *bpB = sm + 7 * nh, *bqB = sm + 8 * nh, *pvB = sm + 9 * nh;
        int *dead = sm + 10 * nh;
        int *pos = sm + 11 * nh;  // nh + 1
        int *hb = sm + 12 * nh + 1;  // nh + 1: offset of segment c's hood in the shared store
        float *xpre = reinterpret_cast<float *>(sm + 13 * nh + 2);
        float *xsuf = xpre + 32;
        int *xsum = reinterpret_cast<int *>(xpre + 64);
        int *ctl = xsum + 32;  // [0] = live count, [1] = some kept hood not staged, [2] = hoods in shared memory
        // hood coordinate store: shared memory between the scratch and the
        // staging areas (whole CTA only)
        const size_t store_off = (need + 15) / 16 * 16;
        float2 *hstore = reinterpret_cast<float2 *>(cta_base + store_off);
        const long long store_cap =
            (cta && sm == reinterpret_cast<int *>(cta_base)) ? (long long)(kCtaBytes - C::kW * kStg - store_off) / 8
                                                             : 0;

        // Block-wide scans over threads, in thread order.
        auto excl_sum = [&](int v, int &total) {
            const int incl = warp_incl_sum(v);
            if (lane == 31) xsum[gw] = incl;
            sync();
            int before = incl - v;
            total = 0;
            for (int w = 0; w < nw; ++w) {
                const int x = xsum[w];
                if (w < gw) before += x;
                total += x;
            }
            sync();
            return before;
        };

        // 1. hood staircase: each thread a block of consecutive segments
        int nl = 0;
        {
            const int m = (nh + nthreads - 1) / nthreads;
            const int c0 = min(nh, t * m), c1 = min(nh, c0 + m);
            float bm = neg_inf();
            for (int cb = c0; cb < c1; cb += 8) {
                float y[8];
                int r[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (cb + u < c1) {
                        y[u] = __ldcg(ss.ymax + slot0 + cb + u);
                        r[u] = __ldcg(ss.count + slot0 + cb + u);
                    }
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    if (cb + u < c1) {
                        yv[cb + u] = y[u];
                        rv[cb + u] = r[u];
                        bm = fmaxf(bm, y[u]);
                    }
                }
            }
            const float ip = warp_incl_prefix_max(bm), is = warp_incl_suffix_max(bm);
            if (lane == 31) xpre[gw] = ip;
            if (lane == 0) xsuf[gw] = is;
            sync();
            float before = __shfl_up_sync(kFull, ip, 1), later = __shfl_down_sync(kFull, is, 1);
            if (lane == 0) before = neg_inf();
            if (lane == 31) later = neg_inf();
            for (int w = 0; w < gw; ++w) before = fmaxf(before, xpre[w]);
            for (int w = gw + 1; w < nw; ++w) later = fmaxf(later, xsuf[w]);
            // later maxima, right to left, kept in dead[] for now
            for (int c = c1 - 1; c >= c0; --c) {
                dead[c] = __float_as_int(later);
                later = fmaxf(later, yv[c]);
            }
            int nk = 0;
            for (int c = c0; c < c1; ++c) {
                const float ym = yv[c];
                const int r = rv[c];
                const int cn = r < 0 ? -r - 1 : r;
                const bool keep = cn > 0 && !(!(ym > before) && ym < __int_as_float(dead[c]));
                pos[c] = keep;
                nk += keep;
                before = fmaxf(before, ym);
            }
            int k = excl_sum(nk, nl);
            for (int c = c0; c < c1; ++c)
                if (pos[c]) {
                    lidA[k] = c;
                    pvA[k] = 0;
                    ++k;
                }
        }
        sync();
        // the sizes of the remaining hoods; their corners copied into shared
        // memory when they fit, and the bridges of adjacent segments already
        // computed at publication (both in one round of loads)
        {
            const int m = (nl + nthreads - 1) / nthreads;
            const int i0 = min(nl, t * m), i1 = min(nl, i0 + m);
            int hs = 0;
            bool unstaged = false;
            for (int i = i0; i < i1; ++i) {
                const int r = rv[lidA[i]];
                hs += r < 0 ? -r - 1 : r;
                unstaged |= r < 0;
            }
            const bool any_unstaged = cta ? __syncthreads_or(unstaged) : __any_sync(kFull, unstaged);
            int htot = 0;
            int off = excl_sum(hs, htot);
            const bool smem = !any_unstaged && htot <= store_cap;
            constexpr int MB = 2;  // bridge words loaded ahead of the copy, per thread
            unsigned long long bw[MB];
#pragma unroll
            for (int u = 0; u < MB; ++u) {
                const int i = i0 + u;
                bw[u] = 0;
                if (i < i1 && i + 1 < nl && lidA[i + 1] == lidA[i] + 1) bw[u] = __ldcg(ss.bridge + stage0 + lidA[i]);
            }
            if (smem) {
                for (int i = i0; i < i1; ++i) {
                    const int c = lidA[i];
                    hb[c] = off;
                    off += rv[c];
                    pos[i] = hb[c];
                }
                if (t == 0) pos[nl] = htot;
                sync();
                // copy: corner e belongs to the hood i with pos[i] <= e < pos[i + 1]
                constexpr int U = 4;
                for (int e0 = t; e0 < htot; e0 += nthreads * U) {
                    float2 v[U];
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * nthreads;
                        if (e < htot) {
                            int lo = 0, hi = nl - 1;
                            while (lo < hi) {
                                const int mid = (lo + hi + 1) >> 1;
                                if (pos[mid] <= e) lo = mid; else hi = mid - 1;
                            }
                            v[u] = __ldcg(ss.xy + (size_t)(stage0 + lidA[lo]) * C::kRCap + (e - pos[lo]));
                        }
                    }
#pragma unroll
                    for (int u = 0; u < U; ++u) {
                        const int e = e0 + u * nthreads;
                        if (e < htot) hstore[e] = v[u];
                    }
                }
            }
            for (int i = i0; i < i1; ++i) {
                unsigned long long w = 0;
                if (i - i0 < MB) {
#pragma unroll
                    for (int u = 0; u < MB; ++u)
                        if (i - i0 == u) w = bw[u];
                } else if (i + 1 < nl && lidA[i + 1] == lidA[i] + 1) {
                    w = __ldcg(ss.bridge + stage0 + lidA[i]);
                }
                if ((unsigned)(w >> 32) == tag) {
                    bpA[i] = (int)((w >> 16) & 0xffffu);
                    bqA[i] = (int)(w & 0xffffu);
                    pvA[i] = 1;
                }
            }
            if (t == 0) ctl[2] = smem;
        }
        sync();
        const bool smem = ctl[2] != 0;
        auto corner = [&](int c, int j) -> float2 {
            if (smem) return hstore[hb[c] + j];
            return seg_hood(ss, P, out, stage0, c, seg_start(it, item_index, c), rv[c]).pt(j);
        };
        int *lid = lidA, *bp = bpA, *bq = bqA, *pv = pvA;
        int *lid2 = lidB, *bp2 = bpB, *bq2 = bqB, *pv2 = pvB;

        // 2-3. bridges of adjacent hoods; drop the hoods that contribute nothing
        for (int round = 0; round < nh + 1; ++round) {
            for (int i = gw; i < nl - 1; i += nw) {
                if (pv[i]) continue;
                const int c = lid[i], d = lid[i + 1];
                int2 pq;
                if (smem && rv[c] <= 32 && rv[d] <= 32)
                    pq = bridge_small<MODE>(pc, FlatHood{hstore + hb[c]}, rv[c], FlatHood{hstore + hb[d]}, rv[d]);
                else if (smem)
                    pq = bridge_warp<MODE>(pc, FlatHood{hstore + hb[c]}, rv[c], FlatHood{hstore + hb[d]}, rv[d]);
                else
                    pq = bridge_hoods(ss, P, out, stage0, c, rv[c], seg_start(it, item_index, c), d, rv[d],
                                      seg_start(it, item_index, d), stg);
                if (lane == 0) {
                    bp[i] = pq.x;
                    bq[i] = pq.y;
                    pv[i] = 1;
                }
                __syncwarp();
            }
            sync();
            int drop = 0;
            for (int i = t; i < nl; i += nthreads) {
                int dd = 0;
                if (i > 0 && i < nl - 1) {
                    const int si = bq[i - 1], ei = bp[i];
                    if (si > ei) {
                        dd = 1;
                    } else if (si == ei) {
                        const float2 A = corner(lid[i - 1], bp[i - 1]);
                        const float2 B = corner(lid[i], si);
                        const float2 Cc = corner(lid[i + 1], bq[i]);
                        dd = orient<MODE>(pc, A, B, Cc) >= 0;
                    }
                }
                dead[i] = dd;
                drop |= dd;
            }
            const bool any = cta ? __syncthreads_or(drop) : __any_sync(kFull, drop);
            if (!any) break;
            // compaction of the live list; a pair's bridge stays valid when
            // its two hoods were already adjacent
            {
                const int m = (nl + nthreads - 1) / nthreads;
                const int i0 = min(nl, t * m), i1 = min(nl, i0 + m);
                int na = 0;
                for (int i = i0; i < i1; ++i) na += !dead[i];
                int total = 0;
                int k = excl_sum(na, total);
                for (int i = i0; i < i1; ++i) {
                    if (dead[i]) continue;
                    lid2[k] = lid[i];
                    // pair (k, k + 1) stays bridged iff the next alive hood is i + 1
                    if (i + 1 < nl && !dead[i + 1] && pv[i]) {
                        pv2[k] = 1;
                        bp2[k] = bp[i];
                        bq2[k] = bq[i];
                    } else {
                        pv2[k] = 0;
                    }
                    ++k;
                }
                nl = total;
            }
            int *tmp;
            tmp = lid; lid = lid2; lid2 = tmp;
            tmp = bp; bp = bp2; bp2 = tmp;
            tmp = bq; bq = bq2; bq2 = tmp;
            tmp = pv; pv = pv2; pv2 = tmp;
            sync();
        }

        // 4. output: ranges [s_i, e_i] of the kept hoods, packed in order.
        int total_out = 0;
        bool any_unstaged = false;
        {
            const int m = (nl + nthreads - 1) / nthreads;
            const int i0 = min(nl, t * m), i1 = min(nl, i0 + m);
            int sum = 0;
            bool unstaged = false;
            for (int i = i0; i < i1; ++i) {
                const int r = rv[lid[i]];
                const int hi = r < 0 ? -r - 1 : r;
                const int si = i > 0 ? bq[i - 1] : 0, ei = i < nl - 1 ? bp[i] : hi - 1;
                sum += ei - si + 1;
                unstaged |= r < 0;
            }
            any_unstaged = cta ? __syncthreads_or(unstaged) : __any_sync(kFull, unstaged);
            int run = excl_sum(sum, total_out);
            for (int i = i0; i < i1; ++i) {
                pos[i] = run;
                const int r = rv[lid[i]];
                const int hi = r < 0 ? -r - 1 : r;
                const int si = i > 0 ? bq[i - 1] : 0, ei = i < nl - 1 ? bp[i] : hi - 1;
                run += ei - si + 1;
            }
            if (t == 0) pos[nl] = total_out;
        }
        sync();
        int ncopy = nl;
        if (!any_unstaged) {
            // Every kept hood has its indices staged: copy from there, all
            // corners at once (element e belongs to the hood i with
            // pos[i] <= e < pos[i + 1]).
            constexpr int U = 8;
            for (int e0 = t; e0 < total_out; e0 += nthreads * U) {
                int v[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthreads;
                    if (e < total_out) {
                        int lo = 0, hi = nl - 1;
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (pos[mid] <= e) lo = mid; else hi = mid - 1;
                        }
                        const int si = lo > 0 ? bq[lo - 1] : 0;
                        v[u] = __ldcg(ss.sidx + (size_t)(stage0 + lid[lo]) * C::kRCap + si + (e - pos[lo]));
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int e = e0 + u * nthreads;
                    if (e < total_out) out[e] = v[u];
                }
            }
            ncopy = 0;  // nothing left for the batched copy below
        }
        // Copy in batches [i0, i1) whose destinations all lie below every
        // source in the batch (destinations never exceed sources); batches run
        // one after the other.
        int i0 = 0;
        while (i0 < ncopy) {
            const long long a0 = seg_start(it, item_index, lid[i0]) + (i0 > 0 ? bq[i0 - 1] : 0);
            int i1 = i0 + 1;
            while (i1 < nl && (long long)pos[i1 + 1] <= a0) ++i1;
            for (int i = i0 + gw; i < i1; i += nw) {
                const int c = lid[i];
                const long long ac = seg_start(it, item_index, c);
                const int r = rv[c];
                const int hi = r < 0 ? -r - 1 : r;
                const int si = i > 0 ? bq[i - 1] : 0, ei = i < nl - 1 ? bp[i] : hi - 1;
                const int len = ei - si + 1, dst = pos[i];
                if ((long long)dst == ac + si) continue;  // already in place
                for (int b0 = 0; b0 < len; b0 += 32) {
                    const int k = b0 + lane;
                    int v = 0;
                    if (k < len) v = __ldcg(out + ac + si + k);
                    __syncwarp();
                    if (k < len) out[dst + k] = v;
                    __syncwarp();
                }
            }
            __threadfence_block();
            sync();
            i0 = i1;
        }
        if (t == 0) {
            args.out_count[it.set] = total_out;
            args.arrivals[it.set] = 0;
        }
        sync();
    }

    __device__ int *cta_flag() const
    {
        return reinterpret_cast<int *>(base - C::kWarpBytes * (threadIdx.x >> 5) + C::kWarpBytes * C::kW);
    }
};

template <class C, int MODE>
__global__ void __launch_bounds__(C::kNT, 1) fused_kernel(FusedArgs args)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    Warp<C, MODE> Wk(args, smem + C::kWarpBytes * warp);
    uint64_t *bars = Wk.bars();
    if (lane == 0) {
        for (int s = 0; s <= C::kS; ++s) mbar_init(bars + s, 1);
        fence_mbar_init();
    }
    if (threadIdx.x == 0) *Wk.cta_flag() = 0;
    __syncthreads();

    Wk.tag = (__ldcg(&args.hdr->epoch) + 1u) ^ kTagMix;

    // Test hook: one bounded wait on a barrier that nothing completes.
    bool go = true;
    const int stall = args.hdr->stall_test_ns;
    if (stall > 0) {
        bool tmo = false;
        if (lane == 0) tmo = !mbar_wait_bounded(bars + C::kS, 0, (uint64_t)stall);
        if (tmo) record_status(&args.hdr->status, kStTimeout);
        go = !__syncthreads_or(tmo);
    }

    unsigned seq = 0;
    if (!go) {
        // skipped
    } else if (args.queue) {
        // Batched: every warp takes items from a shared queue (the planning
        // kernel puts the large sets first) until it runs dry.
        const int nitems = *args.num_items_dev;
        while (true) {
            int i = 0;
            if (lane == 0) i = (int)atomicAdd(args.queue, 1u);
            i = __shfl_sync(kFull, i, 0);
            if (i >= nitems) break;
            if (!Wk.run_segment(i, seq)) break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(args.done, 1u) == gridDim.x - 1) {
                *args.queue = 0;
                *args.done = 0;
            }
        }
    } else {
        // Single set: warps claim segments dynamically and stream them.
        const bool ok = __syncthreads_and(Wk.run_stream(seq));
        // The CTA whose warp completed the last segment leads the merge of the
        // segment hoods with all its warps; every other warp helps with the
        // pair bridges and the final copy.
        const int flag = *Wk.cta_flag();
        if (args.nseg > 1 && ok) {
            if (flag) {
                // the merge reuses the CTA's shared memory, barriers included
                if (lane == 0)
                    for (int s = 0; s <= C::kS; ++s) mbar_inval(bars + s);
                __syncthreads();
                __threadfence();
                Wk.merge_lead(warp);
            } else {
                Wk.merge_help();
            }
        }
    }

    if (MODE & kModeCount) {
        unsigned long long t = Wk.pc.tests, f = Wk.pc.fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_xor_sync(kFull, t, o);
            f += __shfl_xor_sync(kFull, f, o);
        }
        if (lane == 0) {
            atomicAdd(&args.hdr->tests, t);
            atomicAdd(&args.hdr->fallbacks, f);
        }
    }

    // The last CTA to finish advances the workspace's call counter: every
    // CTA read it at its start, and every tagged word of this call is
    // written by then.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(&args.hdr->done_ctas, 1u) == gridDim.x - 1) {
            args.hdr->done_ctas = 0;
            args.hdr->claim = 0;
            args.hdr->epoch = args.hdr->epoch + 1u;
        }
    }
}

// ---------------------------------------------------------------- launcher
template <class C, int MODE>
static cudaError_t launch_cfg(const FusedArgs &args, int grid, cudaStream_t stream)
{
    auto kern = fused_kernel<C, MODE>;
    // The shared-memory attribute is set once per device (it stays with the
    // function in that device's context), not on every launch.
    static std::atomic<unsigned long long> attr_set{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
    if (!bit || !(attr_set.load(std::memory_order_acquire) & bit)) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kBytes);
        if (e != cudaSuccess) return e;
        attr_set.fetch_or(bit, std::memory_order_release);
    }
    kern<<<grid, C::kNT, C::kBytes, stream>>>(args);
    return cudaGetLastError();
}

template <class C>
static cudaError_t launch_mode(const FusedArgs &args, int grid, int mode, cudaStream_t stream)
{
    switch (mode) {
    case 0: return launch_cfg<C, 0>(args, grid, stream);
    case 1: return launch_cfg<C, 1>(args, grid, stream);
    case 2: return launch_cfg<C, 2>(args, grid, stream);
    default: return launch_cfg<C, 3>(args, grid, stream);
    }
}

template <class C>
static cudaError_t occupancy_cfg(int *blocks)
{
    auto kern = fused_kernel<C, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kBytes);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks, kern, C::kNT, C::kBytes);
}

// The tile configurations (index 1..kNumTileCfgs in the ABI): warps per CTA,
// points per lane (odd), tile buffers per warp, running window, pending list.
using Cfg1 = Cfg<8, 23, 4, 128, 128>;
using Cfg2 = Cfg<12, 15, 4, 128, 128>;
using Cfg3 = Cfg<8, 31, 3, 128, 128>;
using Cfg4 = Cfg<6, 31, 4, 128, 128>;

}  // namespace wg
