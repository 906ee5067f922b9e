// wg_fused.cuh -- the fused upper-hood kernel (one launch per call).
//
// The paper's stage loop (Section 2, main) merges hoods of size d into hoods
// of size 2d for d = 1, 2, 4, ... with one launch per stage and the hood array
// copied to the host and back every stage. Here the whole schedule runs in one
// persistent launch of warp streams:
//
//  * Every warp owns a segment: a contiguous range of one set. It streams the
//    segment through its own shared-memory ring of S tiles (32 * K points
//    each), filled by 1-D bulk copies (TMA) and tracked by its own mbarriers,
//    so warps never wait for each other.
//  * Per tile ("stages d = 1 .. 32K", fused):
//      - exact elimination: a point p is dropped when some earlier point is at
//        least as high and some later point (this tile, or the next tile,
//        already resident) is strictly higher; p then lies on or below a
//        segment between two input points and cannot be a corner. A lane whose
//        whole strip of K points is dropped this way learns it from the strip
//        maximum alone (no per-point pass). A repeat of the previous input
//        point is dropped too (first occurrence wins).
//      - a lane with survivors builds the hood of its strip serially (the
//        paper's Section 3 strips);
//      - surviving strip corners are appended, in order, to the warp's pending
//        list, which collects several tiles.
//  * A full pending list is merged by the paper's stages: d <= 16 in
//    registers (warp_hood_regs), larger d over chunk hoods in shared memory
//    with the bridge search (bridge_warp) and mam 6 compaction; the result is
//    merged into the warp's running segment hood (a shared-memory window of
//    its right end; older corners spill to the output array).
//  * At the end of its segment a warp publishes the segment hood (indices in
//    the output array, coordinates in the workspace), its count and the
//    segment's maximum y. The warp that completes the last segment of a set
//    (an atomic arrival count, no waiting) merges the segment hoods: a segment
//    whose maximum is at most the maximum of all earlier segments and below
//    that of some later segment is dropped whole (the same exact rule), and
//    the corners of the remaining segments are streamed through the same tile
//    pass.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "wg_device.cuh"
#include "wg_internal.h"

namespace wg {

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s bound on any device wait

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

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
    static constexpr size_t kOffDesc = kOffRidx + size_t(RCAP) * 4;
    static constexpr size_t kOffBar = kOffDesc + size_t(PCAP / 32) * 8;
    static constexpr size_t kWarpBytes = ((kOffBar + 8 * (S + 1)) + 127) / 128 * 128;
    static constexpr size_t kBytes = kWarpBytes * W;
    static_assert(K % 2 == 1 && K < 32, "K must be odd (bank-conflict-free strips) and < 32");
    static_assert(S >= 3, "three tile buffers: current, look-ahead, in flight");
    static_assert(RCAP % 64 == 0 && PCAP % 32 == 0 && PCAP >= 64, "window / list sizes");
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
    int *live;       // per stage slot: scratch of the final merge (4 ints each)
};

template <class C, int MODE>
struct Warp {
    const FusedArgs &args;
    unsigned char *base;  // this warp's region
    PredCount pc;
    int lane;
    int pn;               // corners in the pending list

    __device__ Warp(const FusedArgs &a, unsigned char *b) : args(a), base(b), pn(0) { lane = threadIdx.x & 31; }

    __device__ float2 *buf(int b) const { return reinterpret_cast<float2 *>(base + C::kOffTiles) + size_t(b) * C::kBuf; }
    __device__ float2 *pxy() const { return reinterpret_cast<float2 *>(base + C::kOffPxy); }
    __device__ int *pidx() const { return reinterpret_cast<int *>(base + C::kOffPidx); }
    __device__ float2 *rxy() const { return reinterpret_cast<float2 *>(base + C::kOffRxy); }
    __device__ int *ridx() const { return reinterpret_cast<int *>(base + C::kOffRidx); }
    __device__ int2 *desc() const { return reinterpret_cast<int2 *>(base + C::kOffDesc); }
    __device__ uint64_t *bars() const { return reinterpret_cast<uint64_t *>(base + C::kOffBar); }

    // ------------------------------------------------------------------ items
    __device__ SegItem item(int i) const
    {
        if (args.items) return args.items[i];
        SegItem it;
        const long long lo = (long long)i * args.tiles / args.nseg;
        const long long hi = (long long)(i + 1) * args.tiles / args.nseg;
        it.set_base = 0;
        it.a = lo * C::kT;
        it.b = hi * C::kT < args.n ? hi * C::kT : args.n;
        it.set = 0;
        it.c = i;
        it.nseg = args.nseg;
        it.slot = i;
        it.slot0 = 0;
        it.pad = i;  // stage slot
        return it;
    }

    __device__ SegStore store() const
    {
        SegStore s;
        s.count = args.seg_count;
        s.ymax = args.seg_ymax;
        s.xy = reinterpret_cast<float2 *>(args.seg_xy);
        s.live = args.seg_live;
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
            bulk_g2s(dst + 2 * shift, src + shift, (unsigned)nint * 8u, bar);
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

    // Append H[from..to) to the running hood.
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
    // bridge (p, q), then R = R[0..p] ++ H[q..h).
    __device__ __forceinline__ void r_merge(RState &R, const float2 *hxy, const int *hid, int h)
    {
        if (R.g + R.w == 0) {
            r_append(R, hxy, hid, 0, h);
            return;
        }
        const RunAcc ra{rxy(), R.g, R.gout, R.pts};
        const int2 pq = bridge_warp<MODE>(pc, ra, R.g + R.w, PtrHood{hxy}, h);
        if (pq.x < R.g) {
            R.g = pq.x + 1;
            R.w = 0;
        } else {
            R.w = pq.x + 1 - R.g;
        }
        __syncwarp();
        r_append(R, hxy, hid, pq.y, h);
    }

    // --------------------------------------------- merge of the pending list
    // Hoods of 32-corner chunks in registers, then the paper's stages over the
    // chunk hoods (bridge + mam 6 compaction in place), then the result into
    // the running hood.
    __device__ __forceinline__ void flush_pending(RState &R)
    {
        const int m = pn;
        pn = 0;
        if (m == 0) return;
        float2 *L = pxy();
        int *Lid = pidx();
        if (m <= 2) {
            r_merge(R, L, Lid, m);
            __syncwarp();
            return;
        }
        const int nc = (m + 31) >> 5;
        int2 *ds = desc();
        for (int c = 0; c < nc; ++c) {
            const int e = c * 32 + lane;
            const int mc = min(32, m - c * 32);
            float2 pt = make_float2(0.f, 0.f);
            int id = 0;
            if (lane < mc) {
                pt = L[e];
                id = Lid[e];
            }
            const int h = mc <= 2 ? mc : warp_hood_regs<MODE>(pc, pt, id, mc);
            __syncwarp();
            if (lane < h) {
                L[c * 32 + lane] = pt;
                Lid[c * 32 + lane] = id;
            }
            if (lane == 0) ds[c] = make_int2(c * 32, h);
            __syncwarp();
        }
        for (int st = 1; st < nc; st <<= 1) {
            for (int a = 0; a + st < nc; a += 2 * st) {
                const int2 P = ds[a], Q = ds[a + st];
                __syncwarp();
                if (Q.y == 0) continue;
                if (P.y == 0) {
                    if (lane == 0) ds[a] = Q;
                    __syncwarp();
                    continue;
                }
                const int2 pq = bridge_warp<MODE>(pc, PtrHood{L + P.x}, P.y, PtrHood{L + Q.x}, Q.y);
                const int dst = P.x + pq.x + 1, src = Q.x + pq.y, cnt = Q.y - pq.y;
                for (int b0 = 0; b0 < cnt; b0 += 32) {
                    const int k2 = b0 + lane;
                    float2 v = make_float2(0.f, 0.f);
                    int id = 0;
                    if (k2 < cnt) {
                        v = L[src + k2];
                        id = Lid[src + k2];
                    }
                    __syncwarp();
                    if (k2 < cnt) {
                        L[dst + k2] = v;
                        Lid[dst + k2] = id;
                    }
                    __syncwarp();
                }
                if (lane == 0) ds[a] = make_int2(P.x, pq.x + 1 + cnt);
                __syncwarp();
            }
        }
        const int2 H = ds[0];
        __syncwarp();
        if (H.y > 0) r_merge(R, L + H.x, Lid + H.x, H.y);
        __syncwarp();
    }

    // Survivors of one strip (not all dropped): per-point elimination, first
    // occurrence, then the strip's hood by a monotone scan whose stack is a bit
    // mask (top two corners in registers, deeper ones re-read).
    __device__ __forceinline__ unsigned strip_corners(const float2 *tb, int sbase, int nvalid, float pm0,
                                                   float sm0, float2 prev_pt, bool has_prev)
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
        unsigned hm = 0;
        int hn = 0;
        float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
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
            if (hv && same_point(pv, Pj)) continue;  // a repeat: first occurrence wins
            while (hn >= 2 && orient<MODE>(pc, A, B, Pj) >= 0) {
                hm &= ~(1u << (31 - __clz(hm)));
                --hn;
                B = A;
                if (hn >= 2) {
                    const unsigned below = hm & ~(1u << (31 - __clz(hm)));
                    A = tb[sbase + (31 - __clz(below))];
                }
            }
            if (hn >= 1) A = B;
            B = Pj;
            hm |= 1u << j;
            ++hn;
        }
        return hm;
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
    // ymax_mine = max y of this lane's strip; ynext = max y of the look-ahead
    // tile (or -inf). If IDX_SMEM the input indices are in idx_arr, else
    // start + position. Survivor corners go to the pending list.
    template <bool IDX_SMEM>
    __device__ __forceinline__ void decide(const float2 *tb, int cnt, long long start, const int *idx_arr,
                                           float ymax_mine, float ynext, float &pm_carry, float2 &prev_pt,
                                           bool &has_prev, RState &R)
    {
        constexpr int K = C::kK;
        const float ipre = warp_incl_prefix_max(ymax_mine);
        const float isuf = warp_incl_suffix_max(ymax_mine);
        float epre = __shfl_up_sync(kFull, ipre, 1);
        float esuf = __shfl_down_sync(kFull, isuf, 1);
        if (lane == 0) epre = neg_inf();
        if (lane == 31) esuf = neg_inf();
        const float tmax = __shfl_sync(kFull, ipre, 31);
        const float pm0 = fmaxf(pm_carry, epre);
        const float sm0 = fmaxf(esuf, ynext);

        const int sbase = lane * K;
        const int nvalid = cnt - sbase;
        unsigned hm = 0;
        // Whole strip dropped: everything before it is at least as high as its
        // maximum, and something after it is strictly higher.
        const bool dead = !(ymax_mine > pm0) && ymax_mine < sm0;
        if (!dead && nvalid > 0) hm = strip_corners(tb, sbase, nvalid, pm0, sm0, prev_pt, has_prev);
        if (args.validate && nvalid > 0) validate_strip(tb, sbase, nvalid, prev_pt, has_prev);

        pm_carry = fmaxf(pm_carry, tmax);
        prev_pt = tb[cnt - 1];
        has_prev = true;

        const int hc = __popc(hm);
        if (__any_sync(kFull, hc > 0)) {
            const int incl = warp_incl_sum(hc);
            const int m = __shfl_sync(kFull, incl, 31);
            const int rank0 = incl - hc;
            for (int r0 = 0; r0 < m;) {
                if (pn == C::kPCap) flush_pending(R);
                const int take = min(C::kPCap - pn, m - r0);
                if (hm) {
                    int r = rank0;
                    unsigned bits = hm;
                    while (bits) {
                        const int j = __ffs(bits) - 1;
                        bits &= bits - 1;
                        if (r >= r0 && r < r0 + take) {
                            pxy()[pn + r - r0] = tb[sbase + j];
                            pidx()[pn + r - r0] = IDX_SMEM ? idx_arr[sbase + j] : (int)(start + sbase + j);
                        }
                        ++r;
                    }
                }
                __syncwarp();
                pn += take;
                r0 += take;
            }
            if (pn >= 32) flush_pending(R);
        }
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
        float pm_carry = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        if (a > 0) {
            prev_pt = P[a - 1];
            has_prev = true;
        }
        const int npre = M < C::kS ? M : C::kS;
        if (lane == 0)
            for (int k = 0; k < npre; ++k) issue(P, a, b, k, seq + k);
        unsigned issued = seq + npre;
        __syncwarp();

        float ymax_prev = neg_inf();
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
                decide<false>(buf(s % C::kS) + tile_shift(P, st), cnt, st, nullptr, ymax_prev, ynext,
                              pm_carry, prev_pt, has_prev, R);
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
        }
        seq += M;
        flush_pending(R);
        write_r(R);
        const int count = R.g + R.w;
        if (it.nseg == 1) {
            if (lane == 0) args.out_count[it.set] = count;
            return true;
        }
        return publish_and_merge(it, item_index, R, pm_carry);
    }

    // End of a segment of a multi-segment set: publish the segment hood (its
    // indices are already in the output array; its coordinates go to the
    // workspace when it fits one window), its count and its max y. The warp
    // that completes the set's last segment merges the segment hoods.
    __device__ bool publish_and_merge(const SegItem &it, int item_index, RState &R, float segmax)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points) + it.set_base;
        int32_t *out = args.out_idx + it.set_base;
        const SegStore ss = store();
        const int count = R.g + R.w;
        const int stage0 = args.items ? args.items[item_index - it.c].pad : 0;
        if (R.g == 0) {
            float2 *dst = ss.xy + (size_t)(stage0 + it.c) * C::kRCap;
            for (int k = lane; k < R.w; k += 32) dst[k] = rxy()[k];
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
        if (old != (unsigned)(it.nseg - 1)) return true;
        __threadfence();
        const GlobSrc src{ss, out, P, args.items ? args.items + (item_index - it.c) : nullptr, it.slot0, stage0,
                          (long long)args.tiles, args.nseg, it.nseg};
        int *scratch = merge_scratch(it.nseg, ss.live + 4 * (size_t)stage0);
        RState F{0, 0, out, P};
        merge_hoods(src, scratch, F);
        write_r(F);
        if (lane == 0) {
            args.out_count[it.set] = F.g + F.w;
            args.arrivals[it.set] = 0;
        }
        __syncwarp();
        return true;
    }

    // ------------------------------------------------------- hood sources
    // A merge pass takes a list of hoods, left to right, each with the max y
    // over the points it came from, its corner count (negative, -count - 1,
    // when its coordinates must be gathered through the indices) and its
    // corners. fetch() loads a batch of up to 8 corners with all loads in
    // flight at once.

    // Hoods published in the workspace by other warps.
    struct GlobSrc {
        SegStore ss;
        const int32_t *out;
        const float2 *P;
        const SegItem *items;  // batched: the set's items; else nullptr
        int slot0;             // count / max-y slot of entry 0
        int stage0;            // stage slot of entry 0
        long long tiles;       // single set: tiles and segments, to locate
        int nseg;              //   segment starts
        int n;                 // number of entries
        __device__ float ymax(int i) const { return __ldcg(ss.ymax + slot0 + i); }
        __device__ int rawcount(int i) const { return __ldcg(ss.count + slot0 + i); }
        __device__ long long start(int i) const
        {
            if (items) return items[i].a;
            return ((long long)i * tiles / nseg) * C::kT;
        }
        // corner `off` of hood c (raw count, start a) for each u with bit u set
        __device__ __forceinline__ void fetch(unsigned valid, const int *c, const int *off, const int *raw,
                                              const long long *a, float2 *p, int *id) const
        {
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if ((valid >> u) & 1u) id[u] = __ldcg(out + a[u] + off[u]);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (((valid >> u) & 1u) && raw[u] >= 0)
                    p[u] = __ldcg(ss.xy + (size_t)(stage0 + c[u]) * C::kRCap + off[u]);
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (((valid >> u) & 1u) && raw[u] < 0) p[u] = P[id[u]];
        }
    };

    // ------------------------------------------------------- merge pass
    // Merge the hoods of src (left to right) into R. Hood staircase first: a
    // hood is dropped whole when its max y is at most the max over all earlier
    // hoods' points and below the max over some later hood's points (every
    // corner of it then lies on or below a segment between two input points).
    // The corners of the remaining hoods, concatenated in order, are streamed
    // through the tile pass (no look-ahead). scratch: 4 * src.n + 1 ints.
    template <class Src>
    __device__ void merge_hoods(const Src &src, int *scratch, RState &R)
    {
        const int nh = src.n;
        float *yv = reinterpret_cast<float *>(scratch);
        int *nv = scratch + nh;        // raw counts
        int *live_seg = scratch + 2 * nh;
        int *live_pre = scratch + 3 * nh;
        // Metadata, with many loads in flight.
        for (int c0 = 0; c0 < nh; c0 += 256) {
            float y[8];
            int r[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + u * 32 + lane;
                if (c < nh) {
                    y[u] = src.ymax(c);
                    r[u] = src.rawcount(c);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int c = c0 + u * 32 + lane;
                if (c < nh) {
                    yv[c] = y[u];
                    nv[c] = r[u];
                }
            }
        }
        __syncwarp();
        // Backward sweep: max over later hoods (kept in live_pre for now).
        float carry_suf = neg_inf();
        for (int b0 = ((nh - 1) >> 5) << 5; b0 >= 0; b0 -= 32) {
            const int c = b0 + lane;
            const float ym = c < nh ? yv[c] : neg_inf();
            const float isuf = warp_incl_suffix_max(ym);
            float esuf = __shfl_down_sync(kFull, isuf, 1);
            if (lane == 31) esuf = neg_inf();
            if (c < nh) live_pre[c] = __float_as_int(fmaxf(esuf, carry_suf));
            carry_suf = fmaxf(carry_suf, __shfl_sync(kFull, isuf, 0));
        }
        __syncwarp();
        // Forward sweep: max over earlier hoods; keep the live hoods and the
        // prefix of their corner counts.
        float carry_pre = neg_inf();
        int nlive = 0, total = 0;
        for (int b0 = 0; b0 < nh; b0 += 32) {
            const int c = b0 + lane;
            float ym = neg_inf(), later = neg_inf();
            int cntc = 0;
            if (c < nh) {
                ym = yv[c];
                later = __int_as_float(live_pre[c]);
                const int r = nv[c];
                cntc = r < 0 ? -r - 1 : r;
            }
            const float ipre = warp_incl_prefix_max(ym);
            float epre = __shfl_up_sync(kFull, ipre, 1);
            if (lane == 0) epre = neg_inf();
            const float before = fmaxf(epre, carry_pre);
            const bool keep = c < nh && cntc > 0 && !(!(ym > before) && ym < later);
            const unsigned km = __ballot_sync(kFull, keep);
            const int kr = __popc(km & ((1u << lane) - 1u));
            const int kc = keep ? cntc : 0;
            const int incl = warp_incl_sum(kc);
            __syncwarp();
            if (keep) {
                live_seg[nlive + kr] = c;
                live_pre[nlive + kr] = total + incl - kc;
            }
            __syncwarp();
            nlive += __popc(km);
            total += __shfl_sync(kFull, incl, 31);
            carry_pre = fmaxf(carry_pre, __shfl_sync(kFull, ipre, 31));
        }
        if (lane == 0) live_pre[nlive] = total;
        __syncwarp();

        pn = 0;
        float pm_carry = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        float2 *t0 = buf(0);
        int *ti = reinterpret_cast<int *>(buf(1));
        int cur = 0;  // live hood holding the first entry of the tile
        for (int v0 = 0; v0 < total; v0 += C::kT) {
            const int cnt = total - v0 < C::kT ? total - v0 : C::kT;
            // Each lane gathers its strip of K consecutive entries, walking
            // forward through the live hoods, 8 corners per batch of loads.
            const int e0 = lane * C::kK;
            int l = cur;
            if (e0 < cnt)
                while (l + 1 < nlive && live_pre[l + 1] <= v0 + e0) ++l;
            for (int jb = 0; jb < C::kK; jb += 8) {
                int cc[8], off[8], raw[8];
                long long aa[8];
                float2 p[8];
                int id[8];
                unsigned valid = 0;
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = e0 + jb + u;
                    cc[u] = 0;
                    off[u] = 0;
                    raw[u] = 0;
                    aa[u] = 0;
                    p[u] = make_float2(0.f, 0.f);
                    id[u] = 0;
                    if (jb + u < C::kK && e < cnt) {
                        const int v = v0 + e;
                        while (live_pre[l + 1] <= v) ++l;
                        cc[u] = live_seg[l];
                        off[u] = v - live_pre[l];
                        raw[u] = nv[cc[u]];
                        aa[u] = src.start(cc[u]);
                        valid |= 1u << u;
                    }
                }
                if (__any_sync(kFull, valid != 0)) {
                    src.fetch(valid, cc, off, raw, aa, p, id);
#pragma unroll
                    for (int u = 0; u < 8; ++u)
                        if ((valid >> u) & 1u) {
                            t0[e0 + jb + u] = p[u];
                            ti[e0 + jb + u] = id[u];
                        }
                }
            }
            while (cur + 1 < nlive && live_pre[cur + 1] <= v0 + C::kT) ++cur;
            __syncwarp();
            const float ym = strip_max(t0, cnt);
            decide<true>(t0, cnt, 0, ti, ym, neg_inf(), pm_carry, prev_pt, has_prev, R);
            __syncwarp();
        }
        flush_pending(R);
    }

    // Scratch for a merge pass over nh hoods (4 nh + 1 ints). Single set: the
    // merging warp completed the last segment, so every other warp of its CTA
    // has finished with its shared memory; use the larger run of their
    // regions. Batched: this warp's free tile buffers, else the workspace.
    __device__ int *merge_scratch(int nh, int *global_scratch) const
    {
        const size_t need = (size_t)(4 * nh + 1) * 4;
        if (!args.items) {
            const int w = threadIdx.x >> 5;
            unsigned char *cta = base - C::kWarpBytes * w;
            const int after = C::kW - 1 - w;
            if (after >= w && (size_t)after * C::kWarpBytes >= need)
                return reinterpret_cast<int *>(cta + C::kWarpBytes * (w + 1));
            if (w > after && (size_t)w * C::kWarpBytes >= need) return reinterpret_cast<int *>(cta);
        }
        if (need <= (size_t)(C::kS - 2) * C::kBuf * 8) return reinterpret_cast<int *>(buf(2));
        return global_scratch;
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
    __syncwarp();

    // Test hook: one bounded wait on a barrier that nothing completes.
    const int stall = args.hdr->stall_test_ns;
    if (stall > 0) {
        bool tmo = false;
        if (lane == 0) tmo = !mbar_wait_bounded(bars + C::kS, 0, (uint64_t)stall);
        if (__any_sync(kFull, tmo)) {
            if (lane == 0) record_status(&args.hdr->status, kStTimeout);
            return;
        }
    }

    unsigned seq = 0;
    if (args.queue) {
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
        const int nitems = args.items ? args.num_items : args.nseg;
        const int gw = blockIdx.x * C::kW + warp, nw = gridDim.x * C::kW;
        for (int i = gw; i < nitems; i += nw)
            if (!Wk.run_segment(i, seq)) break;
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
}

// ---------------------------------------------------------------- launcher
template <class C, int MODE>
static cudaError_t launch_cfg(const FusedArgs &args, int grid, cudaStream_t stream)
{
    auto kern = fused_kernel<C, MODE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::kBytes);
    if (e != cudaSuccess) return e;
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
using Cfg1 = Cfg<8, 23, 4, 128, 64>;
using Cfg2 = Cfg<12, 15, 4, 128, 64>;
using Cfg3 = Cfg<8, 31, 3, 128, 64>;
using Cfg4 = Cfg<6, 31, 4, 128, 64>;

}  // namespace wg
