// wg_fused.cuh -- the fused upper-hood kernel (one launch per call).
//
// The paper's stage loop (Section 2, main) merges hoods of size d into hoods
// of size 2d for d = 1, 2, 4, ... with one launch per stage and the hood array
// copied to the host and back every stage. Here the whole schedule runs in one
// persistent launch:
//
//  * The input is split into segments of consecutive tiles (T = threads * K
//    points); each CTA owns whole segments. Tiles are staged into shared
//    memory by 1-D bulk copies (TMA) through an S-deep mbarrier pipeline.
//  * Per tile ("stages d = 1 .. T", fused):
//      - exact elimination pass: a point p is dropped when some earlier point
//        is at least as high and some later point (this tile, or the next
//        tile, already resident) is strictly higher; then p lies on or below a
//        segment between two input points and cannot be a corner. Repeats of
//        the previous input point are dropped (first occurrence wins).
//      - each thread builds the hood of its strip of K points serially (the
//        paper's Section 3 strips);
//      - the surviving strip corners are packed densely (block scan) and
//        merged by the paper's stages: d <= 16 inside a warp in registers
//        (warp_hood_regs), larger d across warps in shared memory with the
//        warp bridge search (bridge_warp) and mam 6 compaction.
//  * The CTA keeps a running hood of its segment (a shared-memory window of
//    its right end; older corners spill to the output array) and merges each
//    tile hood into it with one more bridge + compaction.
//  * The CTA that finishes the last segment of a set (an atomic arrival
//    count, no waiting) merges the segment hoods, by running the same tile
//    pass over their concatenation, and writes the result.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "wg_device.cuh"
#include "wg_internal.h"

namespace wg {

constexpr uint64_t kWaitNs = 1000000000ull;  // 1 s bound on any device wait

__device__ __forceinline__ float neg_inf() { return __int_as_float(0xff800000); }

template <int NT, int K, int S, int RCAP>
struct Cfg {
    static constexpr int kNT = NT, kNW = NT / 32, kK = K, kT = NT * K, kS = S, kRCap = RCAP;
    static constexpr int kBuf = kT + 2;  // points per tile buffer (+2: alignment shift)
    static constexpr int kMaxChunks = (kT + 31) / 32;
    static constexpr size_t kOffTiles = 0;
    static constexpr size_t kOffIdx = kOffTiles + size_t(S) * kBuf * 8;
    static constexpr size_t kOffRxy = kOffIdx + ((size_t(kT) * 4 + 15) / 16) * 16;
    static constexpr size_t kOffRidx = kOffRxy + size_t(RCAP) * 8;
    static constexpr size_t kOffDesc = kOffRidx + size_t(RCAP) * 4;
    static constexpr size_t kOffWarp = kOffDesc + ((size_t(kMaxChunks) * 8 + 15) / 16) * 16;
    static constexpr size_t kOffBar = kOffWarp + 3 * 32 * 4;
    static constexpr size_t kOffMisc = kOffBar + 8 * (S + 1);
    static constexpr size_t kBytes = kOffMisc + 16;
    static_assert(K % 2 == 1 && K < 32, "K must be odd (bank-conflict-free strips) and < 32");
    static_assert(kT % 2 == 0, "tile must hold an even number of points");
    static_assert(S >= 2, "two tile buffers at least");
    static_assert(RCAP % 64 == 0, "window must split in halves of whole warps");
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

template <class C, int MODE>
struct Fused {
    const FusedArgs &args;
    unsigned char *base;
    PredCount pc;
    int tid, lane, warp;

    __device__ Fused(const FusedArgs &a, unsigned char *b) : args(a), base(b)
    {
        tid = threadIdx.x;
        lane = tid & 31;
        warp = tid >> 5;
    }

    __device__ float2 *buf(int b) const { return reinterpret_cast<float2 *>(base + C::kOffTiles) + size_t(b) * C::kBuf; }
    __device__ int *tidx() const { return reinterpret_cast<int *>(base + C::kOffIdx); }
    __device__ float2 *rxy() const { return reinterpret_cast<float2 *>(base + C::kOffRxy); }
    __device__ int *ridx() const { return reinterpret_cast<int *>(base + C::kOffRidx); }
    __device__ int2 *desc() const { return reinterpret_cast<int2 *>(base + C::kOffDesc); }
    __device__ float *wA() const { return reinterpret_cast<float *>(base + C::kOffWarp); }
    __device__ float *wTot() const { return reinterpret_cast<float *>(base + C::kOffWarp) + 32; }
    __device__ int *wCnt() const { return reinterpret_cast<int *>(base + C::kOffWarp) + 64; }
    __device__ uint64_t *full() const { return reinterpret_cast<uint64_t *>(base + C::kOffBar); }
    __device__ int *misc() const { return reinterpret_cast<int *>(base + C::kOffMisc); }

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
        it.pad = 0;
        return it;
    }

    // ------------------------------------------------------- tile staging
    // Tile k of segment [a, b) of set points P goes to buffer (seq % S).
    // The 16-byte-aligned interior is one bulk copy; at most one point at each
    // end (when the tile start or end is not 16-byte aligned) is a plain load.
    // The plain stores precede the mbarrier arrive, whose release semantics
    // make them visible to threads that pass the wait.
    __device__ void issue(const float2 *P, long long a, long long b, int k, unsigned seq) const
    {
        const int bi = seq % C::kS;
        uint64_t *bar = full() + bi;
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
    __device__ void r_flush_half(RState &R) const
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

    // Append H[from..to) to the running hood (warp 0).
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
    // bridge (p, q), then R = R[0..p] ++ H[q..h) (warp 0).
    __device__ void r_merge(RState &R, const float2 *hxy, const int *hid, int h)
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

    // --------------------------------------------- merge of packed corners
    // Corners L[0..m) (m > 32) in shared memory: hoods of 32-point chunks in
    // registers, then the paper's stages over chunk hoods across warps.
    // Returns the hood as (start, count) into L.
    __device__ int2 cta_stages(float2 *L, int *Lid, int m)
    {
        const int nc = (m + 31) >> 5;
        int2 *ds = desc();
        for (int c = warp; c < nc; c += C::kNW) {
            const int e = c * 32 + lane;
            const int mc = min(32, m - c * 32);
            float2 pt = make_float2(0.f, 0.f);
            int id = 0;
            if (lane < mc) {
                pt = L[e];
                id = Lid[e];
            }
            const int h = warp_hood_regs<MODE>(pc, pt, id, mc);
            if (lane < h) {
                L[c * 32 + lane] = pt;
                Lid[c * 32 + lane] = id;
            }
            if (lane == 0) ds[c] = make_int2(c * 32, h);
            __syncwarp();
        }
        __syncthreads();
        for (int st = 1; st < nc; st <<= 1) {
            for (int k = warp;; k += C::kNW) {
                const int a = 2 * st * k, bq = a + st;
                if (bq >= nc) break;
                const int2 P = ds[a], Q = ds[bq];
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
            __syncthreads();
        }
        return ds[0];
    }

    // ------------------------------------------------ one tile, decided
    // Tile in buffer bi (points at buf(bi) + shift, cnt of them, the first at
    // set-relative index `start`); ymax_mine = max y of this thread's strip.
    // If IDX_SMEM the input indices are in tidx(), else start + position.
    // Returns false if the CTA must stop (timeout seen by some thread).
    template <bool IDX_SMEM>
    __device__ bool decide(int bi, int shift, int cnt, long long start, float ymax_mine,
                           bool lookahead, bool timed_out, float &pm_carry, float2 &prev_pt,
                           bool &has_prev, RState &R)
    {
        constexpr int K = C::kK;
        float2 *tb0 = buf(bi);
        const float2 *tb = tb0 + shift;

        // Block-level exclusive prefix / suffix maxima of the strip maxima.
        const float ipre = warp_incl_prefix_max(ymax_mine);
        const float isuf = warp_incl_suffix_max(ymax_mine);
        float epre = __shfl_up_sync(kFull, ipre, 1);
        float esuf = __shfl_down_sync(kFull, isuf, 1);
        if (lane == 0) epre = neg_inf();
        if (lane == 31) esuf = neg_inf();
        if (lane == 31) wTot()[warp] = ipre;
        if (__syncthreads_or(timed_out)) return false;  // S1
        float bpre = pm_carry, bsuf = neg_inf(), tmax = neg_inf(), ynext = neg_inf();
#pragma unroll 4
        for (int w = 0; w < C::kNW; ++w) {
            const float v = wTot()[w];
            tmax = fmaxf(tmax, v);
            if (w < warp) bpre = fmaxf(bpre, v);
            if (w > warp) bsuf = fmaxf(bsuf, v);
            if (lookahead) ynext = fmaxf(ynext, wA()[w]);
        }
        const float pm0 = fmaxf(bpre, epre);
        const float sm0 = fmaxf(fmaxf(bsuf, esuf), ynext);

        // Load my strip.
        const int sbase = tid * K;
        float px[K], py[K];
        int pid[IDX_SMEM ? K : 1];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int e = sbase + j;
            if (e < cnt) {
                const float2 v = tb[e];
                px[j] = v.x;
                py[j] = v.y;
                if (IDX_SMEM) pid[IDX_SMEM ? j : 0] = tidx()[e];
            } else {
                px[j] = 0.f;
                py[j] = neg_inf();
            }
        }
        const int nvalid = cnt - sbase;
        const unsigned vmask = nvalid >= K ? ((1u << K) - 1u) : (nvalid > 0 ? ((1u << nvalid) - 1u) : 0u);

        // Exact elimination: drop p when (some earlier y >= y_p) and (some
        // later y > y_p).
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
            const bool ks = py[j] < smx;
            if (!(((kpre >> j) & 1u) && ks)) surv |= 1u << j;
            smx = fmaxf(smx, py[j]);
        }
        surv &= vmask;

        // Previous input point of my first point.
        const float2 mylast = make_float2(px[K - 1], py[K - 1]);
        const float2 up = shfl2(mylast, lane > 0 ? lane - 1 : 0);
        float2 prev0 = prev_pt;
        bool has0 = has_prev;
        if (lane > 0) {
            prev0 = up;
            has0 = true;
        } else if (tid > 0) {
            prev0 = tb[sbase - 1];
            has0 = true;
        }

        if (args.validate && vmask) {
            int bad = 0;
#pragma unroll
            for (int j = 0; j < K; ++j) {
                if (!((vmask >> j) & 1u)) continue;
                const float x = px[j], y = py[j];
                const float sx = x * 16777216.f, sy = y * 16777216.f;
                if (!(x >= 0.f && x < 1.f && y >= 0.f && y < 1.f && sx == truncf(sx) && sy == truncf(sy)))
                    bad = kStOffGrid;
                const float2 pv = j == 0 ? prev0 : make_float2(px[j - 1], py[j - 1]);
                const bool hv = j == 0 ? has0 : true;
                if (hv && (pv.x > x || (pv.x == x && pv.y > y))) bad = bad ? bad : kStUnsorted;
            }
            if (bad) record_status(&args.hdr->status, bad);
        }

        // First occurrence wins.
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!((surv >> j) & 1u)) continue;
            const float2 pv = j == 0 ? prev0 : make_float2(px[j - 1], py[j - 1]);
            const bool hv = j == 0 ? has0 : true;
            if (hv && pv.x == px[j] && pv.y == py[j]) surv &= ~(1u << j);
        }

        // Hood of my strip's survivors (monotone scan; stack as a bit mask,
        // top two corners in registers, deeper ones re-read from the tile).
        unsigned hm = 0;
        int hn = 0;
        float2 A = make_float2(0.f, 0.f), B = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!((surv >> j) & 1u)) continue;
            const float2 Pj = make_float2(px[j], py[j]);
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

        const float2 next_prev = tb[cnt - 1];

        // Pack the strip hoods densely at the front of this buffer.
        const int hc = __popc(hm);
        const int icnt = warp_incl_sum(hc);
        if (lane == 31) wCnt()[warp] = icnt;
        __syncthreads();  // S2: every read of this tile is done
        int off = icnt - hc, m = 0;
        for (int w = 0; w < C::kNW; ++w) {
            const int v = wCnt()[w];
            if (w < warp) off += v;
            m += v;
        }
        int *Lid = tidx();
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (!((hm >> j) & 1u)) continue;
            const int pos = off + __popc(hm & ((1u << j) - 1u));
            tb0[pos] = make_float2(px[j], py[j]);
            Lid[pos] = IDX_SMEM ? pid[IDX_SMEM ? j : 0] : (int)(start + sbase + j);
        }
        fence_proxy_async_smem();
        __syncthreads();  // S3

        pm_carry = fmaxf(pm_carry, tmax);
        prev_pt = next_prev;
        has_prev = true;
        if (m == 0) return true;

        if (m <= 32) {
            if (warp == 0) {
                float2 pt = make_float2(0.f, 0.f);
                int id = 0;
                if (lane < m) {
                    pt = tb0[lane];
                    id = Lid[lane];
                }
                const int h = m <= 2 ? m : warp_hood_regs<MODE>(pc, pt, id, m);
                __syncwarp();
                if (lane < h) {
                    tb0[lane] = pt;
                    Lid[lane] = id;
                }
                __syncwarp();
                r_merge(R, tb0, Lid, h);
            }
        } else {
            const int2 H = cta_stages(tb0, Lid, m);
            if (warp == 0 && H.y > 0) r_merge(R, tb0 + H.x, Lid + H.x, H.y);
        }
        fence_proxy_async_smem();
        __syncthreads();  // S4
        return true;
    }

    // Max y over this thread's strip of a tile.
    __device__ float strip_max(const float2 *tb, int cnt) const
    {
        float ym = neg_inf();
        const int sbase = tid * C::kK;
#pragma unroll
        for (int j = 0; j < C::kK; ++j) {
            const int e = sbase + j;
            if (e < cnt) ym = fmaxf(ym, tb[e].y);
        }
        return ym;
    }

    // Wait (bounded) for tiles [from, to) of this CTA's sequence after a
    // timeout, so that no bulk copy is still writing when the CTA exits.
    __device__ void drain(unsigned from, unsigned to) const
    {
        if (tid != 0) return;
        for (unsigned s = from; s < to; ++s)
            mbar_wait_bounded(full() + (s % C::kS), (s / C::kS) & 1u, kWaitNs / 10);
    }

    __device__ void write_r(RState &R) const
    {
        if (warp == 0)
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
        float pm_carry = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        if (a > 0) {
            prev_pt = P[a - 1];
            has_prev = true;
        }
        const int npre = M < C::kS ? M : C::kS;
        if (tid == 0)
            for (int k = 0; k < npre; ++k) issue(P, a, b, k, seq + k);
        unsigned issued = seq + npre;

        float ymax_prev = neg_inf();
        for (int i = 0; i <= M; ++i) {
            float ymax_cur = neg_inf();
            bool tmo = false;
            if (i < M) {
                const unsigned s = seq + i;
                const int bi = s % C::kS;
                tmo = !mbar_wait_bounded(full() + bi, (s / C::kS) & 1u, kWaitNs);
                if (!tmo) {
                    const long long st = a + (long long)i * C::kT;
                    const int cnt = (int)((b - st) < C::kT ? (b - st) : C::kT);
                    ymax_cur = strip_max(buf(bi) + tile_shift(P, st), cnt);
                }
                const float wm = warp_max(ymax_cur);
                if (lane == 0) wA()[warp] = wm;
            }
            if (i == 0) {
                if (__syncthreads_or(tmo)) {
                    record_status(&args.hdr->status, kStTimeout);
                    drain(seq, issued);
                    return false;
                }
            } else {
                const unsigned s = seq + i - 1;
                const long long st = a + (long long)(i - 1) * C::kT;
                const int cnt = (int)((b - st) < C::kT ? (b - st) : C::kT);
                if (!decide<false>(s % C::kS, tile_shift(P, st), cnt, st, ymax_prev, i < M, tmo,
                                   pm_carry, prev_pt, has_prev, R)) {
                    record_status(&args.hdr->status, kStTimeout);
                    drain(s + 1, issued);
                    return false;
                }
                if (tid == 0 && i - 1 + C::kS < M) {
                    issue(P, a, b, i - 1 + C::kS, seq + i - 1 + C::kS);
                    ++issued;
                }
            }
            ymax_prev = ymax_cur;
        }
        seq += M;

        write_r(R);
        int *mi = misc();
        if (tid == 0) mi[1] = R.g + R.w;
        __syncthreads();
        const int count = mi[1];
        if (it.nseg == 1) {
            if (tid == 0) args.out_count[it.set] = count;
            __syncthreads();
            return true;
        }
        if (tid == 0) args.seg_count[it.slot] = count;
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const unsigned old = atomicAdd(args.arrivals + it.set, 1u);
            mi[0] = (old == (unsigned)(it.nseg - 1)) ? 1 : 0;
        }
        __syncthreads();
        const bool last = mi[0] != 0;
        __syncthreads();
        if (last) {
            __threadfence();
            if (!final_pass(it, item_index)) return false;
            if (tid == 0) args.arrivals[it.set] = 0;
        }
        return true;
    }

    // Segment a_c of segment c of the set that item `it` belongs to.
    __device__ long long seg_start(const SegItem &it, int item_index, int c) const
    {
        if (args.items) return args.items[item_index - it.c + c].a;
        return ((long long)c * args.tiles / args.nseg) * C::kT;
    }

    // ------------------------------------------------------- final merge
    // The segment hoods of the set, concatenated in order, are themselves a
    // sorted point sequence whose hood is the set's hood; run the tile pass
    // over them (gathered with plain loads, no look-ahead).
    __device__ bool final_pass(const SegItem &it, int item_index)
    {
        const float2 *P = reinterpret_cast<const float2 *>(args.points) + it.set_base;
        int32_t *out = args.out_idx + it.set_base;
        const int nseg = it.nseg;
        int *pre = reinterpret_cast<int *>(buf(1));  // nseg + 1 prefix sums
        int *sa = pre + (nseg + 1);                  // segment starts
        for (int c = tid; c < nseg; c += C::kNT) {
            pre[c] = __ldcg(args.seg_count + it.slot0 + c);
            sa[c] = (int)seg_start(it, item_index, c);
        }
        __syncthreads();
        if (warp == 0) {
            int carry = 0;
            for (int b0 = 0; b0 < nseg; b0 += 32) {
                const int c = b0 + lane;
                const int v = c < nseg ? pre[c] : 0;
                const int inc = warp_incl_sum(v);
                __syncwarp();
                if (c < nseg) pre[c] = carry + inc - v;
                carry += __shfl_sync(kFull, inc, 31);
                __syncwarp();
            }
            if (lane == 0) pre[nseg] = carry;
        }
        __syncthreads();
        const int E = pre[nseg];

        RState R{0, 0, out, P};
        float pm_carry = neg_inf();
        float2 prev_pt = make_float2(0.f, 0.f);
        bool has_prev = false;
        float2 *t0 = buf(0);
        int *ti = tidx();
        for (int v0 = 0; v0 < E; v0 += C::kT) {
            const int cnt = E - v0 < C::kT ? E - v0 : C::kT;
            for (int e = tid; e < cnt; e += C::kNT) {
                const int v = v0 + e;
                int lo = 0, hi = nseg - 1;  // last c with pre[c] <= v
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (pre[mid] <= v) lo = mid; else hi = mid - 1;
                }
                const int id = __ldcg(out + sa[lo] + (v - pre[lo]));
                t0[e] = P[id];
                ti[e] = id;
            }
            __syncthreads();
            const float ym = strip_max(t0, cnt);
            if (!decide<true>(0, 0, cnt, 0, ym, false, false, pm_carry, prev_pt, has_prev, R))
                return false;
        }
        write_r(R);
        __syncthreads();
        if (tid == 0) args.out_count[it.set] = R.g + R.w;
        return true;
    }
};

template <class C, int MODE>
__global__ void __launch_bounds__(C::kNT) fused_kernel(FusedArgs args)
{
    extern __shared__ __align__(128) unsigned char smem[];
    Fused<C, MODE> F(args, smem);
    uint64_t *bars = F.full();
    if (threadIdx.x == 0) {
        for (int s = 0; s <= C::kS; ++s) mbar_init(bars + s, 1);
        fence_mbar_init();
    }
    __syncthreads();

    // Test hook: one bounded wait on a barrier that nothing completes.
    const int stall = args.hdr->stall_test_ns;
    if (stall > 0) {
        bool tmo = false;
        if (threadIdx.x == 0) tmo = !mbar_wait_bounded(bars + C::kS, 0, (uint64_t)stall);
        if (__syncthreads_or(tmo)) {
            if (threadIdx.x == 0) record_status(&args.hdr->status, kStTimeout);
            return;
        }
    }

    unsigned seq = 0;
    if (args.queue) {
        // Batched: items are taken from a shared queue, largest sets first
        // (the planning kernel orders them), until it runs dry.
        const int nitems = *args.num_items_dev;
        int *mi = F.misc();
        while (true) {
            if (threadIdx.x == 0) mi[2] = (int)atomicAdd(args.queue, 1u);
            __syncthreads();
            const int i = mi[2];
            __syncthreads();
            if (i >= nitems) break;
            if (!F.run_segment(i, seq)) break;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(args.done, 1u) == gridDim.x - 1) {
                *args.queue = 0;
                *args.done = 0;
            }
        }
    } else {
        const int nitems = args.items ? args.num_items : args.nseg;
        for (int i = blockIdx.x; i < nitems; i += gridDim.x)
            if (!F.run_segment(i, seq)) break;
    }

    if (MODE & kModeCount) {
        unsigned long long t = F.pc.tests, f = F.pc.fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_xor_sync(kFull, t, o);
            f += __shfl_xor_sync(kFull, f, o);
        }
        if ((threadIdx.x & 31) == 0) {
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

// The tile configurations (index 1..kNumTileCfgs in the ABI).
using Cfg1 = Cfg<256, 17, 3, 1024>;
using Cfg2 = Cfg<256, 9, 4, 1024>;
using Cfg3 = Cfg<512, 9, 3, 1024>;

}  // namespace wg
