// wg_device.cuh -- device building blocks of the upper-hood path (sm_103a).
//
// Notation follows the paper (Section 2): a hood H(P) is the upper hull of a
// block P of consecutive points, stored as its corners left to right. Merging
// hoods P (left) and Q (right) needs the bridge (p, q): the corners where the
// upper common tangent touches H(P) and H(Q); the merged hood is
// P[0..p] ++ Q[q..] (match_and_merge, mam 6). The bridge is found with the
// paper's two classifications:
//   g(p, q_j): is q_j LOW / EQUAL / HIGH relative to the tangent corner of
//              H(Q) seen from p (mam 1, mam 2, mam 4);
//   f(p_i, q): is p_i LOW / EQUAL / HIGH relative to the tangent corner of
//              H(P) seen from q (mam 3, mam 5);
// and the Theorem after mam 2: with q'_i the tangent corner from p_i,
// f(p_i, q'_i) is LOW left of the bridge corner, EQUAL at it, HIGH right of
// it. Only the LOW tests are needed to locate the first non-LOW entry:
//   gLOW(p, j) = j < hq-1  and orient(p, Q[j], Q[j+1]) >= 0
//   fLOW(i)    = i < hp-1  and orient(P[i], Q[T(P[i])], P[i+1]) > 0
// where T(p) = first j with !gLOW(p, j). The ">= 0" in g and "> 0" in f fix
// the tie rule: on a bridge line the leftmost P corner and the rightmost Q
// corner are kept, so collinear points are never corners. Hood ends are
// handled by the index tests, not by the paper's "point directly below"
// sentinels, which mis-classify vertical bridges.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace wg {

constexpr unsigned kFull = 0xffffffffu;

// Status codes recorded on the device (same values as wg_status).
enum : int { kStOk = 0, kStUnsorted = 3, kStOffGrid = 4, kStTimeout = 5 };

// Predicate mode bits (template parameter MODE of every routine below).
enum : int { kModeFp64Only = 1, kModeCount = 2 };

// ---------------------------------------------------------------------------
// Orientation predicate (the paper's left_of, Section 2): sign of
// det(a - o, b - o), > 0 when b is left of the directed line o -> a.
//
// Inputs are grid points k * 2^-24 in [0, 1), so every coordinate difference
// is exact in float32. With t1 = fl(dx1 dy2), t2 = fl(dy1 dx2) and
// D = fl(t1 - t2) (round to nearest, no fused multiply-add), each rounding
// error is at most u = 2^-24 times the magnitude of its result, so
//   |D - det| <= u |t1 - t2| + u |t1| + u |t2| <= 2u (|t1| + |t2|).
// S = fl(|t1| + |t2|) >= (|t1| + |t2|) / (1 + u), and B = 2^-22 S is exact,
// so |D| > B implies |D| > 2u (|t1| + |t2|) >= |D - det|: sign(D) = sign(det)
// and det != 0. No underflow occurs: a nonzero product of grid differences is
// at least 2^-48. The bound is zero when nothing was rounded: both exact
// products are integer multiples of 2^-48, so if max(|t1|, |t2|) < 2^-25
// (rounding is monotone and 2^-25 is a float, so the exact products are below
// it too) they have fewer than 23 significant bits and are exact, and their
// difference, a multiple of 2^-48 below 2^-24, is exact as well: D = det and
// its sign, zero included, is final. Otherwise, when |D| <= B, the
// determinant is recomputed in float64, where both products (48 significant
// bits) and their difference (49 bits) are exact. The __f*_rn / __d*_rn
// intrinsics are never contracted into FMAs.
// ---------------------------------------------------------------------------
struct PredCount {
    unsigned long long tests = 0;
    unsigned long long fallbacks = 0;
};

template <int MODE>
__device__ __forceinline__ int orient(PredCount &pc, float2 o, float2 a, float2 b)
{
    const float dx1 = __fsub_rn(a.x, o.x), dy1 = __fsub_rn(a.y, o.y);
    const float dx2 = __fsub_rn(b.x, o.x), dy2 = __fsub_rn(b.y, o.y);
    if (MODE & kModeCount) pc.tests++;
    if (!(MODE & kModeFp64Only)) {
        const float t1 = __fmul_rn(dx1, dy2);
        const float t2 = __fmul_rn(dy1, dx2);
        const float d = __fsub_rn(t1, t2);
        if (fmaxf(fabsf(t1), fabsf(t2)) < 0x1p-25f) return (d > 0.f) - (d < 0.f);  // exact
        const float bound = __fmul_rn(__fadd_rn(fabsf(t1), fabsf(t2)), 0x1p-22f);
        if (fabsf(d) > bound) return d > 0.f ? 1 : -1;
        if (MODE & kModeCount) pc.fallbacks++;
    }
    const double e = __dsub_rn(__dmul_rn((double)dx1, (double)dy2),
                               __dmul_rn((double)dy1, (double)dx2));
    return (e > 0.0) - (e < 0.0);
}

__device__ __forceinline__ bool same_point(float2 a, float2 b)
{
    return a.x == b.x && a.y == b.y;
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

__device__ __forceinline__ float2 shfl2(float2 v, int src)
{
    return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}

// ---------------------------------------------------------------------------
// Warp scans.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_incl_prefix_max(float v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v = fmaxf(v, t);
    }
    return v;
}

__device__ __forceinline__ float warp_incl_suffix_max(float v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float t = __shfl_down_sync(kFull, v, o);
        if (lane + o < 32) v = fmaxf(v, t);
    }
    return v;
}

__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ int warp_incl_sum(int v)
{
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// ---------------------------------------------------------------------------
// Hood accessors: pt(i) returns corner i of a hood.
// ---------------------------------------------------------------------------
struct PtrHood {  // contiguous float2 corners (shared or global memory)
    const float2 *xy;
    __device__ __forceinline__ float2 pt(int i) const { return xy[i]; }
};

// Tangent corner T(p) of hood Q seen from p (p lex-left of all of Q): the
// first j with !gLOW(p, j). gLOW is true on a prefix of Q (g is LOW, then
// EQUAL, then HIGH along H(Q)), so binary search finds it.
template <int MODE, class QA>
__device__ __forceinline__ int tangent_from(PredCount &pc, float2 p, const QA &Q, int hq)
{
    int lo = 0, hi = hq - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (orient<MODE>(pc, p, Q.pt(mid), Q.pt(mid + 1)) >= 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

// Bridge of hoods P (hp >= 1 corners) and Q (hq >= 1), P lex-left of Q, by
// one warp (all 32 lanes call it with the same arguments). Sampled search in
// the spirit of mam 1-5: each round probes up to 32 corners of P (one per
// lane); every probing lane finds its tangent corner on Q and evaluates f; a
// ballot of the LOW votes narrows the bracket of the bridge corner p to one
// sampling interval. Rounds: ceil(log32 hp); per lane ~log2(hq) + 1 tests.
// Returns (p, q) in every lane.
template <int MODE, class PA, class QA>
__device__ __noinline__ int2 bridge_warp_range(PredCount &pc, const PA &P, int lo, int hi, int thi, const QA &Q, int hq)
{
    // invariant: lo <= p* <= hi and !fLOW(hi); thi = tangent corner from
    // P[hi] once a probe found it, else -1
    const int lane = lane_id();
    while (lo < hi) {
        const int span = hi - lo;
        const int step = (span + 31) >> 5;
        const int i = lo + lane * step;
        const bool valid = i < hi;
        bool low = false;
        int t = 0;
        if (valid) {
            const float2 p = P.pt(i);
            t = tangent_from<MODE>(pc, p, Q, hq);
            low = orient<MODE>(pc, p, Q.pt(t), P.pt(i + 1)) > 0;
        }
        const unsigned vm = __ballot_sync(kFull, valid);
        const unsigned nl = __ballot_sync(kFull, valid && !low);
        if (nl) {
            const int f = __ffs(nl) - 1;
            const int nhi = lo + f * step;
            lo = f > 0 ? lo + (f - 1) * step + 1 : lo;
            hi = nhi;
            thi = __shfl_sync(kFull, t, f);
        } else {
            lo = lo + (31 - __clz(vm)) * step + 1;
        }
    }
    const int q = thi >= 0 ? thi : tangent_from<MODE>(pc, P.pt(lo), Q, hq);
    return make_int2(lo, q);
}

template <int MODE, class PA, class QA>
__device__ int2 bridge_warp(PredCount &pc, const PA &P, int hp, const QA &Q, int hq)
{
    return bridge_warp_range<MODE>(pc, P, 0, hp - 1, -1, Q, hq);
}

// The same bridge when p* is expected near the end of P (a running hood
// meeting the next chunk of points): the first round probes the last 32
// candidates P[hp-33 .. hp-2] (one per lane). The f votes are LOW exactly
// before p*, so a first non-LOW vote after the first probe fixes p*, no
// non-LOW vote gives p* = hp - 1, and a non-LOW first probe leaves
// p* <= hp - 33 to the sampled search.
template <int MODE, class PA, class QA>
__device__ int2 bridge_tail(PredCount &pc, const PA &P, int hp, const QA &Q, int hq)
{
    if (hp <= 33) return bridge_warp<MODE>(pc, P, hp, Q, hq);
    const int lane = lane_id();
    const int i0 = hp - 33;
    const int i = i0 + lane;
    const float2 p = P.pt(i);
    const int t = tangent_from<MODE>(pc, p, Q, hq);
    const bool low = orient<MODE>(pc, p, Q.pt(t), P.pt(i + 1)) > 0;
    const unsigned nl = __ballot_sync(kFull, !low);
    if (!nl) return make_int2(hp - 1, tangent_from<MODE>(pc, P.pt(hp - 1), Q, hq));
    const int f = __ffs(nl) - 1;
    const int tf = __shfl_sync(kFull, t, f);
    if (f > 0) return make_int2(i0 + f, tf);
    return bridge_warp_range<MODE>(pc, P, 0, i0, tf, Q, hq);
}

// The same bridge for small hoods (1 <= hp, hq <= 32), corners held one per
// lane: lane i holds P[i] and Q[i]. Every P corner finds its tangent corner on
// Q by tangent_from's binary search (a fixed ceil(log2 hq) steps for the
// whole warp, lanes that are done keep their bracket), with Q's corners
// fetched by shuffles; one round of f votes over all of P then gives the
// bridge corner: the first corner whose vote is not LOW, else the last one.
// These are the probes bridge_warp makes when it samples every corner of P,
// so the result is the same.
template <int MODE, class PA, class QA>
__device__ int2 bridge_small(PredCount &pc, const PA &P, int hp, const QA &Q, int hq)
{
    const int lane = lane_id();
    const float2 pi = lane < hp ? P.pt(lane) : make_float2(0.f, 0.f);
    const float2 qi = lane < hq ? Q.pt(lane) : make_float2(0.f, 0.f);
    int lo = 0, hi = hq - 1;
    const int steps = hq > 1 ? 32 - __clz(hq - 1) : 0;
    for (int k = 0; k < steps; ++k) {
        const int mid = (lo + hi) >> 1;
        const float2 a = shfl2(qi, mid), b = shfl2(qi, min(mid + 1, 31));
        if (lo < hi && lane < hp) {
            if (orient<MODE>(pc, pi, a, b) >= 0)
                lo = mid + 1;
            else
                hi = mid;
        }
    }
    const float2 qt = shfl2(qi, lo);
    const float2 pn = shfl2(pi, (lane + 1) & 31);
    const bool vote = lane < hp - 1 && !(orient<MODE>(pc, pi, qt, pn) > 0);
    const unsigned nl = __ballot_sync(kFull, vote);
    const int p = nl ? __ffs(nl) - 1 : hp - 1;
    return make_int2(p, __shfl_sync(kFull, lo, p));
}

// Tangent corner T(p) of hood Q seen from p by the whole warp: each round the
// 32 lanes test gLOW at 32 evenly spaced corners of the current bracket and
// a ballot keeps the interval before the first corner that is not LOW, so a
// round divides the bracket by 32 (ceil(log32 hq) rounds instead of
// ceil(log2 hq) dependent steps). Returns T(p) in every lane.
template <int MODE, class QA>
__device__ int tangent_warp(PredCount &pc, float2 p, const QA &Q, int hq)
{
    const int lane = lane_id();
    int lo = 0, hi = hq - 1;  // T(p) in [lo, hi]; gLOW(p, hi) is false
    while (lo < hi) {
        const int step = (hi - lo + 31) >> 5;
        const int j = lo + lane * step;
        const bool valid = j < hi;
        bool low = false;
        if (valid) low = orient<MODE>(pc, p, Q.pt(j), Q.pt(j + 1)) >= 0;
        const unsigned nl = __ballot_sync(kFull, valid && !low);
        const unsigned vm = __ballot_sync(kFull, valid);
        if (nl) {
            const int f = __ffs(nl) - 1;
            hi = lo + f * step;
            lo = f > 0 ? lo + (f - 1) * step + 1 : lo;
        } else {
            lo = lo + (31 - __clz(vm)) * step + 1;
        }
    }
    return lo;
}

// Bridge of hoods P and Q by a whole CTA (every thread calls it with the
// same arguments; nw = blockDim.x / 32 warps, at most 32), for hoods of many
// thousands of corners: the multi-level bracketing of the paper's closing
// section, with sampling on both hoods. Each round samples nw corners of
// P's bracket, one per warp; each warp finds its corner's tangent corner on
// Q with the 32-way search (tangent_warp) and evaluates the f vote; the
// first corner whose vote is not LOW narrows P's bracket to one sampling
// interval. Rounds: ceil(log_nw hp), each of ceil(log32 hq) warp rounds.
// sh: 2 nw + 2 ints of shared memory. Returns (p, q) in every thread.
template <int MODE, class PA, class QA>
__device__ int2 bridge_cta(PredCount &pc, const PA &P, int hp, const QA &Q, int hq, int *sh)
{
    const int lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int *vote = sh, *tang = sh + nw, *ctl = sh + 2 * nw;
    int lo = 0, hi = hp - 1, thi = -1;  // p* in [lo, hi]; fLOW(hi) is false
    while (lo < hi) {
        const int step = (hi - lo + nw - 1) / nw;
        const int i = lo + warp * step;
        const bool valid = i < hi;
        int t = 0;
        bool low = false;
        if (valid) {
            const float2 pi = P.pt(i);
            t = tangent_warp<MODE>(pc, pi, Q, hq);
            low = orient<MODE>(pc, pi, Q.pt(t), P.pt(i + 1)) > 0;
        }
        if (lane == 0) {
            vote[warp] = valid ? (low ? 1 : 0) : 2;
            tang[warp] = t;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int f = -1, last = -1;
            for (int w = 0; w < nw; ++w) {
                if (vote[w] == 2) break;
                last = w;
                if (vote[w] == 0) {
                    f = w;
                    break;
                }
            }
            ctl[0] = f;
            ctl[1] = last;
        }
        __syncthreads();
        const int f = ctl[0], last = ctl[1];
        if (f >= 0) {
            thi = tang[f];
            hi = lo + f * step;
            lo = f > 0 ? lo + (f - 1) * step + 1 : lo;
        } else {
            lo = lo + last * step + 1;
        }
        __syncthreads();
    }
    const int q = thi >= 0 ? thi : tangent_warp<MODE>(pc, P.pt(lo), Q, hq);
    return make_int2(lo, q);
}

// ---------------------------------------------------------------------------
// Hood of up to 32 sorted, distinct points held one per lane (lanes [0, m)),
// computed in registers by the paper's stages d = 1, 2, 4, 8, 16: at stage d
// every group of 2d lanes merges its left hood P (lanes [g, g+d), hp corners,
// left-packed) with its right hood Q (lanes [g+d, g+2d), hq corners). Each P
// lane finds its tangent corner on Q by binary search over shuffled Q corners,
// a ballot of the f votes gives the bridge (p, q), and one shuffle per field
// packs P[0..p] ++ Q[q..] to the left of the group (mam 6).
// On return lanes [0, h) hold the corners (pt, id) left to right; returns h.
// ---------------------------------------------------------------------------
template <int MODE>
__device__ int warp_hood_regs(PredCount &pc, float2 &pt, int &id, int m)
{
    const int lane = lane_id();
    int cnt = lane < m ? 1 : 0;  // size of the hood of my group
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        if (d >= m) break;  // one group left: P holds every point, Q none
        const int g = lane & ~(2 * d - 1);
        const int r = lane - g;
        const int hp = __shfl_sync(kFull, cnt, g);
        const int hq = __shfl_sync(kFull, cnt, g + d);
        const bool act = (r < hp) && (hq > 0);
        int lo = 0, hi = hq > 0 ? hq - 1 : 0;
#pragma unroll
        for (int s = 1; s < d; s <<= 1) {
            const int mid = (lo + hi) >> 1;
            const int src = g + d + mid;
            const float2 qm = shfl2(pt, src);
            const float2 qn = shfl2(pt, min(src + 1, 31));
            if (act && lo < hi) {
                if (orient<MODE>(pc, pt, qm, qn) >= 0)
                    lo = mid + 1;
                else
                    hi = mid;
            }
        }
        const float2 qt = shfl2(pt, g + d + lo);
        const float2 pn = shfl2(pt, min(lane + 1, 31));
        bool low = false;
        if (act && r < hp - 1) low = orient<MODE>(pc, pt, qt, pn) > 0;
        const unsigned nl = __ballot_sync(kFull, act && !low);
        const unsigned gmask = (d >= 16) ? 0xffffu : ((1u << d) - 1u);
        const int pstar = __ffs((nl >> g) & gmask) - 1;
        const int qstar = __shfl_sync(kFull, lo, g + max(pstar, 0));
        int ncnt, src;
        if (hp > 0 && hq > 0) {
            ncnt = pstar + 1 + hq - qstar;
            src = r <= pstar ? lane : g + d + qstar + (r - pstar - 1);
        } else if (hp == 0) {
            ncnt = hq;
            src = g + d + r;
        } else {
            ncnt = hp;
            src = lane;
        }
        src = (r < ncnt) ? min(src, 31) : lane;
        const float2 np = shfl2(pt, src);
        const int nid = __shfl_sync(kFull, id, src);
        pt = np;
        id = nid;
        cnt = ncnt;
    }
    return cnt;
}

// ---------------------------------------------------------------------------
// Shared-memory, bulk-copy and timing helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

// Ends a barrier's life before its shared memory is put to another use.
__device__ __forceinline__ void mbar_inval(uint64_t *bar)
{
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> shared (the TMA engine's non-tensor form). dst, src
// 16-byte aligned, bytes a multiple of 16; completion is signalled on `bar`.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// L2 policy for data read once: evicted first, so that a stream much larger
// than L2 does not push out the workspace, the code and other reused lines.
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// The same bulk copy with an L2 cache policy.
__device__ __forceinline__ void bulk_g2s_hint(void *dst, const void *src, unsigned bytes, uint64_t *bar,
                                              uint64_t policy)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity of an mbarrier, for at most about
// `limit_ns` nanoseconds. Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
    }
    return false;
}

__device__ __forceinline__ void record_status(int *status, int code)
{
    atomicCAS(status, 0, code);
}

}  // namespace wg
