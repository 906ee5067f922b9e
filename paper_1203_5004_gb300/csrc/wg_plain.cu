// wg_plain.cu -- the paper's stage loop kept on the device, unfused.
//
// Section 2 (main): hoods of size d are merged pairwise into hoods of size 2d,
// d = 1, 2, 4, ..., one launch per stage; the paper copies the padded hood
// array host <-> device around every launch and uses REMOTE padding. Here the
// hoods stay on the device and are stored densely with explicit offsets:
// stage s reads hoods [off[h], off[h+1]) and writes the merged hood of every
// pair (2k, 2k+1) at an offset found by a single-pass scan with decoupled
// look-back (Merrill and Garland, 2016) over the merged lengths.
//
// Each thread owns one pair. Its bridge is found by the nested search on the
// paper's classifications (binary search on the f votes of P, each with a
// binary search of the g votes on Q); pairs whose hoods hold more than 64
// corners together are handed to the whole warp (bridge_warp, the sampled
// 32-way form of mam 1-5) and copied by the warp; pairs of more than 4096
// corners (the late stages of dense hoods) are bridged by the whole block
// with the multi-level search (bridge_cta).
#include <cuda_runtime.h>
#include <cstdint>

#include "wg_device.cuh"
#include "wg_internal.h"

namespace wg {

constexpr int kPlainThreads = 256;
constexpr int kSmallPair = 64;
constexpr int kHugePair = 4096;  // larger pairs: the whole block bridges them
constexpr unsigned long long kLbFlagA = 1ull << 62, kLbFlagP = 2ull << 62;
constexpr unsigned long long kLbMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_volatile_int(const int *p)
{
    return *reinterpret_cast<const volatile int *>(p);
}

// Per-thread bridge by nested binary searches (P, Q global hoods).
template <int MODE>
__device__ int2 bridge_serial(PredCount &pc, const PtrHood &P, int hp, const PtrHood &Q, int hq)
{
    int lo = 0, hi = hp - 1;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        const float2 p = P.pt(mid);
        const int t = tangent_from<MODE>(pc, p, Q, hq);
        if (orient<MODE>(pc, p, Q.pt(t), P.pt(mid + 1)) > 0)
            lo = mid + 1;
        else
            hi = mid;
    }
    return make_int2(lo, tangent_from<MODE>(pc, P.pt(lo), Q, hq));
}

template <int MODE, bool FIRST>
__global__ void __launch_bounds__(kPlainThreads) plain_stage_kernel(PlainArgs a)
{
    __shared__ int s_bid;
    __shared__ int s_wsum[kPlainThreads / 32];
    __shared__ long long s_prefix;
    __shared__ int s_nhuge, s_huge[kPlainThreads], s_pair[4], s_cta[2 * (kPlainThreads / 32) + 2];
    PredCount pc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_bid = (int)atomicAdd(a.ticket, 1u);
    __syncthreads();
    const int bid = s_bid;
    const long long pair = (long long)bid * kPlainThreads + tid;
    const bool valid = pair < a.out_hoods;
    const float2 *pts = reinterpret_cast<const float2 *>(a.points);
    const float2 *ixy = reinterpret_cast<const float2 *>(a.in_xy);

    // The two hoods of my pair.
    int pa = 0, hp = 0, qa = 0, hq = 0;
    float2 fp = make_float2(0.f, 0.f), fq = make_float2(0.f, 0.f);
    if (valid) {
        if (FIRST) {
            const long long i0 = 2 * pair, i1 = i0 + 1;
            fp = pts[i0];
            hp = (i0 == 0 || !same_point(pts[i0 - 1], fp)) ? 1 : 0;
            if (i1 < a.n) {
                fq = pts[i1];
                hq = same_point(fp, fq) ? 0 : 1;
            }
        } else {
            const long long h0 = 2 * pair;
            pa = a.in_off[h0];
            const int pe = a.in_off[h0 + 1];
            hp = pe - pa;
            if (h0 + 1 < a.in_hoods) {
                qa = pe;
                hq = a.in_off[h0 + 2] - pe;
            }
        }
    }
    // Bridge of small pairs by the thread itself.
    int bp = -1, bq = 0, len = 0;
    bool large = false, huge = false;
    if (valid) {
        if (hp == 0 || hq == 0) {
            len = hp + hq;
        } else if (FIRST) {
            bp = 0;
            bq = 0;
            len = 2;
        } else if (hp + hq <= kSmallPair) {
            const int2 r = bridge_serial<MODE>(pc, PtrHood{ixy + pa}, hp, PtrHood{ixy + qa}, hq);
            bp = r.x;
            bq = r.y;
            len = bp + 1 + hq - bq;
        } else if (hp + hq <= kHugePair) {
            large = true;
        } else {
            huge = true;
        }
    }
    // Huge pairs (the late stages): the whole block finds each bridge with
    // the multi-level search, one pair after the other.
    if (tid == 0) s_nhuge = 0;
    __syncthreads();
    if (huge) s_huge[atomicAdd(&s_nhuge, 1)] = tid;
    __syncthreads();
    for (int k = 0; k < s_nhuge; ++k) {
        const int owner = s_huge[k];
        if (tid == owner) {
            s_pair[0] = pa;
            s_pair[1] = hp;
            s_pair[2] = qa;
            s_pair[3] = hq;
        }
        __syncthreads();
        const int2 r = bridge_cta<MODE>(pc, PtrHood{ixy + s_pair[0]}, s_pair[1], PtrHood{ixy + s_pair[2]},
                                        s_pair[3], s_cta);
        if (tid == owner) {
            bp = r.x;
            bq = r.y;
            len = bp + 1 + hq - bq;
        }
        __syncthreads();
    }
    // Large pairs: the warp finds each bridge together.
    unsigned lm = __ballot_sync(kFull, large);
    while (lm) {
        const int L = __ffs(lm) - 1;
        lm &= lm - 1;
        const int Lpa = __shfl_sync(kFull, pa, L), Lhp = __shfl_sync(kFull, hp, L);
        const int Lqa = __shfl_sync(kFull, qa, L), Lhq = __shfl_sync(kFull, hq, L);
        const int2 r = bridge_warp<MODE>(pc, PtrHood{ixy + Lpa}, Lhp, PtrHood{ixy + Lqa}, Lhq);
        if (lane == L) {
            bp = r.x;
            bq = r.y;
            len = bp + 1 + hq - bq;
        }
    }
    large = large || huge;  // both are copied by the warp

    // Block exclusive scan of merged lengths, then decoupled look-back.
    const int incl = warp_incl_sum(len);
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    int local = incl - len, agg = 0;
    for (int w = 0; w < kPlainThreads / 32; ++w) {
        const int v = s_wsum[w];
        if (w < warp) local += v;
        agg += v;
    }
    if (tid == 0) {
        long long excl = 0;
        unsigned long long *lb = a.lookback;
        if (bid == 0) {
            st_release_u64(lb, kLbFlagP | (unsigned long long)agg);
        } else {
            st_release_u64(lb + bid, kLbFlagA | (unsigned long long)agg);
            int j = bid - 1;
            uint64_t t0 = 0;
            unsigned spins = 0;
            bool ok = true;
            while (true) {
                const unsigned long long v = ld_acquire_u64(lb + j);
                const unsigned long long flag = v >> 62;
                if (flag == 0) {
                    if ((++spins & 255u) == 0) {
                        if (t0 == 0) t0 = global_ns();
                        else if (global_ns() - t0 > 1000000000ull || ld_volatile_int(&a.hdr->status) != 0) {
                            ok = false;
                            break;
                        }
                    }
                    continue;
                }
                excl += (long long)(v & kLbMask);
                if (flag == 2) break;
                --j;
            }
            if (!ok) {
                record_status(&a.hdr->status, kStTimeout);
                excl = -1;
            } else {
                st_release_u64(lb + bid, kLbFlagP | (unsigned long long)(excl + agg));
            }
        }
        s_prefix = excl;
    }
    __syncthreads();
    const long long prefix = s_prefix;
    if (prefix < 0) return;  // timed out: output invalid, status recorded
    const int obase = (int)(prefix + local);

    const bool fin = a.final_idx != nullptr;
    int32_t *oidx = fin ? a.final_idx : a.out_idx;
    float2 *oxy = reinterpret_cast<float2 *>(a.out_xy);
    if (valid) {
        if (!fin) {
            a.out_off[pair] = obase;
            if (pair == a.out_hoods - 1) a.out_off[a.out_hoods] = obase + len;
        } else if (pair == 0) {
            *a.final_count = len;
        }
    }
    // Copy the merged hoods: P[0..bp] ++ Q[bq..hq) (or the non-empty side).
    if (valid && !large) {
        if (FIRST) {
            int o = obase;
            const long long i0 = 2 * pair;
            if (hp) {
                if (!fin) oxy[o] = fp;
                oidx[o++] = (int)i0;
            }
            if (hq) {
                if (!fin) oxy[o] = fq;
                oidx[o++] = (int)(i0 + 1);
            }
        } else {
            const int pend = (hq == 0) ? hp : (hp == 0 ? 0 : bp + 1);
            const int qbeg = (hp == 0) ? 0 : (hq == 0 ? hq : bq);
            int o = obase;
            for (int k = 0; k < pend; ++k, ++o) {
                if (!fin) oxy[o] = ixy[pa + k];
                oidx[o] = a.in_idx[pa + k];
            }
            for (int k = qbeg; k < hq; ++k, ++o) {
                if (!fin) oxy[o] = ixy[qa + k];
                oidx[o] = a.in_idx[qa + k];
            }
        }
    }
    lm = __ballot_sync(kFull, large);
    while (lm) {
        const int L = __ffs(lm) - 1;
        lm &= lm - 1;
        const int Lpa = __shfl_sync(kFull, pa, L), Lqa = __shfl_sync(kFull, qa, L);
        const int Lhq = __shfl_sync(kFull, hq, L);
        const int Lbp = __shfl_sync(kFull, bp, L), Lbq = __shfl_sync(kFull, bq, L);
        const int Lo = __shfl_sync(kFull, obase, L);
        for (int k = lane; k <= Lbp; k += 32) {
            if (!fin) oxy[Lo + k] = ixy[Lpa + k];
            oidx[Lo + k] = a.in_idx[Lpa + k];
        }
        const int nq = Lhq - Lbq;
        for (int k = lane; k < nq; k += 32) {
            if (!fin) oxy[Lo + Lbp + 1 + k] = ixy[Lqa + Lbq + k];
            oidx[Lo + Lbp + 1 + k] = a.in_idx[Lqa + Lbq + k];
        }
    }
    if (MODE & kModeCount) {
        unsigned long long t = pc.tests, f = pc.fallbacks;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            t += __shfl_xor_sync(kFull, t, o);
            f += __shfl_xor_sync(kFull, f, o);
        }
        if (lane == 0) {
            atomicAdd(&a.hdr->tests, t);
            atomicAdd(&a.hdr->fallbacks, f);
        }
    }
}

template <int MODE>
static cudaError_t plain_launch_mode(const PlainArgs &a, bool first, cudaStream_t st)
{
    const long long blocks = (a.out_hoods + kPlainThreads - 1) / kPlainThreads;
    if (first)
        plain_stage_kernel<MODE, true><<<(unsigned)blocks, kPlainThreads, 0, st>>>(a);
    else
        plain_stage_kernel<MODE, false><<<(unsigned)blocks, kPlainThreads, 0, st>>>(a);
    return cudaGetLastError();
}

long long plain_blocks(long long hoods) { return (hoods + kPlainThreads - 1) / kPlainThreads; }

cudaError_t plain_stage_launch(const PlainArgs &a, bool first, int mode, cudaStream_t st)
{
    switch (mode) {
    case 0: return plain_launch_mode<0>(a, first, st);
    case 1: return plain_launch_mode<1>(a, first, st);
    case 2: return plain_launch_mode<2>(a, first, st);
    default: return plain_launch_mode<3>(a, first, st);
    }
}

}  // namespace wg
