// wg_sort.cu -- the step before the path: unsorted grid points sorted by
// (x, y), with the permutation (Section 2 assumes its input sorted left to
// right; this supplies that order on the device).
//
// A point (x, y) on the 2^-24 grid has integer coordinates kx = x 2^24 and
// ky = y 2^24 below 2^24; the 48-bit key kx 2^24 + ky orders points exactly
// as (x, y) lexicographically. Keys are sorted by a least-significant-digit
// radix sort, six passes of 8 bits, each pass stable:
//   1. per block of 4096 keys, a histogram of the pass's digit;
//   2. an exclusive scan of the histograms in digit-major order (all
//      blocks' counts of digit 0, then of digit 1, ...), which gives every
//      block the first output position of each of its digits;
//   3. per block, each warp's 512 keys are ranked among the block's keys
//      of the same digit (counts per warp and digit, scanned over the
//      warps; then, 32 keys at a time in input order, the lanes holding
//      the same digit found by a match and ranked by lane), and scattered.
// Stability makes the whole sort stable: copies of a point keep their input
// order, so the first copy in sorted order is the first in the input.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "wg.h"
#include "wg_internal.h"
#include "wg_sort.h"

namespace wg {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortPerThread = 16;
constexpr int kSortTile = kSortThreads * kSortPerThread;  // 4096 keys per block
constexpr int kSortPerWarp = kSortTile / kSortWarps;      // 512
constexpr int kDigits = 256;
constexpr int kPasses = 6;
constexpr int kScanThreads = 1024;
constexpr int kScanPerThread = 8;
constexpr int kScanChunk = kScanThreads * kScanPerThread;  // 8192 entries per scan block
constexpr int kScatterDynSmem = kSortTile * (8 + 4);
static_assert(kSortThreads == kDigits, "the scatter's digit scan takes one thread per digit");

__global__ void sort_keys_kernel(const float2 *__restrict__ p, long long n, unsigned long long *__restrict__ key,
                                 int *__restrict__ val)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float2 v = p[i];
        const unsigned long long kx = (unsigned long long)(v.x * 16777216.f);
        const unsigned long long ky = (unsigned long long)(v.y * 16777216.f);
        key[i] = (kx << 24) | ky;
        val[i] = (int)i;
    }
}

__global__ void sort_out_kernel(const unsigned long long *__restrict__ key, long long n, float2 *__restrict__ out)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long k = key[i];
        out[i] = make_float2((float)(k >> 24) * 0x1p-24f, (float)(k & 0xffffffull) * 0x1p-24f);
    }
}

// 1. hist[d * nb + b] = keys of block b with digit d
__global__ void __launch_bounds__(kSortThreads) sort_hist_kernel(const unsigned long long *__restrict__ key,
                                                                 long long n, int shift, int nb,
                                                                 unsigned *__restrict__ hist)
{
    __shared__ unsigned cnt[kDigits];
    for (int d = threadIdx.x; d < kDigits; d += kSortThreads) cnt[d] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int k = threadIdx.x; k < kSortTile; k += kSortThreads) {
        const long long i = base + k;
        if (i < n) atomicAdd(&cnt[(unsigned)(key[i] >> shift) & (kDigits - 1)], 1u);
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kDigits; d += kSortThreads) hist[(size_t)d * nb + blockIdx.x] = cnt[d];
}

// Block-wide exclusive scan of v (kScanThreads threads); returns the total.
__device__ __forceinline__ unsigned scan_block(unsigned &v, unsigned *wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned s = lane < kScanThreads / 32 ? wsum[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < kScanThreads / 32) wsum[lane] = s;
    }
    __syncthreads();
    const unsigned before = (w > 0 ? wsum[w - 1] : 0u) + x - v;
    const unsigned total = wsum[kScanThreads / 32 - 1];
    __syncthreads();
    v = before;
    return total;
}

// 2a. exclusive scan of each chunk of kScanChunk entries in place; chunk sums out
__global__ void __launch_bounds__(kScanThreads) sort_scan_chunks_kernel(unsigned *__restrict__ a, long long m,
                                                                        unsigned *__restrict__ sums)
{
    __shared__ unsigned wsum[kScanThreads / 32];
    const long long c0 = (long long)blockIdx.x * kScanChunk + (long long)threadIdx.x * kScanPerThread;
    unsigned v[kScanPerThread];
    unsigned t = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        v[j] = c0 + j < m ? a[c0 + j] : 0u;
        t += v[j];
    }
    unsigned before = t;
    const unsigned total = scan_block(before, wsum);
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        if (c0 + j < m) a[c0 + j] = before;
        before += v[j];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// 2b. exclusive scan of the chunk sums (at most kScanChunk of them), one block
__global__ void __launch_bounds__(kScanThreads) sort_scan_sums_kernel(unsigned *__restrict__ sums, int m)
{
    __shared__ unsigned wsum[kScanThreads / 32];
    const int c0 = threadIdx.x * kScanPerThread;
    unsigned v[kScanPerThread];
    unsigned t = 0;
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        v[j] = c0 + j < m ? sums[c0 + j] : 0u;
        t += v[j];
    }
    unsigned before = t;
    scan_block(before, wsum);
#pragma unroll
    for (int j = 0; j < kScanPerThread; ++j) {
        if (c0 + j < m) sums[c0 + j] = before;
        before += v[j];
    }
}

// 2c. add each chunk's offset
__global__ void sort_scan_add_kernel(unsigned *__restrict__ a, long long m, const unsigned *__restrict__ sums)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        a[i] += sums[i / kScanChunk];
}

// 3. stable scatter of block b's keys to off[d * nb + b] + rank: ranked in
// shared memory first (the block's keys in digit order), then written out
// in that order, so that each digit's run leaves as consecutive stores
__global__ void __launch_bounds__(kSortThreads) sort_scatter_kernel(
    const unsigned long long *__restrict__ key, const int *__restrict__ val, long long n, int shift, int nb,
    const unsigned *__restrict__ off, unsigned long long *__restrict__ key_out, int *__restrict__ val_out)
{
    __shared__ unsigned wcnt[kSortWarps][kDigits];  // per warp and digit: count, then its first local position
    __shared__ unsigned dstart[kDigits];            // the block's first local position of each digit
    extern __shared__ __align__(16) unsigned char sdyn[];  // the block's keys and values in digit order
    unsigned long long *skey = reinterpret_cast<unsigned long long *>(sdyn);
    int *sval = reinterpret_cast<int *>(sdyn + 8 * kSortTile);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int k = threadIdx.x; k < kSortWarps * kDigits; k += kSortThreads) (&wcnt[0][0])[k] = 0;
    __syncthreads();
    // this warp's keys: [base, base + 512), lane l holding keys base + 32 r + l
    const long long b0 = (long long)blockIdx.x * kSortTile;
    const long long base = b0 + (long long)w * kSortPerWarp;
    const int nblk = (int)min((long long)kSortTile, n - b0);
    unsigned long long k[kSortPerThread];
    int vv[kSortPerThread];
    unsigned dg[kSortPerThread];
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const long long i = base + 32 * r + lane;
        const bool in = i < n;
        k[r] = in ? key[i] : 0ull;
        vv[r] = in ? val[i] : 0;
        dg[r] = in ? (unsigned)(k[r] >> shift) & (kDigits - 1) : kDigits;  // kDigits: no key
    }
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r)
        if (dg[r] < kDigits) atomicAdd(&wcnt[w][dg[r]], 1u);
    __syncthreads();
    // thread d: the block's count of digit d, then (after a scan over the
    // digits) each warp's first local position of digit d
    {
        const int d = threadIdx.x;  // kSortThreads == kDigits
        unsigned c = 0;
        for (int q = 0; q < kSortWarps; ++q) c += wcnt[q][d];
        // exclusive scan of c over the 256 digits
        unsigned x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        __shared__ unsigned ws[kSortWarps];
        if (lane == 31) ws[w] = x;
        __syncthreads();
        unsigned before = x - c;
        for (int q = 0; q < w; ++q) before += ws[q];
        dstart[d] = before;
        unsigned pos = before;
        for (int q = 0; q < kSortWarps; ++q) {
            const unsigned cq = wcnt[q][d];
            wcnt[q][d] = pos;
            pos += cq;
        }
    }
    __syncthreads();
    // 32 keys at a time, in input order: lanes with the same digit ranked by
    // lane, placed at their local position
    const unsigned lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < kSortPerThread; ++r) {
        const unsigned peers = __match_any_sync(0xffffffffu, dg[r]);
        if (dg[r] < kDigits) {
            const unsigned lp = wcnt[w][dg[r]] + __popc(peers & lt);
            skey[lp] = k[r];
            sval[lp] = vv[r];
        }
        __syncwarp();
        // the highest lane of each group advances the digit's position
        if (dg[r] < kDigits && (peers >> lane) == 1u) wcnt[w][dg[r]] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // local position i holds digit d's (i - dstart[d])-th key of the block
    for (int i = threadIdx.x; i < nblk; i += kSortThreads) {
        const unsigned long long kk = skey[i];
        const unsigned d = (unsigned)(kk >> shift) & (kDigits - 1);
        const unsigned g = off[(size_t)d * nb + blockIdx.x] + (unsigned)i - dstart[d];
        key_out[g] = kk;
        val_out[g] = sval[i];
    }
}

}  // namespace

size_t sort_workspace_bytes(long long n)
{
    const size_t nn = (size_t)(n > 0 ? n : 1);
    const size_t nb = (nn + kSortTile - 1) / kSortTile;
    const size_t m = nb * kDigits;
    const size_t nchunks = (m + kScanChunk - 1) / kScanChunk;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    return 2 * up(8 * nn) + 2 * up(4 * nn) + up(4 * m) + up(4 * nchunks);
}

cudaError_t sort_launch(const float *points, long long n, float *sorted, int32_t *perm, void *ws, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const size_t nn = (size_t)n;
    const int nb = (int)((nn + kSortTile - 1) / kSortTile);
    const long long m = (long long)nb * kDigits;
    const int nchunks = (int)((m + kScanChunk - 1) / kScanChunk);
    if (nchunks > kScanChunk) return cudaErrorInvalidValue;  // n beyond kSortMaxN
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    unsigned char *p = static_cast<unsigned char *>(ws);
    unsigned long long *key[2];
    int *val[2];
    key[0] = reinterpret_cast<unsigned long long *>(p);
    p += up(8 * nn);
    key[1] = reinterpret_cast<unsigned long long *>(p);
    p += up(8 * nn);
    val[0] = reinterpret_cast<int *>(p);
    p += up(4 * nn);
    val[1] = perm;  // the last pass (an even count) ends in key[0] / val[0]; val[1] is scratch
    unsigned *hist = reinterpret_cast<unsigned *>(p);
    p += up(4 * (size_t)m);
    unsigned *sums = reinterpret_cast<unsigned *>(p);
    static bool attr = false;  // set once (the same value every time, so a race is harmless)
    if (!attr) {
        if (cudaFuncSetAttribute(sort_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kScatterDynSmem) !=
            cudaSuccess)
            return cudaGetLastError();
        attr = true;
    }
    const int eb = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    sort_keys_kernel<<<eb, 256, 0, s>>>(reinterpret_cast<const float2 *>(points), n, key[0], val[0]);
    for (int pass = 0; pass < kPasses; ++pass) {
        const int in = pass & 1, out = in ^ 1;
        const int shift = 8 * pass;
        sort_hist_kernel<<<nb, kSortThreads, 0, s>>>(key[in], n, shift, nb, hist);
        sort_scan_chunks_kernel<<<nchunks, kScanThreads, 0, s>>>(hist, m, sums);
        sort_scan_sums_kernel<<<1, kScanThreads, 0, s>>>(sums, nchunks);
        const int ab = (int)std::min<long long>((m + 255) / 256, 152LL * 16);
        sort_scan_add_kernel<<<ab, 256, 0, s>>>(hist, m, sums);
        sort_scatter_kernel<<<nb, kSortThreads, kScatterDynSmem, s>>>(key[in], val[in], n, shift, nb, hist,
                                                                     key[out], val[out]);
    }
    // six passes: the result is in key[0] / val[0]
    sort_out_kernel<<<eb, 256, 0, s>>>(key[0], n, reinterpret_cast<float2 *>(sorted));
    if (cudaMemcpyAsync(perm, val[0], 4 * nn, cudaMemcpyDeviceToDevice, s) != cudaSuccess) return cudaGetLastError();
    return cudaGetLastError();
}

// out[i] = perm[out[i]] for i < *count
__global__ void sort_map_kernel(int32_t *__restrict__ out, const int32_t *__restrict__ count,
                                const int32_t *__restrict__ perm)
{
    const int c = *count;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c; i += gridDim.x * blockDim.x) out[i] = perm[out[i]];
}

cudaError_t sort_map_launch(int32_t *out, const int32_t *count, const int32_t *perm, long long n, cudaStream_t s)
{
    const int b = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
    sort_map_kernel<<<std::max(b, 1), 256, 0, s>>>(out, count, perm);
    return cudaGetLastError();
}

}  // namespace wg
