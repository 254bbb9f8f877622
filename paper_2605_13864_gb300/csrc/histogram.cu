// histogram.cu -- counts of int32 values in equal-width integer bins
// (the thesis names histograms as future work, Sec. 9):
//   counts[b] = #{ i : lo + b*width <= src[i] < lo + (b+1)*width },  b < nbins.
//
// Each CTA of a persistent grid keeps its own copy of the histogram in shared
// memory (32-bit counters, shared-memory atomics), walks the input with
// 16-byte loads (grid-stride, four in flight per thread), and finally adds
// its non-zero counters into
// the int64 result with one global integer atomic each.  Counting is exact
// whatever the order, so the result is bit-exact.  Histograms with more bins
// than fit in shared memory count directly with global atomics.
#include <algorithm>
#include <climits>

#include "internal.h"

namespace optigpu {
namespace {

constexpr int kHistThreads = 512;
constexpr int kSmemBins = 12288; // 48 KiB of 32-bit counters

struct BinRule {
    int64_t lo;
    int64_t width;
    int64_t nbins;
    int shift; // log2(width) when width is a power of two, else -1

    __device__ __forceinline__ int64_t bin(int32_t x) const
    {
        const int64_t d = int64_t(x) - lo;
        if (d < 0)
            return -1;
        const int64_t b = shift >= 0 ? (d >> shift) : d / width;
        return b < nbins ? b : -1;
    }
};

// The same rule in 32-bit arithmetic, valid when lo is an int32 and
// width < 2^32: for x >= lo, x - lo lies in [0, 2^32) and is exact as an
// unsigned 32-bit value.  A width that is not a power of two divides by a
// multiply-high with a precomputed constant (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994, Fig. 4.1):
// with l = ceil(log2 width) and m = floor(2^32 (2^l - width) / width) + 1,
// floor(d / width) = (t + ((d - t) >> 1)) >> (l - 1), t = mulhi(m, d), for
// every 32-bit d.
struct BinRule32 {
    int32_t lo;
    uint32_t width;
    uint32_t nbins;
    int shift;      // log2(width) when width is a power of two, else -1
    uint32_t magic; // m, when shift < 0
    int l;          // ceil(log2 width), when shift < 0

    __device__ __forceinline__ int64_t bin(int32_t x) const
    {
        if (x < lo)
            return -1;
        const uint32_t d = uint32_t(x) - uint32_t(lo);
        uint32_t b;
        if (shift >= 0) {
            b = d >> shift;
        } else {
            const uint32_t t = __umulhi(magic, d);
            b = (t + ((d - t) >> 1)) >> (l - 1);
        }
        return b < nbins ? int64_t(b) : -1;
    }
};

// Host side of BinRule32's division by a width that is not a power of two
// (3 <= width < 2^32).
void invariant_divisor(uint64_t width, uint32_t *magic, int *l)
{
    int k = 0;
    while ((uint64_t(1) << k) < width)
        ++k;
    // 2^32 (2^k - width) < 2^63 since 2^k - width < width <= 2^32 and 2^k - width <= 2^31.
    *magic = uint32_t(((uint64_t(1) << 32) * ((uint64_t(1) << k) - width)) / width + 1);
    *l = k;
}

template <bool SMEM, typename Rule>
__global__ void __launch_bounds__(kHistThreads, 3)
histogram_kernel(const int32_t *__restrict__ src, int64_t n, Rule rule, int64_t nbins, unsigned long long *counts,
                 int vec_ok)
{
    extern __shared__ unsigned int local[];
    if (SMEM) {
        for (int64_t b = threadIdx.x; b < nbins; b += kHistThreads)
            local[b] = 0u;
        __syncthreads();
    }
    auto count = [&](int32_t x) {
        const int64_t b = rule.bin(x);
        if (b >= 0) {
            if (SMEM)
                atomicAdd(&local[b], 1u);
            else
                atomicAdd(&counts[b], 1ull);
        }
    };
    const int64_t tid = int64_t(blockIdx.x) * kHistThreads + threadIdx.x;
    const int64_t stride = int64_t(gridDim.x) * kHistThreads;
    if (vec_ok) {
        const int64_t nv = n / 4;
        const int4 *v = reinterpret_cast<const int4 *>(src);
        // kUnroll 16-byte loads per thread in flight before any is counted.
        constexpr int kUnroll = 4;
        int64_t i = tid;
        for (; i + (kUnroll - 1) * stride < nv; i += kUnroll * stride) {
            int4 q[kUnroll];
#pragma unroll
            for (int u = 0; u < kUnroll; ++u)
                q[u] = __ldcs(v + i + u * stride);
#pragma unroll
            for (int u = 0; u < kUnroll; ++u) {
                count(q[u].x);
                count(q[u].y);
                count(q[u].z);
                count(q[u].w);
            }
        }
        for (; i < nv; i += stride) {
            const int4 q = __ldcs(v + i);
            count(q.x);
            count(q.y);
            count(q.z);
            count(q.w);
        }
        for (int64_t j = nv * 4 + tid; j < n; j += stride)
            count(src[j]);
    } else {
        for (int64_t i = tid; i < n; i += stride)
            count(src[i]);
    }
    if (SMEM) {
        __syncthreads();
        for (int64_t b = threadIdx.x; b < nbins; b += kHistThreads)
            if (local[b])
                atomicAdd(&counts[b], static_cast<unsigned long long>(local[b]));
    }
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" optigpu_status optigpu_histogram_i32(const int32_t *src, int64_t n, int64_t lo, int64_t width,
                                                int32_t nbins, int64_t *counts, optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_histogram_i32");
    if (n < 0 || width < 1 || nbins < 1 || nbins > (1 << 26))
        return fail(OPTIGPU_ERR_INVALID_ARG, "histogram: need n >= 0, width >= 1, 1 <= nbins <= 2^26");
    if (!counts || reinterpret_cast<uintptr_t>(counts) % 8 || (n > 0 && (!src || reinterpret_cast<uintptr_t>(src) % 4)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "histogram: null or misaligned pointer");
    if (lo < -(int64_t(1) << 40) || lo > (int64_t(1) << 40) || width > (int64_t(1) << 40))
        return fail(OPTIGPU_ERR_INVALID_ARG, "histogram: lo and width must lie within +-2^40");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    optigpu_status st = check_cuda(cudaMemsetAsync(counts, 0, 8 * size_t(nbins), s), "histogram: clear counts");
    if (st != OPTIGPU_OK || n == 0)
        return st;
    DeviceInfo dev;
    if ((st = current_device(dev)) != OPTIGPU_OK)
        return st;
    BinRule rule{lo, width, nbins, -1};
    if ((width & (width - 1)) == 0) {
        int l = 0;
        while ((int64_t(1) << l) < width)
            ++l;
        rule.shift = l;
    }
    const bool smem = nbins <= kSmemBins;
    const size_t smem_bytes = smem ? sizeof(unsigned) * size_t(nbins) : 0;
    const bool narrow = lo >= INT32_MIN && lo <= INT32_MAX && width < (int64_t(1) << 32);
    const void *fn = narrow ? (smem ? reinterpret_cast<const void *>(&histogram_kernel<true, BinRule32>)
                                    : reinterpret_cast<const void *>(&histogram_kernel<false, BinRule32>))
                            : (smem ? reinterpret_cast<const void *>(&histogram_kernel<true, BinRule>)
                                    : reinterpret_cast<const void *>(&histogram_kernel<false, BinRule>));
    // One wave: as many CTAs as are resident at once (every CTA walks the
    // input grid-stride, so a second wave would run alone at the end).
    int per_sm = 0;
    if ((st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kHistThreads, smem_bytes),
                         "cudaOccupancyMaxActiveBlocksPerMultiprocessor(histogram)")) != OPTIGPU_OK)
        return st;
    const int64_t want = (n + int64_t(kHistThreads) * 16 - 1) / (int64_t(kHistThreads) * 16);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(want, int64_t(std::max(per_sm, 1)) * dev.num_sms));
    const int vec_ok = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 ? 1 : 0;
    auto *c = reinterpret_cast<unsigned long long *>(counts);
    const int64_t nb = nbins;
    if (narrow) {
        BinRule32 r32{int32_t(lo), uint32_t(width), uint32_t(nbins), rule.shift, 0u, 0};
        if (rule.shift < 0)
            invariant_divisor(uint64_t(width), &r32.magic, &r32.l);
        if (smem)
            histogram_kernel<true><<<unsigned(grid), kHistThreads, smem_bytes, s>>>(src, n, r32, nb, c, vec_ok);
        else
            histogram_kernel<false><<<unsigned(grid), kHistThreads, 0, s>>>(src, n, r32, nb, c, vec_ok);
    } else if (smem) {
        histogram_kernel<true><<<unsigned(grid), kHistThreads, smem_bytes, s>>>(src, n, rule, nb, c, vec_ok);
    } else {
        histogram_kernel<false><<<unsigned(grid), kHistThreads, 0, s>>>(src, n, rule, nb, c, vec_ok);
    }
    return check_cuda(cudaGetLastError(), "launch histogram");
}
