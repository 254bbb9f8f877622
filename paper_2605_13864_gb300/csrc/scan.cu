// scan.cu -- inclusive prefix sums, dst[i] = src[0] + ... + src[i]
// (the thesis names parallel prefix sum as future work, Sec. 9; the running
// sum of Listing 2.1's loop, keeping every intermediate value).
//
// Three launches, all in a fixed order, so results are bit-identical from run
// to run (a single-pass decoupled look-back would combine floats in a
// timing-dependent order):
//   1. chunk sums: the sum's own kernel (reduce_band) writes one FP64 / int64
//      partial per 16384-element chunk;
//   2. carries: one CTA turns the partials into exclusive prefixes (thread t
//      scans a contiguous run sequentially, then a block scan of the run
//      totals), carry[c] = partial[0] + ... + partial[c-1];
//   3. chunk scans: each chunk is scanned in four 4096-element sub-blocks,
//      staged through padded shared memory so that global loads and stores
//      are coalesced; thread t owns 16 consecutive elements, scans them
//      sequentially, the 256 thread totals are scanned with warp shuffles and
//      a shared-memory pass over the 8 warp totals, and every output adds the
//      FP64 carry of the chunk and of the preceding sub-blocks.
// int32 input gives exact int64 output.  Float input (fp32, bf16, fp16) is
// scanned in FP32 inside a sub-block, carried in FP64 between sub-blocks
// and chunks (the carry reaches each element as an FP32 hi + lo pair), and
// written as fp32.
#include <algorithm>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "reduce_core.cuh"

namespace optigpu {
namespace {

constexpr int kScanThreads = 256;
constexpr int kPerThread = 16;
constexpr int kSub = kScanThreads * kPerThread; // 4096 elements per sub-block
static_assert(kReduceChunk % kSub == 0, "chunks split into whole sub-blocks");

template <int DT>
struct ScanTraits;
// FP64 runs at a small fraction of the FP32 rate on this part, so a float
// carry is split once per sub-block into hi + lo (hi = the carry rounded to
// FP32, lo = the rounding error, also in FP32) and each output costs two FP32
// additions: hi + (lo + v), within an FP32 ulp of the exact carry + v.
struct SplitCarry {
    float hi, lo;
};

__device__ __forceinline__ SplitCarry split_carry(double c)
{
    const float hi = float(c);
    return SplitCarry{hi, float(c - double(hi))};
}

template <>
struct ScanTraits<OPTIGPU_INT32> {
    using Acc = long long; // in-sub-block accumulator
    using Carry = long long;
    using Split = long long;
    using Out = long long;
    __device__ static Acc load(const void *p, int64_t i) { return static_cast<const int32_t *>(p)[i]; }
    __device__ static Split split(Carry c) { return c; }
    __device__ static Out finish(Split c, Acc v) { return c + v; }
};

struct FloatFinish {
    using Carry = double;
    using Split = SplitCarry;
    using Out = float;
    __device__ static Split split(Carry c) { return split_carry(c); }
    __device__ static Out finish(Split c, float v) { return c.hi + (c.lo + v); }
};
template <>
struct ScanTraits<OPTIGPU_FLOAT32> : FloatFinish {
    using Acc = float;
    __device__ static Acc load(const void *p, int64_t i) { return static_cast<const float *>(p)[i]; }
};
template <>
struct ScanTraits<OPTIGPU_BFLOAT16> : FloatFinish {
    using Acc = float;
    __device__ static Acc load(const void *p, int64_t i)
    {
        return __uint_as_float(uint32_t(static_cast<const uint16_t *>(p)[i]) << 16);
    }
};
template <>
struct ScanTraits<OPTIGPU_FLOAT16> : FloatFinish {
    using Acc = float;
    __device__ static Acc load(const void *p, int64_t i)
    {
        return __half2float(__ushort_as_half(static_cast<const unsigned short *>(p)[i]));
    }
};

// Block-wide exclusive scan of one value per thread (fixed order: Kogge-Stone
// inside each warp, then the 8 warp totals by warp 0).  Returns the exclusive
// prefix; *total receives the block total (valid in every thread).
template <typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T *warp_tot, T *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T up = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d)
            incl += up;
    }
    if (lane == 31)
        warp_tot[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        T w = lane < kScanThreads / 32 ? warp_tot[lane] : T(0);
#pragma unroll
        for (int d = 1; d < kScanThreads / 32; d <<= 1) {
            const T up = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d)
                w += up;
        }
        if (lane < kScanThreads / 32)
            warp_tot[lane] = w; // inclusive prefix of warp totals
    }
    __syncthreads();
    const T before = warp > 0 ? warp_tot[warp - 1] : T(0);
    *total = warp_tot[kScanThreads / 32 - 1];
    __syncthreads(); // warp_tot is reused by the next call
    return before + (incl - v);
}

// Phase 2: carry[c] = sum of partial[0 .. c) (one CTA, fixed order).
template <typename P>
__global__ void __launch_bounds__(kScanThreads) scan_carries_kernel(const P *partials, P *carry, int64_t count)
{
    __shared__ P warp_tot[kScanThreads / 32];
    const int64_t per = (count + kScanThreads - 1) / kScanThreads;
    const int64_t lo = int64_t(threadIdx.x) * per, hi = min(count, lo + per);
    P run = 0;
    for (int64_t i = lo; i < hi; ++i)
        run += partials[i];
    P total;
    P before = block_exclusive_scan<P>(run, warp_tot, &total);
    for (int64_t i = lo; i < hi; ++i) {
        carry[i] = before;
        before += partials[i];
    }
}

// Shared staging of one sub-block.  Element e of the input lives at word
// e + e / 32 (one pad word per 32): both the coalesced fill (consecutive e
// across lanes) and the per-thread read of 16 consecutive elements (lanes 16
// elements apart) hit 32 distinct banks.  8-byte outputs use one pad slot
// per 16 elements for the same reason.
__device__ __forceinline__ int pad4(int e) { return e + (e >> 5); }
__device__ __forceinline__ int pad8(int e) { return e + (e >> 4); }

// Phase 3: scan every chunk (persistent grid-stride over chunks).  Global
// loads and stores are coalesced (thread t touches elements t + 256 k); the
// per-thread contiguous runs are gathered from and scattered to shared memory.
template <int DT>
__global__ void __launch_bounds__(kScanThreads)
scan_chunks_kernel(const void *__restrict__ src, void *__restrict__ dst, int64_t n, const void *carries,
                   int64_t num_chunks)
{
    using T = ScanTraits<DT>;
    using Acc = typename T::Acc;
    using Carry = typename T::Carry;
    using Out = typename T::Out;
    constexpr bool kWide = sizeof(Out) == 8;
    __shared__ Acc warp_tot[kScanThreads / 32];
    __shared__ union {
        Acc in[kSub + kSub / 32];
        Out out[kWide ? kSub + kSub / 16 : kSub + kSub / 32];
    } stage;
    const Carry *carry = static_cast<const Carry *>(carries);
    Out *out = static_cast<Out *>(dst);
    const int t = threadIdx.x;
    for (int64_t c = blockIdx.x; c < num_chunks; c += gridDim.x) {
        Carry run = carry[c];
        for (int sb = 0; sb < int(kReduceChunk / kSub); ++sb) {
            const int64_t base = c * kReduceChunk + int64_t(sb) * kSub;
            if (base >= n)
                break; // uniform across the CTA
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const int e = t + k * kScanThreads;
                stage.in[pad4(e)] = (base + e < n) ? T::load(src, base + e) : Acc(0);
            }
            __syncthreads();
            Acc v[kPerThread];
#pragma unroll
            for (int j = 0; j < kPerThread; ++j)
                v[j] = stage.in[pad4(t * kPerThread + j)];
#pragma unroll
            for (int j = 1; j < kPerThread; ++j)
                v[j] += v[j - 1];
            Acc total;
            const Acc before = block_exclusive_scan<Acc>(v[kPerThread - 1], warp_tot, &total);
            // (block_exclusive_scan ends with a barrier: stage.in is free.)
            const typename T::Split sc = T::split(run);
#pragma unroll
            for (int j = 0; j < kPerThread; ++j) {
                const int e = t * kPerThread + j;
                stage.out[kWide ? pad8(e) : pad4(e)] = T::finish(sc, before + v[j]);
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kPerThread; ++k) {
                const int e = t + k * kScanThreads;
                if (base + e < n)
                    out[base + e] = stage.out[kWide ? pad8(e) : pad4(e)];
            }
            __syncthreads();
            run += Carry(total);
        }
    }
}

template <int DT>
optigpu_status launch_scan(const void *src, void *dst, int64_t n, cudaStream_t stream)
{
    using T = ScanTraits<DT>;
    using P = typename std::conditional<DT == OPTIGPU_INT32, long long, double>::type;
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const int64_t num_chunks = (n + kReduceChunk - 1) / kReduceChunk;
    void *ws = nullptr;
    if ((st = stream_workspace(stream, size_t(num_chunks) * 16 + 256, &ws, 2)) != OPTIGPU_OK)
        return st;
    P *partials = static_cast<P *>(ws);
    P *carries = partials + num_chunks;
    if ((st = reduce_band(src, n, DT, 0u, partials, 0, stream)) != OPTIGPU_OK)
        return st;
    scan_carries_kernel<P><<<1, kScanThreads, 0, stream>>>(partials, carries, num_chunks);
    if ((st = check_cuda(cudaGetLastError(), "launch scan carries")) != OPTIGPU_OK)
        return st;
    const int64_t grid = std::min<int64_t>(num_chunks, int64_t(8) * dev.num_sms);
    scan_chunks_kernel<DT><<<unsigned(grid), kScanThreads, 0, stream>>>(src, dst, n, carries, num_chunks);
    (void)sizeof(T);
    return check_cuda(cudaGetLastError(), "launch scan chunks");
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" optigpu_status optigpu_scan_inclusive(const void *src, void *dst, int64_t n, optigpu_dtype dtype,
                                                 optigpu_stream_t stream)
{
    if (!dtype_valid(int(dtype)))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "scan: unknown dtype");
    if (n < 0 || n > (int64_t(1) << 40))
        return fail(OPTIGPU_ERR_INVALID_ARG, "scan: n out of range [0, 2^40]");
    if (n == 0)
        return OPTIGPU_OK;
    const size_t ies = esize_of(dtype), oes = dtype == OPTIGPU_INT32 ? 8 : 4;
    if (!src || !dst || reinterpret_cast<uintptr_t>(src) % ies || reinterpret_cast<uintptr_t>(dst) % oes)
        return fail(OPTIGPU_ERR_INVALID_ARG, "scan: null or misaligned pointer");
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
    if (a < b + uintptr_t(n) * oes && b < a + uintptr_t(n) * ies)
        return fail(OPTIGPU_ERR_OVERLAP, "scan: src and dst overlap");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    switch (dtype) {
    case OPTIGPU_INT32: return launch_scan<OPTIGPU_INT32>(src, dst, n, s);
    case OPTIGPU_FLOAT32: return launch_scan<OPTIGPU_FLOAT32>(src, dst, n, s);
    case OPTIGPU_BFLOAT16: return launch_scan<OPTIGPU_BFLOAT16>(src, dst, n, s);
    default: return launch_scan<OPTIGPU_FLOAT16>(src, dst, n, s);
    }
}
