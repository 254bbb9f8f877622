// reduce_core.cuh -- the per-chunk partial sum and the final combine of the
// sum reduction, shared by the single-call kernel (reduce.cu) and the batched
// persistent kernel, so that both produce bit-identical partials.
//
// Fixed summation structure (depends only on n, dtype and the mode):
//   chunk c       elements [c * kReduceChunk, min(n, (c + 1) * kReduceChunk))
//   thread t      16-byte vectors t, t + 256, ... of the chunk, in that order
//   vector        its V elements in a pairwise tree ((e0+e1)+(e2+e3))...
//   block         butterfly over the 32 lanes (xor 16, 8, 4, 2, 1), then the
//                 8 warp sums by a butterfly over lanes 0..7 (xor 4, 2, 1)
// Elements past n count as zero.  A chunk read from a source that is not
// 16-byte aligned, or that ends past n, loads the same vectors element by
// element and runs exactly the same arithmetic.
#pragma once

#include <cstdint>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "../../include/optigpu.h"
#include "ptx.cuh"

namespace optigpu {

constexpr int kReduceThreads = 256;
constexpr int64_t kReduceChunk = OPTIGPU_REDUCE_CHUNK;
constexpr size_t kReduceCounterBytes = 256; // counter region ahead of the partials

// Element traits: V elements per 16-byte vector, vector sums, scalar reads.
template <int DT>
struct ElemTraits;

template <>
struct ElemTraits<OPTIGPU_INT32> {
    static constexpr int V = 4;
    using Sum = long long;
    __device__ static Sum vec_sum(uint4 w)
    {
        return (static_cast<long long>(int(w.x)) + int(w.y)) + (static_cast<long long>(int(w.z)) + int(w.w));
    }
    __device__ static uint32_t scalar_bits(const void *p, int64_t i)
    {
        return static_cast<const uint32_t *>(p)[i];
    }
};

template <>
struct ElemTraits<OPTIGPU_FLOAT32> {
    static constexpr int V = 4;
    using Sum = float;
    __device__ static float vec_sum(uint4 w)
    {
        return (__uint_as_float(w.x) + __uint_as_float(w.y)) + (__uint_as_float(w.z) + __uint_as_float(w.w));
    }
    __device__ static uint32_t scalar_bits(const void *p, int64_t i)
    {
        return static_cast<const uint32_t *>(p)[i];
    }
};

// bfloat16 is the upper half of a binary32, so widening is a 16-bit shift.
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

template <>
struct ElemTraits<OPTIGPU_BFLOAT16> {
    static constexpr int V = 8;
    using Sum = float;
    __device__ static float pair(uint32_t w) { return bf16_lo(w) + bf16_hi(w); }
    __device__ static float vec_sum(uint4 w)
    {
        return (pair(w.x) + pair(w.y)) + (pair(w.z) + pair(w.w));
    }
    __device__ static uint32_t scalar_bits(const void *p, int64_t i)
    {
        return static_cast<const uint16_t *>(p)[i];
    }
};

template <>
struct ElemTraits<OPTIGPU_FLOAT16> {
    static constexpr int V = 8;
    using Sum = float;
    __device__ static float pair(uint32_t w)
    {
        return __half2float(__ushort_as_half(static_cast<unsigned short>(w & 0xffffu))) +
               __half2float(__ushort_as_half(static_cast<unsigned short>(w >> 16)));
    }
    __device__ static float vec_sum(uint4 w)
    {
        return (pair(w.x) + pair(w.y)) + (pair(w.z) + pair(w.w));
    }
    __device__ static uint32_t scalar_bits(const void *p, int64_t i)
    {
        return static_cast<const uint16_t *>(p)[i];
    }
};

// Builds a 16-byte vector of a chunk from scalar reads: its elements are
// chunk[first .. first + V), where `chunk` points at the chunk's first
// element and `rem` elements of the chunk lie before n; elements at or past
// rem are zero bits.  32-bit offsets inside the chunk (at most 16384).
template <int DT>
__device__ __forceinline__ uint4 gather_vector(const void *chunk, int rem, int first)
{
    constexpr int V = ElemTraits<DT>::V;
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < V; ++e) {
        const int i = first + e;
        const uint32_t b = i < rem ? ElemTraits<DT>::scalar_bits(chunk, i) : 0u;
        if (V == 4)
            w[e] = b;
        else
            w[e >> 1] |= (e & 1) ? (b << 16) : b;
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

// Knuth's TwoSum: s + e == a + b exactly, for any order of a and b.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// Per-thread accumulator of one mode (trivially constructible so that it
// can live in shared memory; start from zero()).
template <int DT, bool COMP>
struct Acc;

template <int DT>
struct Acc<DT, false> {
    typename ElemTraits<DT>::Sum s;
    __device__ static Acc zero()
    {
        Acc a;
        a.s = 0;
        return a;
    }
    __device__ void add(typename ElemTraits<DT>::Sum v) { s += v; }
    __device__ void merge(const Acc &o) { s += o.s; }
    __device__ Acc shfl_xor(int lane_mask) const
    {
        Acc r;
        r.s = __shfl_xor_sync(0xffffffffu, s, lane_mask);
        return r;
    }
};

// Neumaier's compensated summation (ZAMM 54, 1974): s carries the sum, c the
// low-order parts lost by each addition.
template <int DT>
struct Acc<DT, true> {
    float s, c;
    __device__ static Acc zero()
    {
        Acc a;
        a.s = 0.f;
        a.c = 0.f;
        return a;
    }
    __device__ void add(float v)
    {
        const float t = s + v;
        if (fabsf(s) >= fabsf(v))
            c += (s - t) + v;
        else
            c += (v - t) + s;
        s = t;
    }
    __device__ void merge(const Acc &o)
    {
        float t, e;
        two_sum(s, o.s, t, e);
        s = t;
        c = (c + o.c) + e;
    }
    __device__ Acc shfl_xor(int lane_mask) const
    {
        Acc r;
        r.s = __shfl_xor_sync(0xffffffffu, s, lane_mask);
        r.c = __shfl_xor_sync(0xffffffffu, c, lane_mask);
        return r;
    }
};

// MAX_BATCH bounds the 16-byte loads a thread has in flight (8: the
// throughput form; 4: fewer registers, so more CTAs fit on an SM).  It only
// changes when loads are issued, never the order of the additions, so both
// forms give the same bits.
template <int DT, bool COMP, int MAX_BATCH = 8>
struct ReduceCore {
    using T = ElemTraits<DT>;
    using A = Acc<DT, COMP>;
    static constexpr int V = T::V;
    static constexpr int VPT = int(kReduceChunk / V / kReduceThreads); // vectors per thread
    static constexpr int BATCH = VPT < MAX_BATCH ? VPT : MAX_BATCH;     // loads in flight
    static_assert(VPT % BATCH == 0, "chunk must split into whole load batches");
    static constexpr bool kInt = (DT == OPTIGPU_INT32);
    using Partial = typename std::conditional<kInt, long long, double>::type;

    struct Shared {
        A warp[kReduceThreads / 32];
        Partial fin[kReduceThreads / 32];
    };

    // Block-wide fixed-order combine; the result is valid in thread 0.
    __device__ static A block_combine(A a, Shared &sh)
    {
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1)
            a.merge(a.shfl_xor(m));
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0)
            sh.warp[warp] = a;
        __syncthreads();
        if (warp == 0) {
            A b = lane < kReduceThreads / 32 ? sh.warp[lane] : A::zero();
#pragma unroll
            for (int m = (kReduceThreads / 32) / 2; m >= 1; m >>= 1)
                b.merge(b.shfl_xor(m));
            a = b;
        }
        __syncthreads(); // sh.warp may be reused by the next chunk
        return a;
    }

    __device__ static Partial to_partial(const A &a)
    {
        if constexpr (kInt)
            return a.s;
        else if constexpr (COMP)
            return double(a.s) + double(a.c);
        else
            return double(a.s);
    }

    // Partial sum of chunk c; valid in thread 0.  All threads must call it.
    __device__ static Partial chunk_partial(const void *src, int64_t n, int64_t c, bool vec_ok, Shared &sh)
    {
        const int64_t base = c * kReduceChunk;
        const int t = threadIdx.x;
        A acc = A::zero();
        if (vec_ok && base + kReduceChunk <= n) {
            const uint4 *vsrc = reinterpret_cast<const uint4 *>(
                static_cast<const char *>(src) + base * int64_t(16 / V));
#pragma unroll
            for (int k0 = 0; k0 < VPT; k0 += BATCH) {
                uint4 buf[BATCH];
#pragma unroll
                for (int u = 0; u < BATCH; ++u)
                    buf[u] = __ldcs(vsrc + (k0 + u) * kReduceThreads + t);
#pragma unroll
                for (int u = 0; u < BATCH; ++u)
                    acc.add(T::vec_sum(buf[u]));
            }
        } else {
            // Ragged or unaligned chunk: the same vectors in the same order,
            // gathered from scalar reads.  A batch's reads are all issued
            // before any is added, so they are in flight together; vectors
            // that start at or past n are not added (as in the full path,
            // where none exist).  Offsets are 32-bit and relative to the
            // chunk, so each element costs a compare and a load.
            const char *chunk = static_cast<const char *>(src) + base * int64_t(16 / V);
            const int rem = n - base < kReduceChunk ? int(n - base) : int(kReduceChunk);
#pragma unroll
            for (int k0 = 0; k0 < VPT; k0 += BATCH) {
                uint4 buf[BATCH];
#pragma unroll
                for (int u = 0; u < BATCH; ++u) {
                    const int first = ((k0 + u) * kReduceThreads + t) * V;
                    buf[u] = first < rem ? gather_vector<DT>(chunk, rem, first) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < BATCH; ++u)
                    if (((k0 + u) * kReduceThreads + t) * V < rem)
                        acc.add(T::vec_sum(buf[u]));
            }
        }
        return to_partial(block_combine(acc, sh));
    }

    __device__ static void store_partial(void *partials, int64_t c, Partial v)
    {
        static_cast<Partial *>(partials)[c] = v;
    }

    // Fixed-order combine of partials[0 .. count): thread t sums entries
    // t, t + 256, ... sequentially, then the same shuffle trees.  Thread 0
    // writes the result to *out.  Each thread issues the loads of 4 entries
    // before adding them (in the same order), so a combine of up to 1024
    // partials costs one round trip to L2 instead of one per entry.
    __device__ static void final_combine(const void *partials, int64_t count, void *out, Shared &sh)
    {
        constexpr int U = 4;
        const Partial *p = static_cast<const Partial *>(partials);
        Partial s = 0;
        for (int64_t i0 = threadIdx.x; i0 < count; i0 += int64_t(U) * kReduceThreads) {
            Partial v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t i = i0 + int64_t(u) * kReduceThreads;
                v[u] = i < count ? __ldcg(p + i) : Partial(0);
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + int64_t(u) * kReduceThreads < count)
                    s += v[u];
        }
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1)
            s += __shfl_xor_sync(0xffffffffu, s, m);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        if (lane == 0)
            sh.fin[warp] = s;
        __syncthreads();
        if (warp == 0) {
            Partial b = lane < kReduceThreads / 32 ? sh.fin[lane] : Partial(0);
#pragma unroll
            for (int m = (kReduceThreads / 32) / 2; m >= 1; m >>= 1)
                b += __shfl_xor_sync(0xffffffffu, b, m);
            if (lane == 0)
                *static_cast<Partial *>(out) = b;
        }
        __syncthreads();
    }
};

} // namespace optigpu
