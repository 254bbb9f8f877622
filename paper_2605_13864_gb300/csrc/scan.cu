// scan.cu -- inclusive prefix sums, dst[i] = src[0] + ... + src[i]
// (the thesis names parallel prefix sum as future work, Sec. 9; the running
// sum of Listing 2.1's loop, keeping every intermediate value).
//
// Default: one pass (scan_deferred_kernel below): 4096-element chunks (8192
// for 16-bit input) claimed in order, TMA-staged, each carried by a sum of
// radix-32 blocks of earlier chunk totals whose expression depends on the
// chunk index alone, so results are bit-identical from run to run and no
// chunk waits on another's carry.
// Each carry is fetched one chunk after the scan that publishes its own
// chunk and used one chunk later still; scan_onepass_kernel, configuration
// 2, is the same pass reading each carry at once.
// The three-launch form, kept as configuration 1, runs in a fixed order too:
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
#include <atomic>
#include <cstring>
#include <type_traits>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"
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
    // An infinite or NaN carry passes through hi alone (inf - inf in lo
    // would turn an infinite prefix into NaN).
    return SplitCarry{hi, isfinite(hi) ? float(c - double(hi)) : 0.0f};
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
template <int BAR>
__device__ __forceinline__ void scan_barrier()
{
    if constexpr (BAR == 0)
        __syncthreads();
    else
        ptx::named_bar_sync(BAR, kScanThreads);
}

template <typename T, int BAR = 0>
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
    scan_barrier<BAR>();
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
    scan_barrier<BAR>();
    const T before = warp > 0 ? warp_tot[warp - 1] : T(0);
    *total = warp_tot[kScanThreads / 32 - 1];
    scan_barrier<BAR>(); // warp_tot is reused by the next call
    // The exclusive value is the left neighbour's inclusive one (incl - v
    // would round, and turn an infinite own value into NaN).
    const T left = __shfl_up_sync(0xffffffffu, incl, 1);
    return lane > 0 ? before + left : before;
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

// ----------------------------------------------------- single pass

// Carries of the single pass, fixed by the chunk index alone.  Chunk c
// (4096 elements, 8192 for 16-bit input) publishes its total a_c = B(0, c).  Block (k, m) is the
// aligned run of chunks [m 32^k, (m+1) 32^k); its sum is defined by a fixed
// tree over its 32 children,
//     B(k+1, m) = tree( B(k, 32m), ..., B(k, 32m + 31) )
// (the lane-0 result of a 5-step XOR butterfly).  Writing c in base 32 with
// digits d_k, the exclusive carry of chunk c adds, level by level from the
// top, the complete blocks before c inside its level-(k+1) group:
//     S_k = tree( B(k, 32 (c >> 5(k+1)) + i) for i < d_k, zeros after ),
//     carry(c) = ((S_top + S_top-1) + ...) + S_0.
// Every term and every addition order depend on c alone, so results are
// bit-identical from run to run whatever the timing.  A chunk never waits on
// another chunk's carry, only on complete blocks of earlier totals, so there
// is no serial chain.  Block (k+1, m) is formed by whichever child arrives
// 32nd (a counter per group): one load of the 32 children by a warp, one
// reduction, one publish -- so the blocks a carry needs are at most a level
// or two away from the chunk totals themselves.
constexpr int kRadixLog = 5;
constexpr int kMaxLevels = 7; // 2^40 elements = 2^28 chunks -> 7 levels of radix 32

struct ScanLevels {
    int levels;                     // block levels 0 .. levels-1
    int64_t count[kMaxLevels];      // blocks at level k: ceil(chunks / 32^k)
    uint64_t block_off[kMaxLevels]; // first block slot of level k
    uint64_t group_off[kMaxLevels]; // first group counter of level k (k < levels-1)
};

// A published block sum is two 64-bit words, each holding one 32-bit half
// of the value (low bits) under its bitwise complement (high bits).  Slots
// start zeroed every launch, and (0, 0) fails the check, so a reader that
// sees both words check has the whole value: no fence orders the halves.
// The check also holds for any mix of a word's zeroed and written 32-bit
// halves: (~h, 0) passes only when h == 0 and (0, h) only when
// h == 0xffffffff, and in both cases that is exactly the written word.  So
// copies that promise no single-copy atomicity above 32 bits (the default
// form's bulk copies) still see each word as either written or not yet.
__device__ __forceinline__ void st_relaxed_v2(unsigned long long *p, unsigned long long a, unsigned long long b)
{
    asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1, %2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2(const unsigned long long *p, unsigned long long &a,
                                              unsigned long long &b)
{
    asm volatile("ld.relaxed.gpu.global.v2.u64 {%0, %1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

template <typename C>
__device__ __forceinline__ void publish_block(unsigned long long *slot, C v)
{
    static_assert(sizeof(C) == 8, "64-bit carries");
    unsigned long long bits;
    memcpy(&bits, &v, 8);
    const unsigned long long lo = bits & 0xffffffffull, hi = bits >> 32;
    st_relaxed_v2(slot, ((lo ^ 0xffffffffull) << 32) | lo, ((hi ^ 0xffffffffull) << 32) | hi);
}

// A word is published when its high half is the complement of its low half.
__device__ __forceinline__ bool word_published(unsigned long long w)
{
    return uint32_t(w >> 32) == ~uint32_t(w);
}

// Decodes the two words of a slot; false while either is not yet published.
template <typename C>
__device__ __forceinline__ bool decode_block(unsigned long long a, unsigned long long b, C &v)
{
    if (!word_published(a) || !word_published(b))
        return false;
    const unsigned long long bits = (a & 0xffffffffull) | (b << 32);
    memcpy(&v, &bits, 8);
    return true;
}

template <typename C>
__device__ __forceinline__ bool try_block(const unsigned long long *slot, C &v)
{
    unsigned long long a, b;
    ld_relaxed_v2(slot, a, b);
    return decode_block<C>(a, b, v);
}

// Bounded wait for a block sum; gives up after limit_ns (value 0).
template <typename C>
__device__ bool wait_block(const unsigned long long *slot, C &v, uint64_t limit_ns)
{
    if (try_block(slot, v))
        return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (try_block(slot, v))
            return true;
        if ((spin & 63u) == 0u && ptx::globaltimer_ns() - t0 > limit_ns) {
            v = C(0);
            return false;
        }
    }
}

// Shared-memory image of the 128-byte swizzle that TMA applies (the 16-byte
// chunk index within each 128-byte row is XORed with the row index mod 8;
// buffers are 1024-byte aligned).  Applied to a logical byte offset.
__device__ __forceinline__ uint32_t swz128(uint32_t b) { return b ^ (((b >> 7) & 7u) << 4); }

template <int DT>
struct OnePass {
    using T = ScanTraits<DT>;
    using Out = typename T::Out;
    static constexpr int kInBytes = (DT == OPTIGPU_BFLOAT16 || DT == OPTIGPU_FLOAT16) ? 2 : 4;
    static constexpr int kOutBytes = int(sizeof(Out));
    // Elements per thread and per chunk.  The rate follows the chunks an SM
    // has in flight more than the bytes: every chunk pays the same claim,
    // publication and carry round trips.  16-bit input uses 8192-element
    // chunks (16 KiB in, like fp32's 4096) at two CTAs per SM: 2^28 bf16 ->
    // fp32 in 0.326 ms against 0.406 ms with 4096-element chunks at three
    // (four CTAs per SM at 4096 gained nothing).  fp32 keeps 4096: 6144-
    // element chunks at two CTAs per SM took 0.541 ms against 0.459 ms, and
    // 8192 at two 0.92 ms against 0.56 ms (an earlier kernel).
    static constexpr int kPer = kInBytes == 2 ? 2 * kPerThread : kPerThread;
    static constexpr int kChunk = kScanThreads * kPer; // 4096, or 8192 for 16-bit input
    static constexpr int kWords = kPer * kInBytes / 4;  // raw 32-bit words per thread (16)
    static constexpr int kInStage = kChunk * kInBytes;   // 16 KiB
    static constexpr int kOutStage = kChunk * kOutBytes; // 16 KiB or 32 KiB
    static constexpr int kSmem = 2 * kInStage + kOutStage + 1024;
    static constexpr int kInRow = 128 / kInBytes;  // elements per 128-byte row
    static constexpr int kOutRow = 128 / kOutBytes;
    static constexpr int kMinBlocks = kInBytes == 2 ? 2 : 3; // CTAs per SM the register budget is sized for
    // Deferred-carry form: a three-stage input ring; int32 (8-byte outputs)
    // and 16-bit input (32 KiB out stages) fit two CTAs per SM, fp32 three.
    static constexpr int kSmemDeferred = 3 * kInStage + kOutStage + 1024;
    static constexpr int kMinBlocksDeferred = (kOutBytes == 8 || kInBytes == 2) ? 2 : 3;
};

// Element bits (the low 16 bits for 2-byte types) -> in-chunk accumulator.
template <int DT>
__device__ __forceinline__ typename ScanTraits<DT>::Acc acc_of_bits(uint32_t w)
{
    if constexpr (DT == OPTIGPU_INT32)
        return static_cast<long long>(static_cast<int32_t>(w));
    else if constexpr (DT == OPTIGPU_FLOAT32)
        return __uint_as_float(w);
    else if constexpr (DT == OPTIGPU_BFLOAT16)
        return __uint_as_float(w << 16);
    else
        return __half2float(__ushort_as_half(static_cast<unsigned short>(w & 0xffffu)));
}

// Chunk c staged from plain loads (the ragged last chunk, or a source that
// is not 16-byte aligned) in the swizzled layout a TMA load gives; elements
// past n are zero.
template <int DT>
__device__ __forceinline__ void stage_chunk_plain(unsigned char *in_ptr, const void *src, int64_t n, int64_t base)
{
    using P = OnePass<DT>;
#pragma unroll
    for (int k = 0; k < P::kPer; ++k) {
        const int e = int(threadIdx.x) + k * kScanThreads;
        const int64_t i = base + e;
        const uint32_t off = swz128(uint32_t(e * P::kInBytes));
        if constexpr (P::kInBytes == 4)
            *reinterpret_cast<uint32_t *>(in_ptr + off) = i < n ? static_cast<const uint32_t *>(src)[i] : 0u;
        else
            *reinterpret_cast<uint16_t *>(in_ptr + off) =
                i < n ? static_cast<const uint16_t *>(src)[i] : uint16_t(0);
    }
}

// Thread t's raw words: elements kPer t .. kPer t + kPer - 1 of the staged
// chunk.
template <int DT>
__device__ __forceinline__ void load_raw(uint32_t in_addr, uint32_t (&raw)[OnePass<DT>::kWords])
{
    using P = OnePass<DT>;
    const uint32_t region = uint32_t(threadIdx.x) * P::kPer * P::kInBytes;
#pragma unroll
    for (int q = 0; q < P::kWords / 4; ++q) {
        const uint4 w = ptx::lds_v4(in_addr + swz128(region + 16u * q));
        raw[4 * q] = w.x;
        raw[4 * q + 1] = w.y;
        raw[4 * q + 2] = w.z;
        raw[4 * q + 3] = w.w;
    }
}

// Sequential sum of the thread's elements, in element order.
template <int DT>
__device__ __forceinline__ typename ScanTraits<DT>::Acc thread_run(const uint32_t (&raw)[OnePass<DT>::kWords])
{
    using Acc = typename ScanTraits<DT>::Acc;
    Acc run = Acc(0);
#pragma unroll
    for (int w = 0; w < OnePass<DT>::kWords; ++w) {
        if constexpr (OnePass<DT>::kInBytes == 4) {
            run += acc_of_bits<DT>(raw[w]);
        } else {
            run += acc_of_bits<DT>(raw[w] & 0xffffu);
            run += acc_of_bits<DT>(raw[w] >> 16);
        }
    }
    return run;
}

// Publishes B(0, c) = total, then forms every block chunk c completes as the
// 32nd arrival of its group.  Called by one whole warp; false in a lane whose
// wait for a child gave up.
template <typename Carry>
__device__ __forceinline__ bool publish_and_form(unsigned long long *blocks, unsigned *groups, const ScanLevels &L,
                                                 int64_t c, Carry total, uint64_t wait_limit_ns)
{
    const int lane = int(threadIdx.x) & 31;
    bool ok = true;
    if (lane == 0)
        publish_block<Carry>(blocks + 2 * (L.block_off[0] + uint64_t(c)), total);
    int64_t j = c;
    for (int k = 0; k + 1 < L.levels; ++k) {
        const int64_t parent = j >> kRadixLog;
        if (((parent + 1) << kRadixLog) > L.count[k])
            break; // an incomplete group is never needed
        unsigned last = 0;
        if (lane == 0)
            last = atomicAdd(groups + L.group_off[k] + uint64_t(parent), 1u) == 31u;
        if (!__shfl_sync(0xffffffffu, last, 0))
            break; // later arrivals form it
        Carry x;
        if (!wait_block<Carry>(blocks + 2 * (L.block_off[k] + uint64_t((parent << kRadixLog) + lane)), x,
                               wait_limit_ns))
            ok = false;
#pragma unroll
        for (int d = 16; d; d >>= 1)
            x += __shfl_xor_sync(0xffffffffu, x, d);
        if (lane == 0)
            publish_block<Carry>(blocks + 2 * (L.block_off[k + 1] + uint64_t(parent)), x);
        j = parent;
    }
    return ok;
}

// The outputs of one chunk into the swizzled out stage: the thread's
// sequential run again (the same operations, so the same bits), plus its
// block prefix, plus the carry.
template <int DT>
__device__ __forceinline__ void finish_chunk(const uint32_t (&raw)[OnePass<DT>::kWords],
                                             typename ScanTraits<DT>::Acc before, typename ScanTraits<DT>::Split sc,
                                             uint32_t out_addr)
{
    using P = OnePass<DT>;
    using T = ScanTraits<DT>;
    using Acc = typename T::Acc;
    Acc v[P::kPer];
#pragma unroll
    for (int w = 0; w < P::kWords; ++w) {
        if constexpr (P::kInBytes == 4) {
            v[w] = acc_of_bits<DT>(raw[w]);
        } else {
            v[2 * w] = acc_of_bits<DT>(raw[w] & 0xffffu);
            v[2 * w + 1] = acc_of_bits<DT>(raw[w] >> 16);
        }
    }
#pragma unroll
    for (int j = 1; j < P::kPer; ++j)
        v[j] += v[j - 1];
    const uint32_t oregion = uint32_t(threadIdx.x) * P::kPer * P::kOutBytes;
    if constexpr (P::kOutBytes == 4) {
#pragma unroll
        for (int q = 0; q < P::kPer / 4; ++q) {
            uint4 w;
            w.x = __float_as_uint(T::finish(sc, before + v[4 * q]));
            w.y = __float_as_uint(T::finish(sc, before + v[4 * q + 1]));
            w.z = __float_as_uint(T::finish(sc, before + v[4 * q + 2]));
            w.w = __float_as_uint(T::finish(sc, before + v[4 * q + 3]));
            ptx::sts_v4(out_addr + swz128(oregion + 16u * q), w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < P::kPer / 2; ++q) {
            const unsigned long long a = static_cast<unsigned long long>(T::finish(sc, before + v[2 * q]));
            const unsigned long long b2 = static_cast<unsigned long long>(T::finish(sc, before + v[2 * q + 1]));
            ptx::sts_v4(out_addr + swz128(oregion + 16u * q),
                        make_uint4(uint32_t(a), uint32_t(a >> 32), uint32_t(b2), uint32_t(b2 >> 32)));
        }
    }
}

// A finished chunk from the out stage to dst with plain coalesced stores (the
// ragged last chunk, or a destination that is not 16-byte aligned).
template <int DT>
__device__ __forceinline__ void store_chunk_plain(void *dst, int64_t n, int64_t chunk, const unsigned char *out_stage)
{
    using P = OnePass<DT>;
    using Out = typename ScanTraits<DT>::Out;
    Out *out = static_cast<Out *>(dst);
    const int64_t pbase = chunk * P::kChunk;
#pragma unroll
    for (int k = 0; k < P::kPer; ++k) {
        const int e = int(threadIdx.x) + k * kScanThreads;
        if (pbase + e < n)
            out[pbase + e] = *reinterpret_cast<const Out *>(out_stage + swz128(uint32_t(e * P::kOutBytes)));
    }
}

// Single-pass scan.  A persistent grid claims chunks in order through an
// integer ticket, and every CTA runs a three-stage software pipeline so that
// no chunk total ever waits for a carry:
//   iteration k:  thread 0 starts the TMA load of chunk k+1 (128-byte
//                 swizzle) into the other half of a two-stage buffer and
//                 claims chunk k+2; the CTA scans chunk k; then, side by
//                 side, warp 1 publishes the total of chunk k and forms every
//                 block it completes, while warp 0 gathers the carry of
//                 chunk k-1; finally chunk k-1 (kept in registers) gets its
//                 carry and leaves through a swizzled stage and one TMA store.
// Totals are published as soon as they exist, so no chain forms: a carry is
// read about one iteration after the totals it needs were published.  The
// ragged last chunk, or pointers that are not 16-byte aligned, use the same
// stages with plain coalesced loads and stores.
template <int DT>
__global__ void __launch_bounds__(kScanThreads, OnePass<DT>::kMinBlocks)
scan_onepass_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_map,
                    const void *__restrict__ src, void *__restrict__ dst, int64_t n, int64_t num_chunks,
                    int64_t full_chunks, int in_tma, int out_tma, unsigned long long *ticket, unsigned *groups,
                    unsigned long long *blocks, const __grid_constant__ ScanLevels L, uint64_t wait_limit_ns,
                    unsigned *err)
{
    using P = OnePass<DT>;
    using T = ScanTraits<DT>;
    using Acc = typename T::Acc;
    using Carry = typename T::Carry;
    constexpr int kWords = P::kWords;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[2];
    __shared__ Acc warp_tot[kScanThreads / 32];
    __shared__ int64_t s_chunk[3];
    __shared__ Carry s_excl;

    const uint32_t raw_addr = ptx::smem_addr(smem_raw);
    const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
    unsigned char *stage = smem_raw + pad;
    const uint32_t stage_addr = raw_addr + pad; // in[0] | in[1] | out
    const uint32_t out_addr = stage_addr + 2 * P::kInStage;
    unsigned char *out_stage = stage + 2 * P::kInStage;
    const uint32_t bar0 = ptx::smem_addr(&full_bar[0]);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    bool failed = false;

    if (t == 0) {
        if (in_tma) {
            ptx::mbar_init(bar0, 1);
            ptx::mbar_init(bar0 + 8, 1);
            ptx::fence_mbar_init();
            ptx::prefetch_tensormap(&in_map);
        }
        if (out_tma)
            ptx::prefetch_tensormap(&out_map);
        const int64_t c0 = int64_t(atomicAdd(ticket, 1ull));
        s_chunk[0] = c0;
        if (in_tma && c0 < full_chunks) {
            ptx::mbar_arrive_expect_tx(bar0, P::kInStage);
            ptx::tma_load_3d(stage_addr, &in_map, 0, 0, int32_t(c0), bar0);
        }
        s_chunk[1] = c0 < num_chunks ? int64_t(atomicAdd(ticket, 1ull)) : num_chunks;
    }
    __syncthreads();

    uint32_t raw_prev[kWords];
    Acc before_prev = Acc(0);
    int64_t prev = -1;  // chunk whose carry is pending (uniform)
    uint32_t phase = 0; // bit b: parity of the next completion of stage b
    for (int it = 0;; ++it) {
        const int buf = it & 1;
        const int64_t c = s_chunk[it % 3];
        const bool has_cur = c < num_chunks;
        if (!has_cur && prev < 0)
            break;
        const int64_t base = c * P::kChunk;
        const uint32_t in_addr = stage_addr + uint32_t(buf) * P::kInStage;
        unsigned long long claim = 0;
        uint32_t raw[kWords];
        Acc before = Acc(0);
        if (has_cur) {
            if (in_tma && c < full_chunks) {
                const bool ok = ptx::mbar_wait_bounded(bar0 + 8u * uint32_t(buf), (phase >> buf) & 1u, wait_limit_ns);
                phase ^= 1u << buf;
                if (__syncthreads_or(!ok)) {
                    // The copy did not arrive in time: give it one more
                    // bounded wait, report, and stop.
                    if (t == 0) {
                        ptx::mbar_wait_bounded(bar0 + 8u * uint32_t(buf), ((phase >> buf) & 1u) ^ 1u, wait_limit_ns);
                        atomicOr(err, DEV_ERR_WAIT_TIMEOUT);
                    }
                    break;
                }
            } else {
                stage_chunk_plain<DT>(stage + buf * P::kInStage, src, n, base);
                __syncthreads();
            }
            if (t == 0) {
                // Load the chunk claimed last iteration into the other stage
                // (its previous contents went to registers one iteration
                // ago) and claim the one after it; the claim is stored only
                // after the scan, so its round trip overlaps the scan.
                const int64_t cn = s_chunk[(it + 1) % 3];
                if (in_tma && cn < full_chunks) {
                    const uint32_t nb = bar0 + 8u * uint32_t(buf ^ 1);
                    ptx::mbar_arrive_expect_tx(nb, P::kInStage);
                    ptx::tma_load_3d(stage_addr + uint32_t(buf ^ 1) * P::kInStage, &in_map, 0, 0, int32_t(cn), nb);
                }
                claim = cn < num_chunks ? atomicAdd(ticket, 1ull) : (unsigned long long)num_chunks;
            }
            load_raw<DT>(in_addr, raw);
            const Acc run = thread_run<DT>(raw);
            Acc total;
            before = block_exclusive_scan<Acc>(run, warp_tot, &total);
            // Warp 1 publishes the total of chunk c and forms the blocks it
            // completes, beside warp 0's carry below.
            if (warp == 1 && !publish_and_form<Carry>(blocks, groups, L, c, Carry(total), wait_limit_ns))
                failed = true;
        }

        const bool pending = prev >= 0;
        if (warp == 0) {
            // Carry of the pending chunk: start every block load, then wait,
            // reduce each level, add from the top level down.
            Carry excl = Carry(0);
            if (prev > 0) {
                Carry xk[kMaxLevels];
                unsigned ready = 0;
#pragma unroll
                for (int k = 0; k < kMaxLevels; ++k) {
                    xk[k] = Carry(0);
                    if (k < L.levels && lane < int((prev >> (kRadixLog * k)) & 31) &&
                        try_block<Carry>(blocks + 2 * (L.block_off[k] +
                                                       uint64_t(((prev >> (kRadixLog * (k + 1))) << kRadixLog) + lane)),
                                         xk[k]))
                        ready |= 1u << k;
                }
                bool first = true;
#pragma unroll
                for (int k = kMaxLevels - 1; k >= 0; --k) {
                    if (k >= L.levels)
                        continue;
                    const int d = int((prev >> (kRadixLog * k)) & 31);
                    if (d == 0)
                        continue; // uniform across the warp
                    if (lane < d && !((ready >> k) & 1u) &&
                        !wait_block<Carry>(blocks + 2 * (L.block_off[k] +
                                                         uint64_t(((prev >> (kRadixLog * (k + 1))) << kRadixLog) + lane)),
                                           xk[k], wait_limit_ns))
                        failed = true;
                    Carry x = lane < d ? xk[k] : Carry(0);
#pragma unroll
                    for (int dd = 16; dd; dd >>= 1)
                        x += __shfl_xor_sync(0xffffffffu, x, dd);
                    x = __shfl_sync(0xffffffffu, x, 0);
                    excl = first ? x : excl + x;
                    first = false;
                }
            }
            if (t == 0) {
                s_excl = excl;
                if (has_cur)
                    s_chunk[(it + 2) % 3] = int64_t(claim);
                if (out_tma)
                    ptx::bulk_wait_group_read<0>(); // the previous store has left the out stage
            }
        }
        __syncthreads();

        if (pending) {
            // Outputs of the pending chunk: its sequential run again (the
            // same operations, so the same bits), plus the thread's block
            // prefix, plus the carry.
            finish_chunk<DT>(raw_prev, before_prev, T::split(s_excl), out_addr);
            const bool store_tma = out_tma && prev < full_chunks;
            if (store_tma)
                ptx::fence_proxy_async_smem();
            __syncthreads();
            if (store_tma) {
                if (t == 0) {
                    ptx::tma_store_3d(&out_map, 0, 0, int32_t(prev), out_addr);
                    ptx::bulk_commit_group();
                }
            } else {
                store_chunk_plain<DT>(dst, n, prev, out_stage);
            }
        }
        if (!has_cur)
            break;
#pragma unroll
        for (int w = 0; w < kWords; ++w)
            raw_prev[w] = raw[w];
        before_prev = before;
        prev = c;
    }
    if (t == 0 && out_tma)
        ptx::bulk_wait_group<0>();
    if (failed)
        atomicOr(err, DEV_ERR_WAIT_TIMEOUT);
}

// The same single pass with every carry used one iteration later.  Warp w
// (w < levels) fetches level w of the carry of chunk k-1 right after the scan
// of chunk k -- when the form above reads it -- with one bulk copy into
// shared memory, and reduces it after the scan of chunk k+1.  The round trip
// overlaps a whole iteration, and no CTA barrier waits for it: a bulk copy
// completes on an mbarrier of its own.  Chunk k-1 stays in the third stage
// of a three-stage input ring and is reloaded into registers at the end of
// iteration k, so it is finished from its raw words by the same operations
// as in the form above, giving the same bits.  Warp 7 publishes totals and
// forms blocks.
//   iteration k:  wait for chunk k in in[k % 3]; thread 0 loads chunk k+1
//                 into in[(k+1) % 3] (its previous chunk, k-2, went to
//                 registers one iteration ago) and claims chunk k+2; scan
//                 chunk k; warp 7 publishes it; warps 0..levels-1 reduce the
//                 carry levels of chunk k-2 and start the copies for chunk
//                 k-1; chunk k-2 gets its carry and leaves through the
//                 swizzled out stage and one TMA store; chunk k-1 is reloaded
//                 from in[(k-1) % 3].
template <int DT>
__global__ void __launch_bounds__(kScanThreads, OnePass<DT>::kMinBlocksDeferred)
scan_deferred_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_map,
                     const void *__restrict__ src, void *__restrict__ dst, int64_t n, int64_t num_chunks,
                     int64_t full_chunks, int in_tma, int out_tma, unsigned long long *ticket, unsigned *groups,
                     unsigned long long *blocks, const __grid_constant__ ScanLevels L, uint64_t wait_limit_ns,
                     unsigned *err)
{
    using P = OnePass<DT>;
    using T = ScanTraits<DT>;
    using Acc = typename T::Acc;
    using Carry = typename T::Carry;
    constexpr int kWords = P::kWords;
    constexpr int kPubWarp = kScanThreads / 32 - 1;
    static_assert(kMaxLevels <= kPubWarp, "one warp per carry level, one to publish");
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[3];
    __shared__ __align__(8) uint64_t slot_bar[kMaxLevels];
    __shared__ __align__(16) unsigned long long s_slot[kMaxLevels][64]; // 32 slots of two words per level
    __shared__ Acc warp_tot[kScanThreads / 32];
    __shared__ int64_t s_chunk[3];
    __shared__ Carry s_level[kMaxLevels];

    const uint32_t raw_addr = ptx::smem_addr(smem_raw);
    const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
    unsigned char *stage = smem_raw + pad;
    const uint32_t stage_addr = raw_addr + pad; // in[0] | in[1] | in[2] | out
    const uint32_t out_addr = stage_addr + 3 * P::kInStage;
    const unsigned char *out_stage = stage + 3 * P::kInStage;
    const uint32_t bar0 = ptx::smem_addr(&full_bar[0]);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const uint32_t my_slot_bar = ptx::smem_addr(&slot_bar[warp < kMaxLevels ? warp : 0]);
    bool failed = false;

    if (t == 0) {
        for (int s = 0; s < 3; ++s)
            ptx::mbar_init(bar0 + 8u * s, 1);
        for (int k = 0; k < kMaxLevels; ++k)
            ptx::mbar_init(ptx::smem_addr(&slot_bar[k]), 1);
        ptx::fence_mbar_init();
        if (in_tma)
            ptx::prefetch_tensormap(&in_map);
        if (out_tma)
            ptx::prefetch_tensormap(&out_map);
        const int64_t c0 = int64_t(atomicAdd(ticket, 1ull));
        s_chunk[0] = c0;
        if (in_tma && c0 < full_chunks) {
            ptx::mbar_arrive_expect_tx(bar0, P::kInStage);
            ptx::tma_load_3d(stage_addr, &in_map, 0, 0, int32_t(c0), bar0);
        }
        s_chunk[1] = c0 < num_chunks ? int64_t(atomicAdd(ticket, 1ull)) : num_chunks;
    }
    __syncthreads();

    uint32_t raw_prev2[kWords]; // raw words of chunk prev2 (reloaded one iteration ago)
    Acc before_p1 = Acc(0), before_p2 = Acc(0);
    int64_t prev1 = -1, prev2 = -1; // chunks scanned one and two iterations ago (uniform)
    bool drained = false;
    bool slot_pending = false; // this warp's slot copy is in flight
    uint32_t phase = 0;        // bit s: parity of the next completion of in[s]
    uint32_t slot_phase = 0;   // parity of the next completion of this warp's slot copy
    for (int it = 0;; ++it) {
        const int sidx = it % 3;
        const int64_t c = drained ? num_chunks : s_chunk[sidx];
        const bool has_cur = c < num_chunks;
        drained = !has_cur;
        if (!has_cur && prev1 < 0 && prev2 < 0)
            break;
        const int64_t base = c * P::kChunk;
        const uint32_t in_addr = stage_addr + uint32_t(sidx) * P::kInStage;
        unsigned long long claim = 0;
        Acc before = Acc(0);
        if (has_cur) {
            if (in_tma && c < full_chunks) {
                const uint32_t fb = bar0 + 8u * uint32_t(sidx);
                const bool ok = ptx::mbar_wait_bounded(fb, (phase >> sidx) & 1u, wait_limit_ns);
                phase ^= 1u << sidx;
                if (__syncthreads_or(!ok)) {
                    // The copy did not arrive in time: give it one more
                    // bounded wait, report, and stop.
                    if (t == 0) {
                        ptx::mbar_wait_bounded(fb, ((phase >> sidx) & 1u) ^ 1u, wait_limit_ns);
                        atomicOr(err, DEV_ERR_WAIT_TIMEOUT);
                    }
                    break;
                }
            } else {
                stage_chunk_plain<DT>(stage + sidx * P::kInStage, src, n, base);
                __syncthreads();
            }
            if (t == 0) {
                // Load the chunk claimed last iteration into the next stage
                // of the ring and claim the one after it; the claim is
                // stored only after the scan, so its round trip overlaps it.
                const int nidx = (it + 1) % 3;
                const int64_t cn = s_chunk[nidx];
                if (in_tma && cn < full_chunks) {
                    const uint32_t nb = bar0 + 8u * uint32_t(nidx);
                    ptx::mbar_arrive_expect_tx(nb, P::kInStage);
                    ptx::tma_load_3d(stage_addr + uint32_t(nidx) * P::kInStage, &in_map, 0, 0, int32_t(cn), nb);
                }
                claim = cn < num_chunks ? atomicAdd(ticket, 1ull) : (unsigned long long)num_chunks;
            }
            // Thread t scans elements 16 t .. 16 t + 15 of the chunk.
            uint32_t raw[kWords];
            load_raw<DT>(in_addr, raw);
            const Acc run = thread_run<DT>(raw);
            Acc total;
            before = block_exclusive_scan<Acc>(run, warp_tot, &total);
            if (warp == kPubWarp && !publish_and_form<Carry>(blocks, groups, L, c, Carry(total), wait_limit_ns))
                failed = true;
        }

        if (warp < L.levels) {
            // Level `warp` of the carry of chunk prev2 (its slots were copied
            // one iteration ago), then the copy for chunk prev1.
            const int lvl = warp;
            if (prev2 > 0) {
                const int d = int((prev2 >> (kRadixLog * lvl)) & 31);
                Carry x = Carry(0);
                if (d > 0) { // uniform across the warp
                    if (!ptx::mbar_wait_bounded(my_slot_bar, slot_phase, wait_limit_ns))
                        failed = true;
                    slot_phase ^= 1u;
                    slot_pending = false;
                    if (lane < d && !decode_block<Carry>(s_slot[lvl][2 * lane], s_slot[lvl][2 * lane + 1], x) &&
                        !wait_block<Carry>(blocks + 2 * (L.block_off[lvl] +
                                                         uint64_t(((prev2 >> (kRadixLog * (lvl + 1))) << kRadixLog) +
                                                                  lane)),
                                           x, wait_limit_ns))
                        failed = true; // copied before it was published: read it again
                    if (lane >= d)
                        x = Carry(0);
#pragma unroll
                    for (int dd = 16; dd; dd >>= 1)
                        x += __shfl_xor_sync(0xffffffffu, x, dd);
                }
                if (lane == 0)
                    s_level[lvl] = x;
            }
            if (prev1 > 0) {
                const int d = int((prev1 >> (kRadixLog * lvl)) & 31);
                if (d > 0) { // uniform across the warp
                    __syncwarp(); // every lane has read its slot of the last copy
                    if (lane == 0) {
                        ptx::fence_proxy_async_smem();
                        ptx::mbar_arrive_expect_tx(my_slot_bar, 16u * uint32_t(d));
                        ptx::bulk_load(ptx::smem_addr(&s_slot[lvl][0]),
                                       blocks + 2 * (L.block_off[lvl] +
                                                     uint64_t((prev1 >> (kRadixLog * (lvl + 1))) << kRadixLog)),
                                       16u * uint32_t(d), my_slot_bar);
                    }
                    slot_pending = true;
                }
            }
        }
        if (t == 0) {
            if (has_cur)
                s_chunk[(it + 2) % 3] = int64_t(claim);
            if (out_tma)
                ptx::bulk_wait_group_read<0>(); // the previous store has left the out stage
        }
        __syncthreads();

        if (prev2 >= 0 || prev1 >= 0) { // uniform
            if (prev2 >= 0) {
                // Chunk prev2: its sequential run again (the same operations,
                // so the same bits), plus the thread's block prefix, plus the
                // carry added from the top level down.
                Carry excl = Carry(0);
                if (prev2 > 0) {
                    bool first = true;
                    for (int k = L.levels - 1; k >= 0; --k) {
                        if (((prev2 >> (kRadixLog * k)) & 31) == 0)
                            continue;
                        excl = first ? s_level[k] : excl + s_level[k];
                        first = false;
                    }
                }
                finish_chunk<DT>(raw_prev2, before_p2, T::split(excl), out_addr);
            }
            if (prev1 >= 0) {
                // Chunk prev1 to registers: its stage takes chunk it+2 next
                // iteration.
                load_raw<DT>(stage_addr + uint32_t((it + 2) % 3) * P::kInStage, raw_prev2);
            }
            const bool store_tma = prev2 >= 0 && out_tma && prev2 < full_chunks;
            if (store_tma)
                ptx::fence_proxy_async_smem();
            __syncthreads();
            if (prev2 >= 0) {
                if (store_tma) {
                    if (t == 0) {
                        ptx::tma_store_3d(&out_map, 0, 0, int32_t(prev2), out_addr);
                        ptx::bulk_commit_group();
                    }
                } else {
                    store_chunk_plain<DT>(dst, n, prev2, out_stage);
                }
            }
        }
        before_p2 = before_p1;
        before_p1 = before;
        prev2 = prev1;
        prev1 = has_cur ? c : -1;
    }
    if (slot_pending && !ptx::mbar_wait_bounded(my_slot_bar, slot_phase, wait_limit_ns))
        failed = true; // no copy is left in flight into this CTA's shared memory
    if (t == 0 && out_tma)
        ptx::bulk_wait_group<0>();
    if (failed)
        atomicOr(err, DEV_ERR_WAIT_TIMEOUT);
}

// ----------------------------------------------------- windowed single pass

// Carries fixed by the slice index through 32 interleaved running sums.
// Slice s (kSubs sub-chunks of 4096 elements) publishes its total T_s.  For
// each lane l < 32 let
//     A_l(s) = sum of T_j over j < s with j = l (mod 32), added left to right,
// and let the exclusive carry of slice s be the lane-0 result of a 5-step
// XOR butterfly over A_0(s) .. A_31(s).  Every CTA extends the 32 running
// sums itself (lane l adds the new T_j of its residue class in increasing j)
// from the published totals, so no CTA waits on another's carry, only on
// totals; and every term and addition order is fixed by s alone (not by the
// grid or the timing), so results are bit-identical from run to run.  Sums
// are int64 for int32 input and FP32 hi + lo pairs (TwoSum) for float input.
// Inside a slice, sub-chunk q adds the totals of sub-chunks 0 .. q-1 (left
// to right) to the carry.
constexpr int kWinWarps = kScanThreads / 32;
constexpr int kWinMaxCtas = kWinWarps * 32; // 256 CTAs at most
constexpr int kCarryWarps = 2;               // carry warps, taking alternate slices of their CTA
constexpr int kWinSlotCap = kCarryWarps * kWinMaxCtas; // totals one copy may bring in

// Float carries of the windowed form are FP32 pairs hi + lo (about 44
// significant bits), added with Knuth's TwoSum and a final fast two-sum:
// FP64 runs at a small fraction of the FP32 rate on this part, and the
// carry path is serial.  A non-finite sum passes through hi alone (lo = 0),
// so infinities and NaN propagate as in a plain running sum.
struct F2 {
    float hi, lo;
    F2() = default;
    __device__ explicit F2(float h, float l = 0.0f) : hi(h), lo(l) {}
};

__device__ __forceinline__ F2 f2_add(F2 a, F2 b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = ((a.hi - (s - bb)) + (b.hi - bb)) + (a.lo + b.lo);
    const float h = s + e;
    const float l = e - (h - s);
    // Selects, not branches: the carry warps keep several sums in flight.
    const float hi = isfinite(s) ? h : s;
    return F2(hi, isfinite(hi) ? l : 0.0f);
}
__device__ __forceinline__ long long win_add(long long a, long long b) { return a + b; }
__device__ __forceinline__ F2 win_add(F2 a, F2 b) { return f2_add(a, b); }
__device__ __forceinline__ long long win_shfl_xor(long long x, int d) { return __shfl_xor_sync(0xffffffffu, x, d); }
__device__ __forceinline__ F2 win_shfl_xor(F2 x, int d)
{
    return F2(__shfl_xor_sync(0xffffffffu, x.hi, d), __shfl_xor_sync(0xffffffffu, x.lo, d));
}
__device__ __forceinline__ long long win_of(long long v) { return v; }
__device__ __forceinline__ F2 win_of(float v) { return F2(v); }
__device__ __forceinline__ long long win_split(long long c) { return c; }
__device__ __forceinline__ SplitCarry win_split(F2 c) { return SplitCarry{c.hi, c.lo}; }

template <int DT>
struct WinPass {
    using T = ScanTraits<DT>;
    using Out = typename T::Out;
    static constexpr int kInBytes = (DT == OPTIGPU_BFLOAT16 || DT == OPTIGPU_FLOAT16) ? 2 : 4;
    static constexpr int kOutBytes = int(sizeof(Out));
    static constexpr int kPer = kPerThread;                 // 16 consecutive elements per thread
    static constexpr int kSubN = kScanThreads * kPer;       // 4096 elements per sub-chunk
    static constexpr int kWords = kPer * kInBytes / 4;      // raw 32-bit words per thread (16 or 8)
    static constexpr int kInSub = kSubN * kInBytes;         // 16 or 8 KiB
    static constexpr int kOutSub = kSubN * kOutBytes;       // 16 or 32 KiB
    // Sub-chunks per slice: 32 KiB of fp32 in, 24 KiB of 16-bit input (48
    // KiB out), 16 KiB of int32 (32 KiB of int64 out).
    static constexpr int kSubs = kOutBytes == 8 ? 1 : (kInBytes == 2 ? 3 : 2);
    static constexpr int kSlice = kSubs * kSubN;
    static constexpr int kInStage = kSubs * kInSub, kOutStage = kSubs * kOutSub;
    // Input stages: slice j being scanned, j-1 .. j-3 waiting for or taking
    // their carries, j+1 and j+2 loading.
    static constexpr int kRing = 6;
    // fp32 is finished in place in its input stage (the same layout in and
    // out); wider outputs take an out stage.
    static constexpr bool kInPlace = kInBytes == kOutBytes;
    static constexpr int kSmem = kRing * kInStage + (kInPlace ? 0 : kOutStage) + 1024;
    static constexpr int kInRow = 128 / kInBytes, kOutRow = 128 / kOutBytes;
    // Slice totals, running sums and carries: int64 for int32 input, FP32
    // pairs for float input.
    using Carry = typename std::conditional<DT == OPTIGPU_INT32, long long, F2>::type;
};

// Every sub-chunk of a slice is scanned by its own group of kScanThreads
// threads (eight warps); `tid` is the thread's index inside its group.

// Sub-chunk staged from plain loads (the ragged last slice, or a source that
// is not 16-byte aligned) in the swizzled layout of a TMA load; elements past
// n are zero.
template <int DT>
__device__ __forceinline__ void win_stage_plain(unsigned char *sub_ptr, const void *src, int64_t n, int64_t base,
                                                int tid)
{
    using P = WinPass<DT>;
#pragma unroll 4
    for (int k = 0; k < P::kPer; ++k) {
        const int e = tid + k * kScanThreads;
        const int64_t i = base + e;
        const uint32_t off = swz128(uint32_t(e * P::kInBytes));
        if constexpr (P::kInBytes == 4)
            *reinterpret_cast<uint32_t *>(sub_ptr + off) = i < n ? static_cast<const uint32_t *>(src)[i] : 0u;
        else
            *reinterpret_cast<uint16_t *>(sub_ptr + off) = i < n ? static_cast<const uint16_t *>(src)[i] : uint16_t(0);
    }
}

template <int DT>
__device__ __forceinline__ void win_load_raw(uint32_t sub_addr, uint32_t (&raw)[WinPass<DT>::kWords], int tid)
{
    using P = WinPass<DT>;
    const uint32_t region = uint32_t(tid) * P::kPer * P::kInBytes;
#pragma unroll
    for (int q = 0; q < P::kWords / 4; ++q) {
        const uint4 w = ptx::lds_v4(sub_addr + swz128(region + 16u * q));
        raw[4 * q] = w.x;
        raw[4 * q + 1] = w.y;
        raw[4 * q + 2] = w.z;
        raw[4 * q + 3] = w.w;
    }
}

template <int DT>
__device__ __forceinline__ void win_unpack(const uint32_t (&raw)[WinPass<DT>::kWords],
                                           typename ScanTraits<DT>::Acc (&v)[WinPass<DT>::kPer])
{
#pragma unroll
    for (int w = 0; w < WinPass<DT>::kWords; ++w) {
        if constexpr (WinPass<DT>::kInBytes == 4) {
            v[w] = acc_of_bits<DT>(raw[w]);
        } else {
            v[2 * w] = acc_of_bits<DT>(raw[w] & 0xffffu);
            v[2 * w + 1] = acc_of_bits<DT>(raw[w] >> 16);
        }
    }
}

// Exclusive scan of one value per thread over a group of kScanThreads (the
// same fixed order as block_exclusive_scan: Kogge-Stone inside each warp,
// then warp 0 of the group scans the 8 warp totals), with two syncs of the
// group's named barrier `bar`.  warp_tot must not be reused before a later
// barrier of the group.
template <typename T>
__device__ __forceinline__ T group_exclusive_scan(T v, T *warp_tot, uint32_t bar, int tid, T *total)
{
    const int lane = tid & 31, warp = tid >> 5;
    T incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T up = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d)
            incl += up;
    }
    if (lane == 31)
        warp_tot[warp] = incl;
    ptx::named_bar_sync(bar, kScanThreads);
    if (warp == 0) {
        T w = lane < kWinWarps ? warp_tot[lane] : T(0);
#pragma unroll
        for (int d = 1; d < kWinWarps; d <<= 1) {
            const T up = __shfl_up_sync(0xffffffffu, w, d);
            if (lane >= d)
                w += up;
        }
        if (lane < kWinWarps)
            warp_tot[lane] = w; // inclusive prefix of the warp totals
    }
    ptx::named_bar_sync(bar, kScanThreads);
    const T bw = warp > 0 ? warp_tot[warp - 1] : T(0);
    *total = warp_tot[kWinWarps - 1];
    // The left neighbour's inclusive value (incl - v would round, and turn an
    // infinite own value into NaN).
    const T left = __shfl_up_sync(0xffffffffu, incl, 1);
    return lane > 0 ? bw + left : bw;
}

// The outputs of a sub-chunk into its swizzled out buffer: the thread's run
// again, plus its group prefix, plus the carry.
template <int DT>
__device__ __forceinline__ void win_finish(const uint32_t (&raw)[WinPass<DT>::kWords],
                                           typename ScanTraits<DT>::Acc before, typename ScanTraits<DT>::Split sc,
                                           uint32_t out_addr, int tid)
{
    using P = WinPass<DT>;
    using T = ScanTraits<DT>;
    typename T::Acc v[P::kPer];
    win_unpack<DT>(raw, v);
#pragma unroll
    for (int j = 1; j < P::kPer; ++j)
        v[j] += v[j - 1];
    const uint32_t oregion = uint32_t(tid) * P::kPer * P::kOutBytes;
    if constexpr (P::kOutBytes == 4) {
        // hi + ((lo + before) + v): the carry's low part and the thread's
        // group prefix are added once, then each output costs two additions.
        const float lb = sc.lo + before;
#pragma unroll
        for (int q = 0; q < P::kPer / 4; ++q) {
            uint4 w;
            w.x = __float_as_uint(sc.hi + (lb + v[4 * q]));
            w.y = __float_as_uint(sc.hi + (lb + v[4 * q + 1]));
            w.z = __float_as_uint(sc.hi + (lb + v[4 * q + 2]));
            w.w = __float_as_uint(sc.hi + (lb + v[4 * q + 3]));
            ptx::sts_v4(out_addr + swz128(oregion + 16u * q), w);
        }
    } else {
#pragma unroll
        for (int q = 0; q < P::kPer / 2; ++q) {
            const unsigned long long a = static_cast<unsigned long long>(T::finish(sc, before + v[2 * q]));
            const unsigned long long b2 = static_cast<unsigned long long>(T::finish(sc, before + v[2 * q + 1]));
            ptx::sts_v4(out_addr + swz128(oregion + 16u * q),
                        make_uint4(uint32_t(a), uint32_t(a >> 32), uint32_t(b2), uint32_t(b2 >> 32)));
        }
    }
}

template <int DT>
__device__ __forceinline__ void win_store_plain(void *dst, int64_t n, int64_t base, const unsigned char *out_sub,
                                                int tid)
{
    using P = WinPass<DT>;
    using Out = typename ScanTraits<DT>::Out;
    Out *out = static_cast<Out *>(dst);
#pragma unroll 4
    for (int k = 0; k < P::kPer; ++k) {
        const int e = tid + k * kScanThreads;
        const int64_t i = base + e;
        if (i < n)
            out[i] = *reinterpret_cast<const Out *>(out_sub + swz128(uint32_t(e * P::kOutBytes)));
    }
}

// Bounded spin until a shared counter reaches `target`; false on timeout or
// when the CTA aborts.
__device__ __forceinline__ bool win_wait_count(const unsigned long long *counter, unsigned long long target,
                                               const volatile int *abort, uint64_t limit_ns)
{
    const volatile unsigned long long *c = counter;
    if (*c >= target)
        return true;
    const uint64_t t0 = ptx::globaltimer_ns();
    for (uint32_t spin = 1;; ++spin) {
        if (*c >= target)
            return true;
        if (*abort)
            return false;
        if ((spin & 63u) == 0u && ptx::globaltimer_ns() - t0 > limit_ns)
            return false;
    }
}

// Windowed single pass.  One CTA per SM (a cooperative launch, so every CTA
// is resident while others wait for its totals); CTA b takes slices
// b, b + G, b + 2G, ... in order.  Group g (eight warps) owns sub-chunk g of
// every slice and runs its own software pipeline over a six-stage ring:
//   iteration j:  load sub-chunk g of slice j+2 into the buffer that of
//                 slice j-4 left; wait for slice j; scan it and hand its total
//                 to the slice (the last group to arrive adds the S totals and
//                 publishes the slice total); finish slice j-3 with the
//                 carry a carry warp prepared, and store it (TMA).
// Two carry warps, taking alternate slices, build the carry of each slice k
// once this CTA has published slice k+1 (by then the totals of the slices
// before k are usually published too): one bulk copy of the totals since the
// warp's previous slice, the 32 running sums and their butterfly, and every
// sub-chunk's carry as an FP32 hi + lo pair (int64 for int32 input), handed
// over through shared memory.  Slot words are read with the same complement
// check as the radix form: a slot copied before it was published is read
// again (bounded).  fp32 is finished in place in its input buffer; wider
// outputs go through an out stage.
template <int DT>
__global__ void __launch_bounds__(WinPass<DT>::kSubs * kScanThreads + 32 * kCarryWarps, 1)
scan_window_kernel(const __grid_constant__ CUtensorMap in_map, const __grid_constant__ CUtensorMap out_map,
                   const void *__restrict__ src, void *__restrict__ dst, int64_t n, int64_t num_slices,
                   int64_t full_slices, int in_tma, int out_tma, unsigned long long *totals,
                   uint64_t wait_limit_ns, unsigned *err)
{
    using P = WinPass<DT>;
    using T = ScanTraits<DT>;
    using Acc = typename T::Acc;
    using Carry = typename P::Carry;
    using Split = typename T::Split;
    constexpr int S = P::kSubs, R = P::kRing, kW = P::kWords;
    constexpr int kSplitRing = 4;
    constexpr bool kInPlace = P::kInPlace;
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[R][S];
    __shared__ __align__(8) uint64_t slot_bar[kCarryWarps];
    __shared__ __align__(16) unsigned long long s_slot[kCarryWarps][2 * kWinSlotCap];
    __shared__ Acc warp_tot[2][S][kWinWarps];
    __shared__ Acc s_tot[R][S];              // sub-chunk totals of slice j, at j % R
    __shared__ unsigned s_arrive[R];         // groups done with slice j, at j % R
    __shared__ Split s_split[kSplitRing][S]; // carry of each sub-chunk of slice k, at k % 4
    __shared__ unsigned long long s_published; // slices of this CTA published
    __shared__ unsigned long long s_ready[kCarryWarps]; // carry warp c: its slices up to s_ready[c] - 1 are in s_split
    __shared__ volatile int s_abort;

    const uint32_t raw_addr = ptx::smem_addr(smem_raw);
    const uint32_t pad = ((raw_addr + 1023u) & ~1023u) - raw_addr;
    unsigned char *stage = smem_raw + pad;
    const uint32_t stage_addr = raw_addr + pad; // in[0..R) | out (unless in place)
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = warp / kWinWarps, tid = t - g * kScanThreads; // group, thread in group
    const int64_t G = gridDim.x, b = blockIdx.x;
    const int64_t K = b < num_slices ? (num_slices - 1 - b) / G + 1 : 0; // slices of this CTA
    auto tma_slice = [&](int64_t k) { return in_tma && b + k * G < full_slices; };

    if (t == 0) {
        for (int r = 0; r < R; ++r) {
            for (int q = 0; q < S; ++q)
                ptx::mbar_init(ptx::smem_addr(&full_bar[r][q]), 1);
            s_arrive[r] = 0;
        }
        for (int c = 0; c < kCarryWarps; ++c) {
            ptx::mbar_init(ptx::smem_addr(&slot_bar[c]), 1);
            s_ready[c] = 0;
        }
        ptx::fence_mbar_init();
        s_published = 0;
        s_abort = 0;
    }
    __syncthreads();
    bool failed = false;

    if (g == S) {
        // ------------------------------------------------ a carry warp
        // Carry warp c takes this CTA's slices k = c (mod kCarryWarps), so
        // two slices' carries are built at once.
        const int c = warp - S * kWinWarps;
        const uint32_t sbar = ptx::smem_addr(&slot_bar[c]);
        unsigned long long *slots = s_slot[c];
        Carry acc = Carry(0); // A_lane(next): the running sum of this lane's residue class
        int64_t next = 0;     // totals [0, next) are in acc
        uint32_t slot_phase = 0;
        for (int64_t k = c; k < K; k += kCarryWarps) {
            const int64_t s = b + k * G;
            // Wait until this CTA has published slice k+1 (its own totals
            // up to there; the other CTAs' earlier slices are mostly out).
            if (!win_wait_count(&s_published, (unsigned long long)(k + 2 < K ? k + 2 : K), &s_abort,
                                wait_limit_ns)) {
                failed = !s_abort;
                s_abort = 1;
                break;
            }
            __threadfence_block();
            const int cnt = int(s - next); // the totals since this warp's last slice: at most kWinSlotCap
            if (cnt > 0) {
                if (lane == 0) {
                    ptx::fence_proxy_async_smem();
                    ptx::mbar_arrive_expect_tx(sbar, 16u * uint32_t(cnt));
                    ptx::bulk_load(ptx::smem_addr(slots), totals + 2 * uint64_t(next), 16u * uint32_t(cnt), sbar);
                }
                if (!ptx::mbar_wait_bounded(sbar, slot_phase, wait_limit_ns)) {
                    failed = true; // the copy is still owed: give it one more bounded wait
                    ptx::mbar_wait_bounded(sbar, slot_phase, wait_limit_ns);
                    s_abort = 1;
                    break;
                }
                slot_phase ^= 1u;
                // Lane l adds T_j for the j = l (mod 32) in [next, s), in
                // increasing j.
                for (int o = int((uint32_t(lane) - uint32_t(next)) & 31u); o < cnt; o += 32) {
                    Carry x;
                    if (!decode_block<Carry>(slots[2 * o], slots[2 * o + 1], x) &&
                        !wait_block<Carry>(totals + 2 * (uint64_t(next) + uint64_t(o)), x, wait_limit_ns))
                        failed = true; // copied before it was published: read it again
                    acc = win_add(acc, x);
                }
            }
            next = s;
            __syncwarp(); // every lane has read s_slot before the next copy
            Carry e = acc;
#pragma unroll
            for (int d = 16; d; d >>= 1)
                e = win_add(e, win_shfl_xor(e, d));
            if (lane == 0) {
                // Sub-chunk q adds the totals of sub-chunks 0 .. q-1, left
                // to right.
                const int r = int(k % R), e4 = int(k % kSplitRing);
                Carry cq = e;
#pragma unroll
                for (int q = 0; q < S; ++q) {
                    if (q > 0)
                        cq = win_add(cq, win_of(s_tot[r][q - 1]));
                    s_split[e4][q] = win_split(cq);
                }
                __threadfence_block();
                atomicMax(&s_ready[c], (unsigned long long)(k + 1));
            }
        }
    } else {
        // ------------------------------------------- compute group g
        const uint32_t gbar = 1u + uint32_t(g); // the group's named barrier
        const bool leader = tid == 0;
        auto in_sub = [&](int r) { return uint32_t(r * P::kInStage + g * P::kInSub); };
        auto issue_load = [&](int64_t k) { // leader
            const int r = int(k % R);
            const uint32_t fb = ptx::smem_addr(&full_bar[r][g]);
            ptx::mbar_arrive_expect_tx(fb, uint32_t(P::kInSub));
            ptx::tma_load_3d(stage_addr + in_sub(r), &in_map, 0, 0, int32_t((b + k * G) * S + g), fb);
        };
        if (leader) {
            if (in_tma)
                ptx::prefetch_tensormap(&in_map);
            if (out_tma)
                ptx::prefetch_tensormap(&out_map);
            for (int64_t k = 0; k < 2 && k < K; ++k)
                if (tma_slice(k))
                    issue_load(k);
        }
        Acc before_p1 = Acc(0), before_p2 = Acc(0), before_p3 = Acc(0);
        uint32_t phase = 0;   // bit r: parity of the next completion of this group's buffer of in[r]
        uint32_t pending = 0; // bit r: a load into it is in flight
        for (int r = 0; r < 2 && r < K; ++r)
            if (tma_slice(r))
                pending |= 1u << r;
        for (int64_t j = 0; j < K + 3; ++j) {
            if (leader) {
                // The store issued last iteration has left shared memory, so
                // the buffer of slice j-4 (and the out buffer) may be refilled.
                if (out_tma)
                    ptx::bulk_wait_group_read<0>();
                if (j + 2 < K && tma_slice(j + 2)) {
                    ptx::fence_proxy_async_smem();
                    issue_load(j + 2);
                }
            }
            if (j + 2 < K && tma_slice(j + 2))
                pending |= 1u << int((j + 2) % R);
            Acc before_c = Acc(0);
            if (j < K) {
                // ---- slice j: wait, scan, hand over the total
                const int r = int(j % R);
                const int64_t s = b + j * G;
                if (tma_slice(j)) {
                    const bool ok = ptx::mbar_wait_bounded(ptx::smem_addr(&full_bar[r][g]), (phase >> r) & 1u,
                                                           wait_limit_ns);
                    if (ptx::named_bar_or(gbar, kScanThreads, !ok)) {
                        failed = true; // the buffer stays pending: drained below
                        break;
                    }
                    phase ^= 1u << r;
                    pending &= ~(1u << r);
                } else {
                    win_stage_plain<DT>(stage + in_sub(r), src, n, s * P::kSlice + int64_t(g) * P::kSubN, tid);
                    ptx::named_bar_sync(gbar, kScanThreads);
                }
                uint32_t raw[kW];
                win_load_raw<DT>(stage_addr + in_sub(r), raw, tid);
                Acc v[P::kPer];
                win_unpack<DT>(raw, v);
                Acc run = Acc(0);
#pragma unroll
                for (int e = 0; e < P::kPer; ++e)
                    run += v[e];
                Acc tot;
                before_c = group_exclusive_scan<Acc>(run, warp_tot[j & 1][g], gbar, tid, &tot);
                if (leader) {
                    s_tot[r][g] = tot;
                    __threadfence_block();
                    if (atomicAdd(&s_arrive[r], 1u) == unsigned(S - 1)) {
                        // The last group of the slice publishes its total.
                        __threadfence_block();
                        s_arrive[r] = 0;
                        Carry ts = win_of(s_tot[r][0]);
#pragma unroll
                        for (int q = 1; q < S; ++q)
                            ts = win_add(ts, win_of(s_tot[r][q]));
                        publish_block<Carry>(totals + 2 * uint64_t(s), ts);
                        __threadfence_block();
                        atomicMax(&s_published, (unsigned long long)(j + 1));
                    }
                }
            }

            // ---- finish slice j-3 and store it
            if (j >= 3) {
                const int64_t k3 = j - 3;
                const int r3 = int(k3 % R);
                const int64_t s3 = b + k3 * G;
                if (leader && !win_wait_count(&s_ready[k3 % kCarryWarps], (unsigned long long)(k3 + 1), &s_abort,
                                              wait_limit_ns))
                    failed = true;
                if (ptx::named_bar_or(gbar, kScanThreads, failed)) {
                    failed = true;
                    break;
                }
                __threadfence_block();
                const uint32_t in3 = stage_addr + in_sub(r3);
                const uint32_t out3 = kInPlace ? in3 : stage_addr + uint32_t(R * P::kInStage + g * P::kOutSub);
                uint32_t raw[kW];
                win_load_raw<DT>(in3, raw, tid);
                win_finish<DT>(raw, before_p3, s_split[k3 % kSplitRing][g], out3, tid);
                const bool store_tma = out_tma && s3 < full_slices;
                if (store_tma)
                    ptx::fence_proxy_async_smem();
                ptx::named_bar_sync(gbar, kScanThreads);
                if (store_tma) {
                    if (leader) {
                        ptx::tma_store_3d(&out_map, 0, 0, int32_t(s3 * S + g), out3);
                        ptx::bulk_commit_group();
                    }
                } else {
                    win_store_plain<DT>(dst, n, s3 * P::kSlice + int64_t(g) * P::kSubN,
                                        stage + (out3 - stage_addr), tid);
                    ptx::named_bar_sync(gbar, kScanThreads); // read before it is refilled
                }
            }
            before_p3 = before_p2;
            before_p2 = before_p1;
            before_p1 = before_c;
        }
        if (failed && leader)
            s_abort = 1;
        if (leader) {
            // Nothing may still write this CTA's shared memory when it exits.
            for (int r = 0; r < R; ++r)
                if ((pending >> r) & 1u)
                    ptx::mbar_wait_bounded(ptx::smem_addr(&full_bar[r][g]), (phase >> r) & 1u, wait_limit_ns);
            if (out_tma)
                ptx::bulk_wait_group<0>();
        }
    }
    if (failed)
        atomicOr(err, DEV_ERR_WAIT_TIMEOUT);
}

// 0: single pass, carries used one chunk later (scan_deferred_kernel);
// 1: three passes; 2: single pass, carries read at once (scan_onepass_kernel);
// 3: windowed single pass (scan_window_kernel).
// Kept per input class: [0] int32 input, [1] float input.  The defaults are
// the fastest measured on 2^28 elements: the radix single pass for int32 ->
// int64 (its 32 KiB of output per 4096 elements leave the windowed form one
// group per slice) and the windowed pass for float input.
std::atomic<int> g_scan_choice[2] = {0, 3};
int scan_class(int dtype) { return dtype == OPTIGPU_INT32 ? 0 : 1; }

template <int DT>
optigpu_status launch_scan_onepass(const void *src, void *dst, int64_t n, int form, cudaStream_t stream)
{
    using P = OnePass<DT>;
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const int64_t chunks = (n + P::kChunk - 1) / P::kChunk, full_chunks = n / P::kChunk;
    ScanLevels L{};
    L.levels = 1;
    L.count[0] = chunks;
    while (L.count[L.levels - 1] > 1) {
        if (L.levels == kMaxLevels)
            return fail(OPTIGPU_ERR_INVALID_ARG, "scan: too many chunks for the carry tree");
        L.count[L.levels] = (L.count[L.levels - 1] + 31) >> kRadixLog;
        ++L.levels;
    }
    uint64_t slots = 0, ngroups = 0;
    for (int k = 0; k < L.levels; ++k) {
        L.block_off[k] = slots;
        slots += uint64_t(L.count[k]);
        L.group_off[k] = ngroups;
        if (k + 1 < L.levels)
            ngroups += uint64_t(L.count[k + 1]);
    }
    // [ticket 256 B][group counters][block slots, 16 B each]; all zeroed.
    const size_t off_groups = 256, off_blocks = (off_groups + 4 * ngroups + 255) / 256 * 256;
    const size_t bytes = off_blocks + 16 * slots;
    void *ws = nullptr;
    if ((st = stream_workspace(stream, bytes, &ws, 3)) != OPTIGPU_OK)
        return st;
    char *b = static_cast<char *>(ws);
    if ((st = check_cuda(cudaMemsetAsync(b, 0, bytes, stream), "scan: reset ticket and carries")) != OPTIGPU_OK)
        return st;

    CUtensorMap in_map{}, out_map{};
    const int in_tma = full_chunks > 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0;
    const int out_tma = full_chunks > 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0;
    if (in_tma &&
        (st = encode_tensor_map_3d_swizzled(&in_map, const_cast<void *>(src),
                                            P::kInBytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                             : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                                            P::kInRow, P::kChunk / P::kInRow, uint64_t(full_chunks), 128,
                                            uint64_t(P::kInStage), P::kInRow, P::kChunk / P::kInRow,
                                            CU_TENSOR_MAP_SWIZZLE_128B)) != OPTIGPU_OK)
        return st;
    if (out_tma &&
        (st = encode_tensor_map_3d_swizzled(&out_map, dst,
                                            P::kOutBytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                              : CU_TENSOR_MAP_DATA_TYPE_UINT64,
                                            P::kOutRow, P::kChunk / P::kOutRow, uint64_t(full_chunks), 128,
                                            uint64_t(P::kOutStage), P::kOutRow, P::kChunk / P::kOutRow,
                                            CU_TENSOR_MAP_SWIZZLE_128B)) != OPTIGPU_OK)
        return st;

    const bool deferred = form == 0;
    const void *fn = deferred ? reinterpret_cast<const void *>(&scan_deferred_kernel<DT>)
                              : reinterpret_cast<const void *>(&scan_onepass_kernel<DT>);
    const int smem = deferred ? P::kSmemDeferred : P::kSmem;
    static std::atomic<bool> attr_set[2][64];
    if (dev.device < 0 || dev.device >= 64 || !attr_set[deferred][dev.device].load()) {
        if ((st = check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, smem),
                             "cudaFuncSetAttribute(scan)")) != OPTIGPU_OK)
            return st;
        if (dev.device >= 0 && dev.device < 64)
            attr_set[deferred][dev.device].store(true);
    }
    int per_sm = 0;
    if ((st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kScanThreads, smem),
                         "cudaOccupancyMaxActiveBlocksPerMultiprocessor(scan)")) != OPTIGPU_OK)
        return st;
    const int64_t grid = std::min<int64_t>(chunks, int64_t(std::max(per_sm, 1)) * dev.num_sms);
    unsigned long long *ticket = reinterpret_cast<unsigned long long *>(b);
    unsigned *groups = reinterpret_cast<unsigned *>(b + off_groups);
    unsigned long long *blocks = reinterpret_cast<unsigned long long *>(b + off_blocks);
    if (deferred)
        scan_deferred_kernel<DT><<<unsigned(grid), kScanThreads, smem, stream>>>(
            in_map, out_map, src, dst, n, chunks, full_chunks, in_tma, out_tma, ticket, groups, blocks, L,
            wait_limit_ns(), dev.status_word);
    else
        scan_onepass_kernel<DT><<<unsigned(grid), kScanThreads, smem, stream>>>(
            in_map, out_map, src, dst, n, chunks, full_chunks, in_tma, out_tma, ticket, groups, blocks, L,
            wait_limit_ns(), dev.status_word);
    return check_cuda(cudaGetLastError(), "launch scan (single pass)");
}

template <int DT>
optigpu_status launch_scan_window(const void *src, void *dst, int64_t n, cudaStream_t stream)
{
    using P = WinPass<DT>;
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const int64_t slices = (n + P::kSlice - 1) / P::kSlice, full_slices = n / P::kSlice;
    const int64_t full_chunks = full_slices * P::kSubs;
    if (full_chunks > int64_t(INT32_MAX))
        return fail(OPTIGPU_ERR_INVALID_ARG, "scan: too many chunks for the windowed form");
    // [slice totals, 16 B each], zeroed.
    const size_t bytes = size_t(16) * size_t(slices) + 256;
    void *ws = nullptr;
    if ((st = stream_workspace(stream, bytes, &ws, 3)) != OPTIGPU_OK)
        return st;
    if ((st = check_cuda(cudaMemsetAsync(ws, 0, bytes, stream), "scan: reset slice totals")) != OPTIGPU_OK)
        return st;

    CUtensorMap in_map{}, out_map{};
    const int in_tma = full_chunks > 0 && reinterpret_cast<uintptr_t>(src) % 16 == 0;
    const int out_tma = full_chunks > 0 && reinterpret_cast<uintptr_t>(dst) % 16 == 0;
    if (in_tma &&
        (st = encode_tensor_map_3d_swizzled(&in_map, const_cast<void *>(src),
                                            P::kInBytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                             : CU_TENSOR_MAP_DATA_TYPE_UINT16,
                                            P::kInRow, P::kSubN / P::kInRow, uint64_t(full_chunks), 128,
                                            uint64_t(P::kInSub), P::kInRow, P::kSubN / P::kInRow,
                                            CU_TENSOR_MAP_SWIZZLE_128B)) != OPTIGPU_OK)
        return st;
    if (out_tma &&
        (st = encode_tensor_map_3d_swizzled(&out_map, dst,
                                            P::kOutBytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                                              : CU_TENSOR_MAP_DATA_TYPE_UINT64,
                                            P::kOutRow, P::kSubN / P::kOutRow, uint64_t(full_chunks), 128,
                                            uint64_t(P::kOutSub), P::kOutRow, P::kSubN / P::kOutRow,
                                            CU_TENSOR_MAP_SWIZZLE_128B)) != OPTIGPU_OK)
        return st;

    const void *fn = reinterpret_cast<const void *>(&scan_window_kernel<DT>);
    static std::atomic<bool> attr_set[64];
    if (dev.device < 0 || dev.device >= 64 || !attr_set[dev.device].load()) {
        if ((st = check_cuda(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, P::kSmem),
                             "cudaFuncSetAttribute(scan window)")) != OPTIGPU_OK)
            return st;
        if (dev.device >= 0 && dev.device < 64)
            attr_set[dev.device].store(true);
    }
    // CTAs wait for the totals of other CTAs' slices, so all of them must be
    // resident at once: one per SM, launched cooperatively.
    const int64_t grid = std::min<int64_t>({slices, int64_t(dev.num_sms), int64_t(kWinMaxCtas)});
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(P::kSubs * kScanThreads + 32 * kCarryWarps); // a group of eight warps per sub-chunk, the carry warps
    cfg.dynamicSmemBytes = size_t(P::kSmem);
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    unsigned long long *totals = static_cast<unsigned long long *>(ws);
    return check_cuda(cudaLaunchKernelEx(&cfg, scan_window_kernel<DT>, in_map, out_map, src, dst, n, slices,
                                         full_slices, in_tma, out_tma, totals, wait_limit_ns(), dev.status_word),
                      "launch scan (windowed single pass)");
}

template <int DT>
optigpu_status launch_scan(const void *src, void *dst, int64_t n, cudaStream_t stream)
{
    const int choice = g_scan_choice[scan_class(DT)].load();
    if (choice == 3)
        return launch_scan_window<DT>(src, dst, n, stream);
    if (choice != 1)
        return launch_scan_onepass<DT>(src, dst, n, choice, stream);
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

int scan_num_configs() { return 4; }
const char *scan_config_name(int c)
{
    return c == 0   ? "scan single pass (carries used one chunk later)"
           : c == 1 ? "scan three passes"
           : c == 2 ? "scan single pass (carries read at once)"
           : c == 3 ? "scan single pass (windowed carries, one CTA per SM)"
                    : nullptr;
}
int scan_selected(int dtype) { return g_scan_choice[scan_class(dtype)].load(); }
void scan_select(int dtype, int c) { g_scan_choice[scan_class(dtype)].store(c); }

} // namespace optigpu

using namespace optigpu;

extern "C" optigpu_status optigpu_scan_inclusive(const void *src, void *dst, int64_t n, optigpu_dtype dtype,
                                                 optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_scan_inclusive");
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
