// tma_tile.cuh -- the register micro-block transpose shared by the TMA
// transpose kernels (out-of-place in transpose.cu, in place in inplace.cu).
// A thread holds a V x V block of elements (V = 16 / element size) as V
// 16-byte rows and writes its transpose as V 16-byte rows.
#pragma once

#include <cstdint>

#include "ptx.cuh"

namespace optigpu {

__device__ __forceinline__ uint32_t word_of(const uint4 &v, int j)
{
    return j == 0 ? v.x : j == 1 ? v.y : j == 2 ? v.z : v.w;
}

// Writes the transpose of the V x V micro-block held in r[0..V) (row i of
// the block = r[i]) as V 16-byte rows at out, out + pitch, ...
template <int ESIZE>
__device__ __forceinline__ void store_transposed(const uint4 *r, uint32_t out, uint32_t pitch);

template <>
__device__ __forceinline__ void store_transposed<4>(const uint4 *r, uint32_t out, uint32_t pitch)
{
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        uint4 o = make_uint4(word_of(r[0], j), word_of(r[1], j), word_of(r[2], j), word_of(r[3], j));
        ptx::sts_v4(out + j * pitch, o);
    }
}

template <>
__device__ __forceinline__ void store_transposed<2>(const uint4 *r, uint32_t out, uint32_t pitch)
{
    // Output row j = 2w + h holds column j of the 8 input rows; its word k
    // packs rows 2k (low half) and 2k+1 (high half).  Selector 0x5410 takes
    // the low halves of both words, 0x7632 the high halves.
#pragma unroll
    for (int w = 0; w < 4; ++w) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const unsigned sel = h ? 0x7632u : 0x5410u;
            uint4 o;
            o.x = __byte_perm(word_of(r[0], w), word_of(r[1], w), sel);
            o.y = __byte_perm(word_of(r[2], w), word_of(r[3], w), sel);
            o.z = __byte_perm(word_of(r[4], w), word_of(r[5], w), sel);
            o.w = __byte_perm(word_of(r[6], w), word_of(r[7], w), sel);
            ptx::sts_v4(out + (2 * w + h) * pitch, o);
        }
    }
}

// Same, with output row j written at row_addr(j) (any layout, e.g. a
// swizzled one).
template <int ESIZE, typename RowAddr>
__device__ __forceinline__ void store_transposed_at(const uint4 *r, RowAddr row_addr)
{
    if constexpr (ESIZE == 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            ptx::sts_v4(row_addr(j), make_uint4(word_of(r[0], j), word_of(r[1], j), word_of(r[2], j),
                                                word_of(r[3], j)));
    } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const unsigned sel = h ? 0x7632u : 0x5410u;
                uint4 o;
                o.x = __byte_perm(word_of(r[0], w), word_of(r[1], w), sel);
                o.y = __byte_perm(word_of(r[2], w), word_of(r[3], w), sel);
                o.z = __byte_perm(word_of(r[4], w), word_of(r[5], w), sel);
                o.w = __byte_perm(word_of(r[6], w), word_of(r[7], w), sel);
                ptx::sts_v4(row_addr(2 * w + h), o);
            }
        }
    }
}

// Byte offset of 16-byte unit `unit` of row `row` in a tile stored as
// 128-byte-wide boxes (TMA's 128-byte swizzle): rows of `box_rows` 128-byte
// lines per box, boxes side by side in memory, and inside each 1024-byte
// group of 8 lines the unit index XORed with the line index mod 8.
__device__ __forceinline__ uint32_t swz128_offset(uint32_t row, uint32_t unit, uint32_t box_rows)
{
    return (unit >> 3) * box_rows * 128u + row * 128u + (((unit & 7u) ^ (row & 7u)) << 4);
}

template <int ESIZE, int TR, int TC>
struct TmaTile {
    static constexpr int V = 16 / ESIZE;        // elements per 16-byte vector
    static constexpr int MR = TR / V;           // micro-block rows
    static constexpr int MC = TC / V;           // micro-block columns
    static constexpr int THREADS = MR * MC;     // one micro-block per consumer thread
    static constexpr uint32_t BYTES = TR * TC * ESIZE;
    static constexpr uint32_t IN_PITCH = TC * ESIZE;  // source tile row
    static constexpr uint32_t OUT_PITCH = TR * ESIZE; // output tile row
    static_assert(MR % 8 == 0 && MC % 8 == 0, "micro-block grid must be a multiple of 8");
    static_assert(IN_PITCH % 128 == 0 && OUT_PITCH % 128 == 0, "tile rows must span whole bank cycles");
    static_assert(TR <= 256 && TC <= 256, "TMA box dimensions are at most 256");
    static_assert(THREADS % 32 == 0 && THREADS <= 512, "consumer threads");
};

} // namespace optigpu
