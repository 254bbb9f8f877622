// transpose.cu -- out-of-place matrix transpose, dst (cols x rows) = src^T
// (thesis arxiv 2605.13864, Listing 3.5, Sec. 3.1: out[x][y] = in[y][x]).
//
// Two kernels:
//
//  * tile32: one 32x32 shared-memory tile per CTA, rows padded so that a
//    column read touches 32 distinct banks, 32x8 threads moving 4 elements
//    each, one barrier between the coalesced row reads and the coalesced row
//    writes.  It is the classic bank-conflict-free form of the kernel the
//    thesis derives (Listings 3.6, 3.10, 6.21; Sec. 7.1 measures against the
//    padded form) and the library's any-shape, any-alignment path.  Tiles are
//    numbered on a 1-D grid and decoded with one division per CTA, instead of
//    the per-thread div/mod chains that cost the generated kernel ~40 GB/s
//    (Sec. 7.2).
//
//  * tma: a persistent kernel (grid = CTAs-per-SM x SMs).  One thread issues
//    2-D TMA tile loads of TR x TC source tiles into a STAGES-deep shared
//    memory ring; completion is tracked by one mbarrier per stage.  Every
//    thread owns one 16-byte x V micro-block of the tile (V = 16 / element
//    size: 4x4 words or 8x8 halves), reads it with V 16-byte shared loads,
//    transposes it in registers (renaming for 4-byte elements, byte permutes
//    for 2-byte ones) and writes V 16-byte rows of the transposed tile into
//    one of two output staging buffers, which a 2-D TMA store writes back.
//    TMA fills out-of-range source elements with zeros and clips the store
//    at the matrix edge, so ragged edges need no predication.  Micro-blocks
//    are assigned so that each group of 8 threads (one shared-memory
//    wavefront of 16-byte accesses) touches 8 distinct 16-byte bank groups on
//    both the read and the write side, which makes the tile conflict-free
//    without a swizzle.
#include <algorithm>
#include <mutex>

#include "internal.h"
#include "ptx.cuh"

namespace optigpu {
namespace {

// ------------------------------------------------------------------ tile32

template <typename T>
__global__ void __launch_bounds__(256)
transpose_tile32_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t rows,
                        int64_t cols, int64_t tiles_c)
{
    // 4-byte rows are padded by one element, 2-byte rows by two, so that a
    // column of the tile spans 32 distinct 4-byte banks.
    constexpr int PAD = sizeof(T) == 4 ? 1 : 2;
    __shared__ T tile[32][32 + PAD];
    const int64_t id = blockIdx.x;
    const int64_t tr = id / tiles_c;
    const int64_t tc = id - tr * tiles_c;
    const int64_t r0 = tr * 32, c0 = tc * 32;
    const int x = threadIdx.x, y = threadIdx.y;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t r = r0 + y + j, c = c0 + x;
        if (r < rows && c < cols)
            tile[y + j][x] = src[r * cols + c];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t orow = c0 + y + j, ocol = r0 + x;
        if (orow < cols && ocol < rows)
            dst[orow * rows + ocol] = tile[x][y + j];
    }
}

// --------------------------------------------------------------------- tma

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

template <int ESIZE, int TR, int TC>
struct TmaTile {
    static constexpr int V = 16 / ESIZE;        // elements per 16-byte vector
    static constexpr int MR = TR / V;           // micro-block rows
    static constexpr int MC = TC / V;           // micro-block columns
    static constexpr int THREADS = MR * MC;     // one micro-block per thread
    static constexpr uint32_t BYTES = TR * TC * ESIZE;
    static constexpr uint32_t IN_PITCH = TC * ESIZE;  // source tile row
    static constexpr uint32_t OUT_PITCH = TR * ESIZE; // output tile row
    static_assert(MR % 8 == 0 && MC % 8 == 0, "micro-block grid must be a multiple of 8");
    static_assert(IN_PITCH % 128 == 0 && OUT_PITCH % 128 == 0, "tile rows must span whole bank cycles");
    static_assert(TR <= 256 && TC <= 256, "TMA box dimensions are at most 256");
};

template <int ESIZE, int TR, int TC, int STAGES>
__global__ void __launch_bounds__(TmaTile<ESIZE, TR, TC>::THREADS)
transpose_tma_kernel(const __grid_constant__ CUtensorMap tm_src,
                     const __grid_constant__ CUtensorMap tm_dst, int32_t tiles_c,
                     int64_t num_tiles, uint64_t wait_limit_ns, unsigned *status)
{
    using Tile = TmaTile<ESIZE, TR, TC>;
    constexpr int V = Tile::V;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t in_base = ptx::smem_addr(smem);
    const uint32_t out_base = in_base + STAGES * Tile::BYTES;
    const uint32_t bar_base = out_base + 2 * Tile::BYTES;

    // Micro-block of this thread.  With q = t % 8 and p = t / 8, the 8
    // threads of a wavefront share p and get rb % 8 = q and
    // cb % 8 = (q + p) % 8: distinct 16-byte bank groups on both sides.
    const int t = threadIdx.x;
    const int q = t & 7, p = t >> 3;
    const int rest = p >> 3;
    const int rb = (rest % (Tile::MR / 8)) * 8 + q;
    const int cb = (rest / (Tile::MR / 8)) * 8 + ((q + (p & 7)) & 7);
    const uint32_t rd_off = uint32_t(rb * V) * Tile::IN_PITCH + uint32_t(cb) * 16u;
    const uint32_t wr_off = uint32_t(cb * V) * Tile::OUT_PITCH + uint32_t(rb) * 16u;

    const int64_t first = blockIdx.x, stride = gridDim.x;
    const int64_t my_count = first < num_tiles ? (num_tiles - 1 - first) / stride + 1 : 0;

    if (t == 0) {
        ptx::prefetch_tensormap(&tm_src);
        ptx::prefetch_tensormap(&tm_dst);
        for (int s = 0; s < STAGES; ++s)
            ptx::mbar_init(bar_base + 8u * s, 1);
        ptx::fence_mbar_init();
    }
    __syncthreads();

    auto issue_load = [&](int64_t k) {
        const int64_t tile = first + k * stride;
        const int32_t tr = int32_t(tile / tiles_c);
        const int32_t tc = int32_t(tile - int64_t(tr) * tiles_c);
        const uint32_t s = uint32_t(k % STAGES);
        ptx::mbar_arrive_expect_tx(bar_base + 8u * s, Tile::BYTES);
        ptx::tma_load_2d(in_base + s * Tile::BYTES, &tm_src, tc * TC, tr * TR, bar_base + 8u * s);
    };

    if (t == 0)
        for (int64_t k = 0; k < STAGES && k < my_count; ++k)
            issue_load(k);

    for (int64_t k = 0; k < my_count; ++k) {
        const uint32_t s = uint32_t(k % STAGES);
        const uint32_t parity = uint32_t(k / STAGES) & 1u;
        const bool ok = ptx::mbar_wait_bounded(bar_base + 8u * s, parity, wait_limit_ns);
        uint4 r[V];
        if (ok) {
#pragma unroll
            for (int i = 0; i < V; ++i)
                r[i] = ptx::lds_v4(in_base + s * Tile::BYTES + rd_off + uint32_t(i) * Tile::IN_PITCH);
        }
        // All threads agree on whether to stop.  This barrier also (a) frees
        // stage s for the next load and (b) publishes thread 0's wait for the
        // store that last used the output buffer written below.
        if (__syncthreads_or(!ok)) {
            if (t == 0) {
                atomicOr(status, DEV_ERR_WAIT_TIMEOUT);
                // Let the loads already issued land (bounded) before exiting.
                for (int64_t kk = k; kk < k + STAGES && kk < my_count; ++kk)
                    ptx::mbar_wait_bounded(bar_base + 8u * uint32_t(kk % STAGES),
                                           uint32_t(kk / STAGES) & 1u, wait_limit_ns);
                ptx::bulk_wait_group<0>();
            }
            return;
        }
        if (t == 0 && k + STAGES < my_count)
            issue_load(k + STAGES);

        const uint32_t obuf = out_base + uint32_t(k & 1) * Tile::BYTES;
        store_transposed<ESIZE>(r, obuf + wr_off, Tile::OUT_PITCH);
        ptx::fence_proxy_async_smem();
        __syncthreads();
        if (t == 0) {
            const int64_t tile = first + k * stride;
            const int32_t tr = int32_t(tile / tiles_c);
            const int32_t tc = int32_t(tile - int64_t(tr) * tiles_c);
            ptx::tma_store_2d(&tm_dst, tr * TR, tc * TC, obuf);
            ptx::bulk_commit_group();
            // The buffer used next iteration was read by the store before
            // this one; wait until at most this store is still reading.
            ptx::bulk_wait_group_read<1>();
        }
    }
    if (t == 0)
        ptx::bulk_wait_group<0>();
}

// ------------------------------------------------------------------- host

struct TmaConfig {
    int esize;
    int tr, tc, stages, threads;
    uint32_t tile_bytes;
    const void *fn;
};

template <int ESIZE, int TR, int TC, int STAGES>
TmaConfig make_config()
{
    using Tile = TmaTile<ESIZE, TR, TC>;
    return TmaConfig{ESIZE, TR, TC, STAGES, Tile::THREADS, Tile::BYTES,
                     reinterpret_cast<const void *>(&transpose_tma_kernel<ESIZE, TR, TC, STAGES>)};
}

const TmaConfig &tma_config(size_t esize)
{
    static const TmaConfig c4 = make_config<4, 64, 64, 4>();
    static const TmaConfig c2 = make_config<2, 64, 128, 4>();
    return esize == 4 ? c4 : c2;
}

size_t tma_smem_bytes(const TmaConfig &c)
{
    return size_t(c.stages + 2) * c.tile_bytes + size_t(c.stages) * 8;
}

// Per (device, config) launch facts: opt-in shared memory set, CTAs per SM.
struct LaunchFacts {
    bool ready = false;
    int ctas_per_sm = 0;
};

std::mutex g_facts_mu;
LaunchFacts g_facts[64][2];

optigpu_status tma_launch_facts(const DeviceInfo &dev, const TmaConfig &c, int &ctas_per_sm)
{
    std::lock_guard<std::mutex> lk(g_facts_mu);
    LaunchFacts &f = g_facts[dev.device & 63][c.esize == 4 ? 0 : 1];
    if (!f.ready) {
        const size_t smem = tma_smem_bytes(c);
        optigpu_status st = check_cuda(
            cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
            "cudaFuncSetAttribute(transpose tma smem)");
        if (st != OPTIGPU_OK)
            return st;
        int n = 0;
        st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, c.fn, c.threads, smem),
                        "cudaOccupancyMaxActiveBlocksPerMultiprocessor(transpose tma)");
        if (st != OPTIGPU_OK)
            return st;
        f.ctas_per_sm = std::max(n, 1);
        f.ready = true;
    }
    ctas_per_sm = f.ctas_per_sm;
    return OPTIGPU_OK;
}

bool tma_eligible(const void *src, const void *dst, int64_t rows, int64_t cols, size_t esize)
{
    if (esize != 2 && esize != 4)
        return false;
    const int64_t per16 = int64_t(16 / esize);
    if ((reinterpret_cast<uintptr_t>(src) & 15u) || (reinterpret_cast<uintptr_t>(dst) & 15u))
        return false;
    if (rows <= 0 || cols <= 0 || rows % per16 || cols % per16)
        return false;
    // TMA coordinates are int32 and global extents at most 2^32.
    if (rows > (int64_t(1) << 30) || cols > (int64_t(1) << 30))
        return false;
    return true;
}

optigpu_status launch_tma(const void *src, void *dst, int64_t rows, int64_t cols, size_t esize,
                          cudaStream_t stream)
{
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const TmaConfig &c = tma_config(esize);
    const CUtensorMapDataType type = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    alignas(64) CUtensorMap ms, md;
    // Source: dim0 = cols (contiguous), dim1 = rows; box TC x TR.
    if ((st = encode_tensor_map_2d(&ms, const_cast<void *>(src), type, uint64_t(cols), uint64_t(rows),
                                   uint64_t(cols) * esize, uint32_t(c.tc), uint32_t(c.tr))) != OPTIGPU_OK)
        return st;
    // Destination: dim0 = rows (contiguous), dim1 = cols; box TR x TC.
    if ((st = encode_tensor_map_2d(&md, dst, type, uint64_t(rows), uint64_t(cols), uint64_t(rows) * esize,
                                   uint32_t(c.tr), uint32_t(c.tc))) != OPTIGPU_OK)
        return st;
    int ctas_per_sm = 1;
    if ((st = tma_launch_facts(dev, c, ctas_per_sm)) != OPTIGPU_OK)
        return st;
    const int64_t tiles_c = (cols + c.tc - 1) / c.tc;
    const int64_t tiles_r = (rows + c.tr - 1) / c.tr;
    const int64_t num_tiles = tiles_r * tiles_c;
    const int64_t grid = std::min<int64_t>(num_tiles, int64_t(ctas_per_sm) * dev.num_sms);
    const size_t smem = tma_smem_bytes(c);
    const uint64_t limit = wait_limit_ns();
    int32_t tiles_c32 = int32_t(tiles_c);
    void *args[] = {&ms, &md, &tiles_c32, const_cast<int64_t *>(&num_tiles), const_cast<uint64_t *>(&limit),
                    &dev.status_word};
    return check_cuda(cudaLaunchKernel(c.fn, dim3(unsigned(grid)), dim3(unsigned(c.threads)), args, smem, stream),
                      "launch transpose tma");
}

optigpu_status launch_tile32(const void *src, void *dst, int64_t rows, int64_t cols, size_t esize,
                             cudaStream_t stream)
{
    const int64_t tiles_c = (cols + 31) / 32;
    const int64_t tiles = tiles_c * ((rows + 31) / 32);
    if (tiles > int64_t(0x7fffffff))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: too many 32x32 tiles for one launch");
    const dim3 block(32, 8);
    if (esize == 4)
        transpose_tile32_kernel<uint32_t><<<unsigned(tiles), block, 0, stream>>>(
            static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst), rows, cols, tiles_c);
    else
        transpose_tile32_kernel<uint16_t><<<unsigned(tiles), block, 0, stream>>>(
            static_cast<const uint16_t *>(src), static_cast<uint16_t *>(dst), rows, cols, tiles_c);
    return check_cuda(cudaGetLastError(), "launch transpose tile32");
}

optigpu_status validate(const void *src, const void *dst, int64_t rows, int64_t cols, int dtype)
{
    if (!dtype_valid(dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "transpose: unknown dtype " + std::to_string(dtype));
    if (rows < 0 || cols < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: negative rows or cols");
    if (rows == 0 || cols == 0)
        return OPTIGPU_OK;
    const size_t es = esize_of(optigpu_dtype(dtype));
    if (rows > (int64_t(1) << 62) / cols || rows * cols > (int64_t(1) << 62) / int64_t(es))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: rows * cols * element size too large");
    if (!src || !dst)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: null pointer");
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % es)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: pointer not aligned to the element size");
    const uintptr_t bytes = uintptr_t(rows * cols) * es;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
    if (a < b + bytes && b < a + bytes)
        return fail(OPTIGPU_ERR_OVERLAP, "transpose: src and dst overlap (the transpose is out-of-place)");
    return OPTIGPU_OK;
}

} // namespace

optigpu_status transpose_dispatch(const void *src, void *dst, int64_t rows, int64_t cols, int dtype,
                                  int kernel, cudaStream_t stream)
{
    optigpu_status st = validate(src, dst, rows, cols, dtype);
    if (st != OPTIGPU_OK)
        return st;
    if (kernel < OPTIGPU_TRANSPOSE_AUTO || kernel > OPTIGPU_TRANSPOSE_TMA)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: unknown kernel " + std::to_string(kernel));
    if (rows == 0 || cols == 0)
        return OPTIGPU_OK;
    const size_t es = esize_of(optigpu_dtype(dtype));
    const bool tma_ok = tma_eligible(src, dst, rows, cols, es);
    if (kernel == OPTIGPU_TRANSPOSE_TMA && !tma_ok)
        return fail(OPTIGPU_ERR_INVALID_ARG,
                    "transpose: TMA kernel needs 16-byte aligned pointers and rows, cols multiples of 16/esize");
    if (kernel == OPTIGPU_TRANSPOSE_TMA || (kernel == OPTIGPU_TRANSPOSE_AUTO && tma_ok))
        return launch_tma(src, dst, rows, cols, es, stream);
    return launch_tile32(src, dst, rows, cols, es, stream);
}

} // namespace optigpu

using namespace optigpu;

extern "C" {

optigpu_status optigpu_transpose(const void *src, void *dst, int64_t rows, int64_t cols,
                                 optigpu_dtype dtype, optigpu_stream_t stream)
{
    return transpose_dispatch(src, dst, rows, cols, int(dtype), OPTIGPU_TRANSPOSE_AUTO,
                              static_cast<cudaStream_t>(stream));
}

optigpu_status optigpu_transpose_ex(const void *src, void *dst, int64_t rows, int64_t cols,
                                    optigpu_dtype dtype, optigpu_transpose_kernel kernel,
                                    optigpu_stream_t stream)
{
    return transpose_dispatch(src, dst, rows, cols, int(dtype), int(kernel), static_cast<cudaStream_t>(stream));
}

int optigpu_transpose_tma_eligible(const void *src, const void *dst, int64_t rows, int64_t cols,
                                   optigpu_dtype dtype)
{
    if (!dtype_valid(int(dtype)))
        return 0;
    return tma_eligible(src, dst, rows, cols, esize_of(dtype)) ? 1 : 0;
}

} // extern "C"
