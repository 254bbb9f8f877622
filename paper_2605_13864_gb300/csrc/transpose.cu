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
#include <atomic>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tma_tile.cuh"

namespace optigpu {
namespace {

// ------------------------------------------------------------------ tile32

template <typename T>
__global__ void __launch_bounds__(256)
transpose_tile32_kernel(const T *__restrict__ src, T *__restrict__ dst, int64_t rows,
                        int64_t cols, int64_t tiles_c, int64_t lds, int64_t ldd,
                        int64_t tiles_per_mat, int64_t bs, int64_t bd)
{
    // 4-byte rows are padded by one element, 2-byte rows by two, so that a
    // column of the tile spans 32 distinct 4-byte banks.
    constexpr int PAD = sizeof(T) == 4 ? 1 : 2;
    __shared__ T tile[32][32 + PAD];
    const int64_t b = int64_t(blockIdx.x) / tiles_per_mat;
    const int64_t id = int64_t(blockIdx.x) - b * tiles_per_mat;
    src += b * bs;
    dst += b * bd;
    const int64_t tr = id / tiles_c;
    const int64_t tc = id - tr * tiles_c;
    const int64_t r0 = tr * 32, c0 = tc * 32;
    const int x = threadIdx.x, y = threadIdx.y;
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t r = r0 + y + j, c = c0 + x;
        if (r < rows && c < cols)
            tile[y + j][x] = src[r * lds + c];
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < 32; j += 8) {
        const int64_t orow = c0 + y + j, ocol = r0 + x;
        if (orow < cols && ocol < rows)
            dst[orow * ldd + ocol] = tile[x][y + j];
    }
}

// --------------------------------------------------------------------- tma

// Tile order.  Tile ids run down `group` tile-rows before moving one
// tile-column right, so the CTAs working at one moment (consecutive ids)
// cover a block of group x (CTAs / group) tiles: each source row band is read
// in runs of several KB and each destination row is written in runs of
// group x TR elements, instead of one short piece per destination row.
struct TileOrder {
    int32_t tiles_r, tiles_c, group;
    int64_t tiles_per_mat; // tiles_r * tiles_c; ids run matrix by matrix
    int32_t rows, cols;    // matrix extent in elements
    __device__ __forceinline__ void coords(int64_t id, int32_t &tr, int32_t &tc, int32_t &b) const
    {
        b = int32_t(id / tiles_per_mat);
        id -= int64_t(b) * tiles_per_mat;
        const int64_t per_group = int64_t(group) * tiles_c;
        const int32_t g = int32_t(id / per_group);
        const int32_t within = int32_t(id - int64_t(g) * per_group);
        const int32_t rows_here = min(group, tiles_r - g * group);
        tc = within / rows_here;
        tr = g * group + (within - tc * rows_here);
    }
};

// Warp roles: warps 0 .. THREADS/32 - 1 are consumers (one micro-block per
// thread); the last warp is the producer, whose lane 0 keeps the STAGES-deep
// ring of source tiles full.  Per stage s: full[s] completes when the TMA
// load has landed (transaction bytes), empty[s] when every consumer warp has
// taken its micro-blocks out.  NOB output buffers let up to NOB - 1 tile
// stores still read shared memory while the next tile is written.
// RANK 2: one matrix; RANK 3: a stack of matrices, the batch index being
// the tensor maps' third coordinate.
// SWZ: tiles move as 128-byte-wide boxes with TMA's 128-byte swizzle (two
// or more boxes per tile and direction) and the consumers address them
// through the same XOR pattern; otherwise one box per tile, unswizzled.
template <int ESIZE, int TR, int TC, int STAGES, int NOB, int RANK = 2, bool SWZ = false>
__global__ void __launch_bounds__(TmaTile<ESIZE, TR, TC>::THREADS + 32, 1)
transpose_tma_kernel(const __grid_constant__ CUtensorMap tm_src,
                     const __grid_constant__ CUtensorMap tm_dst, TileOrder order,
                     int64_t num_tiles, uint64_t wait_limit_ns, unsigned *status)
{
    using Tile = TmaTile<ESIZE, TR, TC>;
    constexpr int V = Tile::V;
    constexpr uint32_t NCONS = Tile::THREADS;
    constexpr uint32_t NWARPS_CONS = NCONS / 32;
    constexpr int BOX = 128 / ESIZE;          // elements per 128-byte box row (SWZ)
    constexpr int NS = SWZ ? TC / BOX : 1;    // source boxes per tile
    constexpr int ND = SWZ ? TR / BOX : 1;    // destination boxes per tile
    extern __shared__ __align__(1024) unsigned char smem[];
    // The swizzle pattern repeats every 1024 bytes from a 1024-byte boundary.
    const uint32_t raw = ptx::smem_addr(smem);
    const uint32_t in_base = SWZ ? (raw + 1023u) & ~1023u : raw;
    const uint32_t out_base = in_base + STAGES * Tile::BYTES;
    const uint32_t full_bar = out_base + NOB * Tile::BYTES;
    const uint32_t empty_bar = full_bar + 8u * STAGES;

    const int t = threadIdx.x;
    const int64_t first = blockIdx.x, stride = gridDim.x;
    const int64_t my_count = first < num_tiles ? (num_tiles - 1 - first) / stride + 1 : 0;

    // Launched with programmatic stream serialisation: wait until the
    // previous kernel on the stream has finished and its writes are visible
    // before any tile moves, then let the next kernel be launched (it waits
    // in turn), so back-to-back calls overlap a launch with this one's tail.
    // Both are no-ops for a plain launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    if (t == 0) {
        ptx::prefetch_tensormap(&tm_src);
        ptx::prefetch_tensormap(&tm_dst);
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(full_bar + 8u * s, 1);
            ptx::mbar_init(empty_bar + 8u * s, NWARPS_CONS);
        }
        ptx::fence_mbar_init();
    }
    __syncthreads();

    if (uint32_t(t) >= NCONS) {
        // ------------------------------------------------------ producer
        if (t != int(NCONS))
            return;
        int64_t k = 0;
        for (; k < my_count; ++k) {
            const uint32_t s = uint32_t(k % STAGES);
            if (k >= STAGES &&
                !ptx::mbar_wait_bounded(empty_bar + 8u * s, uint32_t(k / STAGES - 1) & 1u, wait_limit_ns)) {
                atomicOr(status, DEV_ERR_WAIT_TIMEOUT);
                break;
            }
            int32_t tr, tc, b;
            order.coords(first + k * stride, tr, tc, b);
            // Swizzled boxes that start past the last column are not loaded
            // (their elements lie outside the matrix and are never stored).
            const int ns = SWZ ? min(NS, (order.cols - tc * TC + BOX - 1) / BOX) : 1;
            ptx::mbar_arrive_expect_tx(full_bar + 8u * s, SWZ ? uint32_t(ns) * TR * 128u : Tile::BYTES);
#pragma unroll
            for (int h = 0; h < NS; ++h) {
                if (h >= ns)
                    break;
                const uint32_t dst_smem = in_base + s * Tile::BYTES + uint32_t(h) * TR * 128u;
                if (RANK == 3)
                    ptx::tma_load_3d(dst_smem, &tm_src, tc * TC + h * BOX, tr * TR, b, full_bar + 8u * s);
                else
                    ptx::tma_load_2d(dst_smem, &tm_src, tc * TC + h * BOX, tr * TR, full_bar + 8u * s);
            }
        }
        // Before leaving, let every load still in flight land (bounded), so no
        // copy targets this CTA's shared memory after the consumers are gone.
        for (int64_t kk = (k > STAGES ? k - STAGES : 0); kk < k; ++kk)
            ptx::mbar_wait_bounded(full_bar + 8u * uint32_t(kk % STAGES), uint32_t(kk / STAGES) & 1u,
                                   wait_limit_ns);
        return;
    }

    // ---------------------------------------------------------- consumers
    // Micro-block of this thread.  With q = t % 8 and p = t / 8, the 8
    // threads of a shared-memory wavefront (one quarter warp, 16-byte
    // accesses) share p and get rb % 8 = q and cb % 8 = (q + p) % 8: distinct
    // 16-byte bank groups on both the read and the write side.
    const int q = t & 7, p = t >> 3;
    const int rest = p >> 3;
    const int rb = (rest % (Tile::MR / 8)) * 8 + q;
    const int cb = (rest / (Tile::MR / 8)) * 8 + ((q + (p & 7)) & 7);
    const uint32_t rd_off = uint32_t(rb * V) * Tile::IN_PITCH + uint32_t(cb) * 16u;
    const uint32_t wr_off = uint32_t(cb * V) * Tile::OUT_PITCH + uint32_t(rb) * 16u;
    const bool lane0 = (t & 31) == 0;

    for (int64_t k = 0; k < my_count; ++k) {
        const uint32_t s = uint32_t(k % STAGES);
        const bool ok = ptx::mbar_wait_bounded(full_bar + 8u * s, uint32_t(k / STAGES) & 1u, wait_limit_ns);
        uint4 r[V];
        if (ok) {
#pragma unroll
            for (int i = 0; i < V; ++i)
                r[i] = ptx::lds_v4(in_base + s * Tile::BYTES +
                                   (SWZ ? swz128_offset(uint32_t(rb * V + i), uint32_t(cb), TR)
                                        : rd_off + uint32_t(i) * Tile::IN_PITCH));
        }
        // Output buffer k % NOB is free once the store issued NOB tiles ago
        // has read it: thread 0 (the only thread that issues stores) waits,
        // and the barrier below publishes that to every consumer.  The same
        // barrier lets all consumers agree on a timeout.
        if (t == 0)
            ptx::bulk_wait_group_read<NOB - 1>();
        if (ptx::named_bar_or(1, NCONS, !ok)) {
            if (t == 0) {
                atomicOr(status, DEV_ERR_WAIT_TIMEOUT);
                ptx::bulk_wait_group<0>();
            }
            return;
        }
        const uint32_t obuf = out_base + uint32_t(k % NOB) * Tile::BYTES;
        if (SWZ)
            store_transposed_at<ESIZE>(r, [&](int j) {
                return obuf + swz128_offset(uint32_t(cb * V + j), uint32_t(rb), TC);
            });
        else
            store_transposed<ESIZE>(r, obuf + wr_off, Tile::OUT_PITCH);
        // The values just stored came from stage s, so every lane's read of
        // it is complete: release the stage to the producer, one arrival per
        // warp.
        __syncwarp();
        if (lane0)
            ptx::mbar_arrive(empty_bar + 8u * s);
        ptx::fence_proxy_async_smem();
        ptx::named_bar_sync(2, NCONS);
        if (t == 0) {
            int32_t tr, tc, b;
            order.coords(first + k * stride, tr, tc, b);
#pragma unroll
            for (int h = 0; h < ND; ++h) {
                if (SWZ && tr * TR + h * BOX >= order.rows)
                    break; // a box wholly past the last destination column: nothing to store
                const uint32_t src_smem = obuf + uint32_t(h) * TC * 128u;
                if (RANK == 3)
                    ptx::tma_store_3d(&tm_dst, tr * TR + h * BOX, tc * TC, b, src_smem);
                else
                    ptx::tma_store_2d(&tm_dst, tr * TR + h * BOX, tc * TC, src_smem);
            }
            ptx::bulk_commit_group();
        }
    }
    if (t == 0)
        ptx::bulk_wait_group<0>();
}

// ------------------------------------------------------------------- host

struct TmaConfig {
    int esize;
    int tr, tc, stages, nob, threads;
    uint32_t tile_bytes;
    const void *fn;  // one matrix (2-D tensor maps)
    const void *fn3; // a stack of matrices (3-D tensor maps)
    const char *name;
    bool swz;        // 128-byte-wide swizzled boxes
};

template <int ESIZE, int TR, int TC, int STAGES, int NOB, bool SWZ = false>
TmaConfig make_config(const char *name)
{
    using Tile = TmaTile<ESIZE, TR, TC>;
    static_assert(!SWZ || (TR * ESIZE % 128 == 0 && TC * ESIZE % 128 == 0), "swizzled boxes are 128 bytes wide");
    return TmaConfig{ESIZE, TR, TC, STAGES, NOB, Tile::THREADS + 32, Tile::BYTES,
                     reinterpret_cast<const void *>(&transpose_tma_kernel<ESIZE, TR, TC, STAGES, NOB, 2, SWZ>),
                     reinterpret_cast<const void *>(&transpose_tma_kernel<ESIZE, TR, TC, STAGES, NOB, 3, SWZ>), name,
                     SWZ};
}

// The compiled TMA configurations per element size; index 0 is the default.
const std::vector<TmaConfig> &tma_configs(size_t esize)
{
    // Index 0, the default, is chosen by size (kBySize): measured with CUDA
    // events on square fp32 and bf16 matrices (fraction of the copy peak,
    // inputs cold / left in L2 by the previous call), four stages at two CTAs
    // per SM win below 1 GiB moved (fp32 5120^2-10240^2: 0.94-0.96 / 0.78-0.89,
    // bf16 6144^2-12288^2: 0.93-0.96 / 0.78-0.86), six stages at one CTA per SM
    // from 1 GiB up (fp32 12288^2 0.954 / 0.954 against 0.944 / 0.900, 16384^2
    // 0.968 against 0.91; bf16 16384^2 0.938 against 0.925).  Entry 0 carries
    // the six-stage kernel; launch_tma resolves it by size.  Deeper rings
    // (7-12 stages) and the other shapes measured slower.
    static const std::vector<TmaConfig> c4 = {
        make_config<4, 64, 64, 6, 2>("tma f32 64x64 by size (s4 o2 below 1 GiB moved, s6 o2 from 1 GiB)"),
        make_config<4, 64, 64, 6, 2>("tma f32 64x64 s6 o2"),
        make_config<4, 64, 64, 4, 2>("tma f32 64x64 s4 o2"),
        make_config<4, 64, 64, 3, 3>("tma f32 64x64 s3 o3"),
        make_config<4, 32, 128, 4, 2>("tma f32 32x128 s4 o2"),
        make_config<4, 128, 32, 4, 2>("tma f32 128x32 s4 o2"),
        make_config<4, 32, 64, 6, 3>("tma f32 32x64 s6 o3"),
        make_config<4, 64, 64, 4, 2, true>("tma f32 64x64 s4 o2 swizzle128"),
        make_config<4, 64, 64, 5, 2>("tma f32 64x64 s5 o2"),
        make_config<4, 64, 64, 7, 2>("tma f32 64x64 s7 o2"),
        make_config<4, 64, 64, 8, 2>("tma f32 64x64 s8 o2"),
    };
    static const std::vector<TmaConfig> c2 = {
        make_config<2, 64, 128, 6, 2>("tma 16b 64x128 by size (s4 o2 below 1 GiB moved, s6 o2 from 1 GiB)"),
        make_config<2, 64, 128, 6, 2>("tma 16b 64x128 s6 o2"),
        make_config<2, 64, 128, 4, 2>("tma 16b 64x128 s4 o2"),
        make_config<2, 64, 128, 3, 3>("tma 16b 64x128 s3 o3"),
        make_config<2, 128, 64, 4, 2>("tma 16b 128x64 s4 o2"),
        make_config<2, 128, 128, 3, 2>("tma 16b 128x128 s3 o2"),
        make_config<2, 64, 64, 6, 3>("tma 16b 64x64 s6 o3"),
        make_config<2, 64, 128, 4, 2, true>("tma 16b 64x128 s4 o2 swizzle128"),
        make_config<2, 64, 128, 5, 2>("tma 16b 64x128 s5 o2"),
        make_config<2, 64, 128, 7, 2>("tma 16b 64x128 s7 o2"),
        make_config<2, 64, 128, 8, 2>("tma 16b 64x128 s8 o2"),
    };
    return esize == 4 ? c4 : c2;
}

// Configuration 0 picks one of two entries by the bytes a call moves.
constexpr int kBySize = 0, kDeepRing = 1, kShallowRing = 2;
constexpr uint64_t kBySizeThreshold = uint64_t(1) << 30; // bytes read + written

int resolve_tma_config(int config, uint64_t moved_bytes)
{
    if (config != kBySize)
        return config;
    return moved_bytes < kBySizeThreshold ? kShallowRing : kDeepRing;
}

size_t tma_smem_bytes(const TmaConfig &c)
{
    // Swizzled tiles start on a 1024-byte boundary, found inside 1 KiB slack.
    return size_t(c.stages + c.nob) * c.tile_bytes + size_t(c.stages) * 16 + (c.swz ? 1024 : 0);
}

// Process-wide choice of TMA configuration per element size (autotuner).
std::atomic<int> g_tma_choice[2] = {0, 0};

// Per (device, config) launch facts: opt-in shared memory set, CTAs per SM.
struct LaunchFacts {
    bool ready = false;
    int ctas_per_sm = 0;
};

std::mutex g_facts_mu;
std::map<std::pair<int, const void *>, LaunchFacts> g_facts;

optigpu_status tma_launch_facts(const DeviceInfo &dev, const TmaConfig &c, const void *fn, int &ctas_per_sm)
{
    std::lock_guard<std::mutex> lk(g_facts_mu);
    LaunchFacts &f = g_facts[{dev.device, fn}];
    if (!f.ready) {
        const size_t smem = tma_smem_bytes(c);
        if (smem > dev.max_smem_optin)
            return fail(OPTIGPU_ERR_INVALID_ARG, std::string("transpose config needs too much shared memory: ") + c.name);
        optigpu_status st = check_cuda(
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
            "cudaFuncSetAttribute(transpose tma smem)");
        if (st != OPTIGPU_OK)
            return st;
        int n = 0;
        st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, c.threads, smem),
                        "cudaOccupancyMaxActiveBlocksPerMultiprocessor(transpose tma)");
        if (st != OPTIGPU_OK)
            return st;
        f.ctas_per_sm = std::max(n, 1);
        f.ready = true;
    }
    ctas_per_sm = f.ctas_per_sm;
    return OPTIGPU_OK;
}

// Tile-rows per group of the TMA kernel's tile order.
std::atomic<int> g_group_rows{16};

bool tma_eligible(const void *src, const void *dst, int64_t rows, int64_t cols, int64_t lds, int64_t ldd,
                  size_t esize)
{
    if (esize != 2 && esize != 4)
        return false;
    const int64_t per16 = int64_t(16 / esize);
    if ((reinterpret_cast<uintptr_t>(src) & 15u) || (reinterpret_cast<uintptr_t>(dst) & 15u))
        return false;
    if (rows <= 0 || cols <= 0 || rows % per16 || cols % per16 || lds % per16 || ldd % per16)
        return false;
    // Tensor-map strides are below 2^40 bytes.
    if (lds > (int64_t(1) << 38) || ldd > (int64_t(1) << 38))
        return false;
    // TMA coordinates are int32 and global extents at most 2^32.
    if (rows > (int64_t(1) << 30) || cols > (int64_t(1) << 30))
        return false;
    return true;
}

// A stack of `batch` matrices: matrix b of src starts bs elements after
// matrix b-1 (dst: bd).  batch == 1 is the single-matrix case.
struct Stack {
    int64_t batch = 1, bs = 0, bd = 0;
};

optigpu_status launch_tma(const void *src, void *dst, int64_t rows, int64_t cols, int64_t lds, int64_t ldd,
                          size_t esize, cudaStream_t stream, int config, Stack stack = Stack())
{
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const auto &configs = tma_configs(esize);
    if (config < 0)
        config = g_tma_choice[esize == 4 ? 0 : 1].load();
    if (config < 0 || config >= int(configs.size()))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: unknown TMA configuration");
    config = resolve_tma_config(config, 2 * uint64_t(rows) * uint64_t(cols) * uint64_t(stack.batch) * esize);
    const TmaConfig &c = configs[size_t(config)];
    const bool rank3 = stack.batch > 1;
    const CUtensorMapDataType type = esize == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    // Box widths: the whole tile row, or 128 bytes with the 128-byte swizzle.
    const uint32_t box_s = c.swz ? uint32_t(128 / esize) : uint32_t(c.tc);
    const uint32_t box_d = c.swz ? uint32_t(128 / esize) : uint32_t(c.tr);
    const CUtensorMapSwizzle swz = c.swz ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE;
    alignas(64) CUtensorMap ms, md;
    if (!rank3) {
        // Source: dim0 = cols (contiguous), dim1 = rows; box box_s x TR.
        if ((st = encode_tensor_map_2d(&ms, const_cast<void *>(src), type, uint64_t(cols), uint64_t(rows),
                                       uint64_t(lds) * esize, box_s, uint32_t(c.tr), swz)) != OPTIGPU_OK)
            return st;
        // Destination: dim0 = rows (contiguous), dim1 = cols; box box_d x TC.
        if ((st = encode_tensor_map_2d(&md, dst, type, uint64_t(rows), uint64_t(cols), uint64_t(ldd) * esize,
                                       box_d, uint32_t(c.tc), swz)) != OPTIGPU_OK)
            return st;
    } else {
        // dim2 = the matrix index, strides bs / bd elements.
        if ((st = encode_tensor_map_3d_swizzled(&ms, const_cast<void *>(src), type, uint64_t(cols), uint64_t(rows),
                                                uint64_t(stack.batch), uint64_t(lds) * esize,
                                                uint64_t(stack.bs) * esize, box_s, uint32_t(c.tr), swz)) !=
            OPTIGPU_OK)
            return st;
        if ((st = encode_tensor_map_3d_swizzled(&md, dst, type, uint64_t(rows), uint64_t(cols),
                                                uint64_t(stack.batch), uint64_t(ldd) * esize,
                                                uint64_t(stack.bd) * esize, box_d, uint32_t(c.tc), swz)) !=
            OPTIGPU_OK)
            return st;
    }
    const void *fn = rank3 ? c.fn3 : c.fn;
    int ctas_per_sm = 1;
    if ((st = tma_launch_facts(dev, c, fn, ctas_per_sm)) != OPTIGPU_OK)
        return st;
    const int64_t tiles_c = (cols + c.tc - 1) / c.tc;
    const int64_t tiles_r = (rows + c.tr - 1) / c.tr;
    const int64_t per_mat = tiles_r * tiles_c;
    const int64_t num_tiles = per_mat * stack.batch;
    const int64_t grid = std::min<int64_t>(num_tiles, int64_t(ctas_per_sm) * dev.num_sms);
    const size_t smem = tma_smem_bytes(c);
    const uint64_t limit = wait_limit_ns();
    TileOrder order{int32_t(tiles_r), int32_t(tiles_c), std::max(1, std::min(g_group_rows.load(), int(tiles_r))),
                    per_mat, int32_t(rows), int32_t(cols)};
    void *args[] = {&ms, &md, &order, const_cast<int64_t *>(&num_tiles), const_cast<uint64_t *>(&limit),
                    &dev.status_word};
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(unsigned(c.threads));
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return check_cuda(cudaLaunchKernelExC(&cfg, fn, args), "launch transpose tma");
}

optigpu_status launch_tile32(const void *src, void *dst, int64_t rows, int64_t cols, int64_t lds, int64_t ldd,
                             size_t esize, cudaStream_t stream, Stack stack = Stack())
{
    const int64_t tiles_c = (cols + 31) / 32;
    const int64_t per_mat = tiles_c * ((rows + 31) / 32);
    if (per_mat > int64_t(0x7fffffff) / stack.batch)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: too many 32x32 tiles for one launch");
    const int64_t tiles = per_mat * stack.batch;
    const dim3 block(32, 8);
    if (esize == 4)
        transpose_tile32_kernel<uint32_t><<<unsigned(tiles), block, 0, stream>>>(
            static_cast<const uint32_t *>(src), static_cast<uint32_t *>(dst), rows, cols, tiles_c, lds, ldd, per_mat,
            stack.bs, stack.bd);
    else
        transpose_tile32_kernel<uint16_t><<<unsigned(tiles), block, 0, stream>>>(
            static_cast<const uint16_t *>(src), static_cast<uint16_t *>(dst), rows, cols, tiles_c, lds, ldd, per_mat,
            stack.bs, stack.bd);
    return check_cuda(cudaGetLastError(), "launch transpose tile32");
}

optigpu_status validate(const void *src, int64_t lds, const void *dst, int64_t ldd, int64_t rows, int64_t cols,
                        int dtype)
{
    if (!dtype_valid(dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "transpose: unknown dtype " + std::to_string(dtype));
    if (rows < 0 || cols < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: negative rows or cols");
    if (rows == 0 || cols == 0)
        return OPTIGPU_OK;
    if (lds < cols || ldd < rows)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: leading dimensions must be lds >= cols and ldd >= rows");
    const size_t es = esize_of(optigpu_dtype(dtype));
    const int64_t lim = (int64_t(1) << 62) / int64_t(es);
    if (rows > lim / lds || cols > lim / ldd)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: matrix extent times element size too large");
    if (!src || !dst)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: null pointer");
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % es)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: pointer not aligned to the element size");
    // Byte spans actually touched: the first to the last element of each matrix.
    const uintptr_t sb = uintptr_t((rows - 1) * lds + cols) * es, db = uintptr_t((cols - 1) * ldd + rows) * es;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
    if (a < b + db && b < a + sb)
        return fail(OPTIGPU_ERR_OVERLAP, "transpose: src and dst overlap (the transpose is out-of-place)");
    return OPTIGPU_OK;
}

} // namespace

// ------------------------------------------------------------- tuning hooks

int transpose_num_configs(size_t esize) { return int(tma_configs(esize).size()) + 1; }

const char *transpose_config_name(size_t esize, int config)
{
    const auto &c = tma_configs(esize);
    if (config >= 0 && config < int(c.size()))
        return c[size_t(config)].name;
    if (config == int(c.size()))
        return "tile32 padded 32x33 (no TMA)";
    return nullptr;
}

int transpose_selected(size_t esize) { return g_tma_choice[esize == 4 ? 0 : 1].load(); }

void transpose_select(size_t esize, int config) { g_tma_choice[esize == 4 ? 0 : 1].store(config); }

void transpose_set_group_rows(int g) { g_group_rows.store(g > 0 ? g : 16); }

int transpose_group_rows() { return g_group_rows.load(); }

// Launches configuration `config` (an index of transpose_config_name) on an
// eligible shape; the TMA configurations need tma_eligible().
optigpu_status transpose_launch_config(const void *src, void *dst, int64_t rows, int64_t cols, size_t esize,
                                       int config, cudaStream_t stream)
{
    if (config == int(tma_configs(esize).size()))
        return launch_tile32(src, dst, rows, cols, cols, rows, esize, stream);
    if (!tma_eligible(src, dst, rows, cols, cols, rows, esize))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: shape or alignment not eligible for TMA");
    return launch_tma(src, dst, rows, cols, cols, rows, esize, stream, config);
}

optigpu_status transpose_dispatch_pitched(const void *src, int64_t lds, void *dst, int64_t ldd, int64_t rows,
                                          int64_t cols, int dtype, int kernel, cudaStream_t stream)
{
    optigpu_status st = validate(src, lds, dst, ldd, rows, cols, dtype);
    if (st != OPTIGPU_OK)
        return st;
    if (kernel < OPTIGPU_TRANSPOSE_AUTO || kernel > OPTIGPU_TRANSPOSE_TMA)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose: unknown kernel " + std::to_string(kernel));
    if (rows == 0 || cols == 0)
        return OPTIGPU_OK;
    const size_t es = esize_of(optigpu_dtype(dtype));
    const bool tma_ok = tma_eligible(src, dst, rows, cols, lds, ldd, es);
    if (kernel == OPTIGPU_TRANSPOSE_TMA && !tma_ok)
        return fail(OPTIGPU_ERR_INVALID_ARG,
                    "transpose: TMA kernel needs 16-byte aligned pointers and rows, cols, lds, ldd multiples of "
                    "16/esize");
    const int choice = transpose_selected(es);
    if (kernel == OPTIGPU_TRANSPOSE_TMA)
        return launch_tma(src, dst, rows, cols, lds, ldd, es, stream,
                          choice < int(tma_configs(es).size()) ? choice : 0);
    if (kernel == OPTIGPU_TRANSPOSE_AUTO && tma_ok && choice < int(tma_configs(es).size()))
        return launch_tma(src, dst, rows, cols, lds, ldd, es, stream, choice);
    return launch_tile32(src, dst, rows, cols, lds, ldd, es, stream);
}

optigpu_status transpose_dispatch(const void *src, void *dst, int64_t rows, int64_t cols, int dtype, int kernel,
                                  cudaStream_t stream)
{
    return transpose_dispatch_pitched(src, cols, dst, rows, rows, cols, dtype, kernel, stream);
}

// `batch` dense rows x cols matrices, stride_src / stride_dst elements apart.
optigpu_status transpose_batched_dispatch(const void *src, int64_t stride_src, void *dst, int64_t stride_dst,
                                          int64_t batch, int64_t rows, int64_t cols, int dtype, cudaStream_t stream)
{
    if (!dtype_valid(dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "transpose_batched: unknown dtype " + std::to_string(dtype));
    if (batch < 0 || rows < 0 || cols < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: negative size");
    if (batch == 0 || rows == 0 || cols == 0)
        return OPTIGPU_OK;
    if (batch == 1)
        return transpose_dispatch(src, dst, rows, cols, dtype, OPTIGPU_TRANSPOSE_AUTO, stream);
    const size_t es = esize_of(optigpu_dtype(dtype));
    const int64_t lim = (int64_t(1) << 62) / int64_t(es);
    if (rows > lim / cols || batch > (int64_t(1) << 31))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: sizes too large");
    const int64_t n = rows * cols;
    if (stride_src < n || stride_dst < n)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: strides must be >= rows * cols");
    if (stride_src > lim / batch || stride_dst > lim / batch)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: strides too large");
    if (!src || !dst)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: null pointer");
    if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) % es)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_batched: pointer not aligned to the element size");
    const uintptr_t sb = uintptr_t((batch - 1) * stride_src + n) * es, db = uintptr_t((batch - 1) * stride_dst + n) * es;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
    if (a < b + db && b < a + sb)
        return fail(OPTIGPU_ERR_OVERLAP, "transpose_batched: src and dst overlap");
    Stack stack;
    stack.batch = batch;
    stack.bs = stride_src;
    stack.bd = stride_dst;
    const int64_t per16 = int64_t(16 / es);
    const int choice = transpose_selected(es);
    if (tma_eligible(src, dst, rows, cols, cols, rows, es) && stride_src % per16 == 0 && stride_dst % per16 == 0 &&
        choice < int(tma_configs(es).size()))
        return launch_tma(src, dst, rows, cols, cols, rows, es, stream, choice, stack);
    return launch_tile32(src, dst, rows, cols, cols, rows, es, stream, stack);
}

optigpu_status transpose_band_into(const void *band, void *dst, int64_t b, int64_t cols, int64_t ldd, int dtype,
                                   cudaStream_t stream)
{
    return transpose_dispatch_pitched(band, cols, dst, ldd, b, cols, dtype, OPTIGPU_TRANSPOSE_AUTO, stream);
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
    optigpu::NvtxRange nvtx_range("optigpu_transpose_ex");
    return transpose_dispatch(src, dst, rows, cols, int(dtype), int(kernel), static_cast<cudaStream_t>(stream));
}

optigpu_status optigpu_transpose_strided(const void *src, int64_t lds, void *dst, int64_t ldd, int64_t rows,
                                         int64_t cols, optigpu_dtype dtype, optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_transpose_strided");
    return transpose_dispatch_pitched(src, lds, dst, ldd, rows, cols, int(dtype), OPTIGPU_TRANSPOSE_AUTO,
                                      static_cast<cudaStream_t>(stream));
}

optigpu_status optigpu_transpose_batched(const void *src, int64_t stride_src, void *dst, int64_t stride_dst,
                                         int64_t batch, int64_t rows, int64_t cols, optigpu_dtype dtype,
                                         optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_transpose_batched");
    return transpose_batched_dispatch(src, stride_src, dst, stride_dst, batch, rows, cols, int(dtype),
                                      static_cast<cudaStream_t>(stream));
}

int optigpu_transpose_tma_eligible(const void *src, const void *dst, int64_t rows, int64_t cols,
                                   optigpu_dtype dtype)
{
    if (!dtype_valid(int(dtype)))
        return 0;
    return tma_eligible(src, dst, rows, cols, cols, rows, esize_of(dtype)) ? 1 : 0;
}

int optigpu_transpose_config_for(int64_t rows, int64_t cols, optigpu_dtype dtype)
{
    if (!dtype_valid(int(dtype)) || rows < 0 || cols < 0)
        return -1;
    const size_t es = esize_of(dtype);
    const int64_t per16 = int64_t(16 / es);
    const int tile32 = int(tma_configs(es).size());
    const int choice = transpose_selected(es);
    if (choice >= tile32 || rows == 0 || cols == 0 || rows % per16 || cols % per16 || rows > (int64_t(1) << 30) ||
        cols > (int64_t(1) << 30))
        return choice >= tile32 ? choice : tile32;
    return resolve_tma_config(choice, 2 * uint64_t(rows) * uint64_t(cols) * es);
}

} // extern "C"
