// inplace.cu -- in-place transpose of a square n x n matrix: a[j][i] <- a[i][j]
// (the neighbouring variant of the thesis's out-of-place Listing 3.5).
//
// Work items are pairs of T x T tiles (r, c) and (c, r) of the lower triangle
// (p = r (r + 1) / 2 + c, c <= r); every element belongs to exactly one pair
// and is read before it is written, so no two CTAs touch the same element.
//
//  * TMA kernel (shapes whose rows are 16-byte multiples): a persistent grid;
//    a producer warp loads both tiles of each pair with 2-D TMA into a
//    STAGES-deep ring (full / empty mbarriers, bounded waits); consumer
//    threads transpose one 16-byte micro-block of each tile in registers into
//    output staging buffers; one thread stores tile (r, c)^T at (c, r) and
//    tile (c, r)^T at (r, c) with 2-D TMA.  A diagonal pair is one tile.
//  * padded-tile kernel: any n, any alignment; 64 x 64 tiles through padded
//    shared memory.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <vector>

#include "internal.h"
#include "ptx.cuh"
#include "tma_tile.cuh"

namespace optigpu {
namespace {

// Lower-triangle pair p -> (r, c), c <= r.
__device__ __forceinline__ void pair_coords(int64_t p, int32_t &r, int32_t &c)
{
    int64_t rr = int64_t((sqrt(8.0 * double(p) + 1.0) - 1.0) * 0.5);
    while (rr * (rr + 1) / 2 > p)
        --rr;
    while ((rr + 1) * (rr + 2) / 2 <= p)
        ++rr;
    r = int32_t(rr);
    c = int32_t(p - rr * (rr + 1) / 2);
}

// ---------------------------------------------------------------- in place

// In-place transpose of an n x n matrix: CTA p owns the tile pair (r, c) and
// (c, r) of the lower triangle (p = r (r + 1) / 2 + c, c <= r), loads both
// 64 x 64 tiles into padded shared tiles, and writes each back transposed in
// the other's place (a diagonal tile onto itself).  Every element belongs to
// exactly one pair and is read before it is written, so there is no race.
template <typename T>
__global__ void __launch_bounds__(256)
transpose_inplace_kernel(T *__restrict__ a, int64_t n, int64_t pairs)
{
    constexpr int TS = 64, PAD = sizeof(T) == 4 ? 1 : 2;
    __shared__ T tile[2][TS][TS + PAD];
    const int x = threadIdx.x & (TS - 1), y0 = threadIdx.x >> 6; // 64 x 4 threads
    for (int64_t p = blockIdx.x; p < pairs; p += gridDim.x) {
        int32_t r32, c32;
        pair_coords(p, r32, c32);
        const int64_t r = r32, c = c32;
        const bool diag = (r == c);
        // Tile 0 = block (r, c), tile 1 = block (c, r).
        for (int k = 0; k < TS; k += 4) {
            const int64_t i0 = r * TS + y0 + k, j0 = c * TS + x;
            if (i0 < n && j0 < n)
                tile[0][y0 + k][x] = a[i0 * n + j0];
            if (!diag) {
                const int64_t i1 = c * TS + y0 + k, j1 = r * TS + x;
                if (i1 < n && j1 < n)
                    tile[1][y0 + k][x] = a[i1 * n + j1];
            }
        }
        __syncthreads();
        // Block (c, r) receives tile 0 transposed; block (r, c) tile 1.
        for (int k = 0; k < TS; k += 4) {
            const int64_t i1 = c * TS + y0 + k, j1 = r * TS + x;
            if (i1 < n && j1 < n)
                a[i1 * n + j1] = tile[0][x][y0 + k];
            if (!diag) {
                const int64_t i0 = r * TS + y0 + k, j0 = c * TS + x;
                if (i0 < n && j0 < n)
                    a[i0 * n + j0] = tile[1][x][y0 + k];
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------ TMA pairs

template <int ESIZE, int T, int STAGES, int NOB>
__global__ void __launch_bounds__(TmaTile<ESIZE, T, T>::THREADS + 32, 1)
transpose_inplace_tma_kernel(const __grid_constant__ CUtensorMap tm, int64_t pairs, uint64_t wait_limit_ns,
                             unsigned *status)
{
    using Tile = TmaTile<ESIZE, T, T>;
    constexpr int V = Tile::V;
    constexpr uint32_t NCONS = Tile::THREADS;
    constexpr uint32_t NWARPS_CONS = NCONS / 32;
    constexpr uint32_t PAIR = 2 * Tile::BYTES;
    extern __shared__ __align__(1024) unsigned char smem[];
    const uint32_t in_base = ptx::smem_addr(smem);
    const uint32_t out_base = in_base + STAGES * PAIR;
    const uint32_t full_bar = out_base + NOB * PAIR;
    const uint32_t empty_bar = full_bar + 8u * STAGES;
    const int t = threadIdx.x;
    const int64_t first = blockIdx.x, stride = gridDim.x;
    const int64_t my_count = first < pairs ? (pairs - 1 - first) / stride + 1 : 0;

    if (t == 0) {
        ptx::prefetch_tensormap(&tm);
        for (int s = 0; s < STAGES; ++s) {
            ptx::mbar_init(full_bar + 8u * s, 1);
            ptx::mbar_init(empty_bar + 8u * s, NWARPS_CONS);
        }
        ptx::fence_mbar_init();
    }
    __syncthreads();

    if (uint32_t(t) >= NCONS) {
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
            int32_t r, c;
            pair_coords(first + k * stride, r, c);
            const uint32_t buf = in_base + s * PAIR;
            ptx::mbar_arrive_expect_tx(full_bar + 8u * s, r == c ? Tile::BYTES : PAIR);
            ptx::tma_load_2d(buf, &tm, c * T, r * T, full_bar + 8u * s);
            if (r != c)
                ptx::tma_load_2d(buf + Tile::BYTES, &tm, r * T, c * T, full_bar + 8u * s);
        }
        for (int64_t kk = (k > STAGES ? k - STAGES : 0); kk < k; ++kk)
            ptx::mbar_wait_bounded(full_bar + 8u * uint32_t(kk % STAGES), uint32_t(kk / STAGES) & 1u,
                                   wait_limit_ns);
        return;
    }

    // Consumers: the same bank-conflict-free micro-block assignment as the
    // out-of-place kernel.
    const int q = t & 7, pq = t >> 3;
    const int rest = pq >> 3;
    const int rb = (rest % (Tile::MR / 8)) * 8 + q;
    const int cb = (rest / (Tile::MR / 8)) * 8 + ((q + (pq & 7)) & 7);
    const uint32_t rd_off = uint32_t(rb * V) * Tile::IN_PITCH + uint32_t(cb) * 16u;
    const uint32_t wr_off = uint32_t(cb * V) * Tile::OUT_PITCH + uint32_t(rb) * 16u;
    const bool lane0 = (t & 31) == 0;

    for (int64_t k = 0; k < my_count; ++k) {
        const uint32_t s = uint32_t(k % STAGES);
        int32_t r, c;
        pair_coords(first + k * stride, r, c);
        const bool diag = (r == c);
        const bool ok = ptx::mbar_wait_bounded(full_bar + 8u * s, uint32_t(k / STAGES) & 1u, wait_limit_ns);
        uint4 ra[V], rbv[V];
        if (ok) {
            const uint32_t buf = in_base + s * PAIR;
#pragma unroll
            for (int i = 0; i < V; ++i)
                ra[i] = ptx::lds_v4(buf + rd_off + uint32_t(i) * Tile::IN_PITCH);
            if (!diag) {
#pragma unroll
                for (int i = 0; i < V; ++i)
                    rbv[i] = ptx::lds_v4(buf + Tile::BYTES + rd_off + uint32_t(i) * Tile::IN_PITCH);
            }
        }
        if (t == 0)
            ptx::bulk_wait_group_read<NOB - 1>();
        if (ptx::named_bar_or(1, NCONS, !ok)) {
            if (t == 0) {
                atomicOr(status, DEV_ERR_WAIT_TIMEOUT);
                ptx::bulk_wait_group<0>();
            }
            return;
        }
        const uint32_t obuf = out_base + uint32_t(k % NOB) * PAIR;
        store_transposed<ESIZE>(ra, obuf + wr_off, Tile::OUT_PITCH);
        if (!diag)
            store_transposed<ESIZE>(rbv, obuf + Tile::BYTES + wr_off, Tile::OUT_PITCH);
        __syncwarp();
        if (lane0)
            ptx::mbar_arrive(empty_bar + 8u * s);
        ptx::fence_proxy_async_smem();
        ptx::named_bar_sync(2, NCONS);
        if (t == 0) {
            // Tile (r, c) transposed lands at (c, r): rows c*T.., cols r*T..
            ptx::tma_store_2d(&tm, r * T, c * T, obuf);
            if (!diag)
                ptx::tma_store_2d(&tm, c * T, r * T, obuf + Tile::BYTES);
            ptx::bulk_commit_group();
        }
    }
    if (t == 0)
        ptx::bulk_wait_group<0>();
}

struct InplaceConfig {
    int esize, t, stages, nob, threads;
    uint32_t tile_bytes;
    const void *fn;
};

template <int ESIZE, int T, int STAGES, int NOB>
InplaceConfig make_inplace()
{
    using Tile = TmaTile<ESIZE, T, T>;
    return InplaceConfig{ESIZE, T, STAGES, NOB, Tile::THREADS + 32, Tile::BYTES,
                         reinterpret_cast<const void *>(&transpose_inplace_tma_kernel<ESIZE, T, STAGES, NOB>)};
}

const InplaceConfig &inplace_config(size_t esize)
{
    // Measured with CUDA events (fraction of the copy peak; variants compared
    // only within one run on one GPU).  fp32: 64x64 pairs, one stage and one
    // output buffer (64 KiB) at three CTAs per SM, 0.919-0.934 on 16384^2,
    // against 0.914-0.917 for a 4-stage ring at one CTA per SM and 0.835 for
    // 2 stages; it also wins at 4096^2-12288^2 (e.g. 8192^2 0.870 against
    // 0.840, L2 flushed).  16-bit: 128x128 pairs in a 2-stage ring at one CTA
    // per SM, 0.836-0.886 on 16384^2 against 0.80-0.85 for 64x64 pairs in one
    // stage, and 0.91-0.99 against 0.84-0.91 at 6144^2-8192^2 (64x64 pairs
    // with 2 output buffers 0.849, 2 stages 0.758; 128x128 in one stage
    // 0.729).
    static const InplaceConfig c4 = make_inplace<4, 64, 1, 1>();
    static const InplaceConfig c2 = make_inplace<2, 128, 2, 1>();
    return esize == 4 ? c4 : c2;
}

std::mutex g_inplace_mu;
std::map<std::pair<int, const void *>, int> g_inplace_ctas; // (device, kernel) -> CTAs per SM

optigpu_status launch_inplace_tma(void *a, int64_t n, size_t es, cudaStream_t stream)
{
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const InplaceConfig &c = inplace_config(es);
    const size_t smem = size_t(c.stages + c.nob) * 2 * c.tile_bytes + size_t(c.stages) * 16;
    int per_sm = 1;
    {
        std::lock_guard<std::mutex> lk(g_inplace_mu);
        auto it = g_inplace_ctas.find({dev.device, c.fn});
        if (it == g_inplace_ctas.end()) {
            if ((st = check_cuda(cudaFuncSetAttribute(c.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)),
                                 "cudaFuncSetAttribute(in-place)")) != OPTIGPU_OK)
                return st;
            int k = 0;
            if ((st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, c.fn, c.threads, smem),
                                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor(in-place)")) != OPTIGPU_OK)
                return st;
            it = g_inplace_ctas.emplace(std::make_pair(dev.device, c.fn), std::max(k, 1)).first;
        }
        per_sm = it->second;
    }
    alignas(64) CUtensorMap tm;
    const CUtensorMapDataType type = es == 4 ? CU_TENSOR_MAP_DATA_TYPE_UINT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    if ((st = encode_tensor_map_2d(&tm, a, type, uint64_t(n), uint64_t(n), uint64_t(n) * es, uint32_t(c.t),
                                   uint32_t(c.t))) != OPTIGPU_OK)
        return st;
    const int64_t nt = (n + c.t - 1) / c.t;
    int64_t pairs = nt * (nt + 1) / 2;
    const int64_t grid = std::min<int64_t>(pairs, int64_t(per_sm) * dev.num_sms);
    uint64_t limit = wait_limit_ns();
    void *args[] = {&tm, &pairs, &limit, &dev.status_word};
    return check_cuda(cudaLaunchKernel(c.fn, dim3(unsigned(grid)), dim3(unsigned(c.threads)), args, smem, stream),
                      "launch in-place tma");
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" {

optigpu_status optigpu_transpose_inplace(void *a, int64_t n, optigpu_dtype dtype, optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_transpose_inplace");
    if (!dtype_valid(int(dtype)))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "transpose_inplace: unknown dtype");
    if (n < 0 || n > (int64_t(1) << 30))
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_inplace: n out of range [0, 2^30]");
    if (n <= 1)
        return OPTIGPU_OK;
    const size_t es = esize_of(dtype);
    if (!a || reinterpret_cast<uintptr_t>(a) % es)
        return fail(OPTIGPU_ERR_INVALID_ARG, "transpose_inplace: null or misaligned pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t per16 = int64_t(16 / es);
    if ((reinterpret_cast<uintptr_t>(a) & 15u) == 0 && n % per16 == 0)
        return launch_inplace_tma(a, n, es, s);
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const int64_t nt = (n + 63) / 64;
    const int64_t pairs = nt * (nt + 1) / 2;
    const int64_t grid = std::min<int64_t>(pairs, int64_t(8) * dev.num_sms);
    if (es == 4)
        transpose_inplace_kernel<uint32_t><<<unsigned(grid), 256, 0, s>>>(static_cast<uint32_t *>(a), n, pairs);
    else
        transpose_inplace_kernel<uint16_t><<<unsigned(grid), 256, 0, s>>>(static_cast<uint16_t *>(a), n, pairs);
    return check_cuda(cudaGetLastError(), "launch transpose in place");
}

} // extern "C"
