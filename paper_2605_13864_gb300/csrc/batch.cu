// batch.cu -- many uneven transposes and sums in one persistent launch.
//
// A plan flattens a descriptor table into work items: a transpose of
// rows x cols becomes ceil(rows/TILE) * ceil(cols/TILE) tile items, a sum of
// n elements becomes ceil(n / 16384) chunk items (the same chunks as the
// single-call sum).  A persistent grid (CTAs per SM x SMs) pulls items from a
// device work queue -- one integer atomic counter, each CTA claiming its next
// item while it works on the current one.  A chunk item writes its partial to
// the instance's slot and bumps the instance's completion counter; the CTA
// that finishes an instance's last chunk runs that instance's fixed-order
// FP64 / int64 final combine and resets the counter.  No float atomics; every
// sum is bit-identical to the single-call result, and every transpose is a
// bit copy, whatever the batch mix and the grid size.
//
// The plan owns its device workspace and a CUDA graph of one run (queue
// reset + kernel launch), so a run is one cudaGraphLaunch.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "batch_core.h"
#include "internal.h"
#include "reduce_core.cuh"

namespace optigpu {

namespace {

constexpr int kBatchThreads = 256;
static_assert(sizeof(BatchInst) % 8 == 0 && alignof(BatchInst) >= 8, "descriptors are copied in 8-byte words");

// Largest shared tile, in 32-bit words, for tiles of `AREA` elements: the row
// pitch S is TW + 1 words (TW + 2 halves for 16-bit data), so TH * S is at
// most 1.5 * AREA words (reached at TW = 2 for 4-byte elements).
template <int AREA>
struct BatchShared {
    union {
        uint32_t tile[AREA > 0 ? AREA + AREA / 2 : 1]; // AREA 0: sums only, no transpose tile
        ReduceCore<OPTIGPU_INT32, false>::Shared ri;
        ReduceCore<OPTIGPU_FLOAT32, false>::Shared rf;
        ReduceCore<OPTIGPU_FLOAT32, true>::Shared rfc;
        ReduceCore<OPTIGPU_BFLOAT16, false>::Shared rb;
        ReduceCore<OPTIGPU_BFLOAT16, true>::Shared rbc;
        ReduceCore<OPTIGPU_FLOAT16, false>::Shared rh;
        ReduceCore<OPTIGPU_FLOAT16, true>::Shared rhc;
    } u;
    // Ring of the next items: slot i & 3 holds this CTA's i-th item, its
    // instance index and its descriptor (filled one to three items ahead).
    BatchInst desc[4];
    int64_t item[4];
    uint32_t iidx[4];
    int last;
};

// Asynchronous copies global -> shared (L1-cached: the tables are read-only)
// and their completion, for the descriptor prefetch.
__device__ __forceinline__ void cp_async_4(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_8(void *smem_dst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(static_cast<uint32_t>(__cvta_generic_to_shared(smem_dst))), "l"(gsrc) : "memory");
}

// Row pitch of the shared tile in elements.  Reading a tile column means
// consecutive lanes step by one pitch; an odd pitch in 32-bit words puts them
// in distinct banks (4-byte: TW + 1, or 1 for a one-column tile; 2-byte:
// TW + 2 halves = an odd word count for TW >= 4, one word for TW <= 2).
template <typename T>
__device__ __forceinline__ int tile_pitch(int tw)
{
    if (sizeof(T) == 4)
        return tw == 1 ? 1 : tw + 1;
    return tw <= 2 ? 2 : tw + 2;
}

// One TH x TW tile (TH * TW <= AREA, TH and TW at most 256) of a transpose:
// coalesced reads of source rows into the shared tile, coalesced writes of
// destination rows (= tile columns).  With both sides at most 256, the 256
// threads stride the tile in whole rows: on the load side thread t always
// reads tile column t mod TW (rows t / TW + k * 256 / TW), on the store side
// it always writes tile row t mod TH (columns t / TH + k * 256 / TH).  So a
// thread's k-th address is its first plus k fixed strides, and its edge
// tests are one column (row) test plus a row (column) count: a few integer
// instructions per element instead of a fresh 64-bit index and bound check.
// Each thread issues all of its AREA / 256 loads before the first shared
// store, so they are in flight together.
template <int AREA, typename T>
__device__ __forceinline__ void transpose_tile(const BatchInst &in, int64_t local, T *tile)
{
    constexpr int PER = AREA / kBatchThreads;
    const int th_l = in.th_log2, tw_l = in.tw_log2;
    const int th = 1 << th_l, tw = 1 << tw_l;
    const int S = tile_pitch<T>(tw);
    const int64_t tr = local / in.aux, tc = local - tr * in.aux;
    const int64_t r0 = tr << th_l, c0 = tc << tw_l;
    const int64_t rows = in.rows, cols = in.cols;
    const int nr = int(rows - r0 < th ? rows - r0 : th); // rows of the tile inside the matrix
    const int nc = int(cols - c0 < tw ? cols - c0 : tw); // columns of the tile inside the matrix
    const int t = threadIdx.x;
    // Load side: tile column ct, tile rows rt, rt + dr, ...
    const int ct = t & (tw - 1), rt = t >> tw_l, dr = kBatchThreads >> tw_l;
    const bool col_in = ct < nc;
    const T *p = static_cast<const T *>(in.src) + (r0 + rt) * cols + c0 + ct;
    const int64_t pstep = int64_t(dr) * cols;
    T v[PER];
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        v[k] = (col_in && rt + k * dr < nr) ? *p : T(0);
        p += pstep;
    }
#pragma unroll
    for (int k = 0; k < PER; ++k)
        if (col_in && rt + k * dr < nr)
            tile[(rt + k * dr) * S + ct] = v[k];
    __syncthreads();
    // Store side: tile row rs (destination column r0 + rs), tile columns
    // (destination rows c0 + cs) cs, cs + dc, ...
    const int rs = t & (th - 1), cs = t >> th_l, dc = kBatchThreads >> th_l;
    const bool row_in = rs < nr;
    T *q = static_cast<T *>(in.dst) + (c0 + cs) * rows + r0 + rs;
    const int64_t qstep = int64_t(dc) * rows;
    const T *sp = tile + rs * S + cs;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
        if (row_in && cs + k * dc < nc)
            *q = sp[k * dc];
        q += qstep;
    }
}

template <int DT, bool COMP, int MB, typename Sh>
__device__ __forceinline__ void reduce_chunk(const BatchInst &in, int64_t local, uint32_t inst, void *partials,
                                             unsigned *inst_done, Sh &sh, int &s_last)
{
    using Core = ReduceCore<DT, COMP, MB>;
    using P = typename Core::Partial;
    auto &rs = *reinterpret_cast<typename Core::Shared *>(&sh);
    P *mine = static_cast<P *>(partials) + in.aux;
    const P part = Core::chunk_partial(in.src, in.rows, local, in.vec_ok != 0, rs);
    if (in.nitems == 1) {
        // A one-chunk sum: the fixed-order combine of a single partial is
        // 0 + partial (the other lanes add zeros), written without the
        // partials array, the fence and the completion counter.
        if (threadIdx.x == 0)
            *static_cast<P *>(in.dst) = P(0) + part;
        return;
    }
    if (threadIdx.x == 0) {
        mine[local] = part;
        __threadfence();
        s_last = (atomicAdd(inst_done + inst, 1u) == unsigned(in.nitems) - 1u) ? 1 : 0;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        Core::final_combine(mine, in.nitems, in.dst, rs);
        if (threadIdx.x == 0)
            inst_done[inst] = 0u;
    }
}

// Persistent batch kernel.  Items come from one integer atomic queue in a
// three-stage prefetch, so no round trip sits between two items: while item
// i runs, thread 0 claims item i+3, and warp 0 copies item i+2's instance
// index and item i+1's descriptor into the shared ring (cp.async), all
// completed by the barrier that ends item i.
// SUMS: a batch of sums only (every item a chunk).  No transpose tile in
// shared memory and the sum's 4-loads-in-flight schedule: 48 registers, 5
// CTAs per SM instead of 4 (6 would spill); the arithmetic, and so every
// result, is the same.
template <int AREA, bool SUMS = false>
__global__ void __launch_bounds__(kBatchThreads, SUMS ? 5 : 4)
batch_kernel(const BatchInst *__restrict__ insts, const uint32_t *__restrict__ item_inst, int64_t total_items,
             unsigned long long *queue, unsigned *inst_done, void *partials, int compensated)
{
    constexpr int MB = SUMS ? 4 : 8;
    __shared__ BatchShared<SUMS ? 0 : AREA> sh;
    const int t = threadIdx.x, lane = t & 31;
    if (t == 0) {
        int64_t prev = 0;
        for (int k = 0; k < 3; ++k) {
            const int64_t it = (k == 0 || prev < total_items) ? int64_t(atomicAdd(queue, 1ull)) : total_items;
            sh.item[k] = it;
            prev = it;
        }
        sh.item[3] = total_items;
        if (sh.item[0] < total_items) {
            sh.iidx[0] = item_inst[sh.item[0]];
            sh.desc[0] = insts[sh.iidx[0]];
        }
        if (sh.item[1] < total_items)
            sh.iidx[1] = item_inst[sh.item[1]];
    }
    __syncthreads();
    for (int i = 0;; ++i) {
        const int cur = i & 3;
        const int64_t item = sh.item[cur];
        if (item >= total_items)
            break;
        int64_t next = total_items;
        if (t < 32) {
            const int64_t i2 = sh.item[(i + 2) & 3], i1 = sh.item[(i + 1) & 3];
            if (t == 0 && i2 < total_items)
                next = int64_t(atomicAdd(queue, 1ull)); // item i+3, stored after this item
            if (lane == 0 && i2 < total_items)
                cp_async_4(&sh.iidx[(i + 2) & 3], item_inst + i2);
            if (i1 < total_items && lane < int(sizeof(BatchInst) / 8))
                cp_async_8(reinterpret_cast<char *>(&sh.desc[(i + 1) & 3]) + 8 * lane,
                           reinterpret_cast<const char *>(insts + sh.iidx[(i + 1) & 3]) + 8 * lane);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        const BatchInst in = sh.desc[cur];
        const uint32_t inst = sh.iidx[cur];
        const int64_t local = item - in.first_item;
        if (in.op == OPTIGPU_OP_TRANSPOSE) {
            // (Never reached with SUMS: such batches hold no transpose item.)
            if constexpr (!SUMS) {
                if (in.dtype == OPTIGPU_BFLOAT16 || in.dtype == OPTIGPU_FLOAT16)
                    transpose_tile<AREA, uint16_t>(in, local, reinterpret_cast<uint16_t *>(sh.u.tile));
                else
                    transpose_tile<AREA, uint32_t>(in, local, sh.u.tile);
            }
        } else {
            switch (in.dtype * 2 + (compensated ? 1 : 0)) {
            case OPTIGPU_INT32 * 2:
            case OPTIGPU_INT32 * 2 + 1:
                reduce_chunk<OPTIGPU_INT32, false, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            case OPTIGPU_FLOAT32 * 2:
                reduce_chunk<OPTIGPU_FLOAT32, false, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            case OPTIGPU_FLOAT32 * 2 + 1:
                reduce_chunk<OPTIGPU_FLOAT32, true, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            case OPTIGPU_BFLOAT16 * 2:
                reduce_chunk<OPTIGPU_BFLOAT16, false, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            case OPTIGPU_BFLOAT16 * 2 + 1:
                reduce_chunk<OPTIGPU_BFLOAT16, true, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            case OPTIGPU_FLOAT16 * 2:
                reduce_chunk<OPTIGPU_FLOAT16, false, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            default:
                reduce_chunk<OPTIGPU_FLOAT16, true, MB>(in, local, inst, partials, inst_done, sh.u, sh.last);
                break;
            }
        }
        if (t < 32) {
            if (t == 0)
                sh.item[(i + 3) & 3] = next;
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads(); // publishes the prefetched entries; the tile / reduce scratch may be reused
    }
}

struct BatchConfig {
    int tile; // transpose tile area in elements
    int ctas_per_sm; // 0 = as many as fit
    const void *fn;
    const char *name;
};

const std::vector<BatchConfig> &batch_configs()
{
    static const std::vector<BatchConfig> c = {
        {4096, 0, reinterpret_cast<const void *>(&batch_kernel<4096>), "batch tile area 4096 ctas/SM=max"},
        {4096, 4, reinterpret_cast<const void *>(&batch_kernel<4096>), "batch tile area 4096 ctas/SM=4"},
        {1024, 0, reinterpret_cast<const void *>(&batch_kernel<1024>), "batch tile area 1024 ctas/SM=max"},
        {1024, 8, reinterpret_cast<const void *>(&batch_kernel<1024>), "batch tile area 1024 ctas/SM=8"},
    };
    return c;
}

std::atomic<int> g_batch_choice{0};

} // namespace

int batch_num_configs() { return int(batch_configs().size()); }
const char *batch_config_name(int c)
{
    return (c >= 0 && c < batch_num_configs()) ? batch_configs()[size_t(c)].name : nullptr;
}
int batch_selected() { return g_batch_choice.load(); }
void batch_select(int c) { g_batch_choice.store(c); }

int batch_tile(int config) { return batch_configs()[size_t(config)].tile; }

namespace {
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
} // namespace

BatchLayout batch_layout(int64_t count, int64_t items, int64_t chunks)
{
    BatchLayout L;
    L.off_queue = 0;
    L.off_done = 256;
    L.off_inst = align_up(L.off_done + sizeof(unsigned) * size_t(std::max<int64_t>(count, 1)), 256);
    L.off_items = align_up(L.off_inst + sizeof(BatchInst) * size_t(std::max<int64_t>(count, 1)), 256);
    L.off_part = align_up(L.off_items + sizeof(uint32_t) * size_t(std::max<int64_t>(items, 1)), 256);
    L.total = L.off_part + 8 * size_t(std::max<int64_t>(chunks, 1));
    return L;
}

void batch_tile_shape(int64_t rows, int64_t cols, int area, int &th_log2, int &tw_log2)
{
    // Sides are capped at 256 (2^8), which the batch kernel's transpose
    // relies on (every thread keeps one tile column / row).
    auto log2_ceil = [](int64_t v) {
        int l = 0;
        while ((int64_t(1) << l) < v)
            ++l;
        return l;
    };
    int a_l = log2_ceil(area);
    const int side = a_l / 2;
    const int pr = std::min(log2_ceil(std::max<int64_t>(rows, 1)), a_l);
    const int pc = std::min(log2_ceil(std::max<int64_t>(cols, 1)), a_l);
    if (pr >= side && pc >= side) {
        th_log2 = side;
        tw_log2 = a_l - side;
    } else if (pc < side) {
        tw_log2 = pc;
        th_log2 = std::min(pr, a_l - pc);
    } else {
        th_log2 = pr;
        tw_log2 = std::min(pc, a_l - pr);
    }
    th_log2 = std::min(th_log2, 8);
    tw_log2 = std::min(tw_log2, 8);
}

optigpu_status batch_tables(const optigpu_desc *descs, int32_t count, int area, BatchTables &t)
{
    t.insts.assign(size_t(count), BatchInst{});
    t.item_inst.clear();
    t.items = t.chunks = t.bytes = 0;
    for (int32_t i = 0; i < count; ++i) {
        const optigpu_desc &d = descs[i];
        BatchInst &b = t.insts[size_t(i)];
        std::memset(&b, 0, sizeof b);
        b.src = d.src;
        b.dst = d.dst;
        b.op = d.op;
        b.dtype = d.dtype;
        b.first_item = t.items;
        const int64_t es = int64_t(esize_of(optigpu_dtype(d.dtype)));
        int64_t n_items = 0;
        if (d.op == OPTIGPU_OP_TRANSPOSE) {
            b.rows = d.rows;
            b.cols = d.cols;
            if (d.rows > 0 && d.cols > 0) {
                batch_tile_shape(d.rows, d.cols, area, b.th_log2, b.tw_log2);
                const int64_t th = int64_t(1) << b.th_log2, tw = int64_t(1) << b.tw_log2;
                const int64_t tc = (d.cols + tw - 1) / tw;
                const int64_t trn = (d.rows + th - 1) / th;
                b.aux = tc;
                n_items = tc * trn;
                t.bytes += 2 * d.rows * d.cols * es;
            }
        } else {
            b.rows = d.rows;
            b.cols = 1;
            b.vec_ok = (reinterpret_cast<uintptr_t>(d.src) & 15u) == 0 ? 1 : 0;
            b.aux = t.chunks;
            n_items = (d.rows + kReduceChunk - 1) / kReduceChunk;
            t.chunks += n_items;
            t.bytes += d.rows * es;
        }
        if (n_items > int64_t(0x7fffffff))
            return fail(OPTIGPU_ERR_INVALID_ARG, "batch: instance too large");
        b.nitems = int32_t(n_items);
        t.item_inst.insert(t.item_inst.end(), size_t(n_items), uint32_t(i));
        t.items += n_items;
    }
    return OPTIGPU_OK;
}

namespace {
std::mutex g_occ_mu;
std::map<std::pair<int, const void *>, int> g_occ; // (device, kernel) -> resident CTAs per SM
} // namespace

optigpu_status batch_launch(int config, const BatchInst *d_insts, const uint32_t *d_item_inst, int64_t items,
                            unsigned long long *d_queue, unsigned *d_done, int64_t clear_done, void *d_partials,
                            int compensated, cudaStream_t stream, int *grid_out, bool sums_only)
{
    const BatchConfig &c = batch_configs()[size_t(config)];
    // A batch of sums only runs the kernel form without a transpose tile, at
    // as many CTAs per SM as fit; the configuration's tile and CTA cap are
    // for batches that hold transposes.
    const void *fn = sums_only ? reinterpret_cast<const void *>(&batch_kernel<4096, true>) : c.fn;
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    int per_sm = 0;
    {
        std::lock_guard<std::mutex> lk(g_occ_mu);
        auto it = g_occ.find({dev.device, fn});
        if (it == g_occ.end()) {
            if ((st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kBatchThreads, 0),
                                 "cudaOccupancyMaxActiveBlocksPerMultiprocessor(batch)")) != OPTIGPU_OK)
                return st;
            it = g_occ.emplace(std::make_pair(dev.device, fn), std::max(per_sm, 1)).first;
        }
        per_sm = it->second;
    }
    if (!sums_only && c.ctas_per_sm > 0)
        per_sm = std::min(per_sm, c.ctas_per_sm);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(items, int64_t(per_sm) * dev.num_sms));
    // The counters follow the queue in the layout (batch_layout), so one
    // memset covers both when they must be cleared.
    const size_t clear = clear_done > 0 ? size_t(reinterpret_cast<char *>(d_done + clear_done) -
                                                 reinterpret_cast<char *>(d_queue))
                                        : sizeof(unsigned long long);
    if (clear_done >= 0 &&
        (st = check_cuda(cudaMemsetAsync(d_queue, 0, clear, stream), "batch: reset queue")) != OPTIGPU_OK)
        return st;
    int comp = compensated;
    void *args[] = {&d_insts, &d_item_inst, &items, &d_queue, &d_done, &d_partials, &comp};
    if ((st = check_cuda(cudaLaunchKernel(fn, dim3(unsigned(grid)), dim3(kBatchThreads), args, 0, stream),
                         "launch batch kernel")) != OPTIGPU_OK)
        return st;
    if (grid_out)
        *grid_out = int(grid);
    return OPTIGPU_OK;
}

optigpu_status batch_validate(const optigpu_desc &d, int32_t index);

} // namespace optigpu

// ------------------------------------------------------------------- plans

struct optigpu_batch_plan {
    int device = -1;
    int config = 0;
    uint32_t flags = 0;
    int32_t count = 0;
    int64_t total_items = 0;
    int64_t total_chunks = 0;
    int64_t bytes = 0;            // algorithmic bytes of one run
    std::vector<optigpu_desc> descs;
    // device workspace, one allocation
    void *ws = nullptr;
    optigpu::BatchInst *d_insts = nullptr;
    uint32_t *d_item_inst = nullptr;
    unsigned *d_inst_done = nullptr;
    void *d_partials = nullptr;
    unsigned long long *d_queue = nullptr;
    // graph of one run
    cudaGraphExec_t exec = nullptr;
    int graph_config = -1;
    int grid = 0;
};

namespace optigpu {
namespace {

std::mutex g_batch_mu;

optigpu_status validate_desc_impl(const optigpu_desc &d, int32_t i)
{
    const std::string where = "batch descriptor " + std::to_string(i) + ": ";
    if (d.op != OPTIGPU_OP_TRANSPOSE && d.op != OPTIGPU_OP_REDUCE)
        return fail(OPTIGPU_ERR_INVALID_ARG, where + "unknown op");
    if (!dtype_valid(d.dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, where + "unknown dtype");
    const size_t es = esize_of(optigpu_dtype(d.dtype));
    if (d.op == OPTIGPU_OP_TRANSPOSE) {
        if (d.rows < 0 || d.cols < 0)
            return fail(OPTIGPU_ERR_INVALID_ARG, where + "negative rows or cols");
        if (d.rows == 0 || d.cols == 0)
            return OPTIGPU_OK;
        if (d.rows > (int64_t(1) << 40) / d.cols)
            return fail(OPTIGPU_ERR_INVALID_ARG, where + "rows * cols too large for one batch instance");
        if (!d.src || !d.dst)
            return fail(OPTIGPU_ERR_INVALID_ARG, where + "null pointer");
        if ((reinterpret_cast<uintptr_t>(d.src) | reinterpret_cast<uintptr_t>(d.dst)) % es)
            return fail(OPTIGPU_ERR_INVALID_ARG, where + "pointer not aligned to the element size");
        const uintptr_t bytes = uintptr_t(d.rows * d.cols) * es;
        const uintptr_t a = reinterpret_cast<uintptr_t>(d.src), b = reinterpret_cast<uintptr_t>(d.dst);
        if (a < b + bytes && b < a + bytes)
            return fail(OPTIGPU_ERR_OVERLAP, where + "src and dst overlap");
        return OPTIGPU_OK;
    }
    if (d.rows < 0 || d.rows > (int64_t(1) << 40))
        return fail(OPTIGPU_ERR_INVALID_ARG, where + "n out of range");
    if (!d.dst || reinterpret_cast<uintptr_t>(d.dst) % 8)
        return fail(OPTIGPU_ERR_INVALID_ARG, where + "out must be a non-null 8-byte aligned pointer");
    if (d.rows > 0 && (!d.src || reinterpret_cast<uintptr_t>(d.src) % es))
        return fail(OPTIGPU_ERR_INVALID_ARG, where + "src must be non-null and element-aligned");
    return OPTIGPU_OK;
}

void free_plan_device(optigpu_batch_plan *p)
{
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    if (p->ws) {
        cudaFree(p->ws);
        p->ws = nullptr;
    }
}

// Enqueues one run (queue reset + kernel) of `p` with configuration `config`
// on `stream`.
optigpu_status enqueue_run(optigpu_batch_plan *p, int config, cudaStream_t stream, int *grid_out)
{
    return batch_launch(config, p->d_insts, p->d_item_inst, p->total_items, p->d_queue, p->d_inst_done, 0,
                        p->d_partials, (p->flags & OPTIGPU_REDUCE_COMPENSATED) ? 1 : 0, stream, grid_out,
                        p->total_items == p->total_chunks);
}

// Builds the device tables of `p` for its current configuration (tile size).
optigpu_status build_tables(optigpu_batch_plan *p)
{
    BatchTables t;
    optigpu_status st = batch_tables(p->descs.data(), p->count, batch_tile(p->config), t);
    if (st != OPTIGPU_OK)
        return st;
    p->total_items = t.items;
    p->total_chunks = t.chunks;
    p->bytes = t.bytes;
    const BatchLayout L = batch_layout(p->count, t.items, t.chunks);
    free_plan_device(p);
    if ((st = check_cuda(cudaMalloc(&p->ws, L.total), "batch: cudaMalloc(workspace)")) != OPTIGPU_OK)
        return st;
    char *base = static_cast<char *>(p->ws);
    p->d_queue = reinterpret_cast<unsigned long long *>(base + L.off_queue);
    p->d_inst_done = reinterpret_cast<unsigned *>(base + L.off_done);
    p->d_insts = reinterpret_cast<BatchInst *>(base + L.off_inst);
    p->d_item_inst = reinterpret_cast<uint32_t *>(base + L.off_items);
    p->d_partials = base + L.off_part;
    if ((st = check_cuda(cudaMemset(p->ws, 0, L.off_inst), "batch: clear counters")) != OPTIGPU_OK)
        return st;
    if (p->count > 0 &&
        (st = check_cuda(cudaMemcpy(p->d_insts, t.insts.data(), sizeof(BatchInst) * t.insts.size(),
                                    cudaMemcpyHostToDevice),
                         "batch: upload instances")) != OPTIGPU_OK)
        return st;
    if (t.items > 0 &&
        (st = check_cuda(cudaMemcpy(p->d_item_inst, t.item_inst.data(), sizeof(uint32_t) * t.item_inst.size(),
                                    cudaMemcpyHostToDevice),
                         "batch: upload item map")) != OPTIGPU_OK)
        return st;
    return OPTIGPU_OK;
}

} // namespace

optigpu_status batch_validate(const optigpu_desc &d, int32_t index) { return validate_desc_impl(d, index); }

namespace {

// Captures one run into a CUDA graph on a private stream.
optigpu_status build_graph(optigpu_batch_plan *p)
{
    if (p->exec) {
        cudaGraphExecDestroy(p->exec);
        p->exec = nullptr;
    }
    cudaStream_t cap = nullptr;
    DeviceInfo dev;
    optigpu_status st = current_device(dev); // caches device facts outside the capture
    if (st != OPTIGPU_OK)
        return st;
    if ((st = check_cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "batch: cudaStreamCreate")) !=
        OPTIGPU_OK)
        return st;
    cudaGraph_t graph = nullptr;
    st = check_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "batch: begin capture");
    if (st == OPTIGPU_OK) {
        const optigpu_status run = enqueue_run(p, p->config, cap, &p->grid);
        st = check_cuda(cudaStreamEndCapture(cap, &graph), "batch: end capture");
        if (run != OPTIGPU_OK)
            st = run;
    }
    if (st == OPTIGPU_OK)
        st = check_cuda(cudaGraphInstantiate(&p->exec, graph, 0), "batch: cudaGraphInstantiate");
    if (graph)
        cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
    if (st == OPTIGPU_OK)
        p->graph_config = p->config;
    return st;
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" {

optigpu_status optigpu_batch_plan_create(const optigpu_desc *descs, int32_t count, uint32_t flags,
                                         optigpu_batch_plan **plan)
{
    optigpu::NvtxRange nvtx_range("optigpu_batch_plan_create");
    if (!plan)
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch: null plan pointer");
    *plan = nullptr;
    if (count < 0 || (count > 0 && !descs))
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch: bad descriptor table");
    if (flags & ~(OPTIGPU_REDUCE_COMPENSATED | OPTIGPU_BATCH_NO_GRAPH))
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch: unknown flag bits");
    for (int32_t i = 0; i < count; ++i) {
        optigpu_status st = batch_validate(descs[i], i);
        if (st != OPTIGPU_OK)
            return st;
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    optigpu_batch_plan *p = new (std::nothrow) optigpu_batch_plan();
    if (!p)
        return fail(OPTIGPU_ERR_OOM, "batch: host allocation failed");
    cudaGetDevice(&p->device);
    p->flags = flags;
    p->count = count;
    p->descs.assign(descs, descs + count);
    p->config = batch_selected();
    optigpu_status st = build_tables(p);
    if (st == OPTIGPU_OK && !(flags & OPTIGPU_BATCH_NO_GRAPH) && p->total_items > 0)
        st = build_graph(p);
    if (st != OPTIGPU_OK) {
        free_plan_device(p);
        delete p;
        return st;
    }
    *plan = p;
    return OPTIGPU_OK;
}

optigpu_status optigpu_batch_run(optigpu_batch_plan *plan, optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_batch_run");
    if (!plan)
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch: null plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (plan->total_items == 0) {
        // Only empty instances: sums of nothing are 0.
        for (const optigpu_desc &d : plan->descs)
            if (d.op == OPTIGPU_OP_REDUCE) {
                optigpu_status st = check_cuda(cudaMemsetAsync(d.dst, 0, 8, s), "batch: write 0");
                if (st != OPTIGPU_OK)
                    return st;
            }
        return OPTIGPU_OK;
    }
    // Sums of length 0 inside a batch have no chunk: write their zero first.
    for (const optigpu_desc &d : plan->descs)
        if (d.op == OPTIGPU_OP_REDUCE && d.rows == 0) {
            optigpu_status st = check_cuda(cudaMemsetAsync(d.dst, 0, 8, s), "batch: write 0");
            if (st != OPTIGPU_OK)
                return st;
        }
    if (plan->exec && plan->graph_config == plan->config)
        return check_cuda(cudaGraphLaunch(plan->exec, s), "batch: cudaGraphLaunch");
    return enqueue_run(plan, plan->config, s, &plan->grid);
}

optigpu_status optigpu_batch_plan_info(const optigpu_batch_plan *plan, int64_t *items, int64_t *bytes,
                                       int32_t *grid)
{
    if (!plan)
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch: null plan");
    if (items)
        *items = plan->total_items;
    if (bytes)
        *bytes = plan->bytes;
    if (grid)
        *grid = plan->grid;
    return OPTIGPU_OK;
}

optigpu_status optigpu_batch_autotune(optigpu_batch_plan *plan, int reps, optigpu_stream_t stream,
                                      int *best_config, float *best_ms)
{
    optigpu::NvtxRange nvtx_range("optigpu_batch_autotune");
    if (!plan || reps < 1 || reps > 1000)
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch_autotune: null plan or reps outside [1, 1000]");
    if (plan->total_items == 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "batch_autotune: empty plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t a = nullptr, b = nullptr;
    optigpu_status st = check_cuda(cudaEventCreate(&a), "cudaEventCreate");
    if (st == OPTIGPU_OK)
        st = check_cuda(cudaEventCreate(&b), "cudaEventCreate");
    int best = -1;
    float best_t = 0.f;
    for (int c = 0; st == OPTIGPU_OK && c < batch_num_configs(); ++c) {
        plan->config = c;
        if ((st = build_tables(plan)) != OPTIGPU_OK)
            break;
        std::vector<float> t;
        for (int r = 0; r < reps + 1 && st == OPTIGPU_OK; ++r) {
            cudaEventRecord(a, s);
            st = enqueue_run(plan, c, s, &plan->grid);
            cudaEventRecord(b, s);
            if (st == OPTIGPU_OK)
                st = check_cuda(cudaEventSynchronize(b), "cudaEventSynchronize");
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (r > 0)
                t.push_back(ms);
        }
        if (st != OPTIGPU_OK)
            break;
        std::sort(t.begin(), t.end());
        if (best < 0 || t[t.size() / 2] < best_t) {
            best = c;
            best_t = t[t.size() / 2];
        }
    }
    if (a)
        cudaEventDestroy(a);
    if (b)
        cudaEventDestroy(b);
    if (st != OPTIGPU_OK)
        return st;
    plan->config = best;
    batch_select(best);
    if ((st = build_tables(plan)) != OPTIGPU_OK)
        return st;
    if (!(plan->flags & OPTIGPU_BATCH_NO_GRAPH) && (st = build_graph(plan)) != OPTIGPU_OK)
        return st;
    if (best_config)
        *best_config = best;
    if (best_ms)
        *best_ms = best_t;
    return OPTIGPU_OK;
}

void optigpu_batch_plan_destroy(optigpu_batch_plan *plan)
{
    if (!plan)
        return;
    free_plan_device(plan);
    delete plan;
}

} // extern "C"

// ------------------------------------------------------------ segmented sums

namespace optigpu {
namespace {

// Pinned staging for the per-call tables of optigpu_reduce_segmented: two
// page-locked buffers per (device, stream), each reused only after the copy
// made from it has run (its event), so the upload is a true asynchronous
// copy that never waits for the stream's earlier work.  Held until exit.
struct SegStage {
    void *host[2] = {nullptr, nullptr};
    size_t cap[2] = {0, 0};
    cudaEvent_t done[2] = {nullptr, nullptr};
    unsigned next = 0;
};
std::mutex g_seg_mu;
std::map<std::pair<int, cudaStream_t>, SegStage> g_seg_stage;

optigpu_status seg_stage_buffer(cudaStream_t s, size_t bytes, void **buf, cudaEvent_t *ev)
{
    int dev = -1;
    optigpu_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != OPTIGPU_OK)
        return st;
    std::lock_guard<std::mutex> lk(g_seg_mu);
    SegStage &g = g_seg_stage[std::make_pair(dev, s)];
    const unsigned b = g.next++ & 1u;
    if (g.done[b]) {
        if ((st = check_cuda(cudaEventSynchronize(g.done[b]), "reduce_segmented: staging reuse")) != OPTIGPU_OK)
            return st;
    } else if ((st = check_cuda(cudaEventCreateWithFlags(&g.done[b], cudaEventDisableTiming),
                                "reduce_segmented: staging event")) != OPTIGPU_OK) {
        return st;
    }
    if (g.cap[b] < bytes) {
        if (g.host[b])
            cudaFreeHost(g.host[b]);
        g.host[b] = nullptr;
        g.cap[b] = 0;
        const size_t want = std::max<size_t>(bytes, size_t(1) << 16);
        if (cudaHostAlloc(&g.host[b], want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            g.host[b] = nullptr;
            return fail(OPTIGPU_ERR_OOM, "reduce_segmented: pinned staging allocation failed");
        }
        g.cap[b] = want;
    }
    *buf = g.host[b];
    *ev = g.done[b];
    return OPTIGPU_OK;
}

// The tables of a segmented sum in one launch, one warp per segment: lane 0
// writes instance k (segment k; its items, the 16384-element chunks, start
// at first[k]; an empty segment gets no item and a zero result) and zeroes
// its completion counter, and the warp's lanes write k into the item map for
// every item of the segment; thread 0 also zeroes the work queue.  offsets
// and first may be host memory mapped for the device (one read of each per
// segment, all in flight together).
__global__ void seg_tables_kernel(const char *src, int64_t esize, int dtype, char *out, const int64_t *offsets,
                                  const int64_t *first, int32_t nseg, BatchInst *insts, uint32_t *item_inst,
                                  unsigned long long *queue, unsigned *done)
{
    const int64_t k = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (k == 0 && lane == 0)
        *queue = 0ull;
    if (k >= nseg)
        return;
    const int64_t o0 = offsets[k], o1 = offsets[k + 1], f0 = first[k];
    const int64_t len = o1 - o0;
    const int32_t nitems = int32_t((len + kReduceChunk - 1) / kReduceChunk);
    if (lane == 0) {
        BatchInst b;
        b.src = src + o0 * esize;
        b.dst = out + 8 * k;
        b.rows = len;
        b.cols = 1;
        b.first_item = f0;
        b.aux = f0; // one partial per chunk, in item order
        b.op = OPTIGPU_OP_REDUCE;
        b.dtype = dtype;
        b.nitems = nitems;
        b.vec_ok = (reinterpret_cast<uintptr_t>(b.src) & 15u) == 0 ? 1 : 0;
        b.th_log2 = 0;
        b.tw_log2 = 0;
        insts[k] = b;
        done[k] = 0u;
        if (len == 0)
            *reinterpret_cast<long long *>(out + 8 * k) = 0; // the same bits as int64 0 and double +0.0
    }
    for (int32_t i = lane; i < nitems; i += 32)
        item_inst[f0 + i] = uint32_t(k);
}

} // namespace
} // namespace optigpu

extern "C" optigpu_status optigpu_reduce_segmented(const void *src, const int64_t *offsets, int32_t nseg,
                                                   optigpu_dtype dtype, void *out, uint32_t flags,
                                                   optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_reduce_segmented");
    using namespace optigpu;
    if (!dtype_valid(int(dtype)))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "reduce_segmented: unknown dtype");
    if (flags & ~OPTIGPU_REDUCE_COMPENSATED)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: unknown flag bits");
    if (nseg < 0 || (nseg > 0 && (!offsets || !out)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: bad segment table or output");
    if (nseg == 0)
        return OPTIGPU_OK;
    if (reinterpret_cast<uintptr_t>(out) % 8)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: out must be 8-byte aligned");
    if (offsets[0] < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: negative offset");
    // One pass validates and counts the items (16384-element chunks).
    int64_t items = 0;
    for (int32_t k = 0; k < nseg; ++k) {
        const int64_t len = offsets[k + 1] - offsets[k];
        if (len < 0 || offsets[k + 1] > (int64_t(1) << 40))
            return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: offsets must be non-decreasing and < 2^40");
        items += (len + kReduceChunk - 1) / kReduceChunk;
    }
    const size_t es = esize_of(dtype);
    if (offsets[nseg] > offsets[0] && (!src || reinterpret_cast<uintptr_t>(src) % es))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_segmented: src must be non-null and element-aligned");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int config = 0;
    // Workspace: the batch tables (instance s = segment s), then the offsets
    // and every segment's first item, which the table kernel expands.
    const BatchLayout L = batch_layout(nseg, std::max<int64_t>(items, 1), std::max<int64_t>(items, 1));
    const size_t meta_bytes = 2 * 8 * (size_t(nseg) + 1);
    const size_t off_meta = (L.total + 255) / 256 * 256;
    void *ws = nullptr;
    optigpu_status st;
    if ((st = stream_workspace(s, off_meta + meta_bytes, &ws, 1)) != OPTIGPU_OK)
        return st;
    void *image = nullptr;
    cudaEvent_t copied = nullptr;
    if ((st = seg_stage_buffer(s, meta_bytes, &image, &copied)) != OPTIGPU_OK)
        return st;
    int64_t *h_off = static_cast<int64_t *>(image);
    int64_t *h_first = h_off + (nseg + 1);
    std::memcpy(h_off, offsets, 8 * (size_t(nseg) + 1));
    int64_t it = 0;
    for (int32_t k = 0; k < nseg; ++k) {
        h_first[k] = it;
        it += (offsets[k + 1] - offsets[k] + kReduceChunk - 1) / kReduceChunk;
    }
    h_first[nseg] = it;
    char *base = static_cast<char *>(ws);
    // The table kernel reads the offsets straight from the pinned staging
    // buffer when the device can address it (it always can on this part,
    // over NVLink-C2C); otherwise they are uploaded first.  Either way the
    // staging buffer is reused only after the event that follows its last
    // reader.
    const int64_t *d_off = static_cast<const int64_t *>(device_view_of_host(image, meta_bytes));
    if (!d_off) {
        d_off = reinterpret_cast<const int64_t *>(base + off_meta);
        if ((st = check_cuda(cudaMemcpyAsync(base + off_meta, image, meta_bytes, cudaMemcpyHostToDevice, s),
                             "reduce_segmented: upload offsets")) != OPTIGPU_OK)
            return st;
    }
    const int64_t *d_first = d_off + (nseg + 1);
    BatchInst *d_insts = reinterpret_cast<BatchInst *>(base + L.off_inst);
    uint32_t *d_items = reinterpret_cast<uint32_t *>(base + L.off_items);
    auto *d_queue = reinterpret_cast<unsigned long long *>(base + L.off_queue);
    auto *d_done = reinterpret_cast<unsigned *>(base + L.off_done);
    seg_tables_kernel<<<unsigned((int64_t(nseg) * 32 + 255) / 256), 256, 0, s>>>(
        static_cast<const char *>(src), int64_t(es), int(dtype), static_cast<char *>(out), d_off, d_first, nseg,
        d_insts, d_items, d_queue, d_done);
    if ((st = check_cuda(cudaGetLastError(), "reduce_segmented: tables")) != OPTIGPU_OK)
        return st;
    if ((st = check_cuda(cudaEventRecord(copied, s), "reduce_segmented: staging event")) != OPTIGPU_OK ||
        items == 0)
        return st;
    // The table kernel zeroed the queue and the counters (clear_done < 0).
    return batch_launch(config, d_insts, d_items, items, d_queue, d_done, -1, base + L.off_part,
                        (flags & OPTIGPU_REDUCE_COMPENSATED) ? 1 : 0, s, nullptr, true);
}
