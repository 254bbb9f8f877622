// server.cu -- continuous-batching request server for transposes and sums.
//
// Requests carry host buffers.  submit() queues a request; step() does one
// round of the serving loop:
//   1. completion: every stream whose completion event has fired releases its
//      requests -- their device buffers go back to the arena, their slots are
//      freed, and they are marked done (results are in their host buffers);
//   2. admission: while a stream is free, queued requests are admitted in
//      arrival order as long as a slot is free and their input + output fit
//      in the device-memory budget (an arena carved out of one allocation);
//   3. launch: the admitted requests' inputs are copied in, the step's batch
//      runs as ONE persistent batch kernel built from per-step tables (the
//      kernel of batch.cu: same chunks, same results as the single calls),
//      the outputs are copied back, and an event marks the step's end.
//      Requests whose host buffers are pinned are copied by two copy kernels
//      per step (a gather and a scatter through the device's mapping of the
//      host memory, over NVLink-C2C on GB300) instead of one copy-engine call
//      per buffer, so a step costs a fixed number of launches however many
//      requests it holds; the data still lands in the device arena.
// Requests that arrive while earlier steps run are admitted into the next
// step on another stream, so their copies and kernels overlap on the device.
//
// With OPTIGPU_SERVER_PER_CALL the same loop launches one plain kernel per
// request (optigpu_transpose / optigpu_reduce_sum_ex), one request per
// stream: the per-call baseline.  Two flags hold the copy path fixed across
// both modes, so that batching can be measured apart from it:
// OPTIGPU_SERVER_COPY_ENGINES copies every buffer with a copy-engine call
// (also in batched mode), OPTIGPU_SERVER_COPY_KERNELS moves pinned buffers
// with SM copy kernels in per-call mode too (one gather and one scatter
// launch per request).
//
// If launching a step fails, nothing of it stays on the device: its stream is
// drained, its requests give back their arena space and slots and return to
// the head of the queue in their order, and the error is returned; a later
// step tries them again.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "batch_core.h"
#include "internal.h"
#include "reduce_core.cuh"

namespace optigpu {
namespace {

double now_s()
{
    using clk = std::chrono::steady_clock;
    return std::chrono::duration<double>(clk::now().time_since_epoch()).count();
}

constexpr size_t kAlign = 256;
size_t round_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// One contiguous copy of a step: host<->arena through the device's mapping
// of pinned host memory, done by SMs instead of one copy-engine call each.
struct CopyDesc {
    const char *src;
    char *dst;
    int64_t bytes;
    int64_t first_piece; // prefix of pieces over the step's copies
};

constexpr int64_t kPiece = 32768; // bytes per work piece

// Copies every piece of `count` descriptors; CTAs stride over pieces.  Each
// piece uses the widest unit (16, 4 or 1 bytes) that both addresses allow.
// CTA 0 also zeroes the step's batch queue and its first `ndone` completion
// counters when `queue` is given (the batch kernel runs after this one).
__global__ void __launch_bounds__(256) copy_pieces_kernel(const CopyDesc *__restrict__ d, int32_t count,
                                                          int64_t pieces, unsigned long long *queue,
                                                          unsigned *done, int32_t ndone)
{
    if (queue && blockIdx.x == 0) {
        if (threadIdx.x == 0)
            *queue = 0ull;
        for (int32_t i = threadIdx.x; i < ndone; i += blockDim.x)
            done[i] = 0u;
    }
    for (int64_t p = blockIdx.x; p < pieces; p += gridDim.x) {
        int lo = 0, hi = count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (d[mid].first_piece <= p)
                lo = mid;
            else
                hi = mid - 1;
        }
        const CopyDesc c = d[lo];
        const int64_t off = (p - c.first_piece) * kPiece;
        const int64_t len = min(kPiece, c.bytes - off);
        const char *src = c.src + off;
        char *dst = c.dst + off;
        const uintptr_t al = reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst);
        int64_t done = 0;
        if ((al & 15u) == 0) {
            const int64_t n = len / 16;
            const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
            uint4 *d4 = reinterpret_cast<uint4 *>(dst);
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
                d4[i] = s4[i];
            done = n * 16;
        } else if ((al & 3u) == 0) {
            const int64_t n = len / 4;
            const uint32_t *s1 = reinterpret_cast<const uint32_t *>(src);
            uint32_t *d1 = reinterpret_cast<uint32_t *>(dst);
            for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
                d1[i] = s1[i];
            done = n * 4;
        }
        for (int64_t i = done + threadIdx.x; i < len; i += blockDim.x)
            dst[i] = src[i];
    }
}

// Copies one contiguous range (a request's buffer in per-call mode with copy
// kernels); CTAs stride over 16-byte units when both ends allow, else bytes.
__global__ void __launch_bounds__(256) copy_range_kernel(const char *__restrict__ src, char *__restrict__ dst,
                                                         int64_t bytes)
{
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t first = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    int64_t done = 0;
    if (((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15u) == 0) {
        const int64_t n = bytes / 16;
        const uint4 *s4 = reinterpret_cast<const uint4 *>(src);
        uint4 *d4 = reinterpret_cast<uint4 *>(dst);
        for (int64_t i = first; i < n; i += stride)
            d4[i] = s4[i];
        done = n * 16;
    }
    for (int64_t i = done + first; i < bytes; i += stride)
        dst[i] = src[i];
}

// Best-fit allocator over one device allocation; free ranges coalesce.
struct Arena {
    char *base = nullptr;
    size_t size = 0, used = 0, peak = 0;
    std::map<size_t, size_t> free_ranges; // offset -> length

    void reset(char *b, size_t n)
    {
        base = b;
        size = n;
        used = peak = 0;
        free_ranges.clear();
        if (n)
            free_ranges[0] = n;
    }

    bool alloc(size_t bytes, size_t &off)
    {
        bytes = round_up(std::max<size_t>(bytes, 1));
        auto best = free_ranges.end();
        for (auto it = free_ranges.begin(); it != free_ranges.end(); ++it)
            if (it->second >= bytes && (best == free_ranges.end() || it->second < best->second))
                best = it;
        if (best == free_ranges.end())
            return false;
        off = best->first;
        const size_t len = best->second;
        free_ranges.erase(best);
        if (len > bytes)
            free_ranges[off + bytes] = len - bytes;
        used += bytes;
        peak = std::max(peak, used);
        return true;
    }

    void release(size_t off, size_t bytes)
    {
        bytes = round_up(std::max<size_t>(bytes, 1));
        used -= bytes;
        auto next = free_ranges.lower_bound(off);
        size_t start = off, len = bytes;
        if (next != free_ranges.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_ranges.erase(prev);
            }
        }
        next = free_ranges.lower_bound(off + bytes);
        if (next != free_ranges.end() && next->first == off + bytes) {
            len += next->second;
            free_ranges.erase(next);
        }
        free_ranges[start] = len;
    }
};

enum ReqState { QUEUED = 0, RUNNING = 1, DONE = 2 };

struct Req {
    optigpu_request r{};
    const char *zc_src = nullptr; // device views of pinned host buffers (or null)
    char *zc_dst = nullptr;
    size_t in_bytes = 0, out_bytes = 0;
    size_t off_in = 0, off_out = 0;
    int state = QUEUED;
    double t_submit = 0, t_done = 0;
    int64_t trace_index = -1;
};

struct StreamCtx {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<uint64_t> tickets;
    // per-step batch tables: device workspace and pinned host staging
    void *d_ws = nullptr;
    size_t ws_bytes = 0;
    void *h_stage = nullptr;
    size_t stage_bytes = 0;
};

} // namespace
} // namespace optigpu

struct optigpu_server {
    std::mutex mu;
    size_t budget = 0;
    int32_t max_slots = 0;
    uint32_t flags = 0;
    int device = -1;
    void *arena_mem = nullptr;
    optigpu::Arena arena;
    std::vector<optigpu::StreamCtx> streams;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, optigpu::Req> reqs;
    uint64_t next_ticket = 1;
    int32_t running = 0;
    optigpu_server_stats stats{};
    std::vector<double> *trace_done = nullptr; // completion times by trace index (replay)
    int32_t fail_countdown = 0; // testing hook: the step launch that brings it to 0 fails
};

namespace optigpu {
namespace {

optigpu_status validate_request(const optigpu_server *sv, const optigpu_request &r, size_t &in_b, size_t &out_b)
{
    if (r.op != OPTIGPU_OP_TRANSPOSE && r.op != OPTIGPU_OP_REDUCE)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: unknown op");
    if (!dtype_valid(r.dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "server: unknown dtype");
    const size_t es = esize_of(optigpu_dtype(r.dtype));
    const int64_t cols = r.op == OPTIGPU_OP_TRANSPOSE ? r.cols : 1;
    if (r.rows < 0 || cols < 0 || (cols > 0 && r.rows > (int64_t(1) << 40) / cols))
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: bad size");
    const size_t n = size_t(r.rows) * size_t(cols);
    in_b = n * es;
    out_b = r.op == OPTIGPU_OP_TRANSPOSE ? n * es : 8;
    if ((in_b && !r.host_src) || (out_b && !r.host_dst))
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null host buffer");
    if (round_up(std::max<size_t>(in_b, 1)) + round_up(out_b) > sv->budget)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: request larger than the memory budget");
    return OPTIGPU_OK;
}

// Releases the requests of every stream whose step has finished.
optigpu_status complete_finished(optigpu_server *sv)
{
    for (StreamCtx &sc : sv->streams) {
        if (!sc.busy)
            continue;
        const cudaError_t q = cudaEventQuery(sc.done);
        if (q == cudaErrorNotReady)
            continue;
        if (q != cudaSuccess)
            return check_cuda(q, "server: step failed");
        const double t = now_s();
        for (uint64_t tk : sc.tickets) {
            Req &rq = sv->reqs[tk];
            sv->arena.release(rq.off_in, rq.in_bytes);
            sv->arena.release(rq.off_out, rq.out_bytes);
            rq.state = DONE;
            rq.t_done = t;
            if (sv->trace_done && rq.trace_index >= 0)
                (*sv->trace_done)[size_t(rq.trace_index)] = t;
            --sv->running;
            ++sv->stats.completed;
        }
        sc.tickets.clear();
        sc.busy = false;
    }
    return OPTIGPU_OK;
}

optigpu_status ensure_capacity(StreamCtx &sc, size_t ws_bytes, size_t stage_bytes)
{
    optigpu_status st;
    if (sc.ws_bytes < ws_bytes) {
        if (sc.d_ws)
            cudaFree(sc.d_ws);
        sc.d_ws = nullptr;
        sc.ws_bytes = 0;
        const size_t want = std::max<size_t>(ws_bytes * 2, size_t(1) << 20);
        if ((st = check_cuda(cudaMalloc(&sc.d_ws, want), "server: cudaMalloc(step workspace)")) != OPTIGPU_OK)
            return st;
        if ((st = check_cuda(cudaMemset(sc.d_ws, 0, want), "server: clear step workspace")) != OPTIGPU_OK)
            return st;
        sc.ws_bytes = want;
    }
    if (sc.stage_bytes < stage_bytes) {
        if (sc.h_stage)
            cudaFreeHost(sc.h_stage);
        sc.h_stage = nullptr;
        sc.stage_bytes = 0;
        const size_t want = std::max<size_t>(stage_bytes * 2, size_t(1) << 20);
        if ((st = check_cuda(cudaMallocHost(&sc.h_stage, want), "server: cudaMallocHost(stage)")) != OPTIGPU_OK)
            return st;
        sc.stage_bytes = want;
    }
    return OPTIGPU_OK;
}

// Launches the admitted tickets `adm` on `sc`.
optigpu_status launch_step(optigpu_server *sv, StreamCtx &sc, const std::vector<uint64_t> &adm)
{
    optigpu_status st = OPTIGPU_OK;
    char *base = sv->arena.base;
    for (uint64_t tk : adm) {
        const Req &rq = sv->reqs[tk];
        if (rq.in_bytes && !rq.zc_dst &&
            (st = check_cuda(cudaMemcpyAsync(base + rq.off_in, rq.r.host_src, rq.in_bytes, cudaMemcpyHostToDevice, sc.s),
                             "server: copy in")) != OPTIGPU_OK)
            return st;
    }
    if (sv->fail_countdown > 0 && --sv->fail_countdown == 0)
        return fail(OPTIGPU_ERR_CUDA, "server: injected step failure (testing hook)");
    const bool per_call = (sv->flags & OPTIGPU_SERVER_PER_CALL) != 0;
    const uint32_t rflags = sv->flags & OPTIGPU_REDUCE_COMPENSATED;
    if (per_call) {
        DeviceInfo dev;
        if ((st = current_device(dev)) != OPTIGPU_OK)
            return st;
        auto copy_range = [&](const char *src, char *dst, size_t bytes, const char *what) {
            const int64_t units = int64_t(bytes + 16 * 256 - 1) / (16 * 256);
            const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(units, int64_t(4) * dev.num_sms));
            copy_range_kernel<<<unsigned(grid), 256, 0, sc.s>>>(src, dst, int64_t(bytes));
            ++sv->stats.launches;
            return check_cuda(cudaGetLastError(), what);
        };
        for (uint64_t tk : adm) {
            const Req &rq = sv->reqs[tk];
            if (rq.zc_dst && rq.in_bytes &&
                (st = copy_range(rq.zc_src, base + rq.off_in, rq.in_bytes, "server: gather (per call)")) != OPTIGPU_OK)
                return st;
            if (rq.r.op == OPTIGPU_OP_TRANSPOSE)
                st = transpose_dispatch(base + rq.off_in, base + rq.off_out, rq.r.rows, rq.r.cols, rq.r.dtype,
                                        OPTIGPU_TRANSPOSE_AUTO, sc.s);
            else
                st = reduce_dispatch(base + rq.off_in, rq.r.rows, rq.r.dtype, base + rq.off_out, rflags, sc.s);
            if (st != OPTIGPU_OK)
                return st;
            ++sv->stats.launches;
            if (rq.zc_dst && rq.out_bytes &&
                (st = copy_range(base + rq.off_out, rq.zc_dst, rq.out_bytes, "server: scatter (per call)")) != OPTIGPU_OK)
                return st;
        }
    } else {
        std::vector<optigpu_desc> descs;
        descs.reserve(adm.size());
        for (uint64_t tk : adm) {
            const Req &rq = sv->reqs[tk];
            optigpu_desc d{};
            d.op = rq.r.op;
            d.dtype = rq.r.dtype;
            d.src = base + rq.off_in;
            d.dst = base + rq.off_out;
            d.rows = rq.r.rows;
            d.cols = rq.r.op == OPTIGPU_OP_TRANSPOSE ? rq.r.cols : 1;
            descs.push_back(d);
            if (d.op == OPTIGPU_OP_REDUCE && d.rows == 0 &&
                (st = check_cuda(cudaMemsetAsync(d.dst, 0, 8, sc.s), "server: zero sum")) != OPTIGPU_OK)
                return st;
        }
        const int config = batch_selected();
        BatchTables t;
        if ((st = batch_tables(descs.data(), int32_t(descs.size()), batch_tile(config), t)) != OPTIGPU_OK)
            return st;
        // Copy kernels' descriptors: gathers (host -> arena) then scatters.
        std::vector<CopyDesc> copies;
        int64_t gpieces = 0, spieces = 0;
        for (uint64_t tk : adm) {
            const Req &rq = sv->reqs[tk];
            if (rq.zc_dst && rq.in_bytes) {
                copies.push_back(CopyDesc{rq.zc_src, base + rq.off_in, int64_t(rq.in_bytes), gpieces});
                gpieces += (int64_t(rq.in_bytes) + kPiece - 1) / kPiece;
            }
        }
        const int32_t n_gather = int32_t(copies.size());
        for (uint64_t tk : adm) {
            const Req &rq = sv->reqs[tk];
            if (rq.zc_dst && rq.out_bytes) {
                copies.push_back(CopyDesc{base + rq.off_out, rq.zc_dst, int64_t(rq.out_bytes), spieces});
                spieces += (int64_t(rq.out_bytes) + kPiece - 1) / kPiece;
            }
        }
        const int32_t n_scatter = int32_t(copies.size()) - n_gather;
        // Workspace: the batch layout's queue, counters and tables, then the
        // step's copy list right after the tables (so that tables and list
        // go up in one copy), then the partials.
        const BatchLayout L = batch_layout(int64_t(descs.size()), t.items, t.chunks);
        const size_t table_bytes = L.off_part - L.off_inst;
        const size_t copy_bytes = sizeof(CopyDesc) * copies.size();
        const size_t off_copy = L.off_part;
        const size_t off_part = round_up(off_copy + copy_bytes);
        if ((st = ensure_capacity(sc, off_part + (L.total - L.off_part), table_bytes + copy_bytes)) != OPTIGPU_OK)
            return st;
        char *stage = static_cast<char *>(sc.h_stage);
        char *ws = static_cast<char *>(sc.d_ws);
        if (t.items > 0) {
            std::memcpy(stage, t.insts.data(), sizeof(BatchInst) * t.insts.size());
            std::memcpy(stage + (L.off_items - L.off_inst), t.item_inst.data(), sizeof(uint32_t) * t.item_inst.size());
        }
        if (!copies.empty())
            std::memcpy(stage + table_bytes, copies.data(), copy_bytes);
        if ((t.items > 0 || !copies.empty()) &&
            (st = check_cuda(cudaMemcpyAsync(ws + L.off_inst, stage, table_bytes + copy_bytes, cudaMemcpyHostToDevice,
                                             sc.s),
                             "server: copy step tables and copy list")) != OPTIGPU_OK)
            return st;
        auto *d_queue = reinterpret_cast<unsigned long long *>(ws + L.off_queue);
        auto *d_done = reinterpret_cast<unsigned *>(ws + L.off_done);
        DeviceInfo dev;
        if ((st = current_device(dev)) != OPTIGPU_OK)
            return st;
        const CopyDesc *d_copies = reinterpret_cast<const CopyDesc *>(ws + off_copy);
        // The gather kernel, when there is one, also zeroes the batch queue
        // and counters, and the batch launch then skips its reset memset.
        const bool gather_clears = n_gather > 0 && t.items > 0;
        if (n_gather > 0) {
            const int64_t grid = std::min<int64_t>(gpieces, int64_t(4) * dev.num_sms);
            copy_pieces_kernel<<<unsigned(grid), 256, 0, sc.s>>>(d_copies, n_gather, gpieces,
                                                                 gather_clears ? d_queue : nullptr, d_done,
                                                                 int32_t(descs.size()));
            if ((st = check_cuda(cudaGetLastError(), "server: gather")) != OPTIGPU_OK)
                return st;
            ++sv->stats.launches;
        }
        if (t.items > 0) {
            if ((st = batch_launch(config, reinterpret_cast<BatchInst *>(ws + L.off_inst),
                                   reinterpret_cast<uint32_t *>(ws + L.off_items), t.items, d_queue, d_done,
                                   gather_clears ? -1 : int64_t(descs.size()), ws + off_part, rflags ? 1 : 0,
                                   sc.s, nullptr, t.items == t.chunks)) != OPTIGPU_OK)
                return st;
            ++sv->stats.launches;
        }
        if (n_scatter > 0) {
            const int64_t grid = std::min<int64_t>(spieces, int64_t(4) * dev.num_sms);
            copy_pieces_kernel<<<unsigned(grid), 256, 0, sc.s>>>(d_copies + n_gather, n_scatter, spieces, nullptr,
                                                                 nullptr, 0);
            if ((st = check_cuda(cudaGetLastError(), "server: scatter")) != OPTIGPU_OK)
                return st;
            ++sv->stats.launches;
        }
    }
    for (uint64_t tk : adm) {
        const Req &rq = sv->reqs[tk];
        if (rq.out_bytes && !rq.zc_dst &&
            (st = check_cuda(cudaMemcpyAsync(rq.r.host_dst, base + rq.off_out, rq.out_bytes, cudaMemcpyDeviceToHost,
                                             sc.s),
                             "server: copy out")) != OPTIGPU_OK)
            return st;
    }
    if ((st = check_cuda(cudaEventRecord(sc.done, sc.s), "server: record step event")) != OPTIGPU_OK)
        return st;
    sc.busy = true;
    sc.tickets = adm;
    ++sv->stats.steps;
    return OPTIGPU_OK;
}

// Undoes the admission of `adm` after its launch failed part-way: waits for
// whatever of the step was already enqueued on its stream (so that no copy or
// kernel still touches the arena ranges), gives the ranges and slots back and
// puts the requests back at the head of the queue in their original order.
void rollback_step(optigpu_server *sv, StreamCtx &sc, const std::vector<uint64_t> &adm)
{
    const std::string msg = optigpu_last_error();
    if (cudaStreamSynchronize(sc.s) != cudaSuccess)
        cudaGetLastError();
    for (auto it = adm.rbegin(); it != adm.rend(); ++it) {
        Req &rq = sv->reqs[*it];
        sv->arena.release(rq.off_in, rq.in_bytes);
        sv->arena.release(rq.off_out, rq.out_bytes);
        rq.state = QUEUED;
        --sv->running;
        sv->pending.push_front(*it);
    }
    sc.tickets.clear();
    sc.busy = false;
    fail(OPTIGPU_ERR_CUDA, msg); // keep the launch's own message as the last error
}

optigpu_status step_locked(optigpu_server *sv, int32_t *launched)
{
    if (launched)
        *launched = 0;
    optigpu_status st = complete_finished(sv);
    if (st != OPTIGPU_OK)
        return st;
    const bool per_call = (sv->flags & OPTIGPU_SERVER_PER_CALL) != 0;
    for (StreamCtx &sc : sv->streams) {
        if (sc.busy)
            continue;
        if (sv->pending.empty())
            break;
        // A step takes at most its share of the slots, so that several steps
        // (on different streams) overlap when the queue is long.
        const int32_t per_step = std::max<int32_t>(1, sv->max_slots / int32_t(sv->streams.size()));
        std::vector<uint64_t> adm;
        while (!sv->pending.empty() && sv->running < sv->max_slots && int32_t(adm.size()) < per_step) {
            Req &rq = sv->reqs[sv->pending.front()];
            size_t a = 0, b = 0;
            if (!sv->arena.alloc(rq.in_bytes, a))
                break;
            if (!sv->arena.alloc(rq.out_bytes, b)) {
                sv->arena.release(a, rq.in_bytes);
                break;
            }
            rq.off_in = a;
            rq.off_out = b;
            rq.state = RUNNING;
            ++sv->running;
            adm.push_back(sv->pending.front());
            sv->pending.pop_front();
            if (per_call)
                break; // one request per stream
        }
        if (adm.empty())
            break; // out of slots or budget: wait for completions
        if ((st = launch_step(sv, sc, adm)) != OPTIGPU_OK) {
            rollback_step(sv, sc, adm);
            return st;
        }
        if (launched)
            ++*launched;
    }
    sv->stats.pending = int64_t(sv->pending.size());
    sv->stats.in_flight = sv->running;
    sv->stats.max_in_flight = std::max<int64_t>(sv->stats.max_in_flight, sv->running);
    sv->stats.bytes_in_use = int64_t(sv->arena.used);
    sv->stats.peak_bytes = int64_t(sv->arena.peak);
    return OPTIGPU_OK;
}

optigpu_status submit_locked(optigpu_server *sv, const optigpu_request &r, int64_t trace_index, uint64_t *ticket)
{
    size_t in_b = 0, out_b = 0;
    optigpu_status st = validate_request(sv, r, in_b, out_b);
    if (st != OPTIGPU_OK)
        return st;
    const uint64_t tk = sv->next_ticket++;
    Req rq;
    rq.r = r;
    rq.in_bytes = in_b;
    rq.out_bytes = out_b;
    rq.t_submit = now_s();
    const bool per_call = (sv->flags & OPTIGPU_SERVER_PER_CALL) != 0;
    const bool copy_kernels = per_call ? (sv->flags & OPTIGPU_SERVER_COPY_KERNELS) != 0
                                       : (sv->flags & OPTIGPU_SERVER_COPY_ENGINES) == 0;
    if (copy_kernels) {
        // Pinned host buffers are copied by SM copy kernels; others by the
        // copy engines.
        rq.zc_src = static_cast<const char *>(device_view_of_host(r.host_src, in_b));
        rq.zc_dst = static_cast<char *>(device_view_of_host(r.host_dst, out_b));
        if ((in_b && !rq.zc_src) || !rq.zc_dst)
            rq.zc_src = nullptr, rq.zc_dst = nullptr;
    }
    rq.trace_index = trace_index;
    sv->reqs.emplace(tk, rq);
    sv->pending.push_back(tk);
    ++sv->stats.submitted;
    if (ticket)
        *ticket = tk;
    return OPTIGPU_OK;
}

void destroy_server(optigpu_server *sv)
{
    for (StreamCtx &sc : sv->streams) {
        if (sc.s)
            cudaStreamSynchronize(sc.s);
        if (sc.done)
            cudaEventDestroy(sc.done);
        if (sc.d_ws)
            cudaFree(sc.d_ws);
        if (sc.h_stage)
            cudaFreeHost(sc.h_stage);
        if (sc.s)
            cudaStreamDestroy(sc.s);
    }
    if (sv->arena_mem)
        cudaFree(sv->arena_mem);
    delete sv;
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" {

optigpu_status optigpu_server_create(size_t mem_budget_bytes, int32_t max_slots, int32_t n_streams, uint32_t flags,
                                     optigpu_server **out)
{
    if (!out)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null output pointer");
    *out = nullptr;
    if (mem_budget_bytes < (size_t(1) << 20) || max_slots < 1 || n_streams < 1 || n_streams > 1024)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: budget >= 1 MiB, max_slots >= 1, n_streams in [1, 1024]");
    if (flags & ~(OPTIGPU_REDUCE_COMPENSATED | OPTIGPU_SERVER_PER_CALL | OPTIGPU_SERVER_COPY_ENGINES |
                  OPTIGPU_SERVER_COPY_KERNELS))
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: unknown flag bits");
    if ((flags & OPTIGPU_SERVER_COPY_ENGINES) && (flags & OPTIGPU_SERVER_COPY_KERNELS))
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: COPY_ENGINES and COPY_KERNELS exclude each other");
    optigpu_server *sv = new (std::nothrow) optigpu_server();
    if (!sv)
        return fail(OPTIGPU_ERR_OOM, "server: host allocation failed");
    sv->budget = mem_budget_bytes;
    sv->max_slots = max_slots;
    sv->flags = flags;
    cudaGetDevice(&sv->device);
    optigpu_status st = check_cuda(cudaMalloc(&sv->arena_mem, mem_budget_bytes), "server: cudaMalloc(budget)");
    if (st == OPTIGPU_OK) {
        sv->arena.reset(static_cast<char *>(sv->arena_mem), mem_budget_bytes);
        sv->streams.resize(size_t(n_streams));
        for (StreamCtx &sc : sv->streams) {
            if ((st = check_cuda(cudaStreamCreateWithFlags(&sc.s, cudaStreamNonBlocking), "server: stream")) != OPTIGPU_OK)
                break;
            if ((st = check_cuda(cudaEventCreateWithFlags(&sc.done, cudaEventDisableTiming), "server: event")) !=
                OPTIGPU_OK)
                break;
            // Step tables up to ~8 MiB on the device and 4 MiB of pinned
            // staging from the start: growing them later costs a device-wide
            // synchronisation in the middle of serving.
            if ((st = ensure_capacity(sc, size_t(4) << 20, size_t(2) << 20)) != OPTIGPU_OK)
                break;
        }
    }
    if (st != OPTIGPU_OK) {
        destroy_server(sv);
        return st;
    }
    *out = sv;
    return OPTIGPU_OK;
}

optigpu_status optigpu_server_submit(optigpu_server *sv, const optigpu_request *req, uint64_t *ticket)
{
    if (!sv || !req)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null server or request");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->max_slots > 0 && int64_t(sv->pending.size()) >= int64_t(1) << 24)
        return fail(OPTIGPU_ERR_BUSY, "server: queue full");
    return submit_locked(sv, *req, -1, ticket);
}

optigpu_status optigpu_server_step(optigpu_server *sv, int32_t *launched)
{
    optigpu::NvtxRange nvtx_range("optigpu_server_step");
    if (!sv)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    return step_locked(sv, launched);
}

optigpu_status optigpu_server_poll(optigpu_server *sv, uint64_t ticket, int32_t *done)
{
    if (!sv || !done)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    optigpu_status st = complete_finished(sv);
    if (st != OPTIGPU_OK)
        return st;
    auto it = sv->reqs.find(ticket);
    if (it == sv->reqs.end())
        return fail(OPTIGPU_ERR_NOT_FOUND, "server: unknown ticket");
    *done = it->second.state == DONE ? 1 : 0;
    if (*done)
        sv->reqs.erase(it);
    return OPTIGPU_OK;
}

optigpu_status optigpu_server_drain(optigpu_server *sv)
{
    if (!sv)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null server");
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            optigpu_status st = step_locked(sv, nullptr);
            if (st != OPTIGPU_OK)
                return st;
            if (sv->pending.empty() && sv->running == 0)
                return OPTIGPU_OK;
        }
        std::this_thread::yield();
    }
}

optigpu_status optigpu_server_get_stats(optigpu_server *sv, optigpu_server_stats *out)
{
    if (!sv || !out)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server: null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *out = sv->stats;
    out->pending = int64_t(sv->pending.size());
    out->in_flight = sv->running;
    out->bytes_in_use = int64_t(sv->arena.used);
    out->peak_bytes = int64_t(sv->arena.peak);
    return OPTIGPU_OK;
}

optigpu_status optigpu_server_replay(optigpu_server *sv, const optigpu_request *reqs, const double *arrival_s,
                                     int64_t count, double *latency_s)
{
    optigpu::NvtxRange nvtx_range("optigpu_server_replay");
    if (!sv || count < 0 || (count > 0 && (!reqs || !arrival_s || !latency_s)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "server_replay: bad arguments");
    for (int64_t i = 1; i < count; ++i)
        if (arrival_s[i] < arrival_s[i - 1])
            return fail(OPTIGPU_ERR_INVALID_ARG, "server_replay: arrival times must be non-decreasing");
    std::vector<double> done(size_t(count), -1.0);
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->trace_done = &done;
    const int64_t completed0 = sv->stats.completed;
    const double t0 = now_s();
    int64_t next = 0;
    optigpu_status st = OPTIGPU_OK;
    double prev = 0.0, max_gap = 0.0;
    while (sv->stats.completed - completed0 < count) {
        const double t = now_s() - t0;
        max_gap = std::max(max_gap, t - prev); // a host stall shows up as one long gap
        prev = t;
        while (next < count && arrival_s[next] <= t) {
            if ((st = submit_locked(sv, reqs[next], next, nullptr)) != OPTIGPU_OK)
                break;
            ++next;
        }
        if (st != OPTIGPU_OK || (st = step_locked(sv, nullptr)) != OPTIGPU_OK)
            break;
    }
    sv->trace_done = nullptr;
    sv->stats.replay_max_loop_gap_ns = int64_t(max_gap * 1e9);
    // Replayed tickets are not polled: forget every finished one.
    for (auto it = sv->reqs.begin(); it != sv->reqs.end();)
        it = (it->second.state == DONE && it->second.trace_index >= 0) ? sv->reqs.erase(it) : std::next(it);
    if (st != OPTIGPU_OK)
        return st;
    for (int64_t i = 0; i < count; ++i)
        latency_s[i] = done[size_t(i)] - (t0 + arrival_s[i]);
    return OPTIGPU_OK;
}

optigpu_status optigpu_server_inject_step_failure(optigpu_server *sv, int32_t nth)
{
    if (!sv || nth < 0)
        return fail(OPTIGPU_ERR_INVALID_ARG, "server_inject_step_failure: null server or negative count");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->fail_countdown = nth;
    return OPTIGPU_OK;
}

void optigpu_server_destroy(optigpu_server *sv)
{
    if (sv)
        destroy_server(sv);
}

} // extern "C"
