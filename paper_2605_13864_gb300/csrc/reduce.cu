// reduce.cu -- tree-based sum reduction, *out = sum of src[0 .. n)
// (thesis arxiv 2605.13864, Listing 2.1, Sec. 2.1: reduce_sum(N, A); the
// partial-sum form of Listing 2.2, Sec. 2.2.1; the tree of Sec. 7.2).
//
// One kernel does both passes:
//
//  pass 1  The input is cut into chunks of CHUNK = 16384 elements (the role of
//          Listing 2.2's 128-element tiles).  CTAs of 256 threads take chunks
//          c = blockIdx.x, blockIdx.x + gridDim.x, ...; inside a chunk thread t
//          owns the 16-byte vectors t, t + 256, t + 512, ... and keeps a
//          register accumulator across them (the `mySum` register accumulator
//          whose absence costs the thesis's generated kernel ~50 GB/s,
//          Sec. 7.2).  The elements of one vector are added in a fixed
//          pairwise tree.  Threads are then combined by warp shuffles
//          (butterfly, 5 steps) and the 8 warp sums by a second shuffle tree,
//          giving one partial per chunk in partials[c]:
//            int32 input   int64 everywhere (exact);
//            float input   FP32 sums, widened to FP64 for the partial;
//            compensated   FP32 Neumaier (s, c) pairs per thread, pairs
//                          combined with Knuth's TwoSum, partial = s + c in
//                          FP64.
//  pass 2  The last CTA to finish (an integer completion counter; no float
//          atomics) sums partials[0 .. num_chunks) in FP64 / int64 in a
//          fixed order -- per-thread strided sequential sums, then the same
//          shuffle trees -- writes *out and resets the counter.
//
// The chunk partition, the per-chunk order and the final order depend only
// on (n, dtype, flags): not on the grid size, so results are bit-identical
// from run to run and between this entry point and the batched kernel.
#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"
#include "ptx.cuh"
#include "reduce_core.cuh"

namespace optigpu {
namespace {

// Two forms of one kernel, the same bits (ReduceCore's MAX_BATCH changes
// only when loads are issued):
//   WAVE = false  8 loads in flight per thread, at most 48 registers (5 CTAs
//                 per SM): the throughput form for large sums;
//   WAVE = true   4 loads in flight, at most 32 registers, so 8 CTAs fit on
//                 an SM -- 1216 CTAs on 152 SMs, and a sum of up to that many
//                 chunks (2^24 elements is 1024) starts all its chunks at
//                 once instead of running a second, partial wave.
template <int DT, bool COMP, bool WAVE>
__global__ void __launch_bounds__(kReduceThreads, WAVE ? 8 : 5)
reduce_sum_kernel(const void *__restrict__ src, int64_t n, int vec_ok, void *partials,
                  unsigned *counter, void *out, int64_t num_chunks)
{
    using Core = ReduceCore<DT, COMP, WAVE ? 4 : 8>;
    __shared__ typename Core::Shared sh;
    __shared__ int s_last;
    // Launched with programmatic stream serialisation: wait until the
    // previous kernel on the stream has finished and its writes are visible
    // (it may be the previous sum, on the same workspace), before touching
    // memory; then let the next kernel on the stream be launched, so that its
    // launch overlaps this sum's tail.  Both are no-ops for a plain launch.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    for (int64_t c = blockIdx.x; c < num_chunks; c += gridDim.x) {
        const auto part = Core::chunk_partial(src, n, c, vec_ok != 0, sh);
        if (threadIdx.x == 0)
            Core::store_partial(partials, c, part);
    }
    // Completion: thread 0 wrote every partial of this CTA; it makes them
    // visible GPU-wide, then counts the CTA; the last CTA runs the final
    // combine.
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = (atomicAdd(counter, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    Core::final_combine(partials, num_chunks, out, sh);
    if (threadIdx.x == 0)
        *counter = 0u;
}

// CTAs per SM of the persistent grid for each configuration (0 = as many as
// fit); the partition into chunks, and so the result, does not depend on it.
constexpr int kReduceCtasPerSm[] = {0, 2, 3, 4, 6};
constexpr const char *kReduceConfigNames[] = {"reduce ctas/SM=max", "reduce ctas/SM=2", "reduce ctas/SM=3",
                                              "reduce ctas/SM=4", "reduce ctas/SM=6"};
std::atomic<int> g_reduce_choice{0};

// Partials only, for a band of a larger input: chunk c of the band is
// chunk (chunk_base + c) of the whole vector, and band_src starts at that
// chunk's first element, so each partial is the one the single-pass kernel
// computes.
template <int DT, bool COMP>
__global__ void __launch_bounds__(kReduceThreads)
reduce_band_kernel(const void *__restrict__ band_src, int64_t band_n, int vec_ok, void *partials, int64_t chunk_base,
                   int64_t band_chunks)
{
    using Core = ReduceCore<DT, COMP>;
    __shared__ typename Core::Shared sh;
    for (int64_t c = blockIdx.x; c < band_chunks; c += gridDim.x) {
        const auto part = Core::chunk_partial(band_src, band_n, c, vec_ok != 0, sh);
        if (threadIdx.x == 0)
            Core::store_partial(partials, chunk_base + c, part);
    }
}

// The final combine alone (one CTA).
template <int DT, bool COMP>
__global__ void __launch_bounds__(kReduceThreads) reduce_final_kernel(const void *partials, int64_t count, void *out)
{
    using Core = ReduceCore<DT, COMP>;
    __shared__ typename Core::Shared sh;
    Core::final_combine(partials, count, out, sh);
}

struct KernelFacts {
    bool ready = false;
    int ctas_per_sm = 0;
};
std::mutex g_mu;
KernelFacts g_facts[64][4][2][2];

// Resident CTAs per SM of reduce_sum_kernel<DT, COMP, WAVE> (occupancy,
// looked up once per device and kernel).
template <int DT, bool COMP, bool WAVE>
optigpu_status resident_ctas(const DeviceInfo &dev, int *ctas_per_sm)
{
    std::lock_guard<std::mutex> lk(g_mu);
    KernelFacts &f = g_facts[dev.device & 63][DT][COMP ? 1 : 0][WAVE ? 1 : 0];
    if (!f.ready) {
        const void *fn = reinterpret_cast<const void *>(&reduce_sum_kernel<DT, COMP, WAVE>);
        int k = 0;
        optigpu_status st = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, fn, kReduceThreads, 0),
                                       "cudaOccupancyMaxActiveBlocksPerMultiprocessor(reduce)");
        if (st != OPTIGPU_OK)
            return st;
        f.ctas_per_sm = std::max(k, 1);
        f.ready = true;
    }
    *ctas_per_sm = f.ctas_per_sm;
    return OPTIGPU_OK;
}

// Form and persistent grid of the sum for `num_chunks` chunks on the current
// device.  The one-wave form is taken when all chunks fit in one wave of it;
// otherwise the throughput form, with its resident CTAs per SM capped by the
// tuned configuration.  Neither choice changes the result.
template <int DT, bool COMP>
optigpu_status persistent_grid(int64_t num_chunks, int64_t *grid, bool *wave)
{
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    int per_sm = 1;
    if ((st = resident_ctas<DT, COMP, true>(dev, &per_sm)) != OPTIGPU_OK)
        return st;
    if (num_chunks <= int64_t(per_sm) * dev.num_sms) {
        *wave = true;
        *grid = num_chunks;
        return OPTIGPU_OK;
    }
    if ((st = resident_ctas<DT, COMP, false>(dev, &per_sm)) != OPTIGPU_OK)
        return st;
    const int cap = kReduceCtasPerSm[g_reduce_choice.load()];
    if (cap > 0)
        per_sm = std::min(per_sm, cap);
    *wave = false;
    *grid = std::min<int64_t>(num_chunks, int64_t(per_sm) * dev.num_sms);
    return OPTIGPU_OK;
}

// Programmatic dependent launch: a sum queued right behind another kernel
// may be launched while that kernel finishes (the kernel waits for it before
// touching memory), which takes the launch latency off back-to-back sums.
template <int DT, bool COMP>
cudaError_t launch_sum_kernel(bool wave, int64_t grid, cudaStream_t stream, const void *src, int64_t n, int vec_ok,
                              void *partials, unsigned *counter, void *out, int64_t num_chunks)
{
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(kReduceThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (wave)
        return cudaLaunchKernelEx(&cfg, reduce_sum_kernel<DT, COMP, true>, src, n, vec_ok, partials, counter, out,
                                  num_chunks);
    return cudaLaunchKernelEx(&cfg, reduce_sum_kernel<DT, COMP, false>, src, n, vec_ok, partials, counter, out,
                              num_chunks);
}

template <int DT, bool COMP>
optigpu_status launch(const void *src, int64_t n, void *out, cudaStream_t stream)
{
    const int64_t num_chunks = (n + kReduceChunk - 1) / kReduceChunk;
    int64_t grid = 0;
    bool wave = false;
    optigpu_status st = persistent_grid<DT, COMP>(num_chunks, &grid, &wave);
    if (st != OPTIGPU_OK)
        return st;
    void *ws = nullptr;
    const size_t bytes = kReduceCounterBytes + size_t(num_chunks) * 8;
    if ((st = stream_workspace(stream, bytes, &ws)) != OPTIGPU_OK)
        return st;
    unsigned *counter = static_cast<unsigned *>(ws);
    void *partials = static_cast<char *>(ws) + kReduceCounterBytes;
    const int vec_ok = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 ? 1 : 0;
    return check_cuda(launch_sum_kernel<DT, COMP>(wave, grid, stream, src, n, vec_ok, partials, counter, out,
                                                  num_chunks),
                      "launch reduce");
}

template <int DT, bool COMP>
optigpu_status launch_band(const void *band_src, int64_t band_n, void *partials, int64_t chunk_base,
                           cudaStream_t stream)
{
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    const int64_t chunks = (band_n + kReduceChunk - 1) / kReduceChunk;
    const int64_t grid = std::min<int64_t>(chunks, int64_t(8) * dev.num_sms);
    const int vec_ok = (reinterpret_cast<uintptr_t>(band_src) & 15u) == 0 ? 1 : 0;
    reduce_band_kernel<DT, COMP><<<unsigned(std::max<int64_t>(grid, 1)), kReduceThreads, 0, stream>>>(
        band_src, band_n, vec_ok, partials, chunk_base, chunks);
    return check_cuda(cudaGetLastError(), "launch reduce band");
}

template <int DT, bool COMP>
optigpu_status launch_final(const void *partials, int64_t count, void *out, cudaStream_t stream)
{
    reduce_final_kernel<DT, COMP><<<1, kReduceThreads, 0, stream>>>(partials, count, out);
    return check_cuda(cudaGetLastError(), "launch reduce final");
}

} // namespace

optigpu_status reduce_band(const void *band_src, int64_t band_n, int dtype, uint32_t flags, void *partials,
                           int64_t chunk_base, cudaStream_t stream)
{
    const bool comp = (flags & OPTIGPU_REDUCE_COMPENSATED) != 0;
    switch (dtype) {
    case OPTIGPU_INT32: return launch_band<OPTIGPU_INT32, false>(band_src, band_n, partials, chunk_base, stream);
    case OPTIGPU_FLOAT32:
        return comp ? launch_band<OPTIGPU_FLOAT32, true>(band_src, band_n, partials, chunk_base, stream)
                    : launch_band<OPTIGPU_FLOAT32, false>(band_src, band_n, partials, chunk_base, stream);
    case OPTIGPU_BFLOAT16:
        return comp ? launch_band<OPTIGPU_BFLOAT16, true>(band_src, band_n, partials, chunk_base, stream)
                    : launch_band<OPTIGPU_BFLOAT16, false>(band_src, band_n, partials, chunk_base, stream);
    default:
        return comp ? launch_band<OPTIGPU_FLOAT16, true>(band_src, band_n, partials, chunk_base, stream)
                    : launch_band<OPTIGPU_FLOAT16, false>(band_src, band_n, partials, chunk_base, stream);
    }
}

optigpu_status reduce_final(const void *partials, int64_t count, int dtype, uint32_t flags, void *out,
                            cudaStream_t stream)
{
    const bool comp = (flags & OPTIGPU_REDUCE_COMPENSATED) != 0;
    switch (dtype) {
    case OPTIGPU_INT32: return launch_final<OPTIGPU_INT32, false>(partials, count, out, stream);
    case OPTIGPU_FLOAT32:
        return comp ? launch_final<OPTIGPU_FLOAT32, true>(partials, count, out, stream)
                    : launch_final<OPTIGPU_FLOAT32, false>(partials, count, out, stream);
    case OPTIGPU_BFLOAT16:
        return comp ? launch_final<OPTIGPU_BFLOAT16, true>(partials, count, out, stream)
                    : launch_final<OPTIGPU_BFLOAT16, false>(partials, count, out, stream);
    default:
        return comp ? launch_final<OPTIGPU_FLOAT16, true>(partials, count, out, stream)
                    : launch_final<OPTIGPU_FLOAT16, false>(partials, count, out, stream);
    }
}

int reduce_num_configs() { return int(sizeof(kReduceCtasPerSm) / sizeof(kReduceCtasPerSm[0])); }

const char *reduce_config_name(int config)
{
    return (config >= 0 && config < reduce_num_configs()) ? kReduceConfigNames[config] : nullptr;
}

int reduce_selected() { return g_reduce_choice.load(); }

void reduce_select(int config) { g_reduce_choice.store(config); }

optigpu_status reduce_dispatch(const void *src, int64_t n, int dtype, void *out, uint32_t flags,
                               cudaStream_t stream)
{
    if (!dtype_valid(dtype))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "reduce: unknown dtype " + std::to_string(dtype));
    if (flags & ~OPTIGPU_REDUCE_COMPENSATED)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: unknown flag bits");
    if (n < 0 || n > (int64_t(1) << 62))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: n out of range");
    if (!out)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: null out");
    if (n > 0 && !src)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: null src");
    if (n > 0 && reinterpret_cast<uintptr_t>(src) % esize_of(optigpu_dtype(dtype)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: src not aligned to the element size");
    if (reinterpret_cast<uintptr_t>(out) % 8)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce: out not 8-byte aligned");
    if (n == 0)
        return check_cuda(cudaMemsetAsync(out, 0, 8, stream), "reduce: write 0");
    const bool comp = (flags & OPTIGPU_REDUCE_COMPENSATED) != 0;
    switch (dtype) {
    case OPTIGPU_INT32: return launch<OPTIGPU_INT32, false>(src, n, out, stream);
    case OPTIGPU_FLOAT32:
        return comp ? launch<OPTIGPU_FLOAT32, true>(src, n, out, stream)
                    : launch<OPTIGPU_FLOAT32, false>(src, n, out, stream);
    case OPTIGPU_BFLOAT16:
        return comp ? launch<OPTIGPU_BFLOAT16, true>(src, n, out, stream)
                    : launch<OPTIGPU_BFLOAT16, false>(src, n, out, stream);
    default:
        return comp ? launch<OPTIGPU_FLOAT16, true>(src, n, out, stream)
                    : launch<OPTIGPU_FLOAT16, false>(src, n, out, stream);
    }
}

} // namespace optigpu

using namespace optigpu;

extern "C" {

optigpu_status optigpu_reduce_sum(const void *src, int64_t n, optigpu_dtype dtype, void *out,
                                  optigpu_stream_t stream)
{
    return reduce_dispatch(src, n, int(dtype), out, OPTIGPU_REDUCE_PLAIN, static_cast<cudaStream_t>(stream));
}

optigpu_status optigpu_reduce_sum_ex(const void *src, int64_t n, optigpu_dtype dtype, void *out,
                                     uint32_t flags, optigpu_stream_t stream)
{
    optigpu::NvtxRange nvtx_range("optigpu_reduce_sum_ex");
    return reduce_dispatch(src, n, int(dtype), out, flags, static_cast<cudaStream_t>(stream));
}

optigpu_status optigpu_reduce_reserve(int64_t n, optigpu_stream_t stream)
{
    if (n < 0 || n > (int64_t(1) << 62))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_reserve: n out of range");
    const int64_t num_chunks = (n + kReduceChunk - 1) / kReduceChunk;
    void *ws = nullptr;
    return stream_workspace(static_cast<cudaStream_t>(stream), kReduceCounterBytes + size_t(num_chunks) * 8, &ws);
}

} // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot let a library call cudaMalloc: a host application that
// owns all device memory through its own pool and forbids side allocations,
// a latency-critical loop that must not hit the driver's allocator (which can
// synchronise the device) after start-up, or a process running close to a
// hard device-memory budget.  optigpu_reduce_sum_noalloc serves them.  It
// runs the same kernel as optigpu_reduce_sum_ex, but its partials and its
// completion counter live in the fixed array below, which the CUDA runtime
// places in every device's global memory when this module is loaded there,
// and which stays there until the process exits.  The call itself allocates
// nothing.  The first call on a device looks up the array's address (make it
// before any stream capture).  All calls share the array, so calls whose
// kernels overlap on the GPU race; the limit is 2^29 elements.
// ---------------------------------------------------------------------------

namespace optigpu {
namespace {

// Up to 32768 chunk partials (256 KiB): n <= 32768 * 16384 = 2^29 elements.
constexpr int64_t kNoAllocMaxChunks = 32768;
constexpr size_t kNoAllocScratchBytes = kReduceCounterBytes + size_t(kNoAllocMaxChunks) * 8;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
std::map<int, void *> g_noalloc_addr; // device -> device address of g_noalloc_scratch

// Device address of the scratch array on the current device.  In host code
// the array's name is only a host-side handle, so the address is looked up
// once per device, with that device current.
optigpu_status noalloc_scratch(void **addr)
{
    int dev = -1;
    optigpu_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != OPTIGPU_OK)
        return st;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it == g_noalloc_addr.end()) {
        void *p = nullptr;
        if ((st = check_cuda(cudaGetSymbolAddress(&p, g_noalloc_scratch),
                             "cudaGetSymbolAddress(reduce scratch)")) != OPTIGPU_OK)
            return st;
        it = g_noalloc_addr.emplace(dev, p).first;
    }
    *addr = it->second;
    return OPTIGPU_OK;
}

} // namespace

// Drops the looked-up address of the scratch array on `device` (after
// cudaDeviceReset the module is loaded again and the array may move); the
// next call on that device looks it up afresh.
void noalloc_forget_device(int device)
{
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    g_noalloc_addr.erase(device);
}

namespace {

template <int DT, bool COMP>
optigpu_status launch_noalloc(const void *src, int64_t n, void *out, cudaStream_t stream)
{
    const int64_t num_chunks = (n + kReduceChunk - 1) / kReduceChunk;
    if (num_chunks > kNoAllocMaxChunks)
        return fail(OPTIGPU_ERR_INVALID_ARG,
                    "reduce_sum_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                        std::to_string(kNoAllocMaxChunks * kReduceChunk) + " elements");
    void *scratch = nullptr;
    optigpu_status st = noalloc_scratch(&scratch);
    if (st != OPTIGPU_OK)
        return st;
    // The same kernel form and grid as optigpu_reduce_sum_ex (the result
    // depends on neither; the occupancy is looked up once per device).
    int64_t grid = 0;
    bool wave = false;
    if ((st = persistent_grid<DT, COMP>(num_chunks, &grid, &wave)) != OPTIGPU_OK)
        return st;
    unsigned *counter = static_cast<unsigned *>(scratch);
    void *partials = static_cast<char *>(scratch) + kReduceCounterBytes;
    // The array keeps whatever the previous call left; the counter must start
    // at zero (the partials are all rewritten).
    if ((st = check_cuda(cudaMemsetAsync(counter, 0, sizeof(unsigned), stream),
                         "reduce_sum_noalloc: clear counter")) != OPTIGPU_OK)
        return st;
    const int vec_ok = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 ? 1 : 0;
    return check_cuda(launch_sum_kernel<DT, COMP>(wave, grid, stream, src, n, vec_ok, partials, counter, out,
                                                  num_chunks),
                      "launch reduce (noalloc)");
}

} // namespace
} // namespace optigpu

extern "C" optigpu_status optigpu_reduce_sum_noalloc(const void *src, int64_t n, optigpu_dtype dtype, void *out,
                                                     uint32_t flags, optigpu_stream_t stream)
{
    using namespace optigpu;
    const int dt = int(dtype);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!dtype_valid(dt))
        return fail(OPTIGPU_ERR_UNSUPPORTED_DTYPE, "reduce_sum_noalloc: unknown dtype " + std::to_string(dt));
    if (flags & ~OPTIGPU_REDUCE_COMPENSATED)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_sum_noalloc: unknown flag bits");
    if (n < 0 || n > (int64_t(1) << 62))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_sum_noalloc: n out of range");
    if (!out || reinterpret_cast<uintptr_t>(out) % 8)
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_sum_noalloc: out must be a non-null 8-byte aligned pointer");
    if (n > 0 && (!src || reinterpret_cast<uintptr_t>(src) % esize_of(dtype)))
        return fail(OPTIGPU_ERR_INVALID_ARG, "reduce_sum_noalloc: src must be non-null and element-aligned");
    if ((n + kReduceChunk - 1) / kReduceChunk > kNoAllocMaxChunks)
        return fail(OPTIGPU_ERR_INVALID_ARG,
                    "reduce_sum_noalloc: n = " + std::to_string(n) + " exceeds the fixed scratch limit of " +
                        std::to_string(kNoAllocMaxChunks * kReduceChunk) + " elements");
    if (n == 0)
        return check_cuda(cudaMemsetAsync(out, 0, 8, s), "reduce_sum_noalloc: write 0");
    const bool comp = (flags & OPTIGPU_REDUCE_COMPENSATED) != 0;
    switch (dt) {
    case OPTIGPU_INT32: return launch_noalloc<OPTIGPU_INT32, false>(src, n, out, s);
    case OPTIGPU_FLOAT32:
        return comp ? launch_noalloc<OPTIGPU_FLOAT32, true>(src, n, out, s)
                    : launch_noalloc<OPTIGPU_FLOAT32, false>(src, n, out, s);
    case OPTIGPU_BFLOAT16:
        return comp ? launch_noalloc<OPTIGPU_BFLOAT16, true>(src, n, out, s)
                    : launch_noalloc<OPTIGPU_BFLOAT16, false>(src, n, out, s);
    default:
        return comp ? launch_noalloc<OPTIGPU_FLOAT16, true>(src, n, out, s)
                    : launch_noalloc<OPTIGPU_FLOAT16, false>(src, n, out, s);
    }
}
