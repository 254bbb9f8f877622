// runtime.cu -- host runtime of the library: status strings, the per-thread
// last-error text, per-device facts, the device status word that kernels set
// when a bounded wait gives up, per-stream workspaces, and the TMA descriptor
// encoder (cuTensorMapEncodeTiled fetched through the runtime's driver entry
// point, so the library does not link libcuda directly).
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "internal.h"

namespace optigpu {

// One status word per device; kernels OR DEV_ERR_* bits into it.
__device__ unsigned g_device_status;

namespace {

thread_local std::string t_last_error;

std::mutex g_mu;
std::map<int, DeviceInfo> g_devices;

struct Workspace {
    void *ptr = nullptr;
    size_t bytes = 0;
};
struct WsKey {
    int device;
    cudaStream_t stream;
    int slot;
    bool operator<(const WsKey &o) const
    {
        if (device != o.device)
            return device < o.device;
        if (stream != o.stream)
            return stream < o.stream;
        return slot < o.slot;
    }
};
std::map<WsKey, Workspace> g_workspaces;
// Buffers replaced by larger ones.  A CUDA graph captured while one of them
// was current keeps its address, so they stay allocated until
// optigpu_release_workspaces() (device -> pointers).
std::multimap<int, void *> g_retired;

uint64_t g_wait_limit_ns = 0;

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn g_encode = nullptr;

} // namespace

optigpu_status fail(optigpu_status st, const std::string &msg)
{
    t_last_error = msg;
    return st;
}

optigpu_status check_cuda(cudaError_t err, const char *what)
{
    if (err == cudaSuccess)
        return OPTIGPU_OK;
    std::string msg = std::string(what) + ": " + cudaGetErrorName(err) + " (" +
                      cudaGetErrorString(err) + ")";
    if (err == cudaErrorMemoryAllocation)
        return fail(OPTIGPU_ERR_OOM, msg);
    return fail(OPTIGPU_ERR_CUDA, msg);
}

optigpu_status current_device(DeviceInfo &out)
{
    int dev = -1;
    optigpu_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != OPTIGPU_OK)
        return st;
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_devices.find(dev);
    if (it != g_devices.end()) {
        out = it->second;
        return OPTIGPU_OK;
    }
    DeviceInfo info;
    info.device = dev;
    if ((st = check_cuda(cudaDeviceGetAttribute(&info.num_sms, cudaDevAttrMultiProcessorCount, dev),
                         "cudaDeviceGetAttribute(SMs)")) != OPTIGPU_OK)
        return st;
    int smem = 0;
    if ((st = check_cuda(cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev),
                         "cudaDeviceGetAttribute(smem)")) != OPTIGPU_OK)
        return st;
    info.max_smem_optin = static_cast<size_t>(smem);
    void *word = nullptr;
    if ((st = check_cuda(cudaGetSymbolAddress(&word, g_device_status),
                         "cudaGetSymbolAddress(status word)")) != OPTIGPU_OK)
        return st;
    info.status_word = static_cast<unsigned *>(word);
    g_devices[dev] = info;
    out = info;
    return OPTIGPU_OK;
}

uint64_t wait_limit_ns()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_wait_limit_ns == 0) {
        const char *env = std::getenv("OPTIGPU_WAIT_LIMIT_NS");
        unsigned long long v = env ? std::strtoull(env, nullptr, 10) : 0ull;
        g_wait_limit_ns = v ? v : 2000000000ull;
    }
    return g_wait_limit_ns;
}

optigpu_status stream_workspace(cudaStream_t stream, size_t bytes, void **ptr, int slot)
{
    int dev = -1;
    optigpu_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != OPTIGPU_OK)
        return st;
    std::lock_guard<std::mutex> lk(g_mu);
    Workspace &ws = g_workspaces[WsKey{dev, stream, slot}];
    if (ws.bytes < bytes) {
        size_t want = bytes < (size_t(1) << 16) ? (size_t(1) << 16) : bytes + bytes / 2;
        void *p = nullptr;
        if ((st = check_cuda(cudaMalloc(&p, want), "cudaMalloc(workspace)")) != OPTIGPU_OK)
            return st;
        // Zero once: counters in the workspace start at 0 and every kernel
        // that uses one leaves it at 0 when it finishes.
        if ((st = check_cuda(cudaMemsetAsync(p, 0, want, stream), "cudaMemsetAsync(workspace)")) != OPTIGPU_OK) {
            cudaFree(p);
            return st;
        }
        // The old buffer is retired, not freed: work queued on `stream` and
        // graphs captured from it may still use it.
        if (ws.ptr)
            g_retired.emplace(dev, ws.ptr);
        ws.ptr = p;
        ws.bytes = want;
    }
    *ptr = ws.ptr;
    return OPTIGPU_OK;
}

void *device_view_of_host(const void *p, size_t bytes)
{
    if (!p || bytes == 0)
        return nullptr;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || !a.devicePointer)
        return nullptr;
    const char *last = static_cast<const char *>(p) + bytes - 1;
    cudaPointerAttributes b{};
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (b.type != cudaMemoryTypeHost ||
        static_cast<char *>(b.devicePointer) != static_cast<char *>(a.devicePointer) + bytes - 1)
        return nullptr;
    return a.devicePointer;
}

namespace {
optigpu_status encode_entry();
} // namespace

optigpu_status encode_tensor_map_3d(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                    uint64_t dim0, uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes,
                                    uint64_t stride2_bytes, uint32_t box0, uint32_t box1)
{
    return encode_tensor_map_3d_swizzled(map, base, type, dim0, dim1, dim2, stride1_bytes, stride2_bytes, box0,
                                         box1, CU_TENSOR_MAP_SWIZZLE_NONE);
}

optigpu_status encode_tensor_map_3d_swizzled(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                             uint64_t dim0, uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes,
                                             uint64_t stride2_bytes, uint32_t box0, uint32_t box1,
                                             CUtensorMapSwizzle swizzle)
{
    optigpu_status st = encode_entry();
    if (st != OPTIGPU_OK)
        return st;
    const cuuint64_t dims[3] = {dim0, dim1, dim2};
    const cuuint64_t strides[2] = {stride1_bytes, stride2_bytes};
    const cuuint32_t box[3] = {box0, box1, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = g_encode(map, type, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(OPTIGPU_ERR_CUDA, "cuTensorMapEncodeTiled (3-D) failed with CUresult " + std::to_string(int(r)));
    return OPTIGPU_OK;
}

namespace {
optigpu_status encode_entry()
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
            return fail(OPTIGPU_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
        g_encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    return OPTIGPU_OK;
}
} // namespace

optigpu_status encode_tensor_map_2d(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                    uint64_t dim0, uint64_t dim1, uint64_t stride1_bytes,
                                    uint32_t box0, uint32_t box1, CUtensorMapSwizzle swizzle)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_encode) {
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q{};
            cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                             cudaEnableDefault, &q);
            if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn)
                return fail(OPTIGPU_ERR_CUDA, "cuTensorMapEncodeTiled entry point not available");
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        }
    }
    const cuuint64_t dims[2] = {dim0, dim1};
    const cuuint64_t strides[1] = {stride1_bytes};
    const cuuint32_t box[2] = {box0, box1};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = g_encode(map, type, 2, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(OPTIGPU_ERR_CUDA, "cuTensorMapEncodeTiled failed with CUresult " + std::to_string(int(r)));
    return OPTIGPU_OK;
}

} // namespace optigpu

using namespace optigpu;

extern "C" {

const char *optigpu_status_string(optigpu_status s)
{
    switch (s) {
    case OPTIGPU_OK: return "ok";
    case OPTIGPU_ERR_INVALID_ARG: return "invalid argument";
    case OPTIGPU_ERR_UNSUPPORTED_DTYPE: return "unsupported dtype";
    case OPTIGPU_ERR_OVERLAP: return "source and destination overlap";
    case OPTIGPU_ERR_CUDA: return "CUDA error";
    case OPTIGPU_ERR_OOM: return "out of device memory";
    case OPTIGPU_ERR_TIMEOUT: return "device-side wait timed out";
    case OPTIGPU_ERR_BUSY: return "busy: no slot or memory budget available";
    case OPTIGPU_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

const char *optigpu_last_error(void) { return t_last_error.c_str(); }

int optigpu_version(void) { return OPTIGPU_VERSION; }

void optigpu_set_wait_limit_ns(uint64_t ns)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_wait_limit_ns = ns ? ns : 2000000000ull;
}

optigpu_status optigpu_stream_status(optigpu_stream_t stream)
{
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    optigpu_status st = check_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (st != OPTIGPU_OK)
        return st;
    DeviceInfo dev;
    if ((st = current_device(dev)) != OPTIGPU_OK)
        return st;
    unsigned word = 0;
    if ((st = check_cuda(cudaMemcpyFromSymbol(&word, g_device_status, sizeof word),
                         "read device status word")) != OPTIGPU_OK)
        return st;
    if (word != 0) {
        unsigned zero = 0;
        cudaMemcpyToSymbol(g_device_status, &zero, sizeof zero);
        if (word & DEV_ERR_WAIT_TIMEOUT)
            return fail(OPTIGPU_ERR_TIMEOUT, "a device-side wait exceeded its limit");
        return fail(OPTIGPU_ERR_CUDA, "device status word = " + std::to_string(word));
    }
    return OPTIGPU_OK;
}

optigpu_status optigpu_release_workspaces(void)
{
    int dev = -1;
    optigpu_status st = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (st != OPTIGPU_OK)
        return st;
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto it = g_workspaces.begin(); it != g_workspaces.end();) {
        if (it->first.device == dev) {
            cudaFree(it->second.ptr);
            it = g_workspaces.erase(it);
        } else {
            ++it;
        }
    }
    auto range = g_retired.equal_range(dev);
    for (auto it = range.first; it != range.second; ++it)
        cudaFree(it->second);
    g_retired.erase(range.first, range.second);
    // Cached device addresses of module globals are looked up again on next
    // use (they move if the device was reset).
    g_devices.erase(dev);
    noalloc_forget_device(dev);
    return OPTIGPU_OK;
}

} // extern "C"
