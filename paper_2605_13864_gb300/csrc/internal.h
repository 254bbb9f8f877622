// internal.h -- host-runtime pieces shared by the library's translation units:
// error recording, per-device facts, per-stream workspaces, the TMA
// descriptor encoder and the device status word.  Not part of the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/optigpu.h"

namespace optigpu {

// NVTX range around a public entry point: a named span in Nsight timelines,
// a pointer test when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


// Codes written to the device status word by kernels (bit flags).
enum : unsigned {
    DEV_ERR_WAIT_TIMEOUT = 1u,   // a bounded mbarrier / flag wait gave up
    DEV_ERR_BAD_DESCRIPTOR = 2u, // a kernel met a work item it cannot handle
};

// Records `msg` as the calling thread's last error and returns `st`.
optigpu_status fail(optigpu_status st, const std::string &msg);

// Checks a CUDA runtime result; on failure records the message and returns
// OPTIGPU_ERR_CUDA (OPTIGPU_ERR_OOM for allocation failures).
optigpu_status check_cuda(cudaError_t err, const char *what);

inline size_t esize_of(optigpu_dtype dt)
{
    return (dt == OPTIGPU_BFLOAT16 || dt == OPTIGPU_FLOAT16) ? 2 : 4;
}

inline bool dtype_valid(int dt) { return dt >= OPTIGPU_INT32 && dt <= OPTIGPU_FLOAT16; }

struct DeviceInfo {
    int device = -1;
    int num_sms = 0;
    size_t max_smem_optin = 0;
    unsigned *status_word = nullptr; // device address of the status word
};

// Facts about the current device (cached per device).
optigpu_status current_device(DeviceInfo &out);

// Device-side wait limit handed to kernels that spin (ns).
uint64_t wait_limit_ns();

// A per-(device, stream) scratch buffer.  A later call on the same stream
// that asks for more bytes gets a new, larger buffer; the old one is retired
// (kept allocated), so kernels still queued and CUDA graphs captured with it
// keep valid memory.  Every buffer, current or retired, stays allocated until
// optigpu_release_workspaces() runs.  A new buffer is cleared to zero (on
// `stream`), so counters kept in it start at 0.
// `slot` separates workspaces with different layouts on one stream (0: the
// single-call sum; 1: segmented sums).
optigpu_status stream_workspace(cudaStream_t stream, size_t bytes, void **ptr, int slot = 0);

// Device address of host memory [p, p + bytes) when it is page-locked and
// mapped for the device (checked at both ends of the range), else nullptr.
// Kernels may then read and write it directly (over NVLink-C2C on GB300).
void *device_view_of_host(const void *p, size_t bytes);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no
// shared-memory swizzle unless one is given).
optigpu_status encode_tensor_map_2d(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                    uint64_t dim0, uint64_t dim1, uint64_t stride1_bytes,
                                    uint32_t box0, uint32_t box1,
                                    CUtensorMapSwizzle swizzle = CU_TENSOR_MAP_SWIZZLE_NONE);
// Same with a third dimension (dim2, stride2_bytes) and a box depth of 1.
optigpu_status encode_tensor_map_3d(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                    uint64_t dim0, uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes,
                                    uint64_t stride2_bytes, uint32_t box0, uint32_t box1);
// Same with a chosen shared-memory swizzle (the 3-D form above uses none).
optigpu_status encode_tensor_map_3d_swizzled(CUtensorMap *map, void *base, CUtensorMapDataType type,
                                             uint64_t dim0, uint64_t dim1, uint64_t dim2, uint64_t stride1_bytes,
                                             uint64_t stride2_bytes, uint32_t box0, uint32_t box1,
                                             CUtensorMapSwizzle swizzle);

// Transpose configurations: indices 0 .. n-2 are TMA kernels, n-1 is tile32.
int transpose_num_configs(size_t esize);
const char *transpose_config_name(size_t esize, int config);
int transpose_selected(size_t esize);
void transpose_select(size_t esize, int config);
void transpose_set_group_rows(int g);
int transpose_group_rows();
optigpu_status transpose_launch_config(const void *src, void *dst, int64_t rows, int64_t cols, size_t esize,
                                       int config, cudaStream_t stream);

// Reduction configurations: CTAs per SM of the persistent grid (0 = as many
// as fit).  The result does not depend on the choice.
int reduce_num_configs();
const char *reduce_config_name(int config);
int reduce_selected();
void reduce_select(int config);
optigpu_status reduce_dispatch(const void *src, int64_t n, int dtype, void *out, uint32_t flags,
                               cudaStream_t stream);

// Partials of the chunks of one band (band_src = chunk `chunk_base`'s first
// element, band_n elements) into partials[chunk_base ...], and the final
// combine of `count` partials into *out: together, the single-pass sum.
optigpu_status reduce_band(const void *band_src, int64_t band_n, int dtype, uint32_t flags, void *partials,
                           int64_t chunk_base, cudaStream_t stream);
optigpu_status reduce_final(const void *partials, int64_t count, int dtype, uint32_t flags, void *out,
                            cudaStream_t stream);
// Forgets the allocation-free sum's cached scratch address on `device`.
void noalloc_forget_device(int device);
optigpu_status transpose_dispatch(const void *src, void *dst, int64_t rows, int64_t cols, int dtype, int kernel,
                                  cudaStream_t stream);
// Same with row pitches: dst[c * ldd + r] = src[r * lds + c].
optigpu_status transpose_dispatch_pitched(const void *src, int64_t lds, void *dst, int64_t ldd, int64_t rows,
                                          int64_t cols, int dtype, int kernel, cudaStream_t stream);
// Transpose of a dense b x cols band into dst with row pitch ldd.
optigpu_status transpose_band_into(const void *band, void *dst, int64_t b, int64_t cols, int64_t ldd, int dtype,
                                   cudaStream_t stream);

// Scan configurations: 0 = single pass (ordered look-back), 1 = three passes.
int scan_num_configs();
const char *scan_config_name(int config);
// The scan form is kept per input class (int32; the float types together).
int scan_selected(int dtype);
void scan_select(int dtype, int config);

// Batch kernel configurations (default of new plans).
int batch_num_configs();
const char *batch_config_name(int config);
int batch_selected();
void batch_select(int config);

} // namespace optigpu
