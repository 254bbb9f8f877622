// selftest.cu -- exercises the device-side timeout path without a fault.
//
// One CTA waits on a fresh mbarrier phase that nothing will complete, with
// the same bounded wait the TMA transpose uses (mbar_wait_bounded).  When the
// limit runs out the kernel records DEV_ERR_WAIT_TIMEOUT in the device status
// word and returns normally, so the context stays usable and
// optigpu_stream_status reports OPTIGPU_ERR_TIMEOUT.
#include "internal.h"
#include "ptx.cuh"

namespace optigpu {
namespace {

__global__ void wait_that_times_out(uint64_t limit_ns, unsigned *status)
{
    __shared__ __align__(8) uint64_t bar;
    const uint32_t a = ptx::smem_addr(&bar);
    if (threadIdx.x == 0) {
        // Expected count 1; nobody arrives, so phase 0 never completes.
        ptx::mbar_init(a, 1);
        ptx::fence_mbar_init();
        if (!ptx::mbar_wait_bounded(a, 0u, limit_ns))
            atomicOr(status, DEV_ERR_WAIT_TIMEOUT);
    }
}

} // namespace
} // namespace optigpu

using namespace optigpu;

extern "C" optigpu_status optigpu_selftest_wait_timeout(uint64_t limit_ns, optigpu_stream_t stream)
{
    if (limit_ns == 0 || limit_ns > 10000000000ull)
        return fail(OPTIGPU_ERR_INVALID_ARG, "selftest: limit must be in (0, 10 s]");
    DeviceInfo dev;
    optigpu_status st = current_device(dev);
    if (st != OPTIGPU_OK)
        return st;
    wait_that_times_out<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(limit_ns, dev.status_word);
    return check_cuda(cudaGetLastError(), "launch selftest");
}
