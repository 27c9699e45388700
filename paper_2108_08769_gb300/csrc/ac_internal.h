// ac_internal.h -- helpers shared by the translation units of the library
// (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>

namespace acgb {

// Record the thread's last error message (read by ac_last_error) and
// return `code`.
int set_last_error(int code, const char *fmt, ...);

// Programmatic dependent launch (AC_PDL=0 turns it off): the kernels of a
// pseudo-iteration are launched so that each may be scheduled while its
// predecessor in the stream is still running; every such kernel starts with
// pdl_trigger() + pdl_wait() (ac_kernels.cuh), so it touches nothing before
// the predecessor has finished and its writes are visible.  What overlaps is
// the launch and CTA dispatch, not the work.
inline bool pdl_enabled() {
    static const bool on = [] {
        const char *e = getenv("AC_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

// AC_LOG=1 in the environment: the physical-step calls print one line per
// step on stderr (read at every call, so a process may switch it).
inline bool log_enabled() {
    const char *e = getenv("AC_LOG");
    return e && e[0] == '1';
}

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Args... args) {
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof cfg);
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr;
    memset(&attr, 0, sizeof attr);
    attr.id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr.val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace acgb
