// C ABI of the strip solve (include/boxcode.h, bc_strip_*): argument checks
// and the launch of kernels_strip.cu.
#include <cstdint>

#include "bc_internal.h"

namespace bc {
namespace {
bool strip_on_device(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}
bool strip_shape_ok(int64_t nsys, int64_t N, int m, int r)
{
    return nsys >= 0 && nsys <= INT32_MAX && N >= 1 && m >= 1 && m <= 32 && r >= 1 && r <= 32;
}
}  // namespace
}  // namespace bc

using namespace bc;

bc_status bc_strip_workspace(int64_t nsys, int64_t N, int m, int r, int64_t *bytes)
{
    if (!bytes || !strip_shape_ok(nsys, N, m, r)) {
        set_error("bc_strip_workspace: need nsys >= 0, N >= 1, 1 <= m <= 32, 1 <= r <= 32");
        return BC_ERR_ARG;
    }
    *bytes = int64_t(sizeof(double) * strip_work_doubles(N, m, r)) * nsys;
    return BC_OK;
}

bc_status bc_strip_solve(int64_t nsys, int64_t N, int m, int r, const double *A, const double *B, const double *C,
                         const double *b, double *x, void *work, int32_t *status, void *stream)
{
    if (!strip_shape_ok(nsys, N, m, r)) {
        set_error("bc_strip_solve: need nsys >= 0, N >= 1, 1 <= m <= 32, 1 <= r <= 32");
        return BC_ERR_ARG;
    }
    if (nsys == 0) return BC_OK;
    if (!A || !B || !C || !b || !x || !work) { set_error("bc_strip_solve: NULL argument"); return BC_ERR_ARG; }
    for (const void *p : {(const void *)A, (const void *)B, (const void *)C, (const void *)b, (const void *)x,
                          (const void *)work})
        if (!strip_on_device(p)) { set_error("bc_strip_solve: every array must be device memory"); return BC_ERR_ARG; }
    if (status && !strip_on_device(status)) { set_error("bc_strip_solve: status must be device memory"); return BC_ERR_ARG; }
    const cudaError_t e = launch_strip(nsys, N, m, r, A, B, C, b, x, static_cast<double *>(work), status,
                                       static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) {
        set_error("bc_strip_solve: %s (%s)", cudaGetErrorName(e), cudaGetErrorString(e));
        return BC_ERR_CUDA;
    }
    return BC_OK;
}
