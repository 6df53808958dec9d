// FP64 apply that allocates nothing: the expansion workspaces come from a
// fixed array in the library's device image instead of cudaMalloc.
//
// Who needs it: callers that must not allocate device memory at call time,
// e.g. code running inside another framework whose memory pool owns the free
// device memory, or a sequence being recorded while allocation is forbidden.
// The tree and context (lists, tables) are created beforehand as usual; this
// call only launches kernels.
//
// Sharing rules: every call, on every stream, uses the same array; calls that
// overlap on the GPU race with each other and must be serialised by the
// caller.  The call also uses the tree's own per-box flags and X-list buffer,
// so an overlapping apply of any kind on the same tree races with it too.  The
// array keeps what the last call left in it.  Every workspace element the
// apply reads is written earlier in the same apply, so nothing needs clearing
// between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "bc_internal.h"

namespace bc {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;   // 16 MiB per device, held until exit

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {};

// Device address of the array on `device` (which must be current); looked up
// once per device.
cudaError_t scratch_address(int device, void **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    if (!g_ptr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[device] = p;
    }
    *out = g_ptr[device];
    return cudaSuccess;
}

bool on_device(const void *p)
{
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace bc

using namespace bc;

extern "C" bc_status bc_apply_noalloc(bc_ctx *ctx, const bc_tree *tree, const double *in, double *out, int adjoint,
                                      void *stream)
{
    if (!ctx || !tree || !in || !out) { set_error("bc_apply_noalloc: NULL argument"); return BC_ERR_ARG; }
    if (tree->ctx != ctx) { set_error("bc_apply_noalloc: tree belongs to another context"); return BC_ERR_ARG; }
    if (ctx->device < 0) { set_error("bc_apply_noalloc: host-only context (device -1)"); return BC_ERR_STATE; }
    if (!ctx->tables_ready) { set_error("bc_apply_noalloc: call bc_tables_build first"); return BC_ERR_STATE; }
    if (in == out) { set_error("bc_apply_noalloc: output must not alias input"); return BC_ERR_ARG; }
    const size_t nbox = tree->h.box_level.size();
    const size_t need = 2 * nbox * size_t(ctx->P1) * sizeof(double2);
    if (need > kNoAllocBytes) {
        set_error("bc_apply_noalloc: tree needs %zu bytes of workspace (2 x %zu boxes x %d terms x 16 B), "
                  "above the fixed %zu-byte limit; use bc_apply",
                  need, nbox, ctx->P1, kNoAllocBytes);
        return BC_ERR_ARG;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) { set_error("bc_apply_noalloc: cudaSetDevice: %s", cudaGetErrorString(e)); return BC_ERR_CUDA; }
    if (!on_device(in) || !on_device(out)) {
        set_error("bc_apply_noalloc: input and output must be device memory");
        return BC_ERR_ARG;
    }
    void *base = nullptr;
    e = scratch_address(ctx->device, &base);
    if (e != cudaSuccess) {
        set_error("bc_apply_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return BC_ERR_CUDA;
    }
    DevTree d = tree->d;   // lists as uploaded with the tree; workspaces replaced
    d.expA = static_cast<double2 *>(base);
    d.expB = d.expA + nbox * size_t(ctx->P1);
    const PassArgs a = pass_args(ctx, tree);
    e = launch_apply(a, tree->h, d, ctx->dt, adjoint != 0, in, out, static_cast<cudaStream_t>(stream), 3, nullptr,
                     ctx->m2l_tri, nullptr);
    if (e != cudaSuccess) { set_error("bc_apply_noalloc: launch: %s", cudaGetErrorString(e)); return BC_ERR_CUDA; }
    return BC_OK;
}
