// Filter application that allocates no device memory.
//
// nm_filter_apply keeps its recurrence scratch in a buffer the problem
// allocates with cudaMalloc on first use. Some callers cannot allow that:
// a host whose device memory is handed out by another allocator (a
// framework's caching pool that has already reserved the free HBM, where a
// direct cudaMalloc fails or fragments it), a latency-bound serving loop in
// which cudaMalloc / cudaFree would synchronise the device and stall the
// other streams, or an embedded host that must know its whole device
// footprint when the library is loaded. For them nm_filter_apply_static
// runs the same FP64 recurrence with its scratch in a fixed-size array
// that lives in this file's device image.
//
// Consequences of a file-scope array, which a caller has to respect:
//  - every GPU on which the array is used holds NM_STATIC_SCRATCH_BYTES of
//    device memory until the process exits;
//  - all calls on one device share the array, so two calls whose kernels
//    overlap on that GPU (other streams, threads, contexts or problems)
//    overwrite each other's scratch; serialise them;
//  - the first call on a device looks up the array's device address (and,
//    with lazy module loading, loads this file's device code); make that
//    first call before any stream capture.
#include <mutex>
#include <string>

#include "kernels.h"
#include "nm_internal.h"

namespace nm {
size_t filter_scratch_bytes(const nm_problem* P, int b);
int filter_apply_on(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z, int64_t ldz,
                    int b, double* scratch, cudaStream_t s);
}  // namespace nm

using namespace nm;

namespace {

// In host code this name stands for the device array; it is not a device
// address. The kernels get the address cudaGetSymbolAddress returns for it.
static __device__ __align__(256) double g_static_scratch[NM_STATIC_SCRATCH_BYTES / sizeof(double)];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double* g_scratch_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device (the current device must be `dev`).
int scratch_address(int dev, double** out) {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess || !ptr) {
            cudaGetLastError();
            return fail(NM_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
        }
        g_scratch_addr[dev] = static_cast<double*>(ptr);
    }
    *out = g_scratch_addr[dev];
    return NM_OK;
}

struct ThreadCtx {
    explicit ThreadCtx(nm_ctx* c) { set_thread_ctx(c); }
    ~ThreadCtx() { set_thread_ctx(nullptr); }
};

}  // namespace

extern "C" int nm_filter_apply_static(nm_problem* P, const nm_filter* f, const double* Y, int64_t ldy, double* Z,
                                      int64_t ldz, int b, void* stream) {
    if (!P || !f) return fail(NM_EINVAL, "null argument");
    ThreadCtx tc(P->ctx);
    if (b < 1 || b > 64) return fail(NM_EINVAL, "block width b must be in 1..64");
    if (ldy < b || ldz < b) return fail(NM_EINVAL, "leading dimension must be >= b");
    if (P->info.n > 0 && (!Y || !Z)) return fail(NM_EINVAL, "null device pointer");
    const size_t need = filter_scratch_bytes(P, b);
    if (need > (size_t)NM_STATIC_SCRATCH_BYTES)
        return fail(NM_EINVAL, "nm_filter_apply_static: n = " + std::to_string(P->info.n) + ", Np = " +
                                   std::to_string(P->info.Np) + ", b = " + std::to_string(b) + " needs " +
                                   std::to_string(need) + " bytes of scratch, above the static maximum of " +
                                   std::to_string((size_t)NM_STATIC_SCRATCH_BYTES) +
                                   " bytes; use nm_filter_apply or a smaller b");
    NM_CUDA(cudaSetDevice(P->ctx->device));
    int dev = -1;
    NM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(NM_EUNSUPPORTED, "device ordinal above 63");
    double* scratch = nullptr;
    NM_TRY(scratch_address(dev, &scratch));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Every scratch word is written before it is read within one call; the
    // clear makes each call start from the same state whatever ran before.
    NM_CUDA(cudaMemsetAsync(scratch, 0, need, s));
    return filter_apply_on(P, f, Y, ldy, Z, ldz, b, scratch, s);
}
