// fold_noalloc.cu -- the half-turn folded back-projection for callers that
// must not allocate device memory at call time.
//
// dyn_radon_adj with the fold variant keeps its folded data in a buffer the
// plan allocates with cudaMalloc on first use.  Some callers cannot allow
// that: code running while a stream is being captured into a CUDA graph
// (an allocation inside a capture fails or breaks it), and applications
// whose memory policy forbids any allocation after start-up (a fixed device
// memory budget handed out by their own pool).  dyn_radon_adj_noalloc does
// the same computation with the folded data in a fixed file-scope device
// array instead, and allocates nothing.
//
// The array costs kNoAllocBytes of device memory on every GPU that loads
// this library, for the life of the process.  All calls in the process share
// it, so two calls whose work overlaps on the GPU (different streams, or
// different host threads) race on it; calls issued in order on one stream
// are safe.  Every call overwrites the part it uses completely before
// reading it, so nothing has to start at zero.
#include <algorithm>
#include <cmath>
#include <mutex>

#include <cudaTypedefs.h>

#include "fold_impl.cuh"

namespace dr {

// 8 MiB of folded data: nz * U * ns * MS floats (MS = m padded, see fold_ms).
constexpr size_t kNoAllocBytes = size_t(8) << 20;
constexpr size_t kNoAllocFloats = kNoAllocBytes / sizeof(float);

static __device__ __align__(256) float g_noalloc_fold_scratch[kNoAllocFloats];

// Device address of the array.  Host code must not use the symbol itself as
// a device pointer: the address is looked up with cudaGetSymbolAddress, with
// the device current, once per device and CUDA context, and cached together
// with the context's process-unique id (cuCtxGetId), so that a context torn
// down and re-created (cudaDeviceReset) gets a fresh lookup instead of a
// stale pointer.  If those driver calls cannot be resolved, every call looks
// the address up.
constexpr int kMaxDevices = 64;
struct NoAllocEntry {
    unsigned long long ctx_id;
    float *ptr;
};
static std::mutex g_noalloc_mutex;
static NoAllocEntry g_noalloc_ptr[kMaxDevices];
static std::once_flag g_noalloc_ctx_once;
static PFN_cuCtxGetCurrent_v4000 g_ctx_current = nullptr;
static PFN_cuCtxGetId_v12000 g_ctx_id = nullptr;

static bool current_context_id(unsigned long long *id) {
    std::call_once(g_noalloc_ctx_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    });
    CUcontext ctx = nullptr;
    if (!g_ctx_current || !g_ctx_id || g_ctx_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return g_ctx_id(ctx, id) == CUDA_SUCCESS;
}

static dr_status noalloc_scratch(int device, float **out) {
    if (device < 0 || device >= kMaxDevices) return fail(DR_EINVAL, "dyn_radon_adj_noalloc: device index out of range");
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    NoAllocEntry &e = g_noalloc_ptr[device];
    if (!have_id || !e.ptr || e.ctx_id != id) {
        void *p = nullptr;
        const cudaError_t ce = cudaGetSymbolAddress(&p, g_noalloc_fold_scratch);
        if (ce != cudaSuccess) return cuda_fail(ce, "dyn_radon_adj_noalloc: cudaGetSymbolAddress");
        e.ptr = static_cast<float *>(p);
        e.ctx_id = have_id ? id : 0;
    }
    *out = e.ptr;
    return DR_OK;
}

// The plan's folded adjoint (data fold, then back-projection) with the folded
// data in the fixed array instead of the plan's scratch buffer.
template <typename S, int M>
static dr_status noalloc_adj_t(dr_plan *P, const void *g, void *u, double beta, float *scratch, cudaStream_t st) {
    return fold_adj_launch_t<S, float, M>(P, g, u, 1.0, beta, false, st, scratch);
}

template <typename S>
static dr_status noalloc_dispatch(dr_plan *P, const void *g, void *u, double beta, float *scratch, cudaStream_t st) {
    switch (P->M) {
        case 1: return noalloc_adj_t<S, 1>(P, g, u, beta, scratch, st);
        case 2: return noalloc_adj_t<S, 2>(P, g, u, beta, scratch, st);
        case 4: return noalloc_adj_t<S, 4>(P, g, u, beta, scratch, st);
        case 8: return noalloc_adj_t<S, 8>(P, g, u, beta, scratch, st);
        case 12: return noalloc_adj_t<S, 12>(P, g, u, beta, scratch, st);
        case 16: return noalloc_adj_t<S, 16>(P, g, u, beta, scratch, st);
        case 24: return noalloc_adj_t<S, 24>(P, g, u, beta, scratch, st);
        case 32: return noalloc_adj_t<S, 32>(P, g, u, beta, scratch, st);
    }
    return fail(DR_EINVAL, "dyn_radon_adj_noalloc: unsupported m");
}

}  // namespace dr

using namespace dr;

extern "C" dr_status dyn_radon_adj_noalloc(dr_plan *P, const void *g, void *u, double beta) {
    clear_error();
    if (!P || !g || !u) return fail(DR_EINVAL, "dyn_radon_adj_noalloc: NULL argument");
    if (!std::isfinite(beta)) return fail(DR_EINVAL, "dyn_radon_adj_noalloc: beta must be finite");
    if (P->prec == DR_F64 || P->fold_U == 0)
        return fail(DR_EINVAL, "dyn_radon_adj_noalloc: needs an F32 or BF16 plan (the half-turn fold)");
    const size_t need = sizeof(float) * (size_t)P->nz * P->fold_U * P->ns * fold_ms(P->M);
    if (need > kNoAllocBytes)
        return fail(DR_EINVAL, "dyn_radon_adj_noalloc: folded data needs " + std::to_string(need) +
                                   " bytes, more than the fixed " + std::to_string(kNoAllocBytes) +
                                   "-byte scratch array (use fewer slices per call)");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "dyn_radon_adj_noalloc: cudaGetDevice");
    if (dev != P->device) return fail(DR_EINVAL, "dyn_radon_adj_noalloc: the plan's device must be current");
    float *scratch = nullptr;
    dr_status s = noalloc_scratch(dev, &scratch);
    if (s != DR_OK) return s;
    if (P->prec == DR_BF16_F32ACC) return noalloc_dispatch<bf16>(P, g, u, beta, scratch, P->stream);
    return noalloc_dispatch<float>(P, g, u, beta, scratch, P->stream);
}
