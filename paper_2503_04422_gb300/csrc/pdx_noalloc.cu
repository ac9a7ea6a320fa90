// pdx_search_exact_noalloc: the exact search with its scratch memory in a
// fixed, statically declared device array instead of the stream-ordered
// allocator. It launches the same kernels as pdx_search_exact.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pdx_internal.cuh"

namespace pdx {

// Capacity of the static scratch array. Every GPU that loads the library
// holds this much device memory until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;  // 32 MiB
constexpr int kNoAllocMaxDevices = 64;

// Shared by every call of pdx_search_exact_noalloc on a device. Host code
// must not use this symbol as a device address: its name denotes a host-side
// shadow. The device address is looked up with cudaGetSymbolAddress on every
// call (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of the static scratch array on the current device, looked
// up on every call with that device current. The lookup allocates nothing and
// is cheap; not caching it keeps the address valid after the device's primary
// context is reset and created again (cudaDeviceReset), which moves the array.
static pdx_status noalloc_scratch(unsigned char **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_error("pdx_search_exact_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
        return PDX_ERR_CUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("pdx_search_exact_noalloc: device ordinal %d not supported", dev);
        return PDX_ERR_UNSUPPORTED;
    }
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
        set_error("pdx_search_exact_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                  cudaGetErrorString(e));
        return PDX_ERR_CUDA;
    }
    *out = static_cast<unsigned char *>(p);
    return PDX_OK;
}

static bool noalloc_is_device(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace pdx

using namespace pdx;

extern "C" pdx_status pdx_search_exact_noalloc(const pdx_index *ix, const float *q, int64_t nq, int32_t k,
                                               const pdx_search_opts *opts, float *out_dist, int64_t *out_idx,
                                               void *stream) {
    const char *fn = "pdx_search_exact_noalloc";
    pdx_search_opts o;
    SearchPlan pl;
    pdx_status s = exact_check(ix, q, nq, k, opts, out_dist, out_idx, &o, &pl, fn);
    if (s != PDX_OK) return s;
    if (nq == 0) return PDX_OK;
    if (!noalloc_is_device(q) || !noalloc_is_device(out_dist) || !noalloc_is_device(out_idx)) {
        set_error("%s: q, out_dist and out_idx must be device memory (this entry point stages nothing)", fn);
        return PDX_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms < 1) sms = 1;
    ExactPlan ep;
    s = exact_plan(ix, nq, k, o, pl, sms, &ep);
    if (s != PDX_OK) return s;
    if (ep.bytes > kNoAllocScratchBytes) {
        set_error("%s: this search needs %zu bytes of scratch but the static array holds %zu; "
                  "use fewer queries per call or a smaller start_vectors", fn, ep.bytes, kNoAllocScratchBytes);
        return PDX_ERR_ARG;
    }
    if (o.tau_init && !noalloc_is_device(o.tau_init)) {
        set_error("%s: tau_init must be device memory (this entry point stages nothing)", fn);
        return PDX_ERR_ARG;
    }
    unsigned char *base = nullptr;
    s = noalloc_scratch(&base);
    if (s != PDX_OK) return s;
    // the array keeps the previous call's contents: exact_run resets everything
    // that must start from a known value (thresholds, counters, the work counter)
    unsigned long long *kc = nullptr;
    s = exact_run(ix, q, nq, k, o, pl, ep, base, out_dist, out_idx, &kc, sms, st);
    if (s != PDX_OK) return s;
    if (o.stats_out) {
        unsigned long long c[C_COUNT];
        cudaError_t e = cudaMemcpyAsync(c, kc, sizeof c, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            set_error("%s: reading the counters failed: %s", fn, cudaGetErrorString(e));
            return PDX_ERR_CUDA;
        }
        fill_stats(o.stats_out, c, ix);
    }
    return PDX_OK;
}
