// Transpose without any allocation, for callers that cannot allocate device
// memory themselves: code running where cudaMalloc is not available or not
// allowed (inside a driver-managed memory pool, in a plug-in whose host owns
// all allocations, between graph captures, or under a fixed memory budget),
// and that also cannot hand the library a workspace.  The scratch that
// spg_csc_transpose needs comes from one file-scope device array instead.
//
// The array is a __device__ variable of this library: every GPU on which the
// library's module is loaded holds it (kNoallocScratchBytes) until the
// process exits.  All calls on a device share it and it keeps the contents of
// the last call, so calls whose work overlaps on the GPU (different streams,
// or host threads without ordering) race on it; order them on one stream.
#include <mutex>

#include "kernels.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = SPG_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Id of the calling thread's current CUDA context (driver entry points taken
// through the runtime, so the library needs no link to the driver library);
// false when there is none or the driver does not offer them.
bool current_context_id(unsigned long long &id) {
    using GetCurrent = int (*)(void **);
    using GetId = int (*)(void *, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<GetCurrent>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<GetId>(f);
    });
    void *ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, &id) == 0;
}

// Device address of the array, resolved with the device current (in host
// code the array's name is only a host-side stand-in).  It is looked up once
// per device and context: a reset of the device, or another primary context,
// loads the module again, possibly at another address, so the cached address
// is kept only while the context it was taken in is still the current one.
void *scratch_address(int device, cudaError_t &err) {
    struct Entry {
        void *addr = nullptr;
        unsigned long long ctx = 0;
        bool known = false;  // ctx holds the id of the context addr was taken in
    };
    static std::mutex mu;
    static Entry cache[64];
    err = cudaSuccess;
    if (device < 0 || device >= 64) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    unsigned long long id = 0;
    const bool have = current_context_id(id);
    std::lock_guard<std::mutex> lock(mu);
    Entry &e = cache[device];
    if (e.addr && have && e.known && e.ctx == id) return e.addr;
    void *p = nullptr;
    err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (err != cudaSuccess) return nullptr;
    // the lookup made the device's primary context current if none was
    e.addr = p;
    e.known = current_context_id(id);
    e.ctx = e.known ? id : 0;
    return p;
}

}  // namespace

extern "C" {

spg_status spg_csc_transpose_noalloc(const spg_csc *M, int64_t *T_colptr, int32_t *T_rowidx, void *T_values,
                                     int64_t *perm, spg_stream stream) {
    size_t need = 0;
    spg_status st = spg_transpose_workspace_size(M, &need);
    if (st != SPG_OK) return st;
    if (need > kNoallocScratchBytes) return SPG_ERR_WORKSPACE;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return SPG_ERR_CUDA;
    cudaError_t err;
    void *scratch = scratch_address(device, err);
    if (!scratch || err != cudaSuccess) return SPG_ERR_CUDA;
    // the row counters that must start at zero are cleared inside the call
    return spg_csc_transpose(M, T_colptr, T_rowidx, T_values, perm, scratch, kNoallocScratchBytes, stream);
}

}  // extern "C"
