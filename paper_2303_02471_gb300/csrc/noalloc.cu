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

// Device address of the array, resolved once per device with that device
// current (in host code the array's name is only a host-side stand-in).
void *scratch_address(int device, cudaError_t &err) {
    static std::mutex mu;
    static void *addr[64] = {};
    std::lock_guard<std::mutex> lock(mu);
    err = cudaSuccess;
    if (device < 0 || device >= 64) {
        err = cudaErrorInvalidDevice;
        return nullptr;
    }
    if (!addr[device]) {
        void *p = nullptr;
        err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (err != cudaSuccess) return nullptr;
        addr[device] = p;
    }
    return addr[device];
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
