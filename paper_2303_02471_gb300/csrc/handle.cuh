// Library state that outlives single products on one device (spg_handle of
// the C ABI): the side streams a call forks its lane-group bins onto, and the
// mapped pinned buffer of the small synchronising reads.  Host code only.
#pragma once

#include <mutex>

#include "kernels.cuh"

namespace spg {

// Side streams a numeric (and symbolic) call spreads the lane-group bins
// over, with the events of the fork from and the join back to the caller's
// stream.
constexpr int kNumSideStreams = 2;

struct SideStreams {
    cudaStream_t side[kNumSideStreams] = {};
    cudaEvent_t fork = nullptr, join[kNumSideStreams] = {};

    bool ready() const { return fork != nullptr; }
    // What a failed attempt created is kept and not created again.
    bool create() {
        if (fork) return true;
        for (int i = 0; i < kNumSideStreams; ++i)
            if ((!side[i] && cudaStreamCreateWithFlags(&side[i], cudaStreamNonBlocking) != cudaSuccess) ||
                (!join[i] && cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess))
                return false;
        return cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) == cudaSuccess;
    }
    void release() {
        for (int i = 0; i < kNumSideStreams; ++i) {
            if (side[i]) cudaStreamDestroy(side[i]);
            if (join[i]) cudaEventDestroy(join[i]);
            side[i] = nullptr;
            join[i] = nullptr;
        }
        if (fork) cudaEventDestroy(fork);
        fork = nullptr;
    }
};

}  // namespace spg

struct spg_handle {
    int device = 0;
    spg::SideStreams streams;
    spg::Mirror mirror;
    std::mutex mu;  // serialises read-backs through `mirror`

    ~spg_handle() { streams.release(); }
};

namespace spg {

// Small device -> host read of a call made with handle h (NULL: through the
// calling thread's own buffer).
inline cudaError_t handle_readback(spg_handle *h, void *dst0, const void *src0, size_t n0, void *dst1,
                                   const void *src1, size_t n1, cudaStream_t s) {
    if (!h) return readback(nullptr, dst0, src0, n0, dst1, src1, n1, s);
    std::lock_guard<std::mutex> lock(h->mu);
    return readback(&h->mirror, dst0, src0, n0, dst1, src1, n1, s);
}

}  // namespace spg
