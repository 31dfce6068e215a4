// prof.cuh -- optional timing of the tensor-core kernels with CUDA events.
//
// When enabled (clusco_profile_enable), every launch of the all-pairs kernel, of the
// adjoint kernel, of the dRMSD kernel or of the contact-map kernel is bracketed by two CUDA events recorded on the launch's own stream;
// clusco_profile_read sums the bracketed durations. Off by default; the only cost when off
// is one atomic load per launch.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>
#include <vector>

namespace clusco {

enum ProfKind { PROF_PAIRS = 0, PROF_ADJOINT = 1, PROF_DRMSD = 2, PROF_CMO = 3, PROF_KINDS = 4 };

struct ProfState {
    std::atomic<bool> on{false};
    std::mutex m;
    std::vector<cudaEvent_t> ev[PROF_KINDS];  // begin, end, begin, end, ...
};

inline ProfState &prof_state()
{
    static ProfState p;
    return p;
}

// Record one bracket event for kernel kind k on stream st (a no-op when profiling is off).
inline void prof_mark(int k, cudaStream_t st)
{
    ProfState &p = prof_state();
    if (!p.on.load(std::memory_order_relaxed)) return;
    std::lock_guard<std::mutex> g(p.m);
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return;
    if (cudaEventRecord(e, st) != cudaSuccess) {
        cudaEventDestroy(e);
        return;
    }
    p.ev[k].push_back(e);
}

}  // namespace clusco
