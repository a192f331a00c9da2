// vr_micro.cu -- FP32 FMA throughput probe: the roof the raymarch's arithmetic is
// measured against (the raymarch is bound by the FP32 pipe and L1, not by HBM).
//
// Each thread runs 8 independent FMA chains, 16 steps unrolled per iteration, so
// the FMA pipe, not its latency, limits the rate; the chains' results are stored
// so that nothing is optimised away.
#include "vr_async.cuh"
#include "vr_internal.cuh"

namespace vr {

namespace {

__global__ void __launch_bounds__(256) k_fma_peak(float* __restrict__ out, int iters, float a, float b) {
    const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) x[c] = (float)(tid & 255) * 1e-6f + (float)c * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int c = 0; c < 8; ++c) x[c] = fmaf(x[c], a, b);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) s += x[c];
    out[tid] = s;
}

// One thread waits, with a clock budget, on an mbarrier phase that nothing will
// complete (no arrivals, no transfers) -- the situation of a bulk copy that never
// lands -- and records the expired wait in the status word as the raymarch does.
__global__ void k_wait_probe(unsigned* __restrict__ status, long long budget) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
        if (!mbar_wait_bounded(&bar, 0, budget)) atomicOr(status, kStatusTimeout);
    }
}

// Fails one index check; nothing is read or written either way.
__global__ void k_check_probe(unsigned* status) {
    if (!VR_CHECK(status, threadIdx.x != 0)) return;
}

}  // namespace

cudaError_t launch_check_probe(unsigned* status, cudaStream_t st) {
    k_check_probe<<<1, 32, 0, st>>>(status);
    return cudaGetLastError();
}

cudaError_t launch_wait_probe(unsigned* status, long long budget_cycles, cudaStream_t st) {
    k_wait_probe<<<1, 32, 0, st>>>(status, budget_cycles);
    return cudaGetLastError();
}

// FLOPs of one launch: blocks * 256 threads * iters * 16 * 8 FMAs * 2.
cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t st) {
    k_fma_peak<<<blocks, 256, 0, st>>>(out, iters, 0.999f, 1e-4f);
    return cudaGetLastError();
}

}  // namespace vr
