// vr_micro.cu -- FP32 FMA throughput probe: the roof the raymarch's arithmetic is
// measured against (the raymarch is bound by the FP32 pipe and L1, not by HBM).
//
// Each thread runs 8 independent FMA chains, 16 steps unrolled per iteration, so
// the FMA pipe, not its latency, limits the rate; the chains' results are stored
// so that nothing is optimised away.
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

}  // namespace

// FLOPs of one launch: blocks * 256 threads * iters * 16 * 8 FMAs * 2.
cudaError_t launch_fma_peak(float* out, int blocks, int iters, cudaStream_t st) {
    k_fma_peak<<<blocks, 256, 0, st>>>(out, iters, 0.999f, 1e-4f);
    return cudaGetLastError();
}

}  // namespace vr
