// vr_histogram.cu -- the 256-bin density analysis of Sec. 2.2 and the
// tri-modal tissue-peak extraction behind Tables 1-2.
//
// k_histogram256: every CTA counts its grid-stride share of the normalised
// volume into a private 256-bin shared-memory histogram, then adds it to the
// global one (one atomic per non-empty bin per CTA). The bin of a voxel is the
// integer min(floor(I_norm * 256), 255) taken in float32, where I_norm is the
// float32 normalisation of Eq. 1 already stored for the volume.
// k_tissue_peaks: one CTA; binomial [1 4 6 4 1] smoothing with integer
// weights, local maxima inside [lo, hi], the three largest (ties to the lower
// bin), returned in ascending bin order. Integer arithmetic throughout, so the
// result is exact.
#include "vr_internal.cuh"

namespace vr {

namespace {

__global__ void __launch_bounds__(256) k_histogram256(const float* __restrict__ norm, long long n,
                                                      unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[256];
    h[threadIdx.x] = 0u;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = __fmul_rn(__ldg(norm + i), 256.0f);
        int j = (int)x;
        j = min(max(j, 0), 255);
        atomicAdd(&h[j], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(hist + threadIdx.x, (unsigned long long)h[threadIdx.x]);
}

__global__ void __launch_bounds__(256) k_tissue_peaks(const unsigned long long* __restrict__ hist, int lo, int hi,
                                                      int* __restrict__ peaks) {
    __shared__ unsigned long long s[256];
    const int j = threadIdx.x;
    unsigned long long acc = 0;
    const int w[5] = {1, 4, 6, 4, 1};
#pragma unroll
    for (int t = -2; t <= 2; ++t) acc += (unsigned long long)w[t + 2] * hist[min(max(j + t, 0), 255)];
    s[j] = acc;
    __syncthreads();
    if (j == 0) {
        const int a = max(lo, 1), b = min(hi, 254);
        int best[3] = {-1, -1, -1};
        for (int q = a; q <= b; ++q) {
            if (!(s[q] > s[q - 1] && s[q] >= s[q + 1])) continue;
            for (int r = 0; r < 3; ++r) {
                if (best[r] < 0 || s[q] > s[best[r]]) {
                    for (int u = 2; u > r; --u) best[u] = best[u - 1];
                    best[r] = q;
                    break;
                }
            }
        }
        int out[3], cnt = 0;
        for (int r = 0; r < 3; ++r)
            if (best[r] >= 0) out[cnt++] = best[r];
        for (int x = 0; x < cnt; ++x)
            for (int y = x + 1; y < cnt; ++y)
                if (out[y] < out[x]) {
                    const int t = out[x];
                    out[x] = out[y];
                    out[y] = t;
                }
        for (int r = 0; r < 3; ++r) peaks[r] = r < cnt ? out[r] : -1;
        peaks[3] = cnt;
    }
}

}  // namespace

cudaError_t launch_histogram(const float* norm, long long n, unsigned long long* hist, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    long long blocks = (n + 256LL * 64 - 1) / (256LL * 64);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_histogram256<<<(unsigned)blocks, 256, 0, st>>>(norm, n, hist);
    return cudaGetLastError();
}

cudaError_t launch_tissue_peaks(const unsigned long long* hist, int lo, int hi, int* peaks4, cudaStream_t st) {
    k_tissue_peaks<<<1, 256, 0, st>>>(hist, lo, hi, peaks4);
    return cudaGetLastError();
}

}  // namespace vr
