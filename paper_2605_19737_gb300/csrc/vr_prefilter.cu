// vr_prefilter.cu -- optional pre-filters of the normalised volume (the
// lightweight smoothing or median compute passes proposed in Sec. 5.3 against
// low-SNR and impulsive artefacts), applied before bricking and morphology.
//
// k_median3: one thread per voxel gathers its 27 clamp-to-edge neighbours into
// registers and selects the 14th smallest by rank counting (ties broken by
// position), an exact order statistic.
#include "vr_internal.cuh"

namespace vr {

namespace {

__global__ void __launch_bounds__(256) k_median3(const float* __restrict__ in, float* __restrict__ out, int nx, int ny,
                                                 int nz) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long plane = (long long)nx * ny;
    float w[27];
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int xx = min(max(x + dx, 0), nx - 1), yy = min(max(y + dy, 0), ny - 1),
                          zz = min(max(z + dz, 0), nz - 1);
                w[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = __ldg(in + (long long)zz * plane + (long long)yy * nx + xx);
            }
    float med = w[0];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        int rank = 0;
#pragma unroll
        for (int j = 0; j < 27; ++j) rank += (w[j] < w[i]) || (w[j] == w[i] && j < i);
        if (rank == 13) med = w[i];
    }
    out[(long long)z * plane + (long long)y * nx + x] = med;
}

}  // namespace

cudaError_t launch_median3(const float* in, float* out, const int n[3], cudaStream_t st) {
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, n[2]);
    k_median3<<<grid, 256, 0, st>>>(in, out, n[0], n[1], n[2]);
    return cudaGetLastError();
}

}  // namespace vr
