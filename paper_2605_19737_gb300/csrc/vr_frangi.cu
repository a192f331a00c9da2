// vr_frangi.cu -- per-volume multi-scale Hessian vesselness (the "multi-scale
// Hessian analysis and vesselness measures" of Sec. 1, read as the
// bright-vessel response of Frangi et al., MICCAI 1998), computed once per
// volume like the paper's morphology compute shader (Sec. 2.3).
//
// For each scale sigma (voxels):
//   1. separable Gaussian smoothing, sampled normalised weights exp(-x^2/2s^2)
//      on [-R, R], R = ceil(4 sigma), clamp-to-edge, x then y then z;
//   2. Hessian of the smoothed volume by the central second / mixed differences
//      of Sec. 2.3 in voxel units, times sigma^2 (scale normalisation);
//   3. eigenvalues by cyclic Jacobi rotations in FP32, sorted |l1|<=|l2|<=|l3|;
//   4. pass A: S = ||lambda|| reduced to max_v S; pass B: c = max S / 2 and
//      V_sigma = 0 if l2 > 0 or l3 > 0, else
//      (1 - exp(-Ra^2/2a^2)) exp(-Rb^2/2b^2) (1 - exp(-S^2/2c^2)),
//      Ra = |l2|/|l3|, Rb = |l1|/sqrt|l2 l3|, a = b = 1/2;
//   V = max over scales.
// The smoothing passes are HBM/L1-streaming; the Hessian/eigen passes are ALU.
#include <math.h>

#include "vr_internal.cuh"

namespace vr {

namespace {

constexpr int kMaxRadius = 32;

struct GaussParams {
    float w[2 * kMaxRadius + 1];
    int R;
};

// One 1D Gaussian pass along `axis` (0 = x, 1 = y, 2 = z) with clamp-to-edge.
__global__ void __launch_bounds__(256) k_gauss_axis(const float* __restrict__ in, float* __restrict__ out, int nx,
                                                    int ny, int nz, int axis, const __grid_constant__ GaussParams G) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    const long long plane = (long long)nx * ny;
    float acc = 0.0f;
    if (axis == 0) {
        const float* row = in + (long long)z * plane + (long long)y * nx;
        for (int t = -G.R; t <= G.R; ++t) acc = fmaf(G.w[t + G.R], __ldg(row + min(max(x + t, 0), nx - 1)), acc);
    } else if (axis == 1) {
        const float* col = in + (long long)z * plane + x;
        for (int t = -G.R; t <= G.R; ++t)
            acc = fmaf(G.w[t + G.R], __ldg(col + (long long)min(max(y + t, 0), ny - 1) * nx), acc);
    } else {
        const float* col = in + (long long)y * nx + x;
        for (int t = -G.R; t <= G.R; ++t)
            acc = fmaf(G.w[t + G.R], __ldg(col + (long long)min(max(z + t, 0), nz - 1) * plane), acc);
    }
    out[(long long)z * plane + (long long)y * nx + x] = acc;
}

// Scale-normalised Hessian (xx yy zz xy xz yz) at voxel (x, y, z) of the smoothed volume.
__device__ __forceinline__ void hessian_at(const float* __restrict__ f, int nx, int ny, int nz, int x, int y, int z,
                                           float s2, float H[6]) {
    const long long plane = (long long)nx * ny;
    const int xm = max(x - 1, 0), xp = min(x + 1, nx - 1);
    const int ym = max(y - 1, 0), yp = min(y + 1, ny - 1);
    const int zm = max(z - 1, 0), zp = min(z + 1, nz - 1);
    auto at = [&](int i, int j, int k) { return __ldg(f + (long long)k * plane + (long long)j * nx + i); };
    const float c2 = 2.0f * at(x, y, z);
    H[0] = s2 * (at(xp, y, z) - c2 + at(xm, y, z));
    H[1] = s2 * (at(x, yp, z) - c2 + at(x, ym, z));
    H[2] = s2 * (at(x, y, zp) - c2 + at(x, y, zm));
    H[3] = 0.25f * s2 * ((at(xp, yp, z) - at(xp, ym, z)) - (at(xm, yp, z) - at(xm, ym, z)));
    H[4] = 0.25f * s2 * ((at(xp, y, zp) - at(xp, y, zm)) - (at(xm, y, zp) - at(xm, y, zm)));
    H[5] = 0.25f * s2 * ((at(x, yp, zp) - at(x, yp, zm)) - (at(x, ym, zp) - at(x, ym, zm)));
}

// One Jacobi rotation zeroing a[p][q] of the symmetric 3x3 matrix a.
__device__ __forceinline__ void jacobi_rotate(float a[3][3], int p, int q) {
    const float apq = a[p][q];
    if (apq == 0.0f) return;
    const float theta = (a[q][q] - a[p][p]) / (2.0f * apq);
    const float t = copysignf(1.0f, theta) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.0f)));
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
    }
}

// Eigenvalues sorted by |lambda| ascending (ties by lambda ascending).
__device__ __forceinline__ void eig3_sorted(const float H[6], float l[3]) {
    float a[3][3] = {{H[0], H[3], H[4]}, {H[3], H[1], H[5]}, {H[4], H[5], H[2]}};
    // cyclic sweeps until the off-diagonal part is below float resolution of the
    // diagonal (quadratic convergence: 3-4 sweeps), at most 6
#pragma unroll 1
    for (int sweep = 0; sweep < 6; ++sweep) {
        jacobi_rotate(a, 0, 1);
        jacobi_rotate(a, 0, 2);
        jacobi_rotate(a, 1, 2);
        const float off = fabsf(a[0][1]) + fabsf(a[0][2]) + fabsf(a[1][2]);
        if (off <= 1e-9f * (fabsf(a[0][0]) + fabsf(a[1][1]) + fabsf(a[2][2]))) break;
    }
    l[0] = a[0][0];
    l[1] = a[1][1];
    l[2] = a[2][2];
    auto before = [](float u, float v) { return fabsf(u) < fabsf(v) || (fabsf(u) == fabsf(v) && u < v); };
    if (before(l[1], l[0])) { const float t = l[0]; l[0] = l[1]; l[1] = t; }
    if (before(l[2], l[1])) { const float t = l[1]; l[1] = l[2]; l[2] = t; }
    if (before(l[1], l[0])) { const float t = l[0]; l[0] = l[1]; l[1] = t; }
}

// Per voxel: Hessian of the smoothed volume (x sigma^2), its eigenvalues sorted by
// |lambda| (stored, one plane of the SoA `eig` per eigenvalue, for the second pass)
// and the block maximum of S = |lambda|_2 folded into smax.
__global__ void __launch_bounds__(256) k_frangi_eig(const float* __restrict__ sm, int nx, int ny, int nz, float s2,
                                                    float* __restrict__ eig, float* __restrict__ smax) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    float S = 0.0f;
    if (x < nx && y < ny) {
        float H[6], l[3];
        hessian_at(sm, nx, ny, nz, x, y, z, s2, H);
        eig3_sorted(H, l);
        S = sqrtf(fmaf(l[0], l[0], fmaf(l[1], l[1], l[2] * l[2])));
        const long long nvox = (long long)nx * ny * nz, idx = ((long long)z * ny + y) * nx + x;
        eig[idx] = l[0];
        eig[nvox + idx] = l[1];
        eig[2 * nvox + idx] = l[2];
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) S = fmaxf(S, __shfl_xor_sync(0xffffffffu, S, o));
    __shared__ float ws[8];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = S;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) S = fmaxf(S, ws[w]);
        atomicMax(reinterpret_cast<int*>(smax), __float_as_int(S));
    }
}

// Frangi response of this scale from the stored eigenvalues (c = smax / 2), max-combined into V.
__global__ void __launch_bounds__(256) k_frangi_v(const float* __restrict__ eig, long long nvox,
                                                  const float* __restrict__ smax, float* __restrict__ V) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nvox) return;
    const float l[3] = {__ldg(eig + idx), __ldg(eig + nvox + idx), __ldg(eig + 2 * nvox + idx)};
    const float c = 0.5f * __ldg(smax);
    float v = 0.0f;
    if (!(l[1] > 0.0f || l[2] > 0.0f || l[1] == 0.0f || l[2] == 0.0f || c <= 0.0f)) {
        const float Ra = fabsf(l[1]) / fabsf(l[2]);
        const float Rb = fabsf(l[0]) / sqrtf(fabsf(l[1] * l[2]));
        const float S2 = fmaf(l[0], l[0], fmaf(l[1], l[1], l[2] * l[2]));
        // alpha = beta = 0.5: 2 alpha^2 = 2 beta^2 = 0.5
        v = (1.0f - expf(-Ra * Ra / 0.5f)) * expf(-Rb * Rb / 0.5f) * (1.0f - expf(-S2 / (2.0f * c * c)));
    }
    V[idx] = fmaxf(V[idx], v);
}

}  // namespace

cudaError_t launch_gauss3d(const float* in, float* out, float* tmp, const int n[3], float sigma, cudaStream_t st) {
    GaussParams G;
    G.R = (int)ceil(4.0 * (double)sigma);
    if (G.R > kMaxRadius || !(sigma > 0.0f)) return cudaErrorInvalidValue;
    double sum = 0.0, w[2 * kMaxRadius + 1];
    for (int i = -G.R; i <= G.R; ++i) sum += (w[i + G.R] = exp(-(double)i * i / (2.0 * (double)sigma * sigma)));
    for (int i = 0; i <= 2 * G.R; ++i) G.w[i] = (float)(w[i] / sum);
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, n[2]);
    k_gauss_axis<<<grid, 256, 0, st>>>(in, out, n[0], n[1], n[2], 0, G);
    k_gauss_axis<<<grid, 256, 0, st>>>(out, tmp, n[0], n[1], n[2], 1, G);
    k_gauss_axis<<<grid, 256, 0, st>>>(tmp, out, n[0], n[1], n[2], 2, G);
    return cudaGetLastError();
}

cudaError_t launch_frangi(const float* norm, const int n[3], const float* sigmas, int n_sigmas, float* tmp_a,
                          float* tmp_b /* 3 nvox floats */, float* smax /* n_sigmas floats */, float* V,
                          cudaStream_t st) {
    const long long nvox = (long long)n[0] * n[1] * n[2];
    cudaError_t e = cudaMemsetAsync(V, 0, sizeof(float) * nvox, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(smax, 0, sizeof(float) * n_sigmas, st);
    if (e != cudaSuccess) return e;
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, n[2]);
    for (int si = 0; si < n_sigmas; ++si) {
        const double sg = sigmas[si];
        GaussParams G;
        G.R = (int)ceil(4.0 * sg);
        if (G.R > kMaxRadius) return cudaErrorInvalidValue;
        double sum = 0.0, w[2 * kMaxRadius + 1];
        for (int i = -G.R; i <= G.R; ++i) sum += (w[i + G.R] = exp(-(double)i * i / (2.0 * sg * sg)));
        for (int i = 0; i <= 2 * G.R; ++i) G.w[i] = (float)(w[i] / sum);
        k_gauss_axis<<<grid, 256, 0, st>>>(norm, tmp_a, n[0], n[1], n[2], 0, G);
        k_gauss_axis<<<grid, 256, 0, st>>>(tmp_a, tmp_b, n[0], n[1], n[2], 1, G);
        k_gauss_axis<<<grid, 256, 0, st>>>(tmp_b, tmp_a, n[0], n[1], n[2], 2, G);
        const float s2 = (float)(sg * sg);
        // eigenvalues once (into tmp_b, free after the smoothing), then the response
        k_frangi_eig<<<grid, 256, 0, st>>>(tmp_a, n[0], n[1], n[2], s2, tmp_b, smax + si);
        k_frangi_v<<<(unsigned)((nvox + 255) / 256), 256, 0, st>>>(tmp_b, nvox, smax + si, V);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vr
