// vr_frangi.cu -- per-volume multi-scale Hessian vesselness (the multi-scale
// Hessian analysis with vesselness measures that Sec. 1 mentions, read as the
// bright-vessel response of Frangi et al., MICCAI 1998), computed once per
// volume like the paper's morphology compute shader (Sec. 2.3).
//
// For each scale sigma (voxels):
//   1. separable Gaussian smoothing, sampled normalised weights exp(-x^2/2s^2)
//      on [-R, R], R = ceil(4 sigma), clamp-to-edge, x then y then z;
//   2. Hessian of the smoothed volume by the central second / mixed differences
//      of Sec. 2.3 in voxel units, times sigma^2 (scale normalisation);
//   3. pass A: S = ||lambda|| = ||H||_F (Frobenius norm) reduced to max_v S;
//   4. pass B: the Hessian again, its eigenvalues by cyclic Jacobi rotations in
//      FP32 sorted |l1|<=|l2|<=|l3|, c = max S / 2 and
//      V_sigma = 0 if l2 > 0 or l3 > 0, else
//      (1 - exp(-Ra^2/2a^2)) exp(-Rb^2/2b^2) (1 - exp(-S^2/2c^2)),
//      Ra = |l2|/|l3|, Rb = |l1|/sqrt|l2 l3|, a = b = 1/2;
//   V = max over scales.
// The smoothing passes stream the volume through shared-memory tiles; the
// Hessian/eigen passes are ALU.
#include <math.h>

#include "vr_internal.cuh"

namespace vr {

namespace {

constexpr int kMaxRadius = 32;

struct GaussParams {
    float w[2 * kMaxRadius + 1];
    int R;
};

// The 1D Gaussian passes (clamp-to-edge). Each block stages its input span, halo
// included, in shared memory once, so that every voxel is read from L2/HBM about
// once per pass instead of once per tap; every output sums its 2R+1 taps in the
// order t = -R .. R with one fmaf each.
constexpr int kGaussRow = 256;  // x pass: outputs per block (one row segment)
constexpr int kGaussCol = 64;   // y / z passes: outputs per column, 32 columns per block

// Taps of one output from a staged span (stride `ld` floats between taps): kR > 0
// is the radius known at compile time (the loop unrolls, weights become constant
// operands); kR = 0 reads it from G.R.
template <int kR>
__device__ __forceinline__ float gauss_taps(const float* span, int ld, const GaussParams& G) {
    float acc = 0.0f;
    if (kR > 0) {
#pragma unroll
        for (int t = -kR; t <= kR; ++t) acc = fmaf(G.w[t + kR], span[(t + kR) * ld], acc);
    } else {
        for (int t = -G.R; t <= G.R; ++t) acc = fmaf(G.w[t + G.R], span[(t + G.R) * ld], acc);
    }
    return acc;
}

// x pass: block (x0 .. x0+255, y, z).
template <int kR>
__global__ void __launch_bounds__(256) k_gauss_x(const float* __restrict__ in, float* __restrict__ out, int nx,
                                                 int ny, const __grid_constant__ GaussParams G) {
    __shared__ float s[kGaussRow + 2 * kMaxRadius];
    const int x0 = blockIdx.x * kGaussRow, y = blockIdx.y, z = blockIdx.z;
    const float* row = in + ((long long)z * ny + y) * nx;
#pragma unroll
    for (int k = 0; k < (kGaussRow + 2 * kMaxRadius + 255) / 256; ++k) {  // loads issued back to back
        const int i = threadIdx.x + 256 * k;
        if (i < kGaussRow + 2 * G.R) s[i] = __ldg(row + min(max(x0 - G.R + i, 0), nx - 1));
    }
    __syncthreads();
    const int x = x0 + threadIdx.x;
    if (x >= nx) return;
    out[((long long)z * ny + y) * nx + x] = gauss_taps<kR>(s + threadIdx.x, 1, G);
}

// y or z pass: block = 32 consecutive x times kGaussCol outputs along the pass
// axis (extent na, element stride `stride`); blockIdx.z indexes the remaining axis
// (offset `other` elements per step). 256 threads: 32 columns x 8 rows.
template <int kR>
__global__ void __launch_bounds__(256) k_gauss_col(const float* __restrict__ in, float* __restrict__ out, int nx,
                                                   int na, long long stride, long long other,
                                                   const __grid_constant__ GaussParams G) {
    __shared__ float s[kGaussCol + 2 * kMaxRadius][32];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int x = blockIdx.x * 32 + tx;
    const int a0 = blockIdx.y * kGaussCol;
    const long long base = (long long)blockIdx.z * other + x;
    const bool col = x < nx;
#pragma unroll
    for (int k = 0; k < (kGaussCol + 2 * kMaxRadius) / 8; ++k) {  // loads issued back to back
        const int i = ty + 8 * k;
        if (i < kGaussCol + 2 * G.R)
            s[i][tx] = col ? __ldg(in + base + (long long)min(max(a0 - G.R + i, 0), na - 1) * stride) : 0.0f;
    }
    __syncthreads();
    if (!col) return;
    for (int o = ty; o < kGaussCol && a0 + o < na; o += 8)
        out[base + (long long)(a0 + o) * stride] = gauss_taps<kR>(&s[o][tx], 32, G);
}

// x, then y, then z: in -> out (x) -> tmp (y) -> out (z).
template <int kR>
void gauss_passes_r(const float* in, float* out, float* tmp, const int n[3], const GaussParams& G, cudaStream_t st) {
    const long long plane = (long long)n[0] * n[1];
    k_gauss_x<kR><<<dim3((n[0] + kGaussRow - 1) / kGaussRow, n[1], n[2]), 256, 0, st>>>(in, out, n[0], n[1], G);
    k_gauss_col<kR><<<dim3((n[0] + 31) / 32, (n[1] + kGaussCol - 1) / kGaussCol, n[2]), 256, 0, st>>>(
        out, tmp, n[0], n[1], (long long)n[0], plane, G);
    k_gauss_col<kR><<<dim3((n[0] + 31) / 32, (n[2] + kGaussCol - 1) / kGaussCol, n[1]), 256, 0, st>>>(
        tmp, out, n[0], n[2], plane, (long long)n[0], G);
}

// Radii 4, 8 and 12 (sigma = 1, 2, 3) are unrolled; others take the generic loop.
void gauss_passes(const float* in, float* out, float* tmp, const int n[3], const GaussParams& G, cudaStream_t st) {
    switch (G.R) {
        case 4: gauss_passes_r<4>(in, out, tmp, n, G, st); break;
        case 8: gauss_passes_r<8>(in, out, tmp, n, G, st); break;
        case 12: gauss_passes_r<12>(in, out, tmp, n, G, st); break;
        default: gauss_passes_r<0>(in, out, tmp, n, G, st); break;
    }
}

// Scale-normalised Hessian (xx yy zz xy xz yz) at voxel (x, y, z) of the smoothed
// volume: one 64-bit centre address, clamp-to-edge neighbours as 32-bit offsets.
__device__ __forceinline__ void hessian_at(const float* __restrict__ f, int nx, int ny, int nz, int x, int y, int z,
                                           float s2, float H[6]) {
    const int plane = nx * ny;  // <= 2048^2
    const float* c = f + ((long long)z * ny + y) * nx + x;
    const int xm = x > 0 ? -1 : 0, xp = x < nx - 1 ? 1 : 0;
    const int ym = y > 0 ? -nx : 0, yp = y < ny - 1 ? nx : 0;
    const int zm = z > 0 ? -plane : 0, zp = z < nz - 1 ? plane : 0;
    auto at = [&](int o) { return __ldg(c + o); };
    const float c2 = 2.0f * at(0);
    H[0] = s2 * (at(xp) - c2 + at(xm));
    H[1] = s2 * (at(yp) - c2 + at(ym));
    H[2] = s2 * (at(zp) - c2 + at(zm));
    H[3] = 0.25f * s2 * ((at(xp + yp) - at(xp + ym)) - (at(xm + yp) - at(xm + ym)));
    H[4] = 0.25f * s2 * ((at(xp + zp) - at(xp + zm)) - (at(xm + zp) - at(xm + zm)));
    H[5] = 0.25f * s2 * ((at(yp + zp) - at(yp + zm)) - (at(ym + zp) - at(ym + zm)));
}

// ||H||_F = ||lambda|| (the Frobenius norm is invariant under the orthogonal
// similarity that diagonalises H): S without the eigen-decomposition.
__device__ __forceinline__ float hessian_norm(const float H[6]) {
    const float off = fmaf(H[3], H[3], fmaf(H[4], H[4], H[5] * H[5]));
    return sqrtf(fmaf(2.0f, off, fmaf(H[0], H[0], fmaf(H[1], H[1], H[2] * H[2]))));
}

// One Jacobi rotation of the symmetric 3x3 matrix held as its diagonal d and its
// off-diagonal entries o[0] = a01, o[1] = a02, o[2] = a12, in the plane (p, q) with
// r the third index: the angle makes a_pq exactly zero and the other entries take
// the stable updates of the classical method (tan t of the smaller angle, tau =
// s / (1 + c)); Golub & Van Loan, Sec. 8.5 (the symmetric Schur decomposition).
__device__ __forceinline__ void jacobi_rotate(float d[3], float& opq, float& orp, float& orq, int p, int q) {
    const float apq = opq;
    if (apq == 0.0f) return;
    // The rotation stays orthogonal (c = 1/sqrt(1 + t^2), s = t c) however t is
    // rounded, so t comes from the fast reciprocal; an inexact angle leaves a
    // residual a_pq of a few ulp, which is dropped at the float resolution of H.
    const float theta = 0.5f * __fdividef(d[q] - d[p], apq);
    // t = sign(theta) / (|theta| + sqrt(theta^2 + 1)), with |theta| capped at 1e18
    // (then t ~ 5e-19: a_pq is negligible) so that theta^2 + 1 stays finite and
    // its square root can be taken as r * rsqrt(r)
    const float at = fminf(fabsf(theta), 1e18f);
    const float r = fmaf(at, at, 1.0f);
    float t = __fdividef(1.0f, fmaf(r, rsqrtf(r), at));
    if (theta < 0.0f) t = -t;
    const float c = rsqrtf(fmaf(t, t, 1.0f)), s = t * c, tau = __fdividef(s, 1.0f + c);
    d[p] = fmaf(-t, apq, d[p]);
    d[q] = fmaf(t, apq, d[q]);
    opq = 0.0f;
    const float rp = orp, rq = orq;
    orp = fmaf(-s, fmaf(tau, rp, rq), rp);
    orq = fmaf(s, fmaf(-tau, rq, rp), rq);
}

// Eigenvalues sorted by |lambda| ascending (ties by lambda ascending).
__device__ __forceinline__ void eig3_sorted(const float H[6], float l[3]) {
    float d[3] = {H[0], H[1], H[2]};
    float o01 = H[3], o02 = H[4], o12 = H[5];
    // cyclic sweeps (planes 01, 02, 12) until the off-diagonal part is below float
    // resolution of the diagonal (then every eigenvalue is within that of the
    // diagonal entry, Weyl's inequality; quadratic convergence: 2-3 sweeps), at most 8
#pragma unroll 1
    for (int sweep = 0; sweep < 8; ++sweep) {
        const float off = fabsf(o01) + fabsf(o02) + fabsf(o12);
        if (off <= 6e-8f * (fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]))) break;
        jacobi_rotate(d, o01, o02, o12, 0, 1);  // r = 2: a20 = o02, a21 = o12
        jacobi_rotate(d, o02, o01, o12, 0, 2);  // r = 1: a10 = o01, a12 = o12
        jacobi_rotate(d, o12, o01, o02, 1, 2);  // r = 0: a01 = o01, a02 = o02
    }
    l[0] = d[0];
    l[1] = d[1];
    l[2] = d[2];
    auto before = [](float u, float v) { return fabsf(u) < fabsf(v) || (fabsf(u) == fabsf(v) && u < v); };
    if (before(l[1], l[0])) { const float t = l[0]; l[0] = l[1]; l[1] = t; }
    if (before(l[2], l[1])) { const float t = l[1]; l[1] = l[2]; l[2] = t; }
    if (before(l[1], l[0])) { const float t = l[0]; l[0] = l[1]; l[1] = t; }
}

// Pass A of a scale: the maximum over voxels of S = ||H|| (block maxima folded
// into smax with an integer atomicMax on the non-negative float bits).
__global__ void __launch_bounds__(256) k_frangi_smax(const float* __restrict__ sm, int nx, int ny, int nz, float s2,
                                                     float* __restrict__ smax) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    float S = 0.0f;
    if (x < nx && y < ny) {
        float H[6];
        hessian_at(sm, nx, ny, nz, x, y, z, s2, H);
        S = hessian_norm(H);
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

// Pass B: per voxel the Hessian again, its eigenvalues sorted by |lambda|, and the
// Frangi response of this scale (c = smax / 2), max-combined into V.
__global__ void __launch_bounds__(256) k_frangi_v(const float* __restrict__ sm, int nx, int ny, int nz, float s2,
                                                  const float* __restrict__ smax, float* __restrict__ V) {
    const int x = blockIdx.x * 32 + (threadIdx.x & 31);
    const int y = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int z = blockIdx.z;
    if (x >= nx || y >= ny) return;
    float H[6], l[3];
    hessian_at(sm, nx, ny, nz, x, y, z, s2, H);
    const float c = 0.5f * __ldg(smax);
    const long long idx = ((long long)z * ny + y) * nx + x;
    float v = 0.0f;
    // bright vessels only: l2 < 0 and l3 < 0 (cheap test on the diagonal first:
    // with both negative eigenvalues the trace is negative)
    if (c > 0.0f && H[0] + H[1] + H[2] < 0.0f) {
        eig3_sorted(H, l);
        if (!(l[1] > 0.0f || l[2] > 0.0f || l[1] == 0.0f || l[2] == 0.0f)) {
            // fast reciprocal, reciprocal square root and exponential: a few ulp on
            // factors in [0, 1], far inside the 1e-4 the response is held to
            const float Ra = __fdividef(fabsf(l[1]), fabsf(l[2]));
            const float Rb = fabsf(l[0]) * rsqrtf(fabsf(l[1] * l[2]));
            const float S = hessian_norm(H);
            // alpha = beta = 0.5: 2 alpha^2 = 2 beta^2 = 0.5
            v = (1.0f - __expf(-2.0f * Ra * Ra)) * __expf(-2.0f * Rb * Rb) *
                (1.0f - __expf(-(S * S) * __fdividef(0.5f, c * c)));
        }
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
    gauss_passes(in, out, tmp, n, G, st);
    return cudaGetLastError();
}

cudaError_t launch_frangi(const float* norm, const int n[3], const float* sigmas, int n_sigmas, float* tmp_a,
                          float* tmp_b /* nvox floats */, float* smax /* n_sigmas floats */, float* V,
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
        gauss_passes(norm, tmp_a, tmp_b, n, G, st);
        const float s2 = (float)(sg * sg);
        k_frangi_smax<<<grid, 256, 0, st>>>(tmp_a, n[0], n[1], n[2], s2, smax + si);
        k_frangi_v<<<grid, 256, 0, st>>>(tmp_a, n[0], n[1], n[2], s2, smax + si, V);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace vr
