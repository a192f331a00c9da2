// vr_volume.cu -- per-volume stages: the parallel reductions of Eq. 1 and
// Eq. 4 (Sec. 2.2, Sec. 4), min-max normalisation (Eq. 1), bricking with a
// clamp-to-edge apron, the quantised per-brick min/max grid and the
// transfer-function-driven empty-brick classification (the calvarium culling
// by transfer-function clipping of Sec. 2.2, used for empty-space skipping).
//
// All of these are HBM-bound streaming kernels: coalesced x-fastest access,
// 16-byte vector loads where the layout allows, grids sized in multiples of
// the SM count.
#include <math.h>

#include "vr_internal.cuh"

namespace vr {

namespace {

constexpr int kReduceThreads = 256;
constexpr int kSMs = 152;

__device__ __forceinline__ void warp_minmax(float& lo, float& hi) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
}

// Block-wide min/max; result valid in thread 0.
__device__ __forceinline__ void block_minmax(float& lo, float& hi) {
    __shared__ float slo[32], shi[32];
    warp_minmax(lo, hi);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        slo[w] = lo;
        shi[w] = hi;
    }
    __syncthreads();
    if (w == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        lo = l < nw ? slo[l] : INFINITY;
        hi = l < nw ? shi[l] : -INFINITY;
        warp_minmax(lo, hi);
    }
}

__device__ __forceinline__ void acc(float v, float& lo, float& hi) {
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
}

// Per-block partial min/max over a grid-stride range; float32 input read as float4.
__global__ void __launch_bounds__(kReduceThreads) k_minmax_partials_f32(const float* __restrict__ x, long long n,
                                                                        float* __restrict__ partials) {
    float lo = INFINITY, hi = -INFINITY;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    long long done = 0;
    if (aligned) {
        const long long n4 = n >> 2;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (long long i = tid; i < n4; i += stride) {
            float4 v = __ldg(x4 + i);
            acc(v.x, lo, hi);
            acc(v.y, lo, hi);
            acc(v.z, lo, hi);
            acc(v.w, lo, hi);
        }
        done = n4 << 2;
    }
    for (long long i = done + tid; i < n; i += stride) acc(__ldg(x + i), lo, hi);
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = lo;
        partials[2 * blockIdx.x + 1] = hi;
    }
}

// uint16 input read as 8 values per 16-byte load.
__global__ void __launch_bounds__(kReduceThreads) k_minmax_partials_u16(const uint16_t* __restrict__ x, long long n,
                                                                        float* __restrict__ partials) {
    float lo = INFINITY, hi = -INFINITY;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const bool aligned = (reinterpret_cast<uintptr_t>(x) & 15) == 0;
    long long done = 0;
    if (aligned) {
        const long long n8 = n >> 3;
        const uint4* x8 = reinterpret_cast<const uint4*>(x);
        for (long long i = tid; i < n8; i += stride) {
            uint4 v = __ldg(x8 + i);
            const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                acc((float)(w[q] & 0xffffu), lo, hi);
                acc((float)(w[q] >> 16), lo, hi);
            }
        }
        done = n8 << 3;
    }
    for (long long i = done + tid; i < n; i += stride) acc((float)__ldg(x + i), lo, hi);
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = lo;
        partials[2 * blockIdx.x + 1] = hi;
    }
}

__global__ void __launch_bounds__(1024) k_minmax_final(const float* __restrict__ partials, int nblocks,
                                                       float* __restrict__ out2) {
    float lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        lo = fminf(lo, partials[2 * i]);
        hi = fmaxf(hi, partials[2 * i + 1]);
    }
    block_minmax(lo, hi);
    if (threadIdx.x == 0) {
        out2[0] = lo;
        out2[1] = hi;
    }
}

// Eq. 1 in float32, one IEEE round-to-nearest operation at a time:
// d = x - I_min; I_norm = d / (I_max - I_min). Also publishes the constants.
template <typename T>
__global__ void k_normalize(const T* __restrict__ raw, long long n, const float* __restrict__ mm,
                            VolConst* __restrict__ vc, float* __restrict__ out) {
    const float imin = __ldg(mm), imax = __ldg(mm + 1);
    const float range = __fsub_rn(imax, imin);
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (tid == 0) {
        vc->imin = imin;
        vc->imax = imax;
        vc->range = range;
    }
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = tid; i < n; i += stride) out[i] = __fdiv_rn(__fsub_rn((float)__ldg(raw + i), imin), range);
}

// One CTA per brick: copy voxels [8b-1, 8b+11) per axis (clamped) into the
// brick's 12^3 block. Reads are row-contiguous in x, writes fully contiguous.
__global__ void __launch_bounds__(256) k_make_bricks(const float* __restrict__ norm, int nx, int ny, int nz, int nbx,
                                                     int nby, float* __restrict__ bricks) {
    const long long b = blockIdx.x;
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long long)nbx * nby));
    float* dst = bricks + b * kBrickVox;
#pragma unroll
    for (int q = 0; q < (kBrickVox + 255) / 256; ++q) {  // 256 threads: the loads issue back to back
        const int e = threadIdx.x + 256 * q;
        if (e >= kBrickVox) break;
        const int lx = e % kEdge, ly = (e / kEdge) % kEdge, lz = e / (kEdge * kEdge);
        const int x = min(max(kCells * bx - 1 + lx, 0), nx - 1);
        const int y = min(max(kCells * by - 1 + ly, 0), ny - 1);
        const int z = min(max(kCells * bz - 1 + lz, 0), nz - 1);
        dst[e] = __ldg(norm + ((long long)z * ny + y) * nx + x);
    }
}

// One CTA per skip brick: the voxel-wise intensity, central-difference gradient
// (Eq. 2) and second/mixed differences (Sec. 2.3) of the brick's (B+1)^3 corner
// voxels, with clamp-to-edge neighbours, divided by the spacing -- the per-voxel
// morphology the paper's compute shader produces, laid out for 16-byte loads.
__global__ void __launch_bounds__(256) k_make_derived(const float* __restrict__ norm, int nx, int ny, int nz, int nbx,
                                                      int nby, int bs, float hx, float hy, float hz,
                                                      float* __restrict__ out) {
    // the brick's corner voxels and their neighbours, [Bb - 1, Bb + B + 2) per axis,
    // clamped to the volume (so neighbour i +- 1 of a corner is tile entry t +- 1)
    constexpr int kTMax = (1 << kMaxBrickShift) + 3;
    __shared__ float tile[kTMax * kTMax * kTMax];
    const int B = 1 << bs, E = B + 1, T = B + 3;
    const long long b = blockIdx.x;
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long long)nbx * nby));
    const int x0 = B * bx - 1, y0 = B * by - 1, z0 = B * bz - 1;
    for (int e = threadIdx.x; e < T * T * T; e += blockDim.x) {
        const int tx = e % T, ty = (e / T) % T, tz = e / (T * T);
        const int x = min(max(x0 + tx, 0), nx - 1), y = min(max(y0 + ty, 0), ny - 1), z = min(max(z0 + tz, 0), nz - 1);
        tile[e] = __ldg(norm + ((long long)z * ny + y) * nx + x);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < E * E * E; e += blockDim.x) {
        const int lx = e % E, ly = (e / E) % E, lz = e / (E * E);
        // the corner voxel (clamped as in the per-voxel definition) in tile coordinates
        const int tx = min(B * bx + lx, nx - 1) - x0, ty = min(B * by + ly, ny - 1) - y0,
                  tz = min(B * bz + lz, nz - 1) - z0;
        auto at = [&](int dx, int dy, int dz) { return tile[((tz + dz) * T + (ty + dy)) * T + (tx + dx)]; };
        const float c = at(0, 0, 0), c2 = 2.0f * c;
        float4 a, m, t;
        a.x = c;
        a.y = (at(1, 0, 0) - at(-1, 0, 0)) * (0.5f * hx);
        a.z = (at(0, 1, 0) - at(0, -1, 0)) * (0.5f * hy);
        a.w = (at(0, 0, 1) - at(0, 0, -1)) * (0.5f * hz);
        m.x = (at(1, 0, 0) - c2 + at(-1, 0, 0)) * (hx * hx);
        m.y = (at(0, 1, 0) - c2 + at(0, -1, 0)) * (hy * hy);
        m.z = (at(0, 0, 1) - c2 + at(0, 0, -1)) * (hz * hz);
        m.w = ((at(1, 1, 0) - at(1, -1, 0)) - (at(-1, 1, 0) - at(-1, -1, 0))) * (0.25f * hx * hy);
        t.x = ((at(1, 0, 1) - at(1, 0, -1)) - (at(-1, 0, 1) - at(-1, 0, -1))) * (0.25f * hx * hz);
        t.y = ((at(0, 1, 1) - at(0, 1, -1)) - (at(0, -1, 1) - at(0, -1, -1))) * (0.25f * hy * hz);
        t.z = 0.0f;
        t.w = 0.0f;
        float4* o = reinterpret_cast<float4*>(out + b * der_brick_floats(bs)) + 3 * e;
        o[0] = a;
        o[1] = m;
        o[2] = t;
    }
}

// One warp per skip brick: min/max of I_norm over the brick's corner voxels
// [Bb, min(Bb+B, N-1)] per axis, quantised to qlo = floor(min*65535),
// qhi = ceil(max*65535) (float32 round-to-nearest products).
__global__ void __launch_bounds__(256) k_brick_minmax(const float* __restrict__ norm, int nx, int ny, int nz, int nbx,
                                                      int nby, int bs, long long nbricks, uint16_t* __restrict__ grid) {
    const long long b = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= nbricks) return;
    const int B = 1 << bs;
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long long)nbx * nby));
    const int x0 = B * bx, y0 = B * by, z0 = B * bz;
    const int ex = min(x0 + B, nx - 1) - x0 + 1;
    const int ey = min(y0 + B, ny - 1) - y0 + 1;
    const int ez = min(z0 + B, nz - 1) - z0 + 1;
    float lo = INFINITY, hi = -INFINITY;
    const int cnt = ex * ey * ez;
    for (int e = lane; e < cnt; e += 32) {
        const int lx = e % ex, ly = (e / ex) % ey, lz = e / (ex * ey);
        acc(__ldg(norm + ((long long)(z0 + lz) * ny + (y0 + ly)) * nx + (x0 + lx)), lo, hi);
    }
    warp_minmax(lo, hi);
    if (lane == 0) {
        // codes clamp to [0, 65535]: intensities set outside [0, 1] (vr_set_normalized)
        // look up the transfer function's end entries, which the clamped range covers
        grid[2 * b] = (uint16_t)fminf(fmaxf(floorf(__fmul_rn(lo, 65535.0f)), 0.0f), 65535.0f);
        grid[2 * b + 1] = (uint16_t)fminf(fmaxf(ceilf(__fmul_rn(hi, 65535.0f)), 0.0f), 65535.0f);
    }
}

// |grad I|_max: largest voxel-wise central-difference gradient magnitude
// (Eq. 2 with clamp-to-edge neighbours), reduced per block then combined with
// an integer atomicMax on the (non-negative) float's bit pattern.
__global__ void __launch_bounds__(256) k_gmax(const float* __restrict__ I, int nx, int ny, int nz, float hx, float hy,
                                              float hz, VolConst* __restrict__ vc) {
    const int i = blockIdx.x * 32 + (threadIdx.x & 31);
    const int j = blockIdx.y * 8 + (threadIdx.x >> 5);
    const int k = blockIdx.z;
    float m = 0.0f;
    if (i < nx && j < ny) {
        const long long row = (long long)ny * nx;
        const float* c = I + (long long)k * row + (long long)j * nx + i;
        const float gx = (__ldg(c + (i + 1 < nx ? 1 : 0)) - __ldg(c - (i > 0 ? 1 : 0))) * hx;
        const float gy = (__ldg(c + (j + 1 < ny ? nx : 0)) - __ldg(c - (j > 0 ? nx : 0))) * hy;
        const float gz = (__ldg(c + (k + 1 < nz ? row : 0)) - __ldg(c - (k > 0 ? row : 0))) * hz;
        m = sqrtf(gx * gx + gy * gy + gz * gz);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float sm[8];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, sm[w]);
        atomicMax(reinterpret_cast<int*>(&vc->gmax), __float_as_int(m));
    }
}

// For every intensity column j of the transfer function: 1 if any row has a
// non-zero opacity; then an exclusive prefix count, so that a brick's column
// range can be tested in O(1). One block of 1024 threads: every opacity entry is
// read by its own thread (all loads in flight at once), each thread then owns
// four consecutive columns of the scan (w <= 4096).
__global__ void __launch_bounds__(1024) k_tf_alpha_prefix(const float* __restrict__ tf, int w, int h,
                                                          int* __restrict__ prefix) {
    __shared__ int col[4096];
    __shared__ int warp_sum[32];
    for (int j = threadIdx.x; j < w; j += blockDim.x) col[j] = 0;
    __syncthreads();
    for (long long e = threadIdx.x; e < (long long)w * h; e += blockDim.x)
        if (tf[4 * e + 3] != 0.0f) col[e % w] = 1;  // racing writes all store 1
    __syncthreads();
    const int j0 = 4 * threadIdx.x;
    int c[4], s = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        c[q] = j0 + q < w ? col[j0 + q] : 0;
        s += c[q];
    }
    // exclusive scan of the per-thread sums: within each warp, then over the warps
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int t = warp_sum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += v;
        }
        warp_sum[lane] = t - warp_sum[lane];  // exclusive over warps
    }
    __syncthreads();
    int run = warp_sum[wid] + incl - s;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        if (j0 + q < w) prefix[j0 + q] = run;
        run += c[q];
    }
    if (j0 < w && j0 + 4 >= w) prefix[w] = run;  // the thread holding the last column
}

// A brick is empty when no transfer-function column in
// [floor(qlo*(w-1)/65535) - 1, ceil(qhi*(w-1)/65535) + 1] has any opacity.
__global__ void k_classify(const uint16_t* __restrict__ grid, long long nbricks, const int* __restrict__ prefix,
                           int w, uint8_t* __restrict__ empty) {
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbricks) return;
    const long long ql = grid[2 * b], qh = grid[2 * b + 1];
    long long jl = (ql * (w - 1)) / 65535 - 1;
    long long jh = (qh * (w - 1) + 65534) / 65535 + 1;
    if (jl < 0) jl = 0;
    if (jh > w - 1) jh = w - 1;
    empty[b] = (uint8_t)(prefix[jh + 1] - prefix[jl] == 0);
}

// Per cell of each skip brick -- cell (lx, ly, lz) has corner voxels [Bb + l, Bb + l + 1]
// per axis -- the quantised min/max of I_norm over its 8 corners, with the brick
// grid's rounding. Cells past the volume's last cell (corner index > N - 2) never
// hold a sample and get the empty range (65535, 0). One thread per cell, cells of a
// brick consecutive ((lz B + ly) B + lx).
__global__ void __launch_bounds__(256) k_cell_minmax(const float* __restrict__ norm, int nx, int ny, int nz, int nbx,
                                                     int nby, int bs, long long ncells, uint16_t* __restrict__ cellq) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ncells) return;
    const int B = 1 << bs, m = B - 1;
    const long long b = e >> (3 * bs);
    const int c = (int)(e & ((1 << (3 * bs)) - 1));
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((long long)nbx * nby));
    const int x = B * bx + (c & m), y = B * by + ((c >> bs) & m), z = B * bz + (c >> (2 * bs));
    uint16_t ql = 65535, qh = 0;
    if (x <= nx - 2 && y <= ny - 2 && z <= nz - 2) {
        float lo = INFINITY, hi = -INFINITY;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            acc(__ldg(norm + ((long long)(z + (q >> 2)) * ny + (y + ((q >> 1) & 1))) * nx + (x + (q & 1))), lo, hi);
        ql = (uint16_t)fminf(fmaxf(floorf(__fmul_rn(lo, 65535.0f)), 0.0f), 65535.0f);
        qh = (uint16_t)fminf(fmaxf(ceilf(__fmul_rn(hi, 65535.0f)), 0.0f), 65535.0f);
    }
    cellq[2 * e] = ql;
    cellq[2 * e + 1] = qh;
}

// A cell is empty under the brick rule applied to its own range: no transfer-function
// column in [floor(qlo*(w-1)/65535) - 1, ceil(qhi*(w-1)/65535) + 1] has any opacity
// (every sample in the cell interpolates its 8 corners, so its intensity lies in the
// range). Each warp packs the bits of 32 consecutive cells into one word.
__global__ void __launch_bounds__(256) k_classify_cells(const uint16_t* __restrict__ cellq, long long ncells,
                                                        const int* __restrict__ prefix, int w,
                                                        uint32_t* __restrict__ cellmask) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if ((e & ~31ll) >= ncells) return;  // ncells is a multiple of 64: warps are whole
    const long long ql = cellq[2 * e], qh = cellq[2 * e + 1];
    bool empty = true;
    if (ql <= qh) {
        long long jl = (ql * (w - 1)) / 65535 - 1;
        long long jh = (qh * (w - 1) + 65534) / 65535 + 1;
        if (jl < 0) jl = 0;
        if (jh > w - 1) jh = w - 1;
        empty = prefix[jh + 1] - prefix[jl] == 0;
    }
    const unsigned bits = __ballot_sync(0xffffffffu, empty);
    if ((threadIdx.x & 31) == 0) cellmask[e >> 5] = bits;
}

}  // namespace

cudaError_t launch_cell_minmax(const float* norm, const int n[3], const int nb[3], int bs, uint16_t* cellq,
                               cudaStream_t st) {
    const long long ncells = ((long long)nb[0] * nb[1] * nb[2]) << (3 * bs);
    k_cell_minmax<<<(unsigned)((ncells + 255) / 256), 256, 0, st>>>(norm, n[0], n[1], n[2], nb[0], nb[1], bs, ncells,
                                                                    cellq);
    return cudaGetLastError();
}

cudaError_t launch_classify_cells(const uint16_t* cellq, long long nbricks, int bs, const int* prefix, int tf_w,
                                  uint32_t* cellmask, cudaStream_t st) {
    const long long ncells = nbricks << (3 * bs);
    k_classify_cells<<<(unsigned)((ncells + 255) / 256), 256, 0, st>>>(cellq, ncells, prefix, tf_w, cellmask);
    return cudaGetLastError();
}

int minmax_blocks(long long n) {
    long long want = (n + (long long)kReduceThreads * 16 - 1) / ((long long)kReduceThreads * 16);
    if (want < 1) want = 1;
    if (want > kSMs * 8) want = kSMs * 8;
    return (int)want;
}

cudaError_t launch_minmax_partials(const void* data, vr_dtype dt, long long n, float* partials, int nblocks,
                                   cudaStream_t st) {
    if (dt == VR_F32)
        k_minmax_partials_f32<<<nblocks, kReduceThreads, 0, st>>>((const float*)data, n, partials);
    else
        k_minmax_partials_u16<<<nblocks, kReduceThreads, 0, st>>>((const uint16_t*)data, n, partials);
    return cudaGetLastError();
}

cudaError_t launch_minmax_final(const float* partials, int nblocks, float* out2, cudaStream_t st) {
    k_minmax_final<<<1, 1024, 0, st>>>(partials, nblocks, out2);
    return cudaGetLastError();
}

cudaError_t launch_normalize(const void* raw, vr_dtype dt, long long n, const float* minmax2, VolConst* vc,
                             float* norm, cudaStream_t st) {
    const int blocks = kSMs * 8;
    if (dt == VR_F32)
        k_normalize<float><<<blocks, 256, 0, st>>>((const float*)raw, n, minmax2, vc, norm);
    else
        k_normalize<uint16_t><<<blocks, 256, 0, st>>>((const uint16_t*)raw, n, minmax2, vc, norm);
    return cudaGetLastError();
}

cudaError_t launch_make_bricks(const float* norm, const int n[3], const int nb[3], float* bricks, cudaStream_t st) {
    const long long nbr = (long long)nb[0] * nb[1] * nb[2];
    k_make_bricks<<<(unsigned)nbr, 256, 0, st>>>(norm, n[0], n[1], n[2], nb[0], nb[1], bricks);
    return cudaGetLastError();
}

cudaError_t launch_brick_minmax(const float* norm, const int n[3], const int nb[3], int bs, uint16_t* grid,
                                cudaStream_t st) {
    const long long nbr = (long long)nb[0] * nb[1] * nb[2];
    const unsigned blocks = (unsigned)((nbr + 7) / 8);
    k_brick_minmax<<<blocks, 256, 0, st>>>(norm, n[0], n[1], n[2], nb[0], nb[1], bs, nbr, grid);
    return cudaGetLastError();
}

cudaError_t launch_make_derived(const float* norm, const int n[3], const int nb[3], int bs, const float s[3],
                                float* dbricks, cudaStream_t st) {
    const long long nbr = (long long)nb[0] * nb[1] * nb[2];
    k_make_derived<<<(unsigned)nbr, 256, 0, st>>>(norm, n[0], n[1], n[2], nb[0], nb[1], bs, 1.0f / s[0],
                                                  1.0f / s[1], 1.0f / s[2], dbricks);
    return cudaGetLastError();
}

cudaError_t launch_gmax(const float* norm, const int n[3], const float s[3], VolConst* vc, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&vc->gmax, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    dim3 grid((n[0] + 31) / 32, (n[1] + 7) / 8, n[2]);
    k_gmax<<<grid, 256, 0, st>>>(norm, n[0], n[1], n[2], 0.5f / s[0], 0.5f / s[1], 0.5f / s[2], vc);
    return cudaGetLastError();
}

cudaError_t launch_classify(const uint16_t* grid, long long nbricks, const float* tf, int tf_w, int tf_h,
                            uint8_t* empty, int* prefix_scratch, cudaStream_t st) {
    k_tf_alpha_prefix<<<1, 1024, 0, st>>>(tf, tf_w, tf_h, prefix_scratch);
    k_classify<<<(unsigned)((nbricks + 255) / 256), 256, 0, st>>>(grid, nbricks, prefix_scratch, tf_w, empty);
    return cudaGetLastError();
}

}  // namespace vr

// ---------------------------------------------------------------------------
// Allocation-free brick classification.
//
// Some callers cannot allocate device memory at the point where they need to
// re-classify bricks: a host that hands the GPU to this library with a fixed,
// pre-reserved memory budget, a real-time interaction thread that must not
// enter the allocator, or code running while another component holds the
// device's allocator. For them this entry point runs the same two kernels as
// vr_set_tissue_params' classification, but keeps their scratch (the
// transfer-function column prefix table) in a static device array compiled into
// the library instead of asking for memory.
#include <mutex>

namespace vr {
namespace {

constexpr int kStaticTfMaxW = 4096;  // largest table width the static scratch holds
constexpr int kStaticMaxDevices = 64;

// tf_w + 1 prefix counts; every call rewrites all the entries it reads, so
// nothing here has to start at zero. Each GPU that loads the library holds
// these 16 KB until the process exits.
static __device__ __align__(256) int g_static_prefix[kStaticTfMaxW + 1];

std::mutex g_static_mu;
// Per device: the device address of the static array and the id of the CUDA context
// it was taken in. A device reset (cudaDeviceReset) destroys the context and the
// module with it; the next call sees a new context id and looks the address up again.
int* g_static_prefix_ptr[kStaticMaxDevices] = {};
unsigned long long g_static_ctx_id[kStaticMaxDevices] = {};
// Driver entry points for the current context and its process-unique id, resolved
// through the runtime so that the library does not link the driver library itself.
typedef int (*CtxGetCurrentFn)(void**);
typedef int (*CtxGetIdFn)(void*, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
bool g_ctx_fns_resolved = false;

// Id of the calling thread's current CUDA context, 0 when it cannot be told.
unsigned long long current_ctx_id() {
    if (!g_ctx_fns_resolved) {
        g_ctx_fns_resolved = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f);
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f);
        (void)cudaGetLastError();
    }
    if (!g_ctx_get_current || !g_ctx_get_id) return 0;
    void* cu = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&cu) != 0 || !cu || g_ctx_get_id(cu, &id) != 0) return 0;
    return id;
}

void put_msg(char* buf, int len, const char* msg) {
    if (!buf || len <= 0) return;
    int i = 0;
    for (; i < len - 1 && msg[i]; ++i) buf[i] = msg[i];
    buf[i] = '\0';
}

}  // namespace
}  // namespace vr

extern "C" vr_status vr_classify_bricks_noalloc(const unsigned short* d_grid, long long nbricks, const float* d_tf,
                                                int tf_w, int tf_h, unsigned char* d_empty, void* cuda_stream,
                                                char* h_msg, int msg_len) {
    using namespace vr;
    put_msg(h_msg, msg_len, "");
    if (!d_grid || !d_tf || !d_empty || nbricks < 1 || nbricks > (1LL << 31)) {
        put_msg(h_msg, msg_len, "classify_bricks_noalloc: NULL pointer or brick count outside [1, 2^31]");
        return VR_ERR_INVALID_ARG;
    }
    if (tf_w < 2 || tf_w > kStaticTfMaxW) {
        put_msg(h_msg, msg_len,
                "classify_bricks_noalloc: tf_w must be in [2, 4096]; the static scratch holds 4097 prefix counts");
        return VR_ERR_INVALID_ARG;
    }
    if (tf_h < 1 || tf_h > 256) {
        put_msg(h_msg, msg_len, "classify_bricks_noalloc: tf_h must be in [1, 256]");
        return VR_ERR_INVALID_ARG;
    }
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kStaticMaxDevices) {
        (void)cudaGetLastError();
        put_msg(h_msg, msg_len, "classify_bricks_noalloc: no usable current CUDA device");
        return VR_ERR_CUDA;
    }
    int* prefix = nullptr;
    {
        // once per device and CUDA context, with that device current: the device
        // address of the static array (the host-side symbol is not a device pointer).
        // A context id of 0 (no current context yet, or the driver cannot say) looks
        // the address up on every call.
        std::lock_guard<std::mutex> lock(g_static_mu);
        unsigned long long id = current_ctx_id();
        if (!g_static_prefix_ptr[dev] || id == 0 || id != g_static_ctx_id[dev]) {
            int* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress((void**)&p, g_static_prefix);
            if (e != cudaSuccess || !p) {
                (void)cudaGetLastError();
                put_msg(h_msg, msg_len, "classify_bricks_noalloc: cudaGetSymbolAddress of the static scratch failed");
                return VR_ERR_CUDA;
            }
            if (id == 0) id = current_ctx_id();  // the lookup made the primary context current
            g_static_prefix_ptr[dev] = p;
            g_static_ctx_id[dev] = id;
        }
        prefix = g_static_prefix_ptr[dev];
    }
    const cudaError_t e = launch_classify(reinterpret_cast<const uint16_t*>(d_grid), nbricks, d_tf, tf_w, tf_h,
                                          reinterpret_cast<uint8_t*>(d_empty), prefix, (cudaStream_t)cuda_stream);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        put_msg(h_msg, msg_len, cudaGetErrorString(e));
        return VR_ERR_CUDA;
    }
    return VR_OK;
}
