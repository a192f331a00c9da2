// vr_render.cu -- forward raymarch kernels (Sec. 2.4, Eqs. 4-6).
//
// k_render_gather: one thread per ray, a warp covers an 8x4 pixel packet and a
// CTA a 16x8 tile. Each lane walks its own samples front to back; per sample it
// gathers the 56 weighted voxels of its cell's 4x4x4 neighbourhood straight
// from the bricked volume (L1/L2-resident), evaluates the field, Eq. 4 and the
// shading, and composites by Eqs. 5-6. Samples in bricks classified empty are
// skipped a brick at a time (bit-neutral: their opacity is exactly zero).
#include "vr_sample.cuh"

namespace vr {

namespace {

struct GlobalLoad {
    const float* __restrict__ p;
    __device__ __forceinline__ float operator()(int o) const { return __ldg(p + o); }
};

__device__ __forceinline__ long long brick_index(const VolumeDev& v, const int b[3]) {
    return ((long long)b[2] * v.nb[1] + b[1]) * v.nb[0] + b[0];
}

__device__ __forceinline__ void add_counters(vr_counters* ctr, unsigned rays, unsigned dense, unsigned evald,
                                             unsigned staged) {
    const unsigned r = __reduce_add_sync(0xffffffffu, rays);
    const unsigned d = __reduce_add_sync(0xffffffffu, dense);
    const unsigned e = __reduce_add_sync(0xffffffffu, evald);
    const unsigned s = __reduce_add_sync(0xffffffffu, staged);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctr->rays, (unsigned long long)r);
        atomicAdd(&ctr->dense_samples, (unsigned long long)d);
        atomicAdd(&ctr->evaluated_samples, (unsigned long long)e);
        atomicAdd(&ctr->bricks_staged, (unsigned long long)s);
    }
}

__global__ void __launch_bounds__(128) k_render_gather(const __grid_constant__ RenderLaunch L) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int i = blockIdx.x * 16 + (w & 1) * 8 + (l & 7);
    const int j = blockIdx.y * 8 + (w >> 1) * 4 + (l >> 3);
    const int cam = blockIdx.z;
    const bool inside = i < L.W && j < L.H;
    const VolumeDev& v = L.vol;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const float is[3] = {1.0f / v.s[0], 1.0f / v.s[1], 1.0f / v.s[2]};

    RayDev r;
    const bool hit = inside && setup_ray(L.cams[cam], L.W, L.H, i, j, v.n, v.s, L.tp.step_vox, r);
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    unsigned dense = 0, evald = 0;
    if (hit) {
        int k = 0, kstop = -1;
        while (k < r.ns) {
            const float kk = (float)k + 0.5f;
            int i0[3], bc[3];
            float f[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                cell_of(sample_u(r, q, kk), v.n[q], i0[q], f[q]);
                bc[q] = i0[q] >> 3;
            }
            const long long bi = brick_index(v, bc);
            if (L.skip && __ldg(v.empty + bi)) {
                k = brick_exit_k(r, bc, k, r.ns);
                continue;
            }
            const int base = ((i0[2] - kCells * bc[2]) * kEdge + (i0[1] - kCells * bc[1])) * kEdge +
                             (i0[0] - kCells * bc[0]);
            const long long boff = bi * kBrickVox;
            float fld[10];
            field_eval(GlobalLoad{v.bricks + boff}, base, f[0], f[1], f[2], fld);
            scale_field(fld, is);
            const float vval = v.vbricks ? value_eval(GlobalLoad{v.vbricks + boff}, base, f[0], f[1], f[2]) : 0.0f;
            float alpha, col[3];
            sample_optics(fld, vval, r.dir, L.tp, tf, inv_gmax, alpha, col);
            const float wgt = (1.0f - A) * alpha;  // Eqs. 5-6
            C0 = fmaf(col[0], wgt, C0);
            C1 = fmaf(col[1], wgt, C1);
            C2 = fmaf(col[2], wgt, C2);
            A += wgt;
            ++evald;
            if (A >= L.tp.et_threshold) {
                kstop = k;
                break;
            }
            ++k;
        }
        dense = kstop >= 0 ? (unsigned)(kstop + 1) : (unsigned)r.ns;
    }
    if (inside) {
        const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
        reinterpret_cast<float4*>(L.out)[pix] = make_float4(C0, C1, C2, A);
        if (L.ray_samples) {
            L.ray_samples[2 * pix] = dense;
            L.ray_samples[2 * pix + 1] = evald;
        }
    }
    if (L.counters) add_counters(L.counters, hit ? 1u : 0u, dense, evald, 0u);
}

}  // namespace

cudaError_t launch_render_gather(const RenderLaunch& L, cudaStream_t st) {
    dim3 grid((L.W + 15) / 16, (L.H + 7) / 8, L.n_cams);
    k_render_gather<<<grid, 128, 0, st>>>(L);
    return cudaGetLastError();
}

}  // namespace vr
