// vr_render.cu -- forward raymarch kernels (Sec. 2.4, Eqs. 4-6).
//
// k_render_gather: one thread per ray, a warp covers a packet_w x (32/packet_w)
// pixel packet (4 x 8 by default: 6 % faster than 8 x 4 or 16 x 2 at 1080p) and a
// CTA a 16x8 tile. Each lane walks its own samples front to back; per sample it
// reads its cell straight from HBM/L2 through L1 -- the 8 corners of the derived
// bricks (voxel-wise I, gradient, Hessian: three 16-byte loads per corner) when
// they were built, else the 56 weighted voxels of the 4x4x4 neighbourhood of the
// intensity bricks with the separable stencils -- evaluates Eq. 4 and the
// shading, and composites by Eqs. 5-6. Samples in bricks classified empty are
// skipped a brick at a time (bit-neutral: their opacity is exactly zero).
#include "vr_async.cuh"
#include "vr_march.cuh"

namespace vr {

namespace {

// Registers per thread: 64 for the derived-brick path (8 CTAs of 4 warps per SM:
// equal at 1080p, 2.5 % faster on the 8-view 512^2 workload than 72), 72 when it also
// records the ray state (CTAs of at most 4 warps, 7 per SM: 1.5 % faster than 80 at 6;
// 64 spills ~100 bytes), 80 for the stencils. CTAs of 2, 4 or 8 warps (tile_pixel).
template <bool kDerived, bool kState, int kBS>
__global__ void __launch_bounds__(kState ? 128 : 256, kDerived ? (kState ? 7 : 4) : (kState ? 6 : 3))
    k_render_gather(const __grid_constant__ RenderLaunch L) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int di, dj;
    tile_pixel(L.packet_w, L.tile_sx, w, l, di, dj);
    const int i = blockIdx.x * L.tile_w + di;
    const int j = blockIdx.y * L.tile_h + dj;
    const int cam = blockIdx.z;
    const bool inside = i < L.W && j < L.H;
    const VolumeDev& v = L.vol;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const float is[3] = {1.0f / v.s[0], 1.0f / v.s[1], 1.0f / v.s[2]};

    RayDev r;
    const bool hit = inside && setup_ray(L.cams[cam], L.rc, i, j, v.n, v.s, r);
    float4 px = make_float4(0.f, 0.f, 0.f, 0.f);
    unsigned dense = 0, evald = 0, shaded = 0, interp = 0;
    int kl = -1;
    float tl = 1.0f;
    if (hit)
        march_gather<kDerived, kState, false, true, kBS>(v, L.tp, tf, r, L.skip, inv_gmax, is, px, dense, evald,
                                                         shaded, interp, &kl, &tl);
    if (inside) {
        const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
        reinterpret_cast<float4*>(L.out)[pix] = px;
        if (kState) L.ray_state[pix] = make_float2(__int_as_float(kl), tl);
        if (L.ray_samples) {
            L.ray_samples[2 * pix] = dense;
            L.ray_samples[2 * pix + 1] = evald;
        }
    }
    if (L.counters) add_counters(L.counters, hit ? 1u : 0u, dense, evald, 0u, shaded, interp);
}

}  // namespace

template <int kBS>
void launch_gather_bs(const RenderLaunch& L, dim3 grid, int threads, cudaStream_t st) {
    const bool state = L.ray_state != nullptr;
    if (L.vol.dbricks) {
        if (state)
            k_render_gather<true, true, kBS><<<grid, threads, 0, st>>>(L);
        else
            k_render_gather<true, false, kBS><<<grid, threads, 0, st>>>(L);
    } else {
        if (state)
            k_render_gather<false, true, kBS><<<grid, threads, 0, st>>>(L);
        else
            k_render_gather<false, false, kBS><<<grid, threads, 0, st>>>(L);
    }
}

cudaError_t launch_render_gather(const RenderLaunch& L0, int warps, cudaStream_t st) {
    RenderLaunch L = L0;
    // the state-recording kernels are built for CTAs of at most 4 warps (72 registers,
    // 7 CTAs per SM); the image and the state do not depend on the CTA shape
    if (L.ray_state && warps > 4) warps = 4;
    const int tx = tile_packets_x(L.packet_w, warps);
    L.tile_w = tx * L.packet_w;
    L.tile_h = (warps / tx) * L.packet_h;
    L.tile_sx = __builtin_ctz(tx);
    dim3 grid((L.W + L.tile_w - 1) / L.tile_w, (L.H + L.tile_h - 1) / L.tile_h, L.n_cams);
    switch (L.vol.bs) {
        case 2: launch_gather_bs<2>(L, grid, warps * 32, st); break;
        case 4: launch_gather_bs<4>(L, grid, warps * 32, st); break;
        default: launch_gather_bs<3>(L, grid, warps * 32, st); break;
    }
    return cudaGetLastError();
}

}  // namespace vr

// ---------------------------------------------------------------------------
// k_render_staged: persistent warps pull 32-ray packets (packet_w x packet_h
// pixels) from an atomic work counter. A warp keeps one 12^3 brick (and, for
// the vesselness transfer function, its V brick) in shared memory. Each round
// every live lane skips empty bricks up to its next sample, the warp picks the
// front-most brick any live lane needs (smallest per-axis brick distance from
// the eye, a visibility order of the brick grid), one lane pulls it in with a
// bulk copy completing on an mbarrier, and all lanes whose next sample lies in
// that brick march through it from shared memory. Each lane still walks its own
// samples strictly front to back, so the result equals the gather kernel's
// bit for bit; the brick order only decides how often a brick is re-staged.
namespace vr {
namespace {

struct SmemLoad {
    const float* p;
    __device__ __forceinline__ float operator()(int o) const { return p[o]; }
};

__device__ __forceinline__ unsigned brick_key(const int b[3], const int e[3]) {
    const unsigned dx = min(abs(b[0] - e[0]), 1023), dy = min(abs(b[1] - e[1]), 1023), dz = min(abs(b[2] - e[2]), 1023);
    return (dz << 20) | (dy << 10) | dx;
}

__global__ void __launch_bounds__(256) k_render_staged(const __grid_constant__ RenderLaunch L) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nchan = L.vol.vbricks ? 2 : 1;
    const int per_warp = nchan * kBrickBytes + 128;
    unsigned char* my = smem_raw + (size_t)warp * per_warp;
    float* sbrick = reinterpret_cast<float*>(my);
    float* svbrick = reinterpret_cast<float*>(my + kBrickBytes);
    uint64_t* bar = reinterpret_cast<uint64_t*>(my + nchan * kBrickBytes);
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;

    const VolumeDev& v = L.vol;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const float is[3] = {1.0f / v.s[0], 1.0f / v.s[1], 1.0f / v.s[2]};
    const int ppx = L.packet_w, ppy = L.packet_h;
    unsigned staged = 0, rays_hit = 0, dense_tot = 0, eval_tot = 0;

    while (!failed) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(L.work_counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (unsigned)L.n_work) break;
        const int px = item % L.n_packets_x;
        const int py = (item / L.n_packets_x) % L.n_packets_y;
        const int cam = item / (L.n_packets_x * L.n_packets_y);
        const int i = px * ppx + lane % ppx, j = py * ppy + lane / ppx;
        const bool inside = i < L.W && j < L.H;
        const CamDev& cd = L.cams[cam];
        int eb[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) eb[q] = (int)floorf((cd.eye[q] / v.s[q] - 0.5f) / (float)kCells);

        RayDev r;
        bool live = inside && setup_ray(cd, L.rc, i, j, v.n, v.s, r);
        const bool hit = live;
        int k = 0, kstop = -1, cur = -1, bc[3] = {0, 0, 0};
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
        unsigned evald = 0;

        while (true) {
            // skip empty bricks up to this lane's next evaluated sample
            while (live && cur < 0) {
                if (k >= r.ns) {
                    live = false;
                    break;
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    int i0;
                    float f;
                    sample_cell(r, q, k, v.n[q], i0, f);
                    bc[q] = i0 >> 3;
                }
                if (!VR_CHECK(L.tp.status, (unsigned)bc[0] < (unsigned)v.nb[0] &&
                                               (unsigned)bc[1] < (unsigned)v.nb[1] &&
                                               (unsigned)bc[2] < (unsigned)v.nb[2])) {
                    live = false;
                    break;
                }
                const int bi = (int)brick_index(v, bc);
                if (L.skip && __ldg(v.empty + bi)) {
                    k = brick_exit_k(r, bc, kCells, k, r.ns);
                } else {
                    cur = bi;
                }
            }
            const unsigned key = live ? brick_key(bc, eb) : 0xffffffffu;
            const unsigned mk = __reduce_min_sync(0xffffffffu, key);
            if (mk == 0xffffffffu) break;
            const int leader = __ffs(__ballot_sync(0xffffffffu, key == mk)) - 1;
            const int sel = __shfl_sync(0xffffffffu, cur, leader);
            int sc[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) sc[q] = __shfl_sync(0xffffffffu, bc[q], leader);

            // stage brick `sel` (all lanes are done reading the previous one)
            __syncwarp();
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, nchan * kBrickBytes);
                bulk_g2s(sbrick, v.bricks + (size_t)sel * kBrickVox, kBrickBytes, bar);
                if (nchan == 2) bulk_g2s(svbrick, v.vbricks + (size_t)sel * kBrickVox, kBrickBytes, bar);
                ++staged;
            }
            const bool arrived = __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity));
            if (!arrived) {
                // the copy did not land within the budget: record it, give the copy one
                // more bounded wait so nothing is in flight when the warp leaves, stop.
                (void)mbar_wait_bounded(bar, parity);
                failed = true;
                if (lane == 0) atomicOr(L.status, kStatusTimeout);
                break;
            }
            parity ^= 1u;

            if (live && cur == sel) {
                while (true) {
                    int i0[3], b2[3];
                    float f[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sample_cell(r, q, k, v.n[q], i0[q], f[q]);
                        b2[q] = i0[q] >> 3;
                    }
                    if (b2[0] != sc[0] || b2[1] != sc[1] || b2[2] != sc[2]) {
                        cur = -1;
                        break;
                    }
                    const int base = ((i0[2] - kCells * sc[2]) * kEdge + (i0[1] - kCells * sc[1])) * kEdge +
                                     (i0[0] - kCells * sc[0]);
                    // the 4^3 stencil reads base + a + 12 b + 144 c, a, b, c in [0, 3]
                    if (!VR_CHECK(L.tp.status, base >= 0 && base + 3 * (1 + kEdge + kEdge * kEdge) < kBrickVox)) {
                        live = false;
                        break;
                    }
                    float fld[10];
                    field_eval(SmemLoad{sbrick}, base, f[0], f[1], f[2], fld);
                    scale_field(fld, is);
                    const float vval = nchan == 2 ? value_eval(SmemLoad{svbrick}, base, f[0], f[1], f[2]) : 0.0f;
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
                        live = false;
                        break;
                    }
                    if (++k >= r.ns) {
                        live = false;
                        break;
                    }
                }
            }
        }
        if (failed) break;
        const unsigned dense = hit ? (kstop >= 0 ? (unsigned)(kstop + 1) : (unsigned)r.ns) : 0u;
        if (inside) {
            const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
            reinterpret_cast<float4*>(L.out)[pix] = make_float4(C0, C1, C2, A);
            if (L.ray_samples) {
                L.ray_samples[2 * pix] = dense;
                L.ray_samples[2 * pix + 1] = evald;
            }
        }
        rays_hit += hit ? 1u : 0u;
        dense_tot += dense;
        eval_tot += evald;
    }
    if (L.counters) add_counters(L.counters, rays_hit, dense_tot, eval_tot, lane == 0 ? staged : 0u, eval_tot, eval_tot);
}

// k_render_staged_derived: the staged design on the derived bricks. Persistent
// warps pull packets as k_render_staged does; each warp keeps one derived skip brick
// ((B+1)^3 corners x 48 B: 6000 B for B = 4, 34,992 B for B = 8) in shared memory.
// Every round each live lane advances to its next sample outside empty bricks, the
// warp picks the front-most brick any live lane needs, one lane pulls it in with a
// bulk copy completing on an mbarrier (bounded wait), and the lanes whose next sample
// lies in it march through it reading the 8 corners of their cells from shared
// memory (cell bits and the transfer function still through L1). The warp leaves
// when a vote finds no live lane. Each lane walks its own samples front to back with
// the gather kernel's arithmetic (offset-order corner sums), so the image is the
// same bit for bit. No vesselness channel (mode 2 uses the gather kernels).
template <int kBS>
__global__ void __launch_bounds__(256, 3) k_render_staged_derived(const __grid_constant__ RenderLaunch L) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    constexpr int B = 1 << kBS, E = B + 1;
    constexpr int kFloats = E * E * E * kDerFloats;
    constexpr unsigned kBytes = kFloats * 4;  // a multiple of 16
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    unsigned char* my = smem_raw + (size_t)warp * (kBytes + 128);
    const float4* sbrick = reinterpret_cast<const float4*>(my);
    uint64_t* bar = reinterpret_cast<uint64_t*>(my + kBytes);
    if (lane == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncwarp();
    unsigned parity = 0;
    bool failed = false;
    const VolumeDev& v = L.vol;
    const TissueDev& tp = L.tp;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const int ppx = L.packet_w, ppy = L.packet_h;
    unsigned staged = 0, rays_hit = 0, dense_tot = 0, eval_tot = 0, shade_tot = 0, interp_tot = 0;

    while (!failed) {
        unsigned item = 0;
        if (lane == 0) item = atomicAdd(L.work_counter, 1u);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= (unsigned)L.n_work) break;
        const int px = item % L.n_packets_x;
        const int py = (item / L.n_packets_x) % L.n_packets_y;
        const int cam = item / (L.n_packets_x * L.n_packets_y);
        const int i = px * ppx + lane % ppx, j = py * ppy + lane / ppx;
        const bool inside = i < L.W && j < L.H;
        const CamDev& cd = L.cams[cam];
        int eb[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) eb[q] = (int)floorf((cd.eye[q] / v.s[q] - 0.5f) / (float)B);
        RayDev r;
        bool live = inside && setup_ray(cd, L.rc, i, j, v.n, v.s, r);
        const bool hit = live;
        int k = 0, kstop = -1, cur = -1, bc[3] = {0, 0, 0};
        float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
        unsigned ne = 0, nsh = 0, nip = 0;
        while (true) {
            while (live && cur < 0) {  // this lane's next sample outside empty bricks
                if (k >= r.ns) {
                    live = false;
                    break;
                }
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    int i0;
                    float f;
                    sample_cell(r, q, k, v.n[q], i0, f);
                    bc[q] = i0 >> kBS;
                }
                if (!VR_CHECK(tp.status, (unsigned)bc[0] < (unsigned)v.nb[0] && (unsigned)bc[1] < (unsigned)v.nb[1] &&
                                             (unsigned)bc[2] < (unsigned)v.nb[2])) {
                    live = false;
                    break;
                }
                const int bi = brick_index(v, bc);
                if (L.skip && __ldg(v.empty + bi))
                    k = brick_exit_k(r, bc, B, k, r.ns);
                else
                    cur = bi;
            }
            const unsigned key = live ? brick_key(bc, eb) : 0xffffffffu;
            const unsigned mk = __reduce_min_sync(0xffffffffu, key);
            if (mk == 0xffffffffu) break;  // warp vote: no live lane left
            const int leader = __ffs(__ballot_sync(0xffffffffu, key == mk)) - 1;
            const int sel = __shfl_sync(0xffffffffu, cur, leader);
            int sc[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) sc[q] = __shfl_sync(0xffffffffu, bc[q], leader);
            __syncwarp();  // every lane is done reading the previous brick
            if (lane == 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(bar, kBytes);
                bulk_g2s(my, v.dbricks + (size_t)sel * kFloats, kBytes, bar);
                ++staged;
            }
            const bool arrived = __all_sync(0xffffffffu, mbar_wait_bounded(bar, parity));
            if (!arrived) {
                (void)mbar_wait_bounded(bar, parity);  // nothing in flight when the warp leaves
                failed = true;
                if (lane == 0) atomicOr(L.status, kStatusTimeout);
                break;
            }
            parity ^= 1u;
            if (live && cur == sel) {
                while (true) {
                    int i0[3], b2[3];
                    float f[3];
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        sample_cell(r, q, k, v.n[q], i0[q], f[q]);
                        b2[q] = i0[q] >> kBS;
                    }
                    if (b2[0] != sc[0] || b2[1] != sc[1] || b2[2] != sc[2]) {
                        cur = -1;
                        break;
                    }
                    const int lx = i0[0] & (B - 1), ly = i0[1] & (B - 1), lz = i0[2] & (B - 1);
                    bool done_sample = false;
                    if (L.skip && v.cellmask) {
                        const int c = (((lz << kBS) + ly) << kBS) + lx;
                        if ((__ldg(v.cellmask + (size_t)sel * cell_words(kBS) + (c >> 5)) >> (c & 31)) & 1u)
                            done_sample = true;
                    }
                    if (!done_sample) {
                        ++nip;
                        float fld[10];
                        derived_channels_smem<0, 4>(sbrick, E, lx, ly, lz, f[0], f[1], f[2], fld);
                        if (tp.gk != 0.0f) {
                            derived_channels_smem<4, 6>(sbrick, E, lx, ly, lz, f[0], f[1], f[2], fld + 4);
                        } else {
#pragma unroll
                            for (int q = 4; q < 10; ++q) fld[q] = 0.0f;
                        }
                        SampleOptics o;
                        optics_tf(fld, 0.0f, tp, tf, inv_gmax, o);
                        if (o.c.w != 0.0f) {
                            optics_rest(fld, r.dir, tp, o);
                            ++nsh;
                            const float wgt = (1.0f - A) * o.alpha;  // Eqs. 5-6
                            C0 = fmaf(o.col[0], wgt, C0);
                            C1 = fmaf(o.col[1], wgt, C1);
                            C2 = fmaf(o.col[2], wgt, C2);
                            A += wgt;
                        }
                    }
                    ++ne;
                    if (A >= tp.et_threshold) {
                        kstop = k;
                        live = false;
                        break;
                    }
                    if (++k >= r.ns) {
                        live = false;
                        break;
                    }
                }
            }
        }
        if (failed) break;
        const unsigned dense = hit ? (kstop >= 0 ? (unsigned)(kstop + 1) : (unsigned)r.ns) : 0u;
        if (inside) {
            const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
            reinterpret_cast<float4*>(L.out)[pix] = make_float4(C0, C1, C2, A);
            if (L.ray_samples) {
                L.ray_samples[2 * pix] = dense;
                L.ray_samples[2 * pix + 1] = ne;
            }
        }
        rays_hit += hit ? 1u : 0u;
        dense_tot += dense;
        eval_tot += ne;
        shade_tot += nsh;
        interp_tot += nip;
    }
    if (L.counters) add_counters(L.counters, rays_hit, dense_tot, eval_tot, lane == 0 ? staged : 0u, shade_tot,
                                 interp_tot);
}

template <int kBS>
int staged_derived_bytes() {
    constexpr int E = (1 << kBS) + 1;
    return E * E * E * kDerFloats * 4 + 128;
}

}  // namespace

int staged_derived_smem_bytes(int warps_per_block, int bs) {
    return warps_per_block * (bs == 2 ? staged_derived_bytes<2>() : staged_derived_bytes<3>());
}

cudaError_t staged_derived_config(int warps_per_block, int bs, int* ctas_per_sm) {
    const int smem = staged_derived_smem_bytes(warps_per_block, bs);
    cudaError_t e;
    if (bs == 2) {
        e = cudaFuncSetAttribute(k_render_staged_derived<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 staged_derived_smem_bytes(8, 2));
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_render_staged_derived<2>,
                                                             warps_per_block * 32, smem);
    }
    e = cudaFuncSetAttribute(k_render_staged_derived<3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             staged_derived_smem_bytes(6, 3));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_render_staged_derived<3>, warps_per_block * 32,
                                                         smem);
}

cudaError_t launch_render_staged_derived(const RenderLaunch& L, int warps_per_block, int ctas, cudaStream_t st) {
    const int smem = staged_derived_smem_bytes(warps_per_block, L.vol.bs);
    if (L.vol.bs == 2)
        k_render_staged_derived<2><<<ctas, warps_per_block * 32, smem, st>>>(L);
    else
        k_render_staged_derived<3><<<ctas, warps_per_block * 32, smem, st>>>(L);
    return cudaGetLastError();
}

int staged_smem_bytes(int warps_per_block, bool vessel) {
    return warps_per_block * ((vessel ? 2 : 1) * kBrickBytes + 128);
}

cudaError_t launch_render_staged(const RenderLaunch& L, int warps_per_block, int ctas, cudaStream_t st) {
    const int smem = staged_smem_bytes(warps_per_block, L.vol.vbricks != nullptr);
    k_render_staged<<<ctas, warps_per_block * 32, smem, st>>>(L);
    return cudaGetLastError();
}

cudaError_t staged_config(int warps_per_block, bool vessel, int* ctas_per_sm) {
    const int smem = staged_smem_bytes(warps_per_block, vessel);
    // One limit for every configuration (the largest), so a later call can never lower it.
    cudaError_t e = cudaFuncSetAttribute(k_render_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         staged_smem_bytes(8, true));
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_render_staged, warps_per_block * 32, smem);
}

}  // namespace vr
