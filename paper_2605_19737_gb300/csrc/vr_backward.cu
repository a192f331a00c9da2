// vr_backward.cu -- adjoint raymarch: gradients of a loss on the rendered image
// with respect to the transfer-function entries, the tissue uniforms
// (gamma, ka, kd, ks, opacity_scale) and the normalised voxel intensities.
//
// One thread per ray (the forward kernel's warp packets, 4 warps per CTA). Per ray:
//   1. the ray's stopping sample k_stop and the transmittance T in front of it, from
//      the forward's ray state, or by a forward re-march with the forward kernel's
//      exact arithmetic (empty bricks skipped);
//   2. reverse sweep over every sample k = k_stop .. 0, the lanes of a warp in step
//      by sample index (no skipping: the opacity entries of the transfer function
//      receive gradient from samples whose opacity is zero) with no stored samples:
//      the sample is re-evaluated, T_k = T_{k+1} / (1 - alpha_k) (exact in real
//      arithmetic and well conditioned because early termination keeps
//      1 - alpha_k >= 1 - et before the last sample), R_k = alpha_k c_k +
//      (1 - alpha_k) R_{k+1} and P_k = prod_{j>k} (1 - alpha_j) are carried
//      backwards, and
//        dL/dalpha_k = T_k (<dL/dC, c_k - R_{k+1}> + dL/dA P_k),
//        dL/dc_k     = T_k alpha_k dL/dC              (Eqs. 5-6 differentiated);
//   3. sample_adjoint / field_adjoint_scatter chain these to the parameters.
// Transfer-function gradients are accumulated per lane while its samples stay in
// one lookup cell, then added with 16-byte vector atomics into private global
// copies of the gradient (one 16-float record per cell; CTA c into copy c % n) that
// k_sum_copies gathers afterwards -- contended atomics on one table cost 10x the
// rest of the kernel, and a shared-memory table per CTA 1.6x (1D) to 1.8x (2D
// opacities) the copies. Voxel gradients: on the derived bricks, per-voxel channel
// gradients (vector atomics, neighbouring lanes in one cell merged, corner order
// rotated) and a gather pass through the stencil transposes; otherwise scalar
// global atomics on the voxels. Uniform gradients are warp-reduced first.
#include "vr_adjoint.cuh"

namespace vr {

namespace {

struct GLoad {
    const float* __restrict__ p;
    __device__ __forceinline__ float operator()(int o) const { return __ldg(p + o); }
};

__device__ __forceinline__ long long bidx(const VolumeDev& v, const int b[3]) {
    return ((long long)b[2] * v.nb[1] + b[1]) * v.nb[0] + b[0];
}

// The sample field, from the derived bricks (voxel-wise derivatives) or by the
// per-sample stencils -- the same linear map of the voxels, either way. kHessian:
// the Hessian channels are read even without a curvature term (gamma = 0): the
// forward values do not need them then, but dL/dgamma = sum dL/dw kappa / kappa_ref
// does.
// bi: the skip brick of the sample's cell (derived bricks); sbi, base: its storage
// brick and the stencil origin in it (intensity bricks).
template <bool kDerived, bool kHessian, int kBS>
__device__ __forceinline__ void eval_field(const VolumeDev& v, const TissueDev& tp, long long bi, long long sbi,
                                           const int i0[3], int base, const float f[3], const float is[3],
                                           float fld[10]) {
    if (kDerived) {
        const float4* brick = reinterpret_cast<const float4*>(v.dbricks + bi * der_brick_floats(kBS));
        const int m = (1 << kBS) - 1, E = m + 2;
        derived_channels<true, 0, 4>(brick, E, i0[0] & m, i0[1] & m, i0[2] & m, f[0], f[1], f[2], fld);
        if (kHessian)
            derived_channels<true, 4, 6>(brick, E, i0[0] & m, i0[1] & m, i0[2] & m, f[0], f[1], f[2], fld + 4);
        else
            load_hessian<true>(tp, brick, E, i0[0] & m, i0[1] & m, i0[2] & m, f, fld);
    } else {
        field_eval(GLoad{v.bricks + sbi * kBrickVox}, base, f[0], f[1], f[2], fld);
        scale_field(fld, is);
    }
}

// Adjoint of the derived-field interpolation: the sample's field gradient dfs (I, g, H in the
// derived channels' mm units), trilinearly weighted, into the per-voxel channel
// gradients of the cell's 8 corners -- up to three vector reductions per corner,
// the Hessian ones only when the sample has Hessian gradients (a curvature term):
// without one that removes two thirds of the reduction traffic (8-view 512^2
// backward 36 -> 27 ms).
// Per-voxel channel gradients in three planes: (I, gx, gy, gz) float4 [nvox],
// (Hxx, Hyy, Hzz, Hxy) float4 [nvox], (Hxz, Hyz) float2 [nvox]. Every vector
// reduction then covers one aligned 16- or 8-byte piece, and x-neighbouring voxels'
// pieces share sectors (1080p backward 16.2 -> 14.1 ms against 48-byte records).
// Corner order: a warp's reduction to one address is applied one lane at a time
// (one L1 wavefront per lane: 32 lanes on one address cost 32 wavefronts, on 32
// consecutive addresses one), and the lanes of a warp that scatter in the same
// step are often in the same cell. Each lane therefore starts at the corner given
// by its rank among the lanes in its cell, so that up to 8 of them hit 8 different
// voxels in each reduction instruction. The rank only orders the additions.
// Before that, horizontally neighbouring lanes 2m and 2m + 1 whose samples lie in
// the same cell merge: the even lane receives the odd one's fractions and field
// gradient (13 shuffles) and adds both samples' weighted gradients in each
// reduction, the odd lane issues none (1080p backward 12.1 -> 10.4 ms; at 512^2, where
// fewer neighbours share a cell, within 1 %); lanes left unmerged then pair the same
// way with their vertical neighbour, lane ^ ymask (the packet width): 10.4 -> 10.3 ms.
// A lane adds at most two samples.
// Float index of voxel p's channel ch (0..9).
__device__ __forceinline__ long long chan_index(long long p, long long nvox, int ch) {
    return ch < 4 ? 4 * p + ch : (ch < 8 ? 4 * nvox + 4 * p + (ch - 4) : 8 * nvox + 2 * p + (ch - 8));
}

__device__ __forceinline__ void scatter_channels(float* __restrict__ dgrad, const int n[3], const int i0[3],
                                                 const float f[3], const float dfs[10], int ymask) {
    const long long nvox = (long long)n[0] * n[1] * n[2];
    bool any = false, hess = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) any |= dfs[q] != 0.0f;
#pragma unroll
    for (int q = 4; q < 10; ++q) hess |= dfs[q] != 0.0f;
    if (!any && !hess) return;
    const long long nxy = (long long)n[0] * n[1];
    const long long p0 = (long long)i0[2] * nxy + (long long)i0[1] * n[0] + i0[0];
    // lanes 2m and 2m + 1 that scatter into the same cell: the even lane adds both
    // samples' weighted gradients, the odd one issues nothing
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31;
    const unsigned lo = (unsigned)p0, hi = (unsigned)(p0 >> 32);
    const unsigned plo = __shfl_xor_sync(act, lo, 1), phi = __shfl_xor_sync(act, hi, 1);
    float pf[3], pd[10];
#pragma unroll
    for (int q = 0; q < 3; ++q) pf[q] = __shfl_xor_sync(act, f[q], 1);
#pragma unroll
    for (int q = 0; q < 10; ++q) pd[q] = __shfl_xor_sync(act, dfs[q], 1);
    int phess_v = __shfl_xor_sync(act, (int)hess, 1);
    bool merged = ((act >> (lane ^ 1)) & 1u) && plo == lo && phi == hi;
    if (merged && (lane & 1)) return;
    // second round: lanes left unmerged pair with their vertical neighbour lane ^ ymask
    {
        const unsigned act2 = __activemask();
        const unsigned qlo = __shfl_xor_sync(act2, lo, ymask), qhi = __shfl_xor_sync(act2, hi, ymask);
        const int qfree = __shfl_xor_sync(act2, (int)!merged, ymask);
        float qf[3], qd[10];
#pragma unroll
        for (int q = 0; q < 3; ++q) qf[q] = __shfl_xor_sync(act2, f[q], ymask);
#pragma unroll
        for (int q = 0; q < 10; ++q) qd[q] = __shfl_xor_sync(act2, dfs[q], ymask);
        const int qhess = __shfl_xor_sync(act2, (int)hess, ymask);
        const bool my = !merged && qfree && ((act2 >> (lane ^ ymask)) & 1u) && qlo == lo && qhi == hi;
        if (my && (lane & ymask)) return;
        if (my) {
            merged = true;
#pragma unroll
            for (int q = 0; q < 3; ++q) pf[q] = qf[q];
#pragma unroll
            for (int q = 0; q < 10; ++q) pd[q] = qd[q];
            phess_v = qhess;
        }
    }
    const bool h = hess || (merged && phess_v);
    const unsigned same = __match_any_sync(__activemask(), lo);
    const int rot = __popc(same & ((1u << lane) - 1u)) & 7;
    // instruction i scatters corner i ^ rot: per axis the two factors and offsets
    // are swapped once when that bit of rot is set, so that every corner's weight,
    // ((dx ? fx : 1 - fx) * (dy ? ...)) * (dz ? ...), and address are fixed registers
    const bool sx = rot & 1, sy = (rot >> 1) & 1, sz = (rot >> 2) & 1;
    const float gx = 1.0f - f[0], gy = 1.0f - f[1], gz = 1.0f - f[2];
    const float ax[2] = {sx ? f[0] : gx, sx ? gx : f[0]}, ay[2] = {sy ? f[1] : gy, sy ? gy : f[1]},
                az[2] = {sz ? f[2] : gz, sz ? gz : f[2]};
    const float qx = 1.0f - pf[0], qy = 1.0f - pf[1], qz = 1.0f - pf[2];
    const float bx2[2] = {sx ? pf[0] : qx, sx ? qx : pf[0]}, by2[2] = {sy ? pf[1] : qy, sy ? qy : pf[1]},
                bz2[2] = {sz ? pf[2] : qz, sz ? qz : pf[2]};
    const int nx = n[0], nxy32 = n[0] * n[1];  // < 2^23 for dims <= 2048
    const int ox[2] = {sx ? 1 : 0, sx ? 0 : 1}, oy[2] = {sy ? nx : 0, sy ? 0 : nx},
              oz[2] = {sz ? nxy32 : 0, sz ? 0 : nxy32};
    float4* const c0 = reinterpret_cast<float4*>(dgrad + chan_index(p0, nvox, 0));
    float4* const c1 = reinterpret_cast<float4*>(dgrad + chan_index(p0, nvox, 4));
    float2* const c2 = reinterpret_cast<float2*>(dgrad + chan_index(p0, nvox, 8));
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int ix = i & 1, iy = (i >> 1) & 1, iz = i >> 2;
        const float w = (ax[ix] * ay[iy]) * az[iz];
        const float pw = merged ? (bx2[ix] * by2[iy]) * bz2[iz] : 0.0f;
        if (w == 0.0f && pw == 0.0f) continue;
        const int off = ox[ix] + oy[iy] + oz[iz];
        float4 g0;
        mul2(w, w, dfs[0], dfs[1], g0.x, g0.y);
        mul2(w, w, dfs[2], dfs[3], g0.z, g0.w);
        fma2(pw, pd[0], pd[1], g0.x, g0.y);
        fma2(pw, pd[2], pd[3], g0.z, g0.w);
        atomicAdd(c0 + off, g0);
        if (h) {
            float4 g1;
            float2 g2;
            mul2(w, w, dfs[4], dfs[5], g1.x, g1.y);
            mul2(w, w, dfs[6], dfs[7], g1.z, g1.w);
            mul2(w, w, dfs[8], dfs[9], g2.x, g2.y);
            fma2(pw, pd[4], pd[5], g1.x, g1.y);
            fma2(pw, pd[6], pd[7], g1.z, g1.w);
            fma2(pw, pd[8], pd[9], g2.x, g2.y);
            atomicAdd(c1 + off, g1);
            atomicAdd(c2 + off, g2);
        }
    }
}

// Voxel p's channels read I at clamp(p +- 1) per axis. For voxel v, the p whose
// "+1" (s = 0) or "-1" (s = 1) neighbour along an axis of size nn clamps to v.
__device__ __forceinline__ int clamp_sources(int v, int nn, int sgn, int out[2]) {
    int m = 0;
    if (sgn == 0) {  // clamp(p + 1) == v
        if (v >= 1) out[m++] = v - 1;
        if (v == nn - 1) out[m++] = v;
    } else {  // clamp(p - 1) == v
        if (v <= nn - 2) out[m++] = v + 1;
        if (v == 0) out[m++] = v;
    }
    return m;
}

// dL/dI[v] from the channel gradients: the transpose of the derived channels'
// clamp-to-edge difference stencils (I; g_a = (I[p+a] - I[p-a]) / (2 s_a);
// H_aa = (I[p+a] - 2 I[p] + I[p-a]) / s_a^2; H_ab = the four (p +- a +- b)
// corners / (4 s_a s_b)), gathered per voxel (no atomics).
__global__ void __launch_bounds__(256) k_channels_to_voxels(const float* __restrict__ G, int nx, int ny, int nz,
                                                            float sx, float sy, float sz, float* __restrict__ dvol) {
    const long long nvox = (long long)nx * ny * nz;
    const int nn[3] = {nx, ny, nz};
    const float sp[3] = {sx, sy, sz};
    const int hidx[3][3] = {{4, 7, 8}, {7, 5, 9}, {8, 9, 6}};  // channel of H_ab
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nvox;
         e += (long long)gridDim.x * blockDim.x) {
        const int v[3] = {(int)(e % nx), (int)((e / nx) % ny), (int)(e / ((long long)nx * ny))};
        auto at = [&](const int p[3], int ch) {
            return __ldg(G + chan_index(((long long)p[2] * ny + p[1]) * nx + p[0], nvox, ch));
        };
        float acc = at(v, 0);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float cg = 0.5f / sp[a], ch = 1.0f / (sp[a] * sp[a]);
            acc -= 2.0f * ch * at(v, 4 + a);
#pragma unroll
            for (int sg = 0; sg < 2; ++sg) {
                int src[2];
                const int m = clamp_sources(v[a], nn[a], sg, src);
                for (int u = 0; u < m; ++u) {
                    int p[3] = {v[0], v[1], v[2]};
                    p[a] = src[u];
                    acc += (sg == 0 ? cg : -cg) * at(p, 1 + a) + ch * at(p, 4 + a);
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
#pragma unroll
            for (int b = a + 1; b < 3; ++b) {
                const float cm = 0.25f / (sp[a] * sp[b]);
#pragma unroll
                for (int sa = 0; sa < 2; ++sa) {
#pragma unroll
                    for (int sb = 0; sb < 2; ++sb) {
                        int pa[2], pb[2];
                        const int ma = clamp_sources(v[a], nn[a], sa, pa), mb = clamp_sources(v[b], nn[b], sb, pb);
                        const float sgn = (sa == sb) ? cm : -cm;
                        for (int ua = 0; ua < ma; ++ua)
                            for (int ub = 0; ub < mb; ++ub) {
                                int p[3] = {v[0], v[1], v[2]};
                                p[a] = pa[ua];
                                p[b] = pb[ub];
                                acc += sgn * at(p, hidx[a][b]);
                            }
                    }
                }
            }
        }
        dvol[e] = acc;
    }
}

// 4 resident CTAs per SM (<= 128 registers): measured 1 ms faster at 1080p than
// the 3 that the unbounded register count allows.
// Derived bricks without a curvature term (gamma = 0): with kLazyHessian a sample
// reads the Hessian only when its opacity entry is non-zero (for dL/dgamma); with
// kNoHessian, when no uniform gradient is wanted, never.
// kBS: log2 of the skip-brick edge (2, 3, 4), fixed at compile time.
template <bool kDerived, bool kLazyHessian, bool kNoHessian, int kBS>
__global__ void __launch_bounds__(128, 4) k_render_backward(const __grid_constant__ BackwardLaunch B) {
    const RenderLaunch& L = B.r;
    const size_t ncell = (size_t)L.tp.tf_w * L.tp.tf_h * kTfCellFloats;
    // one of n_copies private global copies of the gradient, so that CTAs working on
    // the same hot entries do not serialise on one address
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    TfGradSink sink(B.dtf_copies + (size_t)(cta % B.n_copies) * ncell, L.tp.tf_h > 1);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    int di, dj;
    tile_pixel(L.packet_w, __ffs(tile_packets_x(L.packet_w, 4)) - 1, w, l, di, dj);
    const int i = blockIdx.x * 16 + di;
    const int j = blockIdx.y * 8 + dj;
    const int cam = blockIdx.z;
    const bool inside = i < L.W && j < L.H;
    const VolumeDev& v = L.vol;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const float is[3] = {1.0f / v.s[0], 1.0f / v.s[1], 1.0f / v.s[2]};
    // the reverse sweep divides by 1 - alpha: stop where A reaches 1 even when early termination is off
    const float et = fminf(L.tp.et_threshold, 1.0f);
    ParamGrad dp{0.f, 0.f, 0.f, 0.f, 0.f};

    RayDev r;
    const bool hit = inside && setup_ray(L.cams[cam], L.rc, i, j, v.n, v.s, r);
    float4 g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int kstop = -1;  // the ray's last sample (-1: none)
    float Tk = 1.0f;
    if (hit) {
        const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
        g4 = __ldg(reinterpret_cast<const float4*>(B.dl_drgba) + pix);
        // 1. the ray's last sample and the transmittance in front of it: recorded by the
        // forward render (ray_state), or re-marched forward here
        kstop = r.ns - 1;
        if (L.ray_state) {
            const float2 st = __ldg(L.ray_state + pix);
            kstop = __float_as_int(st.x);
            Tk = st.y;
            if (!VR_CHECK(L.tp.status, kstop >= -1 && kstop < r.ns)) kstop = -1;  // a state of another image
        } else {
            float A = 0.f, A_prev = 0.f;
            int k = 0, klast = -1;
            while (k < r.ns) {
                int i0[3], bc[3];
                float f[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    sample_cell(r, q, k, v.n[q], i0[q], f[q]);
                    bc[q] = i0[q] >> kBS;
                }
                if (!VR_CHECK(L.tp.status, (unsigned)i0[0] <= (unsigned)(v.n[0] - 2) &&
                                               (unsigned)i0[1] <= (unsigned)(v.n[1] - 2) &&
                                               (unsigned)i0[2] <= (unsigned)(v.n[2] - 2)))
                    break;
                const long long bi = bidx(v, bc);
                if (L.skip && __ldg(v.empty + bi)) {
                    k = brick_exit_k(r, bc, 1 << kBS, k, r.ns);
                    continue;
                }
                int base;
                const long long sbi = storage_brick(v, i0, base);
                float fld[10];
                eval_field<kDerived, false, kBS>(v, L.tp, bi, sbi, i0, base, f, is, fld);
                const float vval =
                    v.vbricks ? value_eval(GLoad{v.vbricks + sbi * kBrickVox}, base, f[0], f[1], f[2]) : 0.f;
                float alpha, col[3];
                sample_optics(fld, vval, r.dir, L.tp, tf, inv_gmax, alpha, col);
                const float wgt = (1.0f - A) * alpha;  // as the forward kernel composites
                A_prev = A;
                A += wgt;
                klast = k;
                if (A >= et) {
                    kstop = k;
                    break;
                }
                ++k;
            }
            // transmittance before the stopping sample (1 when no sample had opacity)
            Tk = (klast == kstop) ? 1.0f - A_prev : 1.0f - A;
        }
    }
    {
            float Tk1 = Tk, R0 = 0.f, R1 = 0.f, R2 = 0.f, P = 1.0f;
            const float dC[3] = {g4.x, g4.y, g4.z};
            // 2. reverse sweep, the lanes of a warp in step: at iteration kr every lane
            // whose ray reaches that far works on its sample kr, so neighbouring rays sit
            // at nearly the same depth and their reads and reductions hit the same cells
            const int kmax = __reduce_max_sync(0xffffffffu, kstop);
            // the position of sample kr, u0 + kr du, carried down by exact integer steps
            long long U[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) U[q] = hit ? r.u0[q] + (long long)kmax * r.du[q] : 0ll;
            for (int kr = kmax; kr >= 0; --kr, U[0] -= r.du[0], U[1] -= r.du[1], U[2] -= r.du[2]) {
                if (kr > kstop) continue;
                int i0[3], bc[3];
                float f[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    cell_at(U[q], v.n[q], i0[q], f[q]);
                    bc[q] = i0[q] >> kBS;
                }
                // No skipping here: a sample in an empty brick has alpha = 0, but its lookup
                // still gives the opacity entries it reads a non-zero gradient.
                if (!VR_CHECK(L.tp.status, (unsigned)i0[0] <= (unsigned)(v.n[0] - 2) &&
                                               (unsigned)i0[1] <= (unsigned)(v.n[1] - 2) &&
                                               (unsigned)i0[2] <= (unsigned)(v.n[2] - 2)))
                    continue;
                const long long bi = bidx(v, bc);
                int base;
                const long long sbi = storage_brick(v, i0, base);
                float fld[10];
                const float vval =
                    v.vbricks ? value_eval(GLoad{v.vbricks + sbi * kBrickVox}, base, f[0], f[1], f[2]) : 0.f;
                SampleOptics so;
                if (kLazyHessian) {
                    // I and the gradient, the table lookup, then the Hessian, which without
                    // a curvature term only dL/dgamma needs -- and not at a zero opacity
                    // entry (dL/dw = 0 there, and w = 1 whatever kappa)
                    const float4* brick = reinterpret_cast<const float4*>(v.dbricks + bi * der_brick_floats(kBS));
                    const int m = (1 << kBS) - 1, E = m + 2;
                    derived_channels<true, 0, 4>(brick, E, i0[0] & m, i0[1] & m, i0[2] & m, f[0], f[1], f[2], fld);
                    optics_tf(fld, vval, L.tp, tf, inv_gmax, so);
                    if (!kNoHessian && so.c.w != 0.0f) {
                        derived_channels<true, 4, 6>(brick, E, i0[0] & m, i0[1] & m, i0[2] & m, f[0], f[1], f[2],
                                                     fld + 4);
                    } else {
#pragma unroll
                        for (int q = 4; q < 10; ++q) fld[q] = 0.0f;
                    }
                    optics_rest(fld, r.dir, L.tp, so);
                } else {
                    eval_field<kDerived, true, kBS>(v, L.tp, bi, sbi, i0, base, f, is, fld);
                    optics_core(fld, vval, r.dir, L.tp, tf, inv_gmax, so);
                }
                const float alpha = so.alpha, col[3] = {so.col[0], so.col[1], so.col[2]};
                // T_k = T_{k+1} / (1 - alpha_k); Tk still holds T_{k+1} here, which a zero
                // alpha leaves unchanged (x / 1 = x), so the division is skipped then
                if (kr != kstop && alpha != 0.0f) Tk = Tk1 / (1.0f - alpha);
                const float da = Tk * (fmaf(dC[0], col[0] - R0, fmaf(dC[1], col[1] - R1, dC[2] * (col[2] - R2))) +
                                       g4.w * P);
                if (so.c.w == 0.0f) {
                    // zero opacity entry: alpha = 0 exactly, so only the table's opacity
                    // entries at the lookup receive a gradient (the one-sided derivative of
                    // the clamp at 0); colour, uniforms and field gradients are all zero
                    float dal = da;
                    if (L.tp.alpha_exp > 0.0f) dal *= L.tp.alpha_exp;
                    const float dr[4] = {0.f, 0.f, 0.f,
                                         (so.raw >= 0.0f && so.raw <= 1.0f) ? dal * L.tp.opacity_scale * so.mg * so.wk
                                                                            : 0.0f};
                    if (L.tp.tf_h == 1)
                        sink.add_cell(so.j, 1.0f - so.t, so.t, 0.0f, 0.0f, dr);
                    else
                        sink.add_cell(so.k * L.tp.tf_w + so.j, (1.0f - so.q) * (1.0f - so.t), (1.0f - so.q) * so.t,
                                      so.q * (1.0f - so.t), so.q * so.t, dr);
                    Tk1 = Tk;
                    continue;
                }
                const float ta = Tk * alpha;
                const float dc[3] = {ta * dC[0], ta * dC[1], ta * dC[2]};
                float dfs[10];
                sample_adjoint(fld, so, r.dir, L.tp, inv_gmax, da, dc, sink, dp, dfs);
                if (kDerived && B.dgrad) {
                    scatter_channels(B.dgrad, v.n, i0, f, dfs, L.packet_w);
                } else if (B.dvol) {
                    const int x0 = i0[0] - 1, y0 = i0[1] - 1, z0 = i0[2] - 1;
                    const int nx = v.n[0], ny = v.n[1], nz = v.n[2];
                    float* dv = B.dvol;
                    field_adjoint_scatter(dfs, is, f[0], f[1], f[2], [&](int a, int b, int c, float g) {
                        if (g == 0.0f) return;
                        const int x = min(max(x0 + a, 0), nx - 1), y = min(max(y0 + b, 0), ny - 1),
                                  z = min(max(z0 + c, 0), nz - 1);
                        atomicAdd(dv + ((long long)z * ny + y) * nx + x, g);
                    });
                }
                R0 = fmaf(alpha, col[0], (1.0f - alpha) * R0);
                R1 = fmaf(alpha, col[1], (1.0f - alpha) * R1);
                R2 = fmaf(alpha, col[2], (1.0f - alpha) * R2);
                P *= (1.0f - alpha);
                Tk1 = Tk;
            }
    }
    sink.flush();
    // uniform gradients: warp sums, one atomic per warp and parameter
    float pv[5] = {dp.gamma, dp.ka, dp.kd, dp.ks, dp.os};
#pragma unroll
    for (int e = 0; e < 5; ++e) {
#pragma unroll
        for (int o = 16; o; o >>= 1) pv[e] += __shfl_xor_sync(0xffffffffu, pv[e], o);
    }
    if (l == 0 && B.dparams) {
#pragma unroll
        for (int e = 0; e < 5; ++e)
            if (pv[e] != 0.0f) atomicAdd(B.dparams + e, pv[e]);
    }
}

// Brick-synchronous variant of the reverse sweep. Phase 1 (the forward
// re-march) is per lane as above. In phase 2 the warp repeatedly picks the
// farthest brick (largest per-axis brick distance from the eye) that a lane's
// next reverse sample lies in; the lanes in that brick sweep their samples in
// it back to front, adding voxel gradients into a 12^3 shared-memory block with
// shared-memory atomics; the warp then adds the touched part of the block to the
// global gradient and clears it. Each lane still sweeps its own samples in
// strictly decreasing order, so every sample sees exactly the arithmetic of
// k_render_backward; only the order of the floating-point additions into the
// voxel gradient differs.
__device__ __forceinline__ unsigned far_key(const int b[3], const int e[3]) {
    const unsigned dx = min(abs(b[0] - e[0]), 1023), dy = min(abs(b[1] - e[1]), 1023), dz = min(abs(b[2] - e[2]), 1023);
    return (dz << 20) | (dy << 10) | dx;
}

__global__ void __launch_bounds__(128) k_render_backward_staged(const __grid_constant__ BackwardLaunch B) {
    extern __shared__ float smem[];
    const RenderLaunch& L = B.r;
    const size_t ncell = (size_t)L.tp.tf_w * L.tp.tf_h * kTfCellFloats;
    const int warp = threadIdx.x >> 5, l = threadIdx.x & 31;
    float* acc = smem + warp * kBrickVox;  // this warp's 12^3 block
    for (int e = l; e < kBrickVox; e += 32) acc[e] = 0.0f;
    __syncthreads();
    const int cta = (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    TfGradSink sink(B.dtf_copies + (size_t)(cta % B.n_copies) * ncell, L.tp.tf_h > 1);
    const int i = blockIdx.x * 16 + (warp & 1) * 8 + (l & 7);
    const int j = blockIdx.y * 8 + (warp >> 1) * 4 + (l >> 3);
    const int cam = blockIdx.z;
    const bool inside = i < L.W && j < L.H;
    const VolumeDev& v = L.vol;
    const float4* tf = reinterpret_cast<const float4*>(L.tf);
    const float gmax = __ldg(&v.vc->gmax);
    const float inv_gmax = gmax > 0.0f ? 1.0f / gmax : 0.0f;
    const float is[3] = {1.0f / v.s[0], 1.0f / v.s[1], 1.0f / v.s[2]};
    const float et = fminf(L.tp.et_threshold, 1.0f);
    const CamDev& cd = L.cams[cam];
    int eb[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) eb[q] = (int)floorf((cd.eye[q] / v.s[q] - 0.5f) / (float)kCells);
    ParamGrad dp{0.f, 0.f, 0.f, 0.f, 0.f};

    RayDev r;
    bool live = inside && setup_ray(cd, L.rc, i, j, v.n, v.s, r);
    float4 g4 = make_float4(0.f, 0.f, 0.f, 0.f);
    int kr = -1;
    float Tk = 1.0f, Tk1 = 1.0f, R0 = 0.f, R1 = 0.f, R2 = 0.f, P = 1.0f;
    int kstop = -1;
    if (live) {
        const long long pix = ((long long)(L.cam_offset + cam) * L.H + j) * L.W + i;
        g4 = __ldg(reinterpret_cast<const float4*>(B.dl_drgba) + pix);
        float A = 0.f, A_prev = 0.f;
        int k = 0, klast = -1;
        kstop = r.ns - 1;
        while (k < r.ns) {
            int i0[3], bc[3];
            float f[3];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                sample_cell(r, q, k, v.n[q], i0[q], f[q]);
                bc[q] = i0[q] >> 3;
            }
            if (!VR_CHECK(L.tp.status, (unsigned)i0[0] <= (unsigned)(v.n[0] - 2) &&
                                           (unsigned)i0[1] <= (unsigned)(v.n[1] - 2) &&
                                           (unsigned)i0[2] <= (unsigned)(v.n[2] - 2)))
                break;
            const long long bi = bidx(v, bc);
            if (L.skip && __ldg(v.empty + bi)) {
                k = brick_exit_k(r, bc, kCells, k, r.ns);
                continue;
            }
            const int base = ((i0[2] - kCells * bc[2]) * kEdge + (i0[1] - kCells * bc[1])) * kEdge +
                             (i0[0] - kCells * bc[0]);
            float fld[10];
            field_eval(GLoad{v.bricks + bi * kBrickVox}, base, f[0], f[1], f[2], fld);
            scale_field(fld, is);
            const float vval = v.vbricks ? value_eval(GLoad{v.vbricks + bi * kBrickVox}, base, f[0], f[1], f[2]) : 0.f;
            float alpha, col[3];
            sample_optics(fld, vval, r.dir, L.tp, tf, inv_gmax, alpha, col);
            A_prev = A;
            A += (1.0f - A) * alpha;
            klast = k;
            if (A >= et) {
                kstop = k;
                break;
            }
            ++k;
        }
        Tk = (klast == kstop) ? 1.0f - A_prev : 1.0f - A;
        Tk1 = Tk;
        kr = kstop;
    }
    const float dC[3] = {g4.x, g4.y, g4.z};
    while (true) {
        // brick of this lane's next reverse sample
        int i0[3] = {0, 0, 0}, bc[3] = {0, 0, 0};
        float f[3] = {0.f, 0.f, 0.f};
        if (live) {
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                sample_cell(r, q, kr, v.n[q], i0[q], f[q]);
                bc[q] = i0[q] >> 3;
            }
        }
        const unsigned key = live ? far_key(bc, eb) + 1u : 0u;
        const unsigned mk = __reduce_max_sync(0xffffffffu, key);
        if (mk == 0u) break;
        const int leader = __ffs(__ballot_sync(0xffffffffu, key == mk)) - 1;
        int sc[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) sc[q] = __shfl_sync(0xffffffffu, bc[q], leader);
        int lo_t[3] = {kEdge, kEdge, kEdge}, hi_t[3] = {-1, -1, -1};  // touched local range
        if (live && bc[0] == sc[0] && bc[1] == sc[1] && bc[2] == sc[2]) {
            const long long bi = bidx(v, sc);
            while (true) {
                const int base = ((i0[2] - kCells * sc[2]) * kEdge + (i0[1] - kCells * sc[1])) * kEdge +
                                 (i0[0] - kCells * sc[0]);
                // the 4^3 stencil and its adjoint touch base + a + 12 b + 144 c, a, b, c in [0, 3]
                if (!VR_CHECK(L.tp.status, base >= 0 && base + 3 * (1 + kEdge + kEdge * kEdge) < kBrickVox)) {
                    live = false;
                    break;
                }
                float fld[10];
                field_eval(GLoad{v.bricks + bi * kBrickVox}, base, f[0], f[1], f[2], fld);
                scale_field(fld, is);
                const float vval =
                    v.vbricks ? value_eval(GLoad{v.vbricks + bi * kBrickVox}, base, f[0], f[1], f[2]) : 0.f;
                SampleOptics so;
                optics_core(fld, vval, r.dir, L.tp, tf, inv_gmax, so);
                const float alpha = so.alpha, col[3] = {so.col[0], so.col[1], so.col[2]};
                if (kr != kstop) Tk = Tk1 / (1.0f - alpha);
                const float da = Tk * (fmaf(dC[0], col[0] - R0, fmaf(dC[1], col[1] - R1, dC[2] * (col[2] - R2))) +
                                       g4.w * P);
                const float ta = Tk * alpha;
                const float dc[3] = {ta * dC[0], ta * dC[1], ta * dC[2]};
                float dfs[10];
                sample_adjoint(fld, so, r.dir, L.tp, inv_gmax, da, dc, sink, dp, dfs);
                if (B.dvol) {
                    const int lx = i0[0] - kCells * sc[0], ly = i0[1] - kCells * sc[1], lz = i0[2] - kCells * sc[2];
                    lo_t[0] = min(lo_t[0], lx), lo_t[1] = min(lo_t[1], ly), lo_t[2] = min(lo_t[2], lz);
                    hi_t[0] = max(hi_t[0], lx + 3), hi_t[1] = max(hi_t[1], ly + 3), hi_t[2] = max(hi_t[2], lz + 3);
                    field_adjoint_scatter(dfs, is, f[0], f[1], f[2], [&](int a, int b, int c, float g) {
                        if (g != 0.0f) atomicAdd(acc + base + (c * kEdge + b) * kEdge + a, g);
                    });
                }
                R0 = fmaf(alpha, col[0], (1.0f - alpha) * R0);
                R1 = fmaf(alpha, col[1], (1.0f - alpha) * R1);
                R2 = fmaf(alpha, col[2], (1.0f - alpha) * R2);
                P *= (1.0f - alpha);
                Tk1 = Tk;
                if (--kr < 0) {
                    live = false;
                    break;
                }
                int b2[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    sample_cell(r, q, kr, v.n[q], i0[q], f[q]);
                    b2[q] = i0[q] >> 3;
                }
                if (b2[0] != sc[0] || b2[1] != sc[1] || b2[2] != sc[2]) break;
            }
        }
        if (B.dvol) {
            // add the touched box of the block to the global gradient (clamped voxel
            // indices: apron cells outside the volume belong to the edge voxel), clear it
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                lo_t[q] = __reduce_min_sync(0xffffffffu, lo_t[q]);
                hi_t[q] = __reduce_max_sync(0xffffffffu, hi_t[q]);
            }
            __syncwarp();
            if (hi_t[0] >= 0) {
                const int ex = hi_t[0] - lo_t[0] + 1, ey = hi_t[1] - lo_t[1] + 1, ez = hi_t[2] - lo_t[2] + 1;
                const int cnt = ex * ey * ez;
                const int nx = v.n[0], ny = v.n[1], nz = v.n[2];
                for (int e = l; e < cnt; e += 32) {
                    const int ax = lo_t[0] + e % ex, ay = lo_t[1] + (e / ex) % ey, az = lo_t[2] + e / (ex * ey);
                    const int o = (az * kEdge + ay) * kEdge + ax;
                    const float g = acc[o];
                    if (g != 0.0f) {
                        acc[o] = 0.0f;
                        const int x = min(max(kCells * sc[0] - 1 + ax, 0), nx - 1);
                        const int y = min(max(kCells * sc[1] - 1 + ay, 0), ny - 1);
                        const int z = min(max(kCells * sc[2] - 1 + az, 0), nz - 1);
                        atomicAdd(B.dvol + ((long long)z * ny + y) * nx + x, g);
                    }
                }
            }
            __syncwarp();
        }
    }
    sink.flush();
    float pv[5] = {dp.gamma, dp.ka, dp.kd, dp.ks, dp.os};
#pragma unroll
    for (int e = 0; e < 5; ++e) {
#pragma unroll
        for (int o = 16; o; o >>= 1) pv[e] += __shfl_xor_sync(0xffffffffu, pv[e], o);
    }
    if (l == 0 && B.dparams) {
#pragma unroll
        for (int e = 0; e < 5; ++e)
            if (pv[e] != 0.0f) atomicAdd(B.dparams + e, pv[e]);
    }
}

// dtf[e] += the sum over copies [16 g, 16 g + 16) of entry e's share of the cells
// around it, one thread per (float e, g): enough threads for a small table with many
// copies (dtf is zeroed before). Entry (j, k) is corner 00 of cell (j, k), 01 of
// (j - 1, k), 10 of (j, k - 1) and 11 of (j - 1, k - 1), where those cells exist (a
// cell's j < w - 1 and, in a 2D table, k < h - 1); in a cell record the opacity of
// corner q is float q, its RGB floats 4 + 3 q .. 6 + 3 q (1D: 2 + 3 q .. 4 + 3 q).
constexpr int kCopiesPerThread = 16;
__global__ void __launch_bounds__(256) k_sum_copies(const float* __restrict__ copies, int n_copies, int w, int h,
                                                   float* __restrict__ out) {
    const long long n = 4ll * w * h;
    const long long stride = (long long)w * h * kTfCellFloats;
    const long long groups = (n_copies + kCopiesPerThread - 1) / kCopiesPerThread;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n * groups;
         t += (long long)gridDim.x * blockDim.x) {
        const long long e = t % n;
        const int ch = (int)(e & 3), entry = (int)(e >> 2), j = entry % w, k = entry / w;
        const int c0 = (int)(t / n) * kCopiesPerThread;
        const int c1 = min(c0 + kCopiesPerThread, n_copies);
        // (cell key, float in its record) of each corner this entry is
        int off[4], m = 0;
        const bool kin = h == 1 || k < h - 1;  // row k holds cells
        auto slot = [&](int q) { return ch == 3 ? q : (h > 1 ? 4 : 2) + 3 * q + ch; };
        if (j < w - 1 && kin) off[m++] = entry * kTfCellFloats + slot(0);
        if (j >= 1 && kin) off[m++] = (entry - 1) * kTfCellFloats + slot(1);
        if (h > 1 && k >= 1 && j < w - 1) off[m++] = (entry - w) * kTfCellFloats + slot(2);
        if (h > 1 && k >= 1 && j >= 1) off[m++] = (long long)(entry - w - 1) * kTfCellFloats + slot(3);
        float acc = 0.0f;
        for (int c = c0; c < c1; ++c)
            for (int u = 0; u < m; ++u) acc += __ldg(copies + (size_t)c * stride + off[u]);
        if (acc != 0.0f) atomicAdd(out + e, acc);
    }
}

}  // namespace

cudaError_t launch_channels_to_voxels(const float* dgrad, const int n[3], const float s[3], float* dvol,
                                      cudaStream_t st) {
    const long long nvox = (long long)n[0] * n[1] * n[2];
    const long long blocks = (nvox + 255) / 256;
    k_channels_to_voxels<<<(unsigned)(blocks < 152 * 16 ? blocks : 152 * 16), 256, 0, st>>>(dgrad, n[0], n[1], n[2],
                                                                                          s[0], s[1], s[2], dvol);
    return cudaGetLastError();
}

cudaError_t launch_sum_copies(const float* copies, int n_copies, int tf_w, int tf_h, float* dtf, cudaStream_t st) {
    const long long n = 4ll * tf_w * tf_h;
    const long long blocks = (n * ((n_copies + kCopiesPerThread - 1) / kCopiesPerThread) + 255) / 256;
    k_sum_copies<<<(unsigned)(blocks < 152 * 8 ? blocks : 152 * 8), 256, 0, st>>>(copies, n_copies, tf_w, tf_h,
                                                                               dtf);
    return cudaGetLastError();
}

template <int kBS>
void launch_backward_bs(const BackwardLaunch& B, dim3 grid, cudaStream_t st) {
    const RenderLaunch& L = B.r;
    if (L.vol.dbricks)
        if (L.tp.gk == 0.0f && !B.dparams)
            k_render_backward<true, true, true, kBS><<<grid, 128, 0, st>>>(B);
        else if (L.tp.gk == 0.0f)
            k_render_backward<true, true, false, kBS><<<grid, 128, 0, st>>>(B);
        else
            k_render_backward<true, false, false, kBS><<<grid, 128, 0, st>>>(B);
    else
        k_render_backward<false, false, false, kBS><<<grid, 128, 0, st>>>(B);
}

cudaError_t launch_render_backward(const BackwardLaunch& B, bool staged, cudaStream_t st) {
    const RenderLaunch& L = B.r;
    dim3 grid((L.W + 15) / 16, (L.H + 7) / 8, L.n_cams);
    if (staged) {
        const int smem = 4 * kBrickBytes;
        cudaError_t e = cudaFuncSetAttribute(k_render_backward_staged, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        k_render_backward_staged<<<grid, 128, smem, st>>>(B);
        return cudaGetLastError();
    }
    switch (L.vol.bs) {
        case 2: launch_backward_bs<2>(B, grid, st); break;
        case 4: launch_backward_bs<4>(B, grid, st); break;
        default: launch_backward_bs<3>(B, grid, st); break;
    }
    return cudaGetLastError();
}

}  // namespace vr
