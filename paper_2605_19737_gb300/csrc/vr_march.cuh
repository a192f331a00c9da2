// vr_march.cuh -- the per-lane front-to-back march of one ray (Sec. 2.4, Eqs. 4-6)
// over the bricked volume, shared by the single-view and batched forward kernels.
#pragma once

#include "vr_sample.cuh"

namespace vr {

struct GlobalLoad {
    const float* __restrict__ p;
    __device__ __forceinline__ float operator()(int o) const { return __ldg(p + o); }
};

// Skip-brick id in 32-bit arithmetic: dims <= 2048 give at most 512^3 = 2^27 bricks.
__device__ __forceinline__ int brick_index(const VolumeDev& v, const int b[3]) {
    return (b[2] * v.nb[1] + b[1]) * v.nb[0] + b[0];
}


__device__ __forceinline__ void add_counters(vr_counters* ctr, unsigned rays, unsigned dense, unsigned evald,
                                             unsigned staged, unsigned shaded, unsigned interp) {
    const unsigned r = __reduce_add_sync(0xffffffffu, rays);
    const unsigned d = __reduce_add_sync(0xffffffffu, dense);
    const unsigned e = __reduce_add_sync(0xffffffffu, evald);
    const unsigned s = __reduce_add_sync(0xffffffffu, staged);
    const unsigned h = __reduce_add_sync(0xffffffffu, shaded);
    const unsigned ip = __reduce_add_sync(0xffffffffu, interp);
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&ctr->rays, (unsigned long long)r);
        atomicAdd(&ctr->dense_samples, (unsigned long long)d);
        atomicAdd(&ctr->evaluated_samples, (unsigned long long)e);
        atomicAdd(&ctr->bricks_staged, (unsigned long long)s);
        atomicAdd(&ctr->shaded_samples, (unsigned long long)h);
        atomicAdd(&ctr->interpolated_samples, (unsigned long long)ip);
    }
}

// Front-to-back march of one ray (Eqs. 4-6) over the bricked volume in HBM/L2,
// skipping bricks classified empty. Shared by the single-view and batched kernels.
// kHessianFirst: the derived path issues the Hessian loads before the table lookup,
// so that they overlap it, or only after its zero-opacity test; the arithmetic, and
// so the image, is the same. Every kernel now takes the first order (the batched
// kernel measured 3 % faster with it once the packed arithmetic and incremental
// positions were in; 1.4 % slower before).
// With kState it also returns the ray's last sample index (kstop) and the
// transmittance in front of that sample (t_last), which the adjoint sweep starts from.
// kBS: log2 of the skip-brick edge in cells, fixed at compile time (2, 3, 4), or 0 to
// take the volume's at run time (batches that mix sizes); a fixed size keeps the
// brick and cell index arithmetic in immediates (the run-time form measured 4-10 %
// slower).
template <bool kDerived, bool kState = false, bool kParity = false, bool kHessianFirst = true, int kBS = 3>
__device__ __forceinline__ void march_gather(const VolumeDev& v, const TissueDev& tp, const float4* __restrict__ tf,
                                             const RayDev& r, int skip, float inv_gmax, const float is[3],
                                             float4& out, unsigned& dense, unsigned& evald, unsigned& shaded,
                                             unsigned& interp, int* klast_out = nullptr, float* t_last = nullptr) {
    float C0 = 0.f, C1 = 0.f, C2 = 0.f, A = 0.f;
    float A_prev = 0.f;  // kState: A before the last evaluated sample
    int klast = -1;      // kState: last evaluated sample
    int k1 = -1;         // kState: first sample with A >= 1 (where the adjoint sweep must start
    float T1 = 1.f;      // when early termination is off) and the transmittance in front of it
    int k = 0, kstop = -1;
    unsigned ne = 0, nsh = 0, nip = 0;
    // The skip flag and the base pointers of the current brick are re-read only
    // when the brick changes (about every 16 samples), keeping a dependent L1 round
    // trip and the 64-bit address arithmetic off the path of every sample.
    int cur_bi = -1;
    bool cur_empty = false;
    const float4* dbrick = nullptr;  // derived brick of cur_bi
    const int bs = kBS ? kBS : v.bs, B = 1 << bs, E = B + 1;
    // the position of sample k, u0 + k du, carried by exact integer additions
    long long U[3] = {r.u0[0], r.u0[1], r.u0[2]};
    auto advance = [&](int k1) {
        if (k1 == k + 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) U[q] += r.du[q];
        } else {
#pragma unroll
            for (int q = 0; q < 3; ++q) U[q] += (long long)(k1 - k) * r.du[q];
        }
        k = k1;
    };
    while (k < r.ns) {
        int i0[3], bc[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            i0[q] = cell_index_at(U[q], v.n[q]);
            bc[q] = i0[q] >> bs;
        }
        if (!VR_CHECK(tp.status, (unsigned)bc[0] < (unsigned)v.nb[0] && (unsigned)bc[1] < (unsigned)v.nb[1] &&
                                     (unsigned)bc[2] < (unsigned)v.nb[2])) {
            advance(k + 1);
            continue;
        }
        const int bi = brick_index(v, bc);
        if (bi != cur_bi) {
            cur_bi = bi;
            if (skip) cur_empty = __ldg(v.empty + bi) != 0;
            if (kDerived)
                dbrick = reinterpret_cast<const float4*>(
                    v.dbricks + (size_t)bi * (kBS ? (size_t)der_brick_floats(kBS) : (size_t)v.der_stride));
        }
        if (skip && cur_empty) {
            advance(brick_exit_k_at(r, U, bc, B, k, r.ns));
            continue;
        }
        // local cell of (i0, j0, k0) within the skip brick: i0 - B bc = i0 & (B - 1)
        const int lx = i0[0] & (B - 1), ly = i0[1] & (B - 1), lz = i0[2] & (B - 1);
        if (skip && v.cellmask) {
            // a cell classified empty holds only samples of opacity exactly 0 (their
            // intensity lies in the range of its 8 corners): nothing to read or add
            const int c = (((lz << bs) + ly) << bs) + lx;
            if ((__ldg(v.cellmask + (size_t)bi * cell_words(bs) + (c >> 5)) >> (c & 31)) & 1u) {
                ++ne;
                advance(k + 1);
                continue;
            }
        }
        ++nip;
        // the sample's fractions, only for samples that are evaluated
        float f[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) f[q] = cell_frac_at(U[q], v.n[q]);
        int base = 0, sbi = 0;
        if (!kDerived || v.vbricks) sbi = storage_brick(v, i0, base);
        const float vval =
            v.vbricks ? value_eval(GlobalLoad{v.vbricks + (size_t)sbi * kBrickVox}, base, f[0], f[1], f[2]) : 0.0f;
        float fld[10], alpha, col[3];
        if (kDerived) {
            // I and the gradient (one 16-byte load per corner) and the Hessian (two), then
            // the transfer function: a zero opacity entry makes alpha exactly 0 whatever
            // the Hessian, and the sample adds nothing (bit-neutral). The Hessian loads are
            // issued before that test so that they overlap the table lookup (measured:
            // equal at 1080p, 2 % faster on the 8-view workload than loading them after it)
            derived_channels<kParity, 0, 4>(dbrick, E, lx, ly, lz, f[0], f[1], f[2], fld);
            if (kHessianFirst) load_hessian<kParity>(tp, dbrick, E, lx, ly, lz, f, fld);
            SampleOptics o;
            optics_tf(fld, vval, tp, tf, inv_gmax, o);
            if (o.c.w == 0.0f) {
                ++ne;
                advance(k + 1);
                continue;
            }
            if (!kHessianFirst) load_hessian<kParity>(tp, dbrick, E, lx, ly, lz, f, fld);
            optics_rest(fld, r.dir, tp, o);
            alpha = o.alpha;
            col[0] = o.col[0];
            col[1] = o.col[1];
            col[2] = o.col[2];
        } else {
            field_eval(GlobalLoad{v.bricks + (size_t)sbi * kBrickVox}, base, f[0], f[1], f[2], fld);
            scale_field(fld, is);
            sample_optics(fld, vval, r.dir, tp, tf, inv_gmax, alpha, col);
        }
        ++nsh;
        const float wgt = (1.0f - A) * alpha;  // Eqs. 5-6
        fma2v(col[0], col[1], wgt, wgt, C0, C1);
        C2 = fmaf(col[2], wgt, C2);
        if (kState) {
            A_prev = A;
            klast = k;
        }
        A += wgt;
        if (kState && k1 < 0 && A >= 1.0f) {
            k1 = k;
            T1 = 1.0f - A_prev;
        }
        ++ne;
        if (A >= tp.et_threshold) {
            kstop = k;
            break;
        }
        advance(k + 1);
    }
    out = make_float4(C0, C1, C2, A);
    dense = kstop >= 0 ? (unsigned)(kstop + 1) : (unsigned)r.ns;
    evald = ne;
    shaded = nsh;
    interp = nip;
    if (kState) {
        // the adjoint sweep starts at the first sample with A >= min(et, 1): the stopping
        // sample, or (early termination off) the first that made A reach 1
        const int kl = (int)dense - 1;
        *klast_out = k1 >= 0 ? k1 : kl;
        *t_last = k1 >= 0 ? T1 : ((klast == kl) ? 1.0f - A_prev : 1.0f - A);  // samples after klast: alpha 0
    }
}

}  // namespace vr
