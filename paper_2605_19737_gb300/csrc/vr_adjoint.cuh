// vr_adjoint.cuh -- adjoint of the per-sample math in vr_sample.cuh.
//
// Given dL/dalpha and dL/dcolour of one sample, sample_adjoint() walks back
// through the shading, Eq. 4, the transfer-function lookup and the curvature
// of Eq. 3 to dL/d(I, grad, Hessian) of the sample field, adding the
// transfer-function and uniform gradients on the way. field_adjoint_scatter()
// is the exact transpose of field_eval(): it spreads those field gradients over
// the 56 weighted voxels of the cell's 4x4x4 neighbourhood. Clamps pass
// gradient only on their identity branch; |x| has derivative sign(x), 0 at 0.
#pragma once

#include "vr_sample.cuh"

namespace vr {

struct ParamGrad {
    float gamma, ka, kd, ks, os;
};

// Transfer-function gradient sink: one of the private global copies of the
// gradient, kept per lookup cell rather than per entry. A lane's consecutive
// samples mostly look up the same transfer-function cell, so the sink accumulates
// the cell's (2 or 4) entry gradients in registers and writes them out only when
// the cell changes (and once at the end of the ray: flush()). A copy holds one
// 16-float record per cell key (k * tf_w + j, the index of its entry (j, k)): the
// opacity gradients of its four corner entries 00, 01, 10, 11, then their RGB
// gradients (3 x 4 floats), written with up to four 16-byte vector reductions, all
// zero pieces skipped; in a 1D table (two corners) the opacities of 00 and 01, then
// the RGB of 00 and of 01 (two pieces). Samples whose opacity entry is zero (most
// of a ray: the sweep does not skip empty space) give gradient to the opacity
// entries only, so most flushes write one 16-byte piece where an entry-major table
// took four (two).
// k_sum_copies gathers each entry's share from the (up to 4) cells around it.
// (Shared-memory tables with scalar atomics measured 1.6x slower on a 1D table:
// the lanes of a CTA contend for the same few entries.)

struct TfGradSink {
    float* p;       // this copy: [cell key][kTfCellFloats]
    bool two_d;
    int key = -1;   // the pending cell, -1 = none
    float4 a00, a01, a10, a11;

    __device__ __forceinline__ TfGradSink(float* p_, bool two_d_) : p(p_), two_d(two_d_) {}

    __device__ __forceinline__ void put(int piece, const float4& v) const {
        // any component not +-0: one OR of the bit patterns, the sign bits shifted out
        const unsigned bits = __float_as_uint(v.x) | __float_as_uint(v.y) | __float_as_uint(v.z) |
                              __float_as_uint(v.w);
        if (bits << 1) atomicAdd(reinterpret_cast<float4*>(p + (size_t)key * kTfCellFloats) + piece, v);
    }
    __device__ __forceinline__ void flush() {
        if (key < 0) return;
        if (two_d) {
            put(0, make_float4(a00.w, a01.w, a10.w, a11.w));
            put(1, make_float4(a00.x, a00.y, a00.z, a01.x));
            put(2, make_float4(a01.y, a01.z, a10.x, a10.y));
            put(3, make_float4(a10.z, a11.x, a11.y, a11.z));
        } else {
            put(0, make_float4(a00.w, a01.w, a00.x, a00.y));
            put(1, make_float4(a00.z, a01.x, a01.y, a01.z));
        }
        key = -1;
    }
    // Add the bilinear weights (w00 .. w11) times d to cell `e00` (= k * w + j).
    __device__ __forceinline__ void add_cell(int e00, float w00, float w01, float w10, float w11, const float d[4]) {
        if (e00 != key) {
            flush();
            key = e00;
            a00 = a01 = a10 = a11 = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        auto acc = [&](float4& a, float c) {
            fma2(c, d[0], d[1], a.x, a.y);
            fma2(c, d[2], d[3], a.z, a.w);
        };
        acc(a00, w00);
        acc(a01, w01);
        if (two_d) {
            acc(a10, w10);
            acc(a11, w11);
        }
    }
};

// Adjoint of one sample's optics, from the forward values `o` that optics_core
// computed for it. da = dL/dalpha and dc = dL/dcolour come in; the transfer-function
// and uniform gradients go to dtf and dp; dfield receives dL/d(I, gx, gy, gz, Hxx,
// Hyy, Hzz, Hxy, Hxz, Hyz) in the same (spacing-scaled) units as the field f.
__device__ __forceinline__ void sample_adjoint(const float f[10], const SampleOptics& o, const float dir[3],
                                               const TissueDev& tp, float inv_gmax, float da, const float dc[3],
                                               TfGradSink& dtf, ParamGrad& dp, float dfield[10]) {
    const float gx = f[1], gy = f[2], gz = f[3];
    const float gg = o.gg, r = o.r, kappa = o.kappa, hx = o.hx, hy = o.hy, hz = o.hz;
    const float Hgx = o.Hgx, Hgy = o.Hgy, Hgz = o.Hgz, gn = o.gn, y = o.y;
    const int w = tp.tf_w, h = tp.tf_h, j = o.j, k = o.k;
    const float I = f[0], t = o.t, q = o.q;
    const float4 c = o.c, T00 = o.T00, T01 = o.T01, T10 = o.T10, T11 = o.T11;
    const float mg = o.mg, wi = o.wi, wk = o.wk, raw = o.raw, dot = o.dot, d = o.d;

    // colour
    float dr[4] = {0.f, 0.f, 0.f, 0.f}, dd = 0.f;
    const float crgb[3] = {c.x, c.y, c.z};
    if (tp.shading) {
        const float d2 = d * d, d4 = d2 * d2, d8 = d4 * d4, d15 = d8 * d4 * d2 * d, d16 = d8 * d8;
        const float lit = fmaf(tp.kd, d, tp.ka);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            dr[ch] = dc[ch] * lit;
            dp.ka += dc[ch] * crgb[ch];
            dp.kd += dc[ch] * crgb[ch] * d;
            dp.ks += dc[ch] * d16;
            dd = fmaf(dc[ch], fmaf(crgb[ch], tp.kd, 16.0f * tp.ks * d15), dd);
        }
    } else {
        dr[0] = dc[0];
        dr[1] = dc[1];
        dr[2] = dc[2];
    }
    // step-size opacity correction alpha' = 1 - (1 - alpha)^e, then Eq. 4
    if (tp.alpha_exp > 0.0f) {
        const float a0 = fminf(fmaxf(raw, 0.0f), 1.0f);
        da = a0 < 1.0f ? da * tp.alpha_exp * expf((tp.alpha_exp - 1.0f) * log1pf(-a0)) : 0.0f;
    }
    const float draw = (raw >= 0.0f && raw <= 1.0f) ? da : 0.0f;
    dp.os += draw * c.w * mg * wk;
    dr[3] = draw * tp.opacity_scale * mg * wk;
    const float dmg = draw * tp.opacity_scale * c.w * wk;
    const float dw = draw * tp.opacity_scale * c.w * mg;
    const float dwi = (wi >= 0.0f && wi <= tp.w_max) ? dw : 0.0f;
    dp.gamma += dwi * kappa * tp.inv_kref;
    const float dkappa = dwi * tp.gk;
    float dgn = (tp.grad_mod && gn < 1.0f) ? dmg : 0.0f;
    // transfer-function lookup
    const bool in_x = I >= 0.0f && I <= 1.0f;
    float dI = 0.f;
    const float T00a[4] = {T00.x, T00.y, T00.z, T00.w}, T01a[4] = {T01.x, T01.y, T01.z, T01.w};
    if (h == 1) {
        dtf.add_cell(j, 1.0f - t, t, 0.0f, 0.0f, dr);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            if (in_x) dI = fmaf(dr[ch], (T01a[ch] - T00a[ch]) * (float)(w - 1), dI);
    } else {
        const float T10a[4] = {T10.x, T10.y, T10.z, T10.w}, T11a[4] = {T11.x, T11.y, T11.z, T11.w};
        const bool in_y = y >= 0.0f && y <= 1.0f;
        float dy = 0.f;
        const int e00 = k * w + j;
        dtf.add_cell(e00, (1.0f - q) * (1.0f - t), (1.0f - q) * t, q * (1.0f - t), q * t, dr);
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            if (in_x)
                dI = fmaf(dr[ch], ((1.0f - q) * (T01a[ch] - T00a[ch]) + q * (T11a[ch] - T10a[ch])) * (float)(w - 1),
                          dI);
            if (in_y)
                dy = fmaf(dr[ch], ((1.0f - t) * (T10a[ch] - T00a[ch]) + t * (T11a[ch] - T01a[ch])) * (float)(h - 1),
                          dy);
        }
        if (tp.tf_mode == 1) dgn += dy;  // mode 2: V is a constant of the volume
    }
    dfield[0] = dI;
    float dgx = 0.f, dgy = 0.f, dgz = 0.f;
#pragma unroll
    for (int e = 4; e < 10; ++e) dfield[e] = 0.f;
    if (gg > 0.0f) {
        if (tp.shading) {
            const float sgn = dot > 0.0f ? 1.0f : (dot < 0.0f ? -1.0f : 0.0f);
            const float ax = dd * sgn * dir[0], ay = dd * sgn * dir[1], az = dd * sgn * dir[2];
            const float proj = fmaf(ax, hx, fmaf(ay, hy, az * hz));
            dgx += (ax - proj * hx) * r;
            dgy += (ay - proj * hy) * r;
            dgz += (az - proj * hz) * r;
        }
        dgx = fmaf(dgn * inv_gmax, hx, dgx);
        dgy = fmaf(dgn * inv_gmax, hy, dgy);
        dgz = fmaf(dgn * inv_gmax, hz, dgz);
        const float s = dkappa * (r * r);
        dgx = fmaf(2.0f * s, Hgx - kappa * gx, dgx);
        dgy = fmaf(2.0f * s, Hgy - kappa * gy, dgy);
        dgz = fmaf(2.0f * s, Hgz - kappa * gz, dgz);
        dfield[4] = s * gx * gx;
        dfield[5] = s * gy * gy;
        dfield[6] = s * gz * gz;
        dfield[7] = 2.0f * s * gx * gy;
        dfield[8] = 2.0f * s * gx * gz;
        dfield[9] = 2.0f * s * gy * gz;
    }
    dfield[1] = dgx;
    dfield[2] = dgy;
    dfield[3] = dgz;
}

// Transpose of field_eval + scale_field: add dL/d(voxel) for the 56 weighted voxels.
// `emit(a, b, c, g)` receives tap (a, b, c) of the 4x4x4 neighbourhood (voxel
// i0-1+a, j0-1+b, k0-1+c) and its gradient g.
template <class Emit>
__device__ __forceinline__ void field_adjoint_scatter(const float dfs[10], const float is[3], float fx, float fy,
                                                      float fz, const Emit& emit) {
    // undo the spacing scale (chain through scale_field)
    const float dI = dfs[0];
    const float dgx = dfs[1] * is[0], dgy = dfs[2] * is[1], dgz = dfs[3] * is[2];
    const float dxx = dfs[4] * is[0] * is[0], dyy = dfs[5] * is[1] * is[1], dzz = dfs[6] * is[2] * is[2];
    const float dxy = dfs[7] * is[0] * is[1], dxz = dfs[8] * is[0] * is[2], dyz = dfs[9] * is[1] * is[2];
    const float gxw = 1.0f - fx, gyw = 1.0f - fy, gzw = 1.0f - fz;
    const float w0x[4] = {0.0f, gxw, fx, 0.0f};
    const float w1x[4] = {-0.5f * gxw, -0.5f * fx, 0.5f * gxw, 0.5f * fx};
    const float w2x[4] = {gxw, fmaf(3.0f, fx, -2.0f), fmaf(-3.0f, fx, 1.0f), fx};
    const float w0y[4] = {0.0f, gyw, fy, 0.0f};
    const float w1y[4] = {-0.5f * gyw, -0.5f * fy, 0.5f * gyw, 0.5f * fy};
    const float w2y[4] = {gyw, fmaf(3.0f, fy, -2.0f), fmaf(-3.0f, fy, 1.0f), fy};
    const float w0z[4] = {0.0f, gzw, fz, 0.0f};
    const float w1z[4] = {-0.5f * gzw, -0.5f * fz, 0.5f * gzw, 0.5f * fz};
    const float w2z[4] = {gzw, fmaf(3.0f, fz, -2.0f), fmaf(-3.0f, fz, 1.0f), fz};
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const bool zmid = (c == 1 || c == 2);
        // transposed z step: adjoints of the y-level sums A.. of field_eval
        float A00 = w1z[c] * dgz + w2z[c] * dzz;
        float A10 = w1z[c] * dxz;
        float A01 = w1z[c] * dyz;
        float A20 = 0.f, A11 = 0.f, A02 = 0.f;
        if (zmid) {
            A00 = fmaf(w0z[c], dI, A00);
            A10 = fmaf(w0z[c], dgx, A10);
            A20 = w0z[c] * dxx;
            A01 = fmaf(w0z[c], dgy, A01);
            A11 = w0z[c] * dxy;
            A02 = w0z[c] * dyy;
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const bool ymid = (b == 1 || b == 2);
            // transposed y step: adjoints of X0, X1, X2
            float X0 = w1y[b] * A01;
            float X1 = 0.f, X2 = 0.f;
            if (ymid) {
                X0 = fmaf(w0y[b], A00, X0);
                X1 = w0y[b] * A10;
                if (zmid) X2 = w0y[b] * A20;
            }
            if (zmid) {
                X1 = fmaf(w1y[b], A11, X1);
                X0 = fmaf(w2y[b], A02, X0);
            }
            // transposed x step
            if (ymid || zmid) {
                emit(0, b, c, fmaf(w1x[0], X1, w2x[0] * X2));
                emit(3, b, c, fmaf(w1x[3], X1, w2x[3] * X2));
            }
            emit(1, b, c, fmaf(w0x[1], X0, fmaf(w1x[1], X1, w2x[1] * X2)));
            emit(2, b, c, fmaf(w0x[2], X0, fmaf(w1x[2], X1, w2x[2] * X2)));
        }
    }
}

}  // namespace vr
