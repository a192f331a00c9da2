// vr_sample.cuh -- per-ray and per-sample device math of the raymarch.
//
// Ray setup (pinhole camera, slab intersection, sample count) runs once per
// ray in FP64; it yields the entry point and per-sample step in voxel
// coordinates as float32 head/tail pairs, from which each sample's cell
// fraction is formed to ~3e-8 at any depth.
//
// The sample field is the trilinear interpolation of the voxel-wise intensity,
// central-difference gradient (Eq. 2) and Hessian (Sec. 2.3). Along one axis,
// with cell origin i0 and fraction f, these are 4-tap filters over voxels
// i0-1 .. i0+2:
//   value        w0 = [0, 1-f, f, 0]
//   d/dx         w1 = [-(1-f), -f, 1-f, f] / 2          (divided by the spacing)
//   d^2/dx^2     w2 = [1-f, 3f-2, 1-3f, f]              (divided by spacing^2)
// and the 3D quantities are separable products of them (mixed second
// derivatives use w1 on both axes). The contraction below reads the 56 voxels
// of the 4x4x4 neighbourhood that carry weight (the 8 outer corners never
// do), contracting x, then y, then z.
#pragma once

#include "vr_internal.cuh"

namespace vr {

struct RayDev {
    int ns;             // number of samples t_k = t_near + (k+1/2) dt < t_far
    long long u0[3];    // voxel coordinate of sample 0 (t_near + dt/2), 32.32 fixed point
    long long du[3];    // voxel-coordinate step per sample, 32.32 fixed point
    float dir[3];       // unit ray direction
};

// 32.32 fixed point from a double-float x (|x| < 2^30), with 32-bit conversions only
// (64-bit float<->integer conversions are slow on this part): the head's whole part
// (truncated), its fraction h - trunc(h) -- exact, h and trunc(h) share sign and
// binade or trunc(h) = 0 -- scaled by 2^31 and doubled (2^-32 resolution), and the
// tail scaled by 2^32.
__device__ __forceinline__ long long df_to_fx(dfloat x) {
    const float t = truncf(x.hi);
    const long long whole = (long long)__float2int_rz(t) << 32;
    const long long frac = 2 * (long long)__float2int_rn((x.hi - t) * 2147483648.0f);
    return whole + frac + (long long)__float2int_rn(x.lo * 4294967296.0f);
}

// A 32.32 fixed-point value as float (|U| < 2^62), again without 64-bit conversions.
__device__ __forceinline__ float fx_to_float(long long U) {
    return fmaf(__uint2float_rn((unsigned)U), 2.3283064365386963e-10f, (float)(int)(U >> 32));
}

// Ray through pixel (i, j): direction normalize(fwd + a right + b up),
// a = 2(i+1/2)/W - 1, b = 1 - 2(j+1/2)/H; slab intersection with the volume box;
// t_near = max(t0, 0); ns = #{k : t_near + (k+1/2) dt < t_far}. Computed in
// double-float arithmetic (~48 bits, vr_df.cuh): FP64 is a small fraction of the
// FP32 rate on this part and its registers come in pairs. Returns false when the
// ray misses the box or has no sample.
__device__ __forceinline__ bool setup_ray(const CamDev& c, const RayConsts& rc, int i, int j, const int n[3],
                                          const float s[3], RayDev& r) {
    // i + 1/2 and j + 1/2 are exact in float for image sizes up to 2^22
    const dfloat tw = {rc.two_over_w.hi, rc.two_over_w.lo}, th = {rc.two_over_h.hi, rc.two_over_h.lo};
    const dfloat a = df_add_f(df_mul_f(tw, (float)i + 0.5f), -1.0f);
    const dfloat b = df_add_f(df_neg(df_mul_f(th, (float)j + 0.5f)), 1.0f);
    dfloat d[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) d[q] = df_add(df_add_f(df_mul_f(a, c.right[q]), c.fwd[q]), df_mul_f(b, c.up[q]));
    const dfloat inv_len = df_rsqrt(df_add(df_add(df_mul(d[0], d[0]), df_mul(d[1], d[1])), df_mul(d[2], d[2])));
#pragma unroll
    for (int q = 0; q < 3; ++q) d[q] = df_mul(d[q], inv_len);
    dfloat t0 = {-INFINITY, 0.0f}, t1 = {INFINITY, 0.0f};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float o = c.eye[q];
        const dfloat hi = df_two_prod((float)n[q], s[q]);  // exact
        if (d[q].hi == 0.0f) {
            if (o < 0.0f || df_lt(hi, dfloat{o, 0.0f})) return false;
            continue;
        }
        const dfloat inv_d = df_recip(d[q]);
        const dfloat ta = df_mul_f(inv_d, -o);
        const dfloat tb = df_mul(df_add_f(hi, -o), inv_d);
        const bool ord = df_lt(ta, tb);
        const dfloat lo_t = ord ? ta : tb, hi_t = ord ? tb : ta;
        if (df_lt(t0, lo_t)) t0 = lo_t;
        if (df_lt(hi_t, t1)) t1 = hi_t;
    }
    const dfloat tn = df_lt(dfloat{0.0f, 0.0f}, t0) ? t0 : dfloat{0.0f, 0.0f}, tf = t1;
    if (!df_lt(tn, tf)) return false;
    const dfloat dt = {rc.dt.hi, rc.dt.lo};
    // estimate, then settle on the exact predicate t_near + (k + 1/2) dt < t_far
    auto before_far = [&](int k) { return df_lt(df_add(tn, df_mul_f(dt, (float)k + 0.5f)), tf); };
    const float est = ceilf(fmaf(__fsub_rn(tf.hi, tn.hi), rc.inv_dt, -0.5f));
    int ns = est > 0.0f ? (est < 4194304.0f ? (int)est : 4194304) : 0;
    while (ns > 0 && !before_far(ns - 1)) --ns;
    while (before_far(ns)) ++ns;
    if (ns == 0) return false;
    r.ns = ns;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const dfloat is = {rc.inv_s[q].hi, rc.inv_s[q].lo};
        const dfloat un = df_add_f(df_mul(df_add_f(df_mul(tn, d[q]), c.eye[q]), is), -0.5f);
        const dfloat st = df_mul(df_mul(dt, d[q]), is);
        // 32.32 fixed point of the step and of sample 0's coordinate u_n + step / 2
        r.du[q] = df_to_fx(st);
        r.u0[q] = df_to_fx(un) + df_to_fx(dfloat{0.5f * st.hi, 0.5f * st.lo});
        r.dir[q] = d[q].hi;
    }
    return true;
}

// Cell of sample k along axis q: u_c = clamp(u, 0, n-1), i0 = min(floor(u_c), n-2),
// f = u_c - i0. u = u_n + (k + 1/2) step is carried in 32.32 fixed point
// (u0 + k du, exact integer arithmetic): the rounding of u0 and du leaves ~(k+1) 2^-33
// voxel, ~1e-7 after thousands of samples, and the same k gives the same cell and
// fraction in every kernel. f is the low word rounded to float once.
__device__ __forceinline__ void sample_cell(const RayDev& r, int q, int k, int n, int& i0, float& f) {
    const long long U = r.u0[q] + (long long)k * r.du[q];
    if (U <= 0) {
        i0 = 0;
        f = 0.0f;
    } else if (U >= ((long long)(n - 1) << 32)) {
        i0 = n - 2;
        f = 1.0f;
    } else {
        i0 = (int)(U >> 32);  // <= n - 2 here
        f = __uint2float_rn((unsigned)U) * 2.3283064365386963e-10f;  // 2^-32
    }
}

// sample_cell from the sample's position U = u0 + k du itself (the march carries U
// from sample to sample by exact integer additions): the same cell and fraction,
// the clamps taken on the high word (U <= 0 gives (0, 0) either way; U >=
// (n - 1) 2^32 exactly when the high word is >= n - 1).
__device__ __forceinline__ int cell_index_at(long long U, int n) { return min(max((int)(U >> 32), 0), n - 2); }
__device__ __forceinline__ float cell_frac_at(long long U, int n) {
    const int hi = (int)(U >> 32);
    const float fl = __uint2float_rn((unsigned)U) * 2.3283064365386963e-10f;  // 2^-32
    return hi < 0 ? 0.0f : (hi > n - 2 ? 1.0f : fl);
}
__device__ __forceinline__ void cell_at(long long U, int n, int& i0, float& f) {
    i0 = cell_index_at(U, n);
    f = cell_frac_at(U, n);
}

// Sample field: out = I, gx, gy, gz, Hxx, Hyy, Hzz, Hxy, Hxz, Hyz (not yet divided
// by the spacing). `load(o)` returns the brick value at flat offset o; `base` is
// the offset of tap (0,0,0) = voxel (i0-1, j0-1, k0-1).
template <class Load>
__device__ __forceinline__ void field_eval(const Load& load, int base, float fx, float fy, float fz, float out[10]) {
    const float gxw = 1.0f - fx, gyw = 1.0f - fy, gzw = 1.0f - fz;
    const float w1x[4] = {-0.5f * gxw, -0.5f * fx, 0.5f * gxw, 0.5f * fx};
    const float w2x[4] = {gxw, fmaf(3.0f, fx, -2.0f), fmaf(-3.0f, fx, 1.0f), fx};
    const float w0y[4] = {0.0f, gyw, fy, 0.0f};
    const float w1y[4] = {-0.5f * gyw, -0.5f * fy, 0.5f * gyw, 0.5f * fy};
    const float w2y[4] = {gyw, fmaf(3.0f, fy, -2.0f), fmaf(-3.0f, fy, 1.0f), fy};
    const float w0z[4] = {0.0f, gzw, fz, 0.0f};
    const float w1z[4] = {-0.5f * gzw, -0.5f * fz, 0.5f * gzw, 0.5f * fz};
    const float w2z[4] = {gzw, fmaf(3.0f, fz, -2.0f), fmaf(-3.0f, fz, 1.0f), fz};
    float I = 0.f, gx = 0.f, gy = 0.f, gz = 0.f, hxx = 0.f, hyy = 0.f, hzz = 0.f, hxy = 0.f, hxz = 0.f, hyz = 0.f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const bool zmid = (c == 1 || c == 2);
        float A00 = 0.f, A10 = 0.f, A20 = 0.f, A01 = 0.f, A11 = 0.f, A02 = 0.f;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const bool ymid = (b == 1 || b == 2);
            const int ro = base + c * (kEdge * kEdge) + b * kEdge;
            const float v1 = load(ro + 1), v2 = load(ro + 2);
            const float X0 = fmaf(fx, v2, gxw * v1);
            float X1 = 0.f, X2 = 0.f;
            if (ymid || zmid) {
                const float v0 = load(ro), v3 = load(ro + 3);
                X1 = fmaf(w1x[3], v3, fmaf(w1x[2], v2, fmaf(w1x[1], v1, w1x[0] * v0)));
                if (ymid && zmid) X2 = fmaf(w2x[3], v3, fmaf(w2x[2], v2, fmaf(w2x[1], v1, w2x[0] * v0)));
            }
            if (ymid) {
                A00 = fmaf(w0y[b], X0, A00);
                A10 = fmaf(w0y[b], X1, A10);
                if (zmid) A20 = fmaf(w0y[b], X2, A20);
            }
            A01 = fmaf(w1y[b], X0, A01);
            if (zmid) {
                A11 = fmaf(w1y[b], X1, A11);
                A02 = fmaf(w2y[b], X0, A02);
            }
        }
        if (zmid) {
            I = fmaf(w0z[c], A00, I);
            gx = fmaf(w0z[c], A10, gx);
            hxx = fmaf(w0z[c], A20, hxx);
            gy = fmaf(w0z[c], A01, gy);
            hxy = fmaf(w0z[c], A11, hxy);
            hyy = fmaf(w0z[c], A02, hyy);
        }
        gz = fmaf(w1z[c], A00, gz);
        hzz = fmaf(w2z[c], A00, hzz);
        hxz = fmaf(w1z[c], A10, hxz);
        hyz = fmaf(w1z[c], A01, hyz);
    }
    out[0] = I;
    out[1] = gx;
    out[2] = gy;
    out[3] = gz;
    out[4] = hxx;
    out[5] = hyy;
    out[6] = hzz;
    out[7] = hxy;
    out[8] = hxz;
    out[9] = hyz;
}

// Sample field from derived bricks: trilinear interpolation of voxel-wise channels
// (already in mm units) over the cell's 8 corners; (lx, ly, lz) is the cell's corner
// voxel (i0, j0, k0) local to the brick's E^3 block (E = B + 1 corners per edge). Channels [kFirst, kFirst +
// kCount): kFirst = 0, kCount = 4 reads (I, gx, gy, gz) -- the first 16-byte vector
// of each corner; kFirst = 4, kCount = 6 the Hessian (Hxx, Hyy, Hzz, Hxy, Hxz, Hyz)
// -- the second and third. Each channel sums its 8 corners in the same order, so
// split and whole evaluations agree bit for bit.
// kParity: the 8 corner loads are issued in order of the corners' parity (even/odd
// voxel index per axis) rather than of their offset from the cell, so that lanes in
// neighbouring cells read the same record in the same instruction and their loads
// coalesce; each lane picks the matching weight. That costs ~30 instructions per
// sample; measured, the adjoint sweep gains 3 %, the 1080p forward frame loses
// 1.3 % (512^2 views gain 3 %). The forward kernels keep the offset order, so that
// single-view and batched renders stay bit-identical; the adjoint uses parity order.
// Read-only 16-byte load that asks L2 to fetch the surrounding 256 bytes from DRAM
// (neighbouring corner records of the same brick row).
__device__ __forceinline__ float4 ldg_l2_256(const float4* p) {
    float4 v;
    asm("ld.global.nc.L2::256B.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
        : "l"(p));
    return v;
}

// (ox, oy) = (fma(w, ax, ox), fma(w, ay, oy)) in one packed instruction
// (fma.rn.f32x2, sm_100 and later): each half rounds exactly as fmaf does, so the
// results are bit-identical to two scalar FMAs in half the issue slots.
__device__ __forceinline__ void fma2(float w, float ax, float ay, float& ox, float& oy) {
    asm("{\n\t.reg .b64 pw, pa, po;\n\t"
        "mov.b64 pw, {%2, %2};\n\t"
        "mov.b64 pa, {%3, %4};\n\t"
        "mov.b64 po, {%0, %1};\n\t"
        "fma.rn.f32x2 po, pw, pa, po;\n\t"
        "mov.b64 {%0, %1}, po;\n\t}"
        : "+f"(ox), "+f"(oy)
        : "f"(w), "f"(ax), "f"(ay));
}

// (cx, cy) = (fma(ax, bx, cx), fma(ay, by, cy)) in one packed instruction.
__device__ __forceinline__ void fma2v(float ax, float ay, float bx, float by, float& cx, float& cy) {
    asm("{\n\t.reg .b64 pa, pb, pc;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mov.b64 pc, {%0, %1};\n\t"
        "fma.rn.f32x2 pc, pa, pb, pc;\n\t"
        "mov.b64 {%0, %1}, pc;\n\t}"
        : "+f"(cx), "+f"(cy)
        : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}

// (ox, oy) = (ax * bx, ay * by) in one packed instruction (mul.rn.f32x2).
__device__ __forceinline__ void mul2(float ax, float ay, float bx, float by, float& ox, float& oy) {
    asm("{\n\t.reg .b64 pa, pb;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "mul.rn.f32x2 pa, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pa;\n\t}"
        : "=f"(ox), "=f"(oy)
        : "f"(ax), "f"(ay), "f"(bx), "f"(by));
}

// Trilinear weights of the 8 corners in offset order c = dx + 2 dy + 4 dz,
// ((dx ? fx : 1 - fx) * (dy ? fy : 1 - fy)) * (dz ? fz : 1 - fz), the x pairs in packed
// multiplies (the same products, rounded the same way).
__device__ __forceinline__ void corner_weights(float fx, float fy, float fz, float w[8]) {
    const float gx = 1.0f - fx, gy = 1.0f - fy, gz = 1.0f - fz;
#pragma unroll
    for (int yz = 0; yz < 4; ++yz) {
        const float wy = (yz & 1) ? fy : gy, wz = (yz & 2) ? fz : gz;
        mul2(gx, fx, wy, wy, w[2 * yz], w[2 * yz + 1]);
        mul2(w[2 * yz], w[2 * yz + 1], wz, wz, w[2 * yz], w[2 * yz + 1]);
    }
}

template <bool kParity, int kFirst, int kCount>
__device__ __forceinline__ void derived_channels(const float4* __restrict__ brick, int E, int lx, int ly, int lz,
                                                 float fx, float fy, float fz, float* out) {
    const int px = kParity ? lx & 1 : 0, py = kParity ? ly & 1 : 0, pz = kParity ? lz & 1 : 0;
    const int base = (lz * E + ly) * E + lx;
    float wo[8];
    if (!kParity) corner_weights(fx, fy, fz, wo);
#pragma unroll
    for (int q = 0; q < kCount; ++q) out[q] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        // kParity: the corner of parity (c & 1, c >> 1 & 1, c >> 2 & 1), i.e. offset
        // parity ^ cell parity; otherwise the corner at offset (c & 1, c >> 1 & 1, c >> 2 & 1)
        const int dx = px ^ (c & 1), dy = py ^ ((c >> 1) & 1), dz = pz ^ ((c >> 2) & 1);
        const float w =
            kParity ? (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz) : wo[c];
        const float4* p = brick + 3 * (base + (dz * E + dy) * E + dx);
        if (kFirst == 0) {
            const float4 a = ldg_l2_256(p);
            fma2(w, a.x, a.y, out[0], out[1]);
            fma2(w, a.z, a.w, out[2], out[3]);
        }
        if (kFirst + kCount > 4) {
            const float4 m = ldg_l2_256(p + 1), t = ldg_l2_256(p + 2);
            float* o = out + (4 - kFirst);
            fma2(w, m.x, m.y, o[0], o[1]);
            fma2(w, m.z, m.w, o[2], o[3]);
            fma2(w, t.x, t.y, o[4], o[5]);
        }
    }
}

// derived_channels over a derived brick staged in shared memory (plain loads).
template <int kFirst, int kCount>
__device__ __forceinline__ void derived_channels_smem(const float4* brick, int E, int lx, int ly, int lz, float fx,
                                                      float fy, float fz, float* out) {
    const int base = (lz * E + ly) * E + lx;
#pragma unroll
    for (int q = 0; q < kCount; ++q) out[q] = 0.0f;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
        const float w = (dx ? fx : 1.0f - fx) * (dy ? fy : 1.0f - fy) * (dz ? fz : 1.0f - fz);
        const float4* p = brick + 3 * (base + (dz * E + dy) * E + dx);
        if (kFirst == 0) {
            const float4 a = p[0];
            fma2(w, a.x, a.y, out[0], out[1]);
            fma2(w, a.z, a.w, out[2], out[3]);
        }
        if (kFirst + kCount > 4) {
            const float4 m = p[1], t = p[2];
            float* o = out + (4 - kFirst);
            fma2(w, m.x, m.y, o[0], o[1]);
            fma2(w, m.z, m.w, o[2], o[3]);
            fma2(w, t.x, t.y, o[4], o[5]);
        }
    }
}

// The Hessian channels fld[4..9] of the derived field -- or zeros when the opacity
// has no curvature term (gamma = 0): the Hessian then enters nothing (w(kappa) =
// fma(0, kappa, 1) = 1 for any kappa, and every Hessian gradient carries the factor
// gamma), so results are unchanged and its 16 loads per sample are saved.
template <bool kParity>
__device__ __forceinline__ void load_hessian(const TissueDev& tp, const float4* __restrict__ brick, int E, int lx,
                                             int ly, int lz, const float f[3], float fld[10]) {
    if (tp.gk != 0.0f) {
        derived_channels<kParity, 4, 6>(brick, E, lx, ly, lz, f[0], f[1], f[2], fld + 4);
    } else {
#pragma unroll
        for (int q = 4; q < 10; ++q) fld[q] = 0.0f;
    }
}


// Trilinear value only (the vesselness channel): 8 corner voxels of the cell.
template <class Load>
__device__ __forceinline__ float value_eval(const Load& load, int base, float fx, float fy, float fz) {
    const int o = base + kEdge * kEdge + kEdge + 1;  // tap (1,1,1) = voxel (i0, j0, k0)
    const float c00 = fmaf(fx, load(o + 1), (1.f - fx) * load(o));
    const float c10 = fmaf(fx, load(o + kEdge + 1), (1.f - fx) * load(o + kEdge));
    const float c01 = fmaf(fx, load(o + kEdge * kEdge + 1), (1.f - fx) * load(o + kEdge * kEdge));
    const float c11 = fmaf(fx, load(o + kEdge * kEdge + kEdge + 1), (1.f - fx) * load(o + kEdge * kEdge + kEdge));
    const float c0 = fmaf(fy, c10, (1.f - fy) * c00);
    const float c1 = fmaf(fy, c11, (1.f - fy) * c01);
    return fmaf(fz, c1, (1.f - fz) * c0);
}

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float t) {
    return make_float4(fmaf(t, b.x - a.x, a.x), fmaf(t, b.y - a.y, a.y), fmaf(t, b.z - a.z, a.z),
                       fmaf(t, b.w - a.w, a.w));
}

// Everything one sample's optics compute on the way to its opacity and colour:
// the forward kernels keep alpha and col, the adjoint reuses the rest.
struct SampleOptics {
    float gg, r, gmag, kappa, hx, hy, hz, Hgx, Hgy, Hgz;  // |g|^2, 1/|g|, |g|, Eq. 3, unit normal, H g
    float gn, y;                                          // |g|/gmax and the second lookup coordinate
    int j, k;                                             // transfer-function cell
    float t, q;                                           // and its fractions
    float4 T00, T01, T10, T11, c;                         // cell entries and the looked-up RGBA
    float mg, wi, wk, raw, dot, d;                        // Eq. 4 factors, shading cosine
    float alpha, col[3];
};

// First half of a sample's optics, from I and the gradient alone (f[0..3]): |g|,
// the unit normal, the lookup coordinates and the transfer-function RGBA. Its
// opacity entry c.w decides whether the sample can be visible at all.
__device__ __forceinline__ void optics_tf(const float f[4], float vval, const TissueDev& tp,
                                          const float4* __restrict__ tf, float inv_gmax, SampleOptics& o) {
    const float gx = f[1], gy = f[2], gz = f[3];
    o.gg = fmaf(gx, gx, fmaf(gy, gy, gz * gz));
    o.r = o.gmag = o.hx = o.hy = o.hz = 0.0f;
    if (o.gg > 0.0f) {
        // one reciprocal square root gives |g|, the unit normal and 1/|g|^2
        o.r = rsqrtf(o.gg);
        o.gmag = o.gg * o.r;
        o.hx = gx * o.r;
        o.hy = gy * o.r;
        o.hz = gz * o.r;
    }
    o.gn = o.gmag * inv_gmax;
    o.y = tp.tf_mode == 1 ? o.gn : (tp.tf_mode == 2 ? vval : 0.0f);
    // piecewise-linear transfer function: x over tf_w entries, y over tf_h rows
    const int w = tp.tf_w, h = tp.tf_h;
    const float xs = fminf(fmaxf(f[0], 0.0f), 1.0f) * (float)(w - 1);
    o.j = min((int)xs, w - 2);
    if (!VR_CHECK(tp.status, o.j >= 0)) o.j = 0;
    o.t = xs - (float)o.j;
    if (h == 1) {
        o.k = 0;
        o.q = 0.0f;
        o.T00 = __ldg(tf + o.j);
        o.T01 = __ldg(tf + o.j + 1);
        o.T10 = o.T11 = make_float4(0.f, 0.f, 0.f, 0.f);
        o.c = lerp4(o.T00, o.T01, o.t);
    } else {
        const float ys = fminf(fmaxf(o.y, 0.0f), 1.0f) * (float)(h - 1);
        o.k = min((int)ys, h - 2);
        if (!VR_CHECK(tp.status, o.k >= 0)) o.k = 0;
        o.q = ys - (float)o.k;
        const float4* r0 = tf + (long long)o.k * w + o.j;
        o.T00 = __ldg(r0);
        o.T01 = __ldg(r0 + 1);
        o.T10 = __ldg(r0 + w);
        o.T11 = __ldg(r0 + w + 1);
        o.c = lerp4(lerp4(o.T00, o.T01, o.t), lerp4(o.T10, o.T11, o.t), o.q);
    }
}

// Second half: curvature (Eq. 3) from the Hessian f[4..9], Eq. 4 opacity, shading.
__device__ __forceinline__ void optics_rest(const float f[10], const float dir[3], const TissueDev& tp,
                                            SampleOptics& o) {
    const float gx = f[1], gy = f[2], gz = f[3];
    o.kappa = o.Hgx = o.Hgy = o.Hgz = 0.0f;
    if (o.gg > 0.0f) {
        // H g: the x and y rows in packed pairs (the same FMA chains)
        float hgx, hgy;
        mul2(f[8], f[9], gz, gz, hgx, hgy);
        fma2v(f[7], f[5], gy, gy, hgx, hgy);
        fma2v(f[4], f[7], gx, gx, hgx, hgy);
        o.Hgx = hgx;
        o.Hgy = hgy;
        o.Hgz = fmaf(f[8], gx, fmaf(f[9], gy, f[6] * gz));
        o.kappa = fmaf(gx, o.Hgx, fmaf(gy, o.Hgy, gz * o.Hgz)) * (o.r * o.r);
    }
    o.mg = tp.grad_mod ? fminf(o.gn, 1.0f) : 1.0f;
    o.wi = fmaf(tp.gk, o.kappa, 1.0f);
    o.wk = fminf(fmaxf(o.wi, 0.0f), tp.w_max);
    o.raw = tp.opacity_scale * o.c.w * o.mg * o.wk;
    o.alpha = fminf(fmaxf(o.raw, 0.0f), 1.0f);
    // optional step-size correction 1 - (1 - alpha)^e = -expm1(e log1p(-alpha)): accurate
    // relative to alpha also for nearly transparent samples
    if (tp.alpha_exp > 0.0f) o.alpha = -expm1f(tp.alpha_exp * log1pf(-o.alpha));
    o.dot = fmaf(o.hx, dir[0], fmaf(o.hy, dir[1], o.hz * dir[2]));
    o.d = fabsf(o.dot);
    if (tp.shading) {
        const float d2 = o.d * o.d, d4 = d2 * d2, d8 = d4 * d4, d16 = d8 * d8;
        const float lit = fmaf(tp.kd, o.d, tp.ka);
        const float spec = tp.ks * d16;
        o.col[0] = o.col[1] = spec;
        fma2v(o.c.x, o.c.y, lit, lit, o.col[0], o.col[1]);
        o.col[2] = fmaf(o.c.z, lit, spec);
    } else {
        o.col[0] = o.c.x;
        o.col[1] = o.c.y;
        o.col[2] = o.c.z;
    }
}

// Opacity (Eq. 4) and colour of one sample from its field (already scaled to
// mm units) and vesselness value, keeping the intermediate values in `o`.
__device__ __forceinline__ void optics_core(const float f[10], float vval, const float dir[3], const TissueDev& tp,
                                            const float4* __restrict__ tf, float inv_gmax, SampleOptics& o) {
    optics_tf(f, vval, tp, tf, inv_gmax, o);
    optics_rest(f, dir, tp, o);
}

// Opacity (Eq. 4) and colour of one sample from its field (already scaled to
// mm units) and vesselness value.
__device__ __forceinline__ void sample_optics(const float f[10], float vval, const float dir[3], const TissueDev& tp,
                                              const float4* __restrict__ tf, float inv_gmax, float& alpha,
                                              float col[3]) {
    SampleOptics o;
    optics_core(f, vval, dir, tp, tf, inv_gmax, o);
    alpha = o.alpha;
    col[0] = o.col[0];
    col[1] = o.col[1];
    col[2] = o.col[2];
}

// Divide the raw stencil sums by the spacing (gradient) and spacing products (Hessian).
__device__ __forceinline__ void scale_field(float f[10], const float is[3]) {
    f[1] *= is[0];
    f[2] *= is[1];
    f[3] *= is[2];
    f[4] *= is[0] * is[0];
    f[5] *= is[1] * is[1];
    f[6] *= is[2] * is[2];
    f[7] *= is[0] * is[1];
    f[8] *= is[0] * is[2];
    f[9] *= is[1] * is[2];
}

// Storage brick (8^3 cells) of cell i0 and the offset of its 4-tap stencil origin
// (voxel i0 - 1 per axis) in the brick's 12^3 block.
__device__ __forceinline__ int storage_brick(const VolumeDev& v, const int i0[3], int& base) {
    base = (((i0[2] & 7) * kEdge) + (i0[1] & 7)) * kEdge + (i0[0] & 7);
    return ((i0[2] >> 3) * v.nsb[1] + (i0[1] >> 3)) * v.nsb[0] + (i0[0] >> 3);
}

// First sample index >= k whose cell lies outside the skip brick (b0, b1, b2) of B
// cells per edge, for a ray currently in that brick; a lower bound (one sample
// earlier is re-tested by the caller), never beyond ns.
// brick_exit_k from the position U[q] = u0 + k du of the current sample k: the
// crossing counted in steps from k (a smaller, so more precise, float quotient);
// conservative in the same way.
__device__ __forceinline__ int brick_exit_k_at(const RayDev& r, const long long U[3], const int bcell[3], int B,
                                               int k, int ns) {
    float kmin = (float)(ns - k);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float st = fx_to_float(r.du[q]);
        if (r.du[q] == 0) continue;
        const int bound = st > 0.0f ? B * (bcell[q] + 1) : B * bcell[q];
        const float ks = fx_to_float(((long long)bound << 32) - U[q]) / st;
        kmin = fminf(kmin, st > 0.0f ? ceilf(ks) : floorf(ks) + 1.0f);
    }
    int ke = k + (int)fmaxf(kmin, 0.0f) - 1;  // back off one sample
    if (ke <= k) ke = k + 1;
    return min(ke, ns);
}

__device__ __forceinline__ int brick_exit_k(const RayDev& r, const int bcell[3], int B, int k, int ns) {
    float kmin = (float)ns;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const float st = fx_to_float(r.du[q]);  // step (voxels)
        if (r.du[q] == 0) continue;
        const int bound = st > 0.0f ? B * (bcell[q] + 1) : B * bcell[q];
        // u(k) = (u0 + k du) 2^-32 crosses `bound` at k* = (bound 2^32 - u0) / du
        const float ks = fx_to_float(((long long)bound << 32) - r.u0[q]) / st;
        kmin = fminf(kmin, st > 0.0f ? ceilf(ks) : floorf(ks) + 1.0f);
    }
    int ke = (int)fmaxf(kmin, 0.0f) - 1;  // back off one sample
    if (ke <= k) ke = k + 1;
    return min(ke, ns);
}

}  // namespace vr
