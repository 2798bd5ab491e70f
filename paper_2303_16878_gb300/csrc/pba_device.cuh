// pba_device.cuh -- device helpers shared by the linearisation and adjoint
// kernels: the arctangent of the spherical projection, texel loads of the
// packed target images, and the column indices of the sampling stencil.
#pragma once

#include "pba_internal.cuh"

namespace pba {

// ------------------------------------------------------------ arctangent

// atan(t) for t in [0, 1] as t + t s Q(s), s = t^2, Q of degree 7
// (gen_atan_poly.py fits Q towards the minimax error in float64 and prints
// the float32 error of this evaluation: below 8e-8 rad, about 1.3 ulp of
// pi / 4; the leading term t is added last, with one rounding).
__device__ __forceinline__ float atan_unit(float t) {
    const float s = t * t;
    float q = 0.0026222029700875282f;
    q = fmaf(q, s, -0.015132364816963673f);
    q = fmaf(q, s, 0.04112157225608826f);
    q = fmaf(q, s, -0.07366681098937988f);
    q = fmaf(q, s, 0.10573919862508774f);
    q = fmaf(q, s, -0.1418597251176834f);
    q = fmaf(q, s, 0.1999039649963379f);
    q = fmaf(q, s, -0.33332985639572144f);
    return fmaf(t * s, q, t);
}

// Spherical projection (Eq. spherical-projection) of pbar = (x, y, z):
// u = cx + fx atan2(y, x), v = cy + fy atan2(z, sqrt(x^2 + y^2)), returned as
// the column c0 = floor(u), its bilinear weight a = u - c0, and v.
// The azimuth is written sgn(y) (B + sigma r) with r = atan(t) in [0, pi/4],
// t = min(|x|, |y|) / max(|x|, |y|) (a reciprocal refined by one Newton
// step), B in {0, pi/2, pi} and sigma = +-1 by octant, so u = U + s with
// U = cx + sgn(y) fx B (fxh = fx pi / 2 and fxp = fx pi are per-pair
// constants; for the spherical intrinsics fx = -W / 2 pi, cx = W / 2 every U
// is an exact integer) and s = sgn(y) sigma fx r, |s| <= |fx| pi / 4.  The
// floor and the fraction are taken of s (float32 spacing at most W / 2^26)
// rather than of u, whose float32 spacing near W is 16 times coarser.
// The elevation is atan(|z| / rxy) with irxy = 1 / rxy given, or
// pi/2 - atan(rxy / |z|) above 45 degrees; NaN or infinite inputs give a v
// that fails every bound.
__device__ __forceinline__ void spherical_project(float x, float y, float z, float irxy, float fx, float fy,
                                                  float cx, float cy, float fxh, float fxp, int& c0, float& a,
                                                  float& v) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float rc = __fdividef(1.f, mx);
    const float t0 = mn * rc;
    const float t = mx > 0.f ? fmaf(fmaf(-t0, mx, mn), rc, t0) : 0.f;
    const float r = atan_unit(t);
    const bool swap = ay > ax, neg_x = x < 0.f;
    const float sg = y < 0.f ? -1.f : 1.f;
    const float U = fmaf(sg, swap ? fxh : (neg_x ? fxp : 0.f), cx);
    const float s = (swap != neg_x ? -sg : sg) * (fx * r);
    const float Ui = floorf(U);
    const float w = (U - Ui) + s;
    const float fw = floorf(w);
    c0 = (int)(Ui + fw);
    a = w - fw;
    const float te = fabsf(z) * irxy;
    const bool steep = te > 1.f;
    const float re = atan_unit(steep ? __fdividef(1.f, te) : te);
    const float el = steep ? 1.57079637f - re : re;
    v = fmaf(fy, z < 0.f ? -el : el, cy);
}

// ------------------------------------------------------------ texel access

struct Texel {
    float d, g, nx, ny, nz;
    bool usable;
};

// An FP16 texel (Tex16 as 4 words) in FP32.
__device__ __forceinline__ Texel texel_of(const uint4 v) {
    Texel t;
    t.d = __uint_as_float(v.x);
    __half2 a = *reinterpret_cast<const __half2*>(&v.y);
    __half2 b = *reinterpret_cast<const __half2*>(&v.z);
    const float2 fa = __half22float2(a), fb = __half22float2(b);
    t.g = fa.x;
    t.nx = fa.y;
    t.ny = fb.x;
    t.nz = fb.y;
    t.usable = v.w != 0u;
    return t;
}

template <int TEXEL>
__device__ __forceinline__ Texel load_texel(const void* __restrict__ base, int idx) {
    Texel t;
    if (TEXEL == 1) {
        t = texel_of(__ldg(reinterpret_cast<const uint4*>(base) + idx));
    } else {
        const float4* p = reinterpret_cast<const float4*>(base) + 2 * idx;
        const float4 v0 = __ldg(p);
        const float2 v1 = __ldg(reinterpret_cast<const float2*>(p + 1));
        t.d = v0.x;
        t.g = v0.y;
        t.nx = v0.z;
        t.ny = v0.w;
        t.nz = v1.x;
        t.usable = __float_as_uint(v1.y) != 0u;
    }
    return t;
}

// A bilinear tap as loaded.  FP16 texels keep their words until a channel other
// than the FP32 depth is needed, so the binary16 conversions are only done for
// points whose taps are usable and that pass the occlusion test.
template <int TEXEL>
struct Tap;
template <>
struct Tap<1> {
    uint4 v;
    __device__ __forceinline__ bool usable() const { return v.w != 0u; }
    __device__ __forceinline__ float depth() const { return __uint_as_float(v.x); }
    __device__ __forceinline__ void rest(float& g, float& nx, float& ny, float& nz) const {
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
        g = a.x;
        nx = a.y;
        ny = b.x;
        nz = b.y;
    }
    // (g, n_x), (n_y, n_z)
    __device__ __forceinline__ void rest2(float2& gnx, float2& nynz) const {
        gnx = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
        nynz = __half22float2(*reinterpret_cast<const __half2*>(&v.z));
    }
};
template <>
struct Tap<0> {
    Texel t;
    __device__ __forceinline__ bool usable() const { return t.usable; }
    __device__ __forceinline__ float depth() const { return t.d; }
    __device__ __forceinline__ void rest(float& g, float& nx, float& ny, float& nz) const {
        g = t.g;
        nx = t.nx;
        ny = t.ny;
        nz = t.nz;
    }
    __device__ __forceinline__ void rest2(float2& gnx, float2& nynz) const {
        gnx = make_float2(t.g, t.nx);
        nynz = make_float2(t.ny, t.nz);
    }
};

// All four taps usable (FP16 texels: the flags are 1 or 0, so one AND of the words).
__device__ __forceinline__ bool all_usable(const Tap<1>& A, const Tap<1>& B, const Tap<1>& C, const Tap<1>& D) {
    return (A.v.w & B.v.w & C.v.w & D.v.w) != 0u;
}
__device__ __forceinline__ bool all_usable(const Tap<0>& A, const Tap<0>& B, const Tap<0>& C, const Tap<0>& D) {
    return A.t.usable && B.t.usable && C.t.usable && D.t.usable;
}

template <int TEXEL>
__device__ __forceinline__ Tap<TEXEL> load_tap(const void* __restrict__ base, int idx) {
    Tap<TEXEL> a;
    if constexpr (TEXEL == 1)
        a.v = __ldg(reinterpret_cast<const uint4*>(base) + idx);
    else
        a.t = load_texel<0>(base, idx);
    return a;
}

__device__ __forceinline__ void channels(const Texel& t, float (&x)[5]) {
    x[0] = t.g;
    x[1] = t.d;
    x[2] = t.nx;
    x[3] = t.ny;
    x[4] = t.nz;
}

// Column indices c0 - 1, c0, c0 + 1, c0 + 2 (wrapped modulo W for the spherical model).
__device__ __forceinline__ void stencil_cols(int c0, int W, bool wrap, int& cm1, int& cc, int& cp1, int& cp2) {
    cc = c0;
    if (wrap) {
        if (cc < 0 || cc >= W) {
            cc %= W;
            if (cc < 0) cc += W;
        }
        cm1 = cc == 0 ? W - 1 : cc - 1;
        cp1 = cc == W - 1 ? 0 : cc + 1;
        cp2 = cp1 == W - 1 ? 0 : cp1 + 1;
    } else {
        cm1 = cc - 1;
        cp1 = cc + 1;
        cp2 = cc + 2;
    }
}

}  // namespace pba
