// pba_device.cuh -- device helpers shared by the linearisation and adjoint
// kernels: the arctangent of the spherical projection, texel loads of the
// packed target images, and the column indices of the sampling stencil.
#pragma once

#include "pba_internal.cuh"

namespace pba {

// ------------------------------------------------------------ arctangent

// atan2(y, x) for the spherical projection: reduce to t = min(|x|,|y|) /
// max(|x|,|y|) in [0, 1], approximate atan(t) = t P(t^2) with a degree-8
// polynomial fitted by least squares (gen_atan_poly.py prints the
// coefficients and its float32 error, max 3e-7 rad), then reflect into the
// octant.  atan2(0, 0) = 0.
__device__ __forceinline__ float atan2_poly(float y, float x) {
    const float ax = fabsf(x), ay = fabsf(y);
    const float mx = fmaxf(ax, ay), mn = fminf(ax, ay);
    const float t = mx > 0.f ? __fdividef(mn, mx) : 0.f;
    const float s = t * t;
    float p = 0.002932762f;
    p = fmaf(p, s, -0.01641319f);
    p = fmaf(p, s, 0.043278243f);
    p = fmaf(p, s, -0.075569004f);
    p = fmaf(p, s, 0.10667487f);
    p = fmaf(p, s, -0.14211106f);
    p = fmaf(p, s, 0.19993694f);
    p = fmaf(p, s, -0.33333138f);
    p = fmaf(p, s, 1.0f);
    float r = t * p;
    if (ay > ax) r = 1.57079637f - r;
    if (x < 0.f) r = 3.14159274f - r;
    return y < 0.f ? -r : r;
}

// ------------------------------------------------------------ texel access

struct Texel {
    float d, g, nx, ny, nz;
    bool usable;
};

template <int TEXEL>
__device__ __forceinline__ Texel load_texel(const void* __restrict__ base, int idx) {
    Texel t;
    if (TEXEL == 1) {
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + idx);
        t.d = __uint_as_float(v.x);
        __half2 a = *reinterpret_cast<const __half2*>(&v.y);
        __half2 b = *reinterpret_cast<const __half2*>(&v.z);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        t.g = fa.x;
        t.nx = fa.y;
        t.ny = fb.x;
        t.nz = fb.y;
        t.usable = v.w != 0u;
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
