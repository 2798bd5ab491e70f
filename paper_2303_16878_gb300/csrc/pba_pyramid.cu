// pba_pyramid.cu -- one pyramid level down (Sec. IV-A: each level of the
// multi-cue pyramid has half the resolution of the previous one).
//
// Coarse pixel (r, c) summarises the fine 2 x 2 block (2r..2r+1, 2c..2c+1).
// It is valid when all four fine pixels are valid (d > 0, range_min <= d <=
// range_max, |n|^2 > 0.25, the rule of the pixel-point builder); then g and d
// are the block means and n the normalised sum of the four normals.  The
// arithmetic is float64 with explicit round-to-nearest operations (no fused
// multiply-add), from the float32 inputs, rounded once to float32 at the end:
// the sums of four floats are exact, so the result does not depend on the
// order of evaluation beyond the one written here.
#include "pba_internal.cuh"

namespace pba {
namespace {

__device__ __forceinline__ bool fine_valid(const float* px, double rmin, double rmax) {
    const double d = px[1];
    const double n2 = (double)px[2] * px[2] + (double)px[3] * px[3] + (double)px[4] * px[4];
    return d > 0.0 && d >= rmin && d <= rmax && n2 > 0.25;
}

__global__ void k_downsample(const float* __restrict__ raw, const FrameInfo* __restrict__ frames,
                             const int* __restrict__ frame_ids, const long long* __restrict__ out_offsets,
                             float* __restrict__ out, double rmin, double rmax) {
    const int f = frame_ids[blockIdx.y];
    const FrameInfo fr = frames[f];
    const int Wc = fr.width / 2, Hc = fr.height / 2;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= Wc * Hc) return;
    const int r = px / Wc, c = px % Wc;
    const float* img = raw + fr.px_offset * 5;
    const float* q[4] = {img + ((long long)(2 * r) * fr.width + 2 * c) * 5,
                         img + ((long long)(2 * r) * fr.width + 2 * c + 1) * 5,
                         img + ((long long)(2 * r + 1) * fr.width + 2 * c) * 5,
                         img + ((long long)(2 * r + 1) * fr.width + 2 * c + 1) * 5};
    float* o = out + (out_offsets[blockIdx.y] + px) * 5;
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 4; ++k) ok = ok && fine_valid(q[k], rmin, rmax);
    double s[5];
#pragma unroll
    for (int ch = 0; ch < 5; ++ch)
        s[ch] = __dadd_rn(__dadd_rn((double)q[0][ch], (double)q[1][ch]), __dadd_rn((double)q[2][ch], (double)q[3][ch]));
    const double nn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(s[2], s[2]), __dmul_rn(s[3], s[3])), __dmul_rn(s[4], s[4])));
    if (!ok || !(nn > 0.0)) {
#pragma unroll
        for (int ch = 0; ch < 5; ++ch) o[ch] = 0.f;
        return;
    }
    o[0] = __double2float_rn(__dmul_rn(s[0], 0.25));
    o[1] = __double2float_rn(__dmul_rn(s[1], 0.25));
    o[2] = __double2float_rn(__ddiv_rn(s[2], nn));
    o[3] = __double2float_rn(__ddiv_rn(s[3], nn));
    o[4] = __double2float_rn(__ddiv_rn(s[4], nn));
}

}  // namespace

cudaError_t launch_downsample(const float* raw, const FrameInfo* frames, const int* frame_ids,
                              const long long* out_offsets, int n, int max_coarse_px, float* out, double range_min,
                              double range_max, cudaStream_t s) {
    if (n <= 0 || max_coarse_px <= 0) return cudaSuccess;
    for (int f0 = 0; f0 < n; f0 += 65535) {  // grid.y limit
        const dim3 grid((max_coarse_px + 255) / 256, n - f0 < 65535 ? n - f0 : 65535);
        k_downsample<<<grid, 256, 0, s>>>(raw, frames, frame_ids + f0, out_offsets + f0, out, range_min, range_max);
    }
    return cudaGetLastError();
}

}  // namespace pba
