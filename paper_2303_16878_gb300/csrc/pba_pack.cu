// pba_pack.cu -- per-frame packing (once per upload).
//
// For every pixel u of a frame (Sec. IV-A five-channel cue image):
//   - a sampling texel: d (FP32, 0 when the pixel is not valid) and g, n in
//     FP16 or FP32, so one bilinear tap is one 16- or 32-byte load;
//   - when the pixel is valid, a pixel-point p_u = R_o pi^-1(u, d) + t_o with
//     its intensity g_u, normal n_u^o = R_o n_u (Supp., p_u) and pixel index,
//     written in raster order to a compacted array (block-wide ballot scan).
// Unprojection pi^-1 (Sec. III): pinhole p = d K^-1 (u, v, 1)^T; spherical
// p = d (cos el cos az, cos el sin az, sin el) with az = (u - c_x) / f_x,
// el = (v - c_y) / f_y.  Validity: range_min <= d <= range_max, d > 0 and
// |n| > 0.5, evaluated in double so that the decision is exact for the
// float32 inputs.
#include "pba_internal.cuh"
#include "pba_device.cuh"

namespace pba {

namespace {

constexpr int kPackThreads = 1024;

__device__ __forceinline__ bool pixel_valid(const float* px, double rmin, double rmax) {
    double d = px[1];
    double n2 = (double)px[2] * px[2] + (double)px[3] * px[3] + (double)px[4] * px[4];
    return d > 0.0 && d >= rmin && d <= rmax && n2 > 0.25;
}

template <int TEXEL>
__global__ void __launch_bounds__(kPackThreads) k_pack(const float* __restrict__ raw,
                                                       const FrameInfo* __restrict__ frames,
                                                       const SensorDev* __restrict__ sensors,
                                                       const int* __restrict__ frame_ids, void* texels,
                                                       float4* __restrict__ pts_pg, float4* __restrict__ pts_n,
                                                       int* __restrict__ pts_pix, int* __restrict__ n_points,
                                                       double rmin, double rmax) {
    __shared__ int s_warp[kPackThreads / 32];
    __shared__ int s_base, s_total;
    const int f = frame_ids[blockIdx.x];
    const FrameInfo fr = frames[f];
    const SensorDev sd = sensors[fr.sensor];
    const int npx = fr.width * fr.height;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int tile = 0; tile < npx; tile += kPackThreads) {
        const int px = tile + threadIdx.x;
        bool valid = false;
        float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (px < npx) {
            const float* src = raw + (fr.px_offset + px) * 5;
            for (int k = 0; k < 5; ++k) c[k] = src[k];
            valid = pixel_valid(c, rmin, rmax);
            // usable: the pixel and its four neighbours are valid, i.e. the
            // central differences of the Supp. are defined at this pixel
            bool usable = valid;
            {
                const int col = px % fr.width, row = px / fr.width;
                const bool wrap = fr.model == 1;
                const int nb[4][2] = {{row - 1, col}, {row + 1, col}, {row, col - 1}, {row, col + 1}};
                for (int q = 0; q < 4 && usable; ++q) {
                    int r = nb[q][0], cc = nb[q][1];
                    if (r < 0 || r >= fr.height) { usable = false; break; }
                    if (cc < 0 || cc >= fr.width) {
                        if (!wrap) { usable = false; break; }
                        cc = cc < 0 ? cc + fr.width : cc - fr.width;
                    }
                    usable = pixel_valid(raw + (fr.px_offset + (long long)r * fr.width + cc) * 5, rmin, rmax);
                }
            }
            const long long t = fr.px_offset + px;
            if (TEXEL == 1) {
                Tex16 tx;
                tx.d = valid ? c[1] : 0.f;
                tx.g_nx = __halves2half2(__float2half_rn(c[0]), __float2half_rn(c[2]));
                tx.ny_nz = __halves2half2(__float2half_rn(c[3]), __float2half_rn(c[4]));
                tx.usable = usable ? 1u : 0u;
                reinterpret_cast<Tex16*>(texels)[t] = tx;
            } else {
                float4* t4 = reinterpret_cast<float4*>(texels) + 2 * t;
                t4[0] = make_float4(valid ? c[1] : 0.f, c[0], c[2], c[3]);
                t4[1] = make_float4(c[4], __uint_as_float(usable ? 1u : 0u), 0.f, 0.f);
            }
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) s_warp[warp] = __popc(ballot);
        __syncthreads();
        if (warp == 0) {
            // exclusive scan of the 32 warp counts; the inclusive total goes to s_total
            const int v = s_warp[lane];
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            s_warp[lane] = incl - v;
            if (lane == 31) s_total = incl;
        }
        __syncthreads();
        if (valid) {
            const int within = __popc(ballot & ((1u << lane) - 1u));
            const int idx = s_base + s_warp[warp] + within;
            const int col = px % fr.width, row = px / fr.width;
            const float d = c[1];
            float p[3];
            if (fr.model == 0) {
                p[0] = d * ((col - fr.cx) / fr.fx);
                p[1] = d * ((row - fr.cy) / fr.fy);
                p[2] = d;
            } else {
                float saz, caz, sel, cel;
                sincosf((col - fr.cx) / fr.fx, &saz, &caz);
                sincosf((row - fr.cy) / fr.fy, &sel, &cel);
                p[0] = d * (cel * caz);
                p[1] = d * (cel * saz);
                p[2] = d * sel;
            }
            float pu[3], no[3];
            for (int r = 0; r < 3; ++r) {
                pu[r] = sd.R[3 * r] * p[0] + sd.R[3 * r + 1] * p[1] + sd.R[3 * r + 2] * p[2] + sd.t[r];
                no[r] = sd.R[3 * r] * c[2] + sd.R[3 * r + 1] * c[3] + sd.R[3 * r + 2] * c[4];
            }
            pts_pg[fr.pt_offset + idx] = make_float4(pu[0], pu[1], pu[2], c[0]);
            pts_n[fr.pt_offset + idx] = make_float4(no[0], no[1], no[2], 0.f);
            pts_pix[fr.pt_offset + idx] = px;
        }
        __syncthreads();
        if (threadIdx.x == 0) s_base += s_total;
        __syncthreads();
    }
    if (threadIdx.x == 0) n_points[f] = s_base;
}

}  // namespace

// Central differences of the Supp. at every usable pixel of the frames
// (d/du = (I(r, c + 1) - I(r, c - 1)) / 2, d/dv = (I(r + 1, c) - I(r - 1, c)) / 2,
// columns wrapping for the spherical model), from the texels as sampled.
template <int TEXEL>
__global__ void k_grad(const void* __restrict__ texels, const FrameInfo* __restrict__ frames,
                       const int* __restrict__ frame_ids, float4* __restrict__ gtex) {
    const FrameInfo fr = frames[frame_ids[blockIdx.y]];
    const int npx = fr.width * fr.height;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npx) return;
    const void* tex = TEXEL == 1 ? (const void*)(reinterpret_cast<const Tex16*>(texels) + fr.px_offset)
                                 : (const void*)(reinterpret_cast<const Tex32*>(texels) + fr.px_offset);
    float4* out = gtex + 3 * (fr.px_offset + px);
    const Texel me = load_texel<TEXEL>(tex, px);
    if (!me.usable) {
        out[0] = out[1] = out[2] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    const int row = px / fr.width, col = px % fr.width;
    const int cl = col == 0 ? fr.width - 1 : col - 1, cr = col == fr.width - 1 ? 0 : col + 1;  // usable: in range
    float L[5], R[5], U[5], D[5];
    channels(load_texel<TEXEL>(tex, row * fr.width + cl), L);
    channels(load_texel<TEXEL>(tex, row * fr.width + cr), R);
    channels(load_texel<TEXEL>(tex, (row - 1) * fr.width + col), U);
    channels(load_texel<TEXEL>(tex, (row + 1) * fr.width + col), D);
    float gu[5], gv[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        gu[c] = 0.5f * (R[c] - L[c]);
        gv[c] = 0.5f * (D[c] - U[c]);
    }
    out[0] = make_float4(gu[0], gu[1], gu[2], gu[3]);
    out[1] = make_float4(gu[4], gv[0], gv[1], gv[2]);
    out[2] = make_float4(gv[3], gv[4], 0.f, 0.f);
}

cudaError_t launch_pack(const float* raw, const FrameInfo* frames, const SensorDev* sensors, const int* frame_ids,
                        int n, int texel_precision, void* texels, float4* pts_pg, float4* pts_n, int* pts_pix,
                        int* n_points, double range_min, double range_max, cudaStream_t s, float4* gtex,
                        int max_px) {
    if (n <= 0) return cudaSuccess;
    if (texel_precision == 1)
        k_pack<1><<<n, kPackThreads, 0, s>>>(raw, frames, sensors, frame_ids, texels, pts_pg, pts_n, pts_pix,
                                             n_points, range_min, range_max);
    else
        k_pack<0><<<n, kPackThreads, 0, s>>>(raw, frames, sensors, frame_ids, texels, pts_pg, pts_n, pts_pix,
                                             n_points, range_min, range_max);
    if (gtex && max_px > 0) {
        for (int f0 = 0; f0 < n; f0 += 65535) {  // grid.y limit
            const dim3 grid((max_px + 255) / 256, n - f0 < 65535 ? n - f0 : 65535);
            if (texel_precision == 1) k_grad<1><<<grid, 256, 0, s>>>(texels, frames, frame_ids + f0, gtex);
            else k_grad<0><<<grid, 256, 0, s>>>(texels, frames, frame_ids + f0, gtex);
        }
    }
    return cudaGetLastError();
}

}  // namespace pba
