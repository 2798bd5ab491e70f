// pba_pack.cu -- per-frame packing (once per upload), in two passes over all
// SMs, then the central differences.
//
// For every pixel u of a frame (Sec. IV-A five-channel cue image):
//   - pass 1 (k_pack_valid): its validity as a byte, and per tile of 1024
//     pixels the count of valid ones;
//   - pass 2 (k_pack_points), from one read of the pixel's channels: a
//     sampling texel: d (FP32, 0 when the pixel is not valid), g and n in FP16
//     or FP32, and the usable flag (the pixel and its four neighbours valid),
//     so one bilinear tap is one 16- or 32-byte load; and, when the pixel is
//     valid, a pixel-point p_u = R_o pi^-1(u, d) + t_o with its intensity g_u,
//     normal n_u^o = R_o n_u (Supp., p_u) and pixel index, written in raster
//     order at the offset given by the counts of the frame's earlier tiles;
//   - k_grad: the central differences of the Supp. at every usable pixel.
// Unprojection pi^-1 (Sec. III): pinhole p = d K^-1 (u, v, 1)^T; spherical
// p = d (cos el cos az, cos el sin az, sin el) with az = (u - c_x) / f_x,
// el = (v - c_y) / f_y.  Validity: range_min <= d <= range_max, d > 0 and
// |n| > 0.5, decided in FP32 exactly as the double evaluation of the float32
// inputs would decide it (see pixel_valid).
#include <cfloat>

#include "pba_internal.cuh"
#include "pba_device.cuh"

namespace pba {

namespace {

constexpr int kPackThreads = 256;
constexpr int kPackTile = 1024;  // pixels per CTA: 4 per thread, pixel tile * 1024 + 256 k + thread

// Validity of a raw pixel (Sec. IV-A): range_min <= d <= range_max, d > 0 and
// |n|^2 > 0.25, decided exactly as the double evaluation of the float inputs
// would: the range limits are their float images rounded inwards (so the float
// comparisons agree with the double ones), and |n|^2 is summed in FP32 (error
// below 2e-7 |n|^2) unless it lies within 1e-6 of the threshold, where the
// double sum decides.
__device__ __forceinline__ bool pixel_valid(const float* px, float rmin, float rmax) {
    const float d = px[1];
    if (!(d > 0.f && d >= rmin && d <= rmax)) return false;
    const float nx = px[2], ny = px[3], nz = px[4];
    const float s = fmaf(nz, nz, fmaf(ny, ny, nx * nx));
    if (fabsf(s - 0.25f) > 1e-6f) return s > 0.25f;
    const double n2 = (double)nx * nx + (double)ny * ny + (double)nz * nz;
    return n2 > 0.25;
}

// Pass 1, one CTA per 1024 pixels of a frame: every pixel's validity as a
// byte and the tile's count of valid pixels.
__global__ void __launch_bounds__(kPackThreads) k_pack_valid(const float* __restrict__ raw,
                                                             const FrameInfo* __restrict__ frames,
                                                             const int* __restrict__ frame_ids,
                                                             unsigned char* __restrict__ valid_px,
                                                             int* __restrict__ tile_counts, int max_tiles, float rmin,
                                                             float rmax) {
    const int f = frame_ids[blockIdx.y];
    const FrameInfo fr = frames[f];
    const int npx = fr.width * fr.height;
    const int tile = blockIdx.x;
    if (tile * kPackTile >= npx) return;
    int count = 0;
#pragma unroll
    for (int k = 0; k < kPackTile / kPackThreads; ++k) {
        const int px = tile * kPackTile + k * kPackThreads + threadIdx.x;
        bool valid = false;
        if (px < npx) {
            const float* src = raw + (fr.px_offset + px) * 5;
            float c[5];
#pragma unroll
            for (int q = 0; q < 5; ++q) c[q] = src[q];
            valid = pixel_valid(c, rmin, rmax);
            valid_px[fr.px_offset + px] = valid ? 1 : 0;
        }
        count += __syncthreads_count(valid);
    }
    if (threadIdx.x == 0) tile_counts[(long long)f * max_tiles + tile] = count;
}

// The sampling texel of a pixel, with its usable flag (the pixel and its four
// neighbours are valid, i.e. the central differences of the Supp. are defined
// there; columns wrap for the spherical model).
template <int TEXEL>
__device__ __forceinline__ void write_texel(const FrameInfo& fr, const unsigned char* __restrict__ vf, int px,
                                            bool valid, const float (&c)[5], void* texels) {
    bool usable = valid;
    if (usable) {
        const int col = px % fr.width, row = px / fr.width;
        const bool wrap = fr.model == 1;
        const int cl = col > 0 ? col - 1 : (wrap ? fr.width - 1 : -1);
        const int cr = col < fr.width - 1 ? col + 1 : (wrap ? 0 : -1);
        usable = row > 0 && row < fr.height - 1 && cl >= 0 && cr >= 0 && vf[px - fr.width] && vf[px + fr.width] &&
                 vf[row * fr.width + cl] && vf[row * fr.width + cr];
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

// Pass 2: every pixel's texel (write_texel) and the tile's valid pixels as
// pixel-points p_u = R_o pi^-1(u, d) + t_o with g_u, n_u^o = R_o n_u and the
// pixel index, written in raster order at the tile's offset (the counts of the
// frame's earlier tiles), from one read of the pixel's channels; the CTA of tile
// 0 also writes the frame's point count.
template <int TEXEL>
__global__ void __launch_bounds__(kPackThreads) k_pack_points(const float* __restrict__ raw,
                                                              const FrameInfo* __restrict__ frames,
                                                              const SensorDev* __restrict__ sensors,
                                                              const int* __restrict__ frame_ids,
                                                              const unsigned char* __restrict__ valid_px,
                                                              const int* __restrict__ tile_counts, int max_tiles,
                                                              void* __restrict__ texels,
                                                              float4* __restrict__ pts_pg, float4* __restrict__ pts_n,
                                                              int* __restrict__ pts_pix, int* __restrict__ n_points) {
    __shared__ int s_warp[kPackThreads / 32];
    __shared__ int s_base;
    const int f = frame_ids[blockIdx.y];
    const FrameInfo fr = frames[f];
    const int npx = fr.width * fr.height;
    const int tile = blockIdx.x;
    if (tile * kPackTile >= npx) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (warp == 0) {
        const int n_tiles = (npx + kPackTile - 1) / kPackTile;
        const int* tc = tile_counts + (long long)f * max_tiles;
        int before = 0, all = 0;
        for (int t = lane; t < n_tiles; t += 32) {
            const int v = tc[t];
            all += v;
            if (t < tile) before += v;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            before += __shfl_xor_sync(0xffffffffu, before, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if (lane == 0) {
            s_base = before;
            if (tile == 0) n_points[f] = all;
        }
    }
    const SensorDev sd = sensors[fr.sensor];
    for (int k = 0; k < kPackTile / kPackThreads; ++k) {
        const int px = tile * kPackTile + k * kPackThreads + threadIdx.x;
        const bool valid = px < npx && valid_px[fr.px_offset + px] != 0;
        float c[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
        if (px < npx) {
            const float* src = raw + (fr.px_offset + px) * 5;
#pragma unroll
            for (int q = 0; q < 5; ++q) c[q] = src[q];
            write_texel<TEXEL>(fr, valid_px + fr.px_offset, px, valid, c, texels);
        }
        const unsigned ballot = __ballot_sync(0xffffffffu, valid);
        if (lane == 0) s_warp[warp] = __popc(ballot);
        __syncthreads();
        int before_warp = 0, total = 0;
#pragma unroll
        for (int w = 0; w < kPackThreads / 32; ++w) {
            const int v = s_warp[w];
            before_warp += w < warp ? v : 0;
            total += v;
        }
        if (valid) {
            const int idx = s_base + before_warp + __popc(ballot & ((1u << lane) - 1u));
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
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                pu[r] = sd.R[3 * r] * p[0] + sd.R[3 * r + 1] * p[1] + sd.R[3 * r + 2] * p[2] + sd.t[r];
                no[r] = sd.R[3 * r] * c[2] + sd.R[3 * r + 1] * c[3] + sd.R[3 * r + 2] * c[4];
            }
            pts_pg[fr.pt_offset + idx] = make_float4(pu[0], pu[1], pu[2], c[0]);
            pts_n[fr.pt_offset + idx] = make_float4(no[0], no[1], no[2], 0.f);
            pts_pix[fr.pt_offset + idx] = px;
        }
        __syncthreads();  // s_warp is rewritten by the next round
        if (threadIdx.x == 0) s_base += total;
        __syncthreads();
    }
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

int pack_tiles(int max_px) { return (max_px + kPackTile - 1) / kPackTile; }

cudaError_t launch_pack(const float* raw, const FrameInfo* frames, const SensorDev* sensors, const int* frame_ids,
                        int n, int texel_precision, void* texels, float4* pts_pg, float4* pts_n, int* pts_pix,
                        int* n_points, double range_min, double range_max, cudaStream_t s, float4* gtex,
                        int max_px, int* tile_counts, unsigned char* valid_px) {
    if (n <= 0) return cudaSuccess;
    // float images of the double range limits, rounded inwards (exact decisions for float depths)
    float rmin = (float)range_min, rmax = range_max > (double)FLT_MAX ? FLT_MAX : (float)range_max;
    if ((double)rmin < range_min) rmin = nextafterf(rmin, FLT_MAX);
    if ((double)rmax > range_max) rmax = nextafterf(rmax, -FLT_MAX);
    const int max_tiles = pack_tiles(max_px);
    for (int f0 = 0; f0 < n; f0 += 65535) {  // grid.y limit
        const int nf = n - f0 < 65535 ? n - f0 : 65535;
        const dim3 grid(max_tiles, nf);
        k_pack_valid<<<grid, kPackThreads, 0, s>>>(raw, frames, frame_ids + f0, valid_px, tile_counts, max_tiles,
                                                   rmin, rmax);
        if (texel_precision == 1)
            k_pack_points<1><<<grid, kPackThreads, 0, s>>>(raw, frames, sensors, frame_ids + f0, valid_px,
                                                           tile_counts, max_tiles, texels, pts_pg, pts_n, pts_pix,
                                                           n_points);
        else
            k_pack_points<0><<<grid, kPackThreads, 0, s>>>(raw, frames, sensors, frame_ids + f0, valid_px,
                                                           tile_counts, max_tiles, texels, pts_pg, pts_n, pts_pix,
                                                           n_points);
    }
    if (gtex && max_px > 0) {
        for (int f0 = 0; f0 < n; f0 += 65535) {
            const dim3 grid((max_px + 255) / 256, n - f0 < 65535 ? n - f0 : 65535);
            if (texel_precision == 1) k_grad<1><<<grid, 256, 0, s>>>(texels, frames, frame_ids + f0, gtex);
            else k_grad<0><<<grid, 256, 0, s>>>(texels, frames, frame_ids + f0, gtex);
        }
    }
    return cudaGetLastError();
}

}  // namespace pba
