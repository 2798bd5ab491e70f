// pba_linearize.cu -- the batched photometric linearisation (hot path).
//
// k_pair_pose     FP64 poses -> FP32 per-pair transform pbar = M p_u + a with
//                 M = R_o^T R_j^T R_i, a = R_o^T (R_j^T (t_i - t_j) - t_o)  (Supp., pbar_u; Eq. uprime)
// k_linearize     one persistent launch over a queue of chunks (pair, points);
//                 per pixel-point: transform, project (Eq. pinhole-projection / spherical-projection), sample the
//                 five target channels bilinearly at the 4 taps and their image
//                 gradients (Supp., image Jacobians: the central differences,
//                 precomputed per pixel at upload, interpolated at the same taps),
//                 residual e = zeta(pbar) - I_j(u') (Supp., Eq. error-jacobian),
//                 Huber weight, Jacobian J_i, and accumulation of the 6x6
//                 H6 = sum w J_i^T Omega J_i, b6 = sum w J_i^T Omega e, cost, count
//                 in FP32 registers; a transposed table in the warp's shared
//                 memory (and shuffles for cost and count) or a shuffle
//                 butterfly, whichever the autotuner keeps, gives one FP32
//                 partial per work item (no global atomics on residuals).
// k_pair_reduce   FP64 sum of a pair's chunk partials in a fixed order, then the
//                 pair's full 12x12 block from J_j = J_i T (see below).
//
// J_j from J_i.  With q = R_j^T (R_i p_u + t_i - t_j), R = R_j^T R_i and
// t = R_j^T (t_i - t_j), the Supp. derivatives are
//   d pbar / d dx_i = R_o^T R [I | -2 [p_u]x],   d pbar / d dx_j = R_o^T [-I | 2 [q]x],
//   d nbar / d dq_i = R_o^T R (-2 [n^o]x),       d nbar / d dq_j = R_o^T 2 [R n^o]x,
// and every one of them satisfies (d/d dx_j) = (d/d dx_i) T with the
// point-independent 6x6 map
//   T = [[-R^T, 2 R^T [t]x], [0, -R^T]]
// (use [R p]x = R [p]x R^T).  Hence J_j = J_i T for every row, H_ij = H6 T,
// H_jj = T^T H6 T and b_j = T^T b6: the kernel accumulates 21 + 6 sums instead
// of 78 + 12, and the parity tests compare against the oracle's independently
// computed J_j.
//
// In the i-frame form used below, J_c = [h_c, 2 p_u x h_c] with
// h_c = M^T (d zeta_c / d pbar - grad I_c d pi / d pbar), plus, for the normal
// rows c = 2 + k, 2 n^o x m_k in the rotation part (m_k = row k of M).
#include "pba_device.cuh"
#include "pba_internal.cuh"
#include "pba_tma.cuh"

namespace pba {

namespace {

constexpr int kLinWarps = kLinThreads / 32;

// ------------------------------------------------------------ pair poses

__global__ void k_pair_pose(const double* __restrict__ poses, const int2* __restrict__ pf,
                            const double* __restrict__ pair_Xo, int m, PairPose* __restrict__ out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m) return;
    const int2 ij = pf[p];
    const double* Xi = poses + 12 * ij.x;
    const double* Xj = poses + 12 * ij.y;
    const double* Xo = pair_Xo + 12 * p;
    double R[9], t[3];
    // R = R_j^T R_i ; t = R_j^T (t_i - t_j)
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            R[3 * r + c] = Xj[r] * Xi[c] + Xj[4 + r] * Xi[4 + c] + Xj[8 + r] * Xi[8 + c];
        t[r] = Xj[r] * (Xi[3] - Xj[3]) + Xj[4 + r] * (Xi[7] - Xj[7]) + Xj[8 + r] * (Xi[11] - Xj[11]);
    }
    PairPose o;
    // M = R_o^T R ; a = R_o^T (t - t_o)
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            o.M[3 * r + c] = (float)(Xo[r] * R[c] + Xo[4 + r] * R[3 + c] + Xo[8 + r] * R[6 + c]);
        o.a[r] = (float)(Xo[r] * (t[0] - Xo[3]) + Xo[4 + r] * (t[1] - Xo[7]) + Xo[8 + r] * (t[2] - Xo[11]));
    }
    out[p] = o;
}

// One lane's 21 + 6 sums of H6 = sum s J J^T (upper triangle) and b6 = sum s J e.
// Where both factors of two sums sit in the same register pairs, the pair is
// updated by one packed FP32 instruction of sm_100-class SMs (FFMA2 / FMUL2: two
// single-precision operations, each rounded as fmaf / a * b would be, so every
// sum gets exactly the operations of the scalar version):
//   d: (H00, H11), (H22, H33), (H44, H55)  = (t0, t1) * (J0, J1), ...
//   o: (H02, H13), (H04, H15), (H24, H35)  = (t0, t1) * (J2, J3), (t0, t1) * (J4, J5), (t2, t3) * (J4, J5)
//   b: (b0, b1), (b2, b3), (b4, b5)         = (t0, t1) * (e, e), ...
// with t = s J; the other nine sums are scalar FMAs (pairing them would need
// swapped copies of J, which cost as many moves as they save).
struct Acc6 {
    float2 d[3], o[3], b[3];
    float h01, h03, h05, h12, h14, h23, h25, h34, h45;
};

__device__ __forceinline__ void acc_zero(Acc6& A) {
#pragma unroll
    for (int i = 0; i < 3; ++i) A.d[i] = A.o[i] = A.b[i] = make_float2(0.f, 0.f);
    A.h01 = A.h03 = A.h05 = A.h12 = A.h14 = A.h23 = A.h25 = A.h34 = A.h45 = 0.f;
}

// Sum k of H6 in upper-triangle row-major order (the partials' layout), k < 21.
__device__ __forceinline__ float acc_h(const Acc6& A, int k) {
    switch (k) {
        case 0: return A.d[0].x;   // H00
        case 1: return A.h01;
        case 2: return A.o[0].x;   // H02
        case 3: return A.h03;
        case 4: return A.o[1].x;   // H04
        case 5: return A.h05;
        case 6: return A.d[0].y;   // H11
        case 7: return A.h12;
        case 8: return A.o[0].y;   // H13
        case 9: return A.h14;
        case 10: return A.o[1].y;  // H15
        case 11: return A.d[1].x;  // H22
        case 12: return A.h23;
        case 13: return A.o[2].x;  // H24
        case 14: return A.h25;
        case 15: return A.d[1].y;  // H33
        case 16: return A.h34;
        case 17: return A.o[2].y;  // H35
        case 18: return A.d[2].x;  // H44
        case 19: return A.h45;
        default: return A.d[2].y;  // H55
    }
}

// H6 += s J J^T ; b6 += s J e for one residual row.
__device__ __forceinline__ void accum_row(Acc6& A, const float (&J)[6], float sw, float e) {
    const float2 j01 = make_float2(J[0], J[1]), j23 = make_float2(J[2], J[3]), j45 = make_float2(J[4], J[5]);
    const float2 s2 = make_float2(sw, sw), e2 = make_float2(e, e);
    const float2 t01 = __fmul2_rn(s2, j01), t23 = __fmul2_rn(s2, j23), t45 = __fmul2_rn(s2, j45);
    A.d[0] = __ffma2_rn(t01, j01, A.d[0]);
    A.d[1] = __ffma2_rn(t23, j23, A.d[1]);
    A.d[2] = __ffma2_rn(t45, j45, A.d[2]);
    A.o[0] = __ffma2_rn(t01, j23, A.o[0]);
    A.o[1] = __ffma2_rn(t01, j45, A.o[1]);
    A.o[2] = __ffma2_rn(t23, j45, A.o[2]);
    A.h01 = fmaf(t01.x, J[1], A.h01);
    A.h03 = fmaf(t01.x, J[3], A.h03);
    A.h05 = fmaf(t01.x, J[5], A.h05);
    A.h12 = fmaf(t01.y, J[2], A.h12);
    A.h14 = fmaf(t01.y, J[4], A.h14);
    A.h23 = fmaf(t23.x, J[3], A.h23);
    A.h25 = fmaf(t23.x, J[5], A.h25);
    A.h34 = fmaf(t23.y, J[4], A.h34);
    A.h45 = fmaf(t45.x, J[5], A.h45);
    A.b[0] = __ffma2_rn(t01, e2, A.b[0]);
    A.b[1] = __ffma2_rn(t23, e2, A.b[1]);
    A.b[2] = __ffma2_rn(t45, e2, A.b[2]);
}

// Sum of value l over the warp's 32 lanes, returned in lane l (a reduce-scatter:
// at the level of offset o each lane keeps the half of its o-value window that
// its bit o selects and adds the partner's copy of that half, so after the
// levels 16, 8, 4, 2, 1 value 0 of lane l holds the full sum of value l).
__device__ __forceinline__ float butterfly_sum(float (&v)[32], int lane) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = up ? v[i] : v[i + o];
            const float keep = up ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

constexpr int kQueue = 64;   // slots of a warp's residual queue (a power of two >= 63)
constexpr int kQItems = 14;  // floats per queued residual: e[5], w, pbar[3], point, r0, c0, a, b

// Stage 2 (a4 gradients + a6 + a7) for one queued residual: the image
// gradients of the five channels at u' (grad_mode 0: the central differences
// of the Supp., precomputed per pixel, interpolated bilinearly at the 4 taps,
// which equals the 12-texel stencil term by term; grad_mode 1: the exact
// bilinear derivative from the 4 texels), d pi / d pbar, the 5 x 6 Jacobian
// J_i and its Huber-weighted accumulation into H6 (upper triangle) and b6.
template <int TEXEL>
__device__ __forceinline__ void jacobian_stage(float (*Q)[kQueue], int slot, int model, float fx, float fy, int W,
                                               bool wrap, const float (&M)[9], const float (&om)[5],
                                               const float4* __restrict__ pg, const float4* __restrict__ pn,
                                               const void* __restrict__ tex, const float4* __restrict__ gtex,
                                               long long tex_off, int grad_mode, Acc6& acc) {
    float e[5];
#pragma unroll
    for (int c = 0; c < 5; ++c) e[c] = Q[c][slot];
    const float w = Q[5][slot];
    const float qx = Q[6][slot], qy = Q[7][slot], qz = Q[8][slot];
    const int k = __float_as_int(Q[9][slot]);
    const int r0 = __float_as_int(Q[10][slot]);
    const int c0 = __float_as_int(Q[11][slot]);
    const float a = Q[12][slot], b = Q[13][slot];

    // c0 was wrapped into [0, W) by stage 1
    const int cc = c0, cp1 = wrap && c0 == W - 1 ? 0 : c0 + 1;
    const int rr0 = r0 * W, rp1 = rr0 + W;
    float gu[5], gv[5];
    if (grad_mode == 0) {
        // central differences at the taps A, B, C, D (precomputed per pixel), interpolated
        const float4* G = gtex + 3 * tex_off;
        const int tap[4] = {rr0 + cc, rr0 + cp1, rp1 + cc, rp1 + cp1};
        const float wt[4] = {(1.f - a) * (1.f - b), a * (1.f - b), (1.f - a) * b, a * b};
#pragma unroll
        for (int c = 0; c < 5; ++c) gu[c] = gv[c] = 0.f;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const float4 g0 = __ldg(G + 3 * tap[t]), g1 = __ldg(G + 3 * tap[t] + 1), g2 = __ldg(G + 3 * tap[t] + 2);
            const float u[5] = {g0.x, g0.y, g0.z, g0.w, g1.x}, vv[5] = {g1.y, g1.z, g1.w, g2.x, g2.y};
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                gu[c] = fmaf(wt[t], u[c], gu[c]);
                gv[c] = fmaf(wt[t], vv[c], gv[c]);
            }
        }
    } else {
        tex = TEXEL == 1 ? (const void*)(reinterpret_cast<const Tex16*>(tex) + tex_off)
                         : (const void*)(reinterpret_cast<const Tex32*>(tex) + tex_off);
        float A[5], B[5], C[5], D[5];
        channels(load_texel<TEXEL>(tex, rr0 + cc), A);
        channels(load_texel<TEXEL>(tex, rr0 + cp1), B);
        channels(load_texel<TEXEL>(tex, rp1 + cc), C);
        channels(load_texel<TEXEL>(tex, rp1 + cp1), D);
#pragma unroll
        for (int c = 0; c < 5; ++c) {
            gu[c] = fmaf(1.f - b, B[c] - A[c], b * (D[c] - C[c]));
            gv[c] = fmaf(1.f - a, C[c] - A[c], a * (D[c] - B[c]));
        }
    }
    const float4 p = __ldg(pg + k);
    const float4 n = __ldg(pn + k);
    // d pi / d pbar (2 x 3) and d zeta^d / d pbar (hardware reciprocal and
    // reciprocal square root: ~1e-7 relative, far below the FP32 Jacobian's use),
    // taken to the i-frame at once: h_c = M^T g_c with g_c = d zeta_c / d pbar -
    // grad I_c d pi / d pbar is linear in those rows, A0 = M^T (d pi / d pbar)_0,
    // A1 = M^T (d pi / d pbar)_1, Az = M^T d zeta^d / d pbar.  The model is the same
    // for the whole warp (one pair per work item), and each branch keeps only the
    // nonzero terms of its model's derivatives.
    float A0[3], A1[3], Az[3];
    if (model == 0) {
        // pinhole: (d pi / d pbar)_0 = (fx / z, 0, -fx x / z^2), _1 = (0, fy / z, -fy y / z^2), d zeta^d = e_z
        const float iz = __fdividef(1.f, qz);
        const float p00 = fx * iz, p02 = -fx * qx * iz * iz;
        const float p11 = fy * iz, p12 = -fy * qy * iz * iz;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A0[j] = fmaf(M[j], p00, M[6 + j] * p02);
            A1[j] = fmaf(M[3 + j], p11, M[6 + j] * p12);
            Az[j] = M[6 + j];
        }
    } else {
        const float rxy2 = fmaf(qx, qx, qy * qy);
        const float irxy = rsqrtf(rxy2);
        const float irxy2 = irxy * irxy;
        const float rxy = rxy2 * irxy;
        const float inv_r = rsqrtf(fmaf(qz, qz, rxy2));
        const float ir2 = inv_r * inv_r;
        // spherical: (d pi / d pbar)_0 = fx (-y, x, 0) / rxy^2, _1 = fy (-z x / (r^2 rxy), -z y / (r^2 rxy), rxy / r^2),
        // d zeta^d = pbar / r
        const float p00 = -fx * qy * irxy2, p01 = fx * qx * irxy2;
        const float k1 = -fy * qz * ir2 * irxy;
        const float p10 = k1 * qx, p11 = k1 * qy, p12 = fy * rxy * ir2;
        const float d0 = qx * inv_r, d1 = qy * inv_r, d2 = qz * inv_r;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            A0[j] = fmaf(M[j], p00, M[3 + j] * p01);
            A1[j] = fmaf(M[j], p10, fmaf(M[3 + j], p11, M[6 + j] * p12));
            Az[j] = fmaf(M[j], d0, fmaf(M[3 + j], d1, M[6 + j] * d2));
        }
    }
    const float4 p2 = make_float4(2.f * p.x, 2.f * p.y, 2.f * p.z, 0.f);
    const float n2x = 2.f * n.x, n2y = 2.f * n.y, n2z = 2.f * n.z;
#pragma unroll
    for (int c = 0; c < 5; ++c) {
        float h[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            h[j] = -fmaf(gu[c], A0[j], gv[c] * A1[j]);
            if (c == 1) h[j] += Az[j];
        }
        // J = [h, 2 p x h] (+ 2 n^o x m_k for the normal rows, m_k = row k of M)
        float J[6];
        J[0] = h[0];
        J[1] = h[1];
        J[2] = h[2];
        J[3] = fmaf(p2.y, h[2], -p2.z * h[1]);
        J[4] = fmaf(p2.z, h[0], -p2.x * h[2]);
        J[5] = fmaf(p2.x, h[1], -p2.y * h[0]);
        if (c >= 2) {
            const int r = c - 2;
            const float mx = M[3 * r], my = M[3 * r + 1], mz = M[3 * r + 2];
            J[3] += fmaf(n2y, mz, -n2z * my);
            J[4] += fmaf(n2z, mx, -n2x * mz);
            J[5] += fmaf(n2x, my, -n2y * mx);
        }
        accum_row(acc, J, w * om[c], e[c]);
    }
}

// One warp per work item (a chunk of up to kWarpChunk points of one pair); no
// block-wide synchronisation.  Stage 1 runs on every point: transform,
// projection, bounds, the 4 bilinear taps (whose usable flags decide the
// 12-texel stencil), sampled values, residual, occlusion test, Huber weight and
// cost.  Valid residuals are compacted into the warp's queue; stage 2 runs on
// full warps of them.
//
// STAGE (FP16 texels): the four taps of each 32-point step are read from a
// kTileRows x kTileCols tile of the target's texels in shared memory, fetched
// by one lane with one TMA tensor copy (the step's taps span a few rows and
// columns: consecutive points of a source row land on neighbouring target
// pixels); a step whose taps do not fit the tile, or straddle the wrap seam of
// a spherical image, reads them from global memory as the unstaged kernel does.
template <int TEXEL, bool FULL, bool MASK, int MINB, bool STAGE>
__global__ void __launch_bounds__(kLinThreads, MINB)
    k_linearize(const int4* __restrict__ chunks, int n_chunks, int* __restrict__ queue,
                const PairStatic* __restrict__ ps, const PairPose* __restrict__ pp,
                const float4* __restrict__ pts_pg, const float4* __restrict__ pts_n,
                const void* __restrict__ tex, const LinParams prm, float* __restrict__ partials,
                uint32_t* __restrict__ mask_bits) {
    static_assert(!STAGE || TEXEL == 1, "tiles are staged for FP16 texels only");
    __shared__ __align__(16) float s_q[FULL ? kLinWarps : 1][kQItems][kQueue];
    __shared__ __align__(128) uint4 s_tile[STAGE ? kLinWarps : 1][STAGE ? kTileRows * kTileCols : 1];
    __shared__ __align__(8) uint64_t s_bar[kLinWarps];
    static_assert(27 * 32 <= kQItems * kQueue, "the reduction table must fit the queue region");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float om[5] = {prm.w_int, prm.w_depth, prm.w_normal, prm.w_normal, prm.w_normal};
    float(*Q)[kQueue] = s_q[FULL ? warp : 0];
    unsigned tile_phase = 0;      // parity of the warp's mbarrier for the next tile
    bool tile_ok = STAGE;         // false once a tile wait ran out (taps read directly)
    if (STAGE) {
        if (lane == 0) tma_mbar_init(&s_bar[warp], 1);
        __syncwarp();
    }

    for (;;) {
        int ci = 0;
        if (lane == 0) ci = atomicAdd(queue, 1);
        ci = __shfl_sync(0xffffffffu, ci, 0);
        if (ci >= n_chunks) break;
        const int4 ch = __ldg(chunks + ci);
        const int pair = ch.x, first = ch.y, count = ch.z;
        const PairStatic& P = ps[pair];
        const int W = P.width, Hh = P.height, model = P.model;
        const float fx = P.fx, fy = P.fy, cx = P.cx, cy = P.cy;
        const long long pt_off = P.src_pt_offset, tex_off = P.tgt_px_offset;
        float M[9], av[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) M[k] = pp[pair].M[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) av[k] = pp[pair].a[k];
        const bool wrap = model == 1;
        const void* tex_j = TEXEL == 1 ? (const void*)(reinterpret_cast<const Tex16*>(tex) + tex_off)
                                       : (const void*)(reinterpret_cast<const Tex32*>(tex) + tex_off);
        const float umax = wrap ? 3.4e38f : (float)(W - 2);
        const float umin = wrap ? -3.4e38f : 1.f;
        const float vmax = (float)(Hh - 2);

        Acc6 acc;
        float cost = 0.f, cnt = 0.f, nonfin = 0.f;
        if (FULL) acc_zero(acc);
        int head = 0, tail = 0;  // warp-uniform queue counters
        const int end = first + count;
        // the point of the next iteration is loaded one iteration ahead (its
        // latency, often a DRAM miss, overlaps this iteration's work)
        float4 p_next = first + lane < end ? __ldg(pts_pg + pt_off + first + lane) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int base = first; base < end; base += 32) {
            const int k = base + lane;
            bool valid = false;
            float e[5], w = 0.f, qx = 0.f, qy = 0.f, qz = 0.f, fa = 0.f, fb = 0.f;
            int r0 = 0, c0 = 0;
            const float4 p = p_next;
            if (k + 32 < end) p_next = __ldg(pts_pg + pt_off + k + 32);
            float zeta_d = 0.f;
            bool ok = false;
            int cp1 = 0;
            if (k < end) {
                // a2: pbar = M p_u + a
                qx = fmaf(M[0], p.x, fmaf(M[1], p.y, fmaf(M[2], p.z, av[0])));
                qy = fmaf(M[3], p.x, fmaf(M[4], p.y, fmaf(M[5], p.z, av[1])));
                qz = fmaf(M[6], p.x, fmaf(M[7], p.y, fmaf(M[8], p.z, av[2])));
                // a3: projection (the column as floor and fraction) and bounds
                float v;
                if (model == 0) {
                    ok = qz > prm.z_min;
                    const float iz = __fdividef(1.f, qz);
                    const float u = fmaf(fx * qx, iz, cx);
                    v = fmaf(fy * qy, iz, cy);
                    zeta_d = qz;
                    ok = ok && u >= umin && u < umax;
                    const float fu = floorf(u);
                    c0 = (int)fu;
                    fa = u - fu;
                } else {
                    // square roots through the hardware reciprocal square root
                    // (~1e-7 relative); a zero radius gives NaN and fails the tests
                    const float rxy2 = fmaf(qx, qx, qy * qy);
                    const float r2 = fmaf(qz, qz, rxy2);
                    zeta_d = r2 * rsqrtf(r2);
                    ok = zeta_d > prm.z_min;
                    spherical_project(qx, qy, qz, rsqrtf(rxy2), fx, fy, cx, cy, P.fxh, P.fxp, c0, fa, v);
                }
                ok = ok && v >= 1.f && v < vmax;
                if (ok) {
                    const float fv = floorf(v);
                    r0 = (int)fv;
                    fb = v - fv;
                    int cm1, cc, cp2;
                    stencil_cols(c0, W, wrap, cm1, cc, cp1, cp2);
                    c0 = cc;
                }
            }
            // staged taps: the warp's tile around this step's taps, one TMA copy
            bool staged = false;
            int t_r = 0, t_c = 0;
            if (STAGE && tile_ok) {
                const int rl = __reduce_min_sync(0xffffffffu, ok ? r0 : 0x7fffffff);
                const int rh = __reduce_max_sync(0xffffffffu, ok ? r0 + 1 : -1);
                const int cl = __reduce_min_sync(0xffffffffu, ok ? c0 : 0x7fffffff);
                const int chh = __reduce_max_sync(0xffffffffu, ok ? c0 + 1 : -1);
                const bool seam = __any_sync(0xffffffffu, ok && cp1 != c0 + 1);
                staged = rh >= 0 && !seam && rh - rl < kTileRows && chh - cl < kTileCols;
                if (staged) {
                    t_r = rl;
                    t_c = cl;
                    __syncwarp();  // every lane's reads of the previous tile are done
                    if (lane == 0)
                        tma_load_tile(s_tile[warp], &s_bar[warp], prm.tmaps + P.tgt, t_c, t_r);
                    if (!tma_wait(&s_bar[warp], tile_phase)) {
                        // the copy did not complete within the limit: raise the flag and read
                        // the taps directly from now on (the tile is not read again)
                        if (lane == 0) atomicExch(prm.tile_err, 1);
                        tile_ok = false;
                        staged = false;
                    }
                    tile_phase ^= 1u;
                }
            }
            if (ok) {
                // a4: the four bilinear taps; their usable flags decide the 12-texel stencil
                Tap<TEXEL> A, B, C, D;
                if constexpr (STAGE) {
                    if (staged) {
                        const uint4* T = s_tile[warp];
                        const int i0 = (r0 - t_r) * kTileCols + (c0 - t_c);
                        A.v = T[i0];
                        B.v = T[i0 + 1];
                        C.v = T[i0 + kTileCols];
                        D.v = T[i0 + kTileCols + 1];
                    }
                }
                if (!(STAGE && staged)) {
                    const int rr0 = r0 * W, rp1 = rr0 + W;
                    A = load_tap<TEXEL>(tex_j, rr0 + c0);
                    B = load_tap<TEXEL>(tex_j, rr0 + cp1);
                    C = load_tap<TEXEL>(tex_j, rp1 + c0);
                    D = load_tap<TEXEL>(tex_j, rp1 + cp1);
                }
                // a5: the depth channel first (FP32 in every texel) and the occlusion
                // test; the other channels are only converted and interpolated for the
                // points that pass
                const float wA = (1.f - fa) * (1.f - fb), wB = fa * (1.f - fb), wC = (1.f - fa) * fb, wD = fa * fb;
                float s[5];
                s[1] = fmaf(wA, A.depth(), fmaf(wB, B.depth(), fmaf(wC, C.depth(), wD * D.depth())));
                const float e_d = zeta_d - s[1];
                ok = all_usable(A, B, C, D) && fabsf(e_d) <= fmaf(prm.occ_rel, zeta_d, prm.occ_abs);
                if (ok) {
                    // (g, n_x) and (n_y, n_z) of the four taps as register pairs, interpolated
                    // with packed FMAs (each rounded as fmaf, in the same order)
                    float2 a0, a1, b0, b1, c0p, c1p, d0, d1;
                    A.rest2(a0, a1);
                    B.rest2(b0, b1);
                    C.rest2(c0p, c1p);
                    D.rest2(d0, d1);
                    const float2 wA2 = make_float2(wA, wA), wB2 = make_float2(wB, wB);
                    const float2 wC2 = make_float2(wC, wC), wD2 = make_float2(wD, wD);
                    const float2 i0 = __ffma2_rn(wA2, a0, __ffma2_rn(wB2, b0, __ffma2_rn(wC2, c0p, __fmul2_rn(wD2, d0))));
                    const float2 i1 = __ffma2_rn(wA2, a1, __ffma2_rn(wB2, b1, __ffma2_rn(wC2, c1p, __fmul2_rn(wD2, d1))));
                    s[0] = i0.x;
                    s[2] = i0.y;
                    s[3] = i1.x;
                    s[4] = i1.y;
                    const float nt2 = fmaf(s[2], s[2], fmaf(s[3], s[3], s[4] * s[4]));
                    ok = nt2 >= 0.25f;
                }
                if (ok) {
                    valid = true;
                    const float4 n = __ldg(pts_n + pt_off + k);
                    const float nbx = fmaf(M[0], n.x, fmaf(M[1], n.y, M[2] * n.z));
                    const float nby = fmaf(M[3], n.x, fmaf(M[4], n.y, M[5] * n.z));
                    const float nbz = fmaf(M[6], n.x, fmaf(M[7], n.y, M[8] * n.z));
                    e[0] = p.w - s[0];
                    e[1] = e_d;
                    e[2] = nbx - s[2];
                    e[3] = nby - s[3];
                    e[4] = nbz - s[4];
                    // chi^2 = e^T Omega e with the three normal rows sharing their weight
                    const float en = fmaf(e[2], e[2], fmaf(e[3], e[3], e[4] * e[4]));
                    const float chi2 = fmaf(om[0] * e[0], e[0], fmaf(om[1] * e[1], e[1], om[2] * en));
                    if (!(chi2 < INFINITY)) {
                        // a NaN or infinite input value (intensity, normal): the residual is
                        // left out of H, b and F and counted in the status word
                        valid = false;
                        nonfin += 1.f;
                    } else {
                        float rho;
                        if (chi2 <= prm.huber_delta2) {
                            w = 1.f;
                            rho = chi2;
                        } else {
                            const float chi = sqrtf(chi2);
                            w = prm.huber_delta / chi;
                            rho = fmaf(2.f * prm.huber_delta, chi, -prm.huber_delta2);
                        }
                        cost += rho;
                        cnt += 1.f;
                    }
                }
            }
            if (MASK) {
                const unsigned bits = __ballot_sync(0xffffffffu, valid);
                if (lane == 0) mask_bits[P.mask_offset + (base >> 5)] = bits;
            }
            if (FULL) {
                const unsigned bal = __ballot_sync(0xffffffffu, valid);
                if (valid) {
                    const int slot = (tail + __popc(bal & ((1u << lane) - 1u))) & (kQueue - 1);
#pragma unroll
                    for (int c = 0; c < 5; ++c) Q[c][slot] = e[c];
                    Q[5][slot] = w;
                    Q[6][slot] = qx;
                    Q[7][slot] = qy;
                    Q[8][slot] = qz;
                    Q[9][slot] = __int_as_float(k);
                    Q[10][slot] = __int_as_float(r0);
                    Q[11][slot] = __int_as_float(c0);
                    Q[12][slot] = fa;
                    Q[13][slot] = fb;
                }
                tail += __popc(bal);
                __syncwarp();
                if (tail - head >= 32) {
                    jacobian_stage<TEXEL>(Q, (head + lane) & (kQueue - 1), model, fx, fy, W, wrap, M, om,
                                          pts_pg + pt_off, pts_n + pt_off, tex, prm.gtex, tex_off, prm.grad_mode, acc);
                    head += 32;
                    __syncwarp();
                }
            }
        }
        if (FULL && tail > head) {
            if (lane < tail - head)
                jacobian_stage<TEXEL>(Q, (head + lane) & (kQueue - 1), model, fx, fy, W, wrap, M, om,
                                      pts_pg + pt_off, pts_n + pt_off, tex, prm.gtex, tex_off, prm.grad_mode, acc);
            __syncwarp();
        }

        // a7: warp reduction, one FP32 partial per work item (lane t writes sum t),
        // by one of two schemes (LinParams::reduction, chosen by the autotuner):
        // 0: H6 and b6 go through the warp's queue region, empty at this point:
        //    lane l writes its 27 sums as column l of a 27 x 32 table, lane j < 27
        //    adds row j; cost, count and the status count by shuffles;
        // 1: all 30 sums by a butterfly of shuffles that halves the values each
        //    lane holds at every level (lane l ends with the warp's sum l).
        float mine = 0.f;
        if (FULL && prm.reduction == 1) {
            float v[32];
#pragma unroll
            for (int j = 0; j < 21; ++j) v[j] = acc_h(acc, j);
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                v[21 + 2 * j] = acc.b[j].x;
                v[22 + 2 * j] = acc.b[j].y;
            }
            v[27] = cost;
            v[28] = cnt;
            v[29] = nonfin;
            v[30] = v[31] = 0.f;
            mine = butterfly_sum(v, lane);
        } else {
            if (FULL) {
                float* tab = &Q[0][0];  // 27 x 32 floats <= kQItems x kQueue
#pragma unroll
                for (int j = 0; j < 21; ++j) tab[j * 32 + lane] = acc_h(acc, j);
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    tab[(21 + 2 * j) * 32 + lane] = acc.b[j].x;
                    tab[(22 + 2 * j) * 32 + lane] = acc.b[j].y;
                }
                __syncwarp();
                if (lane < 27) {
                    // rows start on bank 0: lane j reads its row from float4 (q + j) mod 8 on,
                    // so that the 8 lanes of a quarter-warp hit 8 different bank quads
                    const float4* row = reinterpret_cast<const float4*>(tab + lane * 32);
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 v = row[(q + lane) & 7];
                        s0 += v.x;
                        s1 += v.y;
                        s2 += v.z;
                        s3 += v.w;
                    }
                    mine = (s0 + s1) + (s2 + s3);
                }
                __syncwarp();  // the next work item's queue writes come after these reads
            }
#pragma unroll
            for (int j = 27; j < kNumAcc; ++j) {
                float x = j == 27 ? cost : (j == 28 ? cnt : nonfin);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                if (lane == j) mine = x;
            }
        }
        // the item's partial-sum slot (its index in the plan's own order, whatever
        // order this launch takes the items in)
        const int slot = __ldg(reinterpret_cast<const int*>(chunks + ci) + 3);
        if (lane < kNumAcc && (FULL || lane >= 27)) partials[(long long)slot * kPartialStride + lane] = mine;
    }
}

// ------------------------------------------------------------ pair reduction

constexpr int kPairSlices = 8;  // threads summing one accumulator of a pair (one warp per slice)

__global__ void __launch_bounds__(32 * kPairSlices) k_pair_reduce(const float* __restrict__ partials, const PairStatic* __restrict__ ps,
                              const int2* __restrict__ pf, const double* __restrict__ poses, bool full,
                              double* __restrict__ blocks) {
    const int p = blockIdx.x;
    const int t = threadIdx.x;
    __shared__ double acc[kNumAcc + 3];
    __shared__ double part[kPairSlices][kNumAcc];
    __shared__ double H6[36], T[36], HT[36], R[9], tv[3];
    const PairStatic P = ps[p];
    const int k0 = full ? 0 : 27;
    double* out = blocks + (long long)p * kBlockStride;
    if (t == 64) {
        // status word: 1 when the pair's relative pose is not finite (a NaN or infinite pose)
        const int2 ij = pf[p];
        bool bad = false;
        for (int e = 0; e < 12; ++e) bad = bad || !isfinite(poses[12 * ij.x + e]) || !isfinite(poses[12 * ij.y + e]);
        out[159] = bad ? 1.0 : 0.0;
    }
    // thread (slice, j) sums accumulator j over its contiguous slice of the pair's
    // chunks in chunk order (4 loads in flight), then the slices are added in order
    {
        const int j = t % 32, slice = t / 32;
        const int n = P.chunk_end - P.chunk_begin;
        const int c_lo = P.chunk_begin + (int)((long long)n * slice / kPairSlices);
        const int c_hi = P.chunk_begin + (int)((long long)n * (slice + 1) / kPairSlices);
        if (j >= k0 && j < kNumAcc) {
            double s = 0.0;
            for (int c0 = c_lo; c0 < c_hi; c0 += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = c0 + u < c_hi ? partials[(long long)(c0 + u) * kPartialStride + j] : 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c0 + u < c_hi) s += (double)v[u];
            }
            part[slice][j] = s;
        }
    }
    __syncthreads();
    if (t >= k0 && t < kNumAcc) {
        double s = 0.0;
        for (int slice = 0; slice < kPairSlices; ++slice) s += part[slice][t];
        acc[t] = s;
    }
    __syncthreads();
    if (!full) {
        if (t == 0) {
            out[156] = acc[27];
            out[157] = acc[28];
            out[158] = acc[29];
        }
        return;
    }
    // T = [[-R^T, 2 R^T [t]x], [0, -R^T]],  R = R_j^T R_i, t = R_j^T (t_i - t_j): once per pair
    if (t >= 36 && t < 48) {
        const int2 ij = pf[p];
        const double* Xi = poses + 12 * ij.x;
        const double* Xj = poses + 12 * ij.y;
        const int e = t - 36;
        if (e < 9) {
            const int rr = e / 3, cc = e % 3;
            R[e] = Xj[rr] * Xi[cc] + Xj[4 + rr] * Xi[4 + cc] + Xj[8 + rr] * Xi[8 + cc];
        } else {
            const int rr = e - 9;
            tv[rr] = Xj[rr] * (Xi[3] - Xj[3]) + Xj[4 + rr] * (Xi[7] - Xj[7]) + Xj[8 + rr] * (Xi[11] - Xj[11]);
        }
    }
    __syncthreads();
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        const int a = r < c ? r : c, bb = r < c ? c : r;
        // index of (a, bb) in the row-major upper triangle
        const int idx = a * 6 - a * (a - 1) / 2 + (bb - a);
        H6[t] = acc[idx];
        double val = 0.0;
        if (r < 3 && c < 3) {
            val = -R[3 * c + r];
        } else if (r < 3 && c >= 3) {
            // (2 R^T [t]x)[r][c-3] = 2 sum_k R[k][r] [t]x[k][c-3]
            const double S[9] = {0.0, -tv[2], tv[1], tv[2], 0.0, -tv[0], -tv[1], tv[0], 0.0};
            for (int k = 0; k < 3; ++k) val += 2.0 * R[3 * k + r] * S[3 * k + (c - 3)];
        } else if (r >= 3 && c >= 3) {
            val = -R[3 * (c - 3) + (r - 3)];
        }
        // a pair whose relative pose is not finite has no residual (H6 = 0, b6 = 0):
        // its blocks stay 0 instead of 0 x NaN
        T[t] = isfinite(val) ? val : 0.0;
    }
    __syncthreads();
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += H6[6 * r + k] * T[6 * k + c];
        HT[t] = s;  // H_ij = H6 T
    }
    __syncthreads();
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        out[12 * r + c] = H6[t];                 // H_ii
        out[12 * r + 6 + c] = HT[t];             // H_ij
        out[12 * (6 + c) + r] = HT[t];           // H_ji = H_ij^T
        if (r <= c) {
            // H_jj = T^T H6 T, computed once per unordered entry so it is exactly symmetric
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += T[6 * k + r] * HT[6 * k + c];
            out[12 * (6 + r) + 6 + c] = s;
            out[12 * (6 + c) + 6 + r] = s;
        }
    }
    if (t < 6) {
        out[144 + t] = acc[21 + t];              // b_i = b6
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += T[6 * k + t] * acc[21 + k];
        out[150 + t] = s;                        // b_j = T^T b6
    }
    if (t == 0) {
        out[156] = acc[27];
        out[157] = acc[28];
        out[158] = acc[29];
    }
}

}  // namespace

cudaError_t launch_pair_pose(const double* poses, const int2* pair_frames, const double* pair_Xo, int m,
                             PairPose* out, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_pair_pose<<<(m + 127) / 128, 128, 0, s>>>(poses, pair_frames, pair_Xo, m, out);
    return cudaGetLastError();
}

template <int TEXEL, bool FULL, bool MASK, int MINB, bool STAGE>
static void* lin_kernel() {
    return reinterpret_cast<void*>(&k_linearize<TEXEL, FULL, MASK, MINB, STAGE>);
}

// Occupancy variants (blocks of 128 threads per SM the register budget aims
// at): full pass 4, 6, 7 or 5 (128, 80, 72 or 96 registers: 16 to 28 warps per
// SM), cost-only pass 6, 7, 9 or 10 (72 to 48 registers: 28 to 40 warps) for
// variants 0 .. 3; variants 4 .. 7 are the same budgets with the taps read from
// TMA-staged tiles (FP16 texels without mask export; otherwise they run as
// variants 0 .. 3).  Fewer registers per thread trade spills for warps to hide
// gather latency; the block size only sets the occupancy steps (the warps of a
// block share nothing but their queue and tile regions).
template <int TEXEL, bool FULL, bool MASK, bool STAGE>
static void* pick_minb(int variant) {
    if constexpr (FULL) {
        if (variant == 3) return lin_kernel<TEXEL, FULL, MASK, 5, STAGE>();
        if (variant == 2) return lin_kernel<TEXEL, FULL, MASK, 7, STAGE>();
        return variant ? lin_kernel<TEXEL, FULL, MASK, 6, STAGE>() : lin_kernel<TEXEL, FULL, MASK, 4, STAGE>();
    } else {
        if (variant == 3) return lin_kernel<TEXEL, FULL, MASK, 10, STAGE>();
        if (variant == 2) return lin_kernel<TEXEL, FULL, MASK, 9, STAGE>();
        return variant ? lin_kernel<TEXEL, FULL, MASK, 7, STAGE>() : lin_kernel<TEXEL, FULL, MASK, 6, STAGE>();
    }
}

static void* pick(int texel_precision, bool full, bool mask, int variant) {
    const bool stage = variant >= 4;
    variant &= 3;
    if (texel_precision == 1) {
        if (stage && !mask)
            return full ? pick_minb<1, true, false, true>(variant) : pick_minb<1, false, false, true>(variant);
        if (full) return mask ? pick_minb<1, true, true, false>(variant) : pick_minb<1, true, false, false>(variant);
        return mask ? pick_minb<1, false, true, false>(variant) : pick_minb<1, false, false, false>(variant);
    }
    if (full) return mask ? pick_minb<0, true, true, false>(variant) : pick_minb<0, true, false, false>(variant);
    return mask ? pick_minb<0, false, true, false>(variant) : pick_minb<0, false, false, false>(variant);
}

int linearize_grid(int texel_precision, bool full, int variant) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)pick(texel_precision, full, false, variant),
                                                  kLinThreads, 0);
    if (per_sm < 1) per_sm = 1;
    return sms * per_sm;
}

cudaError_t launch_linearize(bool full, bool mask, int texel_precision, const int4* chunks, int n_chunks, int* queue,
                             const PairStatic* ps, const PairPose* pp, const float4* pts_pg, const float4* pts_n,
                             const void* texels, const LinParams& prm, float* partials, uint32_t* mask_bits,
                             int grid, int variant, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    const int warps = n_chunks;  // one work item per warp at a time
    if (grid * (kLinThreads / 32) > warps) grid = (warps + kLinThreads / 32 - 1) / (kLinThreads / 32);
    // staged variants need the frames' tensor maps
    if (!prm.tmaps) variant &= 3;
    void* fn = pick(texel_precision, full, mask, variant);
    LinParams prm_copy = prm;
    void* args[] = {(void*)&chunks, (void*)&n_chunks, (void*)&queue, (void*)&ps, (void*)&pp, (void*)&pts_pg,
                    (void*)&pts_n, (void*)&texels, (void*)&prm_copy, (void*)&partials, (void*)&mask_bits};
    return cudaLaunchKernel(fn, dim3(grid), dim3(kLinThreads), args, 0, s);
}

cudaError_t launch_pair_reduce(const float* partials, const PairStatic* ps, const int2* pair_frames,
                               const double* poses, const double* pair_Xo, int m, bool full, double* blocks,
                               cudaStream_t s) {
    (void)pair_Xo;
    if (m <= 0) return cudaSuccess;
    k_pair_reduce<<<m, 32 * kPairSlices, 0, s>>>(partials, ps, pair_frames, poses, full, blocks);
    return cudaGetLastError();
}

}  // namespace pba
