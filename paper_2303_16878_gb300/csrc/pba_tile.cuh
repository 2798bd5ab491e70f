// pba_tile.cuh -- 32 x 32 FP32 tile helpers of the Cholesky solves
// (pba_solve_cluster.cu, pba_solve_sparse.cu): the tile geometry, a 16-byte
// load through L2, row-by-row tile products and the factorisation and
// inversion of one diagonal tile by a CTA of 256 threads.
#pragma once

#include "pba_internal.cuh"

namespace pba {
namespace tile {

constexpr int kT = kTile;             // tile edge (32)
constexpr int kLd = kT + 4;           // padded row stride: rows stay 16-byte aligned for float4 loads
constexpr int kTF = kT * kLd;         // floats per stored tile
constexpr int kCsThreads = 256;       // 8 warps; one 16-byte piece of a 32 x 32 tile per thread
constexpr int kCsWarps = kCsThreads / 32;
constexpr int kRpt = kT / kCsWarps;   // tile rows per warp (thread (warp, lane) owns rows warp + 8 h of column lane)

// 16-byte load that bypasses L1 (data written by another CTA of the cluster
// before a cluster barrier)
__device__ __forceinline__ float4 ld_cg4(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }

__device__ __forceinline__ float dot4(const float4 a, const float4 b, float s) {
    s = fmaf(a.x, b.x, s);
    s = fmaf(a.y, b.y, s);
    s = fmaf(a.z, b.z, s);
    return fmaf(a.w, b.w, s);
}

// s[h] = sum_m X[r][m] Y[c][m] for the rows r = warp + 8 h and the column
// c = lane of the calling thread (X rows broadcast, Y rows 16-byte vectors;
// with the 36-float stride 8 lanes read 8 distinct bank quads).
__device__ __forceinline__ void tile_rows_dot(const float* X, const float* Y, float (&s)[kRpt]) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int h = 0; h < kRpt; ++h) s[h] = 0.f;
#pragma unroll
    for (int m = 0; m < kT; m += 4) {
        const float4 y = *reinterpret_cast<const float4*>(Y + lane * kLd + m);
#pragma unroll
        for (int h = 0; h < kRpt; ++h)
            s[h] = dot4(*reinterpret_cast<const float4*>(X + (warp + kCsWarps * h) * kLd + m), y, s[h]);
    }
}

// L L^T = T in place (lower triangle; the upper one is set to 0) and Dv = L^-1
// (lower, row-major, upper 0), by the whole CTA with one barrier per pivot.
// Thread (warp, lane) keeps the elements (r, c) = (warp + 8 h, lane) of the
// Schur complement S and of B in registers (B = I initially).  Pivot j: the
// threads holding column j of S and row j of B publish them (double buffer pv),
// then every thread applies S_rc -= S_rj S_cj / S_jj (r, c > j) and
// B_rw -= S_rj B_jw / S_jj (r > j).  At the end S_rc (r >= c) is column c of
// the factor before scaling: L_rc = S_rc / sqrt(S_cc), and L^-1_rw = B_rw /
// sqrt(S_rr) (right-looking forward substitution of L X = I).  Called by every
// thread of the CTA.
__device__ __forceinline__ void cs_diag(float* T, float* Dv, float* pv, int* fail, float* gDv) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float a[kRpt], bm[kRpt], dr[kRpt], dc = 1.f;
#pragma unroll
    for (int h = 0; h < kRpt; ++h) {
        a[h] = T[(warp + kCsWarps * h) * kLd + lane];
        bm[h] = warp + kCsWarps * h == lane ? 1.f : 0.f;
        dr[h] = 1.f;
    }
    bool bad = false;
#pragma unroll 4
    for (int j = 0; j < kT; ++j) {
        float* col = pv + (j & 1) * 2 * kT;  // column j of S
        float* row = col + kT;                // row j of B
        if (lane == j) {
#pragma unroll
            for (int h = 0; h < kRpt; ++h) col[warp + kCsWarps * h] = a[h];
        }
#pragma unroll
        for (int h = 0; h < kRpt; ++h)
            if (warp + kCsWarps * h == j) row[lane] = bm[h];
        __syncthreads();
        const float d = col[j];
        bad = bad || !(d > 0.f);
        const float id = __fdividef(1.f, d);  // the factor only preconditions the FP64 refinement
        const float scj = col[lane] * id, bj = row[lane];
        if (lane == j) dc = d;
#pragma unroll
        for (int h = 0; h < kRpt; ++h) {
            const int r = warp + kCsWarps * h;
            if (r == j) dr[h] = d;
            if (r > j) {
                const float srj = col[r];
                if (lane > j) a[h] = fmaf(-srj, scj, a[h]);
                bm[h] = fmaf(-srj * id, bj, bm[h]);
            }
        }
    }
    const float rc = rsqrtf(dc);
#pragma unroll
    for (int h = 0; h < kRpt; ++h) {
        const int r = warp + kCsWarps * h;
        T[r * kLd + lane] = r >= lane ? a[h] * rc : 0.f;
        const float xr = bm[h] * rsqrtf(dr[h]);
        Dv[r * kLd + lane] = xr;
        gDv[r * kT + lane] = xr;  // the global copy the other CTAs read
    }
    if (bad && threadIdx.x == 0) *fail = 1;
    __syncthreads();
}

}  // namespace tile
}  // namespace pba
