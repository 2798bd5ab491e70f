// pba_solve_sparse.cu -- the damped solve of one Levenberg-Marquardt step
// (Sec. IV-C) for pose graphs too large for one dense factor.  The system in
// pose variables is gathered block by block straight from the pair blocks
// (nothing of size (6N)^2 is formed), ordered so that its envelope is small,
// Jacobi-scaled, damped and factorised in FP32 in tile-envelope storage, and
// solved to FP64 accuracy by iterative refinement.  Each independent
// component of the variable graph (a connected set of pose variables, such as
// one problem of a batch) is solved by its own thread-block cluster, all
// components in one launch.
//
// Arithmetic (that of launch_solve_mixed and k_solve_cluster):
//   D = diag(H_ff + lambda I)^-1/2 (formed in FP32), A' = D (H_ff + lambda I) D,
//   b' = -D b_f;  L L^T = fl32(A');  x = 0, r = b';
//   `refinements` times: z = (L L^T)^-1 r in FP32, x += z, r = b' - A' x in FP64;
//   dx_f = D x.  The step fails (chol_fail) when a pivot is not positive or a
//   component's last |r| exceeds kRefineTol |b'|.
//
// Structure.  The variables of a component are ordered (natural order or
// reverse Cuthill-McKee, whichever has the smaller envelope), 6 unknowns
// each, and padded to whole tile rows of 32 unknowns (identity on the
// padding).  Row s of A' has its first nonzero in column f(s); the Cholesky
// factor has no nonzero left of f(s) either (fill stays inside the
// envelope), so tile row I stores only the tiles (I, F(I) .. I), F(I) the
// smallest tile column of f(s) over its rows.
//
// Cluster schedule.  Tile row I of a component is owned by CTA I mod C of
// its cluster; tiles and vectors live in global memory (L2-resident) and data
// written by another CTA is read through L2 after a cluster barrier.  One
// cluster barrier per step:
//   factorisation, step k: (a) A_IJ -= L_I,k-1 L_J,k-1^T for the own rows
//     I > k and k <= J <= I (deferred from step k-1); (b) L_Ik = A_Ik Dinv_k^T;
//     (c) look-ahead: the owner of row k+1 applies column k to its diagonal
//     tile, then factorises and inverts it, so step k+1 finds Dinv_k+1 ready;
//   forward L y = r, step k: the owner of row k forms y_k = Dinv_k r_k; then
//     every CTA subtracts L_Ik y_k from its rows I > k;
//   backward L^T z = y, step k descending: the owner of row k forms
//     z_k = Dinv_k^T (y_k - acc_k); then every CTA adds L_kM^T z_k to acc_M of
//     its rows M < k.
// Failures are data (flags), never early exits: every thread of every CTA
// reaches every cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "pba_internal.cuh"
#include "pba_tile.cuh"

namespace pba {

namespace {

namespace cg = cooperative_groups;
using namespace tile;

constexpr int kSpStage = 4;  // target tiles per round of the trailing update
constexpr int kSpMaxCluster = 16;

// ------------------------------------------------------------ gathering

// Lower block e of H_ff in pose variables (permuted positions): the sum of its
// pair-block contributions (pair, row role, column role).  Thread t < 36 sums
// entry (t / 6, t % 6).
__global__ void k_sp_blocks(const double* __restrict__ blocks, const SpPlanDev pl) {
    const int e = blockIdx.x, t = threadIdx.x;
    if (t >= 36) return;
    const int r = t / 6, c = t % 6;
    double s = 0.0;
    for (int k = pl.blk_start[e]; k < pl.blk_start[e + 1]; ++k) {
        const int4 q = pl.blk_contrib[k];
        s += blocks[(long long)q.x * kBlockStride + 12 * (6 * q.y + r) + 6 * q.z + c];
    }
    pl.Hv[36 * (long long)e + t] = s;
}

// b of every position: the sum of its pair-block contributions (pair, role).
__global__ void k_sp_rhs(const double* __restrict__ blocks, const SpPlanDev pl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * pl.nv) return;
    const int v = i / 6, r = i % 6;
    double s = 0.0;
    for (int k = pl.b_start[v]; k < pl.b_start[v + 1]; ++k) {
        const int2 q = pl.b_contrib[k];
        s += blocks[(long long)q.x * kBlockStride + 144 + 6 * q.y + r];
    }
    pl.bvec[i] = s;
}

// lambda for this step (explicit >= 0, the schedule's value, or automatic:
// 1e-4 x max diag H_ff), as k_lm_prepare.
__global__ void k_sp_prepare(const SpPlanDev pl, LmState* st, double explicit_lambda) {
    __shared__ double smax[256];
    double mx = 0.0;
    for (int i = threadIdx.x; i < 6 * pl.nv; i += blockDim.x) {
        const int v = i / 6, r = i % 6;
        mx = fmax(mx, pl.Hv[36 * (long long)pl.diag_blk[v] + 7 * r]);
    }
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double lam;
        if (explicit_lambda >= 0.0) lam = explicit_lambda;
        else if (st->lambda >= 0.0) lam = st->lambda;
        else lam = 1e-4 * smax[0];
        st->lambda_used = lam;
        st->chol_fail = 0;
        st->status = 0;
        st->accepted = 0;
    }
}

// Per unknown s (permuted, padded): D (FP32, as the dense solves), b' = -D b,
// x = 0; the padding gets D = 1, b' = 0 and a unit diagonal in its tile.
__global__ void k_sp_scale(const SpPlanDev pl, const LmState* __restrict__ st) {
    const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (s >= 32LL * pl.n_rows) return;
    const int v = pl.pos_of_scalar[s];
    float d = 1.f;
    double bs = 0.0;
    if (v >= 0) {
        const int r = (int)(s - pl.scal_of_pos[v]);
        const float h = (float)(pl.Hv[36 * (long long)pl.diag_blk[v] + 7 * r] + st->lambda_used);
        d = h > 0.f ? rsqrtf(h) : 0.f;
        bs = -pl.bvec[6 * v + r] * (double)d;
    } else {
        const int I = (int)(s / kT), w = (int)(s % kT);
        pl.L[(pl.tile_off[I] + (I - pl.tile_first[I])) * (kT * kT) + w * kT + w] = 1.f;
    }
    pl.dsc[s] = (double)d;
    pl.dsc32[s] = d;
    pl.bsc[s] = bs;
    pl.x[s] = 0.0;
}

// A' = D (H_ff + lambda I) D in FP32 into the envelope tiles: the lower
// triangle of every lower block (the diagonal blocks' lower halves).
__global__ void k_sp_fill(const SpPlanDev pl, const LmState* __restrict__ st) {
    const int e = blockIdx.x, t = threadIdx.x;
    if (t >= 36) return;
    const int2 uv = pl.blk[e];
    const int r = t / 6, c = t % 6;
    if (uv.x == uv.y && c > r) return;
    const long long s = pl.scal_of_pos[uv.x] + r, q = pl.scal_of_pos[uv.y] + c;
    const double h = pl.Hv[36 * (long long)e + t] + (s == q ? st->lambda_used : 0.0);
    const int I = (int)(s / kT), J = (int)(q / kT);
    pl.L[(pl.tile_off[I] + (J - pl.tile_first[I])) * (kT * kT) + (s % kT) * kT + (q % kT)] =
        (float)h * pl.dsc32[s] * pl.dsc32[q];
}

// ------------------------------------------------------------ the cluster solve

__device__ __forceinline__ float* gtile(const SpPlanDev& pl, int I, int J) {
    return pl.L + (pl.tile_off[I] + (J - pl.tile_first[I])) * (kT * kT);
}

// 32 x 32 tiles from global memory (stride 32, read through L2) into shared
// memory (stride kLd): all loads of a thread in flight before the stores.
template <int MAXN>
__device__ __forceinline__ void load_tiles(float* const (&dst)[MAXN], const float* const (&src)[MAXN], int n) {
    const int r = threadIdx.x >> 3, c = 4 * (threadIdx.x & 7);
    float4 v[MAXN];
#pragma unroll
    for (int t = 0; t < MAXN; ++t)
        if (t < n) v[t] = ld_cg4(src[t] + r * kT + c);
#pragma unroll
    for (int t = 0; t < MAXN; ++t)
        if (t < n) *reinterpret_cast<float4*>(dst[t] + r * kLd + c) = v[t];
}

__device__ __forceinline__ void store_tile(float* g, const float* s) {
    const int r = threadIdx.x >> 3, c = 4 * (threadIdx.x & 7);
    *reinterpret_cast<float4*>(g + r * kT + c) = *reinterpret_cast<const float4*>(s + r * kLd + c);
}

// y[r] = sum_m M[r][m] v[m] (transposed: y[c] = sum_m M[m][c] v[m]) for a
// global tile M (stride 32) and a 32-vector v in shared memory; the result
// (32 floats) goes to out (shared).  Called by the whole CTA.
template <bool TRANS>
__device__ __forceinline__ void tile_matvec(const float* M, const float* v, float* out, float* red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread (warp, lane): rows (or columns) of its 4-row slice m = 4 warp .. 4 warp + 3
    float s = 0.f;
    if (TRANS) {
        // lane = column c; warp sums the rows m = 4 warp + h
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int m = 4 * warp + h;
            s = fmaf(__ldcg(M + m * kT + lane), v[m], s);
        }
    } else {
        // lane = column m of rows r = 4 warp + h: reduce over the lanes
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            float p = __ldcg(M + (4 * warp + h) * kT + lane) * v[lane];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
            if (lane == h) s = p;
        }
    }
    red[warp * kT + lane] = s;
    __syncthreads();
    if (threadIdx.x < kT) {
        float y = 0.f;
        if (TRANS) {
#pragma unroll
            for (int w = 0; w < kCsWarps; ++w) y += red[w * kT + threadIdx.x];
        } else {
            y = red[(threadIdx.x / 4) * kT + (threadIdx.x % 4)];
        }
        out[threadIdx.x] = y;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kCsThreads, 1)
    k_sp_solve(const SpPlanDev pl, LmState* st, int refinements, double* __restrict__ dx) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int C = pl.C;
    const int rank = (int)cl.block_rank();
    const int comp = blockIdx.x / C;
    const int2 cr = pl.comp_rows[comp];
    const int row0 = cr.x, T = cr.y;
    const int tid = threadIdx.x;
    float* sLi = reinterpret_cast<float*>(smem);  // L_I,k-1 (update) / A_Ik then L_Ik (b)
    float* sLj = sLi + kTF;                       // kSpStage operand tiles L_J,k-1
    float* sA = sLj + kSpStage * kTF;             // kSpStage target tiles A_IJ
    float* sD = sA + kSpStage * kTF;              // Dinv_k
    float* sT = sD + kTF;                         // diagonal tile of the look-ahead
    float* sDn = sT + kTF;                        // its inverse
    float* pv = sDn + kTF;                        // 4 x 32: pivot exchange of cs_diag
    float* sv = pv + 4 * kT;                      // 32: vector operand
    float* so = sv + kT;                          // 32: vector result
    float* red = so + kT;                         // kCsWarps x 32: reduction scratch
    int* sflag = reinterpret_cast<int*>(red + kCsWarps * kT);  // [0] pivot failure
    double* sred = reinterpret_cast<double*>(sflag + 4);       // kCsWarps x 2

    if (tid == 0) sflag[0] = 0;
    __syncthreads();
    const int* F = pl.tile_first;
    auto owner = [&](int k) { return k % C; };

    // ---- factorisation
    if (rank == 0) {
        const int I = row0;
        float* d[1] = {sT};
        const float* s[1] = {gtile(pl, I, I)};
        load_tiles<1>(d, s, 1);
        __syncthreads();
        cs_diag(sT, sDn, pv, sflag, pl.Dinv + (long long)I * kT * kT);
        store_tile(gtile(pl, I, I), sT);
    }
    cl.sync();
    for (int k = 0; k < T; ++k) {
        const int K = row0 + k;
        bool have_b = false;
        for (int il = rank; il < T; il += C) have_b = have_b || (il > k && F[row0 + il] <= K);
        if (have_b) {
            float* d[1] = {sD};
            const float* s[1] = {pl.Dinv + (long long)K * kT * kT};
            load_tiles<1>(d, s, 1);
        }
        for (int il = rank; il < T; il += C) {
            if (il <= k) continue;
            const int I = row0 + il;
            if (F[I] > K) continue;  // no tile in columns <= K yet
            // (a) column k-1 into the tiles (I, J), K <= J <= I, with L_J,k-1 != 0
            if (k >= 1 && F[I] <= K - 1) {
                {
                    float* d[1] = {sLi};
                    const float* s[1] = {gtile(pl, I, K - 1)};
                    load_tiles<1>(d, s, 1);
                }
                int J = K;
                while (J <= I) {
                    int js[kSpStage], nj = 0;
                    while (J <= I && nj < kSpStage) {
                        if (F[J] <= K - 1) js[nj++] = J;
                        ++J;
                    }
                    if (nj == 0) continue;
                    // operands L_J,k-1 and targets A_IJ of the round: 2 nj loads in flight per thread
                    {
                        const int r = tid >> 3, c = 4 * (tid & 7);
                        float4 v[2 * kSpStage];
#pragma unroll
                        for (int t = 0; t < kSpStage; ++t)
                            if (t < nj) {
                                v[t] = ld_cg4(gtile(pl, js[t], K - 1) + r * kT + c);
                                v[kSpStage + t] = ld_cg4(gtile(pl, I, js[t]) + r * kT + c);
                            }
#pragma unroll
                        for (int t = 0; t < kSpStage; ++t)
                            if (t < nj) {
                                *reinterpret_cast<float4*>(sLj + t * kTF + r * kLd + c) = v[t];
                                *reinterpret_cast<float4*>(sA + t * kTF + r * kLd + c) = v[kSpStage + t];
                            }
                    }
                    __syncthreads();
                    for (int t = 0; t < nj; ++t) {
                        float acc[kRpt];
                        tile_rows_dot(sLi, sLj + t * kTF, acc);
                        const int lane = tid & 31, warp = tid >> 5;
                        float* A = sA + t * kTF;
#pragma unroll
                        for (int h = 0; h < kRpt; ++h) A[(warp + kCsWarps * h) * kLd + lane] -= acc[h];
                    }
                    __syncthreads();
                    for (int t = 0; t < nj; ++t) store_tile(gtile(pl, I, js[t]), sA + t * kTF);
                    __syncthreads();
                }
            }
            // (b) L_IK = A_IK Dinv_K^T
            {
                float* d[1] = {sA};
                const float* s[1] = {gtile(pl, I, K)};
                load_tiles<1>(d, s, 1);
                __syncthreads();
                float acc[kRpt];
                tile_rows_dot(sA, sD, acc);
                const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
                for (int h = 0; h < kRpt; ++h) sLi[(warp + kCsWarps * h) * kLd + lane] = acc[h];
                __syncthreads();
                store_tile(gtile(pl, I, K), sLi);
            }
            // (c) look-ahead: the diagonal tile of row K+1 gets column K, then is factorised
            if (il == k + 1) {
                float* d[1] = {sT};
                const float* s[1] = {gtile(pl, I, I)};
                load_tiles<1>(d, s, 1);
                __syncthreads();
                float acc[kRpt];
                tile_rows_dot(sLi, sLi, acc);
                const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
                for (int h = 0; h < kRpt; ++h) sT[(warp + kCsWarps * h) * kLd + lane] -= acc[h];
                __syncthreads();
                cs_diag(sT, sDn, pv, sflag, pl.Dinv + (long long)I * kT * kT);
                store_tile(gtile(pl, I, I), sT);
            }
            __syncthreads();
        }
        // a row K+1 whose envelope starts at K+1 has no column-K update: factorise it as it is
        if (k + 1 < T && owner(k + 1) == rank && F[K + 1] > K) {
            float* d[1] = {sT};
            const float* s[1] = {gtile(pl, K + 1, K + 1)};
            load_tiles<1>(d, s, 1);
            __syncthreads();
            cs_diag(sT, sDn, pv, sflag, pl.Dinv + (long long)(K + 1) * kT * kT);
            store_tile(gtile(pl, K + 1, K + 1), sT);
            __syncthreads();
        }
        cl.sync();
    }

    // ---- refinement: x = 0, r = b' (FP32 copy); |b'|^2 of the own rows
    const double lam = st->lambda_used;
    double nb = 0.0, nr = 0.0;
    for (int il = rank; il < T; il += C) {
        const long long s0 = (long long)(row0 + il) * kT;
        if (tid < kT) {
            const double b = pl.bsc[s0 + tid];
            pl.rv[s0 + tid] = (float)b;
            nb += b * b;
        }
    }
    for (int pass = 0; pass < refinements; ++pass) {
        // forward: L y = r
        for (int k = 0; k < T; ++k) {
            const int K = row0 + k;
            if (owner(k) == rank) {
                if (tid < kT) sv[tid] = pl.rv[(long long)K * kT + tid];
                __syncthreads();
                tile_matvec<false>(pl.Dinv + (long long)K * kT * kT, sv, so, red);
                if (tid < kT) pl.yv[(long long)K * kT + tid] = so[tid];
            }
            cl.sync();
            bool any = false;
            for (int il = rank; il < T; il += C) any = any || (il > k && F[row0 + il] <= K);
            if (any) {
                if (tid < kT) sv[tid] = __ldcg(pl.yv + (long long)K * kT + tid);
                __syncthreads();
                for (int il = rank; il < T; il += C) {
                    const int I = row0 + il;
                    if (il <= k || F[I] > K) continue;
                    tile_matvec<false>(gtile(pl, I, K), sv, so, red);
                    if (tid < kT) pl.rv[(long long)I * kT + tid] -= so[tid];
                }
            }
        }
        // backward: L^T z = y
        for (int il = rank; il < T; il += C)
            if (tid < kT) pl.acc[(long long)(row0 + il) * kT + tid] = 0.f;
        for (int k = T - 1; k >= 0; --k) {
            const int K = row0 + k;
            if (owner(k) == rank) {
                __syncthreads();
                if (tid < kT) sv[tid] = pl.yv[(long long)K * kT + tid] - pl.acc[(long long)K * kT + tid];
                __syncthreads();
                tile_matvec<true>(pl.Dinv + (long long)K * kT * kT, sv, so, red);
                if (tid < kT) pl.zv[(long long)K * kT + tid] = so[tid];
            }
            cl.sync();
            bool any = false;
            for (int il = rank; il < k; il += C) any = any || (row0 + il >= F[K]);
            if (any) {
                if (tid < kT) sv[tid] = __ldcg(pl.zv + (long long)K * kT + tid);
                __syncthreads();
                for (int il = rank; il < k; il += C) {
                    const int M = row0 + il;
                    if (M < F[K]) continue;
                    tile_matvec<true>(gtile(pl, K, M), sv, so, red);
                    if (tid < kT) pl.acc[(long long)M * kT + tid] += so[tid];
                }
            }
        }
        // x += z (own rows), then r = b' - A' x in FP64 for the own rows
        for (int il = rank; il < T; il += C) {
            const long long s0 = (long long)(row0 + il) * kT;
            if (tid < kT) pl.x[s0 + tid] += (double)pl.zv[s0 + tid];
        }
        cl.sync();
        nr = 0.0;
        for (int il = rank; il < T; il += C) {
            const long long s0 = (long long)(row0 + il) * kT;
            // warp w handles the unknowns s0 + 4 w .. s0 + 4 w + 3, its lanes the row's blocks
            const int lane = tid & 31, warp = tid >> 5;
            for (int h = 0; h < 4; ++h) {
                const long long s = s0 + 4 * warp + h;
                const int v = pl.pos_of_scalar[s];
                double acc = 0.0;
                if (v >= 0) {
                    const int rr = (int)(s - pl.scal_of_pos[v]);
                    for (int it = pl.row_start[v] + lane; it < pl.row_start[v + 1]; it += 32) {
                        const int2 bi = pl.row_items[it];
                        const int2 uv = pl.blk[bi.x];
                        const int other = bi.y ? uv.x : uv.y;
                        const long long q0 = pl.scal_of_pos[other];
                        const double* Hb = pl.Hv + 36 * (long long)bi.x;
#pragma unroll
                        for (int c = 0; c < 6; ++c) {
                            const double h = bi.y ? Hb[6 * c + rr] : Hb[6 * rr + c];
                            acc += h * (pl.dsc[q0 + c] * __ldcg(pl.x + q0 + c));
                        }
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                if (lane == 0) {
                    double r = 0.0;
                    if (v >= 0) {
                        const double xs = pl.dsc[s] * pl.x[s];
                        r = pl.bsc[s] - pl.dsc[s] * (acc + lam * xs);
                    }
                    pl.r64[s] = r;
                    pl.rv[s] = (float)r;
                    nr += r * r;
                }
            }
        }
        __syncthreads();  // rv is written by every warp and read by warp 0 in the next forward solve
    }

    // ---- convergence (per component) and the step dx_f = D x in variable order
    {
        const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            nb += __shfl_xor_sync(0xffffffffu, nb, o);
            nr += __shfl_xor_sync(0xffffffffu, nr, o);
        }
        if (lane == 0) {
            sred[2 * warp] = nb;
            sred[2 * warp + 1] = nr;
        }
        __syncthreads();
        if (tid == 0) {
            double a = 0.0, b = 0.0;
            for (int w = 0; w < kCsWarps; ++w) {
                a += sred[2 * w];
                b += sred[2 * w + 1];
            }
            pl.nrm[2 * (long long)blockIdx.x] = a;
            pl.nrm[2 * (long long)blockIdx.x + 1] = b;
        }
    }
    for (int il = rank; il < T; il += C) {
        const long long s0 = (long long)(row0 + il) * kT;
        if (tid < kT) {
            const long long s = s0 + tid;
            const int v = pl.pos_of_scalar[s];
            if (v >= 0) dx[6 * (long long)pl.var_of_pos[v] + (s - pl.scal_of_pos[v])] = pl.dsc[s] * pl.x[s];
        }
    }
    cl.sync();
    if (rank == 0 && tid == 0) {
        double a = 0.0, b = 0.0;
        for (int c = 0; c < C; ++c) {
            a += __ldcg(pl.nrm + 2 * ((long long)comp * C + c));
            b += __ldcg(pl.nrm + 2 * ((long long)comp * C + c) + 1);
        }
        if (!(b <= kRefineTol * kRefineTol * a)) atomicExch(&st->chol_fail, 1);
    }
    if (tid == 0 && sflag[0]) atomicExch(&st->chol_fail, 1);
}

int g_sp_cmax[16];
bool g_sp_init_done = false;
std::mutex g_sp_mutex;

constexpr int kSpSmemFloats = 4 * kTF + 2 * kSpStage * kTF + 4 * kT + 2 * kT + kCsWarps * kT + 4;
constexpr int kSpSmemBytes = 4 * kSpSmemFloats + 8 * 2 * kCsWarps + 16;

// The largest cluster (<= 16) the device schedules with this kernel's shared memory.
int sp_cluster_max() {
    std::lock_guard<std::mutex> lock(g_sp_mutex);
    if (!g_sp_init_done) {
        for (int d = 0; d < 16; ++d) g_sp_cmax[d] = -1;
        g_sp_init_done = true;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 16) return 0;
    int& cmax = g_sp_cmax[dev];
    if (cmax >= 0) return cmax;
    cmax = 0;
    if (cudaFuncSetAttribute(k_sp_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpSmemBytes) != cudaSuccess ||
        cudaFuncSetAttribute(k_sp_solve, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    for (int c = kSpMaxCluster; c >= 1; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kCsThreads);
        cfg.dynamicSmemBytes = kSpSmemBytes;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_sp_solve, &cfg) == cudaSuccess && clusters > 0) {
            cmax = c;
            break;
        }
        cudaGetLastError();
    }
    return cmax;
}

}  // namespace

// ------------------------------------------------------------ host plan

// Envelope size (sum over positions of position - first coupled position) of an ordering.
static long long envelope_of(const std::vector<std::vector<int>>& adj, const std::vector<int>& order,
                             std::vector<int>& pos_tmp) {
    for (size_t k = 0; k < order.size(); ++k) pos_tmp[order[k]] = (int)k;
    long long e = 0;
    for (size_t k = 0; k < order.size(); ++k) {
        int lo = (int)k;
        for (int v : adj[order[k]]) lo = std::min(lo, pos_tmp[v]);
        e += (long long)k - lo;
    }
    return e;
}

// Reverse Cuthill-McKee order of one component (`nodes`, in any order): a
// breadth-first search from a pseudo-peripheral node (the far end of two
// searches from a node of smallest degree), neighbours taken by increasing
// degree, reversed.
static std::vector<int> rcm_order(const std::vector<std::vector<int>>& adj, const std::vector<int>& nodes,
                                  std::vector<int>& mark, int stamp0) {
    auto bfs = [&](int start, int stamp, std::vector<int>& out) {
        out.clear();
        out.push_back(start);
        mark[start] = stamp;
        for (size_t h = 0; h < out.size(); ++h) {
            std::vector<int> nb;
            for (int v : adj[out[h]])
                if (mark[v] != stamp) {
                    mark[v] = stamp;
                    nb.push_back(v);
                }
            std::stable_sort(nb.begin(), nb.end(), [&](int a, int b) { return adj[a].size() < adj[b].size(); });
            out.insert(out.end(), nb.begin(), nb.end());
        }
    };
    int start = nodes[0];
    for (int v : nodes)
        if (adj[v].size() < adj[start].size()) start = v;
    std::vector<int> order;
    for (int rep = 0; rep < 2; ++rep) {
        bfs(start, stamp0 + rep, order);
        start = order.back();
    }
    bfs(start, stamp0 + 2, order);
    std::reverse(order.begin(), order.end());
    return order;
}

bool sparse_plan(int n_vars, const std::vector<int>& frame_var, const std::vector<int32_t>& pairs, int cmax,
                 SpPlanHost* out) {
    SpPlanHost P;
    const int nv = n_vars;
    const int m = (int)(pairs.size() / 2);
    P.nv = nv;
    if (nv <= 0 || cmax < 1) return false;
    // variable graph
    std::vector<std::vector<int>> adj(nv);
    for (int q = 0; q < m; ++q) {
        const int u = frame_var[pairs[2 * q]], v = frame_var[pairs[2 * q + 1]];
        if (u < 0 || v < 0 || u == v) continue;
        adj[u].push_back(v);
        adj[v].push_back(u);
    }
    for (auto& a : adj) {
        std::sort(a.begin(), a.end());
        a.erase(std::unique(a.begin(), a.end()), a.end());
    }
    // components (by smallest variable), each ordered naturally or by RCM
    std::vector<int> comp_of(nv, -1), mark(nv, -1), pos_tmp(nv, 0), order_all;
    std::vector<int> comp_first;  // start of each component in order_all
    int stamp = 0;
    for (int s = 0; s < nv; ++s) {
        if (comp_of[s] >= 0) continue;
        const int c = (int)comp_first.size();
        std::vector<int> nodes{s};
        comp_of[s] = c;
        for (size_t h = 0; h < nodes.size(); ++h)
            for (int v : adj[nodes[h]])
                if (comp_of[v] < 0) {
                    comp_of[v] = c;
                    nodes.push_back(v);
                }
        std::sort(nodes.begin(), nodes.end());
        std::vector<int> best = nodes;
        if (nodes.size() > 2) {
            std::vector<int> rcm = rcm_order(adj, nodes, mark, stamp);
            stamp += 3;
            if (envelope_of(adj, rcm, pos_tmp) < envelope_of(adj, nodes, pos_tmp)) best = rcm;
        }
        comp_first.push_back((int)order_all.size());
        order_all.insert(order_all.end(), best.begin(), best.end());
    }
    const int n_comp = (int)comp_first.size();
    comp_first.push_back(nv);
    // positions, unknowns and tile rows: each component starts on a tile row
    P.var_of_pos = order_all;
    std::vector<int> pos_of_var(nv);
    for (int k = 0; k < nv; ++k) pos_of_var[order_all[k]] = k;
    P.scal_of_pos.assign(nv, 0);
    int rows = 0;
    for (int c = 0; c < n_comp; ++c) {
        const int n = comp_first[c + 1] - comp_first[c];
        const int T = (6 * n + kT - 1) / kT;
        P.comp_rows.push_back(make_int2(rows, T));
        for (int l = 0; l < n; ++l) P.scal_of_pos[comp_first[c] + l] = kT * rows + 6 * l;
        rows += T;
    }
    P.n_rows = rows;
    P.pos_of_scalar.assign((size_t)rows * kT, -1);
    for (int v = 0; v < nv; ++v)
        for (int r = 0; r < 6; ++r) P.pos_of_scalar[(size_t)P.scal_of_pos[v] + r] = v;
    // lower blocks (row position >= column position) and their contributions
    std::vector<std::vector<int4>> contrib_of;
    std::vector<std::pair<long long, int>> keyed;  // (row * nv + col, block) for lookup
    std::vector<int2> blk;
    auto block_index = [&](int a, int b) {
        const long long key = (long long)a * nv + b;
        auto it = std::lower_bound(keyed.begin(), keyed.end(), std::make_pair(key, -1));
        return (it != keyed.end() && it->first == key) ? it->second : -1;
    };
    {
        std::vector<long long> keys;
        for (int v = 0; v < nv; ++v) keys.push_back((long long)v * nv + v);
        for (int q = 0; q < m; ++q) {
            const int u = frame_var[pairs[2 * q]], v = frame_var[pairs[2 * q + 1]];
            if (u < 0 || v < 0) continue;
            const int a = std::max(pos_of_var[u], pos_of_var[v]), b = std::min(pos_of_var[u], pos_of_var[v]);
            keys.push_back((long long)a * nv + b);
        }
        std::sort(keys.begin(), keys.end());
        keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
        for (size_t e = 0; e < keys.size(); ++e) {
            keyed.emplace_back(keys[e], (int)e);
            blk.push_back(make_int2((int)(keys[e] / nv), (int)(keys[e] % nv)));
        }
        contrib_of.resize(blk.size());
        for (int q = 0; q < m; ++q) {
            const int fr[2] = {pairs[2 * q], pairs[2 * q + 1]};
            for (int rr = 0; rr < 2; ++rr)
                for (int cc = 0; cc < 2; ++cc) {
                    const int u = frame_var[fr[rr]], v = frame_var[fr[cc]];
                    if (u < 0 || v < 0) continue;
                    const int a = pos_of_var[u], b = pos_of_var[v];
                    if (a < b) continue;  // its transpose (cc, rr) is the lower one
                    contrib_of[block_index(a, b)].push_back(make_int4(q, rr, cc, 0));
                }
        }
    }
    P.blk = blk;
    P.blk_start.push_back(0);
    for (auto& cv : contrib_of) {
        P.blk_contrib.insert(P.blk_contrib.end(), cv.begin(), cv.end());
        P.blk_start.push_back((int)P.blk_contrib.size());
    }
    P.diag_blk.assign(nv, 0);
    for (int v = 0; v < nv; ++v) P.diag_blk[v] = block_index(v, v);
    // b contributions per position
    {
        std::vector<std::vector<int2>> bc(nv);
        for (int q = 0; q < m; ++q)
            for (int r = 0; r < 2; ++r) {
                const int u = frame_var[pairs[2 * q + r]];
                if (u >= 0) bc[pos_of_var[u]].push_back(make_int2(q, r));
            }
        P.b_start.push_back(0);
        for (auto& v : bc) {
            P.b_contrib.insert(P.b_contrib.end(), v.begin(), v.end());
            P.b_start.push_back((int)P.b_contrib.size());
        }
    }
    // block rows for the FP64 product with both triangles: (block, used transposed)
    {
        std::vector<std::vector<int2>> ri(nv);
        for (size_t e = 0; e < blk.size(); ++e) {
            ri[blk[e].x].push_back(make_int2((int)e, 0));
            if (blk[e].x != blk[e].y) ri[blk[e].y].push_back(make_int2((int)e, 1));
        }
        P.row_start.push_back(0);
        for (auto& v : ri) {
            P.row_items.insert(P.row_items.end(), v.begin(), v.end());
            P.row_start.push_back((int)P.row_items.size());
        }
    }
    // tile envelope: F(I) = smallest tile column of the first nonzero of its rows
    P.tile_first.assign(rows, 0);
    for (int I = 0; I < rows; ++I) P.tile_first[I] = I;
    for (const int2& e : blk) {
        const int I0 = P.scal_of_pos[e.x] / kT, I1 = (P.scal_of_pos[e.x] + 5) / kT;
        const int J = P.scal_of_pos[e.y] / kT;
        for (int I = I0; I <= I1; ++I) P.tile_first[I] = std::min(P.tile_first[I], J);
    }
    P.tile_off.assign(rows, 0);
    long long tiles = 0;
    for (int I = 0; I < rows; ++I) {
        P.tile_off[I] = tiles;
        tiles += I - P.tile_first[I] + 1;
    }
    P.n_tiles = tiles;
    // cluster size: up to cmax CTAs per component, no more than the largest component's rows
    int max_rows = 1;
    for (auto& c : P.comp_rows) max_rows = std::max(max_rows, c.y);
    int C = 1;
    while (C * 2 <= std::min(cmax, max_rows)) C *= 2;
    P.C = C;
    *out = std::move(P);
    return true;
}

int sparse_cluster_max() { return sp_cluster_max(); }

cudaError_t launch_sparse_solve(const SpPlanDev& pl, const double* blocks, LmState* st, double explicit_lambda,
                                int refinements, double* dx, cudaStream_t s, int* n_launches) {
    k_sp_blocks<<<pl.nblk, 64, 0, s>>>(blocks, pl);
    k_sp_rhs<<<(6 * pl.nv + 255) / 256, 256, 0, s>>>(blocks, pl);
    k_sp_prepare<<<1, 256, 0, s>>>(pl, st, explicit_lambda);
    cudaError_t e = cudaMemsetAsync(pl.L, 0, sizeof(float) * kT * kT * (size_t)pl.n_tiles, s);
    if (e != cudaSuccess) return e;
    k_sp_scale<<<(int)((32LL * pl.n_rows + 255) / 256), 256, 0, s>>>(pl, st);
    k_sp_fill<<<pl.nblk, 64, 0, s>>>(pl, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = pl.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(pl.n_comp * pl.C);
    cfg.blockDim = dim3(kCsThreads);
    cfg.dynamicSmemBytes = kSpSmemBytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (n_launches) *n_launches += 6;  // kernels (the memset aside)
    return cudaLaunchKernelEx(&cfg, k_sp_solve, pl, st, refinements < 1 ? 1 : refinements, dx);
}

}  // namespace pba
