// pba_solve.cu -- FP64 assembly, the damped gauge-fixed solve in per-tile-step
// launches, box-plus update and the Levenberg-Marquardt accept / reject, all
// on the device.
//
// The paper minimises Eq. total-error-multicue with Levenberg-Marquardt (Sec. IV-C, srrg2_solver);
// the normal equations are H = sum w J^T Omega J, b = sum w J^T Omega e over all
// residuals.  Each step solves (H_ff + lambda I) dx_f = -b_f, where _f drops
// frame 0 (gauge freedom), and applies X_k <- X_k [+] dx_k (Supp.):
// X [+] dx = [R R(dq), R dt + t], R(dq) from the unit quaternion (sqrt(1 - |dq|^2), dq),
// normalised (1, dq) when |dq| >= 1.  The step is kept when the cost decreased
// (lambda / 10), otherwise the poses are restored and lambda grows (x 10).
// Assembly, damping, update and accept are FP64.  The tiled Cholesky kernels
// are templates: FP64 for the FP64 solver, FP32 on the Jacobi-scaled matrix for
// the mixed-precision solver, whose solution is refined with FP64 residuals
// (k_refine_*); the one-launch cluster version of the mixed solve is in
// pba_solve_cluster.cu.
#include <algorithm>

#include "pba_internal.cuh"
#include "../../include/pba.h"

namespace pba {

namespace {

// ------------------------------------------------------------------ assembly

// One block per task: sums the 6x6 sub-blocks of the contributing pairs in a
// fixed order (deterministic) and writes block (a, b) of H and its transpose;
// diagonal tasks also write b_a.  The task's contribution list is staged in
// shared memory and each thread keeps 8 block loads in flight (the sum order
// is unchanged).
constexpr int kAsmStage = 128;
constexpr int kAsmUnroll = 8;

__global__ void __launch_bounds__(64) k_assemble(const AsmTask* __restrict__ tasks,
                                                 const AsmContrib* __restrict__ contrib,
                                                 const double* __restrict__ blocks, int n6, double* __restrict__ H,
                                                 double* __restrict__ b) {
    __shared__ AsmContrib sc[kAsmStage];
    const AsmTask T = tasks[blockIdx.x];
    const int t = threadIdx.x;
    const bool diag = T.a == T.b;
    // thread t < 36: H entry (r, c); 36 <= t < 42 on diagonal tasks: b entry t - 36
    const int r = t < 36 ? t / 6 : t - 36, c = t < 36 ? t % 6 : 0;
    const bool h_entry = t < 36 && (!diag || r <= c), b_entry = t >= 36 && t < 42 && diag;
    double s = 0.0;
    for (int k0 = T.contrib_begin; k0 < T.contrib_end; k0 += kAsmStage) {
        const int nk = min(kAsmStage, T.contrib_end - k0);
        __syncthreads();  // the previous round's reads of sc are done
        for (int k = t; k < nk; k += blockDim.x) sc[k] = contrib[k0 + k];
        __syncthreads();
        if (h_entry || b_entry) {
            for (int k = 0; k < nk; k += kAsmUnroll) {
                double v[kAsmUnroll];
#pragma unroll
                for (int u = 0; u < kAsmUnroll; ++u) {
                    v[u] = 0.0;
                    if (k + u < nk) {
                        const AsmContrib C = sc[k + u];
                        const long long base = (long long)C.pair * kBlockStride;
                        if (h_entry) v[u] = blocks[base + 12 * (6 * C.row_role + r) + 6 * C.col_role + c];
                        else if (C.add_b) v[u] = blocks[base + 144 + 6 * C.row_role + r];
                    }
                }
#pragma unroll
                for (int u = 0; u < kAsmUnroll; ++u)
                    if (k + u < nk && (h_entry || sc[k + u].add_b)) s += v[u];
            }
        }
    }
    if (h_entry) {
        // diagonal blocks: one sum per unordered entry, mirrored, so H is exactly symmetric
        H[(long long)(6 * T.a + r) * n6 + 6 * T.b + c] = s;
        H[(long long)(6 * T.b + c) * n6 + 6 * T.a + r] = s;
    } else if (b_entry) {
        b[6 * T.a + r] = s;
    }
}

// Sum of the pairs' cost and count (fixed order: strided per thread, then a tree).
__global__ void k_total_cost(const double* __restrict__ blocks, int m, LmState* st, bool candidate) {
    __shared__ double sc[256];
    __shared__ double sn[256];
    __shared__ long long snf[256], snp[256];
    double c = 0.0, n = 0.0;
    long long nf = 0, np = 0;  // status word: non-finite residuals and pairs (exact integer sums)
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        nf += (long long)blocks[(long long)p * kBlockStride + 158];
        np += (long long)blocks[(long long)p * kBlockStride + 159];
    }
    snf[threadIdx.x] = nf;
    snp[threadIdx.x] = np;
    // strided per thread (loads 4 at a time, added in the same order), then a tree
    for (int p0 = threadIdx.x; p0 < m; p0 += 4 * blockDim.x) {
        double vc[4], vn[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = p0 + u * blockDim.x;
            vc[u] = p < m ? blocks[(long long)p * kBlockStride + 156] : 0.0;
            vn[u] = p < m ? blocks[(long long)p * kBlockStride + 157] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            if (p0 + u * blockDim.x < m) {
                c += vc[u];
                n += vn[u];
            }
    }
    sc[threadIdx.x] = c;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sc[threadIdx.x] += sc[threadIdx.x + o];
            sn[threadIdx.x] += sn[threadIdx.x + o];
            snf[threadIdx.x] += snf[threadIdx.x + o];
            snp[threadIdx.x] += snp[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (candidate) {
            st->new_cost = sc[0];
            st->n_valid_new = (long long)sn[0];
            st->nf_res_new = snf[0];
            st->nf_pairs_new = snp[0];
        } else {
            st->cost = sc[0];
            st->n_valid = (long long)sn[0];
            st->nf_res = snf[0];
            st->nf_pairs = snp[0];
        }
    }
}

// ------------------------------------------------------------------ damping

// lambda for this step: explicit (>= 0), the schedule's value, or automatic
// (1e-4 x max diag H_ff) when the schedule holds a negative value.
__global__ void k_lm_prepare(const double* __restrict__ H, int n_frames, LmState* st, double explicit_lambda) {
    __shared__ double smax[256];
    const int n6 = 6 * n_frames;
    double mx = 0.0;
    for (int i = 6 + threadIdx.x; i < n6; i += blockDim.x) mx = fmax(mx, H[(long long)i * n6 + i]);
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

// A = H_ff + lambda I padded to n_pad (identity on the padding); rhs = -b_f.
__global__ void k_damp(const double* __restrict__ H, const double* __restrict__ b, int n_frames, int n_pad,
                       const LmState* __restrict__ st, double* __restrict__ A, double* __restrict__ rhs) {
    const int n6 = 6 * n_frames, n = n6 - 6;
    const long long total = (long long)n_pad * n_pad;
    const double lam = st->lambda_used;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n_pad), j = (int)(idx % n_pad);
        double v;
        if (i < n && j < n) v = H[(long long)(i + 6) * n6 + (j + 6)] + (i == j ? lam : 0.0);
        else v = (i == j) ? 1.0 : 0.0;
        A[idx] = v;
        if (j == 0) rhs[i] = i < n ? -b[i + 6] : 0.0;
    }
}

// ------------------------------------------------------------------ Cholesky
// Right-looking tiled factorisation A = L L^T in place (lower triangle),
// tiles of 32 x 32: factor the diagonal tile, solve the panel below it,
// update the trailing lower triangle.

// Diagonal tile (used for FP64, where one warp's long dependent FP64 chains
// would serialise the tile), 256 threads (thread (c, g) owns column c, rows g, g+8, g+16,
// g+24).  The trailing update of pivot j uses the unscaled column:
// T[r][c] -= T[r][j] T[c][j] / T[j][j], so each step needs one barrier and one
// reciprocal, computed by the owner of the next pivot right after its own
// update.  The same row operations applied to an identity block R give
// R = Lh^-1 for the unit-lower factor of T = Lh diag(d) Lh^T, so the tile
// inverse L^-1 = diag(d)^-1/2 R comes out of the same 31 steps (columns c <= j
// update R while columns c > j update T).  The columns are scaled by
// 1 / sqrt(pivot) once at the end.
template <typename F>
__global__ void __launch_bounds__(256) k_potrf(F* __restrict__ A, int n_pad, int k, LmState* st, F* __restrict__ Dinv) {
    if (st->chol_fail) return;
    __shared__ F T[kTile][kTile + 1];
    __shared__ F R[kTile][kTile + 1];
    __shared__ F inv_piv[kTile];
    __shared__ int fail;
    const int c = threadIdx.x, g = threadIdx.y;  // 32 x 8
    const long long base = (long long)(k * kTile) * n_pad + k * kTile;
    for (int r = g; r < kTile; r += 8) {
        T[r][c] = A[base + (long long)r * n_pad + c];
        R[r][c] = r == c ? F(1) : F(0);
    }
    if (c == 0 && g == 0) fail = 0;
    __syncthreads();
    if (c == 0 && g == 0) {
        const F p0 = T[0][0];
        if (!(p0 > F(0))) fail = 1;
        else inv_piv[0] = F(1) / p0;
    }
    __syncthreads();
    for (int j = 0; j < kTile - 1; ++j) {
        if (fail) break;
        const F ip = inv_piv[j];
        if (c > j) {
            const F tcj = T[c][j] * ip;
            for (int r = g; r < kTile; r += 8)
                if (r >= c) T[r][c] -= T[r][j] * tcj;
        } else {
            // row operation on the identity block: R[r] -= (T[r][j] / T[j][j]) R[j], r > j
            const F rjc = R[j][c] * ip;
            for (int r = g; r < kTile; r += 8)
                if (r > j) R[r][c] -= T[r][j] * rjc;
        }
        // the owner of the next pivot (row j+1, column j+1) computes its reciprocal
        if (c == j + 1 && ((j + 1) & 7) == g) {
            const F pn = T[j + 1][j + 1];
            if (!(pn > F(0))) fail = 1;
            else inv_piv[j + 1] = F(1) / pn;
        }
        __syncthreads();
    }
    if (fail) {
        if (c == 0 && g == 0) st->chol_fail = 1;
        return;
    }
    // L[r][c] = T[r][c] / sqrt(T[c][c]) for r >= c, L^T into the upper triangle;
    // L^-1[r][c] = R[r][c] / sqrt(T[r][r]) for r >= c
    const F s = sqrt(inv_piv[c]);
    F* Dk = Dinv ? Dinv + (long long)k * kTile * kTile : nullptr;
    for (int r = g; r < kTile; r += 8) {
        if (r >= c) {
            const F l = T[r][c] * s;
            A[base + (long long)r * n_pad + c] = l;
            A[base + (long long)c * n_pad + r] = l;
        }
        if (Dk) Dk[r * kTile + c] = r >= c ? R[r][c] * sqrt(inv_piv[r]) : F(0);
    }
}

// Diagonal tile by one warp (FP32): lane i holds row i of the tile in registers.
// Step j: L[j][j] = sqrt(T[j][j]); L[i][j] = T[i][j] / L[j][j] (i > j); the
// rank-1 update T[i][k] -= L[i][j] L[k][j] (j < k <= i) takes L[k][j] from lane
// k by a shuffle.  Then lane c forms column c of L^-1 by forward substitution
// on e_c, reading L from shared memory (the same entry for every lane at each
// step: broadcasts).  Loads and stores go through shared memory so that global
// accesses are row-contiguous; L^T is written into the upper tile.
template <typename F>
__global__ void __launch_bounds__(32) k_potrf_warp(F* __restrict__ A, int n_pad, int k, LmState* st,
                                                   F* __restrict__ Dinv) {
    if (st->chol_fail) return;
    __shared__ F S[kTile][kTile + 1];
    const int lane = threadIdx.x;
    const long long base = (long long)(k * kTile) * n_pad + k * kTile;
    for (int r = 0; r < kTile; ++r) S[r][lane] = A[base + (long long)r * n_pad + lane];
    __syncwarp();
    F a[kTile];
#pragma unroll
    for (int c = 0; c < kTile; ++c) a[c] = S[lane][c];
    bool bad = false;
#pragma unroll
    for (int j = 0; j < kTile; ++j) {
        const F piv = __shfl_sync(0xffffffffu, a[j], j);
        bad = bad || !(piv > F(0));
        const F ljj = sqrt(piv);
        const F lij = lane > j ? a[j] / ljj : (lane == j ? ljj : F(0));
        a[j] = lij;
#pragma unroll
        for (int c = j + 1; c < kTile; ++c) {
            const F lcj = __shfl_sync(0xffffffffu, lij, c);
            if (c <= lane) a[c] -= lij * lcj;
        }
    }
    if (bad) {
        if (lane == 0) st->chol_fail = 1;
        return;
    }
#pragma unroll
    for (int c = 0; c < kTile; ++c) S[lane][c] = c <= lane ? a[c] : F(0);
    __syncwarp();
    // L into the lower tile and L^T into the upper tile, row-contiguous
    for (int r = 0; r < kTile; ++r) A[base + (long long)r * n_pad + lane] = lane <= r ? S[r][lane] : S[lane][r];
    if (Dinv) {
        // column `lane` of L^-1: x_i = (delta_{i,lane} - sum_{lane <= m < i} L[i][m] x_m) / L[i][i]
        F x[kTile];
#pragma unroll
        for (int i = 0; i < kTile; ++i) {
            F s = i == lane ? F(1) : F(0);
#pragma unroll
            for (int m = 0; m < i; ++m) s -= S[i][m] * x[m];
            x[i] = i >= lane ? s / S[i][i] : F(0);
        }
        __syncwarp();
        // Dinv row-major: Dinv[i][lane] = x_i
        F* Dk = Dinv + (long long)k * kTile * kTile;
#pragma unroll
        for (int i = 0; i < kTile; ++i) S[i][lane] = x[i];
        __syncwarp();
        for (int r = 0; r < kTile; ++r) Dk[r * kTile + lane] = S[r][lane];
    }
}

// L_ik = A_ik L_kk^{-T} for tiles i > k (one block per tile, 256 threads).
// Row r: x[m] = (a[m] - sum_{c<m} x[c] L[m][c]) / L[m][m].  With the
// column-normalised factor U[c][m] = L[c][m] / L[m][m] the recurrence runs on
// y[m] = x[m] L[m][m]: y[c] -= y[m] U[c][m], one barrier per column.
template <typename F>
__global__ void __launch_bounds__(256) k_trsm(F* __restrict__ A, int n_pad, int k, const LmState* st) {
    if (st->chol_fail) return;
    __shared__ F U[kTile][kTile + 1];
    __shared__ F Y[kTile][kTile + 1];
    __shared__ F inv[kTile];
    const int i = k + 1 + blockIdx.x;
    const int c = threadIdx.x, g = threadIdx.y;
    const long long lk = (long long)(k * kTile) * n_pad + k * kTile;
    const long long ak = (long long)(i * kTile) * n_pad + k * kTile;
    if (g == 0) inv[c] = F(1) / A[lk + (long long)c * n_pad + c];
    for (int r = g; r < kTile; r += 8) Y[r][c] = A[ak + (long long)r * n_pad + c];
    __syncthreads();
    for (int r = g; r < kTile; r += 8) U[r][c] = r > c ? A[lk + (long long)r * n_pad + c] * inv[c] : F(0);
    __syncthreads();
    for (int m = 0; m < kTile - 1; ++m) {
        if (c > m) {
            const F u = U[c][m];
            for (int r = g; r < kTile; r += 8) Y[r][c] -= Y[r][m] * u;
        }
        __syncthreads();
    }
    // L_ik, and L_ik^T into the upper tile (k, i)
    const long long at = (long long)(k * kTile) * n_pad + i * kTile;
    for (int r = g; r < kTile; r += 8) {
        const F l = Y[r][c] * inv[c];
        A[ak + (long long)r * n_pad + c] = l;
        A[at + (long long)c * n_pad + r] = l;
    }
}

// A_ij -= L_ik L_jk^T for k < j <= i (one block per tile of the trailing lower triangle).
template <typename F>
__global__ void __launch_bounds__(1024) k_syrk(F* __restrict__ A, int n_pad, int k, int nt, const LmState* st) {
    if (st->chol_fail) return;
    __shared__ F Li[kTile][kTile + 1];
    __shared__ F Lj[kTile][kTile + 1];
    // decode blockIdx.x -> (i, j), k < j <= i < nt, column-major over j
    int idx = blockIdx.x, j = k + 1;
    while (idx >= nt - j) {
        idx -= nt - j;
        ++j;
    }
    const int i = j + idx;
    const int tx = threadIdx.x, ty = threadIdx.y;
    Li[ty][tx] = A[(long long)(i * kTile + ty) * n_pad + k * kTile + tx];
    Lj[ty][tx] = A[(long long)(j * kTile + ty) * n_pad + k * kTile + tx];
    __syncthreads();
    F s = F(0);
#pragma unroll 8
    for (int m = 0; m < kTile; ++m) s += Li[ty][m] * Lj[tx][m];
    A[(long long)(i * kTile + ty) * n_pad + j * kTile + tx] -= s;
}

// ------------------------------------------------------------------ triangular solves
// One block of 1024 threads: L y = rhs, then L^T x = y, tile by tile, with the
// inverses Dinv_k of the diagonal tiles (from k_potrf): y_k = Dinv_k (r_k -
// sum_{j<k} L_kj y_j), x_k = Dinv_k^T (y_k - sum_{j>k} (L^T)_kj x_j).  Warp w
// handles row w of the tile; rows of L (lower part) and of L^T (upper part)
// are read with coalesced loads and reduced with warp shuffles.  x overwrites rhs.
template <typename F>
__global__ void __launch_bounds__(1024) k_trsv(const F* __restrict__ A, const F* __restrict__ Dinv, int n_pad,
                                               F* __restrict__ x, const LmState* st) {
    if (st->chol_fail) return;
    __shared__ F t[kTile];
    __shared__ F D[kTile][kTile + 1];
    const int nt = n_pad / kTile;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    // forward
    for (int k = 0; k < nt; ++k) {
        const int row = k * kTile + w;
        const F* Lr = A + (long long)row * n_pad;
        F s = F(0);
        for (int c = lane; c < k * kTile; c += 32) s += Lr[c] * x[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        D[w][lane] = Dinv[(long long)k * kTile * kTile + w * kTile + lane];
        if (lane == 0) t[w] = x[row] - s;
        __syncthreads();
        F y = D[w][lane] * t[lane];
        for (int o = 16; o > 0; o >>= 1) y += __shfl_xor_sync(0xffffffffu, y, o);
        __syncthreads();
        if (lane == 0) x[row] = y;
        __syncthreads();
    }
    // backward
    for (int k = nt - 1; k >= 0; --k) {
        const int row = k * kTile + w;
        const F* Ur = A + (long long)row * n_pad;  // row of L^T (upper part)
        F s = F(0);
        for (int c = (k + 1) * kTile + lane; c < n_pad; c += 32) s += Ur[c] * x[c];
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        D[w][lane] = Dinv[(long long)k * kTile * kTile + w * kTile + lane];
        if (lane == 0) t[w] = x[row] - s;
        __syncthreads();
        F xv = D[lane][w] * t[lane];  // (Dinv^T)[w][lane]
        for (int o = 16; o > 0; o >>= 1) xv += __shfl_xor_sync(0xffffffffu, xv, o);
        __syncthreads();
        if (lane == 0) x[row] = xv;
        __syncthreads();
    }
}

// ------------------------------------------------------------------ mixed-precision solve
// GB300 runs FP32 at ~64x its FP64 rate, so the damped system is factorised in
// FP32 after Jacobi scaling and the solution is refined in FP64 (iterative
// refinement, as in LAPACK's dsposv):
//   D = diag(H_ff + lambda I)^-1/2,  A' = D (H_ff + lambda I) D (unit diagonal),
//   b' = -D b_f;  L L^T = fl32(A');  x = 0, r = b';
//   repeat: z = (L L^T)^-1 r (FP32), x += z (FP64), r = b' - A' x (FP64);
//   dx_f = D x.
// The step is declared failed (chol_fail, then rejected with lambda x 10) when
// the final FP64 residual exceeds kRefineTol |b'|.


// A32 = fl32(D (H_ff + lambda I) D) padded with identity; bs = -D b_f (FP64); x = 0; dscale = D.
__global__ void k_damp_mixed(const double* __restrict__ H, const double* __restrict__ b, int n_frames, int n_pad,
                             const LmState* __restrict__ st, float* __restrict__ A32, double* __restrict__ bs,
                             double* __restrict__ x, double* __restrict__ dscale) {
    const int n6 = 6 * n_frames, n = n6 - 6;
    const long long total = (long long)n_pad * n_pad;
    const double lam = st->lambda_used;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / n_pad), j = (int)(idx % n_pad);
        float v;
        if (i < n && j < n) {
            const double hii = H[(long long)(i + 6) * n6 + (i + 6)] + lam;
            const double hjj = H[(long long)(j + 6) * n6 + (j + 6)] + lam;
            const double hij = H[(long long)(i + 6) * n6 + (j + 6)] + (i == j ? lam : 0.0);
            v = (float)(hij / sqrt(hii * hjj));
        } else {
            v = (i == j) ? 1.f : 0.f;
        }
        A32[idx] = v;
        if (j == 0) {
            double d = 1.0;
            if (i < n) {
                const double hii = H[(long long)(i + 6) * n6 + (i + 6)] + lam;
                d = hii > 0.0 ? 1.0 / sqrt(hii) : 0.0;
            }
            dscale[i] = d;
            bs[i] = i < n ? -b[i + 6] * d : 0.0;
            x[i] = 0.0;
        }
    }
}

// r = b' - A' x in FP64 (one warp per row, A' = D (H_ff + lambda I) D evaluated
// from H), r32 = fl32(r); the last call also records |r|^2 and |b'|^2.
__global__ void k_refine_residual(const double* __restrict__ H, int n_frames, int n_pad, const LmState* st,
                                  const double* __restrict__ dscale, const double* __restrict__ bs,
                                  const double* __restrict__ x, float* __restrict__ r32, double* __restrict__ norms,
                                  int first) {
    if (st->chol_fail) return;
    const int n6 = 6 * n_frames, n = n6 - 6;
    const int lane = threadIdx.x & 31;
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (row >= n_pad) return;
    double r;
    if (first) {
        r = bs[row];
    } else {
        double s = 0.0;
        if (row < n) {
            const double lam = st->lambda_used;
            const double* Hr = H + (long long)(row + 6) * n6 + 6;
            for (int j = lane; j < n; j += 32) s += (Hr[j] + (j == row ? lam : 0.0)) * dscale[j] * x[j];
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
            s *= dscale[row];
        } else {
            s = x[row];  // identity padding
        }
        r = bs[row] - s;
    }
    if (lane == 0) {
        r32[row] = (float)r;
        if (norms) {
            atomicAdd(norms, r * r);
            atomicAdd(norms + 1, bs[row] * bs[row]);
        }
    }
}

// x += z (FP64)
__global__ void k_refine_update(const LmState* st, const float* __restrict__ z, double* __restrict__ x, int n_pad) {
    if (st->chol_fail) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n_pad) x[i] += (double)z[i];
}

// dx_f = D x; mark the step failed when the refinement did not converge.
__global__ void k_refine_finish(LmState* st, const double* __restrict__ dscale, const double* __restrict__ x,
                                double* __restrict__ dx, const double* __restrict__ norms, int n_pad) {
    if (st->chol_fail) return;
    const bool ok = norms[0] <= kRefineTol * kRefineTol * norms[1] || norms[1] == 0.0;
    for (int i = threadIdx.x; i < n_pad; i += blockDim.x) dx[i] = dscale[i] * x[i];
    __syncthreads();
    if (threadIdx.x == 0 && !ok) st->chol_fail = 1;
}

// ------------------------------------------------------------------ update
// cand_k = X_k [+] dx_k (dx_0 = 0); on a failed factorisation cand = poses.
// Gauss-Newton system in pose variables when frames share variables or are
// held fixed: Hr = S^T H S, br = S^T b, S the 0/1 selection of 6 x 6 identity
// blocks (frame f moves with variable v).  Hr gets a leading 6 x 6 zero block
// (a fixed dummy variable) so that the gauge-fixed solve, which drops the
// first block, applies unchanged.  Both triangles sum the same terms in the
// same order (outer loop over the lower index's frames), so Hr is exactly
// symmetric like H.
__global__ void k_reduce_vars(const double* __restrict__ H, const double* __restrict__ b, int n_frames,
                              const int* __restrict__ var_start, const int* __restrict__ var_frames, int n_vars,
                              double* __restrict__ Hr, double* __restrict__ br) {
    const long long n6 = 6LL * n_frames;
    const int nr = 6 * (n_vars + 1);
    const long long total = (long long)nr * nr;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(idx / nr), j = (int)(idx % nr);
        double v = 0.0;
        if (i >= 6 && j >= 6) {
            const int lo = i < j ? i : j, hi = i < j ? j : i;
            const int va = (lo - 6) / 6, x = (lo - 6) % 6, vb = (hi - 6) / 6, y = (hi - 6) % 6;
            for (int fa = var_start[va]; fa < var_start[va + 1]; ++fa) {
                const long long row = 6LL * var_frames[fa] + x;
                for (int gb = var_start[vb]; gb < var_start[vb + 1]; ++gb)
                    v += H[row * n6 + 6LL * var_frames[gb] + y];
            }
        }
        Hr[idx] = v;
        if (j == 0) {
            double s = 0.0;
            if (i >= 6) {
                const int va = (i - 6) / 6, x = (i - 6) % 6;
                for (int fa = var_start[va]; fa < var_start[va + 1]; ++fa) s += b[6LL * var_frames[fa] + x];
            }
            br[i] = s;
        }
    }
}

__global__ void k_boxplus(const double* __restrict__ poses, const double* __restrict__ dx_ff, int n_frames,
                          const int* __restrict__ frame_var, const LmState* st, double* __restrict__ cand) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_frames) return;
    const double* X = poses + 12 * k;
    double* out = cand + 12 * k;
    // pose variable of frame k: frame 0 fixed and frame k -> k - 1 by default; -1 = held fixed
    const int v = frame_var ? frame_var[k] : k - 1;
    if (v < 0 || st->chol_fail) {
        for (int e = 0; e < 12; ++e) out[e] = X[e];
        return;
    }
    const double* dx = dx_ff + 6 * v;
    double qx = dx[3], qy = dx[4], qz = dx[5];
    const double n2 = qx * qx + qy * qy + qz * qz;
    double qw;
    if (n2 < 1.0) {
        qw = sqrt(1.0 - n2);
    } else {
        const double nn = sqrt(1.0 + n2);
        qw = 1.0 / nn;
        qx /= nn;
        qy /= nn;
        qz /= nn;
    }
    const double dR[9] = {1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz),     2 * (qx * qz + qw * qy),
                          2 * (qx * qy + qw * qz),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
                          2 * (qx * qz - qw * qy),     2 * (qy * qz + qw * qx),     1 - 2 * (qx * qx + qy * qy)};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c)
            out[4 * r + c] = X[4 * r] * dR[c] + X[4 * r + 1] * dR[3 + c] + X[4 * r + 2] * dR[6 + c];
        out[4 * r + 3] = X[4 * r] * dx[0] + X[4 * r + 1] * dx[1] + X[4 * r + 2] * dx[2] + X[4 * r + 3];
    }
}

// Keep the candidate when the cost decreased (and the factorisation succeeded).
__global__ void k_accept(LmState* st, double* __restrict__ poses, const double* __restrict__ cand, int n_frames,
                         bool speculative) {
    __shared__ int acc;
    if (threadIdx.x == 0) {
        const bool ok = !st->chol_fail && st->new_cost < st->cost;
        acc = ok ? 1 : 0;
        st->accepted = acc;
        st->status = st->chol_fail ? PBA_ENOTPD : PBA_OK;
        st->lambda = ok ? st->lambda_used * 0.1 : st->lambda_used * 10.0;
        st->iter_cost = st->cost;
        st->iter_n_valid = speculative ? st->n_valid_new : st->n_valid;
        st->iter_nf_res = speculative ? st->nf_res_new : st->nf_res;
        st->iter_nf_pairs = speculative ? st->nf_pairs_new : st->nf_pairs;
        if (ok && speculative) {
            st->cost = st->new_cost;
            st->n_valid = st->n_valid_new;
            st->nf_res = st->nf_res_new;
            st->nf_pairs = st->nf_pairs_new;
        }
    }
    __syncthreads();
    if (acc)
        for (int e = threadIdx.x; e < 12 * n_frames; e += blockDim.x) poses[e] = cand[e];
}

// After an accepted speculative step: the candidate's linearisation becomes current.
__global__ void k_accept_copy(const LmState* st, double* __restrict__ H, const double* __restrict__ H_cand,
                              long long nH, double* __restrict__ b, const double* __restrict__ b_cand, int nb,
                              double* __restrict__ blocks, const double* __restrict__ blocks_cand, long long nblk) {
    if (!st->accepted) return;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    for (long long i = i0; i < nH; i += stride) H[i] = H_cand[i];
    for (long long i = i0; i < nb; i += stride) b[i] = b_cand[i];
    for (long long i = i0; i < nblk; i += stride) blocks[i] = blocks_cand[i];
}

}  // namespace

cudaError_t launch_assemble(const AsmTask* tasks, int n_tasks, const AsmContrib* contrib, const double* blocks,
                            int n_frames, double* H, double* b, cudaStream_t s) {
    if (n_tasks <= 0) return cudaSuccess;
    k_assemble<<<n_tasks, 64, 0, s>>>(tasks, contrib, blocks, 6 * n_frames, H, b);
    return cudaGetLastError();
}

cudaError_t launch_total_cost(const double* blocks, int m, LmState* st, bool candidate, cudaStream_t s) {
    k_total_cost<<<1, 256, 0, s>>>(blocks, m, st, candidate);
    return cudaGetLastError();
}

cudaError_t launch_lm_prepare(const double* H, int n_frames, LmState* st, double explicit_lambda, cudaStream_t s) {
    k_lm_prepare<<<1, 256, 0, s>>>(H, n_frames, st, explicit_lambda);
    return cudaGetLastError();
}

cudaError_t launch_damp(const double* H, const double* b, int n_frames, int n_pad, const LmState* st, double* A,
                        double* rhs, cudaStream_t s) {
    const long long total = (long long)n_pad * n_pad;
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    k_damp<<<grid, 256, 0, s>>>(H, b, n_frames, n_pad, st, A, rhs);
    return cudaGetLastError();
}

cudaError_t launch_cholesky(double* A, double* Dinv, int n_pad, LmState* st, cudaStream_t s, int* n_launches) {
    const int nt = n_pad / kTile;
    const dim3 blk(kTile, kTile);
    const dim3 blk8(kTile, 8);
    int nl = 0;
    for (int k = 0; k < nt; ++k) {
        k_potrf<double><<<1, blk8, 0, s>>>(A, n_pad, k, st, Dinv);
        ++nl;
        const int rest = nt - k - 1;
        if (rest > 0) {
            k_trsm<double><<<rest, blk8, 0, s>>>(A, n_pad, k, st);
            k_syrk<double><<<rest * (rest + 1) / 2, blk, 0, s>>>(A, n_pad, k, nt, st);
            nl += 2;
        }
    }
    if (n_launches) *n_launches = nl;
    return cudaGetLastError();
}

cudaError_t launch_trsv(const double* A, const double* Dinv, int n_pad, double* rhs, const LmState* st,
                        cudaStream_t s) {
    k_trsv<double><<<1, 1024, 0, s>>>(A, Dinv, n_pad, rhs, st);
    return cudaGetLastError();
}

cudaError_t launch_solve_mixed(const double* H, const double* b, int n_frames, int n_pad, LmState* st,
                               MixedWork& w, int refinements, double* dx, cudaStream_t s, int* n_launches) {
    const long long total = (long long)n_pad * n_pad;
    int grid = (int)((total + 255) / 256);
    if (grid > 4096) grid = 4096;
    int nl = 0;
    k_damp_mixed<<<grid, 256, 0, s>>>(H, b, n_frames, n_pad, st, w.A32, w.bs, w.x, w.dscale);
    ++nl;
    const int nt = n_pad / kTile;
    const dim3 blk(kTile, kTile), blk8(kTile, 8);
    for (int k = 0; k < nt; ++k) {
        k_potrf_warp<float><<<1, 32, 0, s>>>(w.A32, n_pad, k, st, w.D32);
        ++nl;
        const int rest = nt - k - 1;
        if (rest > 0) {
            k_trsm<float><<<rest, blk8, 0, s>>>(w.A32, n_pad, k, st);
            k_syrk<float><<<rest * (rest + 1) / 2, blk, 0, s>>>(w.A32, n_pad, k, nt, st);
            nl += 2;
        }
    }
    cudaMemsetAsync(w.norms, 0, 2 * sizeof(double), s);
    const int rgrid = (n_pad + 7) / 8;  // 8 warps per block, one row per warp
    for (int it = 0; it < refinements; ++it) {
        k_refine_residual<<<rgrid, 256, 0, s>>>(H, n_frames, n_pad, st, w.dscale, w.bs, w.x, w.r32, nullptr,
                                                it == 0 ? 1 : 0);
        k_trsv<float><<<1, 1024, 0, s>>>(w.A32, w.D32, n_pad, w.r32, st);
        k_refine_update<<<(n_pad + 255) / 256, 256, 0, s>>>(st, w.r32, w.x, n_pad);
        nl += 3;
    }
    k_refine_residual<<<rgrid, 256, 0, s>>>(H, n_frames, n_pad, st, w.dscale, w.bs, w.x, w.r32, w.norms, 0);
    k_refine_finish<<<1, 256, 0, s>>>(st, w.dscale, w.x, dx, w.norms, n_pad);
    nl += 2;
    if (n_launches) *n_launches = nl;
    return cudaGetLastError();
}

cudaError_t launch_boxplus(const double* poses, const double* dx_ff, int n_frames, const int* frame_var,
                           const LmState* st, double* cand, cudaStream_t s) {
    k_boxplus<<<(n_frames + 127) / 128, 128, 0, s>>>(poses, dx_ff, n_frames, frame_var, st, cand);
    return cudaGetLastError();
}

cudaError_t launch_reduce_vars(const double* H, const double* b, int n_frames, const int* var_start,
                               const int* var_frames, int n_vars, double* Hr, double* br, cudaStream_t s) {
    const long long nr = 6LL * (n_vars + 1);
    const int blocks = (int)std::min<long long>((nr * nr + 255) / 256, 4096);
    k_reduce_vars<<<blocks, 256, 0, s>>>(H, b, n_frames, var_start, var_frames, n_vars, Hr, br);
    return cudaGetLastError();
}

cudaError_t launch_accept(LmState* st, double* poses, const double* cand, int n_frames, bool speculative,
                          double* H, const double* H_cand, double* b, const double* b_cand, double* blocks,
                          const double* blocks_cand, int m, cudaStream_t s) {
    k_accept<<<1, 256, 0, s>>>(st, poses, cand, n_frames, speculative);
    if (speculative) {
        // H == nullptr: no dense system is kept (block-sparse solve), only the pair blocks move
        const long long n6 = H ? 6LL * n_frames : 0;
        const long long nblk = (long long)kBlockStride * m;
        long long most = n6 * n6 > nblk ? n6 * n6 : nblk;
        int grid = (int)((most + 255) / 256);
        if (grid > 1024) grid = 1024;
        k_accept_copy<<<grid, 256, 0, s>>>(st, H, H_cand, n6 * n6, b, b_cand, (int)n6, blocks, blocks_cand, nblk);
    }
    return cudaGetLastError();
}

}  // namespace pba
