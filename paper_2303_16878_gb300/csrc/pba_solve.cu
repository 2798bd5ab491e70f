// pba_solve.cu -- FP64 assembly, damped gauge-fixed Cholesky solve, box-plus
// update and the Levenberg-Marquardt accept / reject, all on the device.
//
// The paper minimises Eq. total-error-multicue with Levenberg-Marquardt (Sec. IV-C, srrg2_solver);
// the normal equations are H = sum w J^T Omega J, b = sum w J^T Omega e over all
// residuals.  Each step solves (H_ff + lambda I) dx_f = -b_f, where _f drops
// frame 0 (gauge freedom), and applies X_k <- X_k [+] dx_k (Supp.):
// X [+] dx = [R R(dq), R dt + t], R(dq) from the unit quaternion (sqrt(1 - |dq|^2), dq).
// The step is kept when the cost decreased (lambda / 10), otherwise the poses
// are restored and lambda grows (x 10).  Double precision throughout.
#include "pba_internal.cuh"
#include "../../include/pba.h"

namespace pba {

namespace {

// ------------------------------------------------------------------ assembly

// One block per task: sums the 6x6 sub-blocks of the contributing pairs in a
// fixed order (deterministic) and writes block (a, b) of H and its transpose;
// diagonal tasks also write b_a.
__global__ void k_assemble(const AsmTask* __restrict__ tasks, const AsmContrib* __restrict__ contrib,
                           const double* __restrict__ blocks, int n6, double* __restrict__ H,
                           double* __restrict__ b) {
    const AsmTask T = tasks[blockIdx.x];
    const int t = threadIdx.x;
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        const bool diag = T.a == T.b;
        if (!diag || r <= c) {
            double s = 0.0;
            for (int k = T.contrib_begin; k < T.contrib_end; ++k) {
                const AsmContrib C = contrib[k];
                s += blocks[(long long)C.pair * kBlockStride + 12 * (6 * C.row_role + r) + 6 * C.col_role + c];
            }
            // diagonal blocks: one sum per unordered entry, mirrored, so H is exactly symmetric
            H[(long long)(6 * T.a + r) * n6 + 6 * T.b + c] = s;
            H[(long long)(6 * T.b + c) * n6 + 6 * T.a + r] = s;
        }
    } else if (t < 42 && T.a == T.b) {
        const int r = t - 36;
        double s = 0.0;
        for (int k = T.contrib_begin; k < T.contrib_end; ++k) {
            const AsmContrib C = contrib[k];
            if (C.add_b) s += blocks[(long long)C.pair * kBlockStride + 144 + 6 * C.row_role + r];
        }
        b[6 * T.a + r] = s;
    }
}

// Sum of the pairs' cost and count (fixed order: strided per thread, then a tree).
__global__ void k_total_cost(const double* __restrict__ blocks, int m, LmState* st, bool candidate) {
    __shared__ double sc[256];
    __shared__ double sn[256];
    double c = 0.0, n = 0.0;
    for (int p = threadIdx.x; p < m; p += blockDim.x) {
        c += blocks[(long long)p * kBlockStride + 156];
        n += blocks[(long long)p * kBlockStride + 157];
    }
    sc[threadIdx.x] = c;
    sn[threadIdx.x] = n;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sc[threadIdx.x] += sc[threadIdx.x + o];
            sn[threadIdx.x] += sn[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (candidate) {
            st->new_cost = sc[0];
            st->n_valid_new = (long long)sn[0];
        } else {
            st->cost = sc[0];
            st->n_valid = (long long)sn[0];
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

__global__ void __launch_bounds__(1024) k_potrf(double* __restrict__ A, int n_pad, int k, LmState* st) {
    if (st->chol_fail) return;
    __shared__ double T[kTile][kTile + 1];
    __shared__ double inv_d;
    __shared__ int fail;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long base = (long long)(k * kTile) * n_pad + k * kTile;
    T[ty][tx] = A[base + (long long)ty * n_pad + tx];
    if (tx == 0 && ty == 0) fail = 0;
    __syncthreads();
    for (int j = 0; j < kTile; ++j) {
        if (tx == j && ty == j) {
            const double v = T[j][j];
            if (!(v > 0.0)) {
                fail = 1;
            } else {
                const double d = sqrt(v);
                T[j][j] = d;
                inv_d = 1.0 / d;
            }
        }
        __syncthreads();
        if (fail) break;
        if (tx == j && ty > j) T[ty][j] *= inv_d;
        __syncthreads();
        if (ty > j && tx > j && tx <= ty) T[ty][tx] -= T[ty][j] * T[tx][j];
        __syncthreads();
    }
    if (fail) {
        if (tx == 0 && ty == 0) st->chol_fail = 1;
        return;
    }
    if (tx <= ty) A[base + (long long)ty * n_pad + tx] = T[ty][tx];
}

// L_ik = A_ik L_kk^{-T} for tiles i > k (one block per tile).
__global__ void __launch_bounds__(1024) k_trsm(double* __restrict__ A, int n_pad, int k, const LmState* st) {
    if (st->chol_fail) return;
    __shared__ double L[kTile][kTile + 1];
    __shared__ double X[kTile][kTile + 1];
    __shared__ double inv[kTile];
    const int i = k + 1 + blockIdx.x;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const long long lk = (long long)(k * kTile) * n_pad + k * kTile;
    const long long ak = (long long)(i * kTile) * n_pad + k * kTile;
    L[ty][tx] = A[lk + (long long)ty * n_pad + tx];
    X[ty][tx] = A[ak + (long long)ty * n_pad + tx];
    if (ty == 0) inv[tx] = 1.0 / A[lk + (long long)tx * n_pad + tx];
    __syncthreads();
    // row ty: x L^T = a  <=>  x[m] = (a[m] - sum_{c<m} x[c] L[m][c]) / L[m][m]
    for (int m = 0; m < kTile; ++m) {
        if (tx == m) X[ty][m] *= inv[m];
        __syncthreads();
        if (tx > m) X[ty][tx] -= X[ty][m] * L[tx][m];
        __syncthreads();
    }
    A[ak + (long long)ty * n_pad + tx] = X[ty][tx];
}

// A_ij -= L_ik L_jk^T for k < j <= i (one block per tile of the trailing lower triangle).
__global__ void __launch_bounds__(1024) k_syrk(double* __restrict__ A, int n_pad, int k, int nt, const LmState* st) {
    if (st->chol_fail) return;
    __shared__ double Li[kTile][kTile + 1];
    __shared__ double Lj[kTile][kTile + 1];
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
    double s = 0.0;
#pragma unroll 8
    for (int m = 0; m < kTile; ++m) s += Li[ty][m] * Lj[tx][m];
    A[(long long)(i * kTile + ty) * n_pad + j * kTile + tx] -= s;
}

// ------------------------------------------------------------------ triangular solves
// One block: L y = rhs, then L^T x = y, tile by tile; x overwrites rhs.
__global__ void __launch_bounds__(1024) k_trsv(const double* __restrict__ A, int n_pad, double* __restrict__ x,
                                               const LmState* st) {
    if (st->chol_fail) return;
    const int nt = n_pad / kTile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // forward
    for (int k = 0; k < nt; ++k) {
        if (warp == 0) {
            double r = x[k * kTile + lane];
            const double dinv = 1.0 / A[(long long)(k * kTile + lane) * n_pad + k * kTile + lane];
            for (int m = 0; m < kTile; ++m) {
                const double ym = __shfl_sync(0xffffffffu, r, m) * __shfl_sync(0xffffffffu, dinv, m);
                if (lane == m) r = ym;
                if (lane > m) r -= A[(long long)(k * kTile + lane) * n_pad + k * kTile + m] * ym;
            }
            x[k * kTile + lane] = r;
        }
        __syncthreads();
        for (int row = (k + 1) * kTile + threadIdx.x; row < n_pad; row += blockDim.x) {
            double s = 0.0;
            for (int m = 0; m < kTile; ++m) s += A[(long long)row * n_pad + k * kTile + m] * x[k * kTile + m];
            x[row] -= s;
        }
        __syncthreads();
    }
    // backward: L^T x = y
    for (int k = nt - 1; k >= 0; --k) {
        if (warp == 0) {
            double r = x[k * kTile + lane];
            const double dinv = 1.0 / A[(long long)(k * kTile + lane) * n_pad + k * kTile + lane];
            for (int m = kTile - 1; m >= 0; --m) {
                const double xm = __shfl_sync(0xffffffffu, r, m) * __shfl_sync(0xffffffffu, dinv, m);
                if (lane == m) r = xm;
                if (lane < m) r -= A[(long long)(k * kTile + m) * n_pad + k * kTile + lane] * xm;
            }
            x[k * kTile + lane] = r;
        }
        __syncthreads();
        for (int row = threadIdx.x; row < k * kTile; row += blockDim.x) {
            double s = 0.0;
            for (int m = 0; m < kTile; ++m) s += A[(long long)(k * kTile + m) * n_pad + row] * x[k * kTile + m];
            x[row] -= s;
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ update
// cand_k = X_k [+] dx_k (dx_0 = 0); on a failed factorisation cand = poses.
__global__ void k_boxplus(const double* __restrict__ poses, const double* __restrict__ dx_ff, int n_frames,
                          const LmState* st, double* __restrict__ cand) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n_frames) return;
    const double* X = poses + 12 * k;
    double* out = cand + 12 * k;
    if (k == 0 || st->chol_fail) {
        for (int e = 0; e < 12; ++e) out[e] = X[e];
        return;
    }
    const double* dx = dx_ff + 6 * (k - 1);
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
__global__ void k_accept(LmState* st, double* __restrict__ poses, const double* __restrict__ cand, int n_frames) {
    __shared__ int acc;
    if (threadIdx.x == 0) {
        const bool ok = !st->chol_fail && st->new_cost < st->cost;
        acc = ok ? 1 : 0;
        st->accepted = acc;
        st->status = st->chol_fail ? PBA_ENOTPD : PBA_OK;
        st->lambda = ok ? st->lambda_used * 0.1 : st->lambda_used * 10.0;
    }
    __syncthreads();
    if (acc)
        for (int e = threadIdx.x; e < 12 * n_frames; e += blockDim.x) poses[e] = cand[e];
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

cudaError_t launch_cholesky(double* A, int n_pad, LmState* st, cudaStream_t s, int* n_launches) {
    const int nt = n_pad / kTile;
    const dim3 blk(kTile, kTile);
    int nl = 0;
    for (int k = 0; k < nt; ++k) {
        k_potrf<<<1, blk, 0, s>>>(A, n_pad, k, st);
        ++nl;
        const int rest = nt - k - 1;
        if (rest > 0) {
            k_trsm<<<rest, blk, 0, s>>>(A, n_pad, k, st);
            k_syrk<<<rest * (rest + 1) / 2, blk, 0, s>>>(A, n_pad, k, nt, st);
            nl += 2;
        }
    }
    if (n_launches) *n_launches = nl;
    return cudaGetLastError();
}

cudaError_t launch_trsv(const double* A, int n_pad, double* rhs, const LmState* st, cudaStream_t s) {
    k_trsv<<<1, 1024, 0, s>>>(A, n_pad, rhs, st);
    return cudaGetLastError();
}

cudaError_t launch_boxplus(const double* poses, const double* dx_ff, int n_frames, const LmState* st, double* cand,
                           cudaStream_t s) {
    k_boxplus<<<(n_frames + 127) / 128, 128, 0, s>>>(poses, dx_ff, n_frames, st, cand);
    return cudaGetLastError();
}

cudaError_t launch_accept(LmState* st, double* poses, const double* cand, int n_frames, cudaStream_t s) {
    k_accept<<<1, 256, 0, s>>>(st, poses, cand, n_frames);
    return cudaGetLastError();
}

}  // namespace pba
