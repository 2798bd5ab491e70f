// pba_offset.cu -- sensor offsets X_o as variables of the damped solve.
//
// The paper holds X_o fixed (Supp., offset form); refining it uses the first-
// order identity of the offset Jacobian: right-perturbing X_o by exp(d) acts on
// pbar = X_o^-1 X_j^-1 X_i X_o pi^-1(u, d) like right-perturbing both X_i and
// X_j by X_o exp(d) X_o^-1, so J_o = (J_i + J_j) A_o with
// A_o = [[R_o, 2 [t_o]x R_o], [0, R_o]] in the [dt, dq] coordinates.  The
// offset blocks of a pair therefore follow from its H12 / b12 in FP64:
//   H_io = (H_ii + H_ij) A_o,  H_jo = (H_ji + H_jj) A_o,
//   H_oo = A_o^T (H_ii + H_ij + H_ji + H_jj) A_o,  b_o = A_o^T (b_i + b_j).
#include "pba_internal.cuh"

namespace pba {
namespace {

// A_o (row-major 6 x 6) of a 3x4 offset.
__device__ void offset_map(const double* __restrict__ X, double A[36]) {
    for (int k = 0; k < 36; ++k) A[k] = 0.0;
    const double t0 = X[3], t1 = X[7], t2 = X[11];
    for (int c = 0; c < 3; ++c) {
        const double r0 = X[c], r1 = X[4 + c], r2 = X[8 + c];  // column c of R_o
        const double x[3] = {t1 * r2 - t2 * r1, t2 * r0 - t0 * r2, t0 * r1 - t1 * r0};
        const double col[3] = {r0, r1, r2};
        for (int r = 0; r < 3; ++r) {
            A[6 * r + c] = col[r];
            A[6 * r + 3 + c] = 2.0 * x[r];
            A[6 * (3 + r) + 3 + c] = col[r];
        }
    }
}

// One block of 64 threads per pair: out (114 per pair) = [H_io, H_jo, H_oo, b_o].
__global__ void k_pair_offset(const double* __restrict__ blocks, const double* __restrict__ pair_Xo, int m,
                              double* __restrict__ out) {
    const int q = blockIdx.x;
    if (q >= m) return;
    __shared__ double A[36], Si[36], Sj[36], P[36], bs[6];
    const double* B = blocks + (long long)q * kBlockStride;
    const int t = threadIdx.x;
    if (t == 0) offset_map(pair_Xo + 12LL * q, A);
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        // Si = H_ii + H_ij (rows of i), Sj = H_ji + H_jj (rows of j)
        Si[t] = B[12 * r + c] + B[12 * r + 6 + c];
        Sj[t] = B[12 * (6 + r) + c] + B[12 * (6 + r) + 6 + c];
    } else if (t < 42) {
        bs[t - 36] = B[144 + (t - 36)] + B[150 + (t - 36)];
    }
    __syncthreads();
    double* o = out + 114LL * q;
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        double hi = 0.0, hj = 0.0;
        for (int k = 0; k < 6; ++k) {
            hi += Si[6 * r + k] * A[6 * k + c];
            hj += Sj[6 * r + k] * A[6 * k + c];
        }
        o[t] = hi;
        o[36 + t] = hj;
        P[t] = hi + hj;  // (H_ii + H_ij + H_ji + H_jj) A_o
    }
    __syncthreads();
    if (t < 36) {
        const int r = t / 6, c = t % 6;
        // H_oo = A^T P, computed on the upper triangle and mirrored (exactly symmetric)
        if (r <= c) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += A[6 * k + r] * P[6 * k + c];
            o[72 + 6 * r + c] = s;
            o[72 + 6 * c + r] = s;
        }
    } else if (t < 42) {
        const int r = t - 36;
        double s = 0.0;
        for (int k = 0; k < 6; ++k) s += A[6 * k + r] * bs[k];
        o[108 + r] = s;
    }
}

// Blocks [0, N): Hfo[f] = sum over the pairs touching frame f (its sensor's
// offset, when free) of H_io or H_jo by the frame's role; blocks [N, N + S):
// Hoo[s], bo[s] over the pairs of sensor s.  Fixed order: deterministic.
__global__ void k_assemble_offset(const double* __restrict__ pext, const int* __restrict__ f_start,
                                  const int2* __restrict__ f_items, const int* __restrict__ s_start,
                                  const int* __restrict__ s_items, const int* __restrict__ frame_sensor,
                                  const int* __restrict__ sensor_var, int n_frames, double* __restrict__ Hfo,
                                  double* __restrict__ Hoo, double* __restrict__ bo) {
    const int blk = blockIdx.x, t = threadIdx.x;
    if (blk < n_frames) {
        if (t >= 36) return;
        double s = 0.0;
        if (sensor_var[frame_sensor[blk]] >= 0)
            for (int k = f_start[blk]; k < f_start[blk + 1]; ++k) {
                const int2 it = f_items[k];  // (pair, role)
                s += pext[114LL * it.x + 36 * it.y + t];
            }
        Hfo[36LL * blk + t] = s;
    } else {
        const int sn = blk - n_frames;
        if (t >= 42) return;
        double s = 0.0;
        if (sensor_var[sn] >= 0)
            for (int k = s_start[sn]; k < s_start[sn + 1]; ++k) s += pext[114LL * s_items[k] + 72 + t];
        if (t < 36) Hoo[36LL * sn + t] = s;
        else bo[6LL * sn + (t - 36)] = s;
    }
}

// Hr = S^T H S, br = S^T b over frame blocks [0, N) and offset blocks [N, N + S)
// (leading fixed dummy block); the H of an offset with a frame is Hfo of that
// frame when the offset belongs to the frame's sensor, else zero.  Both
// triangles sum the same terms in the same order.
__device__ __forceinline__ double h_full(const double* __restrict__ H, long long n6, const double* __restrict__ Hfo,
                                         const double* __restrict__ Hoo, const int* __restrict__ frame_sensor,
                                         int n_frames, int A, int x, int B, int y) {
    if (A < n_frames && B < n_frames) return H[(6LL * A + x) * n6 + 6LL * B + y];
    if (A < n_frames) return frame_sensor[A] == B - n_frames ? Hfo[36LL * A + 6 * x + y] : 0.0;
    if (B < n_frames) return frame_sensor[B] == A - n_frames ? Hfo[36LL * B + 6 * y + x] : 0.0;
    return A == B ? Hoo[36LL * (A - n_frames) + 6 * x + y] : 0.0;
}

__global__ void k_reduce_vars_offset(const double* __restrict__ H, const double* __restrict__ b,
                                     const double* __restrict__ Hfo, const double* __restrict__ Hoo,
                                     const double* __restrict__ bo, const int* __restrict__ frame_sensor,
                                     int n_frames, const int* __restrict__ var_start,
                                     const int* __restrict__ var_blocks, int n_vars, double* __restrict__ Hr,
                                     double* __restrict__ br) {
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
            for (int fa = var_start[va]; fa < var_start[va + 1]; ++fa)
                for (int gb = var_start[vb]; gb < var_start[vb + 1]; ++gb)
                    v += h_full(H, n6, Hfo, Hoo, frame_sensor, n_frames, var_blocks[fa], x, var_blocks[gb], y);
        }
        Hr[idx] = v;
        if (j == 0) {
            double s = 0.0;
            if (i >= 6) {
                const int va = (i - 6) / 6, x = (i - 6) % 6;
                for (int fa = var_start[va]; fa < var_start[va + 1]; ++fa) {
                    const int B = var_blocks[fa];
                    s += B < n_frames ? b[6LL * B + x] : bo[6LL * (B - n_frames) + x];
                }
            }
            br[i] = s;
        }
    }
}

// Candidate offsets: X_o [+] dx of the offset's variable (Supp. box-plus), else a copy.
__global__ void k_boxplus_offset(const double* __restrict__ extr, const double* __restrict__ dx,
                                 const int* __restrict__ sensor_var, int n_sensors, const LmState* st,
                                 double* __restrict__ cand) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n_sensors) return;
    const double* X = extr + 12 * s;
    double* out = cand + 12 * s;
    const int v = sensor_var[s];
    if (v < 0 || st->chol_fail) {
        for (int e = 0; e < 12; ++e) out[e] = X[e];
        return;
    }
    const double* d = dx + 6 * v;
    double qx = d[3], qy = d[4], qz = d[5];
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
        out[4 * r + 3] = X[4 * r] * d[0] + X[4 * r + 1] * d[1] + X[4 * r + 2] * d[2] + X[4 * r + 3];
    }
}

// After the accept decision: the candidate offsets become current when the step was taken.
__global__ void k_accept_offset(const LmState* st, double* __restrict__ extr, const double* __restrict__ cand,
                                int n) {
    if (!st->accepted) return;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 12 * n; e += gridDim.x * blockDim.x) extr[e] = cand[e];
}

// The offsets' copies used by the kernels: per pair (FP64, the source frame's
// sensor) and per sensor (FP32 R_o, t_o for the pixel-point builder).
__global__ void k_refresh_offset(const double* __restrict__ extr, int n_sensors, const int2* __restrict__ pf,
                                 const int* __restrict__ frame_sensor, int m, double* __restrict__ pair_Xo,
                                 SensorDev* __restrict__ sensors) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) {
        const double* X = extr + 12 * frame_sensor[pf[k].x];
        for (int e = 0; e < 12; ++e) pair_Xo[12LL * k + e] = X[e];
    }
    if (k < n_sensors) {
        const double* X = extr + 12 * k;
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) sensors[k].R[3 * r + c] = (float)X[4 * r + c];
            sensors[k].t[r] = (float)X[4 * r + 3];
        }
    }
}

}  // namespace

cudaError_t launch_offset_system(const double* blocks, const double* pair_Xo, int m, double* pext,
                                 const int* f_start, const int2* f_items, const int* s_start, const int* s_items,
                                 const int* frame_sensor, const int* sensor_var, int n_frames, int n_sensors,
                                 double* Hfo, double* Hoo, double* bo, cudaStream_t s) {
    if (m > 0) k_pair_offset<<<m, 64, 0, s>>>(blocks, pair_Xo, m, pext);
    k_assemble_offset<<<n_frames + n_sensors, 64, 0, s>>>(pext, f_start, f_items, s_start, s_items, frame_sensor,
                                                         sensor_var, n_frames, Hfo, Hoo, bo);
    return cudaGetLastError();
}

cudaError_t launch_reduce_vars_offset(const double* H, const double* b, const double* Hfo, const double* Hoo,
                                      const double* bo, const int* frame_sensor, int n_frames, const int* var_start,
                                      const int* var_blocks, int n_vars, double* Hr, double* br, cudaStream_t s) {
    const long long nr = 6LL * (n_vars + 1);
    const int blocks = (int)((nr * nr + 255) / 256 < 4096 ? (nr * nr + 255) / 256 : 4096);
    k_reduce_vars_offset<<<blocks, 256, 0, s>>>(H, b, Hfo, Hoo, bo, frame_sensor, n_frames, var_start, var_blocks,
                                                n_vars, Hr, br);
    return cudaGetLastError();
}

cudaError_t launch_offset_step(const double* extr, const double* dx, const int* sensor_var, int n_sensors,
                               const LmState* st, double* cand, cudaStream_t s) {
    k_boxplus_offset<<<(n_sensors + 63) / 64, 64, 0, s>>>(extr, dx, sensor_var, n_sensors, st, cand);
    return cudaGetLastError();
}

cudaError_t launch_offset_accept(const LmState* st, double* extr, const double* cand, int n_sensors,
                                 cudaStream_t s) {
    k_accept_offset<<<1, 128, 0, s>>>(st, extr, cand, n_sensors);
    return cudaGetLastError();
}

cudaError_t launch_offset_refresh(const double* extr, int n_sensors, const int2* pf, const int* frame_sensor, int m,
                                  double* pair_Xo, SensorDev* sensors, cudaStream_t s) {
    const int n = m > n_sensors ? m : n_sensors;
    k_refresh_offset<<<(n + 127) / 128, 128, 0, s>>>(extr, n_sensors, pf, frame_sensor, m, pair_Xo, sensors);
    return cudaGetLastError();
}

}  // namespace pba
