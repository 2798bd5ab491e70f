// pba_plain.cu -- the plain GPU linearisation: one launch per directed pair.
//
// The straightforward mapping of the method onto a GPU, kept as the reference
// the batched path is measured against: one thread per source pixel, FP32
// interleaved cue images read directly (five scalar loads per texel, validity
// recomputed per texel), the full 5 x 12 Jacobian [J_i J_j] formed from the
// Supp. derivatives of both frames, and the 78 + 12 entries of
// w J^T Omega J, w J^T Omega e (plus cost and count) reduced per block and
// added to the pair's FP32 accumulator with global atomics.  The same
// definitions as the batched path (Eq. pinhole-projection, spherical-projection, uprime, total-error-multicue, Supp.): only the
// organisation of the work differs.
#include "pba_internal.cuh"

namespace pba {

namespace {

constexpr int kPlainThreads = 256;
constexpr int kPlainAcc = 92;      // 78 + 12 + cost + count
constexpr int kPlainStride = 96;

__device__ __forceinline__ bool valid_px(const float* c, float rmin, float rmax) {
    const float n2 = c[2] * c[2] + c[3] * c[3] + c[4] * c[4];
    (void)n2;
    return plain_pixel_valid(c, rmin, rmax);
}

template <bool FULL>
__global__ void __launch_bounds__(kPlainThreads)
    k_plain(int pair, const PairStatic* __restrict__ ps, const PairPose* __restrict__ pp,
            const float* __restrict__ raw, const SensorDev* __restrict__ sensors, int sensor,
            const LinParams prm, float rmin, float rmax, float* __restrict__ acc) {
    __shared__ float s_red[kPlainThreads / 32][kPlainAcc];
    const PairStatic P = ps[pair];
    const PairPose Q = pp[pair];
    const SensorDev S = sensors[sensor];
    const int W = P.width, Hh = P.height;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float om[5] = {prm.w_int, prm.w_depth, prm.w_normal, prm.w_normal, prm.w_normal};

    bool valid = false;
    float e[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, w = 0.f, rho = 0.f;
    float J[5][12];
    if (px < P.src_width * P.src_height) {
        const float* c = raw + (P.src_px_offset + px) * 5;
        float cs[5];
        for (int k = 0; k < 5; ++k) cs[k] = c[k];
        if (valid_px(cs, rmin, rmax)) {
            const int col = px % P.src_width, row = px / P.src_width;
            const float d = cs[1];
            float p[3];
            if (P.model == 0) {
                p[0] = d * ((col - P.cx) / P.fx);
                p[1] = d * ((row - P.cy) / P.fy);
                p[2] = d;
            } else {
                float saz, caz, sel, cel;
                sincosf((col - P.cx) / P.fx, &saz, &caz);
                sincosf((row - P.cy) / P.fy, &sel, &cel);
                p[0] = d * (cel * caz);
                p[1] = d * (cel * saz);
                p[2] = d * sel;
            }
            float pu[3], no[3];
            for (int r = 0; r < 3; ++r) {
                pu[r] = S.R[3 * r] * p[0] + S.R[3 * r + 1] * p[1] + S.R[3 * r + 2] * p[2] + S.t[r];
                no[r] = S.R[3 * r] * cs[2] + S.R[3 * r + 1] * cs[3] + S.R[3 * r + 2] * cs[4];
            }
            float q[3];  // pbar
            for (int r = 0; r < 3; ++r) q[r] = Q.M[3 * r] * pu[0] + Q.M[3 * r + 1] * pu[1] + Q.M[3 * r + 2] * pu[2] + Q.a[r];
            float u, v, zd;
            bool ok;
            if (P.model == 0) {
                ok = q[2] > prm.z_min;
                u = P.fx * q[0] / q[2] + P.cx;
                v = P.fy * q[1] / q[2] + P.cy;
                zd = q[2];
            } else {
                zd = sqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
                ok = zd > prm.z_min;
                u = P.fx * atan2f(q[1], q[0]) + P.cx;
                v = P.fy * atan2f(q[2], sqrtf(q[0] * q[0] + q[1] * q[1])) + P.cy;
            }
            ok = ok && v >= 1.f && v < (float)(Hh - 2);
            if (P.model == 0) ok = ok && u >= 1.f && u < (float)(W - 2);
            if (ok) {
                const int c0 = (int)floorf(u), r0 = (int)floorf(v);
                const float a = u - floorf(u), b = v - floorf(v);
                const float* T = raw + P.tgt_px_offset * 5;
                auto tx = [&](int r, int cc) -> const float* {
                    if (P.model == 1) {
                        cc %= W;
                        if (cc < 0) cc += W;
                    }
                    return T + ((long long)r * W + cc) * 5;
                };
                // 12-texel stencil validity
                const int st[12][2] = {{-1, 0}, {-1, 1}, {0, -1}, {0, 0}, {0, 1}, {0, 2},
                                       {1, -1}, {1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 1}};
                for (int k = 0; k < 12 && ok; ++k) {
                    const float* t = tx(r0 + st[k][0], c0 + st[k][1]);
                    float tc[5] = {t[0], t[1], t[2], t[3], t[4]};
                    ok = valid_px(tc, rmin, rmax);
                }
                if (ok) {
                    const int tr[4] = {0, 0, 1, 1}, tcl[4] = {0, 1, 0, 1};
                    const float wt[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
                    float val[5] = {0, 0, 0, 0, 0}, gu[5] = {0, 0, 0, 0, 0}, gv[5] = {0, 0, 0, 0, 0};
                    for (int t = 0; t < 4; ++t) {
                        const int r = r0 + tr[t], cc = c0 + tcl[t];
                        const float *I = tx(r, cc), *Il = tx(r, cc - 1), *Ir = tx(r, cc + 1), *Iu = tx(r - 1, cc),
                                    *Id = tx(r + 1, cc);
                        for (int ch = 0; ch < 5; ++ch) {
                            val[ch] += wt[t] * I[ch];
                            if (prm.grad_mode == 0) {
                                gu[ch] += wt[t] * 0.5f * (Ir[ch] - Il[ch]);
                                gv[ch] += wt[t] * 0.5f * (Id[ch] - Iu[ch]);
                            }
                        }
                    }
                    if (prm.grad_mode == 1) {
                        for (int ch = 0; ch < 5; ++ch) {
                            const float I00 = tx(r0, c0)[ch], I01 = tx(r0, c0 + 1)[ch];
                            const float I10 = tx(r0 + 1, c0)[ch], I11 = tx(r0 + 1, c0 + 1)[ch];
                            gu[ch] = (1 - b) * (I01 - I00) + b * (I11 - I10);
                            gv[ch] = (1 - a) * (I10 - I00) + a * (I11 - I01);
                        }
                    }
                    float nb[3];  // nbar = M n^o
                    for (int r = 0; r < 3; ++r) nb[r] = Q.M[3 * r] * no[0] + Q.M[3 * r + 1] * no[1] + Q.M[3 * r + 2] * no[2];
                    ok = fabsf(zd - val[1]) <= prm.occ_abs + prm.occ_rel * zd;
                    ok = ok && (val[2] * val[2] + val[3] * val[3] + val[4] * val[4]) >= 0.25f;
                    if (ok) {
                        valid = true;
                        e[0] = cs[0] - val[0];
                        e[1] = zd - val[1];
                        for (int r = 0; r < 3; ++r) e[2 + r] = nb[r] - val[2 + r];
                        float chi2 = 0.f;
                        for (int ch = 0; ch < 5; ++ch) chi2 += om[ch] * e[ch] * e[ch];
                        if (chi2 <= prm.huber_delta2) {
                            w = 1.f;
                            rho = chi2;
                        } else {
                            const float chi = sqrtf(chi2);
                            w = prm.huber_delta / chi;
                            rho = 2.f * prm.huber_delta * chi - prm.huber_delta2;
                        }
                        if (FULL) {
                            // d pi / d pbar
                            float P0[3], P1[3], dz[3];
                            if (P.model == 0) {
                                const float iz = 1.f / q[2];
                                P0[0] = P.fx * iz; P0[1] = 0.f; P0[2] = -P.fx * q[0] * iz * iz;
                                P1[0] = 0.f; P1[1] = P.fy * iz; P1[2] = -P.fy * q[1] * iz * iz;
                                dz[0] = 0.f; dz[1] = 0.f; dz[2] = 1.f;
                            } else {
                                const float rxy2 = q[0] * q[0] + q[1] * q[1], rxy = sqrtf(rxy2);
                                const float r2 = rxy2 + q[2] * q[2];
                                P0[0] = -P.fx * q[1] / rxy2; P0[1] = P.fx * q[0] / rxy2; P0[2] = 0.f;
                                P1[0] = -P.fy * q[0] * q[2] / (rxy * r2);
                                P1[1] = -P.fy * q[1] * q[2] / (rxy * r2);
                                P1[2] = P.fy * rxy / r2;
                                dz[0] = q[0] / zd; dz[1] = q[1] / zd; dz[2] = q[2] / zd;
                            }
                            // q_j = R_j^T (R_i p_u + t_i - t_j) = R_o pbar + t_o ; R_j^T R_i n^o = R_o nbar
                            float qj[3], mj[3];
                            for (int r = 0; r < 3; ++r) {
                                qj[r] = S.R[3 * r] * q[0] + S.R[3 * r + 1] * q[1] + S.R[3 * r + 2] * q[2] + S.t[r];
                                mj[r] = S.R[3 * r] * nb[0] + S.R[3 * r + 1] * nb[1] + S.R[3 * r + 2] * nb[2];
                            }
                            for (int ch = 0; ch < 5; ++ch) {
                                float g[3];
                                for (int k = 0; k < 3; ++k) g[k] = (ch == 1 ? dz[k] : 0.f) - (gu[ch] * P0[k] + gv[ch] * P1[k]);
                                // frame i: g^T M [I | -2 [p_u]x]  -> [h, 2 p_u x h], h = M^T g
                                float h[3], kk[3];
                                for (int k = 0; k < 3; ++k) {
                                    h[k] = Q.M[k] * g[0] + Q.M[3 + k] * g[1] + Q.M[6 + k] * g[2];
                                    kk[k] = S.R[3 * k] * g[0] + S.R[3 * k + 1] * g[1] + S.R[3 * k + 2] * g[2];
                                }
                                J[ch][0] = h[0]; J[ch][1] = h[1]; J[ch][2] = h[2];
                                J[ch][3] = 2.f * (pu[1] * h[2] - pu[2] * h[1]);
                                J[ch][4] = 2.f * (pu[2] * h[0] - pu[0] * h[2]);
                                J[ch][5] = 2.f * (pu[0] * h[1] - pu[1] * h[0]);
                                // frame j: g^T R_o^T [-I | 2 [q_j]x] -> [-k, 2 k x q_j], k = R_o g
                                J[ch][6] = -kk[0]; J[ch][7] = -kk[1]; J[ch][8] = -kk[2];
                                J[ch][9] = 2.f * (kk[1] * qj[2] - kk[2] * qj[1]);
                                J[ch][10] = 2.f * (kk[2] * qj[0] - kk[0] * qj[2]);
                                J[ch][11] = 2.f * (kk[0] * qj[1] - kk[1] * qj[0]);
                                if (ch >= 2) {
                                    const int r = ch - 2;
                                    // d nbar_r / d dq_i = e_r^T M (-2 [n^o]x) = 2 (n^o x m_r)^T
                                    const float mx = Q.M[3 * r], my = Q.M[3 * r + 1], mz = Q.M[3 * r + 2];
                                    J[ch][3] += 2.f * (no[1] * mz - no[2] * my);
                                    J[ch][4] += 2.f * (no[2] * mx - no[0] * mz);
                                    J[ch][5] += 2.f * (no[0] * my - no[1] * mx);
                                    // d nbar_r / d dq_j = e_r^T R_o^T 2 [m_j]x = 2 (c_r x m_j)^T, c_r = column r of R_o
                                    const float cx_ = S.R[r], cy_ = S.R[3 + r], cz_ = S.R[6 + r];
                                    J[ch][9] += 2.f * (cy_ * mj[2] - cz_ * mj[1]);
                                    J[ch][10] += 2.f * (cz_ * mj[0] - cx_ * mj[2]);
                                    J[ch][11] += 2.f * (cx_ * mj[1] - cy_ * mj[0]);
                                }
                            }
                        }
                    }
                }
            }
        }
    }
    // block reduction of the 92 sums, then one atomic per entry and block
    const int kfirst = FULL ? 0 : 90;
    auto put = [&](int k, float x) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[warp][k] = x;
    };
    if (FULL) {
        int k = 0;
#pragma unroll
        for (int a = 0; a < 12; ++a) {
#pragma unroll
            for (int c = a; c < 12; ++c) {
                float x = 0.f;
                if (valid) {
#pragma unroll
                    for (int ch = 0; ch < 5; ++ch) x += w * om[ch] * J[ch][a] * J[ch][c];
                }
                put(k++, x);
            }
        }
#pragma unroll
        for (int a = 0; a < 12; ++a) {
            float x = 0.f;
            if (valid) {
#pragma unroll
                for (int ch = 0; ch < 5; ++ch) x += w * om[ch] * J[ch][a] * e[ch];
            }
            put(78 + a, x);
        }
    }
    put(90, valid ? rho : 0.f);
    put(91, valid ? 1.f : 0.f);
    __syncthreads();
    if ((int)threadIdx.x >= kfirst && threadIdx.x < kPlainAcc) {
        float x = 0.f;
        for (int k = 0; k < kPlainThreads / 32; ++k) x += s_red[k][threadIdx.x];
        atomicAdd(acc + (long long)pair * kPlainStride + threadIdx.x, x);
    }
}

__global__ void k_plain_expand(const float* __restrict__ acc, int m, bool full, double* __restrict__ blocks) {
    const int p = blockIdx.x;
    const float* a = acc + (long long)p * kPlainStride;
    double* out = blocks + (long long)p * kBlockStride;
    const int t = threadIdx.x;
    if (full) {
        if (t < 144) {
            const int r = t / 12, c = t % 12;
            const int lo = r < c ? r : c, hi = r < c ? c : r;
            const int idx = lo * 12 - lo * (lo - 1) / 2 + (hi - lo);
            out[t] = (double)a[idx];
        }
        if (t < 12) out[144 + t] = (double)a[78 + t];
    }
    if (t == 0) {
        out[156] = (double)a[90];
        out[157] = (double)a[91];
        out[158] = 0.0;  // the plain path keeps no status word
        out[159] = 0.0;
    }
}

}  // namespace

cudaError_t launch_plain(bool full, int pair, const PairStatic* ps, const PairPose* pp, const float* raw,
                         const SensorDev* sensors, int src_sensor, const LinParams& prm, double range_min,
                         double range_max, float* acc, int width, int height, cudaStream_t s) {
    const int npx = width * height;
    const int grid = (npx + kPlainThreads - 1) / kPlainThreads;
    float rmin, rmax;
    float_range_limits(range_min, range_max, &rmin, &rmax);
    if (full)
        k_plain<true><<<grid, kPlainThreads, 0, s>>>(pair, ps, pp, raw, sensors, src_sensor, prm, rmin, rmax, acc);
    else
        k_plain<false><<<grid, kPlainThreads, 0, s>>>(pair, ps, pp, raw, sensors, src_sensor, prm, rmin, rmax, acc);
    return cudaGetLastError();
}

cudaError_t launch_plain_expand(const float* acc, int m, bool full, double* blocks, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_plain_expand<<<m, 160, 0, s>>>(acc, m, full, blocks);
    return cudaGetLastError();
}

}  // namespace pba
