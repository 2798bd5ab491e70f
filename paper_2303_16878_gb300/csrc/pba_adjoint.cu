// pba_adjoint.cu -- gradient of the total robust cost F (Eq. total-error-multicue)
// with respect to the poses, the sensor offsets and the cue images.
//
// F is a function of the pose matrices through, per directed pair,
//   pbar = M p_u + a,  nbar = M n^o,  M = R_o^T R_j^T R_i,  a = R_o^T (R_j^T (t_i - t_j) - t_o)
// (Supp., pbar_u and the normal error), of the target images through the
// bilinear samples at u' = pi(pbar), and of the source pixels through g_u,
// p_u = R_o pi^-1(u, d) + t_o and n^o = R_o n_u.  The validity decisions
// (bounds, stencil, occlusion, Huber branch) are held fixed.
//
// k_adjoint recomputes every residual (no Jacobian is stored): stage 1 of the
// linearisation, then, per valid residual,
//   g_p = dF/dpbar = 2 w sum_c Omega_c e_c (d zeta_c / d pbar - grad I_c d pi / d pbar)
//   g_n = dF/dnbar = 2 w Omega_n e_n
// with grad I the exact derivative of the bilinear interpolant (the true
// derivative of F, whatever grad_mode the linearisation uses), and per work
// item the sums  P1 = sum g_p p_u^T,  g_a = sum g_p,  N1 = sum g_n n^o^T,
// Q = sum pbar g_p^T,  Nn = sum nbar g_n^T  (39 floats) plus cost and count.
// Image gradients go straight to the caller's buffer with atomics.  The launch
// is persistent (warps take work items from a counter) with 256-thread blocks
// held to 128 registers so that two blocks share an SM: at the 156 registers
// the compiler takes otherwise, one block (8 warps) per SM left the gathers'
// latency unhidden.
// k_adjoint_pairs turns a pair's FP64 sums into
//   dF/dR_i = R_j R_o G_M,  dF/dt_i = R_j R_o g_a = -dF/dt_j,
//   dF/dR_j = R_i G_M^T R_o^T + (t_i - t_j) g_a^T R_o^T,        G_M = P1 + N1,
//   dF/dR_o = R_o (Q + Nn) + C^T R_o ((P1 - g_a t_o^T) + N1) R_o,
//   dF/dt_o = (C - I)^T R_o g_a,                                 C = R_j^T R_i,
// and k_adjoint_frames / k_adjoint_sensors sum them per frame and per sensor.
#include "pba_device.cuh"
#include "pba_internal.cuh"

namespace pba {
namespace {

constexpr int kAdjThreads = 256;
constexpr int kAdjAcc = 41;        // 39 sums + cost + count
constexpr int kAdjStride = 48;     // floats per work-item partial
constexpr int kAdjPairStride = 40; // doubles per pair: dR_i dt_i dR_j dt_j (24), dR_o dt_o (12), cost, count

template <int TEXEL>
__global__ void __launch_bounds__(kAdjThreads, 2)
    k_adjoint(const int4* __restrict__ chunks, int n_chunks, int* __restrict__ queue, const PairStatic* __restrict__ ps,
              const PairPose* __restrict__ pp, const float4* __restrict__ pts_pg, const float4* __restrict__ pts_n,
              const int* __restrict__ pts_pix, const void* __restrict__ tex, const SensorDev* __restrict__ sensors,
              const int* __restrict__ frame_sensor, const LinParams prm, float* __restrict__ partials,
              float* __restrict__ d_img) {
    const int lane = threadIdx.x & 31;
    const float om[5] = {prm.w_int, prm.w_depth, prm.w_normal, prm.w_normal, prm.w_normal};
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
        const long long pt_off = P.src_pt_offset;
        const SensorDev S = sensors[frame_sensor[P.src]];
        float M[9], av[3];
#pragma unroll
        for (int k = 0; k < 9; ++k) M[k] = pp[pair].M[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) av[k] = pp[pair].a[k];
        const bool wrap = model == 1;
        const void* tex_j = TEXEL == 1 ? (const void*)(reinterpret_cast<const Tex16*>(tex) + P.tgt_px_offset)
                                       : (const void*)(reinterpret_cast<const Tex32*>(tex) + P.tgt_px_offset);
        const float umax = wrap ? 3.4e38f : (float)(W - 2);
        const float umin = wrap ? -3.4e38f : 1.f;
        const float vmax = (float)(Hh - 2);

        float acc[kAdjAcc];
#pragma unroll
        for (int k = 0; k < kAdjAcc; ++k) acc[k] = 0.f;
        const int end = first + count;
        for (int base = first; base < end; base += 32) {
            const int k = base + lane;
            if (k >= end) continue;
            const float4 p = __ldg(pts_pg + pt_off + k);
            const float qx = fmaf(M[0], p.x, fmaf(M[1], p.y, fmaf(M[2], p.z, av[0])));
            const float qy = fmaf(M[3], p.x, fmaf(M[4], p.y, fmaf(M[5], p.z, av[1])));
            const float qz = fmaf(M[6], p.x, fmaf(M[7], p.y, fmaf(M[8], p.z, av[2])));
            float v, zeta_d, fa, rxy2 = 0.f;
            int c0;
            bool ok;
            if (model == 0) {
                ok = qz > prm.z_min;
                const float iz = 1.f / qz;
                const float u = fmaf(fx * qx, iz, cx);
                v = fmaf(fy * qy, iz, cy);
                zeta_d = qz;
                ok = ok && u >= umin && u < umax;
                const float fu = floorf(u);
                c0 = (int)fu;
                fa = u - fu;
            } else {
                rxy2 = fmaf(qx, qx, qy * qy);
                zeta_d = sqrtf(fmaf(qz, qz, rxy2));
                ok = zeta_d > prm.z_min;
                spherical_project(qx, qy, qz, rsqrtf(rxy2), fx, fy, cx, cy, P.fxh, P.fxp, c0, fa, v);
            }
            ok = ok && v >= 1.f && v < vmax;
            if (!ok) continue;
            const float fv = floorf(v);
            const int r0 = (int)fv;
            const float fb = v - fv;
            int cm1, cc, cp1, cp2;
            stencil_cols(c0, W, wrap, cm1, cc, cp1, cp2);
            const int rr0 = r0 * W, rp1 = rr0 + W;
            const Texel A = load_texel<TEXEL>(tex_j, rr0 + cc), B = load_texel<TEXEL>(tex_j, rr0 + cp1);
            const Texel C = load_texel<TEXEL>(tex_j, rp1 + cc), D = load_texel<TEXEL>(tex_j, rp1 + cp1);
            if (!(A.usable && B.usable && C.usable && D.usable)) continue;
            float xa[5], xb[5], xc[5], xd[5], s[5], gu[5], gv[5];
            channels(A, xa);
            channels(B, xb);
            channels(C, xc);
            channels(D, xd);
            const float wA = (1.f - fa) * (1.f - fb), wB = fa * (1.f - fb), wC = (1.f - fa) * fb, wD = fa * fb;
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                s[c] = fmaf(wA, xa[c], fmaf(wB, xb[c], fmaf(wC, xc[c], wD * xd[c])));
                gu[c] = fmaf(1.f - fb, xb[c] - xa[c], fb * (xd[c] - xc[c]));
                gv[c] = fmaf(1.f - fa, xc[c] - xa[c], fa * (xd[c] - xb[c]));
            }
            const float e_d = zeta_d - s[1];
            if (!(fabsf(e_d) <= fmaf(prm.occ_rel, zeta_d, prm.occ_abs))) continue;
            if (!(fmaf(s[2], s[2], fmaf(s[3], s[3], s[4] * s[4])) >= 0.25f)) continue;
            const float4 n = __ldg(pts_n + pt_off + k);
            const float nb[3] = {fmaf(M[0], n.x, fmaf(M[1], n.y, M[2] * n.z)),
                                 fmaf(M[3], n.x, fmaf(M[4], n.y, M[5] * n.z)),
                                 fmaf(M[6], n.x, fmaf(M[7], n.y, M[8] * n.z))};
            float e[5] = {p.w - s[0], e_d, nb[0] - s[2], nb[1] - s[3], nb[2] - s[4]};
            float chi2 = 0.f;
#pragma unroll
            for (int c = 0; c < 5; ++c) chi2 = fmaf(om[c] * e[c], e[c], chi2);
            float w, rho;
            if (chi2 <= prm.huber_delta2) {
                w = 1.f;
                rho = chi2;
            } else {
                const float chi = sqrtf(chi2);
                w = prm.huber_delta / chi;
                rho = fmaf(2.f * prm.huber_delta, chi, -prm.huber_delta2);
            }
            acc[39] += rho;
            acc[40] += 1.f;
            // d pi / d pbar and d zeta^d / d pbar
            float P0[3], P1[3], dz[3];
            if (model == 0) {
                const float iz = 1.f / qz;
                P0[0] = fx * iz; P0[1] = 0.f; P0[2] = -fx * qx * iz * iz;
                P1[0] = 0.f; P1[1] = fy * iz; P1[2] = -fy * qy * iz * iz;
                dz[0] = 0.f; dz[1] = 0.f; dz[2] = 1.f;
            } else {
                const float irxy2 = 1.f / rxy2, rxy = sqrtf(rxy2), ir = 1.f / zeta_d, ir2 = ir * ir;
                P0[0] = -fx * qy * irxy2; P0[1] = fx * qx * irxy2; P0[2] = 0.f;
                const float k1 = -fy * qz * ir2 / rxy;
                P1[0] = k1 * qx; P1[1] = k1 * qy; P1[2] = fy * rxy * ir2;
                dz[0] = qx * ir; dz[1] = qy * ir; dz[2] = qz * ir;
            }
            // g_p = 2 w sum_c Omega_c e_c (d zeta_c / d pbar - grad I_c d pi / d pbar); g_n = 2 w Omega_n e_n
            float gp[3] = {0.f, 0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 5; ++c) {
                const float sc = 2.f * w * om[c] * e[c];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float gj = -fmaf(gu[c], P0[j], gv[c] * P1[j]);
                    if (c == 1) gj += dz[j];
                    gp[j] = fmaf(sc, gj, gp[j]);
                }
            }
            const float gn[3] = {2.f * w * om[2] * e[2], 2.f * w * om[3] * e[3], 2.f * w * om[4] * e[4]};
            const float pu[3] = {p.x, p.y, p.z}, no[3] = {n.x, n.y, n.z}, pb[3] = {qx, qy, qz};
#pragma unroll
            for (int r = 0; r < 3; ++r) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc[3 * r + c] = fmaf(gp[r], pu[c], acc[3 * r + c]);         // P1
                    acc[12 + 3 * r + c] = fmaf(gn[r], no[c], acc[12 + 3 * r + c]); // N1
                    acc[21 + 3 * r + c] = fmaf(pb[r], gp[c], acc[21 + 3 * r + c]); // Q
                    acc[30 + 3 * r + c] = fmaf(nb[r], gn[c], acc[30 + 3 * r + c]); // Nn
                }
                acc[9 + r] += gp[r];  // g_a
            }
            if (d_img) {
                // target: dF/dI_j^c(tap) = -2 w Omega_c e_c (bilinear weight of the tap)
                float* tj = d_img + P.tgt_px_offset * 5;
                const int taps[4] = {rr0 + cc, rr0 + cp1, rp1 + cc, rp1 + cp1};
                const float wt[4] = {wA, wB, wC, wD};
#pragma unroll
                for (int c = 0; c < 5; ++c) {
                    const float sc = -2.f * w * om[c] * e[c];
                    // channel order of the images: g, d, nx, ny, nz
#pragma unroll
                    for (int t = 0; t < 4; ++t) atomicAdd(tj + (long long)taps[t] * 5 + c, sc * wt[t]);
                }
                // source pixel: intensity, depth (p_u = R_o pi^-1(u, d) + t_o), normal (n^o = R_o n)
                float* ti = d_img + (P.src_px_offset + __ldg(pts_pix + pt_off + k)) * 5;
                atomicAdd(ti + 0, 2.f * w * om[0] * e[0]);
                // p_s = R_o^T (p_u - t_o); d = p_s.z (pinhole) or |p_s| (spherical); d pbar / d d = M (p_u - t_o) / d
                const float dp[3] = {p.x - S.t[0], p.y - S.t[1], p.z - S.t[2]};
                float ps[3];
#pragma unroll
                for (int r = 0; r < 3; ++r) ps[r] = S.R[r] * dp[0] + S.R[3 + r] * dp[1] + S.R[6 + r] * dp[2];
                const float dd = model == 0 ? ps[2] : sqrtf(ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
                float gd = 0.f;
#pragma unroll
                for (int r = 0; r < 3; ++r) gd += gp[r] * (M[3 * r] * dp[0] + M[3 * r + 1] * dp[1] + M[3 * r + 2] * dp[2]);
                atomicAdd(ti + 1, gd / dd);
                // dF/dn_s = R_o^T M^T g_n
                float mg[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) mg[c] = M[c] * gn[0] + M[3 + c] * gn[1] + M[6 + c] * gn[2];
#pragma unroll
                for (int r = 0; r < 3; ++r)
                    atomicAdd(ti + 2 + r, S.R[r] * mg[0] + S.R[3 + r] * mg[1] + S.R[6 + r] * mg[2]);
            }
        }
        // warp reduction, one partial per work item
        float mine = 0.f;
#pragma unroll
        for (int j = 0; j < kAdjAcc; ++j) {
            float x = acc[j];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (lane == (j & 31)) {
                if (j < 32) mine = x;
                else partials[(long long)ci * kAdjStride + j] = x;
            }
        }
        partials[(long long)ci * kAdjStride + lane] = mine;
    }
}

// Per pair: FP64 sums of its work items, then the matrix gradients.
constexpr int kAdjSlices = 8;  // slices of a pair's work items summed in parallel

__global__ void k_adjoint_pairs(const float* __restrict__ partials, const PairStatic* __restrict__ ps,
                                const int2* __restrict__ pf, const double* __restrict__ poses,
                                const double* __restrict__ pair_Xo, int m, double* __restrict__ out) {
    const int q = blockIdx.x;
    if (q >= m) return;
    __shared__ double S[kAdjAcc];
    __shared__ double part[kAdjSlices][kAdjAcc];
    const PairStatic P = ps[q];
    // thread (slice, t) sums sum t over its contiguous slice of the pair's work
    // items in order (4 loads in flight); the slices are then added in order
    {
        const int n = P.chunk_end - P.chunk_begin;
        for (int e = threadIdx.x; e < kAdjSlices * kAdjAcc; e += blockDim.x) {
            const int slice = e / kAdjAcc, t = e % kAdjAcc;
            const int c_lo = P.chunk_begin + (int)((long long)n * slice / kAdjSlices);
            const int c_hi = P.chunk_begin + (int)((long long)n * (slice + 1) / kAdjSlices);
            double s = 0.0;
            for (int c0 = c_lo; c0 < c_hi; c0 += 4) {
                float v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = c0 + u < c_hi ? partials[(long long)(c0 + u) * kAdjStride + t] : 0.f;
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (c0 + u < c_hi) s += (double)v[u];
            }
            part[slice][t] = s;
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kAdjAcc; t += blockDim.x) {
        double s = 0.0;
        for (int slice = 0; slice < kAdjSlices; ++slice) s += part[slice][t];
        S[t] = s;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    const int2 ij = pf[q];
    const double* Xi = poses + 12 * ij.x;
    const double* Xj = poses + 12 * ij.y;
    const double* Xo = pair_Xo + 12 * q;
    double Ri[9], Rj[9], Ro[9], ti[3], tj[3], to[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            Ri[3 * r + c] = Xi[4 * r + c];
            Rj[3 * r + c] = Xj[4 * r + c];
            Ro[3 * r + c] = Xo[4 * r + c];
        }
        ti[r] = Xi[4 * r + 3];
        tj[r] = Xj[4 * r + 3];
        to[r] = Xo[4 * r + 3];
    }
    const double* P1 = S;
    const double* ga = S + 9;
    const double* N1 = S + 12;
    const double* Q = S + 21;
    const double* Nn = S + 30;
    double GM[9], RjRo[9], C[9];
    for (int k = 0; k < 9; ++k) GM[k] = P1[k] + N1[k];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 3; ++k) {
                a += Rj[3 * r + k] * Ro[3 * k + c];
                b += Rj[3 * k + r] * Ri[3 * k + c];  // C = R_j^T R_i
            }
            RjRo[3 * r + c] = a;
            C[3 * r + c] = b;
        }
    double* o = out + (long long)q * kAdjPairStride;
    // dR_i = R_j R_o G_M ; dt_i = R_j R_o g_a ; dt_j = -dt_i
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += RjRo[3 * r + k] * GM[3 * k + c];
            o[4 * r + c] = s;
        }
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += RjRo[3 * r + k] * ga[k];
        o[4 * r + 3] = s;
        o[12 + 4 * r + 3] = -s;
    }
    // dR_j = R_i G_M^T R_o^T + (t_i - t_j) g_a^T R_o^T
    double RiGt[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += Ri[3 * r + k] * GM[3 * c + k];
            RiGt[3 * r + c] = s;
        }
    double gaRoT[3];
    for (int c = 0; c < 3; ++c) gaRoT[c] = ga[0] * Ro[3 * c] + ga[1] * Ro[3 * c + 1] + ga[2] * Ro[3 * c + 2];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += RiGt[3 * r + k] * Ro[3 * c + k];
            o[12 + 4 * r + c] = s + (ti[r] - tj[r]) * gaRoT[c];
        }
    // dR_o = R_o (Q + Nn) + C^T R_o ((P1 - g_a t_o^T) + N1) R_o ; dt_o = (C - I)^T R_o g_a
    double QN[9], K[9], CtRo[9];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            QN[3 * r + c] = Q[3 * r + c] + Nn[3 * r + c];
            K[3 * r + c] = P1[3 * r + c] - ga[r] * to[c] + N1[3 * r + c];
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += C[3 * k + r] * Ro[3 * k + c];
            CtRo[3 * r + c] = s;
        }
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < 3; ++k) a += Ro[3 * r + k] * QN[3 * k + c];
            for (int k = 0; k < 3; ++k) {
                double kr = 0.0;
                for (int l = 0; l < 3; ++l) kr += K[3 * k + l] * Ro[3 * l + c];
                b += CtRo[3 * r + k] * kr;
            }
            o[24 + 4 * r + c] = a + b;
        }
    double Rg[3];
    for (int r = 0; r < 3; ++r) Rg[r] = Ro[3 * r] * ga[0] + Ro[3 * r + 1] * ga[1] + Ro[3 * r + 2] * ga[2];
    for (int r = 0; r < 3; ++r) {
        double s = 0.0;
        for (int k = 0; k < 3; ++k) s += (C[3 * k + r] - (k == r ? 1.0 : 0.0)) * Rg[k];
        o[24 + 4 * r + 3] = s;
    }
    o[36] = S[39];
    o[37] = S[40];
}

// Per frame: sum of its pairs' pose gradients (fixed order, from the assembly
// tasks' diagonal contributions: role 0 = source i, role 1 = target j).
__global__ void k_adjoint_frames(const AsmTask* __restrict__ tasks, int n_tasks, const AsmContrib* __restrict__ contrib,
                                 const double* __restrict__ pair_out, double* __restrict__ d_poses) {
    const int t = blockIdx.x;
    if (t >= n_tasks) return;
    const AsmTask T = tasks[t];
    if (T.a != T.b) return;
    const int e = threadIdx.x;
    if (e >= 12) return;
    double s = 0.0;
    for (int k = T.contrib_begin; k < T.contrib_end; ++k) {
        const AsmContrib C = contrib[k];
        if (!C.add_b) continue;
        s += pair_out[(long long)C.pair * kAdjPairStride + 12 * C.row_role + e];
    }
    d_poses[12 * T.a + e] = s;
}

// Per sensor: extrinsic gradient and total cost / count over all pairs (fixed order).
__global__ void k_adjoint_sensors(const PairStatic* __restrict__ ps, const int* __restrict__ frame_sensor, int m,
                                  const double* __restrict__ pair_out, int n_sensors, double* __restrict__ d_ext,
                                  double* __restrict__ totals) {
    const int sensor = blockIdx.x;
    const int e = threadIdx.x;
    if (e < 12) {
        double s = 0.0;
        for (int q = 0; q < m; ++q)
            if (frame_sensor[ps[q].src] == sensor) s += pair_out[(long long)q * kAdjPairStride + 24 + e];
        if (d_ext) d_ext[12 * sensor + e] = s;
    } else if (e < 14 && sensor == 0) {
        double s = 0.0;
        for (int q = 0; q < m; ++q) s += pair_out[(long long)q * kAdjPairStride + 36 + (e - 12)];
        totals[e - 12] = s;
    }
}

}  // namespace

int adjoint_partial_stride() { return kAdjStride; }
int adjoint_pair_stride() { return kAdjPairStride; }

int adjoint_grid(int texel_precision) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &per_sm, texel_precision == 1 ? (const void*)k_adjoint<1> : (const void*)k_adjoint<0>, kAdjThreads, 0);
    return sms * (per_sm < 1 ? 1 : per_sm);
}

cudaError_t launch_adjoint(int texel_precision, const int4* chunks, int n_chunks, int* queue, const PairStatic* ps,
                           const PairPose* pp, const float4* pts_pg, const float4* pts_n, const int* pts_pix,
                           const void* texels, const SensorDev* sensors, const int* frame_sensor,
                           const LinParams& prm, float* partials, float* d_img, int grid, cudaStream_t s) {
    if (n_chunks <= 0) return cudaSuccess;
    if (grid * (kAdjThreads / 32) > n_chunks) grid = (n_chunks + kAdjThreads / 32 - 1) / (kAdjThreads / 32);
    if (texel_precision == 1)
        k_adjoint<1><<<grid, kAdjThreads, 0, s>>>(chunks, n_chunks, queue, ps, pp, pts_pg, pts_n, pts_pix, texels,
                                                  sensors, frame_sensor, prm, partials, d_img);
    else
        k_adjoint<0><<<grid, kAdjThreads, 0, s>>>(chunks, n_chunks, queue, ps, pp, pts_pg, pts_n, pts_pix, texels,
                                                  sensors, frame_sensor, prm, partials, d_img);
    return cudaGetLastError();
}

namespace {

// dF/d dx in the box-plus chart of Supp. (X [+] dx = [R R(dq), R dt + t], R(dq)
// from the unit quaternion with imaginary part dq, so R(dq) = I + 2 [dq]x to
// first order) from the matrix gradient G = dF/dX of a 3x4 transform X:
// d/d dt = R^T G_t and, with W = R^T G_R, d/d dq = 2 (W_zy - W_yz, W_xz - W_zx,
// W_yx - W_xy) (the derivative of tr(G_R^T R 2 [dq]x)).  One thread per transform.
__global__ void k_tangent(const double* __restrict__ X, const double* __restrict__ G, int n, double* __restrict__ g) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double* x = X + 12 * k;
    const double* d = G + 12 * k;
    double W[9];
    for (int r = 0; r < 3; ++r) {
        // (R^T G_t)_r and row r of R^T G_R: sums over the rows a of R and G
        double t = 0.0;
        for (int a = 0; a < 3; ++a) t += x[4 * a + r] * d[4 * a + 3];
        g[6 * k + r] = t;
        for (int c = 0; c < 3; ++c) {
            double w = 0.0;
            for (int a = 0; a < 3; ++a) w += x[4 * a + r] * d[4 * a + c];
            W[3 * r + c] = w;
        }
    }
    g[6 * k + 3] = 2.0 * (W[7] - W[5]);
    g[6 * k + 4] = 2.0 * (W[2] - W[6]);
    g[6 * k + 5] = 2.0 * (W[3] - W[1]);
}

}  // namespace

cudaError_t launch_tangent(const double* X, const double* G, int n, double* g, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_tangent<<<(n + 127) / 128, 128, 0, s>>>(X, G, n, g);
    return cudaGetLastError();
}

cudaError_t launch_adjoint_reduce(const float* partials, const PairStatic* ps, const int2* pf, const double* poses,
                                  const double* pair_Xo, int m, double* pair_out, const AsmTask* tasks, int n_tasks,
                                  const AsmContrib* contrib, const int* frame_sensor, int n_sensors,
                                  double* d_poses, double* d_ext, double* totals, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_adjoint_pairs<<<m, 256, 0, s>>>(partials, ps, pf, poses, pair_Xo, m, pair_out);
    if (d_poses) k_adjoint_frames<<<n_tasks, 32, 0, s>>>(tasks, n_tasks, contrib, pair_out, d_poses);
    k_adjoint_sensors<<<n_sensors, 32, 0, s>>>(ps, frame_sensor, m, pair_out, n_sensors, d_ext, totals);
    return cudaGetLastError();
}

}  // namespace pba
