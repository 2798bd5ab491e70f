// pba_solve_cluster.cu -- the mixed-precision damped solve of one Levenberg-
// Marquardt step (Sec. IV-C) in a single launch of one thread-block cluster.
//
// The arithmetic is that of launch_solve_mixed (iterative refinement as in
// LAPACK's dsposv):
//   D = diag(H_ff + lambda I)^-1/2,  A' = D (H_ff + lambda I) D,  b' = -D b_f,
//   L L^T = fl32(A');  x = 0, r = b';
//   `refinements` times: z = (L L^T)^-1 r in FP32, x += z, r = b' - A' x in FP64;
//   dx_f = D x, and the step fails (chol_fail) when a pivot is not positive or
//   the last |r| exceeds kRefineTol |b'|.
// What changes is where it runs.  The FP32 factor is computed in shared memory:
// tile row i (tiles (i, 0..i) of 32 x 32) lives on CTA i mod C of a cluster of
// C <= 16 CTAs, and the steps are separated by cluster barriers instead of
// kernel boundaries.  Finished tiles that other CTAs need (the columns of L
// and the diagonal inverses) are also written to a global scratch copy and
// read from L2, which moves 4 KB tiles several times faster than distributed
// shared memory (measured on GB300: ~29 GB/s of remote shared-memory reads per
// CTA); the short vectors of the triangular solves are pushed through
// distributed shared memory.  The FP64 residual rows are split over the CTAs
// like the tile rows.
//
// Factorisation, right-looking over tile columns with one cluster barrier per
// step p (Dinv_k = L_kk^-1):
//   (a) trailing update by column p-1, deferred from step p-1:
//       A_ij -= L_i,p-1 L_j,p-1^T for p <= j <= i (the owner of row j serves L_j,p-1);
//   (b) L_ip = A_ip Dinv_p^T for the CTA's rows i > p (Dinv_p from its owner);
//   (c) look-ahead on the owner of row p+1: A_p+1,p+1 -= L_p+1,p L_p+1,p^T, then
//       the factorisation and inverse of that diagonal tile, so that step p+1
//       finds Dinv_p+1 ready (that tile is skipped in step p+1's (a)).
// Triangular solves, one cluster barrier per tile row:
//   forward  L y = r:   the owner of row k forms y_k = Dinv_k r_k; after the
//                       barrier every CTA subtracts L_ik y_k from its rows i > k;
//   backward L^T z = y: the owner of row k gathers c_ik = L_ik^T z_i from the
//                       owners of the rows i > k, forms z_k = Dinv_k^T (y_k - sum
//                       c_ik) and its own contributions L_km^T z_k for m < k.
// Every thread of every CTA reaches every cluster barrier (failures are data,
// not early exits), and the last barrier keeps each CTA's shared memory alive
// until the others have finished reading it.
#include <cooperative_groups.h>

#include <mutex>

#include "pba_internal.cuh"
#include "pba_tile.cuh"

namespace pba {

namespace {

namespace cg = cooperative_groups;
using namespace tile;

constexpr int kStage = 4;             // remote tiles staged per round of the trailing update
constexpr int kCsMaxCluster = 16;

__host__ __device__ __forceinline__ int cs_rows(int rank, int nt, int C) {
    return rank < nt ? (nt - 1 - rank) / C + 1 : 0;
}
// slot of tile (row q-th own row, column j) on CTA `rank`: rows before it hold
// rank + C q' + 1 tiles each
__host__ __device__ __forceinline__ int cs_slot(int rank, int C, int q, int j) {
    return q * (rank + 1) + C * q * (q - 1) / 2 + j;
}

// Distributed shared memory through explicit shared::cluster addresses (mapa):
// the address of `p` (this CTA's shared memory) in the CTA of cluster rank `rank`.
__device__ __forceinline__ unsigned dsm_addr(const void* p, int rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;"
                 : "=r"(r)
                 : "r"((unsigned)__cvta_generic_to_shared(p)), "r"(rank));
    return r;
}
__device__ __forceinline__ int dsm_ld_s32(unsigned a) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ void dsm_st(unsigned a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void dsm_st(unsigned a, double v) {
    asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

__global__ void __launch_bounds__(kCsThreads, 1)
    k_solve_cluster(const double* __restrict__ H, const double* __restrict__ b, int n_frames, const CsGeom g,
                    LmState* st, int refinements, double* __restrict__ dx, float* __restrict__ gL,
                    float* __restrict__ gD) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ __align__(16) unsigned char smem[];
    const int rank = (int)cl.block_rank();
    const int C = g.C, nt = g.nt, n_pad = g.n_pad;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* x = reinterpret_cast<double*>(smem + g.o_x);      // full copy of x (FP64)
    double* dsc = reinterpret_cast<double*>(smem + g.o_dsc);  // full copy of D
    double* bsv = reinterpret_cast<double*>(smem + g.o_bs);   // b' of the own rows
    double* rsq = reinterpret_cast<double*>(smem + g.o_rsq);  // r^2 of the own rows (last residual)
    int* flag = reinterpret_cast<int*>(smem + g.o_flag);      // [0] pivot failure
    float* tiles = reinterpret_cast<float*>(smem + g.o_tiles);
    float* dinv = reinterpret_cast<float*>(smem + g.o_dinv);  // Dinv of the own rows
    float* dk = reinterpret_cast<float*>(smem + g.o_dk);      // copy of the current Dinv_p
    float* stage = reinterpret_cast<float*>(smem + g.o_stage);
    float* rv = reinterpret_cast<float*>(smem + g.o_rv);      // r of the own rows (FP32)
    float* yfull = reinterpret_cast<float*>(smem + g.o_yv);   // y, each y_k pushed by its owner
    float* zfull = reinterpret_cast<float*>(smem + g.o_zv);   // z, each z_k pushed by its owner
    float* cbin = reinterpret_cast<float*>(smem + g.o_cb);    // [own row m][source row i][32]: L_im^T z_i, pushed
    float* pv = reinterpret_cast<float*>(smem + g.o_pv);      // pivot column / row exchange of cs_diag
    double* nrmall = reinterpret_cast<double*>(smem + g.o_nrm); // [2][C]: |r|^2 and |b'|^2 of every CTA, pushed
    float* dsc32 = reinterpret_cast<float*>(smem + g.o_dsc32); // D in FP32 (scaling of the FP32 tiles)
    double* xs = reinterpret_cast<double*>(smem + g.o_xs);    // D x (FP64)
    int* conv = flag + 1;                                     // [1] refinement converged

    const int rows = cs_rows(rank, nt, C);
    const int n6 = 6 * n_frames, n = n6 - 6;
    const double lam = st->lambda_used;
    auto own_tile = [&](int q, int j) { return tiles + cs_slot(rank, C, q, j) * kTF; };

    // ---- setup: D, b', x = 0 and the own tiles of A' (padding: identity)
    if (tid == 0) flag[0] = flag[1] = 0;
    for (int i = tid; i < n_pad; i += kCsThreads) {
        // any positive D gives the same solution; it is formed in FP32 and used
        // unchanged (as an FP64 value) everywhere below
        float d = 1.f;
        if (i < n) {
            const float hii = (float)(H[(long long)(i + 6) * n6 + (i + 6)] + lam);
            d = hii > 0.f ? rsqrtf(hii) : 0.f;
        }
        dsc[i] = (double)d;
        dsc32[i] = d;
        x[i] = 0.0;
    }
    __syncthreads();
    for (int q = 0; q < rows; ++q) {
        const int i = rank + C * q;
        if (tid < kT) {
            const int row = kT * i + tid;
            bsv[q * kT + tid] = row < n ? -b[row + 6] * dsc[row] : 0.0;
        }
        // two tiles per round, the 8 loads of a thread in flight together
        for (int j0 = 0; j0 <= i; j0 += 2) {
            double hv[2][kRpt];
#pragma unroll
            for (int t = 0; t < 2; ++t)
#pragma unroll
                for (int h = 0; h < kRpt; ++h) {
                    const int gr = kT * i + warp + kCsWarps * h, gc = kT * (j0 + t) + lane;
                    hv[t][h] = j0 + t <= i && gr < n && gc < n ? H[(long long)(gr + 6) * n6 + (gc + 6)] : 0.0;
                }
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                if (j0 + t > i) break;
                float* T = own_tile(q, j0 + t);
#pragma unroll
                for (int h = 0; h < kRpt; ++h) {
                    const int r = warp + kCsWarps * h, gr = kT * i + r, gc = kT * (j0 + t) + lane;
                    float v;
                    if (gr < n && gc < n) {
                        // the scaling in FP32: fl32(A') only preconditions the FP64 refinement
                        v = (float)(gr == gc ? hv[t][h] + lam : hv[t][h]) * dsc32[gr] * dsc32[gc];
                    } else {
                        v = gr == gc ? 1.f : 0.f;
                    }
                    T[r * kLd + lane] = v;
                }
            }
        }
    }
    __syncthreads();
    if (rank == 0) cs_diag(own_tile(0, 0), dinv, pv, flag, gD);
    cl.sync();

    // ---- factorisation
    for (int p = 0; p < nt; ++p) {
        // (a) trailing update by column p-1
        if (p >= 1) {
            for (int q = 0; q < rows; ++q) {
                const int i = rank + C * q;
                if (i <= p) continue;  // row p's only target (p, p) was done by the look-ahead
                const float* Li = own_tile(q, p - 1);
                for (int j0 = p; j0 <= i; j0 += kStage) {
                    const int nj = min(kStage, i + 1 - j0);
                    // stage the other CTAs' L_j,p-1 from their global copies (L2): thread tid
                    // moves the 16-byte piece (row tid / 8, columns 4 (tid % 8) ..) of each tile
                    const int vr = tid >> 3, vc = 4 * (tid & 7), vo = vr * kLd + vc;
                    float4 v[kStage];
#pragma unroll
                    for (int t = 0; t < kStage; ++t) {
                        const int j = j0 + t;
                        if (t < nj && j % C != rank)
                            v[t] = ld_cg4(gL + (long long)(kT * j + vr) * n_pad + kT * (p - 1) + vc);
                    }
#pragma unroll
                    for (int t = 0; t < kStage; ++t) {
                        const int j = j0 + t;
                        if (t < nj && j % C != rank) *reinterpret_cast<float4*>(stage + t * kTF + vo) = v[t];
                    }
                    __syncthreads();
                    // A_ij[r][c] -= sum_m Li[r][m] Lj[c][m] for the nj targets together: the Li
                    // rows are loaded once per m for all of them (16 independent FMA chains)
                    const float* Lj[kStage];
#pragma unroll
                    for (int t = 0; t < kStage; ++t) {
                        const int j = t < nj ? j0 + t : j0;
                        Lj[t] = (j % C != rank ? stage + t * kTF : own_tile(j / C, p - 1)) + lane * kLd;
                    }
                    float sv[kStage][kRpt];
#pragma unroll
                    for (int t = 0; t < kStage; ++t)
#pragma unroll
                        for (int h = 0; h < kRpt; ++h) sv[t][h] = 0.f;
#pragma unroll
                    for (int m = 0; m < kT; m += 4) {
                        float4 xr[kRpt];
#pragma unroll
                        for (int h = 0; h < kRpt; ++h)
                            xr[h] = *reinterpret_cast<const float4*>(Li + (warp + kCsWarps * h) * kLd + m);
#pragma unroll
                        for (int t = 0; t < kStage; ++t) {
                            if (t < nj) {
                                const float4 y = *reinterpret_cast<const float4*>(Lj[t] + m);
#pragma unroll
                                for (int h = 0; h < kRpt; ++h) sv[t][h] = dot4(xr[h], y, sv[t][h]);
                            }
                        }
                    }
#pragma unroll
                    for (int t = 0; t < kStage; ++t) {
                        if (t < nj) {
                            float* A = own_tile(q, j0 + t);
#pragma unroll
                            for (int h = 0; h < kRpt; ++h) A[(warp + kCsWarps * h) * kLd + lane] -= sv[t][h];
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // (b) L_ip = A_ip Dinv_p^T for the own rows i > p
        bool below = false;
        for (int q = 0; q < rows; ++q) below = below || rank + C * q > p;
        if (below) {
            const float* Dp;
            if (p % C == rank) {
                Dp = dinv + (p / C) * kTF;
            } else {
                const int vr = tid >> 3, vc = 4 * (tid & 7);
                *reinterpret_cast<float4*>(dk + vr * kLd + vc) = ld_cg4(gD + p * kT * kT + vr * kT + vc);
                __syncthreads();
                Dp = dk;
            }
            for (int q = 0; q < rows; ++q) {
                if (rank + C * q <= p) continue;
                float* A = own_tile(q, p);
                float sv[kRpt];
                tile_rows_dot(A, Dp, sv);
                __syncwarp();  // a warp reads and writes only its own rows of A
                const int i = rank + C * q;
#pragma unroll
                for (int h = 0; h < kRpt; ++h) {
                    A[(warp + kCsWarps * h) * kLd + lane] = sv[h];
                    gL[(long long)(kT * i + warp + kCsWarps * h) * n_pad + kT * p + lane] = sv[h];
                }
                __syncwarp();
            }
        }
        // (c) look-ahead: the next diagonal tile
        if (p + 1 < nt && (p + 1) % C == rank) {
            __syncthreads();  // L_p+1,p from (b) was written row by row by all warps
            const int q = (p + 1) / C;
            const float* Lp = own_tile(q, p);
            float* A = own_tile(q, p + 1);
            float sv[kRpt];
            tile_rows_dot(Lp, Lp, sv);
#pragma unroll
            for (int h = 0; h < kRpt; ++h) A[(warp + kCsWarps * h) * kLd + lane] -= sv[h];
            __syncthreads();
            cs_diag(A, dinv + q * kTF, pv, flag, gD + (p + 1) * kT * kT);
        }
        cl.sync();
    }

    // ---- iterative refinement (results are pushed into the consumers' shared
    // memory before each barrier, so that every read after it is local)
    if (tid == 0) {
        double c = 0.0;
        for (int q = 0; q < rows; ++q)
            for (int rr = 0; rr < kT; ++rr) c += bsv[q * kT + rr] * bsv[q * kT + rr];
        for (int k = 0; k < C; ++k) dsm_st(dsm_addr(nrmall + C + rank, k), c);
    }
    for (int it = 0; it <= refinements; ++it) {
        // r = b' - A' x (FP64) for the own rows, A' x = D ((H_ff + lambda I) (D x)); x = 0 on the first pass
        if (it > 0) {
            for (int i = tid; i < n_pad; i += kCsThreads) xs[i] = dsc[i] * x[i];
            __syncthreads();
        }
        for (int q = 0; q < rows; ++q) {
            const int i = rank + C * q;
            double sv[kRpt];
#pragma unroll
            for (int h = 0; h < kRpt; ++h) sv[h] = 0.0;
            if (it > 0) {
                // rows warp + 8 h: s_h = sum_j H_row,j (D x)_j, the loads of the kRpt rows interleaved
                for (int j = lane; j < n; j += 32) {
                    const double xj = xs[j];
#pragma unroll
                    for (int h = 0; h < kRpt; ++h) {
                        const int row = kT * i + warp + kCsWarps * h;
                        if (row < n) sv[h] = fma(H[(long long)(row + 6) * n6 + 6 + j], xj, sv[h]);
                    }
                }
#pragma unroll
                for (int h = 0; h < kRpt; ++h)
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) sv[h] += __shfl_xor_sync(0xffffffffu, sv[h], o);
            }
#pragma unroll
            for (int h = 0; h < kRpt; ++h) {
                const int rr = warp + kCsWarps * h, row = kT * i + rr;
                double r = bsv[q * kT + rr];
                if (it > 0) r -= row < n ? dsc[row] * fma(lam, xs[row], sv[h]) : x[row];  // identity padding
                if (lane == 0) {
                    rv[q * kT + rr] = (float)r;
                    rsq[q * kT + rr] = r * r;
                }
            }
        }
        __syncthreads();
        if (it == refinements) {
            // |r|^2 over the cluster in a fixed order: every CTA takes the same decision
            if (tid == 0) {
                double a = 0.0;
                for (int q = 0; q < rows; ++q)
                    for (int rr = 0; rr < kT; ++rr) a += rsq[q * kT + rr];
                for (int k = 0; k < C; ++k) dsm_st(dsm_addr(nrmall + rank, k), a);
            }
            cl.sync();
            if (tid == 0) {
                double a = 0.0, c = 0.0;
                for (int k = 0; k < C; ++k) {
                    a += nrmall[k];
                    c += nrmall[C + k];
                }
                conv[0] = a <= kRefineTol * kRefineTol * c || c == 0.0;
            }
            __syncthreads();
            break;
        }

        // forward: L y = r
        for (int k = 0; k < nt; ++k) {
            if (k % C == rank && warp == 0) {
                const int q = k / C;
                const float* D = dinv + q * kTF;
                const float* r = rv + q * kT;
                float s0 = 0.f, s1 = 0.f;
#pragma unroll
                for (int m = 0; m < kT; m += 8) {
                    s0 = dot4(*reinterpret_cast<const float4*>(D + lane * kLd + m),
                              *reinterpret_cast<const float4*>(r + m), s0);
                    s1 = dot4(*reinterpret_cast<const float4*>(D + lane * kLd + m + 4),
                              *reinterpret_cast<const float4*>(r + m + 4), s1);
                }
                const float y = s0 + s1;
                for (int d = 0; d < C; ++d) dsm_st(dsm_addr(yfull + k * kT + lane, d), y);
            }
            cl.sync();
            if (warp < rows) {
                const int q = warp, i = rank + C * q;
                if (i > k) {
                    const float* L = own_tile(q, k);
                    const float* y = yfull + k * kT;
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int m = 0; m < kT; m += 8) {
                        s0 = dot4(*reinterpret_cast<const float4*>(L + lane * kLd + m),
                                  *reinterpret_cast<const float4*>(y + m), s0);
                        s1 = dot4(*reinterpret_cast<const float4*>(L + lane * kLd + m + 4),
                                  *reinterpret_cast<const float4*>(y + m + 4), s1);
                    }
                    rv[q * kT + lane] -= s0 + s1;
                }
            }
            __syncthreads();
        }
        // backward: L^T z = y
        for (int k = nt - 1; k >= 0; --k) {
            if (k % C == rank) {
                const int q = k / C;
                if (warp == 0) {
                    float s = 0.f;
                    for (int i = k + 1; i < nt; ++i) s += cbin[(q * nt + i) * kT + lane];
                    // t goes through shared memory (the row's residual slot is free
                    // during the backward sweep) so that it is read back as broadcasts
                    float* tt = rv + q * kT;
                    tt[lane] = yfull[k * kT + lane] - s;
                    __syncwarp();
                    const float* D = dinv + q * kTF;
                    float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;
#pragma unroll
                    for (int m = 0; m < kT; m += 4) {
                        const float4 t4 = *reinterpret_cast<const float4*>(tt + m);
                        z0 = fmaf(D[m * kLd + lane], t4.x, z0);
                        z1 = fmaf(D[(m + 1) * kLd + lane], t4.y, z1);
                        z2 = fmaf(D[(m + 2) * kLd + lane], t4.z, z2);
                        z3 = fmaf(D[(m + 3) * kLd + lane], t4.w, z3);
                    }
                    const float z = (z0 + z1) + (z2 + z3);
                    for (int d = 0; d < C; ++d) dsm_st(dsm_addr(zfull + k * kT + lane, d), z);
                }
                __syncthreads();
                // contributions L_km^T z_k to the rows m < k, pushed to their owners
                for (int m = warp; m < k; m += kCsWarps) {
                    const float* L = own_tile(q, m);
                    const float* z = zfull + k * kT;
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
                    for (int r = 0; r < kT; r += 4) {
                        const float4 z4 = *reinterpret_cast<const float4*>(z + r);
                        s0 = fmaf(L[r * kLd + lane], z4.x, s0);
                        s1 = fmaf(L[(r + 1) * kLd + lane], z4.y, s1);
                        s2 = fmaf(L[(r + 2) * kLd + lane], z4.z, s2);
                        s3 = fmaf(L[(r + 3) * kLd + lane], z4.w, s3);
                    }
                    dsm_st(dsm_addr(cbin + ((m / C) * nt + k) * kT + lane, m % C), (s0 + s1) + (s2 + s3));
                }
            }
            cl.sync();
        }
        // x += z
        for (int row = tid; row < n_pad; row += kCsThreads) x[row] += (double)zfull[row];
        __syncthreads();
    }

    // ---- dx_f = D x for the own rows; failure: a pivot, or no convergence
    for (int q = 0; q < rows; ++q) {
        const int i = rank + C * q;
        if (tid < kT) {
            const int row = kT * i + tid;
            dx[row] = dsc[row] * x[row];
        }
    }
    cl.sync();
    if (rank == 0 && tid == 0) {
        int bad = 0;
        for (int k = 0; k < C; ++k) bad |= dsm_ld_s32(dsm_addr(flag, k));
        if (bad || !conv[0]) st->chol_fail = 1;
    }
    cl.sync();
}

// per device: largest usable cluster size (-1: not queried yet, 0: none) and
// the opt-in shared memory per block
constexpr int kCsMaxDevices = 64;
int g_cs_cmax[kCsMaxDevices];
int g_cs_smem_max[kCsMaxDevices];
bool g_cs_init_done = false;
std::mutex g_cs_mutex;  // problems may be created from several host threads

}  // namespace

bool solve_cluster_init() {
    std::lock_guard<std::mutex> lock(g_cs_mutex);
    if (!g_cs_init_done) {
        for (int d = 0; d < kCsMaxDevices; ++d) g_cs_cmax[d] = -1;
        g_cs_init_done = true;
    }
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kCsMaxDevices) return false;
    int& cmax = g_cs_cmax[dev];
    if (cmax >= 0) return cmax > 0;
    cmax = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    if (cudaFuncSetAttribute(k_solve_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess ||
        cudaFuncSetAttribute(k_solve_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    for (int c = kCsMaxCluster; c >= 1; c /= 2) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = c;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.gridDim = dim3(c);
        cfg.blockDim = dim3(kCsThreads);
        cfg.dynamicSmemBytes = optin;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, k_solve_cluster, &cfg) == cudaSuccess && clusters > 0) {
            cmax = c;
            break;
        }
        cudaGetLastError();
    }
    g_cs_smem_max[dev] = optin;
    return cmax > 0;
}

bool solve_cluster_plan(int n_pad, CsGeom* g) {
    if (!solve_cluster_init() || n_pad <= 0 || n_pad % kT) return false;
    int dev = 0;
    cudaGetDevice(&dev);
    int cmax, smem_max;
    {
        std::lock_guard<std::mutex> lock(g_cs_mutex);
        cmax = g_cs_cmax[dev];
        smem_max = g_cs_smem_max[dev];
    }
    const int nt = n_pad / kT;
    const int C = nt < cmax ? nt : cmax;
    const int R = cs_rows(0, nt, C);
    int slots = 0;
    for (int r = 0; r < C; ++r) {
        const int rows = cs_rows(r, nt, C);
        const int s = rows * (r + 1) + C * rows * (rows - 1) / 2;
        slots = s > slots ? s : slots;
    }
    auto al = [](long long v) { return (v + 15) / 16 * 16; };
    long long o = 0;
    CsGeom h{};
    h.nt = nt;
    h.C = C;
    h.n_pad = n_pad;
    h.o_x = (int)o;
    o = al(o + 8LL * n_pad);
    h.o_dsc = (int)o;
    o = al(o + 8LL * n_pad);
    h.o_xs = (int)o;
    o = al(o + 8LL * n_pad);
    h.o_bs = (int)o;
    o = al(o + 8LL * R * kT);
    h.o_rsq = (int)o;
    o = al(o + 8LL * R * kT);
    h.o_nrm = (int)o;
    o = al(o + 16LL * C);
    h.o_flag = (int)o;
    o = al(o + 16);
    h.o_tiles = (int)o;
    o = al(o + 4LL * slots * kTF);
    h.o_dinv = (int)o;
    o = al(o + 4LL * R * kTF);
    h.o_dk = (int)o;
    o = al(o + 4LL * kTF);
    h.o_stage = (int)o;
    o = al(o + 4LL * kStage * kTF);
    h.o_rv = (int)o;
    o = al(o + 4LL * R * kT);
    h.o_yv = (int)o;
    o = al(o + 4LL * n_pad);
    h.o_zv = (int)o;
    o = al(o + 4LL * n_pad);
    h.o_cb = (int)o;
    o = al(o + 4LL * R * nt * kT);
    h.o_pv = (int)o;
    o = al(o + 4LL * 4 * kT);
    h.o_dsc32 = (int)o;
    o = al(o + 4LL * n_pad);
    if (o > smem_max) return false;
    h.bytes = (int)o;
    *g = h;
    return true;
}

cudaError_t launch_solve_cluster(const double* H, const double* b, int n_frames, const CsGeom& g, LmState* st,
                                 int refinements, double* dx, float* gL, float* gD, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(g.C);
    cfg.blockDim = dim3(kCsThreads);
    cfg.dynamicSmemBytes = g.bytes;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve_cluster, H, b, n_frames, g, st, refinements < 1 ? 1 : refinements, dx, gL,
                              gD);
}

}  // namespace pba
