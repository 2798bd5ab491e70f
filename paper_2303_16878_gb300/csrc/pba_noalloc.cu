// pba_noalloc.cu -- pba_linearize_pairs_noalloc: a linearisation entry point
// that allocates no memory, for callers that cannot call cudaMalloc.
//
// Who needs it: code that only receives device buffers from its host and may
// not allocate (plugins of frameworks that own the device memory pool), and
// loops with a fixed memory budget decided at start-up, where a cudaMalloc
// could fail or stall the device at the wrong moment.  The caller passes the
// inputs (cue images, poses, pairs) and the output buffer; the working memory
// is a fixed-size array in the library's own device memory.
//
// The scratch: `g_noalloc_scratch` below, PBA_NOALLOC_SCRATCH_BYTES per GPU
// that loads the library, held until the process exits.  It holds, per pair,
// the FP32 accumulators of the plain linearisation (78 + 12 sums), an FP64
// cost and an exact integer count, the pair's static data and its FP32
// transform.  Host code never dereferences the symbol: on every call the host
// looks up its device address on the current device with cudaGetSymbolAddress
// and passes that pointer to the kernels.  Every call reuses the same array:
// each call zeroes the accumulators it uses before the kernels run, and calls
// whose device work overlaps (several streams, several threads) race on it.
//
// The kernel is a variant of the plain path's k_plain (pba_plain.cu): one
// thread per source pixel, FP32 cue images read directly, the full 5 x 12
// Jacobian [J_i J_j] from the Supp. derivatives, block reduction and FP32
// atomics into the pair's accumulator (the cost in FP64, the count as an
// integer); here every pair runs in one launch (blockIdx.y = pair).  The
// results match pba_get_pair_system of a plain-path problem on the same inputs
// within the parity tolerances (not bit for bit: the pair transform is formed
// in another order and the atomics sum in no fixed order).
#include "../../include/pba.h"
#include "pba_internal.cuh"

namespace pba {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaAcc = 92;     // 78 + 12 + cost + count
constexpr int kNaStride = 96;

struct NaPair {
    int src, tgt;
    float M[9];
    float a[3];
};

struct NaScratch {
    float acc[PBA_NOALLOC_MAX_PAIRS][kNaStride];  // 78 + 12 FP32 sums (H upper, b)
    double cost[PBA_NOALLOC_MAX_PAIRS];           // FP64 sum of the blocks' FP32 partial costs
    unsigned long long count[PBA_NOALLOC_MAX_PAIRS];  // valid residuals, exact
    NaPair pairs[PBA_NOALLOC_MAX_PAIRS];
};

static_assert(sizeof(NaScratch) <= PBA_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds its stated size");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PBA_NOALLOC_SCRATCH_BYTES];

struct NaSensor {
    int model, width, height;
    float fx, fy, cx, cy;
    float R[9], t[3];
};

__device__ __forceinline__ bool na_valid(const float* c, float rmin, float rmax) {
    const float n2 = c[2] * c[2] + c[3] * c[3] + c[4] * c[4];
    (void)n2;
    return plain_pixel_valid(c, rmin, rmax);
}

// Per pair: zero the accumulator and build the FP32 transform
// pbar = M p_u + a, M = R_o^T R_j^T R_i, a = R_o^T (R_j^T (t_i - t_j) - t_o)  (Supp., pbar_u)
struct Xo12 {
    double v[12];
};

__global__ void k_na_setup(NaScratch* S, const double* __restrict__ poses, const int32_t* __restrict__ pairs, int m,
                           int n_frames, const Xo12 xo) {
    const int q = blockIdx.x;
    if (q >= m) return;
    for (int k = threadIdx.x; k < kNaStride; k += blockDim.x) S->acc[q][k] = 0.f;
    if (threadIdx.x != 0) return;
    S->cost[q] = 0.0;
    S->count[q] = 0ull;
    const double* Xo = xo.v;
    const int i = pairs[2 * q], j = pairs[2 * q + 1];
    if (i < 0 || j < 0 || i >= n_frames || j >= n_frames) {
        // a frame index out of range: the pair contributes nothing (all-zero block)
        S->pairs[q].src = -1;
        S->pairs[q].tgt = -1;
        return;
    }
    const double* Xi = poses + 12 * i;
    const double* Xj = poses + 12 * j;
    double R[9], t[3];
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) R[3 * r + c] = Xj[r] * Xi[c] + Xj[4 + r] * Xi[4 + c] + Xj[8 + r] * Xi[8 + c];
        t[r] = Xj[r] * (Xi[3] - Xj[3]) + Xj[4 + r] * (Xi[7] - Xj[7]) + Xj[8 + r] * (Xi[11] - Xj[11]);
    }
    NaPair P;
    P.src = i;
    P.tgt = j;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) P.M[3 * r + c] = (float)(Xo[r] * R[c] + Xo[4 + r] * R[3 + c] + Xo[8 + r] * R[6 + c]);
        P.a[r] = (float)(Xo[r] * (t[0] - Xo[3]) + Xo[4 + r] * (t[1] - Xo[7]) + Xo[8 + r] * (t[2] - Xo[11]));
    }
    S->pairs[q] = P;
}

__global__ void __launch_bounds__(kNaThreads)
    k_na_plain(NaScratch* S, const float* __restrict__ raw, const NaSensor sen, const LinParams prm, float rmin,
               float rmax) {
    __shared__ float s_red[kNaThreads / 32][kNaAcc];
    const int q = blockIdx.y;
    const NaPair Q = S->pairs[q];
    if (Q.src < 0) return;  // whole block: blockIdx.y is uniform
    const int W = sen.width, Hh = sen.height;
    const long long npx = (long long)W * Hh;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const float om[5] = {prm.w_int, prm.w_depth, prm.w_normal, prm.w_normal, prm.w_normal};
    bool valid = false;
    float e[5] = {0.f, 0.f, 0.f, 0.f, 0.f}, w = 0.f, rho = 0.f;
    float J[5][12];
    if (px < npx) {
        float cs[5];
        const float* c = raw + (Q.src * npx + px) * 5;
        for (int k = 0; k < 5; ++k) cs[k] = c[k];
        if (na_valid(cs, rmin, rmax)) {
            const int col = px % W, row = px / W;
            const float d = cs[1];
            float p[3];
            if (sen.model == 0) {
                p[0] = d * ((col - sen.cx) / sen.fx);
                p[1] = d * ((row - sen.cy) / sen.fy);
                p[2] = d;
            } else {
                float saz, caz, sel, cel;
                sincosf((col - sen.cx) / sen.fx, &saz, &caz);
                sincosf((row - sen.cy) / sen.fy, &sel, &cel);
                p[0] = d * (cel * caz);
                p[1] = d * (cel * saz);
                p[2] = d * sel;
            }
            float pu[3], no[3], qb[3];
            for (int r = 0; r < 3; ++r) {
                pu[r] = sen.R[3 * r] * p[0] + sen.R[3 * r + 1] * p[1] + sen.R[3 * r + 2] * p[2] + sen.t[r];
                no[r] = sen.R[3 * r] * cs[2] + sen.R[3 * r + 1] * cs[3] + sen.R[3 * r + 2] * cs[4];
            }
            for (int r = 0; r < 3; ++r) qb[r] = Q.M[3 * r] * pu[0] + Q.M[3 * r + 1] * pu[1] + Q.M[3 * r + 2] * pu[2] + Q.a[r];
            float u, v, zd;
            bool ok;
            if (sen.model == 0) {
                ok = qb[2] > prm.z_min;
                u = sen.fx * qb[0] / qb[2] + sen.cx;
                v = sen.fy * qb[1] / qb[2] + sen.cy;
                zd = qb[2];
            } else {
                zd = sqrtf(qb[0] * qb[0] + qb[1] * qb[1] + qb[2] * qb[2]);
                ok = zd > prm.z_min;
                u = sen.fx * atan2f(qb[1], qb[0]) + sen.cx;
                v = sen.fy * atan2f(qb[2], sqrtf(qb[0] * qb[0] + qb[1] * qb[1])) + sen.cy;
            }
            ok = ok && v >= 1.f && v < (float)(Hh - 2);
            if (sen.model == 0) ok = ok && u >= 1.f && u < (float)(W - 2);
            if (ok) {
                const int c0 = (int)floorf(u), r0 = (int)floorf(v);
                const float a = u - floorf(u), b = v - floorf(v);
                const float* T = raw + Q.tgt * npx * 5;
                auto tx = [&](int r, int cc) -> const float* {
                    if (sen.model == 1) {
                        cc %= W;
                        if (cc < 0) cc += W;
                    }
                    return T + ((long long)r * W + cc) * 5;
                };
                const int st[12][2] = {{-1, 0}, {-1, 1}, {0, -1}, {0, 0}, {0, 1}, {0, 2},
                                       {1, -1}, {1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 1}};
                for (int k = 0; k < 12 && ok; ++k) {
                    const float* t = tx(r0 + st[k][0], c0 + st[k][1]);
                    float tc[5] = {t[0], t[1], t[2], t[3], t[4]};
                    ok = na_valid(tc, rmin, rmax);
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
                    float nb[3];
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
                        float P0[3], P1[3], dz[3];
                        if (sen.model == 0) {
                            const float iz = 1.f / qb[2];
                            P0[0] = sen.fx * iz; P0[1] = 0.f; P0[2] = -sen.fx * qb[0] * iz * iz;
                            P1[0] = 0.f; P1[1] = sen.fy * iz; P1[2] = -sen.fy * qb[1] * iz * iz;
                            dz[0] = 0.f; dz[1] = 0.f; dz[2] = 1.f;
                        } else {
                            const float rxy2 = qb[0] * qb[0] + qb[1] * qb[1], rxy = sqrtf(rxy2);
                            const float r2 = rxy2 + qb[2] * qb[2];
                            P0[0] = -sen.fx * qb[1] / rxy2; P0[1] = sen.fx * qb[0] / rxy2; P0[2] = 0.f;
                            P1[0] = -sen.fy * qb[0] * qb[2] / (rxy * r2);
                            P1[1] = -sen.fy * qb[1] * qb[2] / (rxy * r2);
                            P1[2] = sen.fy * rxy / r2;
                            dz[0] = qb[0] / zd; dz[1] = qb[1] / zd; dz[2] = qb[2] / zd;
                        }
                        float qj[3], mj[3];
                        for (int r = 0; r < 3; ++r) {
                            qj[r] = sen.R[3 * r] * qb[0] + sen.R[3 * r + 1] * qb[1] + sen.R[3 * r + 2] * qb[2] + sen.t[r];
                            mj[r] = sen.R[3 * r] * nb[0] + sen.R[3 * r + 1] * nb[1] + sen.R[3 * r + 2] * nb[2];
                        }
                        for (int ch = 0; ch < 5; ++ch) {
                            float g[3], h[3], kk[3];
                            for (int k = 0; k < 3; ++k) g[k] = (ch == 1 ? dz[k] : 0.f) - (gu[ch] * P0[k] + gv[ch] * P1[k]);
                            for (int k = 0; k < 3; ++k) {
                                h[k] = Q.M[k] * g[0] + Q.M[3 + k] * g[1] + Q.M[6 + k] * g[2];
                                kk[k] = sen.R[3 * k] * g[0] + sen.R[3 * k + 1] * g[1] + sen.R[3 * k + 2] * g[2];
                            }
                            J[ch][0] = h[0]; J[ch][1] = h[1]; J[ch][2] = h[2];
                            J[ch][3] = 2.f * (pu[1] * h[2] - pu[2] * h[1]);
                            J[ch][4] = 2.f * (pu[2] * h[0] - pu[0] * h[2]);
                            J[ch][5] = 2.f * (pu[0] * h[1] - pu[1] * h[0]);
                            J[ch][6] = -kk[0]; J[ch][7] = -kk[1]; J[ch][8] = -kk[2];
                            J[ch][9] = 2.f * (kk[1] * qj[2] - kk[2] * qj[1]);
                            J[ch][10] = 2.f * (kk[2] * qj[0] - kk[0] * qj[2]);
                            J[ch][11] = 2.f * (kk[0] * qj[1] - kk[1] * qj[0]);
                            if (ch >= 2) {
                                const int r = ch - 2;
                                const float mx = Q.M[3 * r], my = Q.M[3 * r + 1], mz = Q.M[3 * r + 2];
                                J[ch][3] += 2.f * (no[1] * mz - no[2] * my);
                                J[ch][4] += 2.f * (no[2] * mx - no[0] * mz);
                                J[ch][5] += 2.f * (no[0] * my - no[1] * mx);
                                const float cx_ = sen.R[r], cy_ = sen.R[3 + r], cz_ = sen.R[6 + r];
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
    auto put = [&](int k, float x) {
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) s_red[warp][k] = x;
    };
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
    put(90, valid ? rho : 0.f);
    put(91, valid ? 1.f : 0.f);
    __syncthreads();
    if (threadIdx.x < kNaAcc) {
        float x = 0.f;
        for (int w8 = 0; w8 < kNaThreads / 32; ++w8) x += s_red[w8][threadIdx.x];
        if (threadIdx.x < 90) atomicAdd(&S->acc[q][threadIdx.x], x);
        else if (threadIdx.x == 90) atomicAdd(&S->cost[q], (double)x);
        else atomicAdd(&S->count[q], (unsigned long long)x);  // a block's count: an integer <= 256, exact in FP32
    }
}

// FP32 accumulators -> FP64 pair blocks in the caller's buffer (layout of pba_get_pair_system).
__global__ void k_na_expand(const NaScratch* S, double* __restrict__ out) {
    const int q = blockIdx.x, t = threadIdx.x;
    const float* a = S->acc[q];
    double* o = out + (long long)q * PBA_NOALLOC_PAIR_STRIDE;
    if (t < 144) {
        const int r = t / 12, c = t % 12;
        const int lo = r < c ? r : c, hi = r < c ? c : r;
        o[t] = (double)a[lo * 12 - lo * (lo - 1) / 2 + (hi - lo)];
    }
    if (t < 12) o[144 + t] = (double)a[78 + t];
    if (t == 0) {
        o[156] = S->cost[q];
        o[157] = (double)S->count[q];
        o[158] = 0.0;
        o[159] = 0.0;
    }
}

}  // namespace
}  // namespace pba

extern "C" int pba_linearize_pairs_noalloc(const pba_sensor* sensor, const pba_config* cfg, const float* channels,
                                           int n_frames, const double* poses, const int32_t* pairs, int m,
                                           double* pair_out, void* cuda_stream) {
    using namespace pba;
    if (!sensor || !cfg || !channels || !poses || (!pairs && m > 0) || (!pair_out && m > 0) || n_frames < 1 || m < 0)
        return PBA_EINVAL;
    if (sensor->model != PBA_PINHOLE && sensor->model != PBA_SPHERICAL) return PBA_EINVAL;
    if (sensor->width < 4 || sensor->height < 4 || sensor->fx == 0.0 || sensor->fy == 0.0) return PBA_EINVAL;
    if (!(cfg->huber_delta > 0.0) || (cfg->grad_mode != 0 && cfg->grad_mode != 1)) return PBA_EINVAL;
    if (m > PBA_NOALLOC_MAX_PAIRS) return PBA_ETOOBIG;
    if ((long long)sensor->width * sensor->height > (1LL << 30)) return PBA_ETOOBIG;
    if (m == 0) return PBA_OK;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return PBA_ECUDA;
    // the device address of the static array on the current device, looked up on
    // every call (a host-side query; it stays right after a device reset)
    void* sym = nullptr;
    if (cudaGetSymbolAddress(&sym, g_noalloc_scratch) != cudaSuccess || !sym) return PBA_ECUDA;
    NaScratch* S = reinterpret_cast<NaScratch*>(sym);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    LinParams prm{};
    prm.w_int = (float)cfg->w_int;
    prm.w_depth = (float)cfg->w_depth;
    prm.w_normal = (float)cfg->w_normal;
    prm.huber_delta = (float)cfg->huber_delta;
    prm.huber_delta2 = (float)(cfg->huber_delta * cfg->huber_delta);
    prm.occ_abs = (float)cfg->occ_abs;
    prm.occ_rel = (float)cfg->occ_rel;
    prm.z_min = (float)cfg->z_min;
    prm.grad_mode = cfg->grad_mode;
    NaSensor sen{};
    sen.model = sensor->model;
    sen.width = sensor->width;
    sen.height = sensor->height;
    sen.fx = (float)sensor->fx;
    sen.fy = (float)sensor->fy;
    sen.cx = (float)sensor->cx;
    sen.cy = (float)sensor->cy;
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) sen.R[3 * r + c] = (float)sensor->extrinsic[4 * r + c];
        sen.t[r] = (float)sensor->extrinsic[4 * r + 3];
    }
    Xo12 xo;
    for (int k = 0; k < 12; ++k) xo.v[k] = sensor->extrinsic[k];
    float rmin, rmax;
    float_range_limits(cfg->range_min, cfg->range_max, &rmin, &rmax);
    const long long npx = (long long)sensor->width * sensor->height;
    // 1. zero this call's accumulators and build the pair transforms
    k_na_setup<<<m, 128, 0, s>>>(S, poses, pairs, m, n_frames, xo);
    // 2. every pair in one launch
    k_na_plain<<<dim3((unsigned)((npx + kNaThreads - 1) / kNaThreads), (unsigned)m), kNaThreads, 0, s>>>(
        S, channels, sen, prm, rmin, rmax);
    // 3. FP64 pair blocks into the caller's buffer
    k_na_expand<<<m, 160, 0, s>>>(S, pair_out);
    return cudaGetLastError() == cudaSuccess ? PBA_OK : PBA_ECUDA;
}
