// pba_internal.cuh -- device-side data layout shared by the kernels of libpba.
//
// Layout in HBM (one problem):
//   raw       FP32 H x W x 5 per frame (the uploaded cue images, kept for the plain path)
//   texels    per frame H x W sampling texels: Tex16 {float d; half g, nx, ny, nz; usable}
//             or Tex32 {float d, g, nx, ny, nz, usable, pad x 2}; d = 0 marks an invalid
//             pixel, usable = pixel and its 4 neighbours valid
//   points    per frame, compacted valid pixels in raster order:
//             pg = float4(p_u, g_u), pn = float4(n_u^o, 0)   (Supp., p_u = R_o pi^-1(u, d) + t_o),
//             pix = pixel index (row * W + column) of the point
//   pair pose table (FP32, per iteration): pbar = M p_u + a with M = R_o^T R_j^T R_i,
//             a = R_o^T (R_j^T (t_i - t_j) - t_o)   (Supp., pbar_u)
//   chunk list int4 {pair, first point, count, 0}: the persistent launch's work queue
//   partials  FP32 per chunk (one warp's work item): 21 (H6 upper) + 6 (b6) + cost + count
//             + residuals left out as not finite (+2 pad) = 32 floats
//   pair blocks FP64 per pair: H12 (144) + b12 (12) + cost + count + residuals left out as
//             not finite + 1 when the pair's relative pose is not finite = 160 doubles
//   H (6N x 6N) and b (6N) FP64 dense; A = H_ff + lambda I padded to a multiple of 32
#pragma once

#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace pba {

constexpr int kPartialStride = 32;   // floats per chunk partial
constexpr int kNumAcc = 30;          // 21 + 6 + cost + count + non-finite residuals
constexpr int kBlockStride = 160;    // doubles per pair block
constexpr int kTile = 32;            // Cholesky tile
constexpr double kRefineTol = 1e-10; // |r| <= kRefineTol |b'| ends the mixed-precision refinement

// The float32 range limits that decide d >= range_min and d <= range_max for
// every float32 depth d exactly as the double comparisons do: range_min
// rounded up and range_max rounded down to float32 (a limit above the float
// range stays at 3e38).
inline void float_range_limits(double range_min, double range_max, float* rmin, float* rmax) {
    float lo = (float)range_min;
    if ((double)lo < range_min) lo = nextafterf(lo, 3.0e38f);
    float hi = range_max > 3.0e38 ? 3.0e38f : (float)range_max;
    if ((double)hi > range_max) hi = nextafterf(hi, -3.0e38f);
    *rmin = lo;
    *rmax = hi;
}

// Pixel validity of the plain paths (Sec. IV-A): range_min <= d <= range_max
// (limits from float_range_limits), d > 0 and |n|^2 > 0.25, the last summed in
// FP32 unless it lies within 1e-6 of the threshold, where the double sum
// decides (as the double evaluation of the float inputs would).
__device__ __forceinline__ bool plain_pixel_valid(const float* c, float rmin, float rmax) {
    if (!(c[1] > 0.f && c[1] >= rmin && c[1] <= rmax)) return false;
    const float n2 = fmaf(c[4], c[4], fmaf(c[3], c[3], c[2] * c[2]));
    if (fabsf(n2 - 0.25f) > 1e-6f) return n2 > 0.25f;
    return (double)c[2] * c[2] + (double)c[3] * c[3] + (double)c[4] * c[4] > 0.25;
}

struct FrameInfo {
    int width, height, sensor, model;
    float fx, fy, cx, cy;
    long long px_offset;     // pixel offset of the frame in raw / texel buffers
    long long pt_offset;     // point offset of the frame in the point buffers
};

struct SensorDev {
    float R[9];              // R_o row-major (FP32 copy)
    float t[3];              // t_o
    int model, width, height, pad;
    float fx, fy, cx, cy;
};

// Static per-pair data, built on the host by pba_set_pairs.
struct PairStatic {
    int src, tgt, model, width, height;
    int n_points;            // points of the source frame
    int chunk_begin, chunk_end;
    float fx, fy, cx, cy;
    long long src_pt_offset; // into point buffers
    long long tgt_px_offset; // into texel / raw buffers
    long long mask_offset;   // in 32-bit words
    long long src_px_offset; // raw buffer of the source (plain path)
    int src_width, src_height;
    float fxh, fxp;          // spherical: f_x pi / 2 and f_x pi (offsets of the column, spherical_project)
};

// Pose-dependent per-pair constants (FP32), rebuilt on the device each iteration.
struct PairPose {
    float M[9];
    float a[3];
};

// usable = the pixel and its 4 neighbours are valid (central differences defined)
struct Tex16 {
    float d;
    __half2 g_nx;
    __half2 ny_nz;
    unsigned usable;
};

struct Tex32 {
    float d, g, nx, ny, nz;
    unsigned usable;
    float p1, p2;
};

struct LinParams {
    float w_int, w_depth, w_normal;
    float huber_delta, huber_delta2;
    float occ_abs, occ_rel;
    float z_min;
    int grad_mode;
    // per pixel of every frame: the central differences of the Supp. at the pixel,
    // (d/du, d/dv) of (g, d, n_x, n_y, n_z), 12 floats (3 float4, the last two 0);
    // zero where the pixel is not usable
    const float4* gtex;
    // FP16 texels: one TMA tensor map per frame (its texels as 4 words x width x
    // height), read by the staged kernel variants; tile_err is raised when a tile
    // wait ran out
    const CUtensorMap* tmaps;
    int* tile_err;
    // reduction of a work item's 30 sums: 0 a transposed table in shared
    // memory (+ shuffles for the last three), 1 a butterfly of shuffles
    int reduction;
};

// Device-side Levenberg-Marquardt state of one problem.
struct LmState {
    double lambda;          // next damping (< 0: automatic on the next iteration)
    double lambda_used;
    double cost;
    double new_cost;
    long long n_valid;
    long long n_valid_new;
    int accepted;
    int status;             // 0 or PBA_ENOTPD
    int chol_fail;          // set by the factorisation
    int pad;
    double iter_cost;       // F at the poses the last iteration started from
    long long iter_n_valid; // residuals linearised by the last iteration
    // status word: residuals left out because their value is not finite, and pairs
    // whose relative pose is not finite (current system, candidate, last iteration's)
    long long nf_res, nf_res_new, iter_nf_res;
    long long nf_pairs, nf_pairs_new, iter_nf_pairs;
};

// Assembly task: one 6x6 block of H (diagonal when a == b).
struct AsmTask {
    int a, b;               // frames (a <= b)
    int contrib_begin, contrib_end;
};

// Contribution to an assembly task: pair index and the two roles (0 = i, 1 = j)
// selecting the 6x6 sub-block (row role, column role) of the pair's H12.
struct AsmContrib {
    int pair;
    int row_role, col_role;
    int add_b;              // 1: also add the pair's b sub-vector of row_role (diagonal tasks)
};

}  // namespace pba

// ---------------------------------------------------------------- launchers
// (host-callable, defined in the .cu files; all asynchronous on `s`)

namespace pba {

// One pyramid level down (Sec. IV-A): frames frame_ids[0..n) of raw into out at
// out_offsets (coarse pixels), 2 x 2 blocks.
cudaError_t launch_downsample(const float* raw, const FrameInfo* frames, const int* frame_ids,
                              const long long* out_offsets, int n, int max_coarse_px, float* out, double range_min,
                              double range_max, cudaStream_t s);

// Sensor offsets as variables (pba_offset.cu).
cudaError_t launch_offset_system(const double* blocks, const double* pair_Xo, int m, double* pext,
                                 const int* f_start, const int2* f_items, const int* s_start, const int* s_items,
                                 const int* frame_sensor, const int* sensor_var, int n_frames, int n_sensors,
                                 double* Hfo, double* Hoo, double* bo, cudaStream_t s);
cudaError_t launch_reduce_vars_offset(const double* H, const double* b, const double* Hfo, const double* Hoo,
                                      const double* bo, const int* frame_sensor, int n_frames, const int* var_start,
                                      const int* var_blocks, int n_vars, double* Hr, double* br, cudaStream_t s);
cudaError_t launch_offset_step(const double* extr, const double* dx, const int* sensor_var, int n_sensors,
                               const LmState* st, double* cand, cudaStream_t s);
cudaError_t launch_offset_accept(const LmState* st, double* extr, const double* cand, int n_sensors,
                                 cudaStream_t s);
cudaError_t launch_offset_refresh(const double* extr, int n_sensors, const int2* pf, const int* frame_sensor, int m,
                                  double* pair_Xo, SensorDev* sensors, cudaStream_t s);

// Normal estimation (Sec. IV-A), in place on the normal channels of raw.
cudaError_t launch_normals(float* raw, const FrameInfo* frames, const int* frame_ids, int n, int max_px, float scale,
                           int max_radius, double range_min, double range_max, cudaStream_t s);

// max_px: the largest frame's pixel count; tile_counts: n_frames x pack_tiles(max_px) ints of
// scratch; valid_px: one byte per pixel of every frame (scratch, laid out like raw).
int pack_tiles(int max_px);
cudaError_t launch_pack(const float* raw, const FrameInfo* frames, const SensorDev* sensors,
                        const int* frame_ids, int n, int texel_precision, void* texels,
                        float4* pts_pg, float4* pts_n, int* pts_pix, int* n_points, double range_min,
                        double range_max, cudaStream_t s, float4* gtex, int max_px, int* tile_counts,
                        unsigned char* valid_px);

cudaError_t launch_pair_pose(const double* poses, const int2* pair_frames, const double* pair_Xo, int m,
                             PairPose* out, cudaStream_t s);

// chunks: work items (pair, first point, point count, partial-sum slot), taken
// in array order from *queue (counting up to n_chunks); item k writes its sums
// to slot chunks[k].w of partials, so a launch may take a permuted subset.
cudaError_t launch_linearize(bool full, bool mask, int texel_precision, const int4* chunks, int n_chunks,
                             int* queue, const PairStatic* ps, const PairPose* pp, const float4* pts_pg,
                             const float4* pts_n, const void* texels, const LinParams& prm,
                             float* partials, uint32_t* mask_bits, int grid, int variant, cudaStream_t s);

// Threads of a block of the batched linearisation kernel (warps of one block
// share nothing but their queue regions).
constexpr int kLinThreads = 128;

// Persistent grid (SMs x resident blocks) of a linearisation occupancy variant
// (0 .. PBA_N_VARIANTS - 1, see launch_linearize).
int linearize_grid(int texel_precision, bool full, int variant);

cudaError_t launch_pair_reduce(const float* partials, const PairStatic* ps, const int2* pair_frames,
                               const double* poses, const double* pair_Xo, int m, bool full,
                               double* blocks, cudaStream_t s);

cudaError_t launch_plain(bool full, int pair, const PairStatic* ps, const PairPose* pp, const float* raw,
                         const SensorDev* sensors, int src_sensor, const LinParams& prm, double range_min,
                         double range_max, float* acc, int width, int height, cudaStream_t s);

cudaError_t launch_plain_expand(const float* acc, int m, bool full, double* blocks, cudaStream_t s);

cudaError_t launch_assemble(const AsmTask* tasks, int n_tasks, const AsmContrib* contrib,
                            const double* blocks, int n_frames, double* H, double* b, cudaStream_t s);

cudaError_t launch_total_cost(const double* blocks, int m, LmState* st, bool candidate, cudaStream_t s);

cudaError_t launch_lm_prepare(const double* H, int n_frames, LmState* st, double explicit_lambda,
                              cudaStream_t s);

cudaError_t launch_damp(const double* H, const double* b, int n_frames, int n_pad, const LmState* st,
                        double* A, double* rhs, cudaStream_t s);

// Tiled Cholesky A = L L^T in place (L in the lower triangle, L^T copied to the
// upper one); Dinv receives the inverses of the diagonal tiles (n_pad / 32 tiles of 32 x 32).
cudaError_t launch_cholesky(double* A, double* Dinv, int n_pad, LmState* st, cudaStream_t s, int* n_launches);

cudaError_t launch_trsv(const double* A, const double* Dinv, int n_pad, double* rhs, const LmState* st,
                        cudaStream_t s);

// Working buffers of the mixed-precision solve (all n_pad long except A32, n_pad^2).
struct MixedWork {
    float* A32;
    float* D32;     // inverses of the diagonal tiles (n_pad * 32)
    float* r32;
    double* bs;
    double* x;
    double* dscale;
    double* norms;  // 2
};

// Jacobi-scaled FP32 Cholesky + FP64 iterative refinement; writes dx_f (n_pad) = rhs layout
// of launch_trsv.  Sets st->chol_fail when a pivot fails or the refinement misses its tolerance.
cudaError_t launch_solve_mixed(const double* H, const double* b, int n_frames, int n_pad, LmState* st,
                               MixedWork& w, int refinements, double* dx, cudaStream_t s, int* n_launches);

// The same solve as launch_solve_mixed in one launch of a thread-block cluster
// whose shared memory holds the FP32 factor (pba_solve_cluster.cu).
struct CsGeom {
    int nt, C, n_pad, bytes;  // tile rows, CTAs in the cluster, padded size, shared memory per CTA
    int o_x, o_dsc, o_xs, o_bs, o_rsq, o_nrm, o_flag, o_tiles, o_dinv, o_dk, o_stage, o_rv, o_yv, o_zv, o_cb, o_pv,
        o_dsc32;
};
// Largest cluster the device schedules with the full opt-in shared memory (once; false: none).
bool solve_cluster_init();
// Layout for an n_pad system; false when it does not fit the cluster's shared memory.
bool solve_cluster_plan(int n_pad, CsGeom* g);
// gL (n_pad x n_pad FP32) and gD (n_pad x 32 FP32): global scratch for the tiles the CTAs exchange.
cudaError_t launch_solve_cluster(const double* H, const double* b, int n_frames, const CsGeom& g, LmState* st,
                                 int refinements, double* dx, float* gL, float* gD, cudaStream_t s);

// Block-sparse damped solve for large pose graphs (pba_solve_sparse.cu).  Positions
// are the pose variables in the solve's order (components contiguous, each
// ordered for a small envelope); unknown s = 6 position + r within a
// component's tile rows (components start on a tile row; padding unknowns get
// an identity row).  Lower blocks have row position >= column position.
struct SpPlanHost {
    int nv = 0, n_rows = 0, C = 1;
    long long n_tiles = 0;
    std::vector<int> var_of_pos, scal_of_pos, pos_of_scalar, diag_blk;
    std::vector<int2> blk;                 // lower blocks (row position, column position)
    std::vector<int> blk_start;            // contributions of each block ...
    std::vector<int4> blk_contrib;         // ... (pair, row role, column role, 0)
    std::vector<int> b_start;              // b contributions of each position ...
    std::vector<int2> b_contrib;           // ... (pair, role)
    std::vector<int> row_start;            // blocks of each position's block row ...
    std::vector<int2> row_items;           // ... (block, 1 when used transposed)
    std::vector<int> tile_first;           // per tile row I: F(I), the first stored tile column
    std::vector<long long> tile_off;       // per tile row: index of its tile (I, F(I))
    std::vector<int2> comp_rows;           // per component: (first tile row, tile rows)
};
struct SpPlanDev {
    int nv, n_rows, nblk, n_comp, C;
    long long n_tiles;
    const int* var_of_pos;
    const int* scal_of_pos;
    const int* pos_of_scalar;
    const int* diag_blk;
    const int2* blk;
    const int* blk_start;
    const int4* blk_contrib;
    const int* b_start;
    const int2* b_contrib;
    const int* row_start;
    const int2* row_items;
    const int* tile_first;
    const long long* tile_off;
    const int2* comp_rows;
    // work buffers
    double* Hv;    // nblk x 36: the blocks of H_ff (without damping)
    double* bvec;  // nv x 6: b of each position
    double* dsc;   // n_rows x 32: D
    float* dsc32;
    double* bsc;   // b' = -D b
    double* x;     // refined solution of the scaled system
    double* r64;   // its FP64 residual
    float* L;      // n_tiles x 32 x 32: A', then its factor (row-major tiles)
    float* Dinv;   // n_rows x 32 x 32: inverses of the diagonal tiles
    float* rv;     // FP32 right-hand side of the triangular solves (n_rows x 32)
    float* yv;
    float* zv;
    float* acc;    // backward-solve accumulators
    double* nrm;   // 2 per CTA: |b'|^2 and |r|^2 partials
};
// Host plan: variable graph, components, ordering, blocks, envelope; cluster size
// chosen from cmax (the largest cluster the device runs).  False when nothing to solve.
bool sparse_plan(int n_vars, const std::vector<int>& frame_var, const std::vector<int32_t>& pairs, int cmax,
                 SpPlanHost* out);
int sparse_cluster_max();
// Gather, damp, scale, factorise and refine; dx in variable order (6 per variable).
cudaError_t launch_sparse_solve(const SpPlanDev& pl, const double* blocks, LmState* st, double explicit_lambda,
                                int refinements, double* dx, cudaStream_t s, int* n_launches);

cudaError_t launch_boxplus(const double* poses, const double* dx_ff, int n_frames, const int* frame_var,
                           const LmState* st, double* cand, cudaStream_t s);
// Hr = S^T H S, br = S^T b in pose variables (leading fixed dummy block).
cudaError_t launch_reduce_vars(const double* H, const double* b, int n_frames, const int* var_start,
                               const int* var_frames, int n_vars, double* Hr, double* br, cudaStream_t s);

// Keep the candidate when the cost decreased.  speculative: the candidate was
// linearised in full, so on acceptance its system (H_cand, b_cand, blocks_cand,
// cost, count) replaces the current one as well as the poses (H nullptr: only
// the pair blocks, when no dense system is kept).
cudaError_t launch_accept(LmState* st, double* poses, const double* cand, int n_frames, bool speculative,
                          double* H, const double* H_cand, double* b, const double* b_cand, double* blocks,
                          const double* blocks_cand, int m, cudaStream_t s);

// Adjoint of the total cost (pba_adjoint.cu).
int adjoint_partial_stride();  // floats per work-item partial
int adjoint_pair_stride();     // doubles per pair result
int adjoint_grid(int texel_precision);
cudaError_t launch_adjoint(int texel_precision, const int4* chunks, int n_chunks, int* queue, const PairStatic* ps,
                           const PairPose* pp, const float4* pts_pg, const float4* pts_n, const int* pts_pix,
                           const void* texels, const SensorDev* sensors, const int* frame_sensor,
                           const LinParams& prm, float* partials, float* d_img, int grid, cudaStream_t s);
// dF/d dx in the box-plus chart from dF/dX for n transforms (n x 12 -> n x 6).
cudaError_t launch_tangent(const double* X, const double* G, int n, double* g, cudaStream_t s);
cudaError_t launch_adjoint_reduce(const float* partials, const PairStatic* ps, const int2* pf, const double* poses,
                                  const double* pair_Xo, int m, double* pair_out, const AsmTask* tasks, int n_tasks,
                                  const AsmContrib* contrib, const int* frame_sensor, int n_sensors,
                                  double* d_poses, double* d_ext, double* totals, cudaStream_t s);

}  // namespace pba
