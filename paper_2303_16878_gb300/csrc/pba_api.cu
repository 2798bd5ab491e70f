// pba_api.cu -- the C ABI of libpba (declared in include/pba.h): problem
// lifecycle, uploads, the host-side plan of one Gauss-Newton iteration (chunk
// queue, per-pair chunk ranges, assembly tasks) and the enqueueing of the
// kernels, directly or as a captured CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "../../include/pba.h"
#include "pba_internal.cuh"
#include "pba_tma.cuh"

using namespace pba;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kChunk = 1024;     // default points per work item (one warp) of the persistent launch
constexpr int kChunkTail = 256;  // ... in the last stretch of the queue, so that the warps finish closer together
// the work-item sizes pba_autotune tries
constexpr int kTuneChunks[3] = {512, 1024, 2048};
constexpr int kTuneTails[2] = {128, 256};
constexpr int kNumReductions = 2;  // reduction schemes of a work item's sums (LinParams::reduction)
// the order pba_autotune tries them in (the butterfly first: it measured a
// fraction of a per cent faster, within the tie margin, on every workload)
constexpr int kTuneReductions[kNumReductions] = {1, 0};
constexpr float kTuneTie = 0.02f;  // relative time difference the autotuner treats as a tie

}  // namespace

struct pba_problem {
    pba_config cfg{};
    std::vector<pba_sensor> sensors;
    std::vector<int> frame_sensor;
    int N = 0;
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t capture_stream = nullptr;
    // host-to-device uploads are split over the problem's stream and these
    // (one copy keeps one copy engine busy); the events join them back
    static constexpr int kCopyLanes = 4;
    cudaStream_t copy_streams[kCopyLanes - 1] = {};
    cudaEvent_t copy_events[kCopyLanes] = {};
    // pba_iterate_frames: the frames arrive in lanes of whole frames (copied in
    // order on lane_copy, packed on lane_pack, a stream of the greatest
    // priority); the work items of the pairs whose frames have all arrived with
    // lane l form segment l of d_chunks_ready, whose linearisation (on the
    // problem's stream) waits for that lane only
    static constexpr int kFrameLanes = 8;
    cudaStream_t lane_copy = nullptr, lane_pack = nullptr;
    cudaEvent_t lane_start = nullptr;
    cudaEvent_t lane_copied[kFrameLanes] = {}, lane_ready[kFrameLanes] = {};
    int4* d_chunks_ready = nullptr;
    int n_chunks_ready_alloc = 0;
    std::vector<int> ready_first;  // lane boundaries (frames) d_chunks_ready was ordered for
    std::vector<int> ready_seg;    // segment boundaries in d_chunks_ready
    long long plan_serial = 0, ready_serial = -1;
    int* d_seg_queue = nullptr;    // one work-queue counter per segment
    int* h_counts = nullptr;       // pinned: point counts read back after the overlapped pass
    // staged linearisation variants (FP16 texels, frames at least one tile in size):
    // one TMA tensor map per frame and the flag a tile wait raises when it runs out
    bool stage_ok = false;
    CUtensorMap* d_tmaps = nullptr;
    int* d_tile_err = nullptr;
    std::string err;

    // frames
    std::vector<long long> px_off;
    long long total_px = 0;
    std::vector<int> n_points;
    std::vector<char> uploaded;
    bool points_known = false;

    // device buffers (problem lifetime)
    float* raw = nullptr;
    void* tex = nullptr;
    float4* gtex = nullptr;  // central differences per pixel (LinParams::gtex)
    int max_frame_px = 0;
    int* d_tile_counts = nullptr;  // scratch of the two-pass pack: valid pixels per 1024-pixel tile
    unsigned char* d_valid_px = nullptr;  // scratch of the pack: validity of every pixel
    int* d_frame_iota = nullptr;          // 0 .. N-1 (frame lists of contiguous ranges)
    float4* pts_pg = nullptr;
    float4* pts_n = nullptr;
    int* pts_pix = nullptr;
    int* d_frame_sensor = nullptr;
    int* d_npoints = nullptr;
    FrameInfo* d_frames = nullptr;
    SensorDev* d_sensors = nullptr;
    int* d_frame_ids = nullptr;
    double* d_poses = nullptr;
    double* d_cand = nullptr;
    LmState* d_state = nullptr;
    double* d_H = nullptr;
    double* d_b = nullptr;
    double* d_H_cand = nullptr;  // system linearised at the candidate (speculative LM step)
    double* d_b_cand = nullptr;
    double* d_A = nullptr;
    double* d_rhs = nullptr;
    double* d_Dinv = nullptr;  // inverses of the Cholesky diagonal tiles
    int n_pad = 0;        // padded size of the default gauge-fixed system
    int n_pad_alloc = 0;  // padded size the solver buffers hold
    MixedWork mixed{};  // buffers of the mixed-precision solve
    int* d_queue = nullptr;  // two counters: full pass, cost pass

    // pair-dependent buffers
    int M = 0;
    std::vector<int32_t> pairs;
    PairStatic* d_ps = nullptr;
    PairPose* d_pp = nullptr;
    int2* d_pf = nullptr;
    double* d_pair_Xo = nullptr;
    int4* d_chunks = nullptr;
    int n_chunks = 0;
    float* d_partials = nullptr;
    double* d_blocks = nullptr;
    double* d_blocks_cand = nullptr;
    AsmTask* d_tasks = nullptr;
    int n_tasks = 0;
    AsmContrib* d_contrib = nullptr;
    uint32_t* d_mask = nullptr;
    std::vector<long long> mask_off;
    std::vector<int> pair_src_points;
    float* d_plain_acc = nullptr;
    float* d_adj_partials = nullptr;  // adjoint: per work item
    double* d_adj_pair = nullptr;     // adjoint: per pair
    double* d_adj_totals = nullptr;   // adjoint: cost, count

    bool poses_set = false;
    bool mask_export = false;
    bool mask_valid = false;
    bool linearized = false;
    int grid_full = 0, grid_cost = 0;
    int variant_full = 0, variant_cost = 0;  // occupancy variants chosen by pba_autotune
    int chunk = kChunk, chunk_tail = kChunkTail;  // work-item sizes (pba_autotune)
    float tune_ms_full = 0.f, tune_ms_cost = 0.f;
    int tune_from_cache = 0;
    LinParams prm{};

    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int launches_last = 0;

    // pose variables.  fv_user / n_fv_user: the frames' mapping as given to
    // pba_set_variables (n_fv_user < 0: frame 0 fixed, frame k -> variable k - 1);
    // offset_free: sensors whose offset X_o is a variable (pba_set_offset_free).
    // n_vars: the effective number of variables of the solve, < 0 when the default
    // mapping applies and no offset is free (the solve then uses H directly).
    int n_fv_user = -1;
    std::vector<int32_t> fv_user;
    std::vector<char> offset_free;
    bool offsets_free = false;
    int n_vars = -1;
    int* d_frame_var = nullptr;
    int* d_sensor_var = nullptr;
    int* d_var_start = nullptr;
    int* d_var_frames = nullptr;   // blocks of each variable: frames f < N, offsets N + s
    double* d_Hr = nullptr;
    double* d_br = nullptr;
    int n_pad_vars = 0;
    // offsets on the device: current and candidate (S x 12, FP64), per-pair offset
    // blocks, their assembly (Hfo per frame, Hoo and bo per sensor), the pair lists
    // by frame and by sensor, and the frames re-packed when an offset moves
    double* d_extr = nullptr;
    double* d_extr_cand = nullptr;
    double* d_pext = nullptr;
    double* d_Hfo = nullptr;
    double* d_Hoo = nullptr;
    double* d_bo = nullptr;
    int* d_f_start = nullptr;
    int2* d_f_items = nullptr;
    int* d_s_start = nullptr;
    int* d_s_items = nullptr;
    int* d_free_frames = nullptr;
    int n_free_frames = 0;

    // block-sparse solve (pba_solve_sparse.cu): used when `sparse`; its device plan
    // and work buffers (sp_mem: every allocation of the plan, freed together)
    bool sparse = false;
    SpPlanDev sp{};
    std::vector<void*> sp_mem;

    // coarser pyramid levels 1.. (Sec. IV-A), each a problem of its own on the same stream
    std::vector<pba_problem*> levels;
    bool pyramid_stale = true;
};

namespace {

int fail(pba_problem* p, int code, const std::string& msg) {
    if (p) p->err = msg;
    return code;
}

#define CUDA_TRY(p, call)                                                                       \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess)                                                                  \
            return fail((p), e_ == cudaErrorMemoryAllocation ? PBA_ENOMEM : PBA_ECUDA,          \
                        std::string(#call) + ": " + cudaGetErrorString(e_));                   \
    } while (0)

template <typename T>
void dfree(T*& ptr) {
    if (ptr) cudaFree((void*)ptr);
    ptr = nullptr;
}

void free_sparse(pba_problem* p);

void free_pair_buffers(pba_problem* p) {
    free_sparse(p);
    dfree(p->d_ps);
    dfree(p->d_pp);
    dfree(p->d_pf);
    dfree(p->d_pair_Xo);
    dfree(p->d_chunks);
    dfree(p->d_partials);
    dfree(p->d_blocks);
    dfree(p->d_blocks_cand);
    dfree(p->d_tasks);
    dfree(p->d_contrib);
    dfree(p->d_mask);
    dfree(p->d_plain_acc);
    dfree(p->d_adj_partials);
    dfree(p->d_adj_pair);
    dfree(p->d_adj_totals);
    dfree(p->d_pext);
    dfree(p->d_f_start);
    dfree(p->d_f_items);
    dfree(p->d_s_start);
    dfree(p->d_s_items);
    p->d_pext = nullptr;
    p->d_f_start = p->d_s_start = p->d_s_items = nullptr;
    p->d_f_items = nullptr;
    p->M = 0;
    p->n_chunks = 0;
    p->n_tasks = 0;
    ++p->plan_serial;  // any order of the work items built for the previous plan is stale
}

void free_sparse(pba_problem* p) {
    for (void* ptr : p->sp_mem) cudaFree(ptr);
    p->sp_mem.clear();
    p->sp = SpPlanDev{};
    p->sparse = false;
}

void drop_graph(pba_problem* p) {
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->graph_exec = nullptr;
    p->graph = nullptr;
}

int ensure_points(pba_problem* p) {
    if (p->points_known) return PBA_OK;
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    CUDA_TRY(p, cudaMemcpy(p->n_points.data(), p->d_npoints, sizeof(int) * p->N, cudaMemcpyDeviceToHost));
    p->points_known = true;
    return PBA_OK;
}

// Full linearisation at the current poses (or, at_cand, at the candidate
// poses into the candidate buffers): pair pose table, persistent linearise,
// per-pair FP64 reduction, assembly of H and b, total cost.
int enqueue_linearize(pba_problem* p, cudaStream_t s, int* nl, cudaEvent_t* ev = nullptr, bool at_cand = false) {
    const double* poses = at_cand ? p->d_cand : p->d_poses;
    double* blocks = at_cand ? p->d_blocks_cand : p->d_blocks;
    double* H = at_cand ? p->d_H_cand : p->d_H;
    double* b = at_cand ? p->d_b_cand : p->d_b;
    // timing events (speculative timed iteration): [2] before the kernel, [3] after it, [4] after the cost
    CUDA_TRY(p, launch_pair_pose(poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, s));
    ++*nl;
    if (p->cfg.path == PBA_PATH_PLAIN) {
        CUDA_TRY(p, cudaMemsetAsync(p->d_plain_acc, 0, sizeof(float) * 96 * (size_t)p->M, s));
        if (ev) CUDA_TRY(p, cudaEventRecord(ev[2], s));
        for (int q = 0; q < p->M; ++q) {
            const int src = p->pairs[2 * q];
            const pba_sensor& S = p->sensors[p->frame_sensor[src]];
            CUDA_TRY(p, launch_plain(true, q, p->d_ps, p->d_pp, p->raw, p->d_sensors, p->frame_sensor[src], p->prm,
                                     p->cfg.range_min, p->cfg.range_max, p->d_plain_acc, S.width, S.height, s));
            ++*nl;
        }
        if (ev) CUDA_TRY(p, cudaEventRecord(ev[3], s));
        CUDA_TRY(p, launch_plain_expand(p->d_plain_acc, p->M, true, blocks, s));
        ++*nl;
    } else {
        CUDA_TRY(p, cudaMemsetAsync(p->d_queue, 0, sizeof(int), s));
        if (ev) CUDA_TRY(p, cudaEventRecord(ev[2], s));
        const bool mask = p->mask_export && !at_cand;
        CUDA_TRY(p, launch_linearize(true, mask, p->cfg.texel_precision, p->d_chunks, p->n_chunks, p->d_queue,
                                     p->d_ps, p->d_pp, p->pts_pg, p->pts_n, p->tex, p->prm, p->d_partials,
                                     p->d_mask, p->grid_full, p->variant_full, s));
        if (ev) CUDA_TRY(p, cudaEventRecord(ev[3], s));
        CUDA_TRY(p, launch_pair_reduce(p->d_partials, p->d_ps, p->d_pf, poses, p->d_pair_Xo, p->M, true, blocks, s));
        *nl += 2;
    }
    // the block-sparse solve gathers its system from the pair blocks: no dense H
    if (!p->sparse) {
        CUDA_TRY(p, launch_assemble(p->d_tasks, p->n_tasks, p->d_contrib, blocks, p->N, H, b, s));
        ++*nl;
    }
    CUDA_TRY(p, launch_total_cost(blocks, p->M, p->d_state, at_cand, s));
    ++*nl;
    if (ev) CUDA_TRY(p, cudaEventRecord(ev[4], s));
    return PBA_OK;
}

// Damped solve, candidate poses, then either (speculative) a full
// linearisation at the candidate, whose system becomes current on
// acceptance, or only the cost at the candidate; accept / reject.
int enqueue_step(pba_problem* p, double lambda, cudaStream_t s, int* nl, cudaEvent_t* ev = nullptr,
                 bool speculative = false) {
    // timing events (speculative timed iteration only): [1] after the solve, [5] after the accept
    if (!speculative) ev = nullptr;
    // the system in pose variables: H itself by default (the solve drops frame 0),
    // else S^T H S with a leading fixed dummy block
    const double* Hs = p->d_H;
    const double* bs = p->d_b;
    int nf = p->N, npad = p->n_pad;
    const int S = (int)p->sensors.size();
    if (p->sparse) {
        // gathered in pose variables from the pair blocks, damped, factorised and refined
        CUDA_TRY(p, launch_sparse_solve(p->sp, p->d_blocks, p->d_state, lambda, 3, p->d_rhs, s, nl));
    } else if (p->n_vars >= 0 && p->offsets_free) {
        // offset blocks from the current pair blocks (J_o = (J_i + J_j) A_o), then S^T H S
        CUDA_TRY(p, launch_offset_system(p->d_blocks, p->d_pair_Xo, p->M, p->d_pext, p->d_f_start, p->d_f_items,
                                         p->d_s_start, p->d_s_items, p->d_frame_sensor, p->d_sensor_var, p->N, S,
                                         p->d_Hfo, p->d_Hoo, p->d_bo, s));
        CUDA_TRY(p, launch_reduce_vars_offset(p->d_H, p->d_b, p->d_Hfo, p->d_Hoo, p->d_bo, p->d_frame_sensor, p->N,
                                              p->d_var_start, p->d_var_frames, p->n_vars, p->d_Hr, p->d_br, s));
        *nl += p->M > 0 ? 3 : 2;
        Hs = p->d_Hr;
        bs = p->d_br;
        nf = p->n_vars + 1;
        npad = p->n_pad_vars;
    } else if (p->n_vars >= 0) {
        CUDA_TRY(p, launch_reduce_vars(p->d_H, p->d_b, p->N, p->d_var_start, p->d_var_frames, p->n_vars, p->d_Hr,
                                       p->d_br, s));
        ++*nl;
        Hs = p->d_Hr;
        bs = p->d_br;
        nf = p->n_vars + 1;
        npad = p->n_pad_vars;
    }
    int nc = 0;
    CsGeom cg{};
    if (!p->sparse) CUDA_TRY(p, launch_lm_prepare(Hs, nf, p->d_state, lambda, s));
    if (p->sparse) {
        // solved above
    } else if (p->cfg.solver == PBA_SOLVE_MIXED && solve_cluster_plan(npad, &cg)) {
        CUDA_TRY(p, launch_solve_cluster(Hs, bs, nf, cg, p->d_state, 3, p->d_rhs, p->mixed.A32, p->mixed.D32, s));
        *nl += 2;
    } else if (p->cfg.solver != PBA_SOLVE_CHOLESKY_F64) {
        CUDA_TRY(p, launch_solve_mixed(Hs, bs, nf, npad, p->d_state, p->mixed, 3, p->d_rhs, s, &nc));
        *nl += 1 + nc;
    } else {
        CUDA_TRY(p, launch_damp(Hs, bs, nf, npad, p->d_state, p->d_A, p->d_rhs, s));
        CUDA_TRY(p, launch_cholesky(p->d_A, p->d_Dinv, npad, p->d_state, s, &nc));
        CUDA_TRY(p, launch_trsv(p->d_A, p->d_Dinv, npad, p->d_rhs, p->d_state, s));
        *nl += 3 + nc;
    }
    if (ev) CUDA_TRY(p, cudaEventRecord(ev[1], s));
    CUDA_TRY(p, launch_boxplus(p->d_poses, p->d_rhs, p->N, p->n_vars >= 0 ? p->d_frame_var : nullptr, p->d_state,
                               p->d_cand, s));
    ++*nl;
    if (p->offsets_free) {
        // candidate offsets, their per-pair / per-sensor copies, and the pixel-points
        // p_u = R_o pi^-1(u, d) + t_o of the frames they move
        CUDA_TRY(p, launch_offset_step(p->d_extr, p->d_rhs, p->d_sensor_var, S, p->d_state, p->d_extr_cand, s));
        CUDA_TRY(p, launch_offset_refresh(p->d_extr_cand, S, p->d_pf, p->d_frame_sensor, p->M, p->d_pair_Xo,
                                          p->d_sensors, s));
        CUDA_TRY(p, launch_pack(p->raw, p->d_frames, p->d_sensors, p->d_free_frames, p->n_free_frames,
                                p->cfg.texel_precision, p->tex, p->pts_pg, p->pts_n, p->pts_pix, p->d_npoints,
                                p->cfg.range_min, p->cfg.range_max, s, p->gtex, p->max_frame_px, p->d_tile_counts, p->d_valid_px));
        *nl += 3;
    }
    if (speculative) {
        int st = enqueue_linearize(p, s, nl, ev, true);
        if (st) return st;
    } else {
        CUDA_TRY(p, launch_pair_pose(p->d_cand, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, s));
        ++*nl;
        if (p->cfg.path == PBA_PATH_PLAIN) {
            CUDA_TRY(p, cudaMemsetAsync(p->d_plain_acc, 0, sizeof(float) * 96 * (size_t)p->M, s));
            for (int q = 0; q < p->M; ++q) {
                const int src = p->pairs[2 * q];
                const pba_sensor& S = p->sensors[p->frame_sensor[src]];
                CUDA_TRY(p, launch_plain(false, q, p->d_ps, p->d_pp, p->raw, p->d_sensors, p->frame_sensor[src],
                                         p->prm, p->cfg.range_min, p->cfg.range_max, p->d_plain_acc, S.width,
                                         S.height, s));
                ++*nl;
            }
            CUDA_TRY(p, launch_plain_expand(p->d_plain_acc, p->M, false, p->d_blocks_cand, s));
            ++*nl;
        } else {
            CUDA_TRY(p, cudaMemsetAsync(p->d_queue + 1, 0, sizeof(int), s));
            CUDA_TRY(p, launch_linearize(false, false, p->cfg.texel_precision, p->d_chunks, p->n_chunks,
                                         p->d_queue + 1, p->d_ps, p->d_pp, p->pts_pg, p->pts_n, p->tex, p->prm,
                                         p->d_partials, nullptr, p->grid_cost, p->variant_cost, s));
            CUDA_TRY(p, launch_pair_reduce(p->d_partials, p->d_ps, p->d_pf, p->d_cand, p->d_pair_Xo, p->M, false,
                                           p->d_blocks_cand, s));
            *nl += 2;
        }
        CUDA_TRY(p, launch_total_cost(p->d_blocks_cand, p->M, p->d_state, true, s));
        ++*nl;
    }
    CUDA_TRY(p, launch_accept(p->d_state, p->d_poses, p->d_cand, p->N, speculative,
                              p->sparse ? nullptr : p->d_H, p->d_H_cand, p->d_b, p->d_b_cand, p->d_blocks,
                              p->d_blocks_cand, p->M, s));
    *nl += speculative ? 2 : 1;
    if (p->offsets_free) {  // the accepted (or kept) offsets become current again everywhere
        CUDA_TRY(p, launch_offset_accept(p->d_state, p->d_extr, p->d_extr_cand, S, s));
        CUDA_TRY(p, launch_offset_refresh(p->d_extr, S, p->d_pf, p->d_frame_sensor, p->M, p->d_pair_Xo,
                                          p->d_sensors, s));
        CUDA_TRY(p, launch_pack(p->raw, p->d_frames, p->d_sensors, p->d_free_frames, p->n_free_frames,
                                p->cfg.texel_precision, p->tex, p->pts_pg, p->pts_n, p->pts_pix, p->d_npoints,
                                p->cfg.range_min, p->cfg.range_max, s, p->gtex, p->max_frame_px, p->d_tile_counts, p->d_valid_px));
        *nl += 3;
    }
    if (ev) CUDA_TRY(p, cudaEventRecord(ev[5], s));
    return PBA_OK;
}

int read_stats(pba_problem* p, pba_iter_stats* stats) {
    LmState st;
    CUDA_TRY(p, cudaMemcpyAsync(&st, p->d_state, sizeof st, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    if (stats) {
        stats->cost = st.iter_cost;
        stats->new_cost = st.new_cost;
        stats->lambda_used = st.lambda_used;
        stats->lambda_next = st.lambda;
        stats->n_valid = st.iter_n_valid;
        stats->n_nonfinite = st.iter_nf_res;
        stats->nonfinite_pairs = st.iter_nf_pairs;
        stats->accepted = st.accepted;
        stats->status = st.status;
    }
    return PBA_OK;
}

int ready(pba_problem* p) {
    if (!p) return PBA_EINVAL;
    if (!p->poses_set) return fail(p, PBA_ENOTREADY, "poses not set");
    if (p->M <= 0) return fail(p, PBA_ENOTREADY, "pairs not set");
    cudaSetDevice(p->device);
    return PBA_OK;
}

// Texels, pixel-points and central differences of frames first .. first+count-1 on stream s.
int pack_frames(pba_problem* p, int first, int count, cudaStream_t s) {
    CUDA_TRY(p, launch_pack(p->raw, p->d_frames, p->d_sensors, p->d_frame_iota + first, count,
                            p->cfg.texel_precision, p->tex, p->pts_pg, p->pts_n, p->pts_pix, p->d_npoints,
                            p->cfg.range_min, p->cfg.range_max, s, p->gtex, p->max_frame_px, p->d_tile_counts,
                            p->d_valid_px));
    return PBA_OK;
}

// After packing: the frames' point counts on the host, and the pair plan rebuilt
// when they changed.
int finish_repack(pba_problem* p) {
    std::vector<int> before = p->n_points;
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    CUDA_TRY(p, cudaMemcpy(p->n_points.data(), p->d_npoints, sizeof(int) * p->N, cudaMemcpyDeviceToHost));
    p->points_known = true;
    p->linearized = false;
    p->mask_valid = false;
    if (p->M > 0 && before != p->n_points) {
        // the chunk queue depends on the point counts: rebuild the pair plan
        std::vector<int32_t> keep = p->pairs;
        return pba_set_pairs(p, keep.data(), (int)(keep.size() / 2));
    }
    return PBA_OK;
}

// Optionally re-estimates the normals of frames first..first+count-1 (max_radius > 0),
// then rebuilds their texels and pixel-points and, when a point count changed, the
// pair plan.  Synchronises.
int repack(pba_problem* p, int first, int count, float scale, int max_radius) {
    if (max_radius > 0) {
        int max_px = 0;
        for (int k = 0; k < count; ++k) {
            const pba_sensor& S = p->sensors[p->frame_sensor[first + k]];
            max_px = std::max(max_px, S.width * S.height);
        }
        CUDA_TRY(p, launch_normals(p->raw, p->d_frames, p->d_frame_iota + first, count, max_px, scale, max_radius,
                                   p->cfg.range_min, p->cfg.range_max, p->stream));
    }
    int st = pack_frames(p, first, count, p->stream);
    if (st) return st;
    return finish_repack(p);
}

// The effective variables of the solve from the frames' mapping and the free
// offsets: device CSR of the blocks of each variable (frames f < N, offsets
// N + s), the frame and sensor maps used by the box-plus, Hr / br, and the list
// of frames re-packed when an offset moves.  Drops the iteration graph.
int plan_sparse(pba_problem* p);

int rebuild_vars_mapping(pba_problem* p);

// The variables of the solve changed: rebuild their mapping, then the sparse plan.
int rebuild_vars(pba_problem* p) {
    const int st = rebuild_vars_mapping(p);
    return st ? st : plan_sparse(p);
}

int rebuild_vars_mapping(pba_problem* p) {
    drop_graph(p);
    p->pyramid_stale = true;
    const int S = (int)p->sensors.size();
    p->offsets_free = false;
    for (int s = 0; s < S; ++s) p->offsets_free = p->offsets_free || p->offset_free[s];
    dfree(p->d_frame_var);
    dfree(p->d_var_start);
    dfree(p->d_var_frames);
    dfree(p->d_Hr);
    dfree(p->d_br);
    dfree(p->d_free_frames);
    p->n_free_frames = 0;
    p->n_vars = -1;
    std::vector<int> sv(S, -1);
    if (p->n_fv_user < 0 && !p->offsets_free) {
        CUDA_TRY(p, cudaMemcpy(p->d_sensor_var, sv.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
        return PBA_OK;
    }
    std::vector<int32_t> fv(p->N);
    int nf;
    if (p->n_fv_user >= 0) {
        fv = p->fv_user;
        nf = p->n_fv_user;
    } else {
        for (int k = 0; k < p->N; ++k) fv[k] = k - 1;
        nf = p->N - 1;
    }
    int n_total = nf;
    for (int s = 0; s < S; ++s)
        if (p->offset_free[s]) sv[s] = n_total++;
    if (n_total < 1) return fail(p, PBA_EINVAL, "variables: nothing to solve for");
    std::vector<int> count(n_total, 0);
    for (int k = 0; k < p->N; ++k)
        if (fv[k] >= 0) ++count[fv[k]];
    for (int s = 0; s < S; ++s)
        if (sv[s] >= 0) ++count[sv[s]];
    std::vector<int> start(n_total + 1, 0);
    for (int v = 0; v < n_total; ++v) start[v + 1] = start[v] + count[v];
    std::vector<int> fill(start.begin(), start.end() - 1), blocks(start[n_total]);
    for (int k = 0; k < p->N; ++k)
        if (fv[k] >= 0) blocks[fill[fv[k]]++] = k;
    for (int s = 0; s < S; ++s)
        if (sv[s] >= 0) blocks[fill[sv[s]]++] = p->N + s;
    std::vector<int> free_frames;
    for (int k = 0; k < p->N; ++k)
        if (p->offset_free[p->frame_sensor[k]]) free_frames.push_back(k);
    const size_t nr = 6 * (size_t)(n_total + 1);
    if (cudaMalloc((void**)&p->d_frame_var, sizeof(int) * p->N) != cudaSuccess ||
        cudaMalloc((void**)&p->d_var_start, sizeof(int) * (n_total + 1)) != cudaSuccess ||
        cudaMalloc((void**)&p->d_var_frames, sizeof(int) * std::max<size_t>(blocks.size(), 1)) != cudaSuccess ||
        cudaMalloc((void**)&p->d_Hr, sizeof(double) * nr * nr) != cudaSuccess ||
        cudaMalloc((void**)&p->d_br, sizeof(double) * nr) != cudaSuccess ||
        cudaMalloc((void**)&p->d_free_frames, sizeof(int) * std::max<size_t>(free_frames.size(), 1)) != cudaSuccess)
        return fail(p, PBA_ENOMEM, "variables: out of device memory");
    CUDA_TRY(p, cudaMemcpy(p->d_frame_var, fv.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_sensor_var, sv.data(), sizeof(int) * S, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_var_start, start.data(), sizeof(int) * (n_total + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_var_frames, blocks.data(), sizeof(int) * blocks.size(), cudaMemcpyHostToDevice));
    if (!free_frames.empty())
        CUDA_TRY(p, cudaMemcpy(p->d_free_frames, free_frames.data(), sizeof(int) * free_frames.size(),
                               cudaMemcpyHostToDevice));
    p->n_free_frames = (int)free_frames.size();
    p->n_vars = n_total;
    p->n_pad_vars = ((6 * n_total + kTile - 1) / kTile) * kTile;
    if (p->n_pad_vars > p->n_pad_alloc)
        return fail(p, PBA_EINVAL, "variables: more unknowns than the problem's solver buffers hold");
    return PBA_OK;
}

// Whether the block-sparse solve runs, and its plan: for PBA_SOLVE_SPARSE, and for
// PBA_SOLVE_MIXED when the system is too large for the one-launch cluster solve;
// not while a sensor offset is a variable (its dense coupling rows take the
// per-step launches).  The plan follows the pairs and the frames' variables.
int plan_sparse(pba_problem* p) {
    free_sparse(p);
    if (p->M <= 0 || p->offsets_free) return PBA_OK;
    if (p->cfg.solver != PBA_SOLVE_SPARSE) {
        CsGeom cg{};
        const int npad = p->n_vars >= 0 ? p->n_pad_vars : p->n_pad;
        if (p->cfg.solver != PBA_SOLVE_MIXED || solve_cluster_plan(npad, &cg)) return PBA_OK;
    }
    std::vector<int> fv(p->N);
    int nv;
    if (p->n_fv_user >= 0) {
        fv.assign(p->fv_user.begin(), p->fv_user.end());
        nv = p->n_fv_user;
    } else {
        for (int k = 0; k < p->N; ++k) fv[k] = k - 1;
        nv = p->N - 1;
    }
    const int cmax = sparse_cluster_max();
    SpPlanHost h;
    if (cmax < 1 || !sparse_plan(nv, fv, p->pairs, cmax, &h)) return PBA_OK;  // the dense solves remain
    bool ok = true;
    auto up = [&](const void* src, size_t bytes) -> void* {
        void* d = nullptr;
        if (!ok || cudaMalloc(&d, bytes ? bytes : 16) != cudaSuccess) {
            ok = false;
            return nullptr;
        }
        p->sp_mem.push_back(d);
        if (src && bytes && cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
        return d;
    };
    SpPlanDev& d = p->sp;
    d.nv = h.nv;
    d.n_rows = h.n_rows;
    d.nblk = (int)h.blk.size();
    d.n_comp = (int)h.comp_rows.size();
    d.C = h.C;
    d.n_tiles = h.n_tiles;
    d.var_of_pos = (const int*)up(h.var_of_pos.data(), sizeof(int) * h.var_of_pos.size());
    d.scal_of_pos = (const int*)up(h.scal_of_pos.data(), sizeof(int) * h.scal_of_pos.size());
    d.pos_of_scalar = (const int*)up(h.pos_of_scalar.data(), sizeof(int) * h.pos_of_scalar.size());
    d.diag_blk = (const int*)up(h.diag_blk.data(), sizeof(int) * h.diag_blk.size());
    d.blk = (const int2*)up(h.blk.data(), sizeof(int2) * h.blk.size());
    d.blk_start = (const int*)up(h.blk_start.data(), sizeof(int) * h.blk_start.size());
    d.blk_contrib = (const int4*)up(h.blk_contrib.data(), sizeof(int4) * h.blk_contrib.size());
    d.b_start = (const int*)up(h.b_start.data(), sizeof(int) * h.b_start.size());
    d.b_contrib = (const int2*)up(h.b_contrib.data(), sizeof(int2) * h.b_contrib.size());
    d.row_start = (const int*)up(h.row_start.data(), sizeof(int) * h.row_start.size());
    d.row_items = (const int2*)up(h.row_items.data(), sizeof(int2) * h.row_items.size());
    d.tile_first = (const int*)up(h.tile_first.data(), sizeof(int) * h.tile_first.size());
    d.tile_off = (const long long*)up(h.tile_off.data(), sizeof(long long) * h.tile_off.size());
    d.comp_rows = (const int2*)up(h.comp_rows.data(), sizeof(int2) * h.comp_rows.size());
    const size_t ns = (size_t)h.n_rows * kTile;
    d.Hv = (double*)up(nullptr, sizeof(double) * 36 * h.blk.size());
    d.bvec = (double*)up(nullptr, sizeof(double) * 6 * (size_t)h.nv);
    d.dsc = (double*)up(nullptr, sizeof(double) * ns);
    d.dsc32 = (float*)up(nullptr, sizeof(float) * ns);
    d.bsc = (double*)up(nullptr, sizeof(double) * ns);
    d.x = (double*)up(nullptr, sizeof(double) * ns);
    d.r64 = (double*)up(nullptr, sizeof(double) * ns);
    d.L = (float*)up(nullptr, sizeof(float) * kTile * kTile * (size_t)h.n_tiles);
    d.Dinv = (float*)up(nullptr, sizeof(float) * kTile * ns);
    d.rv = (float*)up(nullptr, sizeof(float) * ns);
    d.yv = (float*)up(nullptr, sizeof(float) * ns);
    d.zv = (float*)up(nullptr, sizeof(float) * ns);
    d.acc = (float*)up(nullptr, sizeof(float) * ns);
    d.nrm = (double*)up(nullptr, sizeof(double) * 2 * (size_t)d.n_comp * d.C);
    if (!ok) {
        free_sparse(p);
        return fail(p, PBA_ENOMEM, "sparse solve: device allocation failed");
    }
    p->sparse = true;
    return PBA_OK;
}

// The host copies of the offsets follow the device ones (refined by the solve).
int sync_offsets_to_host(pba_problem* p) {
    const int S = (int)p->sensors.size();
    std::vector<double> X(12 * (size_t)S);
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    CUDA_TRY(p, cudaMemcpy(X.data(), p->d_extr, sizeof(double) * X.size(), cudaMemcpyDeviceToHost));
    for (int s = 0; s < S; ++s)
        for (int e = 0; e < 12; ++e) p->sensors[s].extrinsic[e] = X[12 * s + e];
    return PBA_OK;
}

}  // namespace

extern "C" {

// message of the calling thread's last failed pba_create (no problem exists to hold it)
thread_local std::string t_create_err;

static int create_fail(int code, const std::string& what) {
    t_create_err = "pba_create: " + what;
    return code;
}

const char* pba_last_error(const pba_problem* p) {
    if (!p) return t_create_err.empty() ? "null problem" : t_create_err.c_str();
    return p->err.c_str();
}

// The TMA tensor maps of the staged linearisation: frame k's FP16 texels as a
// 3-D tensor (4 words, width, height; strides 16 B and 16 B x width) with a
// box of one tile (4 words x kTileCols x kTileRows), zero fill outside.  Staging
// is left off for FP32 texels and when a frame is smaller than a tile.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static int build_tile_maps(pba_problem* p) {
    p->stage_ok = false;
    p->prm.tmaps = nullptr;
    p->prm.tile_err = nullptr;
    if (p->cfg.texel_precision != PBA_TEXEL_F16) return PBA_OK;
    for (const pba_sensor& S : p->sensors)
        if (S.width < kTileCols || S.height < kTileRows) return PBA_OK;
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn)
        return fail(p, PBA_ECUDA, "create: the driver has no cuTensorMapEncodeTiled");
    const EncodeTiledFn encode = reinterpret_cast<EncodeTiledFn>(fn);
    std::vector<CUtensorMap> maps(p->N);
    for (int k = 0; k < p->N; ++k) {
        const pba_sensor& S = p->sensors[p->frame_sensor[k]];
        const cuuint64_t dims[3] = {4, (cuuint64_t)S.width, (cuuint64_t)S.height};
        const cuuint64_t strides[2] = {16, 16ull * (cuuint64_t)S.width};
        const cuuint32_t box[3] = {4, (cuuint32_t)kTileCols, (cuuint32_t)kTileRows};
        const cuuint32_t elem[3] = {1, 1, 1};
        void* base = reinterpret_cast<char*>(p->tex) + 16ll * p->px_off[k];
        if (encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, base, dims, strides, box, elem,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return fail(p, PBA_ECUDA, "create: cuTensorMapEncodeTiled refused a frame's texels");
    }
    CUDA_TRY(p, cudaMalloc((void**)&p->d_tmaps, sizeof(CUtensorMap) * (size_t)p->N));
    CUDA_TRY(p, cudaMalloc((void**)&p->d_tile_err, sizeof(int)));
    CUDA_TRY(p, cudaMemcpy(p->d_tmaps, maps.data(), sizeof(CUtensorMap) * (size_t)p->N, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemset(p->d_tile_err, 0, sizeof(int)));
    p->prm.tmaps = p->d_tmaps;
    p->prm.tile_err = p->d_tile_err;
    p->stage_ok = true;
    return PBA_OK;
}

int pba_create(const pba_config* cfg, void* cuda_stream, pba_problem** out) {
    if (!cfg || !out) return create_fail(PBA_EINVAL, "null configuration or output pointer");
    *out = nullptr;
    if (cfg->n_frames < 1 || cfg->n_sensors < 1 || !cfg->sensors)
        return create_fail(PBA_EINVAL, "n_frames and n_sensors must be >= 1 with a sensor array");
    if (!(cfg->huber_delta > 0.0)) return create_fail(PBA_EINVAL, "huber_delta must be > 0");
    if (cfg->grad_mode != 0 && cfg->grad_mode != 1) return create_fail(PBA_EINVAL, "grad_mode must be 0 or 1");
    if (cfg->texel_precision != 0 && cfg->texel_precision != 1)
        return create_fail(PBA_EINVAL, "texel_precision must be PBA_TEXEL_F32 or PBA_TEXEL_F16");
    if (cfg->path != PBA_PATH_BATCHED && cfg->path != PBA_PATH_PLAIN) return create_fail(PBA_EINVAL, "unknown path");
    if (cfg->solver != PBA_SOLVE_CHOLESKY_F64 && cfg->solver != PBA_SOLVE_MIXED &&
        cfg->solver != PBA_SOLVE_MIXED_STEPS && cfg->solver != PBA_SOLVE_SPARSE)
        return create_fail(PBA_EINVAL, "unknown solver");
    for (int s = 0; s < cfg->n_sensors; ++s) {
        const pba_sensor& S = cfg->sensors[s];
        if ((S.model != PBA_PINHOLE && S.model != PBA_SPHERICAL) || S.width < 4 || S.height < 4)
            return create_fail(PBA_EINVAL, "sensor " + std::to_string(s) + ": unknown model or image below 4 x 4");
        if (S.fx == 0.0 || S.fy == 0.0) return create_fail(PBA_EINVAL, "sensor " + std::to_string(s) + ": zero focal length");
        if ((long long)S.width * S.height > (1LL << 30))
            return create_fail(PBA_EINVAL, "sensor " + std::to_string(s) + ": more than 2^30 pixels");
    }
    if (cfg->frame_sensor)
        for (int k = 0; k < cfg->n_frames; ++k)
            if (cfg->frame_sensor[k] < 0 || cfg->frame_sensor[k] >= cfg->n_sensors)
                return create_fail(PBA_EINVAL, "frame_sensor[" + std::to_string(k) + "] out of range");
    {
        int n_dev = 0;
        const cudaError_t e = cudaGetDeviceCount(&n_dev);
        if (e != cudaSuccess || n_dev < 1) {
            const std::string why = e != cudaSuccess ? cudaGetErrorString(e) : "no CUDA device";
            cudaGetLastError();
            return create_fail(PBA_ECUDA, "no usable CUDA device (" + why + "); the library has no CPU path");
        }
    }
    pba_problem* p = new pba_problem();
    p->cfg = *cfg;
    p->N = cfg->n_frames;
    p->sensors.assign(cfg->sensors, cfg->sensors + cfg->n_sensors);
    p->cfg.sensors = nullptr;
    p->frame_sensor.assign(p->N, 0);
    if (cfg->frame_sensor)
        for (int k = 0; k < p->N; ++k) p->frame_sensor[k] = cfg->frame_sensor[k];  // checked above
    p->cfg.frame_sensor = nullptr;
    cudaGetDevice(&p->device);
    auto bail = [&](int code) {
        const cudaError_t e = cudaGetLastError();
        pba_destroy(p);
        return create_fail(code, std::string(code == PBA_ENOMEM ? "device allocation failed" : "CUDA call failed") +
                                     (e != cudaSuccess ? std::string(" (") + cudaGetErrorString(e) + ")" : ""));
    };
    if (cuda_stream) {
        p->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PBA_ECUDA);
        p->stream = p->own_stream;
    }
    if (cudaStreamCreateWithFlags(&p->capture_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(PBA_ECUDA);

    p->px_off.resize(p->N);
    long long off = 0;
    for (int k = 0; k < p->N; ++k) {
        const pba_sensor& S = p->sensors[p->frame_sensor[k]];
        p->px_off[k] = off;
        off += (long long)S.width * S.height;
    }
    p->total_px = off;
    p->n_points.assign(p->N, 0);
    p->uploaded.assign(p->N, 0);

    const size_t texel_bytes = cfg->texel_precision == PBA_TEXEL_F16 ? sizeof(Tex16) : sizeof(Tex32);
    const int n6 = 6 * p->N;
    const int n = n6 - 6;
    p->n_pad = ((n + kTile - 1) / kTile) * kTile;
    if (p->n_pad == 0) p->n_pad = kTile;
    // the solver's buffers also hold the variables of free offsets (6 per sensor)
    const int S = (int)p->sensors.size();
    p->n_pad_alloc = ((n + 6 * S + kTile - 1) / kTile) * kTile;
    p->offset_free.assign(S, 0);
    auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, bytes ? bytes : 16) == cudaSuccess; };
    bool ok = alloc((void**)&p->raw, sizeof(float) * 5 * (size_t)p->total_px) &&
              alloc(&p->tex, texel_bytes * (size_t)p->total_px) &&
              alloc((void**)&p->gtex, sizeof(float4) * 3 * (size_t)p->total_px) &&
              alloc((void**)&p->d_valid_px, (size_t)p->total_px) &&
              alloc((void**)&p->pts_pg, sizeof(float4) * (size_t)p->total_px) &&
              alloc((void**)&p->pts_n, sizeof(float4) * (size_t)p->total_px) &&
              alloc((void**)&p->pts_pix, sizeof(int) * (size_t)p->total_px) &&
              alloc((void**)&p->d_frame_sensor, sizeof(int) * p->N) &&
              alloc((void**)&p->d_npoints, sizeof(int) * p->N) &&
              alloc((void**)&p->d_frames, sizeof(FrameInfo) * p->N) &&
              alloc((void**)&p->d_sensors, sizeof(SensorDev) * p->sensors.size()) &&
              alloc((void**)&p->d_frame_ids, sizeof(int) * p->N) &&
              alloc((void**)&p->d_poses, sizeof(double) * 12 * p->N) &&
              alloc((void**)&p->d_cand, sizeof(double) * 12 * p->N) &&
              alloc((void**)&p->d_state, sizeof(LmState)) &&
              alloc((void**)&p->d_H, sizeof(double) * (size_t)n6 * n6) &&
              alloc((void**)&p->d_b, sizeof(double) * n6) &&
              alloc((void**)&p->d_H_cand, sizeof(double) * (size_t)n6 * n6) &&
              alloc((void**)&p->d_b_cand, sizeof(double) * n6) &&
              alloc((void**)&p->d_A, sizeof(double) * (size_t)p->n_pad_alloc * p->n_pad_alloc) &&
              alloc((void**)&p->d_rhs, sizeof(double) * p->n_pad_alloc) &&
              alloc((void**)&p->d_Dinv, sizeof(double) * (size_t)p->n_pad_alloc * kTile) &&
              alloc((void**)&p->d_extr, sizeof(double) * 12 * S) &&
              alloc((void**)&p->d_extr_cand, sizeof(double) * 12 * S) &&
              alloc((void**)&p->d_sensor_var, sizeof(int) * S) &&
              alloc((void**)&p->d_Hfo, sizeof(double) * 36 * (size_t)p->N) &&
              alloc((void**)&p->d_Hoo, sizeof(double) * 36 * S) &&
              alloc((void**)&p->d_bo, sizeof(double) * 6 * S) &&
              alloc((void**)&p->d_queue, sizeof(int) * 2) &&
              (cfg->solver == PBA_SOLVE_CHOLESKY_F64 ||
               (alloc((void**)&p->mixed.A32, sizeof(float) * (size_t)p->n_pad_alloc * p->n_pad_alloc) &&
                alloc((void**)&p->mixed.D32, sizeof(float) * (size_t)p->n_pad_alloc * kTile) &&
                alloc((void**)&p->mixed.r32, sizeof(float) * p->n_pad_alloc) &&
                alloc((void**)&p->mixed.bs, sizeof(double) * p->n_pad_alloc) &&
                alloc((void**)&p->mixed.x, sizeof(double) * p->n_pad_alloc) &&
                alloc((void**)&p->mixed.dscale, sizeof(double) * p->n_pad_alloc) &&
                alloc((void**)&p->mixed.norms, sizeof(double) * 2)));
    if (!ok) return bail(PBA_ENOMEM);
    // cluster limits of the one-launch mixed solve, queried here (outside any stream capture)
    if (cfg->solver == PBA_SOLVE_MIXED) solve_cluster_init();
    if (cfg->solver == PBA_SOLVE_MIXED || cfg->solver == PBA_SOLVE_SPARSE) sparse_cluster_max();

    std::vector<FrameInfo> fi(p->N);
    for (int k = 0; k < p->N; ++k) {
        const pba_sensor& S = p->sensors[p->frame_sensor[k]];
        fi[k].width = S.width;
        fi[k].height = S.height;
        fi[k].sensor = p->frame_sensor[k];
        fi[k].model = S.model;
        fi[k].fx = (float)S.fx;
        fi[k].fy = (float)S.fy;
        fi[k].cx = (float)S.cx;
        fi[k].cy = (float)S.cy;
        fi[k].px_offset = p->px_off[k];
        fi[k].pt_offset = p->px_off[k];
    }
    std::vector<SensorDev> sd(p->sensors.size());
    for (size_t s = 0; s < p->sensors.size(); ++s) {
        const pba_sensor& S = p->sensors[s];
        for (int r = 0; r < 3; ++r) {
            for (int c = 0; c < 3; ++c) sd[s].R[3 * r + c] = (float)S.extrinsic[4 * r + c];
            sd[s].t[r] = (float)S.extrinsic[4 * r + 3];
        }
        sd[s].model = S.model;
        sd[s].width = S.width;
        sd[s].height = S.height;
        sd[s].fx = (float)S.fx;
        sd[s].fy = (float)S.fy;
        sd[s].cx = (float)S.cx;
        sd[s].cy = (float)S.cy;
    }
    LmState st{};
    st.lambda = -1.0;
    std::vector<double> ex(12 * p->sensors.size());
    for (size_t s = 0; s < p->sensors.size(); ++s)
        for (int e = 0; e < 12; ++e) ex[12 * s + e] = p->sensors[s].extrinsic[e];
    std::vector<int> no_var(p->sensors.size(), -1);
    if (cudaMemcpy(p->d_extr, ex.data(), sizeof(double) * ex.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_extr_cand, ex.data(), sizeof(double) * ex.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_sensor_var, no_var.data(), sizeof(int) * no_var.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(p->d_frames, fi.data(), sizeof(FrameInfo) * p->N, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_sensors, sd.data(), sizeof(SensorDev) * sd.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(p->d_frame_sensor, p->frame_sensor.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(p->d_state, &st, sizeof st, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(p->d_npoints, 0, sizeof(int) * p->N) != cudaSuccess ||
        cudaMemset(p->d_H, 0, sizeof(double) * (size_t)n6 * n6) != cudaSuccess ||
        cudaMemset(p->d_b, 0, sizeof(double) * n6) != cudaSuccess)
        return bail(PBA_ECUDA);

    p->prm.w_int = (float)cfg->w_int;
    p->prm.w_depth = (float)cfg->w_depth;
    p->prm.w_normal = (float)cfg->w_normal;
    p->prm.huber_delta = (float)cfg->huber_delta;
    p->prm.huber_delta2 = (float)(cfg->huber_delta * cfg->huber_delta);
    p->prm.occ_abs = (float)cfg->occ_abs;
    p->prm.occ_rel = (float)cfg->occ_rel;
    p->prm.z_min = (float)cfg->z_min;
    p->prm.grad_mode = cfg->grad_mode;
    p->prm.gtex = p->gtex;
    for (const pba_sensor& S : p->sensors) p->max_frame_px = std::max(p->max_frame_px, S.width * S.height);
    if (!alloc((void**)&p->d_tile_counts, sizeof(int) * (size_t)p->N * pack_tiles(p->max_frame_px)) ||
        !alloc((void**)&p->d_frame_iota, sizeof(int) * (size_t)p->N))
        return bail(PBA_ENOMEM);
    {
        std::vector<int> iota(p->N);
        for (int k = 0; k < p->N; ++k) iota[k] = k;
        if (cudaMemcpy(p->d_frame_iota, iota.data(), sizeof(int) * p->N, cudaMemcpyHostToDevice) != cudaSuccess)
            return bail(PBA_ECUDA);
    }
    if (int st = build_tile_maps(p)) {
        const std::string what = p->err;
        pba_destroy(p);
        return create_fail(st, what);
    }
    p->grid_full = linearize_grid(cfg->texel_precision, true, 0);
    p->grid_cost = linearize_grid(cfg->texel_precision, false, 0);
    *out = p;
    return PBA_OK;
}

void pba_destroy(pba_problem* p) {
    if (!p) return;
    cudaSetDevice(p->device);
    if (p->stream) cudaStreamSynchronize(p->stream);
    for (pba_problem* q : p->levels) pba_destroy(q);
    p->levels.clear();
    drop_graph(p);
    dfree(p->d_frame_var);
    dfree(p->d_var_start);
    dfree(p->d_var_frames);
    dfree(p->d_Hr);
    dfree(p->d_br);
    dfree(p->d_sensor_var);
    dfree(p->d_free_frames);
    dfree(p->d_extr);
    dfree(p->d_extr_cand);
    dfree(p->d_Hfo);
    dfree(p->d_Hoo);
    dfree(p->d_bo);
    free_sparse(p);
    free_pair_buffers(p);
    dfree(p->raw);
    dfree(p->tex);
    dfree(p->gtex);
    dfree(p->d_tile_counts);
    dfree(p->d_valid_px);
    dfree(p->d_frame_iota);
    dfree(p->pts_pg);
    dfree(p->pts_n);
    dfree(p->pts_pix);
    dfree(p->d_frame_sensor);
    dfree(p->d_npoints);
    dfree(p->d_frames);
    dfree(p->d_sensors);
    dfree(p->d_frame_ids);
    dfree(p->d_poses);
    dfree(p->d_cand);
    dfree(p->d_state);
    dfree(p->d_H);
    dfree(p->d_b);
    dfree(p->d_H_cand);
    dfree(p->d_b_cand);
    dfree(p->d_A);
    dfree(p->d_rhs);
    dfree(p->d_Dinv);
    dfree(p->d_queue);
    dfree(p->mixed.A32);
    dfree(p->mixed.D32);
    dfree(p->mixed.r32);
    dfree(p->mixed.bs);
    dfree(p->mixed.x);
    dfree(p->mixed.dscale);
    dfree(p->mixed.norms);
    if (p->capture_stream) cudaStreamDestroy(p->capture_stream);
    for (cudaStream_t& c : p->copy_streams)
        if (c) cudaStreamDestroy(c);
    for (cudaEvent_t& e : p->copy_events)
        if (e) cudaEventDestroy(e);
    dfree(p->d_chunks_ready);
    dfree(p->d_seg_queue);
    dfree(p->d_tmaps);
    dfree(p->d_tile_err);
    if (p->h_counts) cudaFreeHost(p->h_counts);
    for (cudaStream_t c : {p->lane_copy, p->lane_pack})
        if (c) cudaStreamDestroy(c);
    if (p->lane_start) cudaEventDestroy(p->lane_start);
    for (int l = 0; l < p->kFrameLanes; ++l) {
        if (p->lane_copied[l]) cudaEventDestroy(p->lane_copied[l]);
        if (p->lane_ready[l]) cudaEventDestroy(p->lane_ready[l]);
    }
    if (p->own_stream) cudaStreamDestroy(p->own_stream);
    delete p;
}

int pba_set_stream(pba_problem* p, void* cuda_stream) {
    if (!p) return PBA_EINVAL;
    p->stream = cuda_stream ? (cudaStream_t)cuda_stream : p->own_stream;
    if (!p->stream) {
        CUDA_TRY(p, cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking));
        p->stream = p->own_stream;
    }
    return PBA_OK;
}

int pba_upload_frames(pba_problem* p, int first, int count, const float* channels, int is_device) {
    if (!p) return PBA_EINVAL;
    if (!channels || count < 1 || first < 0 || first + count > p->N)
        return fail(p, PBA_EINVAL, "upload: bad frame range or null channels");
    cudaSetDevice(p->device);
    const pba_sensor& S0 = p->sensors[p->frame_sensor[first]];
    for (int k = first; k < first + count; ++k) {
        const pba_sensor& S = p->sensors[p->frame_sensor[k]];
        if (S.width != S0.width || S.height != S0.height)
            return fail(p, PBA_EINVAL, "upload: frames of one call must share the image size");
    }
    const size_t frame_bytes = sizeof(float) * 5 * (size_t)S0.width * S0.height;
    const size_t bytes = frame_bytes * count;
    float* dst = p->raw + 5 * p->px_off[first];
    const int lanes = std::min(p->kCopyLanes, count);
    for (int k = first; k < first + count; ++k) p->uploaded[k] = 1;
    p->pyramid_stale = true;
    if (is_device || bytes < ((size_t)16 << 20) || lanes < 2) {
        CUDA_TRY(p, cudaMemcpyAsync(dst, channels, bytes,
                                    is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
        return repack(p, first, count, 0.f, 0);
    }
    // large host uploads: the frames are split into lanes of whole frames, each
    // copied and packed on its own stream (one copy keeps one copy engine busy,
    // and a lane's packing runs while the other lanes still copy), joined back
    // into the problem's stream
    if (!p->copy_events[0]) {
        for (cudaStream_t& c : p->copy_streams) CUDA_TRY(p, cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
        for (cudaEvent_t& e : p->copy_events) CUDA_TRY(p, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    CUDA_TRY(p, cudaEventRecord(p->copy_events[0], p->stream));
    for (int l = 0; l < lanes; ++l) {
        const int f0 = first + (int)((long long)count * l / lanes), f1 = first + (int)((long long)count * (l + 1) / lanes);
        cudaStream_t cs = l == 0 ? p->stream : p->copy_streams[l - 1];
        if (l > 0) CUDA_TRY(p, cudaStreamWaitEvent(cs, p->copy_events[0], 0));
        CUDA_TRY(p, cudaMemcpyAsync(reinterpret_cast<char*>(dst) + frame_bytes * (f0 - first),
                                    reinterpret_cast<const char*>(channels) + frame_bytes * (f0 - first),
                                    frame_bytes * (f1 - f0), cudaMemcpyHostToDevice, cs));
        int st = pack_frames(p, f0, f1 - f0, cs);
        if (st) return st;
        if (l > 0) {
            CUDA_TRY(p, cudaEventRecord(p->copy_events[l], cs));
            CUDA_TRY(p, cudaStreamWaitEvent(p->stream, p->copy_events[l], 0));
        }
    }
    return finish_repack(p);
}

int pba_estimate_normals(pba_problem* p, int first, int count, float scale, int max_radius) {
    if (!p) return PBA_EINVAL;
    if (count < 1 || first < 0 || first + count > p->N)
        return fail(p, PBA_EINVAL, "estimate_normals: bad frame range");
    if (!(scale >= 0.f) || !(scale < 1e30f) || max_radius < 2 || max_radius > PBA_NORMALS_MAX_RADIUS)
        return fail(p, PBA_EINVAL, "estimate_normals: scale must be finite and >= 0, max_radius in [2, 32]");
    for (int k = first; k < first + count; ++k) {
        const pba_sensor& S = p->sensors[p->frame_sensor[k]];
        if (S.model == PBA_SPHERICAL && 2 * max_radius + 1 > S.width)
            return fail(p, PBA_EINVAL, "estimate_normals: spherical image narrower than the neighbourhood");
        if (!p->uploaded[k]) return fail(p, PBA_ENOTREADY, "estimate_normals: frame not uploaded");
    }
    cudaSetDevice(p->device);
    p->pyramid_stale = true;
    return repack(p, first, count, scale, max_radius);
}

int pba_get_channels(pba_problem* p, int first, int count, float* channels, int is_device) {
    if (!p) return PBA_EINVAL;
    if (!channels || count < 1 || first < 0 || first + count > p->N)
        return fail(p, PBA_EINVAL, "get_channels: bad frame range or null output");
    for (int k = first; k < first + count; ++k)
        if (!p->uploaded[k]) return fail(p, PBA_ENOTREADY, "get_channels: frame not uploaded");
    cudaSetDevice(p->device);
    const long long end = first + count < p->N ? p->px_off[first + count] : p->total_px;
    const size_t bytes = sizeof(float) * 5 * (size_t)(end - p->px_off[first]);
    CUDA_TRY(p, cudaMemcpyAsync(channels, p->raw + 5 * p->px_off[first], bytes,
                                is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_set_extrinsic(pba_problem* p, int sensor, const double* extrinsic) {
    if (!p || !extrinsic || sensor < 0 || sensor >= (int)p->sensors.size())
        return fail(p, PBA_EINVAL, "set_extrinsic: bad argument");
    cudaSetDevice(p->device);
    int sst = sync_offsets_to_host(p);
    if (sst) return sst;
    pba_sensor& S = p->sensors[sensor];
    for (int e = 0; e < 12; ++e) S.extrinsic[e] = extrinsic[e];
    CUDA_TRY(p, cudaMemcpyAsync(p->d_extr + 12 * sensor, S.extrinsic, sizeof(double) * 12, cudaMemcpyHostToDevice,
                                p->stream));
    CUDA_TRY(p, cudaMemcpyAsync(p->d_extr_cand + 12 * sensor, S.extrinsic, sizeof(double) * 12,
                                cudaMemcpyHostToDevice, p->stream));
    SensorDev sd{};
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) sd.R[3 * r + c] = (float)S.extrinsic[4 * r + c];
        sd.t[r] = (float)S.extrinsic[4 * r + 3];
    }
    sd.model = S.model;
    sd.width = S.width;
    sd.height = S.height;
    sd.fx = (float)S.fx;
    sd.fy = (float)S.fy;
    sd.cx = (float)S.cx;
    sd.cy = (float)S.cy;
    CUDA_TRY(p, cudaMemcpyAsync(p->d_sensors + sensor, &sd, sizeof sd, cudaMemcpyHostToDevice, p->stream));
    // the points p_u = R_o pi^-1(u, d) + t_o of this sensor's uploaded frames are rebuilt
    std::vector<int> ids;
    for (int k = 0; k < p->N; ++k)
        if (p->frame_sensor[k] == sensor && p->uploaded[k]) ids.push_back(k);
    if (!ids.empty()) {
        CUDA_TRY(p, cudaMemcpyAsync(p->d_frame_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice,
                                    p->stream));
        CUDA_TRY(p, launch_pack(p->raw, p->d_frames, p->d_sensors, p->d_frame_ids, (int)ids.size(),
                                p->cfg.texel_precision, p->tex, p->pts_pg, p->pts_n, p->pts_pix, p->d_npoints,
                                p->cfg.range_min, p->cfg.range_max, p->stream, p->gtex, p->max_frame_px, p->d_tile_counts, p->d_valid_px));
    }
    // per-pair copies of the extrinsic
    if (p->M > 0) {
        std::vector<double> pxo(12 * (size_t)p->M);
        for (int q = 0; q < p->M; ++q) {
            const pba_sensor& Sq = p->sensors[p->frame_sensor[p->pairs[2 * q]]];
            for (int e = 0; e < 12; ++e) pxo[12 * q + e] = Sq.extrinsic[e];
        }
        CUDA_TRY(p, cudaMemcpyAsync(p->d_pair_Xo, pxo.data(), sizeof(double) * pxo.size(), cudaMemcpyHostToDevice,
                                    p->stream));
    }
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));  // host vectors above are pageable
    p->linearized = false;
    p->mask_valid = false;
    p->pyramid_stale = true;
    return PBA_OK;
}

int pba_frame_points(pba_problem* p, int frame, int32_t* n_points) {
    if (!p || !n_points || frame < 0 || frame >= p->N) return fail(p, PBA_EINVAL, "frame_points: bad argument");
    if (!p->uploaded[frame]) return fail(p, PBA_ENOTREADY, "frame not uploaded");
    cudaSetDevice(p->device);
    int st = ensure_points(p);
    if (st) return st;
    *n_points = p->n_points[frame];
    return PBA_OK;
}

int pba_set_poses(pba_problem* p, const double* poses, int is_device) {
    if (!p || !poses) return fail(p, PBA_EINVAL, "set_poses: null");
    cudaSetDevice(p->device);
    CUDA_TRY(p, cudaMemcpyAsync(p->d_poses, poses, sizeof(double) * 12 * p->N,
                                is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, p->stream));
    if (!is_device) CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    p->poses_set = true;
    p->linearized = false;
    return PBA_OK;
}

int pba_get_poses(pba_problem* p, double* poses) {
    if (!p || !poses) return fail(p, PBA_EINVAL, "get_poses: null");
    cudaSetDevice(p->device);
    CUDA_TRY(p, cudaMemcpyAsync(poses, p->d_poses, sizeof(double) * 12 * p->N, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_set_pairs(pba_problem* p, const int32_t* pairs, int m) {
    if (!p || (!pairs && m > 0) || m < 0) return fail(p, PBA_EINVAL, "set_pairs: bad argument");
    cudaSetDevice(p->device);
    for (int q = 0; q < m; ++q) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        if (i < 0 || j < 0 || i >= p->N || j >= p->N) return fail(p, PBA_EINVAL, "set_pairs: frame out of range");
        if (p->frame_sensor[i] != p->frame_sensor[j])
            return fail(p, PBA_EINVAL, "set_pairs: pair frames use different sensors");
        if (!p->uploaded[i] || !p->uploaded[j]) return fail(p, PBA_ENOTREADY, "set_pairs: frame not uploaded");
    }
    int st = ensure_points(p);
    if (st) return st;
    if ((st = sync_offsets_to_host(p))) return st;
    drop_graph(p);
    p->pyramid_stale = true;
    free_pair_buffers(p);
    p->pairs.assign(pairs, pairs + 2 * (size_t)m);
    p->M = m;
    p->linearized = false;
    p->mask_valid = false;
    if (m == 0) return PBA_OK;

    // processing order: by target frame (its texels stay in L2), then source
    std::vector<int> order(m);
    for (int q = 0; q < m; ++q) order[q] = q;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        if (pairs[2 * a + 1] != pairs[2 * b + 1]) return pairs[2 * a + 1] < pairs[2 * b + 1];
        return pairs[2 * a] < pairs[2 * b];
    });
    std::vector<PairStatic> ps(m);
    std::vector<int2> pf(m);
    std::vector<double> pxo(12 * (size_t)m);
    std::vector<int4> chunks;
    p->mask_off.assign(m, 0);
    p->pair_src_points.assign(m, 0);
    long long mask_words = 0;
    for (int q = 0; q < m; ++q) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        const pba_sensor& S = p->sensors[p->frame_sensor[i]];
        PairStatic& P = ps[q];
        P.src = i;
        P.tgt = j;
        P.model = S.model;
        P.width = S.width;
        P.height = S.height;
        P.n_points = p->n_points[i];
        P.fx = (float)S.fx;
        P.fxh = (float)(S.fx * (0.5 * kPi));
        P.fxp = (float)(S.fx * kPi);
        P.fy = (float)S.fy;
        P.cx = (float)S.cx;
        P.cy = (float)S.cy;
        P.src_pt_offset = p->px_off[i];
        P.tgt_px_offset = p->px_off[j];
        P.src_px_offset = p->px_off[i];
        P.src_width = S.width;
        P.src_height = S.height;
        P.mask_offset = mask_words;
        p->mask_off[q] = mask_words;
        p->pair_src_points[q] = P.n_points;
        mask_words += (P.n_points + 31) / 32;
        pf[q] = make_int2(i, j);
        for (int e = 0; e < 12; ++e) pxo[12 * q + e] = S.extrinsic[e];
    }
    // the queue hands items out in order; about one item per resident warp at its
    // end is cut into short ones, so that the last warps to finish are not left
    // with a whole long item while the others idle
    long long total_pts = 0;
    for (int q = 0; q < m; ++q) total_pts += ps[q].n_points;
    const long long resident = (long long)std::max(p->grid_full, 1) * (kLinThreads / 32);
    const long long tail_start = total_pts - std::min(total_pts / 4, resident * p->chunk);
    long long done_pts = 0;
    for (int oi = 0; oi < m; ++oi) {
        const int q = order[oi];
        ps[q].chunk_begin = (int)chunks.size();
        for (int s = 0; s < ps[q].n_points;) {
            const int size = done_pts + s >= tail_start ? p->chunk_tail : p->chunk;
            const int n = std::min(size, ps[q].n_points - s);
            chunks.push_back(make_int4(q, s, n, (int)chunks.size()));  // pair, first point, count, slot
            s += n;
        }
        done_pts += ps[q].n_points;
        ps[q].chunk_end = (int)chunks.size();
    }
    p->n_chunks = (int)chunks.size();

    // assembly tasks: one per diagonal block and per unordered frame pair
    std::map<std::pair<int, int>, std::vector<AsmContrib>> tasks;
    for (int q = 0; q < m; ++q) {
        const int i = pairs[2 * q], j = pairs[2 * q + 1];
        // roles: 0 = i (rows/cols 0-5 of the pair block), 1 = j
        const int fr[2] = {i, j};
        for (int rr = 0; rr < 2; ++rr)
            for (int cc = 0; cc < 2; ++cc) {
                const int a = fr[rr], b = fr[cc];
                if (a > b) continue;  // the transpose is written by the (b, a) contribution's task
                tasks[{a, b}].push_back(AsmContrib{q, rr, cc, rr == cc ? 1 : 0});
            }
    }
    std::vector<AsmTask> tv;
    std::vector<AsmContrib> cv;
    for (auto& kv : tasks) {
        AsmTask T;
        T.a = kv.first.first;
        T.b = kv.first.second;
        T.contrib_begin = (int)cv.size();
        for (auto& c : kv.second) cv.push_back(c);
        T.contrib_end = (int)cv.size();
        tv.push_back(T);
    }
    p->n_tasks = (int)tv.size();

    // pair lists by frame ((pair, role) with role 0 = source, 1 = target) and by sensor
    const int S = (int)p->sensors.size();
    std::vector<int> f_start(p->N + 1, 0), s_start(S + 1, 0);
    for (int q = 0; q < m; ++q) {
        ++f_start[pairs[2 * q] + 1];
        ++f_start[pairs[2 * q + 1] + 1];
        ++s_start[p->frame_sensor[pairs[2 * q]] + 1];
    }
    for (int k = 0; k < p->N; ++k) f_start[k + 1] += f_start[k];
    for (int s = 0; s < S; ++s) s_start[s + 1] += s_start[s];
    std::vector<int2> f_items(2 * (size_t)m);
    std::vector<int> s_items(m);
    {
        std::vector<int> ff(f_start.begin(), f_start.end() - 1), sf(s_start.begin(), s_start.end() - 1);
        for (int q = 0; q < m; ++q) {
            f_items[ff[pairs[2 * q]]++] = make_int2(q, 0);
            f_items[ff[pairs[2 * q + 1]]++] = make_int2(q, 1);
            s_items[sf[p->frame_sensor[pairs[2 * q]]]++] = q;
        }
    }

    auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, bytes ? bytes : 16) == cudaSuccess; };
    bool ok = alloc((void**)&p->d_ps, sizeof(PairStatic) * m) && alloc((void**)&p->d_pp, sizeof(PairPose) * m) &&
              alloc((void**)&p->d_pf, sizeof(int2) * m) && alloc((void**)&p->d_pair_Xo, sizeof(double) * 12 * m) &&
              alloc((void**)&p->d_chunks, sizeof(int4) * chunks.size()) &&
              alloc((void**)&p->d_partials, sizeof(float) * kPartialStride * chunks.size()) &&
              alloc((void**)&p->d_blocks, sizeof(double) * kBlockStride * m) &&
              alloc((void**)&p->d_blocks_cand, sizeof(double) * kBlockStride * m) &&
              alloc((void**)&p->d_tasks, sizeof(AsmTask) * tv.size()) &&
              alloc((void**)&p->d_contrib, sizeof(AsmContrib) * cv.size()) &&
              alloc((void**)&p->d_mask, sizeof(uint32_t) * (size_t)mask_words) &&
              alloc((void**)&p->d_plain_acc, sizeof(float) * 96 * m) &&
              alloc((void**)&p->d_adj_partials, sizeof(float) * adjoint_partial_stride() * chunks.size()) &&
              alloc((void**)&p->d_adj_pair, sizeof(double) * adjoint_pair_stride() * m) &&
              alloc((void**)&p->d_adj_totals, sizeof(double) * 2) &&
              alloc((void**)&p->d_pext, sizeof(double) * 114 * m) &&
              alloc((void**)&p->d_f_start, sizeof(int) * (p->N + 1)) &&
              alloc((void**)&p->d_f_items, sizeof(int2) * 2 * m) &&
              alloc((void**)&p->d_s_start, sizeof(int) * (S + 1)) &&
              alloc((void**)&p->d_s_items, sizeof(int) * m);
    if (!ok) {
        free_pair_buffers(p);
        return fail(p, PBA_ENOMEM, "set_pairs: device allocation failed");
    }
    CUDA_TRY(p, cudaMemcpy(p->d_ps, ps.data(), sizeof(PairStatic) * m, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_pf, pf.data(), sizeof(int2) * m, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_pair_Xo, pxo.data(), sizeof(double) * 12 * m, cudaMemcpyHostToDevice));
    if (!chunks.empty())
        CUDA_TRY(p, cudaMemcpy(p->d_chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_tasks, tv.data(), sizeof(AsmTask) * tv.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_contrib, cv.data(), sizeof(AsmContrib) * cv.size(), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_f_start, f_start.data(), sizeof(int) * (p->N + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_f_items, f_items.data(), sizeof(int2) * 2 * m, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_s_start, s_start.data(), sizeof(int) * (S + 1), cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemcpy(p->d_s_items, s_items.data(), sizeof(int) * m, cudaMemcpyHostToDevice));
    CUDA_TRY(p, cudaMemset(p->d_blocks, 0, sizeof(double) * kBlockStride * m));
    CUDA_TRY(p, cudaMemset(p->d_blocks_cand, 0, sizeof(double) * kBlockStride * m));
    const int n6 = 6 * p->N;
    CUDA_TRY(p, cudaMemset(p->d_H, 0, sizeof(double) * (size_t)n6 * n6));
    CUDA_TRY(p, cudaMemset(p->d_b, 0, sizeof(double) * n6));
    CUDA_TRY(p, cudaMemset(p->d_H_cand, 0, sizeof(double) * (size_t)n6 * n6));
    CUDA_TRY(p, cudaMemset(p->d_b_cand, 0, sizeof(double) * n6));
    return plan_sparse(p);
}

int pba_build_pairs(pba_problem* p, double max_angle, double max_dist, double min_ratio, int sequential,
                    int32_t* pairs_out, float* ratio_out, int cap, int32_t* m_out) {
    if (!p || !m_out || cap < 0) return fail(p, PBA_EINVAL, "build_pairs: bad argument");
    if (!p->poses_set) return fail(p, PBA_ENOTREADY, "build_pairs: poses not set");
    for (int k = 0; k < p->N; ++k)
        if (!p->uploaded[k]) return fail(p, PBA_ENOTREADY, "build_pairs: frame not uploaded");
    cudaSetDevice(p->device);
    std::vector<double> X(12 * (size_t)p->N);
    CUDA_TRY(p, cudaMemcpyAsync(X.data(), p->d_poses, sizeof(double) * X.size(), cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    // candidates: rotation angle of R_i^T R_j and |t_i - t_j| (FP64)
    std::vector<int32_t> cand;
    std::vector<char> seq;
    for (int i = 0; i < p->N; ++i)
        for (int j = i + 1; j < p->N; ++j) {
            if (p->frame_sensor[i] != p->frame_sensor[j]) continue;
            const double* A = X.data() + 12 * (size_t)i;
            const double* B = X.data() + 12 * (size_t)j;
            double tr = 0.0;
            for (int r = 0; r < 3; ++r)
                for (int c = 0; c < 3; ++c) tr += A[4 * r + c] * B[4 * r + c];  // trace(R_i^T R_j)
            const double ca = std::max(-1.0, std::min(1.0, 0.5 * (tr - 1.0)));
            const double ang = std::acos(ca);
            const double dx = A[3] - B[3], dy = A[7] - B[7], dz = A[11] - B[11];
            const double dist = std::sqrt(dx * dx + dy * dy + dz * dz);
            const bool is_seq = sequential && j == i + 1;
            if ((ang < max_angle && dist < max_dist) || is_seq) {
                cand.push_back(i);
                cand.push_back(j);
                seq.push_back(is_seq ? 1 : 0);
            }
        }
    const int mc = (int)(cand.size() / 2);
    std::vector<double> cost_c(mc), count_c(mc);
    if (mc > 0) {
        // count valid residuals of the candidates with the problem's own machinery, then restore its pairs
        std::vector<int32_t> keep = p->pairs;
        int st = pba_set_pairs(p, cand.data(), mc);
        if (st) return st;
        CUDA_TRY(p, launch_pair_pose(p->d_poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, p->stream));
        if (p->cfg.path == PBA_PATH_BATCHED) {
            CUDA_TRY(p, cudaMemsetAsync(p->d_queue + 1, 0, sizeof(int), p->stream));
            CUDA_TRY(p, launch_linearize(false, false, p->cfg.texel_precision, p->d_chunks, p->n_chunks,
                                         p->d_queue + 1, p->d_ps, p->d_pp, p->pts_pg, p->pts_n, p->tex, p->prm,
                                         p->d_partials, nullptr, p->grid_cost, p->variant_cost, p->stream));
            CUDA_TRY(p, launch_pair_reduce(p->d_partials, p->d_ps, p->d_pf, p->d_poses, p->d_pair_Xo, p->M, false,
                                           p->d_blocks_cand, p->stream));
        } else {
            CUDA_TRY(p, cudaMemsetAsync(p->d_plain_acc, 0, sizeof(float) * 96 * (size_t)p->M, p->stream));
            for (int q = 0; q < p->M; ++q) {
                const int src = p->pairs[2 * q];
                const pba_sensor& S = p->sensors[p->frame_sensor[src]];
                CUDA_TRY(p, launch_plain(false, q, p->d_ps, p->d_pp, p->raw, p->d_sensors, p->frame_sensor[src],
                                         p->prm, p->cfg.range_min, p->cfg.range_max, p->d_plain_acc, S.width,
                                         S.height, p->stream));
            }
            CUDA_TRY(p, launch_plain_expand(p->d_plain_acc, p->M, false, p->d_blocks_cand, p->stream));
        }
        std::vector<double> blk((size_t)kBlockStride * mc);
        CUDA_TRY(p, cudaMemcpyAsync(blk.data(), p->d_blocks_cand, sizeof(double) * blk.size(),
                                    cudaMemcpyDeviceToHost, p->stream));
        CUDA_TRY(p, cudaStreamSynchronize(p->stream));
        for (int q = 0; q < mc; ++q) count_c[q] = blk[(size_t)kBlockStride * q + 157];
        st = keep.empty() ? PBA_OK : pba_set_pairs(p, keep.data(), (int)(keep.size() / 2));
        if (keep.empty()) {
            drop_graph(p);
            free_pair_buffers(p);
            p->pairs.clear();
            p->linearized = false;
        }
        if (st) return st;
    }
    int m = 0;
    for (int q = 0; q < mc; ++q) {
        const int i = cand[2 * q];
        const double np = (double)p->n_points[i];
        const double ratio = np > 0 ? count_c[q] / np : 0.0;
        if (ratio > min_ratio || seq[q]) {
            if (m < cap) {
                if (pairs_out) {
                    pairs_out[2 * m] = i;
                    pairs_out[2 * m + 1] = cand[2 * q + 1];
                }
                if (ratio_out) ratio_out[m] = (float)ratio;
            }
            ++m;
        }
    }
    *m_out = m;
    if (m > cap) return fail(p, PBA_EINVAL, "build_pairs: output capacity too small");
    return PBA_OK;
}

int pba_cost_gradient(pba_problem* p, double* cost, int64_t* n_valid, double* d_poses, double* d_extrinsic,
                      float* d_channels) {
    int st = ready(p);
    if (st) return st;
    if (p->cfg.path != PBA_PATH_BATCHED) return fail(p, PBA_EINVAL, "cost_gradient needs the batched path");
    for (int k = 0; k < p->N; ++k)
        if (!p->uploaded[k]) return fail(p, PBA_ENOTREADY, "cost_gradient: frame not uploaded");
    cudaStream_t s = p->stream;
    CUDA_TRY(p, launch_pair_pose(p->d_poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, s));
    if (d_poses) CUDA_TRY(p, cudaMemsetAsync(d_poses, 0, sizeof(double) * 12 * p->N, s));
    if (d_channels) CUDA_TRY(p, cudaMemsetAsync(d_channels, 0, sizeof(float) * 5 * (size_t)p->total_px, s));
    CUDA_TRY(p, cudaMemsetAsync(p->d_queue + 1, 0, sizeof(int), s));
    CUDA_TRY(p, launch_adjoint(p->cfg.texel_precision, p->d_chunks, p->n_chunks, p->d_queue + 1, p->d_ps, p->d_pp,
                               p->pts_pg, p->pts_n, p->pts_pix, p->tex, p->d_sensors, p->d_frame_sensor, p->prm,
                               p->d_adj_partials, d_channels, adjoint_grid(p->cfg.texel_precision), s));
    CUDA_TRY(p, launch_adjoint_reduce(p->d_adj_partials, p->d_ps, p->d_pf, p->d_poses, p->d_pair_Xo, p->M,
                                      p->d_adj_pair, p->d_tasks, p->n_tasks, p->d_contrib, p->d_frame_sensor,
                                      (int)p->sensors.size(), d_poses, d_extrinsic, p->d_adj_totals, s));
    double tot[2];
    CUDA_TRY(p, cudaMemcpyAsync(tot, p->d_adj_totals, sizeof tot, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(p, cudaStreamSynchronize(s));
    if (cost) *cost = tot[0];
    if (n_valid) *n_valid = (int64_t)tot[1];
    return PBA_OK;
}

int pba_tangent_gradient(pba_problem* p, const double* X, const double* G, int n, double* g) {
    if (!p || n < 0 || (n > 0 && (!X || !G || !g))) return fail(p, PBA_EINVAL, "tangent_gradient: bad arguments");
    if (n == 0) return PBA_OK;
    cudaSetDevice(p->device);
    CUDA_TRY(p, launch_tangent(X, G, n, g, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_linearize(pba_problem* p, double* cost, int64_t* n_valid) {
    int st = ready(p);
    if (st) return st;
    int nl = 0;
    st = enqueue_linearize(p, p->stream, &nl);
    if (st) return st;
    LmState ls;
    CUDA_TRY(p, cudaMemcpyAsync(&ls, p->d_state, sizeof ls, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    p->linearized = true;
    p->mask_valid = p->mask_export && p->cfg.path == PBA_PATH_BATCHED;
    if (cost) *cost = ls.cost;
    if (n_valid) *n_valid = ls.n_valid;
    return PBA_OK;
}

int pba_get_system(pba_problem* p, double* H, double* b) {
    if (!p) return PBA_EINVAL;
    if (!p->linearized) return fail(p, PBA_ENOTREADY, "get_system: no linearisation");
    cudaSetDevice(p->device);
    const int n6 = 6 * p->N;
    // the block-sparse solve keeps no dense system: assemble it from the pair blocks now
    if (p->sparse && p->M > 0)
        CUDA_TRY(p, launch_assemble(p->d_tasks, p->n_tasks, p->d_contrib, p->d_blocks, p->N, p->d_H, p->d_b,
                                    p->stream));
    if (H) CUDA_TRY(p, cudaMemcpyAsync(H, p->d_H, sizeof(double) * (size_t)n6 * n6, cudaMemcpyDeviceToHost, p->stream));
    if (b) CUDA_TRY(p, cudaMemcpyAsync(b, p->d_b, sizeof(double) * n6, cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_get_pair_system(pba_problem* p, double* pair_H, double* pair_b, double* pair_cost, int64_t* pair_count) {
    if (!p) return PBA_EINVAL;
    if (!p->linearized) return fail(p, PBA_ENOTREADY, "get_pair_system: no linearisation");
    cudaSetDevice(p->device);
    std::vector<double> blk((size_t)kBlockStride * p->M);
    CUDA_TRY(p, cudaMemcpyAsync(blk.data(), p->d_blocks, sizeof(double) * blk.size(), cudaMemcpyDeviceToHost,
                                p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    for (int q = 0; q < p->M; ++q) {
        const double* B = blk.data() + (size_t)kBlockStride * q;
        if (pair_H) memcpy(pair_H + 144 * (size_t)q, B, sizeof(double) * 144);
        if (pair_b) memcpy(pair_b + 12 * (size_t)q, B + 144, sizeof(double) * 12);
        if (pair_cost) pair_cost[q] = B[156];
        if (pair_count) pair_count[q] = (int64_t)B[157];
    }
    return PBA_OK;
}

int pba_set_mask_export(pba_problem* p, int enable) {
    if (!p) return PBA_EINVAL;
    if (p->cfg.path != PBA_PATH_BATCHED && enable) return fail(p, PBA_EINVAL, "mask export needs the batched path");
    if ((p->mask_export ? 1 : 0) != (enable ? 1 : 0)) drop_graph(p);
    p->mask_export = enable != 0;
    return PBA_OK;
}

int pba_get_mask(pba_problem* p, int pair, uint32_t* bits, int n_words) {
    if (!p || !bits || pair < 0 || pair >= p->M) return fail(p, PBA_EINVAL, "get_mask: bad argument");
    if (!p->mask_valid) return fail(p, PBA_ENOTREADY, "get_mask: no mask exported");
    const int need = (p->pair_src_points[pair] + 31) / 32;
    if (n_words < need) return fail(p, PBA_EINVAL, "get_mask: buffer too small");
    cudaSetDevice(p->device);
    if (need > 0)
        CUDA_TRY(p, cudaMemcpyAsync(bits, p->d_mask + p->mask_off[pair], sizeof(uint32_t) * need,
                                    cudaMemcpyDeviceToHost, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_solve_step(pba_problem* p, double lambda, pba_iter_stats* stats) {
    int st = ready(p);
    if (st) return st;
    if (!p->linearized) return fail(p, PBA_ENOTREADY, "solve_step: no linearisation");
    if (!(lambda >= 0.0)) return fail(p, PBA_EINVAL, "solve_step: lambda must be >= 0");
    int nl = 0;
    st = enqueue_step(p, lambda, p->stream, &nl);
    if (st) return st;
    p->linearized = false;
    return read_stats(p, stats);
}

int pba_set_lambda(pba_problem* p, double lambda) {
    if (!p) return PBA_EINVAL;
    cudaSetDevice(p->device);
    const double v = lambda >= 0.0 ? lambda : -1.0;
    CUDA_TRY(p, cudaMemcpyAsync(&p->d_state->lambda, &v, sizeof v, cudaMemcpyHostToDevice, p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

// The plan's work items ordered by the lane in which the last of their pair's
// two frames arrives (lanes: frame ranges [first[l], first[l + 1])), within a
// lane the long items first; cached for the plan and lane boundaries.
static int build_ready_order(pba_problem* p, const std::vector<int>& first) {
    if (p->ready_serial == p->plan_serial && p->ready_first == first) return PBA_OK;
    const int L = (int)first.size() - 1;
    std::vector<int4> items(p->n_chunks);
    CUDA_TRY(p, cudaMemcpyAsync(items.data(), p->d_chunks, sizeof(int4) * items.size(), cudaMemcpyDeviceToHost,
                                p->stream));
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    std::vector<int> lane_of(p->N);
    for (int l = 0; l < L; ++l)
        for (int k = first[l]; k < first[l + 1]; ++k) lane_of[k] = l;
    std::vector<int> key(items.size());
    std::vector<int> seg(L + 1, 0);
    for (size_t c = 0; c < items.size(); ++c) {
        const int q = items[c].x;
        key[c] = std::max(lane_of[p->pairs[2 * q]], lane_of[p->pairs[2 * q + 1]]);
        ++seg[key[c] + 1];
    }
    for (int l = 0; l < L; ++l) seg[l + 1] += seg[l];
    std::vector<int4> ordered(items.size());
    std::vector<int> fill(seg.begin(), seg.end() - 1);
    for (size_t c = 0; c < items.size(); ++c) ordered[fill[key[c]]++] = items[c];
    for (int l = 0; l < L; ++l)  // the short items end each segment, as they end the plan
        std::stable_sort(ordered.begin() + seg[l], ordered.begin() + seg[l + 1],
                         [](const int4& a, const int4& b) { return a.z > b.z; });
    if (p->n_chunks_ready_alloc < p->n_chunks) {
        dfree(p->d_chunks_ready);
        p->n_chunks_ready_alloc = 0;
        CUDA_TRY(p, cudaMalloc((void**)&p->d_chunks_ready, sizeof(int4) * (size_t)p->n_chunks));
        p->n_chunks_ready_alloc = p->n_chunks;
    }
    CUDA_TRY(p, cudaMemcpy(p->d_chunks_ready, ordered.data(), sizeof(int4) * ordered.size(), cudaMemcpyHostToDevice));
    p->ready_first = first;
    p->ready_seg = seg;
    p->ready_serial = p->plan_serial;
    return PBA_OK;
}

int pba_iterate_frames(pba_problem* p, const float* channels, const double* poses, pba_iter_stats* stats) {
    if (!p) return PBA_EINVAL;
    if (!channels) return fail(p, PBA_EINVAL, "iterate_frames: channels is NULL");
    cudaSetDevice(p->device);
    int st;
    if (poses && (st = pba_set_poses(p, poses, 0))) return st;
    if ((st = ready(p))) return st;
    bool overlap = p->cfg.path == PBA_PATH_BATCHED && p->points_known && p->n_chunks > 0;
    for (int k = 0; k < p->N && overlap; ++k) overlap = p->uploaded[k] != 0;
    int nl = 0;
    if (!overlap) {
        // frames not uploaded before (no plan to start from): the upload of each run
        // of same-size frames, then the linearisation
        for (int k = 0; k < p->N;) {
            const pba_sensor& S = p->sensors[p->frame_sensor[k]];
            int j = k + 1;
            while (j < p->N && p->sensors[p->frame_sensor[j]].width == S.width &&
                   p->sensors[p->frame_sensor[j]].height == S.height)
                ++j;
            if ((st = pba_upload_frames(p, k, j - k, channels + 5 * p->px_off[k], 0))) return st;
            k = j;
        }
        if ((st = ready(p))) return st;
        if ((st = enqueue_linearize(p, p->stream, &nl))) return st;
    } else {
        // streams, events and buffers of the lanes, created on first use (each one
        // that is still missing, so that a failed earlier attempt is completed)
        if (!p->lane_pack) {
            int least = 0, greatest = 0;
            CUDA_TRY(p, cudaDeviceGetStreamPriorityRange(&least, &greatest));
            CUDA_TRY(p, cudaStreamCreateWithPriority(&p->lane_pack, cudaStreamNonBlocking, greatest));
        }
        if (!p->lane_copy) CUDA_TRY(p, cudaStreamCreateWithFlags(&p->lane_copy, cudaStreamNonBlocking));
        if (!p->lane_start) CUDA_TRY(p, cudaEventCreateWithFlags(&p->lane_start, cudaEventDisableTiming));
        for (int l = 0; l < p->kFrameLanes; ++l) {
            if (!p->lane_copied[l]) CUDA_TRY(p, cudaEventCreateWithFlags(&p->lane_copied[l], cudaEventDisableTiming));
            if (!p->lane_ready[l]) CUDA_TRY(p, cudaEventCreateWithFlags(&p->lane_ready[l], cudaEventDisableTiming));
        }
        if (!p->d_seg_queue) CUDA_TRY(p, cudaMalloc((void**)&p->d_seg_queue, sizeof(int) * p->kFrameLanes));
        if (!p->h_counts) CUDA_TRY(p, cudaMallocHost((void**)&p->h_counts, sizeof(int) * (size_t)p->N));
        // lanes of whole frames, about equal in bytes
        std::vector<int> first(1, 0);
        for (int l = 1; l < p->kFrameLanes; ++l) {
            const long long target = p->total_px * l / p->kFrameLanes;
            int k = first.back() + 1;
            while (k < p->N && p->px_off[k] < target) ++k;
            if (k < p->N) first.push_back(k);
        }
        first.push_back(p->N);
        const int L = (int)first.size() - 1;
        if ((st = build_ready_order(p, first))) return st;
        // the copies start once earlier work on the frames' buffers is done; each
        // lane is packed as soon as it has arrived
        CUDA_TRY(p, cudaEventRecord(p->lane_start, p->stream));
        CUDA_TRY(p, cudaStreamWaitEvent(p->lane_copy, p->lane_start, 0));
        CUDA_TRY(p, cudaStreamWaitEvent(p->lane_pack, p->lane_start, 0));
        for (int l = 0; l < L; ++l) {
            const long long a = p->px_off[first[l]];
            const long long b = first[l + 1] < p->N ? p->px_off[first[l + 1]] : p->total_px;
            CUDA_TRY(p, cudaMemcpyAsync(p->raw + 5 * a, channels + 5 * a, sizeof(float) * 5 * (size_t)(b - a),
                                        cudaMemcpyHostToDevice, p->lane_copy));
            CUDA_TRY(p, cudaEventRecord(p->lane_copied[l], p->lane_copy));
            CUDA_TRY(p, cudaStreamWaitEvent(p->lane_pack, p->lane_copied[l], 0));
            if ((st = pack_frames(p, first[l], first[l + 1] - first[l], p->lane_pack))) return st;
            CUDA_TRY(p, cudaEventRecord(p->lane_ready[l], p->lane_pack));
        }
        p->pyramid_stale = true;
        p->linearized = false;
        p->mask_valid = false;
        // segment l of the linearisation waits for lane l (the copies run ahead of
        // it on the copy engine; the packing, on a stream of greater priority,
        // takes the SMs as a segment drains)
        CUDA_TRY(p, launch_pair_pose(p->d_poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, p->stream));
        CUDA_TRY(p, cudaMemsetAsync(p->d_seg_queue, 0, sizeof(int) * L, p->stream));
        for (int l = 0; l < L; ++l) {
            CUDA_TRY(p, cudaStreamWaitEvent(p->stream, p->lane_ready[l], 0));
            CUDA_TRY(p, launch_linearize(true, false, p->cfg.texel_precision, p->d_chunks_ready + p->ready_seg[l],
                                         p->ready_seg[l + 1] - p->ready_seg[l], p->d_seg_queue + l, p->d_ps,
                                         p->d_pp, p->pts_pg, p->pts_n, p->tex, p->prm, p->d_partials, nullptr,
                                         p->grid_full, p->variant_full, p->stream));
            ++nl;
        }
        // the point counts the plan was built for must still hold
        CUDA_TRY(p, cudaMemcpyAsync(p->h_counts, p->d_npoints, sizeof(int) * (size_t)p->N, cudaMemcpyDeviceToHost,
                                    p->stream));
        CUDA_TRY(p, cudaStreamSynchronize(p->stream));
        if (std::equal(p->n_points.begin(), p->n_points.end(), p->h_counts)) {
            CUDA_TRY(p, launch_pair_reduce(p->d_partials, p->d_ps, p->d_pf, p->d_poses, p->d_pair_Xo, p->M, true,
                                           p->d_blocks, p->stream));
            if (!p->sparse)
                CUDA_TRY(p, launch_assemble(p->d_tasks, p->n_tasks, p->d_contrib, p->d_blocks, p->N, p->d_H, p->d_b,
                                            p->stream));
            CUDA_TRY(p, launch_total_cost(p->d_blocks, p->M, p->d_state, false, p->stream));
        } else {
            // a frame's count changed: the pair plan is rebuilt and the pass redone
            if ((st = finish_repack(p))) return st;
            if ((st = enqueue_linearize(p, p->stream, &nl))) return st;
        }
    }
    // the damped step and the cost at the candidate (the system there is not formed)
    p->linearized = true;
    if ((st = enqueue_step(p, -1.0, p->stream, &nl))) return st;
    p->linearized = false;
    return read_stats(p, stats);
}

int pba_iterate(pba_problem* p, pba_iter_stats* stats) {
    int st = pba_iterate_async(p, 1);
    if (st) return st;
    return read_stats(p, stats);
}

int pba_iterate_async(pba_problem* p, int n) {
    int st = ready(p);
    if (st) return st;
    if (n < 0) return fail(p, PBA_EINVAL, "iterate_async: n < 0");
    if (!p->graph_exec) {
        int nl = 0;
        CUDA_TRY(p, cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal));
        st = enqueue_step(p, -1.0, p->capture_stream, &nl, nullptr, true);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(p->capture_stream, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return fail(p, PBA_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        p->graph = g;
        CUDA_TRY(p, cudaGraphInstantiate(&p->graph_exec, p->graph, 0));
        p->launches_last = nl;
    }
    if (n > 0 && !p->linearized) {
        // the step needs the system at the current poses; every iteration then keeps it current
        int nl = 0;
        st = enqueue_linearize(p, p->stream, &nl);
        if (st) return st;
    }
    for (int k = 0; k < n; ++k) CUDA_TRY(p, cudaGraphLaunch(p->graph_exec, p->stream));
    if (n > 0) p->linearized = true;
    p->mask_valid = false;
    return PBA_OK;
}

int pba_get_stats(pba_problem* p, pba_iter_stats* stats) {
    if (!p) return PBA_EINVAL;
    cudaSetDevice(p->device);
    return read_stats(p, stats);
}

int pba_iterate_timed(pba_problem* p, float* phase_ms, int n_phases, pba_iter_stats* stats) {
    int st = ready(p);
    if (st) return st;
    cudaEvent_t ev[PBA_N_PHASES + 1] = {};
    for (auto& e : ev) CUDA_TRY(p, cudaEventCreate(&e));
    int nl = 0;
    if (!p->linearized) {
        st = enqueue_linearize(p, p->stream, &nl);
        if (st) return st;
    }
    CUDA_TRY(p, cudaEventRecord(ev[0], p->stream));
    st = enqueue_step(p, -1.0, p->stream, &nl, ev, true);
    if (!st) st = read_stats(p, stats);
    if (!st && phase_ms)
        for (int k = 0; k < n_phases && k < PBA_N_PHASES; ++k) {
            float ms = 0.f;
            cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            phase_ms[k] = ms;
        }
    for (auto& e : ev) cudaEventDestroy(e);
    p->linearized = st == PBA_OK;
    return st;
}

}  // extern "C"

namespace {

// Tuned settings per configuration, for the life of the process.
struct TuneEntry {
    int variant_full, variant_cost, chunk, chunk_tail, reduction;
    float ms_full, ms_cost;
};
std::mutex g_tune_mutex;
std::map<std::string, TuneEntry> g_tune_cache;

// What a tuning depends on: device, texel precision, gradient mode, the pairs
// (count, points and sensor models) and the frames' sizes.
std::string tune_key(const pba_problem* p) {
    long long pts = 0, h = 1469598103934665603LL;
    for (int q = 0; q < p->M; ++q) {
        const int i = p->pairs[2 * q], j = p->pairs[2 * q + 1];
        pts += p->n_points[i];
        const pba_sensor& S = p->sensors[p->frame_sensor[i]];
        for (long long v : {(long long)i, (long long)j, (long long)S.model, (long long)S.width, (long long)S.height})
            h = (h ^ v) * 1099511628211LL;
    }
    char buf[160];
    snprintf(buf, sizeof buf, "d%d t%d g%d m%d p%lld h%llx", p->device, p->cfg.texel_precision, p->cfg.grad_mode, p->M,
             pts, (unsigned long long)h);
    return buf;
}

// Rebuild the chunk queue (and everything pba_set_pairs plans) for new work-item sizes.
int set_chunking(pba_problem* p, int chunk, int tail) {
    if (p->chunk == chunk && p->chunk_tail == tail) return PBA_OK;
    p->chunk = chunk;
    p->chunk_tail = tail;
    std::vector<int32_t> keep = p->pairs;
    return pba_set_pairs(p, keep.data(), (int)(keep.size() / 2));
}

// Mean time of `repeats` launches of one linearisation pass (after one untimed launch).
int time_pass(pba_problem* p, bool full, int variant, int repeats, cudaEvent_t e0, cudaEvent_t e1, float* ms_out) {
    const int grid = linearize_grid(p->cfg.texel_precision, full, variant);
    float total = 0.f;
    for (int r = 0; r <= repeats; ++r) {
        CUDA_TRY(p, cudaMemsetAsync(p->d_queue, 0, sizeof(int), p->stream));
        CUDA_TRY(p, cudaEventRecord(e0, p->stream));
        CUDA_TRY(p, launch_linearize(full, false, p->cfg.texel_precision, p->d_chunks, p->n_chunks, p->d_queue,
                                     p->d_ps, p->d_pp, p->pts_pg, p->pts_n, p->tex, p->prm, p->d_partials, nullptr,
                                     grid, variant, p->stream));
        CUDA_TRY(p, cudaEventRecord(e1, p->stream));
        CUDA_TRY(p, cudaEventSynchronize(e1));
        float ms = 0.f;
        CUDA_TRY(p, cudaEventElapsedTime(&ms, e0, e1));
        if (r > 0) total += ms;
    }
    *ms_out = total / repeats;
    return PBA_OK;
}

}  // namespace

extern "C" {

int pba_autotune(pba_problem* p, int repeats, int32_t* variant_full, int32_t* variant_cost) {
    int st = ready(p);
    if (st) return st;
    if (repeats < 1) repeats = 1;
    if (p->cfg.path != PBA_PATH_BATCHED) {
        if (variant_full) *variant_full = 0;
        if (variant_cost) *variant_cost = 0;
        return PBA_OK;
    }
    if ((st = ensure_points(p))) return st;
    const std::string key = tune_key(p);
    TuneEntry best{0, 0, kChunk, kChunkTail, 0, 3.4e38f, 3.4e38f};
    bool cached = false;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            best = it->second;
            cached = true;
        }
    }
    if (!cached) {
        cudaEvent_t e0, e1;
        CUDA_TRY(p, cudaEventCreate(&e0));
        CUDA_TRY(p, cudaEventCreate(&e1));
        // the full pass over work-item size x tail size x occupancy variant x
        // reduction scheme; settings within kTuneTie of the fastest count as equal
        // and the first of them in this order is kept, so that timing noise does
        // not flip the choice
        struct Timed { int chunk, tail, variant, reduction; float ms; };
        std::vector<Timed> full;
        const int n_var = p->stage_ok ? PBA_N_VARIANTS : PBA_N_VARIANTS / 2;  // staged ones need tiles
        for (int c : kTuneChunks)
            for (int t : kTuneTails) {
                if ((st = set_chunking(p, c, t))) return st;
                CUDA_TRY(p, launch_pair_pose(p->d_poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, p->stream));
                for (int v = 0; v < n_var; ++v)
                    for (int red : kTuneReductions) {
                        float ms = 0.f;
                        p->prm.reduction = red;
                        st = time_pass(p, true, v, repeats, e0, e1, &ms);
                        p->prm.reduction = 0;
                        if (st) return st;
                        full.push_back({c, t, v, red, ms});
                    }
            }
        float fastest = 3.4e38f;
        for (const Timed& x : full) fastest = std::min(fastest, x.ms);
        for (const Timed& x : full)
            if (x.ms <= fastest * (1.f + kTuneTie)) {
                best.ms_full = x.ms;
                best.variant_full = x.variant;
                best.chunk = x.chunk;
                best.chunk_tail = x.tail;
                best.reduction = x.reduction;
                break;
            }
        // the cost-only pass at the chosen work items
        if ((st = set_chunking(p, best.chunk, best.chunk_tail))) return st;
        CUDA_TRY(p, launch_pair_pose(p->d_poses, p->d_pf, p->d_pair_Xo, p->M, p->d_pp, p->stream));
        float cost_ms[PBA_N_VARIANTS];
        for (int v = 0; v < n_var; ++v)
            if ((st = time_pass(p, false, v, repeats, e0, e1, &cost_ms[v]))) return st;
        const float cost_fastest = *std::min_element(cost_ms, cost_ms + n_var);
        for (int v = 0; v < n_var; ++v)
            if (cost_ms[v] <= cost_fastest * (1.f + kTuneTie)) {
                best.ms_cost = cost_ms[v];
                best.variant_cost = v;
                break;
            }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune_cache[key] = best;
    } else if ((st = set_chunking(p, best.chunk, best.chunk_tail))) {
        return st;
    }
    // (staged variants only where this problem stages tiles)
    p->variant_full = p->stage_ok ? best.variant_full : (best.variant_full & 3);
    p->variant_cost = p->stage_ok ? best.variant_cost : (best.variant_cost & 3);
    p->prm.reduction = best.reduction;
    p->tune_ms_full = best.ms_full;
    p->tune_ms_cost = best.ms_cost;
    p->tune_from_cache = cached ? 1 : 0;
    p->grid_full = linearize_grid(p->cfg.texel_precision, true, p->variant_full);
    p->grid_cost = linearize_grid(p->cfg.texel_precision, false, p->variant_cost);
    drop_graph(p);
    p->linearized = false;
    if (variant_full) *variant_full = p->variant_full;
    if (variant_cost) *variant_cost = p->variant_cost;
    return PBA_OK;
}

int pba_get_tuning(pba_problem* p, pba_tuning* out) {
    if (!p || !out) return PBA_EINVAL;
    out->variant_full = p->variant_full;
    out->variant_cost = p->variant_cost;
    out->chunk = p->chunk;
    out->chunk_tail = p->chunk_tail;
    out->reduction = p->prm.reduction;
    out->from_cache = p->tune_from_cache;
    out->tile_err = 0;
    if (p->d_tile_err) CUDA_TRY(p, cudaMemcpy(&out->tile_err, p->d_tile_err, sizeof(int), cudaMemcpyDeviceToHost));
    out->ms_full = p->tune_ms_full;
    out->ms_cost = p->tune_ms_cost;
    return PBA_OK;
}

int pba_set_variables(pba_problem* p, const int32_t* frame_var, int n_vars) {
    if (!p) return PBA_EINVAL;
    cudaSetDevice(p->device);
    if (!frame_var) {  // back to the default: frame 0 fixed, every other frame free
        p->n_fv_user = -1;
        p->fv_user.clear();
        return rebuild_vars(p);
    }
    if (n_vars < 1 || n_vars > p->N - 1)
        return fail(p, PBA_EINVAL, "set_variables: n_vars must lie in [1, n_frames - 1]");
    std::vector<int> count(n_vars, 0);
    int fixed = 0;
    for (int k = 0; k < p->N; ++k) {
        if (frame_var[k] < -1 || frame_var[k] >= n_vars)
            return fail(p, PBA_EINVAL, "set_variables: frame_var entry outside [-1, n_vars)");
        if (frame_var[k] < 0) ++fixed;
        else ++count[frame_var[k]];
    }
    if (!fixed) return fail(p, PBA_EINVAL, "set_variables: no frame is held fixed (the gauge would be free)");
    for (int v = 0; v < n_vars; ++v)
        if (!count[v]) return fail(p, PBA_EINVAL, "set_variables: a variable moves no frame");
    p->fv_user.assign(frame_var, frame_var + p->N);
    p->n_fv_user = n_vars;
    return rebuild_vars(p);
}

int pba_set_offset_free(pba_problem* p, int sensor, int is_free) {
    if (!p || sensor < 0 || sensor >= (int)p->sensors.size())
        return fail(p, PBA_EINVAL, "set_offset_free: bad sensor");
    cudaSetDevice(p->device);
    p->offset_free[sensor] = is_free ? 1 : 0;
    return rebuild_vars(p);
}

namespace {

// X [+] d on the host for one 3x4 offset: [R R(dq), R dt + t], R(dq) from the
// unit quaternion (sqrt(1 - |dq|^2), dq), normalised (1, dq) when |dq| >= 1.
void boxplus_host(const double X[12], const double d[6], double out[12]) {
    double qx = d[3], qy = d[4], qz = d[5];
    const double n2 = qx * qx + qy * qy + qz * qz;
    double qw;
    if (n2 < 1.0) {
        qw = std::sqrt(1.0 - n2);
    } else {
        const double nn = std::sqrt(1.0 + n2);
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

// Gradient of F in the box-plus chart at X from the matrix gradient G = dF/dX:
// dt part R^T G_t; dq part 2 (W_zy - W_yz, W_xz - W_zx, W_yx - W_xy), W = R^T G_R
// (R(dq) ~ I + 2 [dq]x).
void tangent_host(const double X[12], const double G[12], double g[6]) {
    double W[9];
    for (int a = 0; a < 3; ++a) {
        g[a] = 0.0;
        for (int r = 0; r < 3; ++r) g[a] += X[4 * r + a] * G[4 * r + 3];
        for (int b = 0; b < 3; ++b) {
            W[3 * a + b] = 0.0;
            for (int r = 0; r < 3; ++r) W[3 * a + b] += X[4 * r + a] * G[4 * r + b];
        }
    }
    g[3] = 2.0 * (W[7] - W[5]);
    g[4] = 2.0 * (W[2] - W[6]);
    g[5] = 2.0 * (W[3] - W[1]);
}

// F and its tangent gradient with respect to sensor `sensor`'s offset set to X.
int extrinsic_eval(pba_problem* p, int sensor, const double X[12], double* dE, double* F, double g[6]) {
    int st = pba_set_extrinsic(p, sensor, X);
    if (st) return st;
    st = pba_cost_gradient(p, F, nullptr, nullptr, dE, nullptr);
    if (st) return st;
    double G[12];
    CUDA_TRY(p, cudaMemcpy(G, dE + 12 * sensor, sizeof G, cudaMemcpyDeviceToHost));
    tangent_host(X, G, g);
    return PBA_OK;
}

}  // namespace

int pba_get_extrinsic(pba_problem* p, int sensor, double* extrinsic) {
    if (!p || !extrinsic || sensor < 0 || sensor >= (int)p->sensors.size())
        return fail(p, PBA_EINVAL, "get_extrinsic: bad argument");
    cudaSetDevice(p->device);
    int st = sync_offsets_to_host(p);
    if (st) return st;
    for (int e = 0; e < 12; ++e) extrinsic[e] = p->sensors[sensor].extrinsic[e];
    return PBA_OK;
}

int pba_refine_extrinsic(pba_problem* p, int sensor, int max_iters, double rel_tol, double* cost_before,
                         double* cost_after, int32_t* iterations) {
    int st = ready(p);
    if (st) return st;
    if (sensor < 0 || sensor >= (int)p->sensors.size() || max_iters < 0)
        return fail(p, PBA_EINVAL, "refine_extrinsic: bad sensor or iteration count");
    if (p->cfg.path != PBA_PATH_BATCHED) return fail(p, PBA_EINVAL, "refine_extrinsic needs the batched path");
    double* dE = nullptr;
    if (cudaMalloc((void**)&dE, sizeof(double) * 12 * p->sensors.size()) != cudaSuccess)
        return fail(p, PBA_ENOMEM, "refine_extrinsic: out of device memory");
    double X[12], F, g[6];
    for (int e = 0; e < 12; ++e) X[e] = p->sensors[sensor].extrinsic[e];
    st = extrinsic_eval(p, sensor, X, dE, &F, g);
    if (st) {
        cudaFree(dE);
        return st;
    }
    if (cost_before) *cost_before = F;
    // BFGS on the 6 tangent coordinates; each iterate is re-expressed in the chart
    // at the new offset (the curvature estimate carries over to first order)
    double Hi[36] = {0};
    for (int a = 0; a < 6; ++a) Hi[7 * a] = 1.0;
    bool scaled = false;
    int it = 0;
    for (; it < max_iters; ++it) {
        double d[6], gn = 0.0, slope = 0.0;
        for (int a = 0; a < 6; ++a) {
            d[a] = 0.0;
            for (int b = 0; b < 6; ++b) d[a] -= Hi[6 * a + b] * g[b];
            gn += g[a] * g[a];
        }
        for (int a = 0; a < 6; ++a) slope += g[a] * d[a];
        if (!(gn > 0.0)) break;
        if (!(slope < 0.0)) {  // not a descent direction: restart from steepest descent
            for (int a = 0; a < 36; ++a) Hi[a] = a % 7 ? 0.0 : 1.0;
            for (int a = 0; a < 6; ++a) d[a] = -g[a];
            slope = -gn;
            scaled = false;
        }
        double alpha = 1.0, dn = 0.0;
        for (int a = 0; a < 6; ++a) dn += d[a] * d[a];
        dn = std::sqrt(dn);
        if (!scaled && dn > 0.01) alpha = 0.01 / dn;  // first step: at most 1 cm / 0.01 in the chart
        double Xn[12], Fn = F, gnew[6];
        bool ok = false;
        for (int ls = 0; ls < 30; ++ls) {
            double step[6];
            for (int a = 0; a < 6; ++a) step[a] = alpha * d[a];
            boxplus_host(X, step, Xn);
            st = extrinsic_eval(p, sensor, Xn, dE, &Fn, gnew);
            if (st) {
                cudaFree(dE);
                return st;
            }
            if (Fn <= F + 1e-4 * alpha * slope) {
                ok = true;
                break;
            }
            alpha *= 0.5;
        }
        if (!ok) {  // no decrease along d: keep the current offset
            st = pba_set_extrinsic(p, sensor, X);
            break;
        }
        double s[6], y[6], sy = 0.0, yy = 0.0;
        for (int a = 0; a < 6; ++a) {
            s[a] = alpha * d[a];
            y[a] = gnew[a] - g[a];
            sy += s[a] * y[a];
            yy += y[a] * y[a];
        }
        const double decrease = F - Fn;
        for (int e = 0; e < 12; ++e) X[e] = Xn[e];
        for (int a = 0; a < 6; ++a) g[a] = gnew[a];
        F = Fn;
        if (sy > 1e-300) {
            if (!scaled) {
                for (int a = 0; a < 36; ++a) Hi[a] = a % 7 ? 0.0 : sy / yy;
                scaled = true;
            }
            // Hi <- (I - rho s y^T) Hi (I - rho y s^T) + rho s s^T
            const double rho = 1.0 / sy;
            double Hy[6], yHy = 0.0;
            for (int a = 0; a < 6; ++a) {
                Hy[a] = 0.0;
                for (int b = 0; b < 6; ++b) Hy[a] += Hi[6 * a + b] * y[b];
                yHy += y[a] * Hy[a];
            }
            for (int a = 0; a < 6; ++a)
                for (int b = 0; b < 6; ++b)
                    Hi[6 * a + b] += -rho * (s[a] * Hy[b] + Hy[a] * s[b]) + (rho * rho * yHy + rho) * s[a] * s[b];
        }
        if (decrease < rel_tol * (F + decrease)) {
            ++it;
            break;
        }
    }
    cudaFree(dE);
    if (st) return st;
    if (cost_after) *cost_after = F;
    if (iterations) *iterations = it;
    return PBA_OK;
}

int pba_build_pyramid(pba_problem* p, int n_levels) {
    if (!p) return PBA_EINVAL;
    if (n_levels < 1 || n_levels > PBA_MAX_LEVELS) return fail(p, PBA_EINVAL, "build_pyramid: n_levels outside [1, 8]");
    for (int k = 0; k < p->N; ++k)
        if (!p->uploaded[k]) return fail(p, PBA_ENOTREADY, "build_pyramid: frame not uploaded");
    cudaSetDevice(p->device);
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    int sst = sync_offsets_to_host(p);
    if (sst) return sst;
    for (pba_problem* q : p->levels) pba_destroy(q);
    p->levels.clear();
    p->pyramid_stale = true;
    pba_problem* prev = p;
    for (int l = 1; l < n_levels; ++l) {
        // intrinsics of the half-resolution level: coarse pixel k is centred on
        // fine coordinate 2k + 1/2, so f' = f / 2 and c' = (c + 1/2) / 2 - 1/2
        std::vector<pba_sensor> cs = prev->sensors;
        for (pba_sensor& S : cs) {
            S.width /= 2;
            S.height /= 2;
            S.fx /= 2.0;
            S.fy /= 2.0;
            S.cx = (S.cx + 0.5) / 2.0 - 0.5;
            S.cy = (S.cy + 0.5) / 2.0 - 0.5;
            if (S.width < 4 || S.height < 4) {
                for (pba_problem* q : p->levels) pba_destroy(q);
                p->levels.clear();
                return fail(p, PBA_EINVAL, "build_pyramid: a level would be smaller than 4 x 4 pixels");
            }
        }
        pba_config cfg = prev->cfg;
        cfg.n_sensors = (int)cs.size();
        cfg.sensors = cs.data();
        cfg.frame_sensor = prev->frame_sensor.data();
        pba_problem* q = nullptr;
        int st = pba_create(&cfg, prev->stream, &q);
        if (st) {
            for (pba_problem* r : p->levels) pba_destroy(r);
            p->levels.clear();
            return fail(p, st, "build_pyramid: creating a level failed");
        }
        p->levels.push_back(q);
        auto bail = [&](int code, const std::string& msg) {
            for (pba_problem* r : p->levels) pba_destroy(r);
            p->levels.clear();
            return fail(p, code, msg);
        };
        float* tmp = nullptr;
        long long* d_off = nullptr;
        if (cudaMalloc((void**)&tmp, sizeof(float) * 5 * (size_t)std::max(q->total_px, 1LL)) != cudaSuccess ||
            cudaMalloc((void**)&d_off, sizeof(long long) * q->N) != cudaSuccess) {
            cudaFree(tmp);
            return bail(PBA_ENOMEM, "build_pyramid: out of device memory");
        }
        std::vector<int> ids(q->N);
        int max_px = 0;
        for (int k = 0; k < q->N; ++k) {
            ids[k] = k;
            const pba_sensor& S = cs[q->frame_sensor[k]];
            max_px = std::max(max_px, S.width * S.height);
        }
        cudaError_t ce = cudaMemcpyAsync(prev->d_frame_ids, ids.data(), sizeof(int) * q->N, cudaMemcpyHostToDevice,
                                         prev->stream);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(d_off, q->px_off.data(), sizeof(long long) * q->N, cudaMemcpyHostToDevice,
                                 prev->stream);
        if (ce == cudaSuccess)
            ce = launch_downsample(prev->raw, prev->d_frames, prev->d_frame_ids, d_off, q->N, max_px, tmp,
                                   prev->cfg.range_min, prev->cfg.range_max, prev->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(prev->stream);
        // upload runs of consecutive frames of one image size
        for (int k0 = 0; ce == cudaSuccess && k0 < q->N;) {
            const pba_sensor& S0 = cs[q->frame_sensor[k0]];
            int k1 = k0 + 1;
            while (k1 < q->N && cs[q->frame_sensor[k1]].width == S0.width &&
                   cs[q->frame_sensor[k1]].height == S0.height)
                ++k1;
            st = pba_upload_frames(q, k0, k1 - k0, tmp + 5 * q->px_off[k0], 1);
            if (st) {
                cudaFree(tmp);
                cudaFree(d_off);
                return bail(st, std::string("build_pyramid: ") + q->err);
            }
            k0 = k1;
        }
        cudaFree(tmp);
        cudaFree(d_off);
        if (ce != cudaSuccess) return bail(PBA_ECUDA, std::string("build_pyramid: ") + cudaGetErrorString(ce));
        if (p->poses_set && (st = pba_set_poses(q, p->d_poses, 1))) return bail(st, "build_pyramid: poses");
        if (p->M > 0 && (st = pba_set_pairs(q, p->pairs.data(), p->M))) return bail(st, "build_pyramid: pairs");
        if (p->n_fv_user >= 0 && (st = pba_set_variables(q, p->fv_user.data(), p->n_fv_user)))
            return bail(st, "build_pyramid: variables");
        for (int s = 0; s < (int)p->sensors.size(); ++s)
            if (p->offset_free[s] && (st = pba_set_offset_free(q, s, 1))) return bail(st, "build_pyramid: offsets");
        prev = q;
    }
    p->pyramid_stale = false;
    return PBA_OK;
}

int pba_pyramid_level(pba_problem* p, int level, pba_problem** level_out) {
    if (!p || !level_out) return PBA_EINVAL;
    if (level < 0 || level > (int)p->levels.size()) return fail(p, PBA_EINVAL, "pyramid_level: no such level");
    if (level > 0 && p->pyramid_stale)
        return fail(p, PBA_ENOTREADY, "pyramid_level: frames, pairs or extrinsics changed since build_pyramid");
    *level_out = level == 0 ? p : p->levels[level - 1];
    return PBA_OK;
}

int pba_optimize(pba_problem* p, int n_levels, const int32_t* max_iters, double rel_tol, pba_level_stats* stats) {
    int st = ready(p);
    if (st) return st;
    if (!max_iters || n_levels < 1 || n_levels > (int)p->levels.size() + 1)
        return fail(p, PBA_EINVAL, "optimize: n_levels exceeds the built pyramid, or max_iters is NULL");
    if (n_levels > 1 && p->pyramid_stale)
        return fail(p, PBA_ENOTREADY, "optimize: frames, pairs or extrinsics changed since build_pyramid");
    for (int l = 0; l < n_levels; ++l)
        if (max_iters[l] < 0) return fail(p, PBA_EINVAL, "optimize: negative iteration count");
    const bool was_stale = p->pyramid_stale;
    const int S = (int)p->sensors.size();
    double X[12];
    for (int l = n_levels - 1; l >= 0; --l) {
        pba_problem* q = l == 0 ? p : p->levels[l - 1];
        if (q != p && (st = pba_set_poses(q, p->d_poses, 1))) return fail(p, st, "optimize: " + q->err);
        for (int s = 0; q != p && s < S; ++s)  // refined offsets travel with the poses
            if (p->offset_free[s] && ((st = pba_get_extrinsic(p, s, X)) || (st = pba_set_extrinsic(q, s, X))))
                return fail(p, st, "optimize: offsets");
        if ((st = pba_set_lambda(q, -1.0))) return fail(p, st, "optimize: " + q->err);
        pba_level_stats ls{};
        ls.level = l;
        ls.status = PBA_OK;
        for (int it = 0; it < max_iters[n_levels - 1 - l]; ++it) {
            pba_iter_stats s{};
            if ((st = pba_iterate(q, &s))) return fail(p, st, "optimize: " + q->err);
            if (it == 0) ls.cost_first = s.cost;
            ++ls.iterations;
            ls.cost_last = s.accepted ? s.new_cost : s.cost;
            if (s.status) ls.status = s.status;
            if (s.accepted) {
                ++ls.accepted;
                if (s.cost - s.new_cost < rel_tol * s.cost) break;  // error variation below the threshold
            }
        }
        if (q != p && (st = pba_set_poses(p, q->d_poses, 1))) return fail(p, st, "optimize: poses");
        for (int s = 0; q != p && s < S; ++s)
            if (p->offset_free[s] && ((st = pba_get_extrinsic(q, s, X)) || (st = pba_set_extrinsic(p, s, X))))
                return fail(p, st, "optimize: offsets");
        if (stats) stats[n_levels - 1 - l] = ls;
    }
    p->pyramid_stale = was_stale;  // offsets carried between levels leave the levels' images valid
    CUDA_TRY(p, cudaStreamSynchronize(p->stream));
    return PBA_OK;
}

int pba_set_variants(pba_problem* p, int variant_full, int variant_cost) {
    if (!p) return PBA_EINVAL;
    if (variant_full < 0 || variant_full >= PBA_N_VARIANTS || variant_cost < 0 || variant_cost >= PBA_N_VARIANTS)
        return fail(p, PBA_EINVAL, "set_variants: variant outside [0, PBA_N_VARIANTS)");
    cudaSetDevice(p->device);
    if (!p->stage_ok) {  // no staged tiles here: variants 4 .. 7 run as 0 .. 3
        variant_full &= 3;
        variant_cost &= 3;
    }
    p->variant_full = variant_full;
    p->variant_cost = variant_cost;
    p->grid_full = linearize_grid(p->cfg.texel_precision, true, variant_full);
    p->grid_cost = linearize_grid(p->cfg.texel_precision, false, variant_cost);
    drop_graph(p);
    return PBA_OK;
}

int pba_set_tuning(pba_problem* p, const pba_tuning* t) {
    if (!p) return PBA_EINVAL;
    if (!t) return fail(p, PBA_EINVAL, "set_tuning: tuning is NULL");
    if (t->chunk < 32 || t->chunk > 8192 || t->chunk % 32 || t->chunk_tail < 32 || t->chunk_tail > t->chunk ||
        t->chunk_tail % 32)
        return fail(p, PBA_EINVAL, "set_tuning: chunk must be a multiple of 32 in [32, 8192], chunk_tail one in [32, chunk]");
    if (t->reduction < 0 || t->reduction >= kNumReductions)
        return fail(p, PBA_EINVAL, "set_tuning: reduction must be 0 (shared-memory table) or 1 (shuffle butterfly)");
    const int old_reduction = p->prm.reduction;
    p->prm.reduction = t->reduction;  // (pba_set_variants drops the iteration graph)
    int st = pba_set_variants(p, t->variant_full, t->variant_cost);
    if (st) {
        p->prm.reduction = old_reduction;
        return st;
    }
    p->tune_ms_full = p->tune_ms_cost = 0.f;
    p->tune_from_cache = 0;
    if (p->cfg.path != PBA_PATH_BATCHED || p->M <= 0) {
        p->chunk = t->chunk;
        p->chunk_tail = t->chunk_tail;
        return PBA_OK;
    }
    p->linearized = false;
    return set_chunking(p, t->chunk, t->chunk_tail);
}

int pba_iteration_launches(pba_problem* p, int32_t* n_launches) {
    if (!p || !n_launches) return PBA_EINVAL;
    if (p->M <= 0) return fail(p, PBA_ENOTREADY, "pairs not set");
    if (!p->graph_exec) {
        // count without running: the same enqueue logic, on a capture that is discarded
        int nl = 0;
        CUDA_TRY(p, cudaStreamBeginCapture(p->capture_stream, cudaStreamCaptureModeThreadLocal));
        int st = enqueue_linearize(p, p->capture_stream, &nl);
        if (!st) st = enqueue_step(p, -1.0, p->capture_stream, &nl);
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(p->capture_stream, &g);
        if (g) cudaGraphDestroy(g);
        if (st) return st;
        *n_launches = nl;
        return PBA_OK;
    }
    *n_launches = p->launches_last;
    return PBA_OK;
}

}  // extern "C"
