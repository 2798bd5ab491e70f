/*
 * pba.h -- C ABI of the GB300 photometric bundle-adjustment library (libpba.so).
 *
 * The library linearises the multi-cue photometric error of Di Giammarino et
 * al., "Photometric LiDAR and RGB-D Bundle Adjustment" (Eq. total-error-multicue with the offset
 * form of the supplementary material), assembles the Gauss-Newton system
 * H dx = -b over all sensor poses, and takes damped (Levenberg-Marquardt)
 * steps X_k <- X_k [+] dx_k, all on one GPU.
 *
 * Conventions shared by every call:
 *   - Status: every int-returning call returns PBA_OK (0) or a negative
 *     PBA_E* code and never throws; pba_last_error() gives a message.
 *   - Ownership: input buffers are borrowed for the duration of the call
 *     only (the library copies what it keeps; the one exception is device
 *     memory given to pba_set_poses, read by a copy ordered on the problem's
 *     stream); outputs are caller-allocated.
 *     The problem object owns all device memory it allocates.
 *   - Host / device pointers: arguments documented "host or device" take an
 *     `is_device` flag; 1 means a pointer into the current CUDA device's
 *     global memory (e.g. a torch tensor's data_ptr()).
 *   - Streams: all device work is ordered on the stream given at creation
 *     (or pba_set_stream); calls that return results synchronise that stream.
 *   - Poses are 3x4 row-major [R | t] (Eq. 1) mapping the platform frame into
 *     the world frame, in double precision, frame k at offset 12 k.
 *   - Pose perturbations dx_k = [dt, dq] (Supp.): dt a translation, dq the
 *     imaginary part of a unit quaternion; X [+] dx = X exp(dx).
 *   - Not thread-safe per problem; distinct problems may be used from
 *     distinct threads.
 */
#ifndef PBA_H
#define PBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define PBA_OK 0
#define PBA_EINVAL (-1)     /* bad argument (null pointer, size, index, sensor mismatch) */
#define PBA_ENOMEM (-2)     /* device or host allocation failed */
#define PBA_ECUDA (-3)      /* a CUDA call failed; the message names it */
#define PBA_ENOTPD (-4)     /* damped system not positive definite; the step was rejected */
/* (-5 is not used: no kernel of the library waits on another) */
#define PBA_ENOTREADY (-6)  /* a required input (frames, poses, pairs) was not set */
#define PBA_ETOOBIG (-7)    /* a size exceeds the fixed maximum of pba_linearize_pairs_noalloc */

/* projection models, Sec. III */
#define PBA_PINHOLE 0       /* pi_p(p) = phi(K p), Eq. pinhole-projection; d is the depth */
#define PBA_SPHERICAL 1     /* pi_s(p) = K_[1,2] psi(p), Eq. spherical-projection; d is the range */

/* linearisation paths */
#define PBA_PATH_BATCHED 0  /* all pairs in one persistent launch, 6x6 reduced accumulation */
#define PBA_PATH_PLAIN 1    /* one launch per pair, full 12x12 accumulation, FP32 atomics */

/* storage of the target-image channels used for sampling (depth always FP32) */
#define PBA_TEXEL_F32 0
#define PBA_TEXEL_F16 1     /* intensity and normal in binary16 (round to nearest even) */

/* damped solve (Sec. IV-C, LM): all deliver the FP64 solution of
 * (H_ff + lambda I) dx_f = -b_f.  CHOLESKY_F64 factorises in FP64;
 * MIXED factorises the Jacobi-scaled system in FP32 and refines the solution
 * with FP64 residuals until |r| <= 1e-10 |b| (else the step is rejected and
 * lambda grows), which suits GB300's FP64 rate of ~1/64 of FP32.  MIXED runs
 * as one launch of a thread-block cluster holding the FP32 factor in shared
 * memory when the system fits (up to about 800 unknowns); larger systems,
 * unless a sensor offset is a variable, take the block-sparse solve of SPARSE;
 * otherwise one launch per tile step.  MIXED_STEPS always takes the per-step
 * launches (same arithmetic, kept for comparison).  SPARSE (same arithmetic)
 * gathers the system in pose variables block by block from the pair blocks,
 * orders each independent component of the pose graph for a small envelope
 * (natural or reverse Cuthill-McKee order), factorises in tile-envelope
 * storage and refines, one thread-block cluster per component in one launch;
 * with a sensor offset as a variable it takes the per-step launches. */
#define PBA_SOLVE_CHOLESKY_F64 0
#define PBA_SOLVE_MIXED 1
#define PBA_SOLVE_MIXED_STEPS 2
#define PBA_SOLVE_SPARSE 3

/* image-gradient modes (Supp., image Jacobians) */
#define PBA_GRAD_CENTRAL 0  /* central differences at pixels, bilinearly interpolated (paper) */
#define PBA_GRAD_BILINEAR 1 /* exact derivative of the bilinear interpolant */

typedef struct pba_problem pba_problem;

/* One sensor: intrinsics K (Eq. camera-matrix-p; for the spherical model f_x, f_y are the
 * azimuth / elevation resolutions in pixels per radian and c_x, c_y their
 * offsets, Eq. spherical-projection) and the extrinsic offset X_o = [R_o | t_o] (row-major 3x4)
 * placing the sensor on the platform (Supp., p_u = R_o pi^-1(u, d) + t_o). */
typedef struct {
    int32_t model;              /* PBA_PINHOLE or PBA_SPHERICAL */
    int32_t width, height;      /* image size in pixels; >= 4 each */
    int32_t reserved;           /* 0 */
    double fx, fy, cx, cy;
    double extrinsic[12];
} pba_sensor;

/* Problem configuration.  A pixel is valid iff range_min <= d <= range_max,
 * d > 0 and |n| > 0.5.  The residual of a pixel-point is the stacked
 * five-channel error e = (g, d, n_x, n_y, n_z) of the Supp. error term with
 * Omega = diag(w_int, w_depth, w_normal, w_normal, w_normal); the Huber
 * function acts on chi = sqrt(e^T Omega e) with threshold huber_delta.
 * A sample is rejected (occlusion suppression, Sec. IV-C) when
 * |zeta^d - I^d(u')| > occ_abs + occ_rel * zeta^d or the sampled normal has
 * norm < 0.5, and when pbar_z (pinhole) or |pbar| (spherical) <= z_min. */
typedef struct {
    int32_t n_frames;           /* N >= 1 */
    int32_t n_sensors;          /* >= 1 */
    const pba_sensor* sensors;  /* n_sensors entries, host memory */
    const int32_t* frame_sensor;/* n_frames entries (host) or NULL: every frame uses sensor 0 */
    double w_int, w_depth, w_normal;
    double huber_delta;         /* > 0 */
    double occ_abs, occ_rel;
    double z_min;
    double range_min, range_max;
    int32_t grad_mode;          /* PBA_GRAD_CENTRAL or PBA_GRAD_BILINEAR */
    int32_t texel_precision;    /* PBA_TEXEL_F32 or PBA_TEXEL_F16 (batched path only) */
    int32_t path;               /* PBA_PATH_BATCHED or PBA_PATH_PLAIN */
    int32_t solver;             /* PBA_SOLVE_CHOLESKY_F64, _MIXED, _MIXED_STEPS or _SPARSE */
} pba_config;

/* Outcome of one Levenberg-Marquardt iteration. */
typedef struct {
    double cost;        /* F (Eq. total-error-multicue) at the poses the iteration started from */
    double new_cost;    /* F at the candidate poses X [+] dx */
    double lambda_used; /* damping of the solved system (H_ff + lambda I) */
    double lambda_next; /* lambda / 10 after an accepted step, lambda * 10 otherwise */
    int64_t n_valid;    /* residuals (valid pixel-points over all pairs) linearised */
    int32_t accepted;   /* 1 when new_cost < cost and the poses were updated */
    int32_t status;     /* PBA_OK, or PBA_ENOTPD when the Cholesky met a non-positive pivot */
    /* status word of the same linearisation as n_valid (batched path; 0 on the
     * plain path): residuals left out of H, b and F because their value was
     * not finite (a NaN or infinite intensity or normal), and pairs whose
     * relative pose X_j^-1 X_i was not finite (a NaN or infinite pose; such a
     * pair yields no residual) */
    int64_t n_nonfinite;
    int64_t nonfinite_pairs;
} pba_iter_stats;

/* Create a problem on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL: the library creates its own non-blocking stream).
 * Allocates every device buffer whose size the configuration fixes.
 * Errors: PBA_EINVAL (bad config), PBA_ENOMEM, PBA_ECUDA. */
int pba_create(const pba_config* cfg, void* cuda_stream, pba_problem** out);

/* Free the problem and its device memory (synchronises its stream). NULL is a no-op. */
void pba_destroy(pba_problem* p);

/* Message of the last failed call on p.  With p NULL: the message of the
 * calling thread's last failed pba_create (which has no problem to hold it;
 * for example no CUDA device: the library has no CPU path), or "null problem"
 * when there was none.  The text stays valid until the next failing call on p
 * (or, for NULL, the thread's next failing pba_create). */
const char* pba_last_error(const pba_problem* p);

/* Order all further device work on cuda_stream (NULL: the problem's own stream).
 * Errors: PBA_EINVAL (p NULL), PBA_ECUDA. */
int pba_set_stream(pba_problem* p, void* cuda_stream);

/* Upload the five-channel cue images (Sec. IV-A) of frames first..first+count-1
 * and build their pixel-point clouds and sampling texels.  channels holds
 * count images back to back, each height x width x 5 float32 (row-major,
 * channel fastest: g, d, n_x, n_y, n_z; normals in the sensor frame), with the
 * frame's sensor size; host or device memory.  All frames of one call must
 * use sensors of the same size.  Errors: PBA_EINVAL, PBA_ECUDA. */
int pba_upload_frames(pba_problem* p, int first, int count, const float* channels, int is_device);

/* Replace the extrinsic offset X_o (row-major 3x4, host memory) of one
 * sensor (Supp., p_u = R_o pi^-1(u, d) + t_o): the pixel-points of that
 * sensor's uploaded frames are rebuilt; the next iteration relinearises.
 * Errors: PBA_EINVAL (bad sensor index, extrinsic NULL), PBA_ECUDA. */
int pba_set_extrinsic(pba_problem* p, int sensor, const double* extrinsic);

/* Normal estimation (Sec. IV-A) for the uploaded frames first..first+count-1,
 * computed from their depth channel and written over their normal channels
 * on the device; their texels and pixel-points are then rebuilt (and the
 * pair plan when a point count changed), as after pba_upload_frames.
 * For every pixel u with valid depth d (d > 0, range_min <= d <= range_max):
 * the valid pixels u' with |u - u'| < r(u) (pixel distance, columns wrapping
 * for the spherical model), r(u) = clamp(scale / d, 1.5, max_radius), are
 * unprojected; n_u is the normal of their least-squares plane (eigenvector
 * of the smallest eigenvalue of their covariance) oriented towards the
 * observer (n_u . p < 0).  A pixel with fewer than 5 such points, or whose
 * points are collinear (middle eigenvalue <= 1e-6 x largest), gets a zero
 * normal and so no pixel-point.  Arithmetic is float32.
 * Errors: PBA_EINVAL (bad range, scale not finite or < 0, max_radius outside
 * [2, PBA_NORMALS_MAX_RADIUS], a spherical image narrower than
 * 2 max_radius + 1 columns), PBA_ENOTREADY (a frame not uploaded),
 * PBA_ECUDA.  Synchronises. */
#define PBA_NORMALS_MAX_RADIUS 32
int pba_estimate_normals(pba_problem* p, int first, int count, float scale, int max_radius);

/* Copy the five-channel images of the uploaded frames first..first+count-1
 * (the layout of pba_upload_frames, frames back to back) to channels (host
 * memory, or device memory with is_device != 0).  Synchronises.
 * Errors: PBA_EINVAL, PBA_ENOTREADY (a frame not uploaded), PBA_ECUDA. */
int pba_get_channels(pba_problem* p, int first, int count, float* channels, int is_device);

/* Number of valid pixel-points of a frame (Sec. IV-A: its valid pixels, after
 * its upload).  Errors: PBA_EINVAL (bad frame, n_points NULL), PBA_ENOTREADY
 * (frame not uploaded). */
int pba_frame_points(pba_problem* p, int frame, int32_t* n_points);

/* Set all N poses X_k (Sec. III; N x 12 doubles in the pose convention above,
 * host or device memory).  The next iteration linearises at them first.
 * Host poses are copied before the call returns; device poses are copied by
 * work ordered on the problem's stream, without waiting, so they must stay
 * unchanged until that stream has passed this call (automatic when the
 * caller works on the same stream).  Errors: PBA_EINVAL (poses NULL),
 * PBA_ECUDA. */
int pba_set_poses(pba_problem* p, const double* poses, int is_device);

/* Read all N poses into host memory (N x 12 doubles); synchronises.
 * Errors: PBA_EINVAL (poses NULL), PBA_ECUDA. */
int pba_get_poses(pba_problem* p, double* poses);

/* Set the directed pairs (source i, target j), m x 2 int32 in host memory,
 * Sec. IV-B.  Both frames must use the same sensor; i == j is allowed.
 * Requires every frame named to have been uploaded.  Errors: PBA_EINVAL
 * (m < 0, pairs NULL with m > 0, a frame out of range, frames of different
 * sensors), PBA_ENOTREADY (a frame not uploaded), PBA_ENOMEM, PBA_ECUDA. */
int pba_set_pairs(pba_problem* p, const int32_t* pairs, int m);

/* Graph construction (Sec. IV-B): directed candidate pairs (i, j), i < j,
 * frames of the same sensor, whose poses differ by a rotation angle below
 * max_angle [rad] and a translation below max_dist [m] are tested in one
 * persistent launch of the cost-only linearisation at the current poses; a
 * pair is kept when the ratio of frame i's pixel-points that give a valid
 * residual against frame j (same validity rules as the residuals) exceeds
 * min_ratio.  With sequential != 0, every (i, i + 1) of the same sensor is
 * kept as well (odometry-like edges).  Writes up to cap pairs (m x 2 int32,
 * ascending i then j) to pairs_out and their ratios to ratio_out (either may
 * be NULL), and the number found to *m_out.  The problem's own pair list is
 * unchanged; pass the result to pba_set_pairs.  Needs poses and every frame
 * uploaded; synchronises.  PBA_EINVAL when cap is too small (*m_out then
 * holds the size needed). */
int pba_build_pairs(pba_problem* p, double max_angle, double max_dist, double min_ratio, int sequential,
                    int32_t* pairs_out, float* ratio_out, int cap, int32_t* m_out);

/* The gradient of F in the box-plus chart of the Supp. (X [+] dx =
 * [R R(dq), R dt + t], dx = [dt, dq]) from matrix gradients: for each of n
 * 3x4 transforms X_k (row-major [R | t]) and G_k = dF/dX_k (as
 * pba_cost_gradient returns them), g_k = dF/d dx_k at dx = 0:
 *   g_k[0..2] = R^T G_t,  g_k[3..5] = 2 (W_zy - W_yz, W_xz - W_zx, W_yx - W_xy),
 *   W = R^T G_R  (R(dq) = I + 2 [dq]x to first order).
 * X, G: n x 12 doubles, g: n x 6 doubles, device buffers of the problem's
 * device (caller-owned; G may be the d_poses of pba_cost_gradient, X the
 * poses it was evaluated at).  Enqueued on the problem's stream;
 * synchronises.  Errors: PBA_EINVAL (p NULL, n < 0, a NULL buffer with
 * n > 0), PBA_ECUDA. */
int pba_tangent_gradient(pba_problem* p, const double* X, const double* G, int n, double* g);

/* Linearise all pairs at the current poses: builds H (6N x 6N, gauge not
 * fixed) and b (6N) on the device and returns the total cost F (Eq. total-error-multicue) and
 * the number of valid residuals; synchronises.  Either output may be NULL.
 * Errors: PBA_EINVAL (p NULL), PBA_ENOTREADY (poses or pairs not set),
 * PBA_ECUDA. */
int pba_linearize(pba_problem* p, double* cost, int64_t* n_valid);

/* Adjoint of the total cost F (Eq. total-error-multicue) at the current
 * poses.  One launch recomputes every residual (no Jacobian is stored) and
 * accumulates the gradient of F, the validity decisions (bounds, stencil,
 * occlusion, Huber branch) held fixed:
 *   d_poses     N x 12 doubles: dF/dX_k, the derivative with respect to the
 *               entries of each 3x4 pose [R_k | t_k] (F evaluated with the
 *               paper's formulas for any 3x4 matrices; pba_tangent_gradient
 *               turns it into the gradient in the box-plus chart);
 *   d_extrinsic S x 12 doubles: dF/dX_o per sensor, likewise;
 *   d_channels  one float per channel of every uploaded pixel (the layout of
 *               pba_upload_frames, frames back to back): dF/d(g, d, n) through
 *               the bilinear samples of the targets and the source pixels.
 * Image derivatives use the exact derivative of the bilinear interpolant.
 * All three are caller-allocated device buffers of the current device (any
 * may be NULL); cost and n_valid (host, may be NULL) receive F and the number
 * of valid residuals.  Batched path only; synchronises. */
int pba_cost_gradient(pba_problem* p, double* cost, int64_t* n_valid, double* d_poses, double* d_extrinsic,
                      float* d_channels);

/* Copy the last linearisation's Gauss-Newton system (Sec. IV-C: H = sum of
 * w J^T Omega J and b = sum of w J^T Omega e over every residual of Eq.
 * total-error-multicue, J = [J_i J_j] from the Supp. Jacobians) to host
 * memory: H (6N x 6N row-major) and b (6N); either may be NULL.  Frame k owns
 * rows and columns 6k..6k+5.  Errors: PBA_EINVAL, PBA_ENOTREADY (no
 * linearisation yet), PBA_ECUDA. */
int pba_get_system(pba_problem* p, double* H, double* b);

/* Copy the last linearisation's per-pair results to host memory: pair_H
 * (m x 12 x 12: rows/cols 0-5 frame i, 6-11 frame j), pair_b (m x 12),
 * pair_cost (m), pair_count (m).  Any may be NULL.  Errors: PBA_EINVAL,
 * PBA_ENOTREADY (no linearisation yet), PBA_ECUDA. */
int pba_get_pair_system(pba_problem* p, double* pair_H, double* pair_b, double* pair_cost,
                        int64_t* pair_count);

/* Enable (1) or disable (0) export of the valid-residual mask (which
 * pixel-points pass the validity and occlusion rules of Sec. IV-C) by later
 * linearisations.  Errors: PBA_EINVAL (p NULL, or enabling on the plain
 * path). */
int pba_set_mask_export(pba_problem* p, int enable);

/* Copy the valid-residual mask of one pair from the last linearisation with
 * mask export on: bit k % 32 of word k / 32 is set when the k-th pixel-point
 * (raster order) of the source frame gave a valid residual.  n_words must be
 * >= ceil(P_i / 32).  Errors: PBA_EINVAL, PBA_ENOTREADY (no mask exported). */
int pba_get_mask(pba_problem* p, int pair, uint32_t* bits, int n_words);

/* One damped (Levenberg-Marquardt, Sec. IV-C) step from the last
 * linearisation with the given lambda >= 0: solve (H_ff + lambda I) dx_f =
 * -b_f with frame 0 held fixed (gauge), evaluate F at X [+] dx, keep the
 * candidate when F decreased.  Fills stats (may be NULL); synchronises.
 * Returns PBA_OK even when the step is rejected; stats->status reports
 * PBA_ENOTPD.  Errors: PBA_EINVAL (lambda < 0 or NaN), PBA_ENOTREADY (poses
 * or pairs not set, no linearisation), PBA_ECUDA. */
int pba_solve_step(pba_problem* p, double lambda, pba_iter_stats* stats);

/* Damping used by pba_iterate (Sec. IV-C, Levenberg-Marquardt): lambda >= 0
 * sets it, lambda < 0 resets it to automatic (1e-4 times the largest diagonal
 * entry of H_ff on the next iteration).  The schedule then divides by 10 on
 * acceptance and multiplies by 10 on rejection, on the device.
 * Errors: PBA_EINVAL (p NULL), PBA_ECUDA. */
int pba_set_lambda(pba_problem* p, double lambda);

/* One full Levenberg-Marquardt iteration (Sec. IV-C) with the device-side lambda
 * schedule: damp and solve the current system, form the candidate poses,
 * linearise fully at the candidate, and accept (the candidate's poses and
 * system become current) or reject (nothing changes).  The first iteration
 * after new poses, frames or pairs first linearises at the current poses.
 * stats->cost is F at the start, stats->new_cost F at the candidate,
 * stats->n_valid the residuals of the candidate's linearisation.  Fills stats
 * (may be NULL) and synchronises.  A rejected or not positive definite step
 * is an outcome (stats), not an error.  Errors: PBA_EINVAL (p NULL),
 * PBA_ENOTREADY (poses or pairs not set), PBA_ECUDA. */
int pba_iterate(pba_problem* p, pba_iter_stats* stats);

/* One Levenberg-Marquardt iteration (Sec. IV-C) on new images of all N
 * frames: sets the poses (host memory, N x 12; NULL keeps the current ones),
 * uploads channels, linearises at the poses, damps and solves, and evaluates
 * F at the candidate (the system there is not formed: the next iteration
 * linearises afresh) before accepting or rejecting it.  channels holds every
 * frame back to back in frame order, each height x width x 5 float32 of its
 * sensor as in pba_upload_frames (the layout pba_get_channels writes for
 * frames 0 .. N-1), in host memory; page-locked memory lets the copies overlap
 * the computation.  Once every frame has been uploaded before, the frames are
 * copied in lanes of whole frames in frame order, each lane packed as soon as
 * it has arrived, and the work items of each pair are linearised as soon as
 * both its frames are packed, while later lanes are still in flight.  That
 * linearisation uses the pair plan of the previous point counts; when a
 * frame's count has changed, the plan is rebuilt and the pass redone before
 * the step (the same result, without the overlap).  Before every frame has
 * been uploaded: pba_upload_frames of each run of same-size frames, then the
 * iteration.  The result equals pba_upload_frames, pba_linearize and one
 * damped step with the device-side lambda schedule.  channels must stay
 * unchanged until the call returns.  Fills stats (may be NULL; n_valid is the
 * residual count of the linearisation at the given poses); synchronises.  Errors: PBA_EINVAL (p or
 * channels NULL), PBA_ENOTREADY (pairs not set, or poses neither given nor
 * set), PBA_ECUDA. */
int pba_iterate_frames(pba_problem* p, const float* channels, const double* poses, pba_iter_stats* stats);

/* Enqueue n iterations as replays of one captured CUDA graph without
 * synchronising; pba_get_stats() then reads the last iteration's outcome.
 * Errors: as pba_iterate, and PBA_EINVAL for n < 0. */
int pba_iterate_async(pba_problem* p, int n);

/* Synchronise and read the outcome of the last iteration.  Errors:
 * PBA_EINVAL (p NULL), PBA_ECUDA. */
int pba_get_stats(pba_problem* p, pba_iter_stats* stats);

/* The current offset X_o of one sensor (row-major 3x4, host memory).
 * Errors: PBA_EINVAL. */
int pba_get_extrinsic(pba_problem* p, int sensor, double* extrinsic);

/* Refine one sensor's offset X_o (Supp., offset form) at the current poses
 * by quasi-Newton (BFGS) descent of F over its 6 box-plus coordinates, with
 * the adjoint gradient of pba_cost_gradient and a backtracking (Armijo)
 * line search; the first step moves at most 0.01 in the chart (1 cm or
 * ~1 deg).  Stops after max_iters iterations or at the first step whose
 * relative decrease of F is below rel_tol.  The refined offset is the
 * sensor's extrinsic afterwards (as after pba_set_extrinsic).  Alternating
 * it with pose iterations (pba_iterate / pba_optimize) refines poses and
 * offset jointly.  Host or device outputs: cost_before, cost_after (F before
 * and after) and iterations (host, any may be NULL).  Needs poses, pairs and
 * the batched path; allocates a small device buffer; synchronises.
 * Errors: PBA_EINVAL, PBA_ENOTREADY, PBA_ENOMEM, PBA_ECUDA. */
int pba_refine_extrinsic(pba_problem* p, int sensor, int max_iters, double rel_tol, double* cost_before,
                         double* cost_after, int32_t* iterations);

/* Pose variables of the damped solve.  By default frame 0 is held fixed (the
 * gauge) and every other frame k moves with its own variable.  frame_var
 * (n_frames entries, host memory) instead maps frame k to variable
 * frame_var[k] in [0, n_vars), or to -1 to hold it fixed: frames sharing a
 * variable move together, e.g. the frames of several sensors rigidly mounted
 * on one platform and captured at one platform pose (the coupled multi-sensor
 * problem of Sec. V, fusion), or a fixed frame per independent sub-problem.
 * The step solves (S^T H S + lambda I) dx_v = -S^T b, S the 0/1 selection
 * (frame k's perturbation is dx_v[frame_var[k]]), and applies dx_v to every
 * frame of each variable; the initial lambda is 1e-4 max diag(S^T H S).
 * Frames tied to one variable should carry equal poses (their common
 * perturbation keeps them equal).  frame_var = NULL restores the default.
 * pba_get_system still returns the per-frame H and b.  Errors: PBA_EINVAL
 * (n_vars outside [1, n_frames - 1], an entry outside [-1, n_vars), no frame
 * held fixed, a variable without frames), PBA_ENOMEM, PBA_ECUDA. */
int pba_set_variables(pba_problem* p, const int32_t* frame_var, int n_vars);

/* Make the offset X_o of one sensor a variable of the damped solve (is_free
 * != 0) or hold it fixed again (0, the default).  The paper holds offsets
 * fixed (Supp., offset form); as a variable its Jacobian follows from the
 * first-order identity J_o = (J_i + J_j) A_o, A_o = [[R_o, 2 [t_o]x R_o],
 * [0, R_o]] (a right perturbation of X_o acts like the perturbation
 * X_o exp(d) X_o^-1 of both poses), so the offset blocks of every pair come
 * from its H12 and b12 in FP64.  Each iteration then moves the free offsets
 * with the poses, rebuilds the pixel-points of their frames for the
 * candidate, and again after the accept decision.  With one sensor the
 * offset and the poses share a 6-dimensional gauge: free an offset when
 * another sensor's offset is fixed and the sensors' frames are tied by
 * pba_set_variables (coupled platforms), or with fixed frames.
 * pba_get_extrinsic reads the refined offsets.  Drops the iteration graph.
 * Errors: PBA_EINVAL (bad sensor, too many unknowns), PBA_ENOMEM, PBA_ECUDA. */
int pba_set_offset_free(pba_problem* p, int sensor, int is_free);

/* ---- Pyramid and coarse-to-fine optimisation (Sec. IV-A, Sec. IV-C) ----
 *
 * Level 0 is the problem itself; level l + 1 halves the resolution of level
 * l (sizes rounded down; each level at least 4 x 4).  A coarse pixel
 * summarises a 2 x 2 block: valid when all four fine pixels are valid, then
 * g and d are the block means and n the normalised sum of the four normals
 * (float64 sums of the float32 inputs, rounded once to float32).  Its
 * intrinsics are f' = f / 2, c' = (c + 1/2) / 2 - 1/2 (the coarse pixel k is
 * centred on fine coordinate 2k + 1/2), for both models; extrinsics,
 * weights, thresholds, path, texels and solver are those of the problem. */
#define PBA_MAX_LEVELS 8

/* Build levels 1..n_levels-1 from the uploaded frames (downsampled on the
 * device), with the problem's poses and pairs.  Each level is a problem of
 * its own, owned by p and on p's stream.  Uploading frames, estimating
 * normals, setting pairs or an extrinsic afterwards makes the pyramid stale
 * (PBA_ENOTREADY from the calls below until it is rebuilt).  Allocates;
 * synchronises.  Errors: PBA_EINVAL (n_levels outside [1, PBA_MAX_LEVELS],
 * a level below 4 x 4), PBA_ENOTREADY (a frame not uploaded), PBA_ENOMEM,
 * PBA_ECUDA. */
int pba_build_pyramid(pba_problem* p, int n_levels);

/* The problem of one level (borrowed: owned by p, valid until the pyramid is
 * rebuilt or p destroyed; level 0 returns p).  Every entry point applies to
 * it, e.g. to linearise at a coarse level.  Errors: PBA_EINVAL (no such
 * level), PBA_ENOTREADY (stale pyramid). */
int pba_pyramid_level(pba_problem* p, int level, pba_problem** level_out);

/* Outcome of one level of pba_optimize. */
typedef struct {
    int32_t level;       /* 0 = finest */
    int32_t iterations;  /* LM iterations run (accepted or not) */
    int32_t accepted;
    int32_t status;      /* PBA_OK, or PBA_ENOTPD when some step met a non-positive pivot */
    double cost_first;   /* F at the level's starting poses */
    double cost_last;    /* F at the level's final poses */
} pba_level_stats;

/* Hierarchical optimisation (Sec. IV-C): Levenberg-Marquardt on level
 * n_levels-1 (coarsest) first, then on each finer level from the poses
 * reached so far, ending on level 0, whose poses are the problem's.  Each
 * level starts with automatic damping and runs at most max_iters[k]
 * iterations (k = 0 the coarsest), ending early at the first accepted step
 * whose relative decrease (F - F_new) / F is below rel_tol (the paper's
 * error-variation criterion).  stats (n_levels entries, coarsest first) may
 * be NULL.  Synchronises after every iteration.  Errors: PBA_EINVAL,
 * PBA_ENOTREADY (stale pyramid, poses or pairs not set), PBA_ECUDA. */
int pba_optimize(pba_problem* p, int n_levels, const int32_t* max_iters, double rel_tol, pba_level_stats* stats);

/* Number of kernel launches one pba_iterate performs (for accounting; captures
 * the iteration graph when there is none).  Errors: PBA_EINVAL,
 * PBA_ENOTREADY (poses or pairs not set), PBA_ECUDA. */
int pba_iteration_launches(pba_problem* p, int32_t* n_launches);

/* Variants of the batched linearisation kernel: register budgets for 4, 6, 7
 * or 5 (full pass) and 6, 7, 9 or 10 (cost-only pass) blocks of 128 threads
 * per SM, variants 0 .. 3; variants 4 .. 7 have the same budgets and read each
 * 32-point step's bilinear taps from a 4 x 48-pixel tile of the target's
 * texels that one TMA tensor copy staged in shared memory (FP16 texels and
 * frames of at least 48 x 4 pixels; otherwise, and for the linearisation with
 * mask export, they run as variants 0 .. 3).  The results agree up to float32
 * summation order. */
#define PBA_N_VARIANTS 8

/* Tune the batched linearisation on this problem by timing it (each setting
 * launched repeats + 1 times, the first as warm-up): for the full pass every
 * work-item size (512, 1024, 2048 points per warp item, i.e. 16, 32 or 64
 * points per lane) x size of the short items that end the queue (128, 256) x
 * variant (0 .. PBA_N_VARIANTS - 1; the staged variants 4 .. 7 only where
 * tiles are staged) x reduction scheme of a work item's sums (0, 1: see
 * pba_tuning), then for the cost-only pass the variants at the chosen work
 * items; settings within 2 % of the fastest count as equal, and the first of
 * them in that order (work-item size, then tail size and variant, each
 * ascending, then reduction 1 before 0) is kept, so that timing noise does
 * not change the choice between runs.  Later
 * iterations use the choice (pba_get_tuning reports it).  The result is
 * cached for the life of the process per configuration (device, texel
 * precision, gradient mode, pairs, point counts, sensors): tuning the same
 * configuration again applies it without timing.  Rebuilds the pair plan
 * when the work items change.  Reports the variants (0 .. PBA_N_VARIANTS - 1)
 * in the optional outputs.  Needs frames, poses and pairs; synchronises.  A
 * no-op on the plain path.  Errors: PBA_EINVAL, PBA_ENOTREADY (poses or pairs
 * not set), PBA_ECUDA. */
int pba_autotune(pba_problem* p, int repeats, int32_t* variant_full, int32_t* variant_cost);

/* The settings the last pba_autotune chose (or the defaults): occupancy
 * variants of the full and the cost-only pass, the work-item size (points per
 * warp work item: 512, 1024 or 2048) and the size of the short items at the
 * end of the queue (128 or 256), the reduction of each work item's 30 FP32
 * sums into its partial (0: each lane writes its sums as one column of a
 * transposed table in the warp's shared memory and lane j adds row j; 1: a
 * butterfly of warp shuffles in which every level halves the values a lane
 * holds, lane j ending with sum j; the two differ only in float32 summation
 * order), whether they came from the process's cache of tuned
 * configurations (same device, texel precision, gradient mode,
 * pairs, point counts and sensors: no timing was done), whether a staged
 * tile's wait ran past its limit since the problem was created (tile_err: 1;
 * the taps are then read directly, the results stay exact), and the mean time
 * of one full and one cost-only pass with them (0 before any tuning).
 * Errors: PBA_EINVAL (a NULL argument). */
typedef struct {
    int32_t variant_full, variant_cost;
    int32_t chunk, chunk_tail;
    int32_t from_cache, tile_err;
    float ms_full, ms_cost;
    int32_t reduction;
} pba_tuning;
int pba_get_tuning(pba_problem* p, pba_tuning* out);

/* Set the variants explicitly (e.g. to reproduce a tuned configuration).
 * Errors: PBA_EINVAL (a variant outside [0, PBA_N_VARIANTS)). */
int pba_set_variants(pba_problem* p, int variant_full, int variant_cost);

/* Apply a tuning given by the caller (e.g. one pba_get_tuning reported in an
 * earlier process) without timing anything: its variants, work-item size,
 * tail item size and reduction scheme; from_cache, ms_full and ms_cost are
 * ignored (reported as 0 afterwards).  Rebuilds the pair plan when the work items change.  On the
 * plain path only the values are recorded.  Errors: PBA_EINVAL (tuning NULL, a
 * variant outside [0, PBA_N_VARIANTS), chunk not a multiple of 32 in
 * [32, 8192], chunk_tail not a multiple of 32 in [32, chunk], reduction not
 * 0 or 1), PBA_ECUDA. */
int pba_set_tuning(pba_problem* p, const pba_tuning* tuning);

/* Instrumentation: one iteration like pba_iterate, enqueued launch by launch
 * (not as a graph) with CUDA events recorded on the problem's stream between
 * its phases; writes min(n_phases, PBA_N_PHASES) device times in
 * milliseconds: [0] damping + solve, [1] box-plus + candidate transforms,
 * [2] the linearisation kernel at the candidate, [3] per-pair reduction +
 * assembly + cost, [4] accept / reject (and the swap of the system).  Fills
 * stats (may be NULL); synchronises.  Errors: as pba_iterate. */
#define PBA_N_PHASES 5
int pba_iterate_timed(pba_problem* p, float* phase_ms, int n_phases, pba_iter_stats* stats);

/* ------------------------------------------------------------------------
 * Linearisation without allocation.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory -- code that is
 * handed its device buffers by a host framework which owns the memory pool,
 * or a loop whose memory budget is fixed at start-up, where a cudaMalloc could
 * fail or stall the device mid-run.  It performs no cudaMalloc, cudaFree or
 * other allocation: its working memory is a static device array of
 * PBA_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits.
 *
 * It linearises m directed pairs (i, j) of frames that share one sensor with
 * the residual, Jacobians, robust weights and validity rules of pba_linearize
 * on the plain path, and agrees with it within the parity tolerances (not bit
 * for bit: sums are formed in another order; cfg->texel_precision,
 * cfg->path and cfg->n_frames / sensors / frame_sensor are ignored), and
 * writes per pair PBA_NOALLOC_PAIR_STRIDE doubles to pair_out: H12 (144,
 * rows/cols 0-5 frame i, 6-11 frame j), b12 (12), cost, count, 2 zeros --
 * the layout of pba_get_pair_system.
 *
 * Arguments: sensor, cfg in host memory; channels (n_frames x H x W x 5
 * float32, layout of pba_upload_frames), poses (n_frames x 12 doubles), pairs
 * (m x 2 int32) and pair_out in device memory of the current device, all
 * owned by the caller; cuda_stream orders the work (NULL: legacy stream); the
 * call does not synchronise.  A pair naming a frame outside [0, n_frames)
 * yields an all-zero block.
 *
 * Limits and errors: PBA_ETOOBIG when m > PBA_NOALLOC_MAX_PAIRS or the image
 * has more than 2^30 pixels; PBA_EINVAL for null pointers or a bad sensor /
 * configuration; PBA_ECUDA when a launch fails.
 *
 * Sharing: every call looks up the array's device address on the current
 * device (a host-side query); make the first call on a device before any
 * stream capture.  Every call reuses the same array and clears the accumulators it uses, so
 * the array keeps the previous call's contents until then; calls whose device
 * work overlaps (other streams or threads) race on it and must be serialised
 * by the caller. */
#define PBA_NOALLOC_MAX_PAIRS 4096
#define PBA_NOALLOC_SCRATCH_BYTES (2u * 1024u * 1024u)
#define PBA_NOALLOC_PAIR_STRIDE 160
int pba_linearize_pairs_noalloc(const pba_sensor* sensor, const pba_config* cfg, const float* channels, int n_frames,
                                const double* poses, const int32_t* pairs, int m, double* pair_out,
                                void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* PBA_H */
