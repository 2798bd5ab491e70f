/*
 * pba_oracle.c -- plain, slow FP64 CPU oracle of the photometric bundle
 * adjustment linearisation and damped Gauss-Newton / Levenberg-Marquardt step
 * (Di Giammarino et al., "Photometric LiDAR and RGB-D Bundle Adjustment").
 *
 * TEST INFRASTRUCTURE ONLY.  It exists to check the CUDA path; the product
 * path never calls it.  It shares no code, header, table or constant with the
 * CUDA library, and neither includes nor links the other.
 *
 * Every function follows the paper's definitions literally, one point at a
 * time, in double precision, with no blocking, fusion or reordering:
 *   - rigid transforms and their inverse ............... Eq. 1
 *   - pinhole projection pi_p = phi(K p) ............... Eq. pinhole-projection
 *   - spherical projection pi_s = K_[1,2] psi(p) ....... Eq. spherical-projection
 *   - unprojection pi^-1(u, d) (depth / range) ......... Sec. III
 *   - five-channel cue image (g, d, n) ................. Sec. IV-A
 *   - u' and the relative transform .................... Eq. uprime
 *   - multi-cue robust error F ......................... Eq. total-error-multicue
 *   - offset points p_u, pbar_u and the error e ........ Supp., Eq. error-jacobian
 *   - perturbed points and their Jacobians ............. Supp., dpbar/dDx_i, dpbar/dDx_j
 *   - projection Jacobians (pinhole, spherical) ........ Supp.
 *   - image Jacobians by central differences ........... Supp.
 *   - cue mapping Jacobians (intensity, depth, range,
 *     normals) and the full J_i, J_j ................... Supp., Eq. normal-error-jacobian
 *   - box-plus X [+] Dx = X exp(Dx), Dx = [Dt, Dq] ..... Supp. (first paragraph)
 *   - Levenberg-Marquardt (the paper uses srrg2_solver;
 *     the normal equations H = sum w J^T Omega J,
 *     b = sum w J^T Omega e, damping H + lambda I,
 *     gauge fixed on frame 0, dense Cholesky) ........ Sec. IV-C
 *
 * Readings taken where the paper is silent or garbled (each also listed in the
 * design notes of the repository):
 *   R1  the Huber rho acts on chi = sqrt(e^T Omega e); w = 1 if chi <= delta,
 *       else delta / chi; rho = chi^2 or 2 delta chi - delta^2.
 *   R2  the channel norm of Eq. total-error-multicue is the stacked weighted norm
 *       sum_c Omega^c (e^c)^2 with Omega = diag(w_g, w_d, w_n, w_n, w_n).
 *   R3  R(Dq) ~ I + 2 [Dq]x, so d(R(Dq) p)/dDq = -2 [p]x with [a]x b = a x b;
 *       the Supp. "2 [p]x" is read with the opposite skew convention.
 *   R4  the normal Jacobian for frame i uses R_j^T (the Supp. prints R_j).
 *   R5  image gradients are the central differences of the Supp. at pixel
 *       centres, bilinearly interpolated at u' (grad_mode 0); grad_mode 1
 *       takes the exact derivative of the bilinear interpolant instead.
 *       Gradient order is (d/du, d/dv) = (d/dcolumn, d/drow), matching pi.
 *   R6  a pixel is valid iff range_min <= d <= range_max, d > 0 and |n| > 0.5;
 *       a sample at u' is usable iff the 12 texels of the central-difference
 *       stencil of its 4 bilinear taps are valid; column indices wrap
 *       modulo W for the spherical model; rows never wrap.
 *   R7  occlusion suppression (Sec. IV-C, mechanism not given): reject when
 *       |zeta^d - I_j^d(u')| > occ_abs + occ_rel * zeta^d, or when the sampled
 *       target normal has norm < 0.5.
 *   R8  pinhole points with pbar_z <= z_min and spherical points with
 *       |pbar| <= z_min are rejected.
 *   R9  integer pixel coordinates are pixel centres; column = u, row = v.
 *   R10 X [+] Dx = [R R(Dq), R Dt + t], R(Dq) from the unit quaternion
 *       (sqrt(1 - |Dq|^2), Dq) (normalised (1, Dq) when |Dq| >= 1).
 *   R24 d pbar / d Dx_j = R_o^T [-I | 2 [q]x]: the Supp. derivation of the
 *       target's perturbation leaves out the rotation R(-Dq) acting on Dt,
 *       which changes nothing at first order, the order a Jacobian keeps.
 *
 * Decision margins: the oracle flags a point when a validity decision lies
 * within `margin_px` pixels (projections against integers) or `margin_rel`
 * (relative, depth and norm tests) of its threshold, because a float32
 * implementation may take the other branch there.  A sample position off by
 * up to margin_px moves an interpolated value by its bilinear slope times
 * margin_px, so the occlusion and normal-norm tests, which compare
 * interpolated values, widen their margins by that amount (large at depth or
 * normal discontinuities).
 *
 * With other_branch set, o_point_residual takes the other branch of every
 * rejection whose decision lies within its margin (z_min, occlusion, normal
 * norm; a sample that is not usable at u' is taken at u' moved by 2
 * margin_px towards the neighbouring cell), so that a test can evaluate the
 * contribution of a point that a float32 implementation counted and the
 * oracle did not.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_PINHOLE 0
#define O_SPHERICAL 1

typedef struct {
    int model;
    int width, height;
    int pad_;
    double fx, fy, cx, cy;
    double Xo[12]; /* extrinsic X_o, row-major 3x4 [R_o | t_o] */
} o_sensor;

typedef struct {
    double w_int, w_depth, w_normal; /* Omega diagonal (R2) */
    double huber_delta;              /* R1 */
    double occ_abs, occ_rel;         /* R7 */
    double z_min;                    /* R8 */
    double range_min, range_max;     /* R6 */
    double margin_px, margin_rel;    /* decision margins */
    int grad_mode;                   /* R5 */
    int other_branch;                /* 1: a rejection whose decision lies within its margin is overruled */
    int texel_f16;                   /* R25: target g and n sampled as binary16 values */
} o_params;

/* ---------------------------------------------------------------- algebra */

/* 3x3 row-major helpers */
static void mat3_mul(const double A[9], const double B[9], double C[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
            C[3 * r + c] = s;
        }
}
static void mat3_T(const double A[9], double T[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) T[3 * c + r] = A[3 * r + c];
}
static void mat3_vec(const double A[9], const double v[3], double out[3]) {
    for (int r = 0; r < 3; ++r) out[r] = A[3 * r] * v[0] + A[3 * r + 1] * v[1] + A[3 * r + 2] * v[2];
}
static void rot_of(const double X[12], double R[9]) {
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) R[3 * r + c] = X[4 * r + c];
}
static void trans_of(const double X[12], double t[3]) {
    t[0] = X[3]; t[1] = X[7]; t[2] = X[11];
}
/* [a]x : the matrix with [a]x b = a x b */
static void skew(const double a[3], double S[9]) {
    S[0] = 0.0;   S[1] = -a[2]; S[2] = a[1];
    S[3] = a[2];  S[4] = 0.0;   S[5] = -a[0];
    S[6] = -a[1]; S[7] = a[0];  S[8] = 0.0;
}

/* ------------------------------------------------------- Sec. III models */

/* Eq. pinhole-projection and Eq. spherical-projection: image coordinates of p. */
void o_project(const o_sensor* s, const double p[3], double uv[2]) {
    if (s->model == O_PINHOLE) {
        /* v = K p ; phi(v) = (v_x / v_z, v_y / v_z) */
        double vx = s->fx * p[0] + s->cx * p[2];
        double vy = s->fy * p[1] + s->cy * p[2];
        double vz = p[2];
        uv[0] = vx / vz;
        uv[1] = vy / vz;
    } else {
        /* psi(p) = (atan2(y, x), atan2(z, sqrt(x^2 + y^2)), 1); K_[1,2] psi */
        double az = atan2(p[1], p[0]);
        double el = atan2(p[2], sqrt(p[0] * p[0] + p[1] * p[1]));
        uv[0] = s->fx * az + s->cx;
        uv[1] = s->fy * el + s->cy;
    }
}

/* Sec. III: p = pi^-1(u, d); d is the depth (pinhole) or the range (spherical). */
void o_unproject(const o_sensor* s, double u, double v, double d, double p[3]) {
    if (s->model == O_PINHOLE) {
        /* p = d K^-1 [u v 1]^T */
        p[0] = d * (u - s->cx) / s->fx;
        p[1] = d * (v - s->cy) / s->fy;
        p[2] = d;
    } else {
        double az = (u - s->cx) / s->fx;
        double el = (v - s->cy) / s->fy;
        p[0] = d * cos(el) * cos(az);
        p[1] = d * cos(el) * sin(az);
        p[2] = d * sin(el);
    }
}

/* Supp., projection Jacobians: d pi / d p (2x3, row-major). */
void o_proj_jacobian(const o_sensor* s, const double p[3], double J[6]) {
    if (s->model == O_PINHOLE) {
        /* (1/v_z^2) [[v_z, 0, -v_x], [0, v_z, -v_y]] K  with v = K p */
        double vx = s->fx * p[0] + s->cx * p[2];
        double vy = s->fy * p[1] + s->cy * p[2];
        double vz = p[2];
        double P[6] = {vz, 0.0, -vx, 0.0, vz, -vy};
        double K[9] = {s->fx, 0.0, s->cx, 0.0, s->fy, s->cy, 0.0, 0.0, 1.0};
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += P[3 * r + k] * K[3 * k + c];
                J[3 * r + c] = acc / (vz * vz);
            }
    } else {
        /* K_[1,2] d psi / d p, v = p */
        double x = p[0], y = p[1], z = p[2];
        double rxy2 = x * x + y * y;
        double rxy = sqrt(rxy2);
        double r2 = rxy2 + z * z;
        double D[9] = {-y / rxy2, x / rxy2, 0.0,
                       -x * z / (rxy * r2), -y * z / (rxy * r2), rxy / r2,
                       0.0, 0.0, 0.0};
        double K12[6] = {s->fx, 0.0, s->cx, 0.0, s->fy, s->cy};
        for (int r = 0; r < 2; ++r)
            for (int c = 0; c < 3; ++c) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += K12[3 * r + k] * D[3 * k + c];
                J[3 * r + c] = acc;
            }
    }
}

/* Supp.: X [+] Dx = X exp(Dx), Dx = [Dt, Dq] (reading R10). */
void o_boxplus(const double X[12], const double dx[6], double out[12]) {
    double qx = dx[3], qy = dx[4], qz = dx[5];
    double n2 = qx * qx + qy * qy + qz * qz;
    double qw;
    if (n2 < 1.0) {
        qw = sqrt(1.0 - n2);
    } else {
        double n = sqrt(1.0 + n2);
        qw = 1.0 / n; qx /= n; qy /= n; qz /= n;
    }
    double dR[9] = {
        1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qw * qz),     2 * (qx * qz + qw * qy),
        2 * (qx * qy + qw * qz),     1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qw * qx),
        2 * (qx * qz - qw * qy),     2 * (qy * qz + qw * qx),     1 - 2 * (qx * qx + qy * qy)};
    double R[9], t[3], RdR[9], Rdt[3];
    rot_of(X, R);
    trans_of(X, t);
    mat3_mul(R, dR, RdR);
    mat3_vec(R, dx, Rdt);
    for (int r = 0; r < 3; ++r) {
        for (int c = 0; c < 3; ++c) out[4 * r + c] = RdR[3 * r + c];
        out[4 * r + 3] = Rdt[r] + t[r];
    }
}

/* ------------------------------------------------------ Sec. IV-A pixels */

static int pixel_valid(const o_params* prm, const float* px) {
    double d = px[1];
    double n2 = (double)px[2] * px[2] + (double)px[3] * px[3] + (double)px[4] * px[4];
    return d > 0.0 && d >= prm->range_min && d <= prm->range_max && n2 > 0.25;
}

/*
 * Pixel-points of one frame in raster order (row-major, column fastest).
 * For each valid pixel u: p_u = R_o pi^-1(u, d) + t_o (Supp., p_u), its
 * intensity g_u and its normal rotated into the platform frame n_u^o = R_o n_u.
 * out[7 k + 0..2] = p_u, out[7 k + 3] = g_u, out[7 k + 4..6] = n_u^o;
 * pix[k] = row * W + column.  Returns the number of points (<= cap).
 */
int o_frame_points(const o_sensor* s, const o_params* prm, const float* ch, double* out,
                   int32_t* pix, int cap) {
    double Ro[9], to[3];
    rot_of(s->Xo, Ro);
    trans_of(s->Xo, to);
    int k = 0;
    for (int r = 0; r < s->height; ++r)
        for (int c = 0; c < s->width; ++c) {
            const float* px = ch + 5 * ((size_t)r * s->width + c);
            if (!pixel_valid(prm, px)) continue;
            if (k >= cap) return -1;
            double p[3], pu[3], n[3] = {px[2], px[3], px[4]}, no[3];
            o_unproject(s, (double)c, (double)r, (double)px[1], p);
            mat3_vec(Ro, p, pu);
            for (int a = 0; a < 3; ++a) pu[a] += to[a];
            mat3_vec(Ro, n, no);
            double* o = out + 7 * (size_t)k;
            o[0] = pu[0]; o[1] = pu[1]; o[2] = pu[2];
            o[3] = px[0];
            o[4] = no[0]; o[5] = no[1]; o[6] = no[2];
            if (pix) pix[k] = r * s->width + c;
            ++k;
        }
    return k;
}

/* ----------------------------------------------------- sampling at u' */

static const float* texel(const o_sensor* s, const float* ch, int r, int c) {
    if (s->model == O_SPHERICAL) {
        c %= s->width;
        if (c < 0) c += s->width;
    }
    return ch + 5 * ((size_t)r * s->width + c);
}

/*
 * Reading R25 (FP16 image channels): with half-precision texels the target's
 * intensity and normal channels are sampled as their binary16 values (depth
 * stays float32; a pixel's validity is still decided on its float32
 * channels).  Rounding to the nearest binary16 number, ties to even, from the
 * format's definition: 11 significant bits, smallest normal exponent -14 (so
 * below 2^-14 the spacing stays 2^-24), largest finite value 65504.
 */
double o_half(float x) {
    double v = (double)x;
    if (v == 0.0 || !isfinite(v)) return v;
    int e;
    (void)frexp(v, &e);        /* |v| = m 2^e, 0.5 <= m < 1 */
    int q = e - 11;            /* spacing of 11-bit significands in [2^(e-1), 2^e) */
    if (q < -24) q = -24;      /* subnormal binary16 numbers */
    double r = ldexp(nearbyint(ldexp(v, -q)), q);  /* exact scaling; nearbyint rounds ties to even */
    if (fabs(r) > 65504.0) return v > 0.0 ? INFINITY : -INFINITY;
    return r;
}

/* channel ci of texel I as the sampled image holds it */
static double tval(const o_params* prm, const float* I, int ci) {
    return (prm->texel_f16 && ci != 1) ? o_half(I[ci]) : (double)I[ci];
}

static double near_int_dist(double x) {
    return fabs(x - floor(x + 0.5));
}

/*
 * Bilinear sample of the five channels of image ch at (u, v) and of their
 * image Jacobians (R5, R6).  val[c], gu[c] = d/du, gv[c] = d/dv.
 * Returns 0 when the sample is not usable.  *flag is raised when u or v lies
 * within margin_px of an integer (the choice of taps, and with it the
 * usability test, may differ in another precision).
 */
static int sample(const o_sensor* s, const o_params* prm, const float* ch, double u, double v,
                  double val[5], double gu[5], double gv[5], double slope[5], int* flag) {
    if (!(v >= 1.0 && v < (double)(s->height - 2))) {
        if (near_int_dist(v) < prm->margin_px) *flag = 1;
        return 0;
    }
    if (s->model == O_PINHOLE && !(u >= 1.0 && u < (double)(s->width - 2))) {
        if (near_int_dist(u) < prm->margin_px) *flag = 1;
        return 0;
    }
    if (near_int_dist(u) < prm->margin_px || near_int_dist(v) < prm->margin_px) *flag = 1;
    int c0 = (int)floor(u), r0 = (int)floor(v);
    double a = u - c0, b = v - r0;
    /* the 12 stencil texels must be valid */
    static const int st[12][2] = {{-1, 0}, {-1, 1}, {0, -1}, {0, 0}, {0, 1}, {0, 2},
                                  {1, -1}, {1, 0}, {1, 1}, {1, 2}, {2, 0}, {2, 1}};
    for (int k = 0; k < 12; ++k)
        if (!pixel_valid(prm, texel(s, ch, r0 + st[k][0], c0 + st[k][1]))) return 0;
    /* taps t = (dr, dc) with bilinear weights */
    const int tr[4] = {0, 0, 1, 1}, tc[4] = {0, 1, 0, 1};
    const double w[4] = {(1 - a) * (1 - b), a * (1 - b), (1 - a) * b, a * b};
    for (int ci = 0; ci < 5; ++ci) { val[ci] = 0.0; gu[ci] = 0.0; gv[ci] = 0.0; }
    for (int t = 0; t < 4; ++t) {
        int r = r0 + tr[t], c = c0 + tc[t];
        const float* I = texel(s, ch, r, c);
        const float* Il = texel(s, ch, r, c - 1);
        const float* Ir = texel(s, ch, r, c + 1);
        const float* Iu = texel(s, ch, r - 1, c);
        const float* Id = texel(s, ch, r + 1, c);
        for (int ci = 0; ci < 5; ++ci) {
            val[ci] += w[t] * tval(prm, I, ci);
            if (prm->grad_mode == 0) {
                /* Supp.: dI/dc = (I_{r,c+1} - I_{r,c-1}) / 2, dI/dr = (I_{r+1,c} - I_{r-1,c}) / 2 */
                gu[ci] += w[t] * 0.5 * (tval(prm, Ir, ci) - tval(prm, Il, ci));
                gv[ci] += w[t] * 0.5 * (tval(prm, Id, ci) - tval(prm, Iu, ci));
            }
        }
    }
    for (int ci = 0; ci < 5; ++ci) {
        /* slopes of the bilinear interpolant in u and v: |d val / du| + |d val / dv| */
        double I00 = tval(prm, texel(s, ch, r0, c0), ci), I01 = tval(prm, texel(s, ch, r0, c0 + 1), ci);
        double I10 = tval(prm, texel(s, ch, r0 + 1, c0), ci), I11 = tval(prm, texel(s, ch, r0 + 1, c0 + 1), ci);
        double su = (1 - b) * (I01 - I00) + b * (I11 - I10);
        double sv = (1 - a) * (I10 - I00) + a * (I11 - I01);
        slope[ci] = fabs(su) + fabs(sv);
        if (prm->grad_mode == 1) {
            gu[ci] = su;
            gv[ci] = sv;
        }
    }
    return 1;
}

/* ----------------------------------------- Supp.: one residual, J_i, J_j */

/*
 * Residual of one pixel-point pt (7 values from o_frame_points of frame i)
 * against target image tgt of frame j, at poses X_i, X_j (3x4 row-major).
 * Outputs: e[5] = zeta(pbar) - I_j(pi(pbar)) ordered (g, d, n_x, n_y, n_z);
 * Ji, Jj (5x6 row-major, columns [Dt, Dq]); rho, w (R1); *flag (margins).
 * Returns 1 for a valid residual, 0 when rejected.
 */
int o_point_residual(const o_sensor* s, const o_params* prm, const float* tgt,
                     const double Xi[12], const double Xj[12], const double pt[7],
                     double e[5], double Ji[30], double Jj[30], double* rho, double* w,
                     int* flag) {
    *flag = 0;
    double Ri[9], Rj[9], RjT[9], Ro[9], RoT[9], ti[3], tj[3], to[3];
    rot_of(Xi, Ri); rot_of(Xj, Rj); rot_of(s->Xo, Ro);
    trans_of(Xi, ti); trans_of(Xj, tj); trans_of(s->Xo, to);
    mat3_T(Rj, RjT);
    mat3_T(Ro, RoT);
    const double pu[3] = {pt[0], pt[1], pt[2]};
    const double gu_src = pt[3];
    const double no[3] = {pt[4], pt[5], pt[6]};

    /* q = R_j^T (R_i p_u + t_i - t_j);  pbar = R_o^T (q - t_o)   (Supp., pbar_u) */
    double Rp[3], tmp[3], q[3], pb[3];
    mat3_vec(Ri, pu, Rp);
    for (int a = 0; a < 3; ++a) tmp[a] = Rp[a] + ti[a] - tj[a];
    mat3_vec(RjT, tmp, q);
    for (int a = 0; a < 3; ++a) tmp[a] = q[a] - to[a];
    mat3_vec(RoT, tmp, pb);

    /* depth cue zeta^d (Supp., Depth / Range) and the R8 test */
    double zd;
    if (s->model == O_PINHOLE) {
        zd = pb[2];
    } else {
        zd = sqrt(pb[0] * pb[0] + pb[1] * pb[1] + pb[2] * pb[2]);
    }
    int near_zmin = fabs(zd - prm->z_min) < prm->margin_rel * (1.0 + fabs(zd));
    if (near_zmin) *flag = 1;
    if (!(zd > prm->z_min) && !(prm->other_branch && near_zmin && zd > 0.0)) return 0;

    /* u' = pi(pbar)  (Eq. uprime) and the sample of I_j at u' */
    double uv[2];
    o_project(s, pb, uv);
    double Iv[5], Igu[5], Igv[5], Islope[5];
    int sflag = 0;
    int ok = sample(s, prm, tgt, uv[0], uv[1], Iv, Igu, Igv, Islope, &sflag);
    if (sflag) *flag = 1;
    if (!ok && prm->other_branch && sflag) {
        const double m2 = 2.0 * prm->margin_px;
        const double du[8] = {-m2, m2, 0.0, 0.0, -m2, -m2, m2, m2}, dv[8] = {0.0, 0.0, -m2, m2, -m2, m2, -m2, m2};
        for (int t = 0; t < 8 && !ok; ++t) {
            int f2 = 0;
            ok = sample(s, prm, tgt, uv[0] + du[t], uv[1] + dv[t], Iv, Igu, Igv, Islope, &f2);
        }
    }
    if (!ok) return 0;

    /* normal cue: nbar = R_o^T R_j^T R_i n_u^o  (Eq. normal-error-jacobian) */
    double Rn[3], RjTRn[3], nb[3];
    mat3_vec(Ri, no, Rn);
    mat3_vec(RjT, Rn, RjTRn);
    mat3_vec(RoT, RjTRn, nb);

    /* occlusion suppression (R7) */
    double thr = prm->occ_abs + prm->occ_rel * zd;
    double dd = fabs(zd - Iv[1]);
    int near_occ = fabs(dd - thr) < prm->margin_rel * (1.0 + fabs(zd)) + prm->margin_px * Islope[1];
    if (near_occ) *flag = 1;
    if (dd > thr && !(prm->other_branch && near_occ)) return 0;
    double nt = sqrt(Iv[2] * Iv[2] + Iv[3] * Iv[3] + Iv[4] * Iv[4]);
    int near_nt = fabs(nt - 0.5) < prm->margin_rel + prm->margin_px * (Islope[2] + Islope[3] + Islope[4]);
    if (near_nt) *flag = 1;
    if (nt < 0.5 && !(prm->other_branch && near_nt)) return 0;

    /* e = zeta(pbar) - I_j(u')  (Supp., Eq. error-jacobian) */
    e[0] = gu_src - Iv[0];
    e[1] = zd - Iv[1];
    e[2] = nb[0] - Iv[2];
    e[3] = nb[1] - Iv[3];
    e[4] = nb[2] - Iv[4];

    /* d pbar / d Dx_i = R_o^T R_j^T R_i [I | -2 [p_u]x]   (R3) */
    double M[9], RoTRjT[9], Spu[9], dPi[18], dPj[18];
    mat3_mul(RoT, RjT, RoTRjT);
    mat3_mul(RoTRjT, Ri, M);
    skew(pu, Spu);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            dPi[6 * r + c] = M[3 * r + c];
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += M[3 * r + k] * (-2.0 * Spu[3 * k + c]);
            dPi[6 * r + 3 + c] = acc;
        }
    /* d pbar / d Dx_j = R_o^T [-I | 2 [q]x]   (R3, R24) */
    double Sq[9];
    skew(q, Sq);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            dPj[6 * r + c] = -RoT[3 * r + c];
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += RoT[3 * r + k] * (2.0 * Sq[3 * k + c]);
            dPj[6 * r + 3 + c] = acc;
        }

    /* d pi / d pbar */
    double Jp[6];
    o_proj_jacobian(s, pb, Jp);

    /* d zeta^d / d pbar: e_z^T (depth) or pbar^T / |pbar| (range) */
    double dz[3];
    if (s->model == O_PINHOLE) {
        dz[0] = 0.0; dz[1] = 0.0; dz[2] = 1.0;
    } else {
        dz[0] = pb[0] / zd; dz[1] = pb[1] / zd; dz[2] = pb[2] / zd;
    }

    /* d nbar / d Dq_i = R_o^T R_j^T R_i (-2 [n_u^o]x);  d nbar / d Dq_j = R_o^T 2 [R_j^T R_i n_u^o]x  (R3, R4) */
    double Sno[9], Sm[9], dNi[9], dNj[9];
    skew(no, Sno);
    skew(RjTRn, Sm);
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) {
            double a1 = 0.0, a2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                a1 += M[3 * r + k] * (-2.0 * Sno[3 * k + c]);
                a2 += RoT[3 * r + k] * (2.0 * Sm[3 * k + c]);
            }
            dNi[3 * r + c] = a1;
            dNj[3 * r + c] = a2;
        }

    /* J = d zeta / d Dx - [dI/du dI/dv] (d pi / d pbar) (d pbar / d Dx)   (Supp., full Jacobians) */
    for (int ci = 0; ci < 5; ++ci) {
        double gI[3];
        for (int c = 0; c < 3; ++c) gI[c] = Igu[ci] * Jp[c] + Igv[ci] * Jp[3 + c];
        for (int col = 0; col < 6; ++col) {
            double img_i = 0.0, img_j = 0.0;
            for (int k = 0; k < 3; ++k) {
                img_i += gI[k] * dPi[6 * k + col];
                img_j += gI[k] * dPj[6 * k + col];
            }
            double map_i = 0.0, map_j = 0.0;
            if (ci == 1) {
                for (int k = 0; k < 3; ++k) {
                    map_i += dz[k] * dPi[6 * k + col];
                    map_j += dz[k] * dPj[6 * k + col];
                }
            } else if (ci >= 2 && col >= 3) {
                map_i = dNi[3 * (ci - 2) + (col - 3)];
                map_j = dNj[3 * (ci - 2) + (col - 3)];
            }
            Ji[6 * ci + col] = map_i - img_i;
            Jj[6 * ci + col] = map_j - img_j;
        }
    }

    /* Huber on chi = sqrt(e^T Omega e)   (R1, R2) */
    const double om[5] = {prm->w_int, prm->w_depth, prm->w_normal, prm->w_normal, prm->w_normal};
    double chi2 = 0.0;
    for (int ci = 0; ci < 5; ++ci) chi2 += om[ci] * e[ci] * e[ci];
    double chi = sqrt(chi2);
    if (chi <= prm->huber_delta) {
        *w = 1.0;
        *rho = chi2;
    } else {
        *w = prm->huber_delta / chi;
        *rho = 2.0 * prm->huber_delta * chi - prm->huber_delta * prm->huber_delta;
    }
    return 1;
}

/* ------------------------------------------------ one directed pair (i, j) */

/*
 * Linearise one directed pair: for every point of frame i (raster order),
 * H12 += w J^T Omega J with J = [J_i J_j] (5x12), b12 += w J^T Omega e,
 * cost += rho, count += 1 (each accumulated in double).  H12 is 12x12
 * row-major (rows/cols 0-5 frame i, 6-11 frame j); any of H12, b12 may be NULL
 * (cost only).  mask / flags (optional) receive one bit per point of frame i
 * (bit k % 32 of word k / 32): valid residual / decision near a threshold.
 * Returns the number of points of frame i, or -1 on allocation failure.
 */
int o_linearize_pair(const o_sensor* s, const o_params* prm, const float* src, const float* tgt,
                     const double Xi[12], const double Xj[12], double* H12, double* b12,
                     double* cost, int64_t* count, uint32_t* mask, uint32_t* flags) {
    int cap = s->width * s->height;
    double* pts = (double*)malloc(sizeof(double) * 7 * (size_t)(cap > 0 ? cap : 1));
    if (!pts) return -1;
    int np = o_frame_points(s, prm, src, pts, NULL, cap);
    const double om[5] = {prm->w_int, prm->w_depth, prm->w_normal, prm->w_normal, prm->w_normal};
    if (mask) memset(mask, 0, sizeof(uint32_t) * (size_t)((np + 31) / 32));
    if (flags) memset(flags, 0, sizeof(uint32_t) * (size_t)((np + 31) / 32));
    double c_acc = 0.0;
    int64_t n_acc = 0;
    for (int k = 0; k < np; ++k) {
        double e[5], Ji[30], Jj[30], rho, w;
        int flag;
        int ok = o_point_residual(s, prm, tgt, Xi, Xj, pts + 7 * (size_t)k, e, Ji, Jj, &rho, &w, &flag);
        if (flags && flag) flags[k >> 5] |= 1u << (k & 31);
        if (!ok) continue;
        if (mask) mask[k >> 5] |= 1u << (k & 31);
        c_acc += rho;
        n_acc += 1;
        if (!H12 && !b12) continue;
        double J[5][12];
        for (int r = 0; r < 5; ++r)
            for (int c = 0; c < 6; ++c) {
                J[r][c] = Ji[6 * r + c];
                J[r][6 + c] = Jj[6 * r + c];
            }
        for (int a = 0; a < 12; ++a) {
            if (b12) {
                double s_b = 0.0;
                for (int r = 0; r < 5; ++r) s_b += J[r][a] * om[r] * e[r];
                b12[a] += w * s_b;
            }
            if (H12)
                for (int c = 0; c < 12; ++c) {
                    double s_h = 0.0;
                    for (int r = 0; r < 5; ++r) s_h += J[r][a] * om[r] * J[r][c];
                    H12[12 * a + c] += w * s_h;
                }
        }
    }
    *cost += c_acc;
    *count += n_acc;
    free(pts);
    return np;
}

/* ------------------------------------------------------- whole problem */

/*
 * Linearise every directed pair and assemble the dense system (gauge not
 * fixed): H (6N x 6N row-major) and b (6N), frame k owning rows 6k..6k+5,
 * plus the total cost F (Eq. total-error-multicue) and the number of valid residuals.
 * channels[k] is frame k's H x W x 5 float image; poses is N x 12.
 * H and b may be NULL (cost only).  Pair k's 12x12 block and 12-vector are
 * also returned in pair_H (M x 144) / pair_b (M x 12) when those are non-NULL,
 * and its cost / count in pair_cost / pair_count.  Returns 0, or -1 on a
 * malformed pair (frames out of range or of different sensors).
 */
/* ----------------------------------------- the sensor offset as a variable */

/*
 * Reading R23 (the paper holds X_o fixed and prints no derivative for it):
 * pbar = X_o^-1 X_j^-1 X_i X_o pi^-1(u, d), and n-bar likewise with the
 * rotations.  Right-perturbing X_o by E = exp(d) gives E^-1 (X_o^-1 X_j^-1
 * X_i X_o) E; right-perturbing X_i by X_o E X_o^-1 produces the right factor
 * and right-perturbing X_j by the same transform the left one.  So, to first
 * order, J_o = (J_i + J_j) A_o with A_o the map d -> [R_o dt + 2 [t_o]x R_o dq,
 * R_o dq] (X_o E X_o^-1 in the [dt, dq] coordinates of Supp., R(dq) ~ I + 2
 * [dq]x).  A is row-major 6 x 6.
 */
void o_offset_map(const double Xo[12], double A[36]) {
    double Ro[9], to[3];
    rot_of(Xo, Ro);
    trans_of(Xo, to);
    memset(A, 0, sizeof(double) * 36);
    /* [t_o]x R_o, column c: t_o x (column c of R_o) */
    for (int c = 0; c < 3; ++c) {
        const double col[3] = {Ro[c], Ro[3 + c], Ro[6 + c]};
        const double x[3] = {to[1] * col[2] - to[2] * col[1], to[2] * col[0] - to[0] * col[2],
                             to[0] * col[1] - to[1] * col[0]};
        for (int r = 0; r < 3; ++r) {
            A[6 * r + c] = Ro[3 * r + c];
            A[6 * r + 3 + c] = 2.0 * x[r];
            A[6 * (3 + r) + 3 + c] = Ro[3 * r + c];
        }
    }
}

/* Jo (5x6) = (Ji + Jj) A_o  (R23). */
void o_offset_jacobian(const double Xo[12], const double Ji[30], const double Jj[30], double Jo[30]) {
    double A[36];
    o_offset_map(Xo, A);
    for (int r = 0; r < 5; ++r)
        for (int c = 0; c < 6; ++c) {
            double s = 0.0;
            for (int k = 0; k < 6; ++k) s += (Ji[6 * r + k] + Jj[6 * r + k]) * A[6 * k + c];
            Jo[6 * r + c] = s;
        }
}

/* Offset blocks of one pair, point by point: out = [H_io (6x6), H_jo (6x6),
 * H_oo (6x6), b_o (6)] = sums of w J_i^T Omega J_o, w J_j^T Omega J_o,
 * w J_o^T Omega J_o, w J_o^T Omega e over the valid residuals. */
int o_pair_offset_blocks(const o_sensor* s, const o_params* prm, const float* src, const float* tgt,
                         const double Xi[12], const double Xj[12], double out[114]) {
    int cap = s->width * s->height;
    double* pts = (double*)malloc(sizeof(double) * 7 * (size_t)(cap > 0 ? cap : 1));
    if (!pts) return -1;
    int np = o_frame_points(s, prm, src, pts, NULL, cap);
    const double om[5] = {prm->w_int, prm->w_depth, prm->w_normal, prm->w_normal, prm->w_normal};
    memset(out, 0, sizeof(double) * 114);
    for (int k = 0; k < np; ++k) {
        double e[5], Ji[30], Jj[30], Jo[30], rho, w;
        int flag;
        if (!o_point_residual(s, prm, tgt, Xi, Xj, pts + 7 * (size_t)k, e, Ji, Jj, &rho, &w, &flag)) continue;
        o_offset_jacobian(s->Xo, Ji, Jj, Jo);
        for (int a = 0; a < 6; ++a) {
            for (int c = 0; c < 6; ++c) {
                double hi = 0.0, hj = 0.0, ho = 0.0;
                for (int r = 0; r < 5; ++r) {
                    hi += Ji[6 * r + a] * om[r] * Jo[6 * r + c];
                    hj += Jj[6 * r + a] * om[r] * Jo[6 * r + c];
                    ho += Jo[6 * r + a] * om[r] * Jo[6 * r + c];
                }
                out[6 * a + c] += w * hi;
                out[36 + 6 * a + c] += w * hj;
                out[72 + 6 * a + c] += w * ho;
            }
            double bo = 0.0;
            for (int r = 0; r < 5; ++r) bo += Jo[6 * r + a] * om[r] * e[r];
            out[108 + a] += w * bo;
        }
    }
    free(pts);
    return np;
}

int o_linearize(int n_frames, const o_sensor* sensors, const int32_t* frame_sensor,
                const float* const* channels, const double* poses, int m, const int32_t* pairs,
                const o_params* prm, double* H, double* b, double* cost, int64_t* count,
                double* pair_H, double* pair_b, double* pair_cost, int64_t* pair_count) {
    int n6 = 6 * n_frames;
    if (H) memset(H, 0, sizeof(double) * (size_t)n6 * n6);
    if (b) memset(b, 0, sizeof(double) * (size_t)n6);
    *cost = 0.0;
    *count = 0;
    for (int k = 0; k < m; ++k) {
        int i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= n_frames || j >= n_frames) return -1;
        if (frame_sensor[i] != frame_sensor[j]) return -1;
        const o_sensor* s = &sensors[frame_sensor[i]];
        double H12[144], b12[12], pc = 0.0;
        int64_t pn = 0;
        memset(H12, 0, sizeof H12);
        memset(b12, 0, sizeof b12);
        if (o_linearize_pair(s, prm, channels[i], channels[j], poses + 12 * (size_t)i,
                             poses + 12 * (size_t)j, H ? H12 : NULL, b ? b12 : NULL, &pc, &pn,
                             NULL, NULL) < 0)
            return -2;
        *cost += pc;
        *count += pn;
        if (pair_H) memcpy(pair_H + 144 * (size_t)k, H12, sizeof H12);
        if (pair_b) memcpy(pair_b + 12 * (size_t)k, b12, sizeof b12);
        if (pair_cost) pair_cost[k] = pc;
        if (pair_count) pair_count[k] = pn;
        const int base[2] = {6 * i, 6 * j};
        for (int ba = 0; ba < 2; ++ba) {
            if (b)
                for (int a = 0; a < 6; ++a) b[base[ba] + a] += b12[6 * ba + a];
            if (H)
                for (int bb = 0; bb < 2; ++bb)
                    for (int a = 0; a < 6; ++a)
                        for (int c = 0; c < 6; ++c)
                            H[(size_t)(base[ba] + a) * n6 + base[bb] + c] += H12[12 * (6 * ba + a) + 6 * bb + c];
        }
    }
    return 0;
}

/* --------------------------------------------------------------- solver */

/*
 * Solve A x = rhs for symmetric positive definite A (n x n row-major) by a
 * plain Cholesky factorisation A = L L^T and two triangular solves.
 * Returns 0, or -1 when a pivot is not positive (A not positive definite).
 */
int o_cholesky_solve(int n, const double* A, const double* rhs, double* x) {
    double* L = (double*)calloc((size_t)n * n + 1, sizeof(double));
    double* y = (double*)calloc((size_t)n + 1, sizeof(double));
    if (!L || !y) { free(L); free(y); return -2; }
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(s > 0.0)) { free(L); free(y); return -1; }
        double d = sqrt(s);
        L[(size_t)j * n + j] = d;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= L[(size_t)i * n + k] * L[(size_t)j * n + k];
            L[(size_t)i * n + j] = t / d;
        }
    }
    for (int i = 0; i < n; ++i) {
        double t = rhs[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * y[k];
        y[i] = t / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        double t = y[i];
        for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * x[k];
        x[i] = t / L[(size_t)i * n + i];
    }
    free(L);
    free(y);
    return 0;
}

/*
 * Damped, gauge-fixed step (Sec. IV-C, LM): (H_ff + lambda I) dx_f = -b_f
 * where _f drops frame 0's six rows and columns; dx (6N) gets dx_0 = 0.
 * Returns 0, or -1 when the damped system is not positive definite.
 */
int o_solve_step(int n_frames, const double* H, const double* b, double lambda, double* dx) {
    int n6 = 6 * n_frames, n = n6 - 6;
    memset(dx, 0, sizeof(double) * (size_t)n6);
    if (n <= 0) return 0;
    double* A = (double*)malloc(sizeof(double) * (size_t)n * n);
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    if (!A || !r) { free(A); free(r); return -2; }
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) A[(size_t)i * n + j] = H[(size_t)(i + 6) * n6 + (j + 6)];
        A[(size_t)i * n + i] += lambda;
        r[i] = -b[i + 6];
    }
    int st = o_cholesky_solve(n, A, r, dx + 6);
    free(A);
    free(r);
    if (st != 0) memset(dx, 0, sizeof(double) * (size_t)n6);
    return st;
}

/* X_k <- X_k [+] dx_k for every frame (Supp., box-plus). */
void o_apply_update(int n_frames, const double* poses, const double* dx, double* out) {
    for (int k = 0; k < n_frames; ++k) o_boxplus(poses + 12 * (size_t)k, dx + 6 * (size_t)k, out + 12 * (size_t)k);
}
