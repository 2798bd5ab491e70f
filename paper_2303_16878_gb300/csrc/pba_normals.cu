// pba_normals.cu -- normal estimation (Sec. IV-A).
//
// For every pixel u with valid depth: the valid pixels u' with |u - u'| < r(u),
// r(u) = clamp(scale / d(u), 1.5, max_radius) pixels (a radius inversely
// proportional to the range; columns wrap for the spherical model), are
// unprojected (Sec. III), the least-squares plane through them is fitted
// (normal = eigenvector of the smallest eigenvalue of their covariance) and
// the normal is oriented towards the observer (n . p_u < 0).  Pixels with
// fewer than kMinCount points, or whose points are collinear (middle
// eigenvalue <= 1e-6 x largest), get a zero normal.  One thread per pixel;
// moments are taken about the centre pixel's point, in FP32; the symmetric
// 3 x 3 eigenproblem is solved by cyclic Jacobi rotations.
#include <algorithm>

#include "pba_internal.cuh"

namespace pba {
namespace {

constexpr int kMinCount = 5;
constexpr float kCollinear = 1e-6f;

// rmin / rmax are the float images of the double range limits, rounded inwards on the
// host, so that these float comparisons decide exactly like the double ones of pack.
__device__ __forceinline__ bool depth_valid(float d, float rmin, float rmax) {
    return d > 0.f && d >= rmin && d <= rmax;
}

__device__ __forceinline__ void unproject(const FrameInfo& fr, int row, int col, float d, float p[3]) {
    if (fr.model == 0) {
        p[0] = d * ((col - fr.cx) / fr.fx);
        p[1] = d * ((row - fr.cy) / fr.fy);
        p[2] = d;
    } else {
        float saz, caz, sel, cel;
        sincosf((col - fr.cx) / fr.fx, &saz, &caz);
        sincosf((row - fr.cy) / fr.fy, &sel, &cel);
        p[0] = d * (cel * caz);
        p[1] = d * (cel * saz);
        p[2] = d * sel;
    }
}

// One Jacobi rotation in the (p, q) plane of the symmetric matrix (app, aqq, apq;
// arp, arq the entries of the third row r), chosen to zero apq: t = tan(angle)
// is the smaller root of t^2 + 2 theta t - 1 = 0, theta = (aqq - app) / (2 apq).
// The eigenvector columns vp, vq (3 entries each) rotate with it.
__device__ __forceinline__ void jacobi_rotate(float& app, float& aqq, float& apq, float& arp, float& arq, float vp[3],
                                              float vq[3]) {
    if (apq == 0.f) return;
    const float theta = (aqq - app) / (2.f * apq);
    float t = fabsf(theta) > 1e18f ? 0.5f / theta : copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
    const float c = rsqrtf(t * t + 1.f), s = t * c;
    app -= t * apq;
    aqq += t * apq;
    apq = 0.f;
    const float rp = arp, rq = arq;
    arp = c * rp - s * rq;
    arq = s * rp + c * rq;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float xp = vp[k], xq = vq[k];
        vp[k] = c * xp - s * xq;
        vq[k] = s * xp + c * xq;
    }
}

// Eigen-decomposition of a symmetric 3 x 3 matrix by cyclic Jacobi sweeps
// (backward stable: eigenvector errors of order u |A| / gap).  Returns the
// eigenvalues ascending in ev and the eigenvector of the smallest in n.
__device__ void eig3_smallest(float a00, float a01, float a02, float a11, float a12, float a22, float n[3],
                              float ev[3]) {
    float v0[3] = {1.f, 0.f, 0.f}, v1[3] = {0.f, 1.f, 0.f}, v2[3] = {0.f, 0.f, 1.f};
#pragma unroll 1
    for (int sweep = 0; sweep < 6; ++sweep) {
        jacobi_rotate(a00, a11, a01, a02, a12, v0, v1);  // plane (0, 1), third row 2
        jacobi_rotate(a00, a22, a02, a01, a12, v0, v2);  // plane (0, 2), third row 1
        jacobi_rotate(a11, a22, a12, a01, a02, v1, v2);  // plane (1, 2), third row 0
    }
    // sort the diagonal
    float l[3] = {a00, a11, a22};
    int lo = 0;
    if (l[1] < l[lo]) lo = 1;
    if (l[2] < l[lo]) lo = 2;
    const float lmax = fmaxf(l[0], fmaxf(l[1], l[2]));
    ev[0] = l[lo];
    ev[2] = lmax;
    ev[1] = (l[0] + l[1] + l[2]) - ev[0] - ev[2];
    const float* v = lo == 0 ? v0 : (lo == 1 ? v1 : v2);
    n[0] = v[0];
    n[1] = v[1];
    n[2] = v[2];
}

// In place: every thread reads only depth channels and writes only the normal
// channels of its own pixel, so no thread reads what another one writes.
__global__ void k_normals(float* raw, const FrameInfo* __restrict__ frames, const int* __restrict__ frame_ids,
                          float scale, int max_radius, float rmin, float rmax) {
    const FrameInfo fr = frames[frame_ids[blockIdx.y]];
    const int npx = fr.width * fr.height;
    const int px = blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= npx) return;
    const int row = px / fr.width, col = px % fr.width;
    float* img = raw + fr.px_offset * 5;
    const float d = img[(long long)px * 5 + 1];
    float nrm[3] = {0.f, 0.f, 0.f};
    if (depth_valid(d, rmin, rmax)) {
        float pc[3];
        unproject(fr, row, col, d, pc);
        const float rad = fminf(fmaxf(scale / d, 1.5f), (float)max_radius);
        const float r2 = rad * rad;
        float s1[3] = {0.f, 0.f, 0.f}, s2[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        int cnt = 0;
        for (int dr = -max_radius; dr <= max_radius; ++dr) {
            const int rr = row + dr;
            if (rr < 0 || rr >= fr.height) continue;
            for (int dc = -max_radius; dc <= max_radius; ++dc) {
                if ((float)(dr * dr + dc * dc) >= r2) continue;
                int cc = col + dc;
                if (cc < 0 || cc >= fr.width) {
                    if (fr.model != 1) continue;
                    cc = cc < 0 ? cc + fr.width : cc - fr.width;
                }
                const float dn = img[((long long)rr * fr.width + cc) * 5 + 1];
                if (!depth_valid(dn, rmin, rmax)) continue;
                float q[3];
                unproject(fr, rr, cc, dn, q);
                q[0] -= pc[0];
                q[1] -= pc[1];
                q[2] -= pc[2];
                s1[0] += q[0];
                s1[1] += q[1];
                s1[2] += q[2];
                s2[0] = fmaf(q[0], q[0], s2[0]);
                s2[1] = fmaf(q[0], q[1], s2[1]);
                s2[2] = fmaf(q[0], q[2], s2[2]);
                s2[3] = fmaf(q[1], q[1], s2[3]);
                s2[4] = fmaf(q[1], q[2], s2[4]);
                s2[5] = fmaf(q[2], q[2], s2[5]);
                ++cnt;
            }
        }
        if (cnt >= kMinCount) {
            const float ic = 1.f / cnt;
            const float m0 = s1[0] * ic, m1 = s1[1] * ic, m2 = s1[2] * ic;
            float ev[3], n[3];
            eig3_smallest(s2[0] * ic - m0 * m0, s2[1] * ic - m0 * m1, s2[2] * ic - m0 * m2, s2[3] * ic - m1 * m1,
                          s2[4] * ic - m1 * m2, s2[5] * ic - m2 * m2, n, ev);
            if (ev[1] > kCollinear * ev[2]) {
                const float sgn = (n[0] * pc[0] + n[1] * pc[1] + n[2] * pc[2]) > 0.f ? -1.f : 1.f;
                nrm[0] = sgn * n[0];
                nrm[1] = sgn * n[1];
                nrm[2] = sgn * n[2];
            }
        }
    }
    float* o = img + (long long)px * 5 + 2;
    o[0] = nrm[0];
    o[1] = nrm[1];
    o[2] = nrm[2];
}

}  // namespace

cudaError_t launch_normals(float* raw, const FrameInfo* frames, const int* frame_ids, int n, int max_px, float scale,
                           int max_radius, double range_min, double range_max, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    // smallest float >= range_min, largest float <= range_max
    float rmin = (float)range_min, rmax = range_max > 3.0e38 ? 3.0e38f : (float)range_max;
    if ((double)rmin < range_min) rmin = nextafterf(rmin, 3.0e38f);
    if ((double)rmax > range_max) rmax = nextafterf(rmax, -3.0e38f);
    for (int f0 = 0; f0 < n; f0 += 65535) {  // grid.y limit
        const dim3 grid((max_px + 255) / 256, std::min(65535, n - f0));
        k_normals<<<grid, 256, 0, s>>>(raw, frames, frame_ids + f0, scale, max_radius, rmin, rmax);
    }
    return cudaGetLastError();
}

}  // namespace pba
