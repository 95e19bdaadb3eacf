// The reduced camera system of cameras with interior parameters, formed on
// the device into a variable-size BSMC system (ba_vbsmc_create_interiors).
//
// Sec. 4 gives block (i, j) of the RCS c_i x c_j entries; Sec. 4.1 counts six
// exterior and five interior unknowns per camera.  The interiors are
// [f, cx, cy, k1, k2]: with xh = x/z, yh = y/z, r2 = xh^2 + yh^2 and
// d = 1 + k1 r2 + k2 r2^2 the projection is u = f d xh + cx, v = f d yh + cy.
// A camera has c_i = 6 (interiors fixed) or 11 unknowns.  Three kernels:
//   k_vbi_linearize  e and J of every observation (Eq. 1), rows of
//                    [J_c (2 x 11) | J_p (2 x 3) | e (2)] in the storage
//                    precision (X_cam in FP64, the rest in that precision);
//   k_vbi_points     per point, in FP64, V_k (damped), its Cholesky factor
//                    L, V_k^-1 and l_p (Eq. 3), and per observation the
//                    factor row P = J_p L^-T and e^ = e + P L^-1 l_p;
//   k_vbi_blocks     a warp per stored block (i, j): the sum over its point
//                    pairs of -J_c,a^T (P_a P_b^T) J_c,b = -W_a V_k^-1 W_b^T
//                    (Eq. 4), plus U_i (damped) and b_i = -sum J_c^T e^ on
//                    the diagonal, in the storage precision.  The pairs of a
//                    block are listed on the host (track order), so the sums
//                    need no atomics and are deterministic.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "vbsmc_internal.h"

namespace ba {

constexpr int VJW = 32;      // J row (T): J_c 2 x 11 at 0, 11 | J_p 2 x 3 at 22, 25 | e at 28, 29 | pad
constexpr int VPW = 8;       // factor row (T): P = J_p L^-T (2 x 3) at 0, 3 | e^ = e + P L^-1 l_p at 6, 7
constexpr int VB_CI = 11;    // unknowns of a self-calibrating camera
constexpr int VB_NT = 4;     // block entries per lane: 4 x 32 >= 11 x 11

// Per camera [R (9), t (3)] in FP64, R = Exp(omega).
__global__ void k_vbi_camcache(int n, const double *__restrict__ cams, double *__restrict__ camc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double q[4], R[9];
    quat_exp(cams + 6 * i, q);
    quat_to_R(q, R);
    for (int k = 0; k < 9; ++k) camc[12 * i + k] = R[k];
    for (int k = 0; k < 3; ++k) camc[12 * i + 9 + k] = cams[6 * i + 3 + k];
}

// X_cam = R X + t in FP64 (no cancellation of the large world coordinates),
// then the projection with interiors in T: xh = x/z, yh = y/z,
// r2 = xh^2 + yh^2, d = 1 + k1 r2 + k2 r2^2, e = (f d xh + cx, f d yh + cy) - u.
template <typename T>
struct VbiProj {
    T Xc[3], xh, yh, r2, d, e0, e1;
};
template <typename T>
__device__ __forceinline__ VbiProj<T> vbi_project(const double *__restrict__ camc, const double *__restrict__ intr,
                                                  const double *__restrict__ pts, int i, int64_t k,
                                                  const double *__restrict__ uv) {
    const double *R = camc + 12 * i, *X = pts + 3 * k, *kk = intr + 5 * i;
    VbiProj<T> o;
    for (int r = 0; r < 3; ++r) o.Xc[r] = (T)(R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + R[9 + r]);
    o.xh = o.Xc[0] / o.Xc[2];
    o.yh = o.Xc[1] / o.Xc[2];
    o.r2 = o.xh * o.xh + o.yh * o.yh;
    o.d = T(1) + (T)kk[3] * o.r2 + (T)kk[4] * o.r2 * o.r2;
    o.e0 = (T)kk[0] * o.d * o.xh + (T)(kk[1] - uv[0]);
    o.e1 = (T)kk[0] * o.d * o.yh + (T)(kk[2] - uv[1]);
    return o;
}

template <typename T>
__global__ void __launch_bounds__(256) k_vbi_linearize(int64_t m, const int *__restrict__ ocam,
                                                       const int *__restrict__ opt, const double *__restrict__ uv,
                                                       const double *__restrict__ camc,
                                                       const double *__restrict__ intr,
                                                       const double *__restrict__ pts, T *__restrict__ J) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const int i = ocam[a], k = opt[a];
        const VbiProj<T> pr = vbi_project<T>(camc, intr, pts, i, k, uv + 2 * a);
        const double *R = camc + 12 * i, *kk = intr + 5 * i;
        const T f = (T)kk[0], k1 = (T)kk[3], k2 = (T)kk[4];
        const T z = pr.Xc[2], xh = pr.xh, yh = pr.yh, r2 = pr.r2, d = pr.d;
        const T g = T(2) * (k1 + T(2) * k2 * r2);
        // image-plane Jacobian D of (f d xh, f d yh) w.r.t. (xh, yh), then A = D d(xh, yh)/dX_cam
        const T D00 = f * (d + g * xh * xh), D01 = f * g * xh * yh, D11 = f * (d + g * yh * yh);
        T A[2][3];
        A[0][0] = D00 / z;
        A[0][1] = D01 / z;
        A[0][2] = -(D00 * xh + D01 * yh) / z;
        A[1][0] = D01 / z;
        A[1][1] = D11 / z;
        A[1][2] = -(D01 * xh + D11 * yh) / z;
        // dX_cam/d(d_omega) = -[X_cam]x (camera-frame update), dX_cam/d(dt) = I, dX_cam/dX = R
        const T *Xc = pr.Xc;
        const T Mx[3][3] = {{T(0), Xc[2], -Xc[1]}, {-Xc[2], T(0), Xc[0]}, {Xc[1], -Xc[0], T(0)}};
        T *o = J + a * VJW;
        const T ph[2] = {xh, yh};
        for (int r = 0; r < 2; ++r) {
            T *jc = o + VB_CI * r, *jp = o + 22 + 3 * r;
            for (int c = 0; c < 3; ++c) {
                jc[c] = A[r][0] * Mx[0][c] + A[r][1] * Mx[1][c] + A[r][2] * Mx[2][c];
                jc[3 + c] = A[r][c];
                jp[c] = A[r][0] * (T)R[c] + A[r][1] * (T)R[3 + c] + A[r][2] * (T)R[6 + c];
            }
            jc[6] = d * ph[r];                 // f
            jc[7] = r == 0 ? T(1) : T(0);      // cx
            jc[8] = r == 0 ? T(0) : T(1);      // cy
            jc[9] = f * ph[r] * r2;            // k1
            jc[10] = f * ph[r] * r2 * r2;      // k2
        }
        o[28] = pr.e0;
        o[29] = pr.e1;
        o[30] = T(0);
        o[31] = T(0);
    }
}

// Per point, in FP64: V_k = sum J_p^T J_p + lambda clamp(diag), its
// Cholesky factor V_k = L L^T (the three pivots must be positive), V_k^-1
// and l_p = -sum J_p^T e for Eq. 5; then per observation of the point the
// factor row P_a = J_p,a L^-T and e^_a = e_a + P_a (L^-1 l_p), in T, so that
// -W_a V^-1 W_b^T = -J_c,a^T (P_a P_b^T) J_c,b and
// -J_c,a^T e_a - W_a V^-1 l_p = -J_c,a^T e^_a (the block kernel's products).
template <typename T>
__global__ void __launch_bounds__(256) k_vbi_points(int64_t P, const int *__restrict__ trk_ptr,
                                                    const T *__restrict__ J, double lambda, double *__restrict__ Vinv,
                                                    double *__restrict__ lp, T *__restrict__ PE, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        double V[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, l[3] = {0, 0, 0};
        for (int a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a) {
            const T *o = J + (int64_t)a * VJW;
            double jp[6];
            for (int q = 0; q < 6; ++q) jp[q] = (double)o[22 + q];
            const double e0 = (double)o[28], e1 = (double)o[29];
            for (int m = 0; m < 3; ++m) {
                for (int n = 0; n < 3; ++n) V[m][n] += jp[m] * jp[n] + jp[3 + m] * jp[3 + n];
                l[m] -= jp[m] * e0 + jp[3 + m] * e1;
            }
        }
        for (int m = 0; m < 3; ++m) V[m][m] += lambda * clampT(V[m][m]);
        // V = L L^T, M = L^-1 (lower)
        const double d0 = sqrt(V[0][0]), c10 = V[0][1] / d0, c20 = V[0][2] / d0;
        const double s11 = V[1][1] - c10 * c10, d1 = sqrt(s11), c21 = (V[1][2] - c20 * c10) / d1;
        const double s22 = V[2][2] - c20 * c20 - c21 * c21, d2 = sqrt(s22);
        const bool ok = V[0][0] > 0.0 && s11 > 0.0 && s22 > 0.0;
        double m00 = 1.0 / d0, m11 = 1.0 / d1, m22 = 1.0 / d2;
        double m10 = -c10 * m00 * m11, m21 = -c21 * m11 * m22, m20 = -(c20 * m00 + c21 * m10) * m22;
        if (!ok) {
            atomicExch(err, (int)BA_ERR_NOT_SPD);
            m00 = m11 = m22 = m10 = m21 = m20 = 0.0;
        }
        // V^-1 = M^T M
        const double Mm[3][3] = {{m00, 0.0, 0.0}, {m10, m11, 0.0}, {m20, m21, m22}};
        double *vi = Vinv + 9 * k;
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) vi[3 * r + c] = Mm[0][r] * Mm[0][c] + Mm[1][r] * Mm[1][c] + Mm[2][r] * Mm[2][c];
        for (int m = 0; m < 3; ++m) lp[3 * k + m] = l[m];
        const double q0 = m00 * l[0], q1 = m10 * l[0] + m11 * l[1], q2 = m20 * l[0] + m21 * l[1] + m22 * l[2];
        for (int a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a) {
            const T *o = J + (int64_t)a * VJW;
            T *pe = PE + (int64_t)a * VPW;
            for (int r = 0; r < 2; ++r) {
                const double j0 = (double)o[22 + 3 * r], j1 = (double)o[23 + 3 * r], j2 = (double)o[24 + 3 * r];
                // P = J_p L^-T: P_c = sum_k J_k (L^-1)_ck over k <= c
                const double P0 = j0 * m00, P1 = j0 * m10 + j1 * m11, P2 = j0 * m20 + j1 * m21 + j2 * m22;
                pe[3 * r] = (T)P0;
                pe[3 * r + 1] = (T)P1;
                pe[3 * r + 2] = (T)P2;
                pe[6 + r] = (T)((double)o[28 + r] + P0 * q0 + P1 * q1 + P2 * q2);
            }
        }
    }
}

// A warp per stored block (beta, gamma) and its list of slot pairs (a, b).
// A slot is an observation's J_c columns that belong to one block: for a
// block of camera i (c_i = 6 or 11) the first c_i columns, for the block of a
// physical camera whose images share interiors the five interior columns;
// jc0[beta] is the first J_c column of block beta's slots (null: 0).  The
// pairs of a block are its slots' pairs within each point (every ordered
// pair, a in beta and b in gamma).  Per pair the 2 x 2 middle factor is
// -P_a P_b^T, or I - P_a P_a^T when both slots belong to one observation
// (that adds U = J_c^T J_c, the coupling of an image and its physical camera
// included); lanes 16.. form its product with the c_gamma columns of J_c,b,
// lanes 0.. stage J_c,a's c_beta columns, and every lane adds
// J_c,a^T (M J_c,b) for its entries.  Summed over a point's slot pairs this is
// U - W_beta V_k^-1 W_gamma^T with W_beta summed over the point's slots in
// beta.  On a diagonal block a slot paired with itself also gives b_beta's
// term -J_c,a^T e^_a and the U diagonal that damps the block at the end.
template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 5 : 4) k_vbi_blocks(int64_t nnzb, const int *__restrict__ brow,
                                                    const int *__restrict__ col, const int *__restrict__ cdim,
                                                    const int *__restrict__ jc0, const int *__restrict__ off,
                                                    const int64_t *__restrict__ boff,
                                                    const int *__restrict__ pptr, const int2 *__restrict__ plist,
                                                    const T *__restrict__ J, const T *__restrict__ PE,
                                                    double lambda, T *__restrict__ val, T *__restrict__ b) {
    __shared__ T sm[8][4 * 16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T *Jca = sm[w], *Tb = Jca + 32;  // J_c,a columns (2 x 16), M J_c,b (2 x 16)
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < nnzb; k += nw) {
        const int i = brow[k], j = col[k], ci = cdim[i], cj = cdim[j], nel = ci * cj;
        const int ai = jc0 ? jc0[i] : 0, aj = jc0 ? jc0[j] : 0;
        const bool diag = i == j;
        T acc[VB_NT], dU[VB_NT], bacc = T(0);
        // this lane's entries (row, column) of the block, fixed for its pairs
        int er[VB_NT], ec[VB_NT];
#pragma unroll
        for (int t = 0; t < VB_NT; ++t) {
            acc[t] = dU[t] = T(0);
            const int E = lane + 32 * t;
            er[t] = E < nel ? E / cj : 0;
            ec[t] = E < nel ? E - er[t] * cj : 0;
        }
        for (int p = pptr[k]; p < pptr[k + 1]; ++p) {  // warp-uniform
            const int2 pr = plist[p];
            const bool same = pr.x == pr.y;
            const T *Ja = J + (int64_t)pr.x * VJW, *Jb = J + (int64_t)pr.y * VJW;
            const T *Pa = PE + (int64_t)pr.x * VPW, *Pb = PE + (int64_t)pr.y * VPW;
            if (lane < 16) {
                const int r = lane;
                if (r < ci) {
                    const T j0 = Ja[ai + r], j1 = Ja[VB_CI + ai + r];
                    Jca[r] = j0;
                    Jca[16 + r] = j1;
                    if (diag && same) bacc -= j0 * Pa[6] + j1 * Pa[7];
                }
            } else {
                const int c = lane - 16;
                if (c < cj) {
                    // M = (same ? I : 0) - P_a P_b^T
                    T M[2][2];
                    for (int u = 0; u < 2; ++u)
                        for (int v = 0; v < 2; ++v)
                            M[u][v] = (same && u == v ? T(1) : T(0)) -
                                      (Pa[3 * u] * Pb[3 * v] + Pa[3 * u + 1] * Pb[3 * v + 1] + Pa[3 * u + 2] * Pb[3 * v + 2]);
                    const T j0 = Jb[aj + c], j1 = Jb[VB_CI + aj + c];
                    Tb[c] = M[0][0] * j0 + M[0][1] * j1;
                    Tb[16 + c] = M[1][0] * j0 + M[1][1] * j1;
                }
            }
            __syncwarp();
#pragma unroll
            for (int t = 0; t < VB_NT; ++t) {
                if (lane + 32 * t < nel) {
                    const int r = er[t], c = ec[t];
                    acc[t] += Jca[r] * Tb[c] + Jca[16 + r] * Tb[16 + c];
                    if (diag && same && r == c) dU[t] += Jca[r] * Jca[r] + Jca[16 + r] * Jca[16 + r];
                }
            }
            __syncwarp();
        }
        for (int t = 0; t < VB_NT; ++t) {
            const int E = lane + 32 * t;
            if (E < nel) {
                const int r = E / cj, c = E - r * cj;
                T v = acc[t];
                if (diag && r == c) v += (T)lambda * clampT(dU[t]);
                val[boff[k] + E] = v;
            }
        }
        if (diag && lane < ci) b[off[i] + lane] = (T)bacc;
    }
}

// ---------------------------------------------------------------------------
// LM iteration with interiors: cost, Eq. 5, the trial state and its cost, and
// the model decrease of the gain ratio (all FP64)
// ---------------------------------------------------------------------------

struct VbiScalars {
    double cost, cost_trial, model;
    unsigned long long n_cheir_trial;
};

// F = 1/2 sum ||e||^2 from the stored rows (after k_vbi_linearize), FP64 sum
template <typename T>
__global__ void __launch_bounds__(256) k_vbi_cost(int64_t m, const T *__restrict__ J, VbiScalars *sc, double *red,
                                                  unsigned *ctr) {
    double v[1] = {0.0};
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const double e0 = (double)J[a * VJW + 28], e1 = (double)J[a * VJW + 29];
        v[0] += e0 * e0 + e1 * e1;
    }
    grid_sum<1>(v, red, ctr, [&](double *t) { sc->cost = 0.5 * t[0]; });
}

// Eq. 5 per point: dx_p = V^-1 (l_p - sum_a W_a^T dx_c,cam(a)) with
// W_a^T dx = J_p,a^T (J_c,a dx) over the camera's c_i columns; the trial
// point X + dx_p.  dxc is the solve's vector (c_i entries per camera at off[i]).
template <typename T>
__global__ void __launch_bounds__(256) k_vbi_backsub(int64_t P, const int *__restrict__ trk_ptr,
                                                     const int *__restrict__ ocam, const T *__restrict__ J,
                                                     const double *__restrict__ Vinv, const double *__restrict__ lp,
                                                     const int *__restrict__ cdim, const int *__restrict__ off,
                                                     const T *__restrict__ dxc, const double *__restrict__ pts,
                                                     double *__restrict__ dxp, double *__restrict__ pts_t) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        double s[3] = {lp[3 * k], lp[3 * k + 1], lp[3 * k + 2]};
        for (int a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a) {
            const T *o = J + (int64_t)a * VJW;
            const int i = ocam[a], ci = cdim[i];
            const T *dc = dxc + off[i];
            double t0 = 0.0, t1 = 0.0;
            for (int c = 0; c < ci; ++c) {
                t0 += (double)o[c] * (double)dc[c];
                t1 += (double)o[VB_CI + c] * (double)dc[c];
            }
            for (int m = 0; m < 3; ++m) s[m] -= (double)o[22 + m] * t0 + (double)o[25 + m] * t1;
        }
        const double *vi = Vinv + 9 * k;
        for (int m = 0; m < 3; ++m) {
            const double d = vi[3 * m] * s[0] + vi[3 * m + 1] * s[1] + vi[3 * m + 2] * s[2];
            dxp[3 * k + m] = d;
            pts_t[3 * k + m] = pts[3 * k + m] + d;
        }
    }
}

// The trial cameras: the pose perturbed in the camera frame,
// R <- Exp(d_omega) R, t <- Exp(d_omega) t + dt (unit quaternions), and the
// interiors of a self-calibrating camera (c_i = 11) moved additively.
template <typename T>
__global__ void k_vbi_update_cams(int n, const double *__restrict__ cams, const double *__restrict__ intr,
                                  const int *__restrict__ cdim, const int *__restrict__ off, const T *__restrict__ dxc,
                                  double *__restrict__ cams_t, double *__restrict__ intr_t) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T *dc = dxc + off[i];
    double w[3], q[4], qd[4], qn[4], Rd[9];
    const double dw[3] = {(double)dc[0], (double)dc[1], (double)dc[2]};
    quat_exp(cams + 6 * i, q);
    quat_exp(dw, qd);
    quat_mul(qd, q, qn);
    const double nn = rsqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
    for (int k = 0; k < 4; ++k) qn[k] *= nn;
    quat_log(qn, w);
    quat_to_R(qd, Rd);
    const double *t = cams + 6 * i + 3;
    for (int r = 0; r < 3; ++r) {
        cams_t[6 * i + r] = w[r];
        cams_t[6 * i + 3 + r] = Rd[3 * r] * t[0] + Rd[3 * r + 1] * t[1] + Rd[3 * r + 2] * t[2] + (double)dc[3 + r];
    }
    const bool self_cal = cdim[i] == VB_CI;
    for (int r = 0; r < 5; ++r) intr_t[5 * i + r] = intr[5 * i + r] + (self_cal ? (double)dc[6 + r] : 0.0);
}

// Per observation the trial residual (trial cost, camc_t the trial cameras'
// [R, t]) and the model decrease term -(2 e^T J dx + ||J dx||^2),
// J dx = J_c dx_c (c_i columns) + J_p dx_p; both summed in FP64, plus the
// trial cheirality count.
template <typename T>
__global__ void __launch_bounds__(256) k_vbi_trial(int64_t m, const int *__restrict__ ocam,
                                                   const int *__restrict__ opt, const double *__restrict__ uv,
                                                   const T *__restrict__ J, const int *__restrict__ cdim,
                                                   const int *__restrict__ off, const T *__restrict__ dxc,
                                                   const double *__restrict__ dxp, const double *__restrict__ camc_t,
                                                   const double *__restrict__ intr_t, const double *__restrict__ pts_t,
                                                   VbiScalars *sc, double *red, unsigned *ctr) {
    double v[3] = {0.0, 0.0, 0.0};
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const int i = ocam[a], k = opt[a], ci = cdim[i];
        const VbiProj<T> pr = vbi_project<T>(camc_t, intr_t, pts_t, i, k, uv + 2 * a);
        v[0] += (double)pr.e0 * (double)pr.e0 + (double)pr.e1 * (double)pr.e1;
        v[2] += pr.Xc[2] <= T(1e-6) ? 1.0 : 0.0;
        const T *o = J + a * VJW;
        const T *dc = dxc + off[i];
        T t0 = T(0), t1 = T(0);
        for (int c = 0; c < ci; ++c) {
            t0 += o[c] * dc[c];
            t1 += o[VB_CI + c] * dc[c];
        }
        for (int c = 0; c < 3; ++c) {
            t0 += o[22 + c] * (T)dxp[3 * (int64_t)k + c];
            t1 += o[25 + c] * (T)dxp[3 * (int64_t)k + c];
        }
        v[1] -= (double)(t0 * (T(2) * o[28] + t0) + t1 * (T(2) * o[29] + t1));
    }
    grid_sum<3>(v, red, ctr, [&](double *t) {
        sc->cost_trial = 0.5 * t[0];
        sc->model = 0.5 * t[1];
        sc->n_cheir_trial = (unsigned long long)t[2];
    });
}

}  // namespace ba

using namespace ba;

namespace {

bool finite_n(const double *x, int64_t cnt) {
    for (int64_t k = 0; k < cnt; ++k)
        if (!std::isfinite(x[k])) return false;
    return true;
}

// Temporary device buffers of one formation, freed on every exit.
struct Scratch {
    std::vector<void *> ptrs;
    cudaError_t alloc(void **d, size_t bytes) {
        cudaError_t e = cudaMalloc(d, bytes < 16 ? 16 : bytes);
        if (e == cudaSuccess) ptrs.push_back(*d);
        return e;
    }
    cudaError_t put(void **d, const void *src, size_t bytes) {
        cudaError_t e = alloc(d, bytes);
        return e != cudaSuccess ? e : cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice);
    }
    ~Scratch() {
        for (void *p : ptrs) cudaFree(p);
    }
};

// The block pattern and the slot-pair lists of k_vbi_blocks.  Every
// observation a (internal order: by point, then camera) has ns slots, slot s
// in block blk(a, s).  The pattern holds every diagonal block and each
// (beta <= gamma) that two slots of one point fall in; the pairs of a block
// are, point by point in track order, the ordered slot pairs (x in beta,
// y in gamma) - all of them when beta == gamma - stored as their
// observations.
struct VbiLayout {
    std::vector<int32_t> row_ptr, col, pptr;
    std::vector<int2> plist;
};

template <class Blk>
ba_status vbi_layout(int32_t nblk, int64_t P, const std::vector<int32_t> &trk_ptr, int ns, Blk blk, VbiLayout &L) {
    std::vector<uint64_t> keys;
    keys.reserve((size_t)nblk + trk_ptr[P] * 4);
    for (int32_t b = 0; b < nblk; ++b) keys.push_back((uint64_t)b * nblk + b);
    std::vector<int32_t> sb;
    for (int64_t k = 0; k < P; ++k) {
        sb.clear();
        for (int32_t a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a)
            for (int s = 0; s < ns; ++s) sb.push_back(blk(a, s));
        for (size_t x = 0; x < sb.size(); ++x)
            for (size_t y = 0; y < sb.size(); ++y)
                if (sb[x] < sb[y]) keys.push_back((uint64_t)sb[x] * nblk + sb[y]);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    if ((int64_t)keys.size() >= (int64_t)INT32_MAX) return set_error(BA_ERR_INVALID_ARG, "too many RCS blocks");
    L.row_ptr.assign(nblk + 1, 0);
    L.col.resize(keys.size());
    for (size_t q = 0; q < keys.size(); ++q) {
        L.row_ptr[keys[q] / nblk + 1]++;
        L.col[q] = (int32_t)(keys[q] % nblk);
    }
    for (int32_t b = 0; b < nblk; ++b) L.row_ptr[b + 1] += L.row_ptr[b];
    const int64_t nnzb = (int64_t)keys.size();
    auto block_of = [&](int32_t beta, int32_t gamma) {
        const int32_t *c0 = L.col.data() + L.row_ptr[beta], *c1 = L.col.data() + L.row_ptr[beta + 1];
        return (int64_t)(std::lower_bound(c0, c1, gamma) - L.col.data());
    };
    std::vector<int64_t> cnt(nnzb + 1, 0);
    std::vector<std::pair<int32_t, int32_t>> sl;  // (block, observation) of the point's slots
    auto each_pair = [&](auto &&fn) {
        for (int64_t k = 0; k < P; ++k) {
            sl.clear();
            for (int32_t a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a)
                for (int s = 0; s < ns; ++s) sl.emplace_back(blk(a, s), a);
            for (size_t x = 0; x < sl.size(); ++x)
                for (size_t y = 0; y < sl.size(); ++y)
                    if (sl[x].first <= sl[y].first) fn(block_of(sl[x].first, sl[y].first), sl[x].second, sl[y].second);
        }
    };
    each_pair([&](int64_t b, int32_t, int32_t) { cnt[b + 1]++; });
    for (int64_t b = 0; b < nnzb; ++b) cnt[b + 1] += cnt[b];
    if (cnt[nnzb] >= (int64_t)INT32_MAX) return set_error(BA_ERR_INVALID_ARG, "more than 2^31 slot pairs");
    L.pptr.assign(cnt.begin(), cnt.end());
    L.plist.resize(cnt[nnzb]);
    std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
    each_pair([&](int64_t b, int32_t x, int32_t y) { L.plist[fill[b]++] = make_int2(x, y); });
    return BA_OK;
}

// Device inputs of the formation, owned by the caller of vbi_form.
struct VbiDev {
    int *ocam = nullptr, *opt = nullptr, *trk = nullptr, *pptr = nullptr, *jc0 = nullptr, *err = nullptr;
    int2 *plist = nullptr;
    double *uv = nullptr, *Vinv = nullptr, *lp = nullptr, *camc = nullptr;
    void *J = nullptr, *PE = nullptr;  // rows in the storage precision: VJW and VPW values per observation
};

// e and J at (cams, intr, pts): the cameras' [R, t] into d.camc, then the rows.
cudaError_t vbi_linearize(ba_vbsmc *h, const VbiDev &d, int64_t m, int n, const double *cams, const double *intr,
                          const double *pts) {
    k_vbi_camcache<<<(n + 127) / 128, 128, 0, h->st>>>(n, cams, d.camc);
    const int g1 = (int)std::min<int64_t>((m + 255) / 256, 152 * 16);
    if (h->fp32)
        k_vbi_linearize<float><<<g1, 256, 0, h->st>>>(m, d.ocam, d.opt, d.uv, d.camc, intr, pts, (float *)d.J);
    else
        k_vbi_linearize<double><<<g1, 256, 0, h->st>>>(m, d.ocam, d.opt, d.uv, d.camc, intr, pts, (double *)d.J);
    return cudaGetLastError();
}

// From the stored rows: V_k^-1, l_p and the factor rows per point, then the
// damped RCS into h's values and b (queued on h's stream; M^-1 is left to
// vb_finish).
cudaError_t vbi_form(ba_vbsmc *h, const VbiDev &d, int64_t P, double lambda) {
    cudaError_t e = cudaMemsetAsync(d.err, 0, sizeof(int), h->st);
    if (e != cudaSuccess) return e;
    const int g2 = (int)std::min<int64_t>((P + 255) / 256, 152 * 16);
    const int g3 = (int)std::min<int64_t>((h->nnzb * 32 + 255) / 256, 152 * 16);
    if (h->fp32) {
        k_vbi_points<float><<<g2, 256, 0, h->st>>>(P, d.trk, (const float *)d.J, lambda, d.Vinv, d.lp, (float *)d.PE,
                                                   d.err);
        k_vbi_blocks<float><<<g3, 256, 0, h->st>>>(h->nnzb, h->brow, h->col, h->cdim, d.jc0, h->off, h->boff, d.pptr,
                                                   d.plist, (const float *)d.J, (const float *)d.PE, lambda,
                                                   (float *)h->val, (float *)h->b);
    } else {
        k_vbi_points<double><<<g2, 256, 0, h->st>>>(P, d.trk, (const double *)d.J, lambda, d.Vinv, d.lp,
                                                    (double *)d.PE, d.err);
        k_vbi_blocks<double><<<g3, 256, 0, h->st>>>(h->nnzb, h->brow, h->col, h->cdim, d.jc0, h->off, h->boff,
                                                    d.pptr, d.plist, (const double *)d.J, (const double *)d.PE,
                                                    lambda, (double *)h->val, (double *)h->b);
    }
    return cudaGetLastError();
}

// F of the stored rows into sc->cost (FP64 sum)
cudaError_t vbi_cost(ba_vbsmc *h, const VbiDev &d, int64_t m, VbiScalars *sc, double *red, unsigned *ctr) {
    const int g = (int)std::min<int64_t>((m + 255) / 256, 152 * 4);
    if (h->fp32)
        k_vbi_cost<float><<<g, 256, 0, h->st>>>(m, (const float *)d.J, sc, red, ctr);
    else
        k_vbi_cost<double><<<g, 256, 0, h->st>>>(m, (const double *)d.J, sc, red, ctr);
    return cudaGetLastError();
}

// One-shot formation of a variable-size RCS (the two creation entry points).
ba_status vbi_create(const ba_options &o, int32_t nblk, const std::vector<int32_t> &cdim,
                     const std::vector<int32_t> *jc0, const HostSetup &hs, const VbiLayout &L, int64_t n_pts,
                     int64_t n_obs, const std::vector<double> &uv, const double *cams, int32_t n_cams,
                     const std::vector<double> &intr, const std::vector<double> &ptsi, double lambda, ba_vbsmc **out) {
    ba_vbsmc *h = nullptr;
    ba_status s = vb_build(o, nblk, cdim.data(), (int64_t)L.col.size(), L.row_ptr.data(), L.col.data(), &h);
    if (s) return s;
    Scratch sc;
    VbiDev d;
    double *d_cams = nullptr, *d_intr = nullptr, *d_pts = nullptr;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    step(sc.put((void **)&d.ocam, hs.obs_cam.data(), n_obs * sizeof(int32_t)));
    step(sc.put((void **)&d.opt, hs.obs_pt.data(), n_obs * sizeof(int32_t)));
    step(sc.put((void **)&d.trk, hs.trk_ptr.data(), (n_pts + 1) * sizeof(int32_t)));
    step(sc.put((void **)&d.pptr, L.pptr.data(), L.pptr.size() * sizeof(int32_t)));
    step(sc.put((void **)&d.plist, L.plist.data(), L.plist.size() * sizeof(int2)));
    if (jc0) step(sc.put((void **)&d.jc0, jc0->data(), jc0->size() * sizeof(int32_t)));
    step(sc.put((void **)&d.uv, uv.data(), uv.size() * sizeof(double)));
    step(sc.put((void **)&d_cams, cams, (size_t)n_cams * 6 * sizeof(double)));
    step(sc.put((void **)&d_intr, intr.data(), intr.size() * sizeof(double)));
    step(sc.put((void **)&d_pts, ptsi.data(), ptsi.size() * sizeof(double)));
    step(sc.alloc((void **)&d.J, (size_t)n_obs * VJW * h->esz));
    step(sc.alloc((void **)&d.PE, (size_t)n_obs * VPW * h->esz));
    step(sc.alloc((void **)&d.camc, (size_t)n_cams * 12 * sizeof(double)));
    step(sc.alloc((void **)&d.Vinv, (size_t)n_pts * 9 * sizeof(double)));
    step(sc.alloc((void **)&d.lp, (size_t)n_pts * 3 * sizeof(double)));
    step(sc.alloc((void **)&d.err, sizeof(int)));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        ba_vbsmc_destroy(h);
        return set_error(BA_ERR_OOM, "cudaMalloc failed");
    }
    if (e == cudaSuccess) e = vbi_linearize(h, d, n_obs, n_cams, d_cams, d_intr, d_pts);
    if (e == cudaSuccess) e = vbi_form(h, d, n_pts, lambda);
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d.err, sizeof(int), cudaMemcpyDeviceToHost, h->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
    if (e != cudaSuccess) {
        ba_vbsmc_destroy(h);
        return set_error(BA_ERR_CUDA, (std::string("forming the RCS with interiors: ") + cudaGetErrorString(e)).c_str());
    }
    if (flag == BA_ERR_NOT_SPD) {
        ba_vbsmc_destroy(h);
        return set_error(BA_ERR_NOT_SPD, "a point's V is not positive definite");
    }
    if ((s = vb_finish(h))) {
        ba_vbsmc_destroy(h);
        return s;
    }
    *out = h;
    return BA_OK;
}

// Observation inputs in the internal order (by point, then camera).
void internal_inputs(const HostSetup &hs, int64_t n_pts, int64_t n_obs, const double *obs_uv, const double *pts,
                     std::vector<double> &uv, std::vector<double> &ptsi) {
    uv.resize(2 * n_obs);
    ptsi.resize(3 * n_pts);
    for (int64_t a = 0; a < n_obs; ++a) {
        uv[2 * a] = obs_uv[2 * hs.obs_perm[a]];
        uv[2 * a + 1] = obs_uv[2 * hs.obs_perm[a] + 1];
    }
    for (int64_t k = 0; k < n_pts; ++k)
        for (int c = 0; c < 3; ++c) ptsi[3 * k + c] = pts[3 * hs.pt_perm[k] + c];
}

ba_status check_scene(int32_t n_cams, const double *cams, int64_t n_pts, const double *pts, int64_t n_obs,
                      const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv, double lambda) {
    if (!cams || !pts || !obs_cam || !obs_pt || !obs_uv) return set_error(BA_ERR_INVALID_ARG, "null input array");
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0) return set_error(BA_ERR_INVALID_ARG, "sizes must be positive");
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return set_error(BA_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    if (!finite_n(cams, (int64_t)n_cams * 6) || !finite_n(pts, n_pts * 3) || !finite_n(obs_uv, n_obs * 2))
        return set_error(BA_ERR_NONFINITE, "non-finite camera, point or observation value");
    return BA_OK;
}

}  // namespace

struct ba_vbi_problem {
    ba_options opt{};
    int32_t n = 0;
    int64_t P = 0, m = 0;
    HostSetup hs;
    std::vector<int32_t> cdim;
    ba_vbsmc *h = nullptr;  // the RCS storage, its block-Jacobi M^-1 and PCG
    VbiDev d;
    double *cams = nullptr, *intr = nullptr, *pts = nullptr, *cams_t = nullptr, *intr_t = nullptr, *pts_t = nullptr;
    double *dxp = nullptr, *red = nullptr, *camc_t = nullptr;
    unsigned *ctr = nullptr;
    VbiScalars *sc = nullptr, *sc_host = nullptr;
    std::vector<void *> allocs;
    cudaEvent_t ev[6] = {};
    double lambda = 1e-4, nu = 2.0, F = 0.0;
    bool linearized = false, stepped = false, dead = false;
    int64_t dev_bytes = 0;
};

namespace {

ba_status vbi_fail(ba_vbi_problem *p, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BA_OK;
    p->dead = true;
    return set_error(BA_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

ba_status vbi_alloc(ba_vbi_problem *p, void **dptr, size_t bytes) {
    bytes = bytes < 16 ? 16 : bytes;
    if (p->opt.device_mem_cap && (size_t)p->dev_bytes + p->h->dev_bytes + bytes > p->opt.device_mem_cap)
        return set_error(BA_ERR_OOM, "device_mem_cap reached");
    cudaError_t e = cudaMalloc(dptr, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(BA_ERR_OOM, "cudaMalloc failed");
    }
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    p->allocs.push_back(*dptr);
    p->dev_bytes += (int64_t)bytes;
    return BA_OK;
}

ba_status vbi_put(ba_vbi_problem *p, void **dptr, const void *src, size_t bytes) {
    ba_status s = vbi_alloc(p, dptr, bytes);
    if (s) return s;
    return vbi_fail(p, cudaMemcpy(*dptr, src, bytes, cudaMemcpyHostToDevice), "upload");
}

void vbi_free(ba_vbi_problem *p) {
    if (!p) return;
    if (p->h) {
        cudaStreamSynchronize(p->h->st);
        ba_vbsmc_destroy(p->h);
    }
    for (auto &e : p->ev)
        if (e) cudaEventDestroy(e);
    for (void *q : p->allocs) cudaFree(q);
    if (p->sc_host) cudaFreeHost(p->sc_host);
    delete p;
}

}  // namespace

extern "C" {

ba_status ba_vbsmc_create_interiors(const ba_options *opt, int32_t n_cams, const double *cams, const double *intr,
                                    const int32_t *cdim, int64_t n_pts, const double *pts, int64_t n_obs,
                                    const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv, double lambda,
                                    ba_vbsmc **out) {
    if (!out) return set_error(BA_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return set_error(BA_ERR_INVALID_ARG, "bad precision");
    ba_status s = check_scene(n_cams, cams, n_pts, pts, n_obs, obs_cam, obs_pt, obs_uv, lambda);
    if (s) return s;
    if (!intr || !cdim) return set_error(BA_ERR_INVALID_ARG, "null input array");
    for (int32_t i = 0; i < n_cams; ++i)
        if (cdim[i] != 6 && cdim[i] != VB_CI) return set_error(BA_ERR_INVALID_ARG, "cdim must be 6 or 11");
    if (!finite_n(intr, (int64_t)n_cams * 5)) return set_error(BA_ERR_NONFINITE, "non-finite interior value");
    HostSetup hs;
    std::string err;
    s = symbolic_setup(n_cams, n_pts, n_obs, obs_cam, obs_pt, nullptr, OBS_MAX_DEFAULT, true, hs, err);
    if (s) return set_error(s, err.c_str());
    VbiLayout L;
    if ((s = vbi_layout(n_cams, n_pts, hs.trk_ptr, 1, [&](int32_t a, int) { return hs.obs_cam[a]; }, L))) return s;
    std::vector<double> uv, ptsi;
    internal_inputs(hs, n_pts, n_obs, obs_uv, pts, uv, ptsi);
    std::vector<int32_t> cd(cdim, cdim + n_cams);
    std::vector<double> in(intr, intr + 5 * (size_t)n_cams);
    return vbi_create(o, n_cams, cd, nullptr, hs, L, n_pts, n_obs, uv, cams, n_cams, in, ptsi, lambda, out);
}

ba_status ba_vbsmc_create_shared(const ba_options *opt, int32_t n_images, const double *cams, int32_t n_phys,
                                 const double *intr_phys, const int32_t *phys, int64_t n_pts, const double *pts,
                                 int64_t n_obs, const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv,
                                 double lambda, ba_vbsmc **out) {
    if (!out) return set_error(BA_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return set_error(BA_ERR_INVALID_ARG, "bad precision");
    ba_status s = check_scene(n_images, cams, n_pts, pts, n_obs, obs_cam, obs_pt, obs_uv, lambda);
    if (s) return s;
    if (!intr_phys || !phys) return set_error(BA_ERR_INVALID_ARG, "null input array");
    if (n_phys <= 0 || (int64_t)n_images + n_phys >= (1 << 30))
        return set_error(BA_ERR_INVALID_ARG, "need 0 < n_phys and n_images + n_phys < 2^30");
    for (int32_t i = 0; i < n_images; ++i)
        if (phys[i] < 0 || phys[i] >= n_phys) return set_error(BA_ERR_INVALID_ARG, "phys index out of range");
    if (!finite_n(intr_phys, (int64_t)n_phys * 5)) return set_error(BA_ERR_NONFINITE, "non-finite interior value");
    HostSetup hs;
    std::string err;
    s = symbolic_setup(n_images, n_pts, n_obs, obs_cam, obs_pt, nullptr, OBS_MAX_DEFAULT, true, hs, err);
    if (s) return set_error(s, err.c_str());
    const int32_t nblk = n_images + n_phys;
    VbiLayout L;
    auto blk = [&](int32_t a, int sl) { return sl == 0 ? hs.obs_cam[a] : n_images + phys[hs.obs_cam[a]]; };
    if ((s = vbi_layout(nblk, n_pts, hs.trk_ptr, 2, blk, L))) return s;
    std::vector<double> uv, ptsi;
    internal_inputs(hs, n_pts, n_obs, obs_uv, pts, uv, ptsi);
    std::vector<int32_t> cd(nblk, 6), jc0(nblk, 0);
    for (int32_t q = n_images; q < nblk; ++q) {
        cd[q] = 5;
        jc0[q] = 6;
    }
    std::vector<double> in(5 * (size_t)n_images);  // each image's interiors: its physical camera's
    for (int32_t i = 0; i < n_images; ++i)
        for (int c = 0; c < 5; ++c) in[5 * i + c] = intr_phys[5 * phys[i] + c];
    return vbi_create(o, nblk, cd, &jc0, hs, L, n_pts, n_obs, uv, cams, n_images, in, ptsi, lambda, out);
}

ba_status ba_vbi_problem_create(const ba_options *opt, int32_t n_cams, const double *cams, const double *intr,
                                const int32_t *cdim, int64_t n_pts, const double *pts, int64_t n_obs,
                                const int32_t *obs_cam, const int64_t *obs_pt, const double *obs_uv,
                                ba_vbi_problem **out) {
    if (!out) return set_error(BA_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return set_error(BA_ERR_INVALID_ARG, "bad precision");
    if (!(o.lambda0 > 0) || !std::isfinite(o.lambda0)) return set_error(BA_ERR_INVALID_ARG, "lambda0 must be > 0");
    if (!(o.pcg_rel_tol > 0) || o.pcg_max_iters < 0) return set_error(BA_ERR_INVALID_ARG, "bad PCG options");
    ba_status s = check_scene(n_cams, cams, n_pts, pts, n_obs, obs_cam, obs_pt, obs_uv, 0.0);
    if (s) return s;
    if (!intr || !cdim) return set_error(BA_ERR_INVALID_ARG, "null input array");
    for (int32_t i = 0; i < n_cams; ++i)
        if (cdim[i] != 6 && cdim[i] != VB_CI) return set_error(BA_ERR_INVALID_ARG, "cdim must be 6 or 11");
    if (!finite_n(intr, (int64_t)n_cams * 5)) return set_error(BA_ERR_NONFINITE, "non-finite interior value");
    ba_vbi_problem *p = new ba_vbi_problem();
    p->opt = o;
    p->n = n_cams;
    p->P = n_pts;
    p->m = n_obs;
    p->lambda = o.lambda0;
    p->cdim.assign(cdim, cdim + n_cams);
    std::string err;
    s = symbolic_setup(n_cams, n_pts, n_obs, obs_cam, obs_pt, nullptr, OBS_MAX_DEFAULT, true, p->hs, err);
    if (s) {
        vbi_free(p);
        return set_error(s, err.c_str());
    }
    VbiLayout L;
    const HostSetup &hs = p->hs;
    if ((s = vbi_layout(n_cams, n_pts, hs.trk_ptr, 1, [&](int32_t a, int) { return hs.obs_cam[a]; }, L))) {
        vbi_free(p);
        return s;
    }
    if ((s = vb_build(o, n_cams, cdim, (int64_t)L.col.size(), L.row_ptr.data(), L.col.data(), &p->h))) {
        p->h = nullptr;
        vbi_free(p);
        return s;
    }
    std::vector<double> uv, ptsi;
    internal_inputs(hs, n_pts, n_obs, obs_uv, pts, uv, ptsi);
    const size_t C6 = (size_t)n_cams * 6 * 8, C5 = (size_t)n_cams * 5 * 8, P3 = (size_t)n_pts * 3 * 8;
    if (!s) s = vbi_put(p, (void **)&p->d.ocam, hs.obs_cam.data(), n_obs * sizeof(int32_t));
    if (!s) s = vbi_put(p, (void **)&p->d.opt, hs.obs_pt.data(), n_obs * sizeof(int32_t));
    if (!s) s = vbi_put(p, (void **)&p->d.trk, hs.trk_ptr.data(), (n_pts + 1) * sizeof(int32_t));
    if (!s) s = vbi_put(p, (void **)&p->d.pptr, L.pptr.data(), L.pptr.size() * sizeof(int32_t));
    if (!s) s = vbi_put(p, (void **)&p->d.plist, L.plist.data(), L.plist.size() * sizeof(int2));
    if (!s) s = vbi_put(p, (void **)&p->d.uv, uv.data(), uv.size() * sizeof(double));
    if (!s) s = vbi_alloc(p, (void **)&p->d.J, (size_t)n_obs * VJW * p->h->esz);
    if (!s) s = vbi_alloc(p, (void **)&p->d.PE, (size_t)n_obs * VPW * p->h->esz);
    if (!s) s = vbi_alloc(p, (void **)&p->d.camc, (size_t)n_cams * 12 * sizeof(double));
    if (!s) s = vbi_alloc(p, (void **)&p->camc_t, (size_t)n_cams * 12 * sizeof(double));
    if (!s) s = vbi_alloc(p, (void **)&p->d.Vinv, (size_t)n_pts * 9 * sizeof(double));
    if (!s) s = vbi_alloc(p, (void **)&p->d.lp, P3);
    if (!s) s = vbi_alloc(p, (void **)&p->d.err, sizeof(int));
    if (!s) s = vbi_put(p, (void **)&p->cams, cams, C6);
    if (!s) s = vbi_put(p, (void **)&p->intr, intr, C5);
    if (!s) s = vbi_put(p, (void **)&p->pts, ptsi.data(), P3);
    if (!s) s = vbi_alloc(p, (void **)&p->cams_t, C6);
    if (!s) s = vbi_alloc(p, (void **)&p->intr_t, C5);
    if (!s) s = vbi_alloc(p, (void **)&p->pts_t, P3);
    if (!s) s = vbi_alloc(p, (void **)&p->dxp, P3);
    if (!s) s = vbi_alloc(p, (void **)&p->red, (size_t)RED_SLOTS * sizeof(double));
    if (!s) s = vbi_alloc(p, (void **)&p->ctr, 64);
    if (!s) s = vbi_alloc(p, (void **)&p->sc, sizeof(VbiScalars));
    if (!s) s = vbi_fail(p, cudaMemset(p->ctr, 0, 64), "memset");
    if (!s) s = vbi_fail(p, cudaMallocHost((void **)&p->sc_host, sizeof(VbiScalars)), "cudaMallocHost");
    for (auto &e : p->ev)
        if (!s) s = vbi_fail(p, cudaEventCreate(&e), "event");
    if (s) {
        vbi_free(p);
        return s;
    }
    *out = p;
    return BA_OK;
}

void ba_vbi_problem_destroy(ba_vbi_problem *p) { vbi_free(p); }

ba_status ba_vbi_lm_step(ba_vbi_problem *p, ba_step_info *info) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (p->dead) return set_error(BA_ERR_STATE, "the problem is unusable after an earlier error");
    ba_vbsmc *h = p->h;
    cudaStream_t st = h->st;
    ba_status s;
    const bool relin = !p->linearized;
    if ((s = vbi_fail(p, cudaEventRecord(p->ev[0], st), "event"))) return s;
    if (relin) {
        if ((s = vbi_fail(p, vbi_linearize(h, p->d, p->m, p->n, p->cams, p->intr, p->pts), "k_vbi_linearize")))
            return s;
        if ((s = vbi_fail(p, vbi_cost(h, p->d, p->m, p->sc, p->red, p->ctr), "k_vbi_cost"))) return s;
    }
    if ((s = vbi_fail(p, cudaEventRecord(p->ev[1], st), "event"))) return s;
    // Eq. 3-4 with c_i unknowns per camera, then the block-Jacobi M^-1
    if ((s = vbi_fail(p, vbi_form(h, p->d, p->P, p->lambda), "forming the RCS"))) return s;
    int flag = 0;
    if ((s = vbi_fail(p, cudaMemcpyAsync(&flag, p->d.err, sizeof(int), cudaMemcpyDeviceToHost, st), "copy")))
        return s;
    if ((s = vb_finish(h))) {  // synchronises
        if (s != BA_ERR_NOT_SPD) p->dead = true;
        return s;
    }
    if (flag == BA_ERR_NOT_SPD) return set_error(BA_ERR_NOT_SPD, "a point's V is not positive definite");
    if (relin) {
        if ((s = vbi_fail(p, cudaMemcpy(p->sc_host, p->sc, sizeof(VbiScalars), cudaMemcpyDeviceToHost), "copy")))
            return s;
        p->F = p->sc_host->cost;
        p->linearized = true;
    }
    if ((s = vbi_fail(p, cudaEventRecord(p->ev[2], st), "event"))) return s;
    // Sec. 3.2: block-Jacobi PCG on S dx_c = b
    int iters = 0;
    double rel = 0.0;
    s = ba_vbsmc_solve(h, p->opt.pcg_rel_tol, p->opt.pcg_max_iters, nullptr, &iters, &rel, nullptr);
    if (s != BA_OK && s != BA_ERR_NO_CONVERGENCE) {
        if (s != BA_ERR_NOT_SPD) p->dead = true;
        return s;
    }
    if ((s = vbi_fail(p, cudaEventRecord(p->ev[3], st), "event"))) return s;
    // Eq. 5, the trial state, its cost and the model decrease
    const int gp = (int)std::min<int64_t>((p->P + 255) / 256, 152 * 16);
    const int go = (int)std::min<int64_t>((p->m + 255) / 256, 152 * 4);
    const int gc = (p->n + 127) / 128;
    if (h->fp32) {
        const float *dxc = (const float *)h->vec[0];
        k_vbi_backsub<float><<<gp, 256, 0, st>>>(p->P, p->d.trk, p->d.ocam, (const float *)p->d.J, p->d.Vinv,
                                                 p->d.lp, h->cdim, h->off, dxc, p->pts, p->dxp, p->pts_t);
        k_vbi_update_cams<float><<<gc, 128, 0, st>>>(p->n, p->cams, p->intr, h->cdim, h->off, dxc, p->cams_t,
                                                     p->intr_t);
        k_vbi_camcache<<<gc, 128, 0, st>>>(p->n, p->cams_t, p->camc_t);
        if ((s = vbi_fail(p, cudaEventRecord(p->ev[4], st), "event"))) return s;
        k_vbi_trial<float><<<go, 256, 0, st>>>(p->m, p->d.ocam, p->d.opt, p->d.uv, (const float *)p->d.J, h->cdim,
                                               h->off, dxc, p->dxp, p->camc_t, p->intr_t, p->pts_t, p->sc, p->red,
                                               p->ctr + 1);
    } else {
        const double *dxc = (const double *)h->vec[0];
        k_vbi_backsub<double><<<gp, 256, 0, st>>>(p->P, p->d.trk, p->d.ocam, (const double *)p->d.J, p->d.Vinv,
                                                  p->d.lp, h->cdim, h->off, dxc, p->pts, p->dxp, p->pts_t);
        k_vbi_update_cams<double><<<gc, 128, 0, st>>>(p->n, p->cams, p->intr, h->cdim, h->off, dxc, p->cams_t,
                                                      p->intr_t);
        k_vbi_camcache<<<gc, 128, 0, st>>>(p->n, p->cams_t, p->camc_t);
        if ((s = vbi_fail(p, cudaEventRecord(p->ev[4], st), "event"))) return s;
        k_vbi_trial<double><<<go, 256, 0, st>>>(p->m, p->d.ocam, p->d.opt, p->d.uv, (const double *)p->d.J, h->cdim,
                                                h->off, dxc, p->dxp, p->camc_t, p->intr_t, p->pts_t, p->sc, p->red,
                                                p->ctr + 1);
    }
    if ((s = vbi_fail(p, cudaGetLastError(), "trial kernels"))) return s;
    if ((s = vbi_fail(p, cudaEventRecord(p->ev[5], st), "event"))) return s;
    if ((s = vbi_fail(p, cudaMemcpyAsync(p->sc_host, p->sc, sizeof(VbiScalars), cudaMemcpyDeviceToHost, st), "copy")))
        return s;
    if ((s = vbi_fail(p, cudaStreamSynchronize(st), "sync"))) return s;
    // gain ratio and Nielsen's damping rule, as the 6-unknown LM step
    const double F0 = p->F, F1 = p->sc_host->cost_trial, pred = p->sc_host->model;
    const double rho = pred > 0 ? (F0 - F1) / pred : -INFINITY;
    const bool ok = pred > 0 && rho > 1e-3 && std::isfinite(F1);
    ba_step_info loc{};
    loc.cost_before = F0;
    loc.cost_trial = F1;
    loc.predicted = pred;
    loc.rho = rho;
    loc.lambda = p->lambda;
    loc.accepted = ok ? 1 : 0;
    loc.pcg_iters = iters;
    loc.rcs_rel_resid = rel;
    loc.n_cheirality = (int64_t)p->sc_host->n_cheir_trial;
    float ms[5] = {0, 0, 0, 0, 0};
    for (int k = 0; k < 5; ++k) cudaEventElapsedTime(&ms[k], p->ev[k], p->ev[k + 1]);
    loc.ms[0] = ms[0];                  // linearize and cost
    loc.ms[1] = ms[1];                  // RCS formation and M^-1
    loc.ms[2] = ms[2];                  // PCG
    loc.ms[3] = ms[3];                  // Eq. 5 and the trial cameras
    loc.ms[4] = ms[4];                  // trial cost and model decrease
    loc.ms[5] = ms[0] + ms[1] + ms[2] + ms[3] + ms[4];
    if (ok) {
        std::swap(p->cams, p->cams_t);
        std::swap(p->intr, p->intr_t);
        std::swap(p->pts, p->pts_t);
        std::swap(p->d.camc, p->camc_t);
        p->F = F1;
        p->linearized = false;
        p->lambda *= std::max(1.0 / 3.0, 1.0 - std::pow(2.0 * rho - 1.0, 3));
        p->nu = 2.0;
    } else {
        p->lambda *= p->nu;
        p->nu *= 2.0;
    }
    loc.cost_after = ok ? F1 : F0;
    p->stepped = true;
    if (info) *info = loc;
    return BA_OK;
}

ba_status ba_vbi_get_state(const ba_vbi_problem *p, double *cams, double *intr, double *pts) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (p->dead) return set_error(BA_ERR_STATE, "the problem is unusable after an earlier error");
    ba_vbi_problem *q = const_cast<ba_vbi_problem *>(p);
    ba_status s;
    if ((s = vbi_fail(q, cudaStreamSynchronize(p->h->st), "sync"))) return s;
    if (cams && (s = vbi_fail(q, cudaMemcpy(cams, p->cams, (size_t)p->n * 48, cudaMemcpyDeviceToHost), "copy")))
        return s;
    if (intr && (s = vbi_fail(q, cudaMemcpy(intr, p->intr, (size_t)p->n * 40, cudaMemcpyDeviceToHost), "copy")))
        return s;
    if (pts) {
        std::vector<double> t(3 * p->P);
        if ((s = vbi_fail(q, cudaMemcpy(t.data(), p->pts, t.size() * 8, cudaMemcpyDeviceToHost), "copy"))) return s;
        for (int64_t k = 0; k < p->P; ++k)
            for (int c = 0; c < 3; ++c) pts[3 * p->hs.pt_perm[k] + c] = t[3 * k + c];
    }
    return BA_OK;
}

ba_status ba_vbi_set_state(ba_vbi_problem *p, const double *cams, const double *intr, const double *pts,
                           double lambda, double nu) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (p->dead) return set_error(BA_ERR_STATE, "the problem is unusable after an earlier error");
    if (!cams || !intr || !pts) return set_error(BA_ERR_INVALID_ARG, "null input array");
    if (!(lambda > 0) || !std::isfinite(lambda) || !(nu > 0) || !std::isfinite(nu))
        return set_error(BA_ERR_INVALID_ARG, "lambda and nu must be finite and > 0");
    if (!finite_n(cams, (int64_t)p->n * 6) || !finite_n(intr, (int64_t)p->n * 5) || !finite_n(pts, p->P * 3))
        return set_error(BA_ERR_NONFINITE, "non-finite state value");
    std::vector<double> t(3 * p->P);
    for (int64_t k = 0; k < p->P; ++k)
        for (int c = 0; c < 3; ++c) t[3 * k + c] = pts[3 * p->hs.pt_perm[k] + c];
    ba_status s;
    if ((s = vbi_fail(p, cudaStreamSynchronize(p->h->st), "sync"))) return s;
    if ((s = vbi_fail(p, cudaMemcpy(p->cams, cams, (size_t)p->n * 48, cudaMemcpyHostToDevice), "copy"))) return s;
    if ((s = vbi_fail(p, cudaMemcpy(p->intr, intr, (size_t)p->n * 40, cudaMemcpyHostToDevice), "copy"))) return s;
    if ((s = vbi_fail(p, cudaMemcpy(p->pts, t.data(), t.size() * 8, cudaMemcpyHostToDevice), "copy"))) return s;
    p->lambda = lambda;
    p->nu = nu;
    p->linearized = false;
    p->stepped = false;
    return BA_OK;
}

ba_status ba_vbi_get_lm_state(const ba_vbi_problem *p, double *lambda, double *nu, double *cost) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (p->dead) return set_error(BA_ERR_STATE, "the problem is unusable after an earlier error");
    if (lambda) *lambda = p->lambda;
    if (nu) *nu = p->nu;
    if (cost) {
        if (!p->linearized) {  // the cost of the current state
            ba_vbi_problem *q = const_cast<ba_vbi_problem *>(p);
            ba_status s;
            if ((s = vbi_fail(q, vbi_linearize(p->h, p->d, p->m, p->n, p->cams, p->intr, p->pts), "k_vbi_linearize")))
                return s;
            if ((s = vbi_fail(q, vbi_cost(p->h, p->d, p->m, p->sc, p->red, p->ctr), "k_vbi_cost"))) return s;
            if ((s = vbi_fail(q, cudaMemcpyAsync(p->sc_host, p->sc, sizeof(VbiScalars), cudaMemcpyDeviceToHost,
                                                 p->h->st), "copy")))
                return s;
            if ((s = vbi_fail(q, cudaStreamSynchronize(p->h->st), "sync"))) return s;
            q->F = p->sc_host->cost;
            q->linearized = true;
        }
        *cost = p->F;
    }
    return BA_OK;
}

ba_status ba_vbi_get_step(const ba_vbi_problem *p, double *dxc, double *dxp) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (p->dead) return set_error(BA_ERR_STATE, "the problem is unusable after an earlier error");
    if (!p->stepped) return set_error(BA_ERR_STATE, "no step taken since creation or the last ba_vbi_set_state");
    ba_vbi_problem *q = const_cast<ba_vbi_problem *>(p);
    ba_status s;
    if ((s = vbi_fail(q, cudaStreamSynchronize(p->h->st), "sync"))) return s;
    if (dxc) {
        std::vector<char> raw(p->h->N * p->h->esz);
        if ((s = vbi_fail(q, cudaMemcpy(raw.data(), p->h->vec[0], raw.size(), cudaMemcpyDeviceToHost), "copy")))
            return s;
        for (int64_t k = 0; k < p->h->N; ++k)
            dxc[k] = p->h->fp32 ? (double)reinterpret_cast<const float *>(raw.data())[k]
                                : reinterpret_cast<const double *>(raw.data())[k];
    }
    if (dxp) {
        std::vector<double> t(3 * p->P);
        if ((s = vbi_fail(q, cudaMemcpy(t.data(), p->dxp, t.size() * 8, cudaMemcpyDeviceToHost), "copy"))) return s;
        for (int64_t k = 0; k < p->P; ++k)
            for (int c = 0; c < 3; ++c) dxp[3 * p->hs.pt_perm[k] + c] = t[3 * k + c];
    }
    return BA_OK;
}

const ba_vbsmc *ba_vbi_system(const ba_vbi_problem *p) { return p ? p->h : nullptr; }

ba_status ba_vbi_info(const ba_vbi_problem *p, int64_t *n_unknowns, int64_t *n_blocks, int64_t *device_bytes) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    if (n_unknowns) *n_unknowns = p->h->N;
    if (n_blocks) *n_blocks = p->h->nnzb;
    if (device_bytes) *device_bytes = p->dev_bytes + (int64_t)p->h->dev_bytes;
    return BA_OK;
}

}  // extern "C"
