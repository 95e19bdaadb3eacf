// Per-observation kernels: state caches, linearization (residuals and
// Jacobians of Eq. 1), the cost F = 1/2 sum rho(||e||^2), the pose update and
// the trial evaluation (cost and model decrease for the LM gain ratio).
//
// Camera model: X_cam = R(omega) X + t, u = fx x/z + cx, v = fy y/z + cy,
// e = (u, v) - u_obs.  The pose is perturbed in the camera frame,
// X_cam <- Exp(d_omega) X_cam + dt, so dX_cam/d(d_omega) = -[X_cam]x,
// dX_cam/d(dt) = I and dX_cam/dX = R.
//
// FP32 mode keeps the state in FP64 and evaluates X_cam = R (X - C) with
// X and the camera centre C = -R^T t split into FP32 hi + lo parts, so the
// subtraction of two large world coordinates loses nothing before the FP32
// rotation.  The cost F (the LM's gain ratio compares F at two states) is
// evaluated in double-float arithmetic from the same parts and the rotation's
// lo parts, against the FP64 observations: near convergence an LM step
// changes F by less than FP32 residuals resolve (~1e-8 of F at 1M points),
// and the accept/reject decision must follow the step, not the rounding.
// Once accepted steps change F by less than 1e-3 of it, the trial cost is F
// plus its change formed in FP32 from the step itself and the state's
// residuals, which each state keeps from its last double-float evaluation
// (updated by accepted steps); the change is then accurate relative to
// itself.
#include "device_util.cuh"
#include "tma_util.cuh"

namespace ba {

struct Intr {
    double fx, fy, cx, cy;
};

// --------------------------------------------------------------------------
// state caches
// --------------------------------------------------------------------------
__global__ void k_prepare_cams64(int n, const double *__restrict__ cams, double *__restrict__ camc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double q[4], R[9];
    quat_exp(cams + 6 * i, q);
    quat_to_R(q, R);
#pragma unroll
    for (int k = 0; k < 9; ++k) camc[12 * i + k] = R[k];
#pragma unroll
    for (int k = 0; k < 3; ++k) camc[12 * i + 9 + k] = cams[6 * i + 3 + k];
}

// FP32 camera cache, CAMC32_W floats per camera:
// [R_hi (9), C_hi (3), C_lo (3), 0, R_lo (9), 0 (7)]
__global__ void k_prepare_cams32(int n, const double *__restrict__ cams, float *__restrict__ camc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double q[4], R[9];
    quat_exp(cams + 6 * i, q);
    quat_to_R(q, R);
    const double *t = cams + 6 * i + 3;
    float *o = camc + CAMC32_W * i;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float hi = (float)R[k];
        o[k] = hi;
        o[16 + k] = (float)(R[k] - (double)hi);
    }
#pragma unroll
    for (int k = 25; k < CAMC32_W; ++k) o[k] = 0.f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const double C = -(R[0 + d] * t[0] + R[3 + d] * t[1] + R[6 + d] * t[2]);
        const float hi = (float)C;
        o[9 + d] = hi;
        o[12 + d] = (float)(C - (double)hi);
    }
    o[15] = 0.f;
}

__global__ void k_split_pts(int64_t P, const double *__restrict__ pts, float *__restrict__ hl) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const double x = pts[3 * k + d];
            const float hi = (float)x;
            hl[6 * k + d] = hi;
            hl[6 * k + 3 + d] = (float)(x - (double)hi);
        }
    }
}

// X_cam of observation (camera i, point k) in the mode precision.
__device__ __forceinline__ void cam_point(const double *camc, const double *pts, const float *, int i, int k,
                                          double *Xc, double *R) {
    const double *c = camc + 12 * i;
    const double X0 = pts[3 * k], X1 = pts[3 * k + 1], X2 = pts[3 * k + 2];
#pragma unroll
    for (int r = 0; r < 9; ++r) R[r] = c[r];
#pragma unroll
    for (int r = 0; r < 3; ++r) Xc[r] = R[3 * r] * X0 + R[3 * r + 1] * X1 + R[3 * r + 2] * X2 + c[9 + r];
}
__device__ __forceinline__ void cam_point(const float *camc, const double *, const float *hl, int i, int k,
                                          float *Xc, float *R) {
    const float4 *c4 = reinterpret_cast<const float4 *>(camc + CAMC32_W * i);
    const float4 a = c4[0], b = c4[1], c = c4[2], d = c4[3];
    R[0] = a.x; R[1] = a.y; R[2] = a.z; R[3] = a.w; R[4] = b.x; R[5] = b.y; R[6] = b.z; R[7] = b.w; R[8] = c.x;
    const float Chi[3] = {c.y, c.z, c.w}, Clo[3] = {d.x, d.y, d.z};
    const float *h = hl + 6 * (int64_t)k;
    float D[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) D[r] = (h[r] - Chi[r]) + (h[3 + r] - Clo[r]);
#pragma unroll
    for (int r = 0; r < 3; ++r) Xc[r] = R[3 * r] * D[0] + R[3 * r + 1] * D[1] + R[3 * r + 2] * D[2];
}

template <typename T>
__device__ __forceinline__ T huber_rho(T s, int on, T delta) {
    if (!on || s <= delta * delta) return s;
    return T(2) * delta * sqrt(s) - delta * delta;
}

// ||e||^2 of observation a (camera i, point given by its hi + lo parts) in
// double-float arithmetic on the FP32 pipe: X - C, the rotation with
// R = R_hi + R_lo, the quotients, the intrinsics and e against the
// observation's hi + lo parts, each to ~2^-44 relative.  behind: z <= 1e-6.
struct IntrDF {
    float fxh, fxl, fyh, fyl, cxh, cxl, cyh, cyl;
};
// Knuth's TwoSum: s + e = a + b exactly
__device__ __forceinline__ df32 two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}
// sum_k (ah_k + al_k)(bh_k + bl_k) for k = 0..2: exact leading products and
// their sums, first-order cross terms
__device__ __forceinline__ df32 df_dot3(const float *ah, const float *al, const df32 *b) {
    float p[3], lo = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        p[k] = ah[k] * b[k].hi;
        lo += __fmaf_rn(ah[k], b[k].hi, -p[k]);
        lo = __fmaf_rn(ah[k], b[k].lo, __fmaf_rn(al[k], b[k].hi, lo));
    }
    const df32 s1 = two_sum(p[0], p[1]);
    const df32 s2 = two_sum(s1.hi, p[2]);
    return df_fast_norm(s2.hi, s2.lo + s1.lo + lo);
}
__device__ __forceinline__ df32 df_rcp(df32 b) {
    const float q1 = __frcp_rn(b.hi);
    float r = __fmaf_rn(-q1, b.hi, 1.0f);  // exact
    r = __fmaf_rn(-q1, b.lo, r);
    return df_fast_norm(q1, r * q1);
}
__device__ __forceinline__ df32 sq_resid_df(const float *__restrict__ camc, int i, const float *hl,
                                            const IntrDF &in, float uh, float ul, float vh, float vl, bool &behind,
                                            float &e0o, float &e1o) {
    const float4 *c4 = reinterpret_cast<const float4 *>(camc + CAMC32_W * i);
    const float4 c0 = c4[0], c1 = c4[1], c2 = c4[2], c3 = c4[3], c5 = c4[4], c6 = c4[5], c7 = c4[6];
    const float Rh[9] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x};
    const float Rl[9] = {c5.x, c5.y, c5.z, c5.w, c6.x, c6.y, c6.z, c6.w, c7.x};
    const float Ch[3] = {c2.y, c2.z, c2.w}, Cl[3] = {c3.x, c3.y, c3.z};
    df32 D[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        const df32 t = two_sum(hl[r], -Ch[r]);
        D[r] = df_fast_norm(t.hi, t.lo + (hl[3 + r] - Cl[r]));
    }
    const df32 X0 = df_dot3(Rh, Rl, D), X1 = df_dot3(Rh + 3, Rl + 3, D), X2 = df_dot3(Rh + 6, Rl + 6, D);
    behind = X2.hi <= 1e-6f;
    const df32 iz = df_rcp(X2);
    const df32 u = df_add(df_mul(df32{in.fxh, in.fxl}, df_mul(X0, iz)), df32{in.cxh, in.cxl});
    const df32 v = df_add(df_mul(df32{in.fyh, in.fyl}, df_mul(X1, iz)), df32{in.cyh, in.cyl});
    const df32 e0 = df_add(u, df32{-uh, -ul}), e1 = df_add(v, df32{-vh, -vl});
    e0o = e0.hi;
    e1o = e1.hi;
    // e0^2 + e1^2: exact squares of the leading parts, first-order cross terms
    const float p0 = e0.hi * e0.hi, p1 = e1.hi * e1.hi;
    const float l0 = __fmaf_rn(e0.hi, e0.hi, -p0) + 2.f * e0.hi * e0.lo;
    const float l1 = __fmaf_rn(e1.hi, e1.hi, -p1) + 2.f * e1.hi * e1.lo;
    const df32 s = two_sum(p0, p1);
    return df_fast_norm(s.hi, s.lo + l0 + l1);
}
// rho(s') - rho(s) from s and the change ds = s' - s formed exactly (FP32):
// the change is kept relative to itself where both lie on one branch.
__device__ __forceinline__ float rho_change(float s, float ds, int huber, float dl) {
    if (!huber) return ds;
    const float s1 = s + ds, d2 = dl * dl;
    if (s <= d2 && s1 <= d2) return ds;
    if (s > d2 && s1 > d2) return 2.f * dl * ds / (sqrtf(s1) + sqrtf(s));
    const float r0 = s <= d2 ? s : 2.f * dl * sqrtf(s) - d2;
    const float r1 = s1 <= d2 ? s1 : 2.f * dl * sqrtf(s1) - d2;
    return r1 - r0;
}

// The change de of the residual of observation (camera i, point) under the
// LM step, formed from the step itself: X_cam' = Exp(dw)(X_cam + R dX) + dt
// (the camera-frame update), so dX_cam = (Exp(dw) - I) v + R dX + dt with
// v = X_cam + R dX, and de = f (dx z - x dz) / (z (z + dz)).  FP32 gives de
// to ~1e-7 of itself, where two FP32 residual evaluations differ by ~1e-4 px
// of rounding.  behind: z' <= 1e-6.
__device__ __forceinline__ void resid_change(const float (&Xc)[3], const float (&R)[9], const float *dw6,
                                             const float *dp, const IntrDF &in, float &du, float &dv,
                                             bool &behind) {
    float RdX[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) RdX[r] = R[3 * r] * dp[0] + R[3 * r + 1] * dp[1] + R[3 * r + 2] * dp[2];
    const float w0 = dw6[0], w1 = dw6[1], w2 = dw6[2];
    const float v0 = Xc[0] + RdX[0], v1 = Xc[1] + RdX[1], v2 = Xc[2] + RdX[2];
    const float c0 = w1 * v2 - w2 * v1, c1 = w2 * v0 - w0 * v2, c2 = w0 * v1 - w1 * v0;
    const float d0 = w1 * c2 - w2 * c1, d1 = w2 * c0 - w0 * c2, d2 = w0 * c1 - w1 * c0;
    const float th2 = w0 * w0 + w1 * w1 + w2 * w2;
    float a, b;
    if (th2 < 1e-8f) {
        a = 1.f - th2 * (1.f / 6.f);
        b = 0.5f - th2 * (1.f / 24.f);
    } else {
        const float th = sqrtf(th2), sh = sinf(0.5f * th);
        a = sinf(th) / th;
        b = 2.f * sh * sh / th2;
    }
    const float dX = a * c0 + b * d0 + RdX[0] + dw6[3];
    const float dY = a * c1 + b * d1 + RdX[1] + dw6[4];
    const float dZ = a * c2 + b * d2 + RdX[2] + dw6[5];
    const float z1 = Xc[2] + dZ;
    behind = z1 <= 1e-6f;
    const float q = 1.f / (Xc[2] * z1);
    du = in.fxh * (dX * Xc[2] - Xc[0] * dZ) * q;
    dv = in.fyh * (dY * Xc[2] - Xc[1] * dZ) * q;
}

// An FP64 sum of rho(||e||^2) over double-float values of ||e||^2: the
// leading parts are added in FP64, the trailing parts (below the leading
// part's last bit, so their FP32 sum is exact to ~2^-24 of a quantity already
// 2^-24 of the total) in FP32 beside it; Huber's bent branch in FP64.
struct RhoSum {
    double s = 0.0;
    float lo = 0.f;
    __device__ __forceinline__ void add(df32 q, int huber, double delta) {
        if (huber && q.hi > (float)(delta * delta)) {
            s += huber_rho<double>((double)q.hi + (double)q.lo, 1, delta);
        } else {
            s += (double)q.hi;
            lo += q.lo;
        }
    }
    __device__ __forceinline__ double get() const { return s + (double)lo; }
};

// --------------------------------------------------------------------------
// K1: residuals and Jacobians, one thread per observation
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_linearize(int64_t m, const int *__restrict__ obs_cam, const int *__restrict__ obs_pt,
                                                   const T *__restrict__ uv, const T *__restrict__ camc,
                                                   const double *__restrict__ pts, const float *__restrict__ pts_hl,
                                                   Intr in, int huber, double delta, T *__restrict__ J) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const int i = obs_cam[a], k = obs_pt[a];
        T Xc[3], R[9];
        cam_point(camc, pts, pts_hl, i, k, Xc, R);
        const T iz = T(1) / Xc[2];
        const T xh = Xc[0] * iz, yh = Xc[1] * iz;
        T e0 = T(in.fx) * xh + T(in.cx) - uv[2 * a];
        T e1 = T(in.fy) * yh + T(in.cy) - uv[2 * a + 1];
        // dpi/dX_cam = [[a0, 0, a2], [0, a1, a3]]
        const T a0 = T(in.fx) * iz, a2 = -T(in.fx) * xh * iz;
        const T a1 = T(in.fy) * iz, a3 = -T(in.fy) * yh * iz;
        T o[JW];
        // rotation columns: dpi/dX_cam * (-[X_cam]x)
        o[0] = a2 * Xc[1];
        o[1] = a0 * Xc[2] - a2 * Xc[0];
        o[2] = -a0 * Xc[1];
        o[6] = -a1 * Xc[2] + a3 * Xc[1];
        o[7] = -a3 * Xc[0];
        o[8] = a1 * Xc[0];
        // translation columns: dpi/dX_cam
        o[3] = a0; o[4] = T(0); o[5] = a2;
        o[9] = T(0); o[10] = a1; o[11] = a3;
        // point columns: dpi/dX_cam * R
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            o[12 + c] = a0 * R[c] + a2 * R[6 + c];
            o[15 + c] = a1 * R[3 + c] + a3 * R[6 + c];
        }
        if (huber) {
            const T s = e0 * e0 + e1 * e1, dl = (T)delta;
            if (s > dl * dl) {
                const T sw = sqrt(dl / sqrt(s));
#pragma unroll
                for (int q = 0; q < 18; ++q) o[q] *= sw;
                e0 *= sw;
                e1 *= sw;
            }
        }
        o[18] = e0;
        o[19] = e1;
        T *dst = J + a * JW;
        if constexpr (sizeof(T) == 4) {
            float4 *d4 = reinterpret_cast<float4 *>(dst);
#pragma unroll
            for (int q = 0; q < 5; ++q) d4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
        } else {
            double2 *d2 = reinterpret_cast<double2 *>(dst);
#pragma unroll
            for (int q = 0; q < 10; ++q) d2[q] = make_double2(o[2 * q], o[2 * q + 1]);
        }
    }
}

// --------------------------------------------------------------------------
// F = 1/2 sum rho(||e||^2) (FP64 sum) and the cheirality count
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_cost(int64_t m, const int *__restrict__ obs_cam, const int *__restrict__ obs_pt,
                                              const T *__restrict__ uv, const T *__restrict__ camc,
                                              const double *__restrict__ pts, const float *__restrict__ pts_hl,
                                              Intr in, int huber, double delta, DevScalars *sc, int trial,
                                              double *red, unsigned *ctr, const float *__restrict__ uv_lo, IntrDF idf,
                                              float *__restrict__ e_out) {
    RunSum<double> f;  // FP64 accumulation (FP64 terms; double-float residuals in FP32 mode)
    RhoSum fdf;
    int ncheir = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(T) == 4) {
        // two observations per pass, their double-float chains independent
        for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += 2 * stride) {
            const bool two = a + stride < m;
            const int64_t b = two ? a + stride : a;
            const int ia = obs_cam[a], ka = obs_pt[a], ib = obs_cam[b], kb = obs_pt[b];
            bool behind_a, behind_b;
            float ea0, ea1, eb0, eb1;
            const df32 sa = sq_resid_df(camc, ia, pts_hl + 6 * (int64_t)ka, idf, uv[2 * a], uv_lo[2 * a],
                                        uv[2 * a + 1], uv_lo[2 * a + 1], behind_a, ea0, ea1);
            const df32 sb = sq_resid_df(camc, ib, pts_hl + 6 * (int64_t)kb, idf, uv[2 * b], uv_lo[2 * b],
                                        uv[2 * b + 1], uv_lo[2 * b + 1], behind_b, eb0, eb1);
            fdf.add(sa, huber, delta);
            ncheir += behind_a ? 1 : 0;
            e_out[2 * a] = ea0;
            e_out[2 * a + 1] = ea1;
            if (two) {
                fdf.add(sb, huber, delta);
                ncheir += behind_b ? 1 : 0;
                e_out[2 * b] = eb0;
                e_out[2 * b + 1] = eb1;
            }
        }
    }
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; sizeof(T) == 8 && a < m; a += stride) {
        const int i = obs_cam[a], k = obs_pt[a];
        {
            T Xc[3], R[9];
            cam_point(camc, pts, pts_hl, i, k, Xc, R);
            const T iz = T(1) / Xc[2];
            const T e0 = T(in.fx) * (Xc[0] * iz) + T(in.cx) - uv[2 * a];
            const T e1 = T(in.fy) * (Xc[1] * iz) + T(in.cy) - uv[2 * a + 1];
            f.add((double)huber_rho<T>(e0 * e0 + e1 * e1, huber, (T)delta));
            ncheir += (Xc[2] <= T(1e-6)) ? 1 : 0;
        }
    }
    double v[2] = {f.get() + fdf.get(), (double)ncheir};
    grid_sum<2>(v, red, ctr, [&](double *t) {
        if (trial) {
            sc->cost_trial = 0.5 * t[0];
            sc->n_cheir_trial = (unsigned long long)t[1];
        } else {
            sc->cost = 0.5 * t[0];
            sc->n_cheir = (unsigned long long)t[1];
        }
    });
}

// --------------------------------------------------------------------------
// trial point: R <- Exp(dw) R, t <- Exp(dw) t + dt, X <- X + dX
// --------------------------------------------------------------------------
template <typename T>
__global__ void k_update_cams(int n, const double *__restrict__ cams, const T *__restrict__ dxc, double *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double w[3], q[4], qd[4], qn[4], Rd[9];
    const double dw[3] = {(double)dxc[6 * i], (double)dxc[6 * i + 1], (double)dxc[6 * i + 2]};
    quat_exp(cams + 6 * i, q);
    quat_exp(dw, qd);
    quat_mul(qd, q, qn);
    const double nn = rsqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
#pragma unroll
    for (int k = 0; k < 4; ++k) qn[k] *= nn;
    quat_log(qn, w);
    quat_to_R(qd, Rd);
    const double *t = cams + 6 * i + 3;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        out[6 * i + r] = w[r];
        out[6 * i + 3 + r] = Rd[3 * r] * t[0] + Rd[3 * r + 1] * t[1] + Rd[3 * r + 2] * t[2] + (double)dxc[6 * i + 3 + r];
    }
}


// One staged observation row (JW values, 16-byte aligned) from shared memory.
__device__ __forceinline__ void load_jrow_s(const float *s, float (&v)[JW]) {
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 4; ++q) {
        const float4 t = s4[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}
__device__ __forceinline__ void load_jrow_s(const double *s, double (&v)[JW]) {
    const double2 *s2 = reinterpret_cast<const double2 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 2; ++q) {
        const double2 t = s2[q];
        v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
}

// X_cam of camera i and a point given by value (FP64; FP32 as hi + lo parts).
__device__ __forceinline__ void cam_point_v(const double *camc, int i, const double *X, const float *, double *Xc) {
    const double *c = camc + 12 * i;
#pragma unroll
    for (int r = 0; r < 3; ++r) Xc[r] = c[3 * r] * X[0] + c[3 * r + 1] * X[1] + c[3 * r + 2] * X[2] + c[9 + r];
}
__device__ __forceinline__ void cam_point_v(const float *camc, int i, const double *, const float *hl, float *Xc) {
    const float4 *c4 = reinterpret_cast<const float4 *>(camc + CAMC32_W * i);
    const float4 a = c4[0], b = c4[1], c = c4[2], d = c4[3];
    const float R[9] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x};
    const float Chi[3] = {c.y, c.z, c.w}, Clo[3] = {d.x, d.y, d.z};
    float D[3];
#pragma unroll
    for (int r = 0; r < 3; ++r) D[r] = (hl[r] - Chi[r]) + (hl[3 + r] - Clo[r]);
#pragma unroll
    for (int r = 0; r < 3; ++r) Xc[r] = R[3 * r] * D[0] + R[3 * r + 1] * D[1] + R[3 * r + 2] * D[2];
}

// The LM step's point pass: the back-substitution of Eq. 5
// (dx_p = V^-1 (l_p - sum_a J_p,a^T J_c,a dx_c), V^-1 = L^-T L^-1), the trial
// point x_p + dx_p (FP64, and its FP32 hi + lo split), and for every
// observation the trial cost F(x (+) dx) and the model decrease
// -1/2 sum_a (J_a dx)^T (2 e_a + J_a dx) (weighted e, J under Huber), summed
// in FP64.  It runs over the RCS formation's point groups (whole tracks,
// <= obs_max observations, contiguous rows): a persistent CTA copies a
// group's rows into shared memory with one bulk copy (one buffer, so that
// three CTAs fit on an SM), a thread per observation forms J_c dx_c and
// J_p^T J_c dx_c, a thread per point solves Eq. 5 from shared
// memory and keeps dx_p and the trial point there, then a thread per
// observation evaluates it from shared memory.  The stored linearization is
// read from DRAM once, in whole contiguous ranges, at any problem size (a
// thread per point re-reading its rows from cache, and a warp-cooperative
// variant over batches of points, both measured slower).  The trial cameras
// (cache included) are formed before.
constexpr int STEP_THREADS = 256;
constexpr int STEP_OBS_PER_THREAD = (OBS_MAX_LIMIT + STEP_THREADS - 1) / STEP_THREADS;

template <typename T>
__global__ void __launch_bounds__(STEP_THREADS, sizeof(T) == 4 ? 3 : 1) k_step_groups(const GroupDesc *__restrict__ grp, int ngroups,
                                                     const int *__restrict__ trk_ptr, const int *__restrict__ obs_cam,
                                                     const int *__restrict__ obs_pt, const T *__restrict__ uv,
                                                     const T *__restrict__ J, const T *__restrict__ dxc,
                                                     const T *__restrict__ Linv, const T *__restrict__ lp,
                                                     const double *__restrict__ pts, const T *__restrict__ camc_trial,
                                                     Intr in, int huber, double delta, T *__restrict__ dxp,
                                                     double *__restrict__ pts_trial, float *__restrict__ hl_trial,
                                                     DevScalars *sc, double *red, unsigned *ctr, int obs_max,
                                                     long long limit, const float *__restrict__ uv_lo, IntrDF idf,
                                                     const float *__restrict__ camc_cur,
                                                     const float *__restrict__ hl_cur, int diff,
                                                     const float *__restrict__ e_cur, float *__restrict__ e_trial) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ GroupDesc sdesc;
    __shared__ int s_ok;
    // one row buffer (more CTAs per SM rather than a second buffer); per point
    // of the current group dx_p (3 T), its trial split (6 float) and, FP64
    // only, the trial point (3 double); per observation J_p^T J_c dx_c (3 T),
    // J_c dx_c (2 T) and the camera.  Each thread keeps J_p and e of its own
    // observations (at most STEP_OBS_PER_THREAD) in registers from the first
    // pass to the trial evaluation, so the row buffer is free for the next
    // group's copy after the first pass.
    const size_t buf_bytes = (size_t)obs_max * JW * sizeof(T);
    const size_t np = (size_t)obs_max / 2;
    unsigned char *aux = smem_raw + buf_bytes;
    T *s_dp = reinterpret_cast<T *>(aux);
    float *s_hl = reinterpret_cast<float *>(s_dp + np * 3);
    double *s_xt = reinterpret_cast<double *>(aux + np * (3 * sizeof(T) + 6 * sizeof(float)));
    T *s_c3 = reinterpret_cast<T *>(reinterpret_cast<unsigned char *>(s_xt) + (sizeof(T) == 8 ? np * 24 : 0));
    T *s_jc = s_c3 + (size_t)obs_max * 3;
    int *s_cam = reinterpret_cast<int *>(s_jc + (size_t)obs_max * 2);
    int *s_pl = s_cam + obs_max;                                   // each observation's point in the group
    float *s_hlc = reinterpret_cast<float *>(s_pl + obs_max);     // FP32: each point's current X (hi, lo)
    if (threadIdx.x == 0) {
        mbar_init(&mbar, 1);
        fence_proxy_async();
    }
    __syncthreads();
    auto issue = [&](int gi) {
        const GroupDesc d = grp[gi];
        sdesc = d;
        const uint32_t jb = (uint32_t)d.nobs * JW * (uint32_t)sizeof(T);
        fence_proxy_async();
        mbar_expect_tx(&mbar, jb);
        bulk_g2s(smem_raw, J + (int64_t)d.obs_begin * JW, jb, &mbar);
    };
    RunSum<double> f, mdl;  // FP64 accumulation of the gain ratio's sums (terms formed in T)
    RhoSum fdf;
    int ncheir = 0;
    const T dl = (T)delta;
    uint32_t parity = 0u;
    int gi = blockIdx.x;
    if (threadIdx.x == 0 && gi < ngroups) issue(gi);
    for (; gi < ngroups; gi += gridDim.x) {
        if (threadIdx.x == 0) s_ok = mbar_wait(&mbar, parity, limit) ? 1 : 0;
        __syncthreads();
        if (!s_ok) {
            // give up: flag it, let the copy still in flight land (bounded), leave
            if (threadIdx.x == 0) {
                atomicExch(&sc->err, (int)BA_ERR_TIMEOUT);
                mbar_wait(&mbar, parity, limit);
            }
            return;
        }
        parity ^= 1u;
        const GroupDesc g = sdesc;
        const T *so = reinterpret_cast<const T *>(smem_raw);
        // per observation: J_c dx_c and its image J_p^T J_c dx_c under J_p
        T pe[STEP_OBS_PER_THREAD][8];
#pragma unroll
        for (int k = 0; k < STEP_OBS_PER_THREAD; ++k) {
            const int al = threadIdx.x + k * STEP_THREADS;
            if (al >= g.nobs) break;
            const int i = __ldg(obs_cam + g.obs_begin + al);
            s_pl[al] = __ldg(obs_pt + g.obs_begin + al) - g.pt_begin;
            const T *dc = dxc + 6 * i;
            T j[JW];
            load_jrow_s(so + al * JW, j);
            T t0 = T(0), t1 = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) { t0 += j[c] * dc[c]; t1 += j[6 + c] * dc[c]; }
#pragma unroll
            for (int d = 0; d < 3; ++d) s_c3[3 * al + d] = j[12 + d] * t0 + j[15 + d] * t1;
            s_jc[2 * al] = t0;
            s_jc[2 * al + 1] = t1;
            s_cam[al] = i;
#pragma unroll
            for (int q = 0; q < 8; ++q) pe[k][q] = j[12 + q];
        }
        __syncthreads();
        // the rows are no longer read: the next group's copy overlaps the rest
        const int gn = gi + gridDim.x;
        if (threadIdx.x == 0 && gn < ngroups) issue(gn);
        // Eq. 5 per point: dx_p = L^-T L^-1 (l_p - sum over the track)
        for (int pl = threadIdx.x; pl < g.npts; pl += blockDim.x) {
            const int64_t kp = (int64_t)g.pt_begin + pl;
            const int a0 = __ldg(trk_ptr + kp) - g.obs_begin, a1 = __ldg(trk_ptr + kp + 1) - g.obs_begin;
            T s0 = lp[3 * kp], s1 = lp[3 * kp + 1], s2 = lp[3 * kp + 2];
            for (int a = a0; a < a1; ++a) {
                s0 -= s_c3[3 * a];
                s1 -= s_c3[3 * a + 1];
                s2 -= s_c3[3 * a + 2];
            }
            const T *mL = Linv + 6 * kp;  // m00 m10 m11 m20 m21 m22
            const T u0 = mL[0] * s0, u1 = mL[1] * s0 + mL[2] * s1, u2 = mL[3] * s0 + mL[4] * s1 + mL[5] * s2;
            const T dp[3] = {mL[0] * u0 + mL[1] * u1 + mL[3] * u2, mL[2] * u1 + mL[4] * u2, mL[5] * u2};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const double x = pts[3 * kp + d] + (double)dp[d];
                const float h = (float)x, l = (float)(x - (double)h);
                dxp[3 * kp + d] = dp[d];
                pts_trial[3 * kp + d] = x;
                if (hl_trial) {
                    hl_trial[6 * kp + d] = h;
                    hl_trial[6 * kp + 3 + d] = l;
                }
                s_dp[3 * pl + d] = dp[d];
                if (sizeof(T) == 8) s_xt[3 * pl + d] = x;
                if (sizeof(T) == 4 && diff) {
                    s_hlc[6 * pl + d] = hl_cur[6 * kp + d];
                    s_hlc[6 * pl + 3 + d] = hl_cur[6 * kp + 3 + d];
                }
                s_hl[6 * pl + d] = h;
                s_hl[6 * pl + 3 + d] = l;
            }
        }
        __syncthreads();
        // the trial cost and the model decrease, one thread per observation
#pragma unroll
        for (int k = 0; k < STEP_OBS_PER_THREAD; ++k) {
            const int al = threadIdx.x + k * STEP_THREADS;
            if (al >= g.nobs) break;
            const int64_t a = (int64_t)g.obs_begin + al;
            const int i = s_cam[al], pl = s_pl[al];
            if constexpr (sizeof(T) == 4) {
                bool behind;
                if (diff) {
                    // the change of rho from the step and the state's residual
                    float Xc[3], R[9], du, dv;
                    cam_point(camc_cur, nullptr, s_hlc, i, pl, Xc, R);
                    resid_change(Xc, R, dxc + 6 * i, s_dp + 3 * pl, idf, du, dv, behind);
                    const float e0 = e_cur[2 * a], e1 = e_cur[2 * a + 1];
                    const float ds = du * (2.f * e0 + du) + dv * (2.f * e1 + dv);
                    f.add((double)rho_change(e0 * e0 + e1 * e1, ds, huber, dl));
                    e_trial[2 * a] = e0 + du;
                    e_trial[2 * a + 1] = e1 + dv;
                } else {
                    float e0, e1;
                    const df32 s = sq_resid_df(camc_trial, i, s_hl + 6 * pl, idf, uv[2 * a], uv_lo[2 * a],
                                               uv[2 * a + 1], uv_lo[2 * a + 1], behind, e0, e1);
                    fdf.add(s, huber, delta);
                    e_trial[2 * a] = e0;
                    e_trial[2 * a + 1] = e1;
                }
                ncheir += behind ? 1 : 0;
            } else {
                T Xc[3];
                cam_point_v(camc_trial, i, s_xt + 3 * pl, s_hl + 6 * pl, Xc);
                const T iz = T(1) / Xc[2];
                const T e0 = T(in.fx) * (Xc[0] * iz) + T(in.cx) - uv[2 * a];
                const T e1 = T(in.fy) * (Xc[1] * iz) + T(in.cy) - uv[2 * a + 1];
                f.add((double)huber_rho<T>(e0 * e0 + e1 * e1, huber, dl));
                ncheir += (Xc[2] <= T(1e-6)) ? 1 : 0;
            }
            const T *jr = pe[k];  // J_p (2 x 3), e
            T jd0 = s_jc[2 * al], jd1 = s_jc[2 * al + 1];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                jd0 += jr[c] * s_dp[3 * pl + c];
                jd1 += jr[3 + c] * s_dp[3 * pl + c];
            }
            mdl.add(-(double)(jd0 * (T(2) * jr[6] + jd0) + jd1 * (T(2) * jr[7] + jd1)));
        }
        // the per-point and per-observation areas are rewritten only after the
        // barrier that follows the next group's copy wait
    }
    double v[3] = {f.get() + fdf.get(), mdl.get(), (double)ncheir};
    grid_sum<3>(v, red, ctr, [&](double *t) {
        sc->cost_trial = 0.5 * t[0];
        sc->model = 0.5 * t[1];
        sc->n_cheir_trial = (unsigned long long)t[2];
    });
}

// Triangulation of the points from the camera poses, the alternative the
// paper gives to the back-substitution of Eq. 5 (Sec. 3.1; Sec. 5): a thread
// per point, in FP64.  Each observation gives two equations linear in the
// point X (the pinhole model with the depth multiplied out):
//   ((u - cx) R_3 - fx R_1) . X = fx t_1 - (u - cx) t_3,
//   ((v - cy) R_3 - fy R_2) . X = fy t_2 - (v - cy) t_3;
// their normal equations are solved by a 3x3 Cholesky factorisation, then
// gn_iters Gauss-Newton steps (J_p^T J_p) dX = -J_p^T e refine X on the
// reprojection error.  A point whose 3x3 matrix is not positive definite, or
// whose result is not finite, keeps its value and is counted.
__device__ __forceinline__ bool chol3_solve(const double (&N)[6], const double (&h)[3], double (&x)[3]) {
    // N = [n00 n01 n02; . n11 n12; . . n22] packed as (00, 01, 02, 11, 12, 22)
    if (!(N[0] > 0.0)) return false;
    const double l00 = sqrt(N[0]), l10 = N[1] / l00, l20 = N[2] / l00;
    const double d1 = N[3] - l10 * l10;
    if (!(d1 > 0.0)) return false;
    const double l11 = sqrt(d1), l21 = (N[4] - l20 * l10) / l11;
    const double d2 = N[5] - l20 * l20 - l21 * l21;
    if (!(d2 > 0.0)) return false;
    const double l22 = sqrt(d2);
    const double y0 = h[0] / l00, y1 = (h[1] - l10 * y0) / l11, y2 = (h[2] - l20 * y0 - l21 * y1) / l22;
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    return true;
}
__device__ __forceinline__ void sym3_add(double (&N)[6], double (&h)[3], const double (&a)[3], double r) {
    N[0] += a[0] * a[0]; N[1] += a[0] * a[1]; N[2] += a[0] * a[2];
    N[3] += a[1] * a[1]; N[4] += a[1] * a[2]; N[5] += a[2] * a[2];
    h[0] += a[0] * r; h[1] += a[1] * r; h[2] += a[2] * r;
}
__global__ void __launch_bounds__(256) k_triangulate(int64_t P, const int *__restrict__ trk_ptr,
                                                     const int *__restrict__ obs_cam, const double *__restrict__ uv,
                                                     const double *__restrict__ cam64, Intr in, int gn_iters,
                                                     double *__restrict__ pts, unsigned long long *nfail) {
    unsigned long long bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        const int a0 = __ldg(trk_ptr + k), a1 = __ldg(trk_ptr + k + 1);
        double N[6] = {0, 0, 0, 0, 0, 0}, h[3] = {0, 0, 0}, X[3];
        for (int a = a0; a < a1; ++a) {
            const double *c = cam64 + 12 * (int64_t)__ldg(obs_cam + a);
            const double du = uv[2 * (int64_t)a] - in.cx, dv = uv[2 * (int64_t)a + 1] - in.cy;
            const double r0[3] = {du * c[6] - in.fx * c[0], du * c[7] - in.fx * c[1], du * c[8] - in.fx * c[2]};
            const double r1[3] = {dv * c[6] - in.fy * c[3], dv * c[7] - in.fy * c[4], dv * c[8] - in.fy * c[5]};
            sym3_add(N, h, r0, in.fx * c[9] - du * c[11]);
            sym3_add(N, h, r1, in.fy * c[10] - dv * c[11]);
        }
        bool ok = chol3_solve(N, h, X);
        for (int it = 0; ok && it < gn_iters; ++it) {
            double M[6] = {0, 0, 0, 0, 0, 0}, g[3] = {0, 0, 0}, dX[3];
            for (int a = a0; a < a1; ++a) {
                const double *c = cam64 + 12 * (int64_t)__ldg(obs_cam + a);
                const double x = c[0] * X[0] + c[1] * X[1] + c[2] * X[2] + c[9];
                const double y = c[3] * X[0] + c[4] * X[1] + c[5] * X[2] + c[10];
                const double z = c[6] * X[0] + c[7] * X[1] + c[8] * X[2] + c[11];
                const double iz = 1.0 / z;
                const double e0 = in.fx * x * iz + in.cx - uv[2 * (int64_t)a];
                const double e1 = in.fy * y * iz + in.cy - uv[2 * (int64_t)a + 1];
                // J_p = d(pi)/d(X_cam) R: rows fx/z (R_1 - x/z R_3), fy/z (R_2 - y/z R_3)
                const double j0[3] = {in.fx * iz * (c[0] - x * iz * c[6]), in.fx * iz * (c[1] - x * iz * c[7]),
                                      in.fx * iz * (c[2] - x * iz * c[8])};
                const double j1[3] = {in.fy * iz * (c[3] - y * iz * c[6]), in.fy * iz * (c[4] - y * iz * c[7]),
                                      in.fy * iz * (c[5] - y * iz * c[8])};
                sym3_add(M, g, j0, -e0);
                sym3_add(M, g, j1, -e1);
            }
            ok = chol3_solve(M, g, dX);
            if (ok) {
                X[0] += dX[0];
                X[1] += dX[1];
                X[2] += dX[2];
            }
        }
        ok = ok && isfinite(X[0]) && isfinite(X[1]) && isfinite(X[2]);
        if (ok) {
            pts[3 * k] = X[0];
            pts[3 * k + 1] = X[1];
            pts[3 * k + 2] = X[2];
        } else {
            ++bad;
        }
    }
    if (bad) atomicAdd(nfail, bad);
}

// The same for FP32 problems on the FP32 pipe, centred on each point's
// current value X0: with X = X0 + d, observation a's equations read
//   ((u - cx) R_3 - fx R_1) . d = fx x0 - (u - cx) z0   (and likewise for v),
// (x0, y0, z0) = R X0 + t formed from the FP32 camera and point caches as
// R ((X0_hi - C_hi) + (X0_lo - C_lo)), exact to the camera-point distance
// rather than the world offset; Gauss-Newton on d; X = X0 + d in FP64.
__device__ __forceinline__ bool chol3_solve(const float (&N)[6], const float (&h)[3], float (&x)[3]) {
    if (!(N[0] > 0.f)) return false;
    const float l00 = sqrtf(N[0]), l10 = N[1] / l00, l20 = N[2] / l00;
    const float d1 = N[3] - l10 * l10;
    if (!(d1 > 0.f)) return false;
    const float l11 = sqrtf(d1), l21 = (N[4] - l20 * l10) / l11;
    const float d2 = N[5] - l20 * l20 - l21 * l21;
    if (!(d2 > 0.f)) return false;
    const float l22 = sqrtf(d2);
    const float y0 = h[0] / l00, y1 = (h[1] - l10 * y0) / l11, y2 = (h[2] - l20 * y0 - l21 * y1) / l22;
    x[2] = y2 / l22;
    x[1] = (y1 - l21 * x[2]) / l11;
    x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
    return true;
}
__device__ __forceinline__ void sym3_add(float (&N)[6], float (&h)[3], const float (&a)[3], float r) {
    N[0] += a[0] * a[0]; N[1] += a[0] * a[1]; N[2] += a[0] * a[2];
    N[3] += a[1] * a[1]; N[4] += a[1] * a[2]; N[5] += a[2] * a[2];
    h[0] += a[0] * r; h[1] += a[1] * r; h[2] += a[2] * r;
}
__global__ void __launch_bounds__(256) k_triangulate32(int64_t P, const int *__restrict__ trk_ptr,
                                                       const int *__restrict__ obs_cam, const float *__restrict__ uv,
                                                       const float *__restrict__ camc, const float *__restrict__ hl,
                                                       Intr in, int gn_iters, double *__restrict__ pts,
                                                       unsigned long long *nfail) {
    const float fx = (float)in.fx, fy = (float)in.fy, cx = (float)in.cx, cy = (float)in.cy;
    unsigned long long bad = 0;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        const int a0 = __ldg(trk_ptr + k), a1 = __ldg(trk_ptr + k + 1);
        float N[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f}, d[3];
        for (int a = a0; a < a1; ++a) {
            float Xc[3], R[9];
            cam_point(camc, nullptr, hl, __ldg(obs_cam + a), (int)k, Xc, R);
            const float du = uv[2 * (int64_t)a] - cx, dv = uv[2 * (int64_t)a + 1] - cy;
            const float r0[3] = {du * R[6] - fx * R[0], du * R[7] - fx * R[1], du * R[8] - fx * R[2]};
            const float r1[3] = {dv * R[6] - fy * R[3], dv * R[7] - fy * R[4], dv * R[8] - fy * R[5]};
            sym3_add(N, h, r0, fx * Xc[0] - du * Xc[2]);
            sym3_add(N, h, r1, fy * Xc[1] - dv * Xc[2]);
        }
        bool ok = chol3_solve(N, h, d);
        for (int it = 0; ok && it < gn_iters; ++it) {
            float M[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, g[3] = {0.f, 0.f, 0.f}, dd[3];
            for (int a = a0; a < a1; ++a) {
                float Xc[3], R[9];
                cam_point(camc, nullptr, hl, __ldg(obs_cam + a), (int)k, Xc, R);
                const float x = Xc[0] + R[0] * d[0] + R[1] * d[1] + R[2] * d[2];
                const float y = Xc[1] + R[3] * d[0] + R[4] * d[1] + R[5] * d[2];
                const float z = Xc[2] + R[6] * d[0] + R[7] * d[1] + R[8] * d[2];
                const float iz = 1.f / z;
                const float e0 = fx * x * iz + cx - uv[2 * (int64_t)a];
                const float e1 = fy * y * iz + cy - uv[2 * (int64_t)a + 1];
                const float j0[3] = {fx * iz * (R[0] - x * iz * R[6]), fx * iz * (R[1] - x * iz * R[7]),
                                     fx * iz * (R[2] - x * iz * R[8])};
                const float j1[3] = {fy * iz * (R[3] - y * iz * R[6]), fy * iz * (R[4] - y * iz * R[7]),
                                     fy * iz * (R[5] - y * iz * R[8])};
                sym3_add(M, g, j0, -e0);
                sym3_add(M, g, j1, -e1);
            }
            ok = chol3_solve(M, g, dd);
            if (ok) {
                d[0] += dd[0];
                d[1] += dd[1];
                d[2] += dd[2];
            }
        }
        ok = ok && isfinite(d[0]) && isfinite(d[1]) && isfinite(d[2]);
        if (ok) {
            pts[3 * k] += (double)d[0];
            pts[3 * k + 1] += (double)d[1];
            pts[3 * k + 2] += (double)d[2];
        } else {
            ++bad;
        }
    }
    if (bad) atomicAdd(nfail, bad);
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
static inline int grid_for(int64_t work, int threads, int cap) {
    int64_t g = (work + threads - 1) / threads;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (int)g;
}
static constexpr int GRID_CAP = 152 * 8;  // 152 SMs x 8 resident 256-thread CTAs

static Intr intr_of(const ba_problem *p) { return Intr{p->opt.fx, p->opt.fy, p->opt.cx, p->opt.cy}; }
static IntrDF intrdf_of(const ba_problem *p) {
    auto hi = [](double x) { return (float)x; };
    auto lo = [](double x) { return (float)(x - (double)(float)x); };
    return IntrDF{hi(p->opt.fx), lo(p->opt.fx), hi(p->opt.fy), lo(p->opt.fy),
                  hi(p->opt.cx), lo(p->opt.cx), hi(p->opt.cy), lo(p->opt.cy)};
}

// Points between the caller's order and the internal (Morton) one:
// internal point k is the caller's point perm[k].
__global__ void k_count_nonfinite(int64_t cnt, const double *__restrict__ a, unsigned *bad) {
    unsigned local = 0;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x)
        local |= isfinite(a[x]) ? 0u : 1u;
    if (__any_sync(0xffffffffu, local) && (threadIdx.x & 31) == 0) atomicOr(bad, 1u);
}
__global__ void k_gather_pts(int64_t P, const int32_t *__restrict__ perm, const double *__restrict__ user,
                             double *__restrict__ internal) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = __ldg(perm + k);
#pragma unroll
        for (int d = 0; d < 3; ++d) internal[3 * k + d] = user[3 * u + d];
    }
}
template <typename T>
__global__ void k_scatter_pts(int64_t P, const int32_t *__restrict__ perm, const T *__restrict__ internal,
                              double *__restrict__ user) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = __ldg(perm + k);
#pragma unroll
        for (int d = 0; d < 3; ++d) user[3 * u + d] = (double)internal[3 * k + d];
    }
}

cudaError_t launch_count_nonfinite(ba_problem *p, const double *a, int64_t cnt, unsigned *bad) {
    k_count_nonfinite<<<grid_for(cnt, 256, GRID_CAP), 256, 0, p->st>>>(cnt, a, bad);
    p->launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_gather_pts(ba_problem *p, const double *user, double *internal) {
    k_gather_pts<<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(p->P, p->d_perm, user, internal);
    p->launches += 1;
    return cudaGetLastError();
}
cudaError_t launch_scatter_pts(ba_problem *p, const void *internal, bool internal_fp32, double *user) {
    if (internal_fp32)
        k_scatter_pts<float><<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(p->P, p->d_perm,
                                                                              (const float *)internal, user);
    else
        k_scatter_pts<double><<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(p->P, p->d_perm,
                                                                               (const double *)internal, user);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_prepare_state(ba_problem *p, StateBuf &s) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PREPARE, &ev);
    const int nb = (p->n + 127) / 128;
    if (p->fp32) {
        k_prepare_cams32<<<nb, 128, 0, p->st>>>(p->n, s.cams, (float *)s.camc);
        k_split_pts<<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(p->P, s.pts, s.pts_hl);
    } else {
        k_prepare_cams64<<<nb, 128, 0, p->st>>>(p->n, s.cams, (double *)s.camc);
    }
    ktimer_end(p, K_PREPARE, ev);
    p->launches += p->fp32 ? 2 : 1;
    return cudaGetLastError();
}

cudaError_t launch_linearize(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_LINEARIZE, &ev);
    const int g = grid_for(p->m, 256, GRID_CAP * 4);
    const int hub = p->opt.robust == BA_LOSS_HUBER;
    if (p->fp32)
        k_linearize<float><<<g, 256, 0, p->st>>>(p->m, p->obs_cam, p->obs_pt, p->uv32, (const float *)p->cur.camc,
                                                 p->cur.pts, p->cur.pts_hl, intr_of(p), hub, p->opt.huber_delta,
                                                 (float *)p->J);
    else
        k_linearize<double><<<g, 256, 0, p->st>>>(p->m, p->obs_cam, p->obs_pt, p->uv64, (const double *)p->cur.camc,
                                                  p->cur.pts, nullptr, intr_of(p), hub, p->opt.huber_delta,
                                                  (double *)p->J);
    ktimer_end(p, K_LINEARIZE, ev);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_cost(ba_problem *p, StateBuf &s, bool trial) {
    cudaEvent_t ev;
    ktimer_begin(p, K_COST, &ev);
    const int g = grid_for(p->m, 256, GRID_CAP);
    const int hub = p->opt.robust == BA_LOSS_HUBER;
    if (p->fp32)
        k_cost<float><<<g, 256, 0, p->st>>>(p->m, p->obs_cam, p->obs_pt, p->uv32, (const float *)s.camc, s.pts,
                                            s.pts_hl, intr_of(p), hub, p->opt.huber_delta, p->sc, trial ? 1 : 0,
                                            p->red, p->counters + 0, p->uv_lo, intrdf_of(p), s.e);
    else
        k_cost<double><<<g, 256, 0, p->st>>>(p->m, p->obs_cam, p->obs_pt, p->uv64, (const double *)s.camc, s.pts,
                                             nullptr, intr_of(p), hub, p->opt.huber_delta, p->sc, trial ? 1 : 0,
                                             p->red, p->counters + 0, p->uv_lo, intrdf_of(p), s.e);
    ktimer_end(p, K_COST, ev);
    p->launches += 1;
    return cudaGetLastError();
}


// trial cameras and their cache (the point pass forms the trial points)
cudaError_t launch_trial_cameras(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_UPDATE, &ev);
    const int nb = (p->n + 127) / 128;
    if (p->fp32) {
        k_update_cams<float><<<nb, 128, 0, p->st>>>(p->n, p->cur.cams, (const float *)p->dxc, p->trial.cams);
        k_prepare_cams32<<<nb, 128, 0, p->st>>>(p->n, p->trial.cams, (float *)p->trial.camc);
    } else {
        k_update_cams<double><<<nb, 128, 0, p->st>>>(p->n, p->cur.cams, (const double *)p->dxc, p->trial.cams);
        k_prepare_cams64<<<nb, 128, 0, p->st>>>(p->n, p->trial.cams, (double *)p->trial.camc);
    }
    ktimer_end(p, K_UPDATE, ev);
    p->launches += 2;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t step_groups_T(ba_problem *p, long long limit) {
    const size_t smem = (size_t)p->obs_max * JW * sizeof(T) +
                        (size_t)p->obs_max / 2 * (3 * sizeof(T) + 6 * sizeof(float) + (sizeof(T) == 8 ? 24 : 0)) +
                        (size_t)p->obs_max * (5 * sizeof(T) + 2 * sizeof(int)) +
                        (size_t)p->obs_max / 2 * 6 * sizeof(float);
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_step_groups<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) !=
        cudaSuccess)
        return e;
    int ctas_per_sm = 0, n_sm = 0;
    if ((e = occupancy((const void *)k_step_groups<T>, STEP_THREADS, smem, &ctas_per_sm, &n_sm)) != cudaSuccess)
        return e;
    const int grid = (int)std::min<int64_t>(p->ngroups, (int64_t)std::max(1, ctas_per_sm) * n_sm);
    const int hub = p->opt.robust == BA_LOSS_HUBER;
    k_step_groups<T><<<grid, STEP_THREADS, smem, p->st>>>(
        p->grp, (int)p->ngroups, p->trk_ptr, p->obs_cam, p->obs_pt, (const T *)(p->fp32 ? (const void *)p->uv32
                                                                                        : (const void *)p->uv64),
        (const T *)p->J, (const T *)p->dxc, (const T *)p->Linv, (const T *)p->lp, p->cur.pts,
        (const T *)p->trial.camc, intr_of(p), hub, p->opt.huber_delta, (T *)p->dxp, p->trial.pts,
        p->fp32 ? p->trial.pts_hl : nullptr, p->sc, p->red, p->counters + 1, p->obs_max, limit, p->uv_lo,
        intrdf_of(p), p->fp32 ? (const float *)p->cur.camc : nullptr, p->fp32 ? p->cur.pts_hl : nullptr,
        p->step_diff ? 1 : 0, p->cur.e, p->trial.e);
    return cudaGetLastError();
}

cudaError_t launch_triangulate(ba_problem *p, int gn_iters) {
    cudaError_t e;
    cudaEvent_t ev;
    if ((e = cudaMemsetAsync(&p->sc->n_tri_fail, 0, sizeof(unsigned long long), p->st)) != cudaSuccess) return e;
    if (p->fp32) {
        // the FP32 caches of the current state are up to date (every state
        // change refreshes them)
        ktimer_begin(p, K_TRIANGULATE, &ev);
        k_triangulate32<<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(
            p->P, p->trk_ptr, p->obs_cam, p->uv32, (const float *)p->cur.camc, p->cur.pts_hl, intr_of(p), gn_iters,
            p->cur.pts, &p->sc->n_tri_fail);
        ktimer_end(p, K_TRIANGULATE, ev);
        p->launches += 1;
        return cudaGetLastError();
    }
    if (!p->tri_cam64) {
        void *d = nullptr;
        if ((e = cudaMalloc(&d, (size_t)p->n * 12 * sizeof(double))) != cudaSuccess) return e;
        p->allocs.push_back(d);
        p->dev_bytes += (size_t)p->n * 12 * sizeof(double);
        p->tri_cam64 = (double *)d;
    }
    ktimer_begin(p, K_TRIANGULATE, &ev);
    k_prepare_cams64<<<(p->n + 127) / 128, 128, 0, p->st>>>(p->n, p->cur.cams, p->tri_cam64);
    k_triangulate<<<grid_for(p->P, 256, GRID_CAP), 256, 0, p->st>>>(p->P, p->trk_ptr, p->obs_cam, p->uv64,
                                                                    p->tri_cam64, intr_of(p), gn_iters, p->cur.pts,
                                                                    &p->sc->n_tri_fail);
    ktimer_end(p, K_TRIANGULATE, ev);
    p->launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_step_points(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_STEP_POINTS, &ev);
    const long long limit = 4000000000LL;  // ~2 s of SM clock per copy wait
    const cudaError_t e = p->fp32 ? step_groups_T<float>(p, limit) : step_groups_T<double>(p, limit);
    ktimer_end(p, K_STEP_POINTS, ev);
    p->launches += 1;
    return e;
}


}  // namespace ba
