// The reduced camera system of cameras with interior parameters, formed on
// the device into a variable-size BSMC system (ba_vbsmc_create_interiors).
//
// Sec. 4 gives block (i, j) of the RCS c_i x c_j entries; Sec. 4.1 counts six
// exterior and five interior unknowns per camera.  The interiors are
// [f, cx, cy, k1, k2]: with xh = x/z, yh = y/z, r2 = xh^2 + yh^2 and
// d = 1 + k1 r2 + k2 r2^2 the projection is u = f d xh + cx, v = f d yh + cy.
// A camera has c_i = 6 (interiors fixed) or 11 unknowns.  Three kernels:
//   k_vbi_linearize  e and J of every observation (Eq. 1), FP64 rows of
//                    [J_c (2 x 11) | J_p (2 x 3) | e (2)];
//   k_vbi_points     per point V_k (damped), V_k^-1 and l_p (Eq. 3);
//   k_vbi_blocks     a warp per stored block (i, j): the sum over its point
//                    pairs of -W_a V_k^-1 W_b^T (Eq. 4), plus U_i (damped) and
//                    b_i on the diagonal.  The pairs of a block are listed on
//                    the host (track order), so the sums need no atomics and
//                    are deterministic.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "vbsmc_internal.h"

namespace ba {

constexpr int VJW = 32;      // FP64 J row: J_c 2 x 11 at 0, 11 | J_p 2 x 3 at 22, 25 | e at 28, 29
constexpr int VB_CI = 11;    // unknowns of a self-calibrating camera
constexpr int VB_NT = 4;     // block entries per lane: 4 x 32 >= 11 x 11

__global__ void k_vbi_linearize(int64_t m, const int *__restrict__ ocam, const int *__restrict__ opt,
                                const double *__restrict__ uv, const double *__restrict__ cams,
                                const double *__restrict__ intr, const double *__restrict__ pts,
                                double *__restrict__ J) {
    for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < m; a += (int64_t)gridDim.x * blockDim.x) {
        const int i = ocam[a], k = opt[a];
        double q[4], R[9];
        quat_exp(cams + 6 * i, q);
        quat_to_R(q, R);
        const double *X = pts + 3 * (int64_t)k, *t = cams + 6 * i + 3, *kk = intr + 5 * i;
        double Xc[3];
        for (int r = 0; r < 3; ++r) Xc[r] = R[3 * r] * X[0] + R[3 * r + 1] * X[1] + R[3 * r + 2] * X[2] + t[r];
        const double f = kk[0], k1 = kk[3], k2 = kk[4];
        const double z = Xc[2], xh = Xc[0] / z, yh = Xc[1] / z;
        const double r2 = xh * xh + yh * yh, d = 1.0 + k1 * r2 + k2 * r2 * r2, g = 2.0 * (k1 + 2.0 * k2 * r2);
        // image-plane Jacobian D of (f d xh, f d yh) w.r.t. (xh, yh), then A = D d(xh, yh)/dX_cam
        const double D00 = f * (d + g * xh * xh), D01 = f * g * xh * yh, D11 = f * (d + g * yh * yh);
        double A[2][3];
        A[0][0] = D00 / z;
        A[0][1] = D01 / z;
        A[0][2] = -(D00 * xh + D01 * yh) / z;
        A[1][0] = D01 / z;
        A[1][1] = D11 / z;
        A[1][2] = -(D01 * xh + D11 * yh) / z;
        // dX_cam/d(d_omega) = -[X_cam]x (camera-frame update), dX_cam/d(dt) = I, dX_cam/dX = R
        const double Mx[3][3] = {{0.0, Xc[2], -Xc[1]}, {-Xc[2], 0.0, Xc[0]}, {Xc[1], -Xc[0], 0.0}};
        double *o = J + a * VJW;
        const double pr[2] = {xh, yh};
        for (int r = 0; r < 2; ++r) {
            double *jc = o + VB_CI * r, *jp = o + 22 + 3 * r;
            for (int c = 0; c < 3; ++c) {
                jc[c] = A[r][0] * Mx[0][c] + A[r][1] * Mx[1][c] + A[r][2] * Mx[2][c];
                jc[3 + c] = A[r][c];
                jp[c] = A[r][0] * R[c] + A[r][1] * R[3 + c] + A[r][2] * R[6 + c];
            }
            jc[6] = d * pr[r];                 // f
            jc[7] = r == 0 ? 1.0 : 0.0;        // cx
            jc[8] = r == 0 ? 0.0 : 1.0;        // cy
            jc[9] = f * pr[r] * r2;            // k1
            jc[10] = f * pr[r] * r2 * r2;      // k2
        }
        o[28] = f * d * xh + kk[1] - uv[2 * a];
        o[29] = f * d * yh + kk[2] - uv[2 * a + 1];
        o[30] = 0.0;
        o[31] = 0.0;
    }
}

// V_k = sum J_p^T J_p + lambda clamp(diag), its inverse (adjugate; the three
// leading minors must be positive) and l_p = -sum J_p^T e, a thread per point.
__global__ void k_vbi_points(int64_t P, const int *__restrict__ trk_ptr, const double *__restrict__ J, double lambda,
                             double *__restrict__ Vinv, double *__restrict__ lp, int *err) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        double V[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, l[3] = {0, 0, 0};
        for (int a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a) {
            const double *o = J + (int64_t)a * VJW;
            for (int m = 0; m < 3; ++m) {
                for (int n = 0; n < 3; ++n) V[m][n] += o[22 + m] * o[22 + n] + o[25 + m] * o[25 + n];
                l[m] -= o[22 + m] * o[28] + o[25 + m] * o[29];
            }
        }
        for (int m = 0; m < 3; ++m) V[m][m] += lambda * clampT(V[m][m]);
        const double c00 = V[1][1] * V[2][2] - V[1][2] * V[2][1], c01 = V[1][2] * V[2][0] - V[1][0] * V[2][2],
                     c02 = V[1][0] * V[2][1] - V[1][1] * V[2][0];
        const double det = V[0][0] * c00 + V[0][1] * c01 + V[0][2] * c02;
        const double m2 = V[0][0] * V[1][1] - V[0][1] * V[1][0];
        double *vi = Vinv + 9 * k;
        if (!(V[0][0] > 0.0) || !(m2 > 0.0) || !(det > 0.0)) {
            atomicExch(err, (int)BA_ERR_NOT_SPD);
            for (int q = 0; q < 9; ++q) vi[q] = 0.0;
        } else {
            const double id = 1.0 / det;
            vi[0] = c00 * id;
            vi[1] = (V[0][2] * V[2][1] - V[0][1] * V[2][2]) * id;
            vi[2] = (V[0][1] * V[1][2] - V[0][2] * V[1][1]) * id;
            vi[3] = c01 * id;
            vi[4] = (V[0][0] * V[2][2] - V[0][2] * V[2][0]) * id;
            vi[5] = (V[0][2] * V[1][0] - V[0][0] * V[1][2]) * id;
            vi[6] = c02 * id;
            vi[7] = (V[0][1] * V[2][0] - V[0][0] * V[2][1]) * id;
            vi[8] = m2 * id;
        }
        for (int m = 0; m < 3; ++m) lp[3 * k + m] = l[m];
    }
}

// A warp per stored block (i, j) and its list of observation pairs (a, b),
// cam(a) = i, cam(b) = j, of the points both cameras see.  Per pair, lanes
// 0..15 form row r of W_a = J_c,a^T J_p,a (c_i x 3) and lanes 16..31 row c of
// Z_b = V_k^-1 W_b^T (3 x c_j) in the warp's shared slot; then every lane
// subtracts (W_a Z_b)(r, c) for its entries.  On a diagonal block the pairs
// are camera i's observations with themselves, which also give U_i =
// sum J_c^T J_c (damped at the end) and b_i = sum (-J_c^T e - W V^-1 l_p).
template <typename T>
__global__ void __launch_bounds__(256) k_vbi_blocks(int64_t nnzb, const int *__restrict__ brow,
                                                    const int *__restrict__ col, const int *__restrict__ cdim,
                                                    const int *__restrict__ off, const int64_t *__restrict__ boff,
                                                    const int *__restrict__ pptr, const int2 *__restrict__ plist,
                                                    const int *__restrict__ opt, const double *__restrict__ J,
                                                    const double *__restrict__ Vinv, const double *__restrict__ lp,
                                                    double lambda, T *__restrict__ val, T *__restrict__ b) {
    __shared__ double sm[8][3 * 16 + 3 * 16 + 2 * 16];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double *Wa = sm[w], *Zb = Wa + 48, *Jca = Zb + 48;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; k < nnzb; k += nw) {
        const int i = brow[k], j = col[k], ci = cdim[i], cj = cdim[j], nel = ci * cj;
        const bool diag = i == j;
        double acc[VB_NT], dU[VB_NT], bacc = 0.0;
        for (int t = 0; t < VB_NT; ++t) acc[t] = dU[t] = 0.0;
        for (int p = pptr[k]; p < pptr[k + 1]; ++p) {  // warp-uniform
            const int2 pr = plist[p];
            const int kp = opt[pr.x];
            const double *Ja = J + (int64_t)pr.x * VJW, *Jb = J + (int64_t)pr.y * VJW, *Vi = Vinv + 9 * (int64_t)kp;
            if (lane < 16) {
                const int r = lane;
                if (r < ci) {
                    const double j0 = Ja[r], j1 = Ja[VB_CI + r];
                    double wr[3];
                    for (int m = 0; m < 3; ++m) {
                        wr[m] = j0 * Ja[22 + m] + j1 * Ja[25 + m];
                        Wa[3 * r + m] = wr[m];
                    }
                    Jca[r] = j0;
                    Jca[16 + r] = j1;
                    if (diag) {
                        const double *l = lp + 3 * (int64_t)kp;
                        double s = -(j0 * Ja[28] + j1 * Ja[29]);
                        for (int m = 0; m < 3; ++m) s -= wr[m] * (Vi[3 * m] * l[0] + Vi[3 * m + 1] * l[1] + Vi[3 * m + 2] * l[2]);
                        bacc += s;
                    }
                }
            } else {
                const int c = lane - 16;
                if (c < cj) {
                    const double j0 = Jb[c], j1 = Jb[VB_CI + c];
                    double wb[3];
                    for (int n = 0; n < 3; ++n) wb[n] = j0 * Jb[22 + n] + j1 * Jb[25 + n];
                    for (int m = 0; m < 3; ++m) Zb[3 * c + m] = Vi[3 * m] * wb[0] + Vi[3 * m + 1] * wb[1] + Vi[3 * m + 2] * wb[2];
                }
            }
            __syncwarp();
            for (int t = 0; t < VB_NT; ++t) {
                const int E = lane + 32 * t;
                if (E < nel) {
                    const int r = E / cj, c = E - r * cj;
                    acc[t] -= Wa[3 * r] * Zb[3 * c] + Wa[3 * r + 1] * Zb[3 * c + 1] + Wa[3 * r + 2] * Zb[3 * c + 2];
                    if (diag) {
                        const double u = Jca[r] * Jca[c] + Jca[16 + r] * Jca[16 + c];
                        acc[t] += u;
                        if (r == c) dU[t] += u;
                    }
                }
            }
            __syncwarp();
        }
        for (int t = 0; t < VB_NT; ++t) {
            const int E = lane + 32 * t;
            if (E < nel) {
                const int r = E / cj, c = E - r * cj;
                double v = acc[t];
                if (diag && r == c) v += lambda * clampT(dU[t]);
                val[boff[k] + E] = (T)v;
            }
        }
        if (diag && lane < ci) b[off[i] + lane] = (T)bacc;
    }
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
    if (!cams || !intr || !cdim || !pts || !obs_cam || !obs_pt || !obs_uv)
        return set_error(BA_ERR_INVALID_ARG, "null input array");
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0) return set_error(BA_ERR_INVALID_ARG, "sizes must be positive");
    if (!(lambda >= 0.0) || !std::isfinite(lambda)) return set_error(BA_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    for (int32_t i = 0; i < n_cams; ++i)
        if (cdim[i] != 6 && cdim[i] != VB_CI) return set_error(BA_ERR_INVALID_ARG, "cdim must be 6 or 11");
    if (!finite_n(cams, (int64_t)n_cams * 6) || !finite_n(intr, (int64_t)n_cams * 5) || !finite_n(pts, n_pts * 3) ||
        !finite_n(obs_uv, n_obs * 2))
        return set_error(BA_ERR_NONFINITE, "non-finite camera, interior, point or observation value");
    HostSetup hs;
    std::string err;
    ba_status s = symbolic_setup(n_cams, n_pts, n_obs, obs_cam, obs_pt, nullptr, OBS_MAX_DEFAULT, true, hs, err);
    if (s) return set_error(s, err.c_str());
    const int64_t nnzb = (int64_t)hs.col.size();
    // the observation pairs of every stored block, in track order
    std::vector<int64_t> cnt(nnzb + 1, 0);
    auto block_of = [&](int32_t ca, int32_t cb) {
        const int32_t *c0 = hs.col.data() + hs.row_ptr[ca], *c1 = hs.col.data() + hs.row_ptr[ca + 1];
        return (int64_t)(std::lower_bound(c0, c1, cb) - hs.col.data());
    };
    for (int64_t k = 0; k < n_pts; ++k)
        for (int32_t p = hs.trk_ptr[k]; p < hs.trk_ptr[k + 1]; ++p)
            for (int32_t q = p; q < hs.trk_ptr[k + 1]; ++q) cnt[block_of(hs.obs_cam[p], hs.obs_cam[q]) + 1]++;
    for (int64_t k = 0; k < nnzb; ++k) cnt[k + 1] += cnt[k];
    if (cnt[nnzb] >= (int64_t)INT32_MAX) return set_error(BA_ERR_INVALID_ARG, "more than 2^31 observation pairs");
    std::vector<int32_t> pptr(cnt.begin(), cnt.end());
    std::vector<int2> plist(cnt[nnzb]);
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t k = 0; k < n_pts; ++k)
            for (int32_t p = hs.trk_ptr[k]; p < hs.trk_ptr[k + 1]; ++p)
                for (int32_t q = p; q < hs.trk_ptr[k + 1]; ++q)
                    plist[fill[block_of(hs.obs_cam[p], hs.obs_cam[q])]++] = make_int2(p, q);
    }
    // inputs in the internal order: observations by (point, camera), points by hs.pt_perm
    std::vector<double> uv(2 * n_obs), ptsi(3 * n_pts);
    for (int64_t a = 0; a < n_obs; ++a) {
        uv[2 * a] = obs_uv[2 * hs.obs_perm[a]];
        uv[2 * a + 1] = obs_uv[2 * hs.obs_perm[a] + 1];
    }
    for (int64_t k = 0; k < n_pts; ++k)
        for (int c = 0; c < 3; ++c) ptsi[3 * k + c] = pts[3 * hs.pt_perm[k] + c];

    ba_vbsmc *h = nullptr;
    if ((s = vb_build(o, n_cams, cdim, nnzb, hs.row_ptr.data(), hs.col.data(), &h))) return s;
    Scratch sc;
    int *d_ocam = nullptr, *d_opt = nullptr, *d_trk = nullptr, *d_pptr = nullptr, *d_err = nullptr;
    int2 *d_plist = nullptr;
    double *d_uv = nullptr, *d_cams = nullptr, *d_intr = nullptr, *d_pts = nullptr, *d_J = nullptr, *d_Vinv = nullptr,
           *d_lp = nullptr;
    cudaError_t e = cudaSuccess;
    auto step = [&](cudaError_t r) {
        if (e == cudaSuccess) e = r;
    };
    step(sc.put((void **)&d_ocam, hs.obs_cam.data(), n_obs * sizeof(int32_t)));
    step(sc.put((void **)&d_opt, hs.obs_pt.data(), n_obs * sizeof(int32_t)));
    step(sc.put((void **)&d_trk, hs.trk_ptr.data(), (n_pts + 1) * sizeof(int32_t)));
    step(sc.put((void **)&d_pptr, pptr.data(), (nnzb + 1) * sizeof(int32_t)));
    step(sc.put((void **)&d_plist, plist.data(), plist.size() * sizeof(int2)));
    step(sc.put((void **)&d_uv, uv.data(), uv.size() * sizeof(double)));
    step(sc.put((void **)&d_cams, cams, (size_t)n_cams * 6 * sizeof(double)));
    step(sc.put((void **)&d_intr, intr, (size_t)n_cams * 5 * sizeof(double)));
    step(sc.put((void **)&d_pts, ptsi.data(), ptsi.size() * sizeof(double)));
    step(sc.alloc((void **)&d_J, (size_t)n_obs * VJW * sizeof(double)));
    step(sc.alloc((void **)&d_Vinv, (size_t)n_pts * 9 * sizeof(double)));
    step(sc.alloc((void **)&d_lp, (size_t)n_pts * 3 * sizeof(double)));
    step(sc.alloc((void **)&d_err, sizeof(int)));
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        ba_vbsmc_destroy(h);
        return set_error(BA_ERR_OOM, "cudaMalloc failed");
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d_err, 0, sizeof(int), h->st);
    if (e == cudaSuccess) {
        const int g1 = (int)std::min<int64_t>((n_obs + 255) / 256, 152 * 16);
        k_vbi_linearize<<<g1, 256, 0, h->st>>>(n_obs, d_ocam, d_opt, d_uv, d_cams, d_intr, d_pts, d_J);
        const int g2 = (int)std::min<int64_t>((n_pts + 255) / 256, 152 * 16);
        k_vbi_points<<<g2, 256, 0, h->st>>>(n_pts, d_trk, d_J, lambda, d_Vinv, d_lp, d_err);
        const int g3 = (int)std::min<int64_t>((nnzb * 32 + 255) / 256, 152 * 16);
        if (h->fp32)
            k_vbi_blocks<float><<<g3, 256, 0, h->st>>>(nnzb, h->brow, h->col, h->cdim, h->off, h->boff, d_pptr, d_plist,
                                                       d_opt, d_J, d_Vinv, d_lp, lambda, (float *)h->val, (float *)h->b);
        else
            k_vbi_blocks<double><<<g3, 256, 0, h->st>>>(nnzb, h->brow, h->col, h->cdim, h->off, h->boff, d_pptr,
                                                        d_plist, d_opt, d_J, d_Vinv, d_lp, lambda, (double *)h->val,
                                                        (double *)h->b);
        e = cudaGetLastError();
    }
    int flag = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&flag, d_err, sizeof(int), cudaMemcpyDeviceToHost, h->st);
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

}  // extern "C"
