// Block-Jacobi PCG on the RCS S y = b (Sec. 3.2, Eqs. 6-7), the BSMC
// matrix-vector product (Sec. 6.2, Fig. 13), the FP64 refinement residual and
// the back-substitution of the points (Eq. 5).
//
// PCG recurrence (y0 = 0): r0 = b, d0 = M^-1 r0; per iteration
//   alpha = r^T M^-1 r / d^T S d, y += alpha d, r -= alpha S d,
//   stop if ||r|| <= T ||r0||, beta = r+^T M^-1 r+ / r^T M^-1 r,
//   d = M^-1 r+ + beta d.
// Two kernels per iteration: the SpMV forms d = z + beta d_old on the fly
// (double-buffered d), q = S d and d^T S d; the update kernel does the axpys,
// z = M^-1 r and the two dot products.  Reductions end in the last CTA (no
// waiting), and a device flag stops the recurrence, so a batch of iterations
// is queued without host round trips.
#include "device_util.cuh"

namespace ba {

// q += S x over BSMC: a warp per block row; each lane takes blocks of the
// row, adds S_ij x_j to its row sum and scatters S_ij^T x_i to q_j.
// PCG variant: x_j = z_j + beta d_old_j, row owner stores d_new_i, and the
// quadratic form d^T S d is accumulated (each off-diagonal block twice).
template <typename TS, typename TV, bool PCG>
__global__ void __launch_bounds__(256) k_spmv(int n, const int *__restrict__ row_ptr, const int *__restrict__ col,
                                              const TS *__restrict__ S, const TV *__restrict__ xz,
                                              const TV *__restrict__ dold, TV *__restrict__ dnew, TV *__restrict__ q,
                                              DevScalars *sc, double *red, unsigned *ctr) {
    if (PCG && sc->done) return;
    const TV beta = PCG ? (TV)sc->beta : TV(0);
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    double pap = 0.0;
    for (int i = warp; i < n; i += nw) {
        TV di[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) di[c] = PCG ? xz[6 * i + c] + beta * dold[6 * i + c] : xz[6 * i + c];
        if (PCG) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                if (lane == c) dnew[6 * i + c] = di[c];
        }
        TV acc[6] = {0, 0, 0, 0, 0, 0};
        const int rb = row_ptr[i], re = row_ptr[i + 1];
        for (int blk = rb + lane; blk < re; blk += 32) {
            const int j = col[blk];
            const TS *Sb = S + (int64_t)blk * BW;
            TV Sv[36];
#pragma unroll
            for (int t = 0; t < 36; ++t) Sv[t] = (TV)Sb[t];
            TV dj[6];
            if (j == i) {
#pragma unroll
                for (int c = 0; c < 6; ++c) dj[c] = di[c];
            } else {
#pragma unroll
                for (int c = 0; c < 6; ++c) dj[c] = PCG ? xz[6 * j + c] + beta * dold[6 * j + c] : xz[6 * j + c];
            }
            double qf = 0.0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                TV t = TV(0);
#pragma unroll
                for (int c = 0; c < 6; ++c) t += Sv[6 * r + c] * dj[c];
                acc[r] += t;
                qf += (double)di[r] * (double)t;
            }
            if (j != i) {
                pap += 2.0 * qf;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    TV u = TV(0);
#pragma unroll
                    for (int r = 0; r < 6; ++r) u += Sv[6 * r + c] * di[r];
                    atomicAdd(q + 6 * j + c, u);
                }
            } else {
                pap += qf;
            }
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[r] = warp_sum(acc[r]);
        if (lane == 0)
#pragma unroll
            for (int r = 0; r < 6; ++r) atomicAdd(q + 6 * i + r, acc[r]);
    }
    if (PCG) {
        double v[1] = {pap};
        grid_sum<1>(v, red, ctr, [&](double *t) {
            sc->pAp = t[0];
            if (!(t[0] > 0.0)) {
                sc->done = 1;
                sc->err = (int)BA_ERR_NOT_SPD;
                sc->alpha = 0.0;
            } else {
                sc->alpha = sc->rz / t[0];
            }
        });
    }
}

template <typename T>
__device__ __forceinline__ void apply_minv(const T *__restrict__ Minv, int i, const T *r, T *z) {
    const T *M = Minv + 36 * (int64_t)i;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        T s = T(0);
#pragma unroll
        for (int c = 0; c < 6; ++c) s += M[6 * a + c] * r[c];
        z[a] = s;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pcg_init(int n, const T *__restrict__ rhs, const T *__restrict__ Minv, T *y, T *r,
                                                  T *z, T *dold, T *q, DevScalars *sc, double tol2, int max_iters,
                                                  double *red, unsigned *ctr) {
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ri[6], zi[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ri[c] = rhs[6 * i + c];
            r[6 * i + c] = ri[c];
            y[6 * i + c] = T(0);
            q[6 * i + c] = T(0);
            dold[6 * i + c] = T(0);
        }
        apply_minv(Minv, i, ri, zi);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[6 * i + c] = zi[c];
            v[0] += (double)ri[c] * (double)zi[c];
            v[1] += (double)ri[c] * (double)ri[c];
        }
    }
    grid_sum<2>(v, red, ctr, [&](double *t) {
        sc->rz = t[0];
        sc->rr = t[1];
        sc->rr0 = t[1];
        sc->beta = 0.0;
        sc->alpha = 0.0;
        sc->iters = 0;
        sc->tol2 = tol2;
        sc->max_iters = max_iters;
        sc->done = (t[1] == 0.0 || max_iters <= 0) ? 1 : 0;
    });
}

template <typename T>
__global__ void __launch_bounds__(256) k_pcg_update(int n, const T *__restrict__ Minv, const T *__restrict__ d, T *q,
                                                    T *y, T *r, T *z, DevScalars *sc, double *red, unsigned *ctr) {
    if (sc->done) return;
    const T alpha = (T)sc->alpha;
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ri[6], zi[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            y[6 * i + c] += alpha * d[6 * i + c];
            ri[c] = r[6 * i + c] - alpha * q[6 * i + c];
            r[6 * i + c] = ri[c];
            q[6 * i + c] = T(0);
        }
        apply_minv(Minv, i, ri, zi);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[6 * i + c] = zi[c];
            v[0] += (double)ri[c] * (double)zi[c];
            v[1] += (double)ri[c] * (double)ri[c];
        }
    }
    grid_sum<2>(v, red, ctr, [&](double *t) {
        const int it = sc->iters + 1;
        sc->iters = it;
        sc->rr = t[1];
        if (t[1] <= sc->tol2 * sc->rr0 || it >= sc->max_iters) {
            sc->done = 1;
        } else {
            sc->beta = t[0] / sc->rz;
            sc->rz = t[0];
        }
    });
}

// r64 = b - q64 (q64 = S x64 from the FP64 SpMV), q64 reset; ||r64||^2, ||b||^2.
template <typename T>
__global__ void __launch_bounds__(256) k_resid_fin(int n, const T *__restrict__ b, double *q64, double *r64, DevScalars *sc,
                                                   double *red, unsigned *ctr) {
    double v[2] = {0.0, 0.0};
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < 6 * n; x += gridDim.x * blockDim.x) {
        const double bi = (double)b[x];
        const double ri = bi - q64[x];
        r64[x] = ri;
        q64[x] = 0.0;
        v[0] += ri * ri;
        v[1] += bi * bi;
    }
    grid_sum<2>(v, red, ctr, [&](double *t) {
        sc->rr64 = t[0];
        sc->bb64 = t[1];
    });
}

template <typename T>
__global__ void k_to_T(int64_t cnt, const double *__restrict__ x, T *__restrict__ o) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        o[i] = (T)x[i];
}
template <typename T>
__global__ void k_acc64(int64_t cnt, const T *__restrict__ y, double *__restrict__ x, int first) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        x[i] = (first ? 0.0 : x[i]) + (double)y[i];
}

// Eq. 5: dx_p = V^-1 (l_p - sum_a J_p,a^T J_c,a dx_c) with V^-1 = L^-T L^-1.
template <typename T>
__global__ void __launch_bounds__(256) k_back_sub(int64_t P, const int *__restrict__ trk_ptr, const int *__restrict__ obs_cam,
                                                  const T *__restrict__ J, const T *__restrict__ dxc,
                                                  const T *__restrict__ Linv, const T *__restrict__ lp,
                                                  T *__restrict__ dxp) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        T s0 = lp[3 * k], s1 = lp[3 * k + 1], s2 = lp[3 * k + 2];
        for (int a = trk_ptr[k]; a < trk_ptr[k + 1]; ++a) {
            const T *j = J + (int64_t)a * JW;
            const T *dc = dxc + 6 * obs_cam[a];
            T t0 = T(0), t1 = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) { t0 += j[c] * dc[c]; t1 += j[6 + c] * dc[c]; }
            s0 -= j[12] * t0 + j[15] * t1;
            s1 -= j[13] * t0 + j[16] * t1;
            s2 -= j[14] * t0 + j[17] * t1;
        }
        const T *m = Linv + 6 * k;  // m00 m10 m11 m20 m21 m22
        const T u0 = m[0] * s0, u1 = m[1] * s0 + m[2] * s1, u2 = m[3] * s0 + m[4] * s1 + m[5] * s2;
        dxp[3 * k] = m[0] * u0 + m[1] * u1 + m[3] * u2;
        dxp[3 * k + 1] = m[2] * u1 + m[4] * u2;
        dxp[3 * k + 2] = m[5] * u2;
    }
}

// --------------------------------------------------------------------------
// launchers
// --------------------------------------------------------------------------
static inline int grid_for(int64_t work, int threads, int cap) {
    int64_t g = (work + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}
static constexpr int VEC_CAP = 152 * 4;

// pv[]: 0 y, 1 r, 2 z, 3 d0, 4 d1, 5 q
cudaError_t launch_pcg_init(ba_problem *p, const void *rhs, double tol, int max_iters) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_INIT, &ev);
    const int g = grid_for(p->n, 256, VEC_CAP);
    if (p->fp32)
        k_pcg_init<float><<<g, 256, 0, p->st>>>(p->n, (const float *)rhs, (const float *)p->Minv, (float *)p->pv[0],
                                                (float *)p->pv[1], (float *)p->pv[2], (float *)p->pv[3],
                                                (float *)p->pv[5], p->sc, tol * tol, max_iters, p->red, p->counters + 2);
    else
        k_pcg_init<double><<<g, 256, 0, p->st>>>(p->n, (const double *)rhs, (const double *)p->Minv,
                                                 (double *)p->pv[0], (double *)p->pv[1], (double *)p->pv[2],
                                                 (double *)p->pv[3], (double *)p->pv[5], p->sc, tol * tol, max_iters,
                                                 p->red, p->counters + 2);
    ktimer_end(p, K_PCG_INIT, ev);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pcg_iter(ba_problem *p, int it) {
    // even iterations read d0 and write d1, odd ones the reverse
    void *dold = p->pv[3 + (it & 1)], *dnew = p->pv[4 - (it & 1)];
    const int gs = grid_for((int64_t)p->n * 32, 256, 152 * 8);
    const int gv = grid_for(p->n, 256, VEC_CAP);
    cudaEvent_t ev;
    ktimer_begin(p, K_SPMV, &ev);
    if (p->fp32)
        k_spmv<float, float, true><<<gs, 256, 0, p->st>>>(p->n, p->row_ptr, p->col, (const float *)p->S,
                                                          (const float *)p->pv[2], (const float *)dold, (float *)dnew,
                                                          (float *)p->pv[5], p->sc, p->red, p->counters + 3);
    else
        k_spmv<double, double, true><<<gs, 256, 0, p->st>>>(p->n, p->row_ptr, p->col, (const double *)p->S,
                                                            (const double *)p->pv[2], (const double *)dold,
                                                            (double *)dnew, (double *)p->pv[5], p->sc, p->red,
                                                            p->counters + 3);
    ktimer_end(p, K_SPMV, ev);
    p->launches += 1;
    ktimer_begin(p, K_PCG_UPDATE, &ev);
    if (p->fp32)
        k_pcg_update<float><<<gv, 256, 0, p->st>>>(p->n, (const float *)p->Minv, (const float *)dnew,
                                                   (float *)p->pv[5], (float *)p->pv[0], (float *)p->pv[1],
                                                   (float *)p->pv[2], p->sc, p->red, p->counters + 4);
    else
        k_pcg_update<double><<<gv, 256, 0, p->st>>>(p->n, (const double *)p->Minv, (const double *)dnew,
                                                    (double *)p->pv[5], (double *)p->pv[0], (double *)p->pv[1],
                                                    (double *)p->pv[2], p->sc, p->red, p->counters + 4);
    ktimer_end(p, K_PCG_UPDATE, ev);
    p->launches += 1;
    return cudaGetLastError();
}

// from_x64: r64 = b - S x64; else r64 = b (x64 = 0).
cudaError_t launch_resid64(ba_problem *p, bool from_x64) {
    cudaEvent_t ev;
    ktimer_begin(p, K_RESID64, &ev);
    if (from_x64) {
        const int gs = grid_for((int64_t)p->n * 32, 256, 152 * 8);
        if (p->fp32)
            k_spmv<float, double, false><<<gs, 256, 0, p->st>>>(p->n, p->row_ptr, p->col, (const float *)p->S,
                                                                p->x64, nullptr, nullptr, p->q64, p->sc, p->red,
                                                                p->counters + 5);
        else
            k_spmv<double, double, false><<<gs, 256, 0, p->st>>>(p->n, p->row_ptr, p->col, (const double *)p->S,
                                                                 p->x64, nullptr, nullptr, p->q64, p->sc, p->red,
                                                                 p->counters + 5);
    }
    const int g = grid_for((int64_t)p->n * 6, 256, VEC_CAP);
    if (p->fp32)
        k_resid_fin<float><<<g, 256, 0, p->st>>>(p->n, (const float *)p->b, p->q64, p->r64, p->sc, p->red,
                                                 p->counters + 6);
    else
        k_resid_fin<double><<<g, 256, 0, p->st>>>(p->n, (const double *)p->b, p->q64, p->r64, p->sc, p->red,
                                                  p->counters + 6);
    ktimer_end(p, K_RESID64, ev);
    p->launches += from_x64 ? 2 : 1;
    return cudaGetLastError();
}

// x64 (+)= y (first: x64 = y)
cudaError_t launch_accumulate_solution(ba_problem *p, bool first) {
    const int64_t cnt = (int64_t)p->n * 6;
    const int g = grid_for(cnt, 256, VEC_CAP);
    if (p->fp32)
        k_acc64<float><<<g, 256, 0, p->st>>>(cnt, (const float *)p->pv[0], p->x64, first ? 1 : 0);
    else
        k_acc64<double><<<g, 256, 0, p->st>>>(cnt, (const double *)p->pv[0], p->x64, first ? 1 : 0);
    p->launches += 1;
    return cudaGetLastError();
}

// rhs_T = (T) r64
cudaError_t launch_refine_rhs(ba_problem *p, void *rhs) {
    const int64_t cnt = (int64_t)p->n * 6;
    const int g = grid_for(cnt, 256, VEC_CAP);
    if (p->fp32)
        k_to_T<float><<<g, 256, 0, p->st>>>(cnt, p->r64, (float *)rhs);
    else
        k_to_T<double><<<g, 256, 0, p->st>>>(cnt, p->r64, (double *)rhs);
    p->launches += 1;
    return cudaGetLastError();
}

// dxc = (T) x64
cudaError_t launch_solution_to_step(ba_problem *p) {
    const int64_t cnt = (int64_t)p->n * 6;
    const int g = grid_for(cnt, 256, VEC_CAP);
    if (p->fp32)
        k_to_T<float><<<g, 256, 0, p->st>>>(cnt, p->x64, (float *)p->dxc);
    else
        k_to_T<double><<<g, 256, 0, p->st>>>(cnt, p->x64, (double *)p->dxc);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_back_substitute(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_BACKSUB, &ev);
    const int g = grid_for(p->P, 256, 152 * 16);
    if (p->fp32)
        k_back_sub<float><<<g, 256, 0, p->st>>>(p->P, p->trk_ptr, p->obs_cam, (const float *)p->J,
                                                (const float *)p->dxc, (const float *)p->Linv, (const float *)p->lp,
                                                (float *)p->dxp);
    else
        k_back_sub<double><<<g, 256, 0, p->st>>>(p->P, p->trk_ptr, p->obs_cam, (const double *)p->J,
                                                 (const double *)p->dxc, (const double *)p->Linv,
                                                 (const double *)p->lp, (double *)p->dxp);
    ktimer_end(p, K_BACKSUB, ev);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace ba
