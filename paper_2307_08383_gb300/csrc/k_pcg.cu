// Block-Jacobi PCG on the RCS S y = b (Sec. 3.2, Eqs. 6-7), the BSMC
// matrix-vector product (Sec. 6.2, Fig. 13), the FP64 refinement residual and
// the back-substitution of the points (Eq. 5).
//
// PCG recurrence (y0 = 0): r0 = b, d0 = M^-1 r0; per iteration
//   alpha = r^T M^-1 r / d^T S d, y += alpha d, r -= alpha S d,
//   stop if ||r|| <= T ||r0||, beta = r+^T M^-1 r+ / r^T M^-1 r,
//   d = M^-1 r+ + beta d.
// The whole recurrence runs in one persistent cooperative kernel: per
// iteration a BSMC SpMV phase forms d = z + beta d_old on the fly (double-
// buffered d), q = S d and d^T S d; a grid barrier; an update phase does the
// axpys, z = M^-1 r and the two dot products; a second barrier.  Every CTA
// sums the per-CTA partials in the same order, so all CTAs take the same
// alpha, beta and stop decision without a third barrier.  Barrier waits are
// bounded; a timeout sets an error flag and every CTA leaves.
#include <algorithm>

#include "device_util.cuh"

namespace ba {

// One 6x6 block (16-byte aligned) into registers, read-only path.
template <typename TS, typename TV>
__device__ __forceinline__ void load_block(const TS *__restrict__ Sb, TV (&v)[36]) {
    if constexpr (sizeof(TS) == 4) {
        const float4 *s4 = reinterpret_cast<const float4 *>(Sb);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 t = __ldg(s4 + q);
            v[4 * q] = (TV)t.x; v[4 * q + 1] = (TV)t.y; v[4 * q + 2] = (TV)t.z; v[4 * q + 3] = (TV)t.w;
        }
    } else {
        const double2 *s2 = reinterpret_cast<const double2 *>(Sb);
#pragma unroll
        for (int q = 0; q < 18; ++q) {
            const double2 t = __ldg(s2 + q);
            v[2 * q] = (TV)t.x; v[2 * q + 1] = (TV)t.y;
        }
    }
}

// Six entries of a camera vector (24 B for FP32, 8-byte aligned; 48 B for FP64).
__device__ __forceinline__ void load6(const float *p, float (&v)[6]) {
    const float2 *p2 = reinterpret_cast<const float2 *>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float2 t = __ldcg(p2 + k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}
__device__ __forceinline__ void load6(const double *p, double (&v)[6]) {
    const double2 *p2 = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double2 t = __ldcg(p2 + k);
        v[2 * k] = t.x;
        v[2 * k + 1] = t.y;
    }
}

template <typename TV, bool PCG>
__device__ __forceinline__ void gather_x(const TV *__restrict__ xz, const TV *__restrict__ dold, TV beta, int j,
                                         TV (&x)[6]) {
    load6(xz + 6 * j, x);
    if (PCG) {
        TV d[6];
        load6(dold + 6 * j, d);
#pragma unroll
        for (int c = 0; c < 6; ++c) x[c] += beta * d[c];
    }
}

template <typename TV>
__device__ __forceinline__ void block_apply(const TV (&Sv)[36], const TV (&x)[6], bool transposed, TV (&acc)[6]) {
    if (!transposed) {
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c = 0; c < 6; ++c) acc[r] += Sv[6 * r + c] * x[c];
    } else {
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
            for (int r = 0; r < 6; ++r) acc[c] += Sv[6 * r + c] * x[r];
    }
}

// q = S x over BSMC without atomics: a warp per block row i walks the row's
// two-sided entry list - the stored blocks (i, j >= i), applied as S_ij x_j,
// then the blocks (j < i, i) of column i, applied as S_ji^T x_j - so q_i is
// one warp's sum: deterministic, no zeroing, no red.add.  (Fig. 13 reads each
// block once and scatters; here each off-diagonal block is read twice, from
// L2.)  A lane takes two entries at a time and issues all their loads before
// any arithmetic, so one L2 round trip covers ~64 blocks of the row.
// PCG variant: x_j = z_j + beta d_old_j, the row owner stores d_new_i, and the
// function returns this thread's share of d^T S d = sum_i d_i^T q_i.
template <typename TS, typename TV, bool PCG>
__device__ __forceinline__ double spmv_rows(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                            const TS *__restrict__ S, const TV *__restrict__ xz,
                                            const TV *__restrict__ dold, TV *__restrict__ dnew, TV *__restrict__ q,
                                            TV beta) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    TV pap = TV(0);
    for (int i = warp; i < n; i += nw) {
        const int tb = __ldg(tw_ptr + i), te = __ldg(tw_ptr + i + 1);
        TV di[6];
        gather_x<TV, PCG>(xz, dold, beta, i, di);
        if (PCG) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                if (lane == c) dnew[6 * i + c] = di[c];
        }
        TV acc[6] = {0, 0, 0, 0, 0, 0};
        for (int t0 = tb + lane; t0 < te; t0 += 64) {
            const int t1 = t0 + 32;
            const bool has1 = t1 < te;
            const int2 ea = __ldg(tw_ent + t0);
            const int2 eb = has1 ? __ldg(tw_ent + t1) : ea;
            TV Sa[36], Sb[36], xa[6], xb[6];
            load_block<TS, TV>(S + (int64_t)(ea.x & 0x7fffffff) * BW, Sa);
            load_block<TS, TV>(S + (int64_t)(eb.x & 0x7fffffff) * BW, Sb);
            gather_x<TV, PCG>(xz, dold, beta, ea.y, xa);
            gather_x<TV, PCG>(xz, dold, beta, eb.y, xb);
            block_apply<TV>(Sa, xa, ea.x < 0, acc);
            if (has1) block_apply<TV>(Sb, xb, eb.x < 0, acc);
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[r] = warp_sum(acc[r]);
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (lane == c) q[6 * i + c] = acc[c];
        if (PCG && lane == 0) {
#pragma unroll
            for (int c = 0; c < 6; ++c) pap += di[c] * acc[c];
        }
    }
    return (double)pap;
}

// q = S x with FP64 accumulation, for the refinement residual.
template <typename TS>
__global__ void __launch_bounds__(256) k_spmv64(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                                const TS *__restrict__ S, const double *__restrict__ x, double *q) {
    spmv_rows<TS, double, false>(n, tw_ptr, tw_ent, S, x, nullptr, nullptr, q, 0.0);
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
                                                  T *z, T *dold, T *q, T *q1, DevScalars *sc, double tol2, int max_iters,
                                                  double *red, unsigned *ctr) {
    T rz_p = T(0), rr_p = T(0);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        T ri[6], zi[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ri[c] = rhs[6 * i + c];
            r[6 * i + c] = ri[c];
            y[6 * i + c] = T(0);
            q[6 * i + c] = T(0);
            q1[6 * i + c] = T(0);
            dold[6 * i + c] = T(0);
        }
        apply_minv(Minv, i, ri, zi);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[6 * i + c] = zi[c];
            rz_p += ri[c] * zi[c];
            rr_p += ri[c] * ri[c];
        }
    }
    double v[2] = {(double)rz_p, (double)rr_p};
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

// The PCG recurrence from the state k_pcg_init left (alpha, beta, stop test
// as in the header comment).  Cooperative launch: all CTAs are resident.
// r is double-buffered by iteration parity: the update phase of iteration k
// reads r_k (all six entries of a camera) and writes r_k+1.  The update runs one thread per vector entry
// e = 6 i + a; each recomputes camera i's six new residual entries (reads
// shared through L1) to form z_e = sum_c M^-1_i[a][c] r_i[c].
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_persist(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                                     const T *__restrict__ S, const T *__restrict__ Minv, T *y, T *r0,
                                                     T *r1, T *z, T *d0, T *d1, T *q, DevScalars *sc, double *red,
                                                     unsigned *bar, long long limit_cycles) {
    __shared__ double sh[40];
    if (sc->done) return;
    double rz = sc->rz;
    const double rr0 = sc->rr0, tol2 = sc->tol2;
    const int max_iters = sc->max_iters;
    double *redA = red, *redB = red + gridDim.x, *bcast = red + 3 * gridDim.x;
    double beta = 0.0;
    int it = 0;
    const int ne = 6 * n;
    for (;;) {
        const bool odd = it & 1;
        T *dold = odd ? d1 : d0, *dnew = odd ? d0 : d1;
        T *rc = odd ? r1 : r0, *rn = odd ? r0 : r1;
        // SpMV phase: d = z + beta d_old, q = S d, d^T S d
        double v1[1] = {spmv_rows<T, T, true>(n, tw_ptr, tw_ent, S, z, dold, dnew, q, (T)beta)};
        block_sum<1>(v1, sh);
        if (!grid_allreduce<1>(v1, redA, bcast, bar, &sc->err, limit_cycles)) return;
        const double pAp = v1[0];
        if (!(pAp > 0.0)) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                sc->err = (int)BA_ERR_NOT_SPD;
                sc->done = 1;
                sc->iters = it;
            }
            return;
        }
        const T alpha = (T)(rz / pAp);
        // update phase: y += alpha d, r -= alpha q, z = M^-1 r, r^T z, r^T r
        T rz_p = T(0), rr_p = T(0);
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
            const int i = e / 6, a = e - 6 * i;
            T ri[6], qi[6];
            load6(rc + 6 * i, ri);
            load6(q + 6 * i, qi);
#pragma unroll
            for (int c = 0; c < 6; ++c) ri[c] -= alpha * qi[c];
            const T *M = Minv + 36 * (int64_t)i + 6 * a;
            T ze = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) ze += __ldg(M + c) * ri[c];
            T ra = ri[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (a == c) ra = ri[c];
            y[e] += alpha * __ldcg(dnew + e);
            rn[e] = ra;
            z[e] = ze;
            rz_p += ra * ze;
            rr_p += ra * ra;
        }
        double v2[2] = {(double)rz_p, (double)rr_p};
        block_sum<2>(v2, sh);
        if (!grid_allreduce<2>(v2, redB, bcast, bar, &sc->err, limit_cycles)) return;
        const double rz_new = v2[0], rr = v2[1];
        ++it;
        if (rr <= tol2 * rr0 || it >= max_iters) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                sc->iters = it;
                sc->rr = rr;
                sc->rz = rz_new;
                sc->done = 1;
            }
            return;
        }
        beta = rz_new / rz;
        rz = rz_new;
    }
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

// pv[]: 0 y, 1 r, 2 z, 3 d0, 4 d1, 5 q, 6 r (odd iterations), 7 q (odd iterations)
cudaError_t launch_pcg_init(ba_problem *p, const void *rhs, double tol, int max_iters) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_INIT, &ev);
    const int g = grid_for(p->n, 256, VEC_CAP);
    if (p->sv.f32)
        k_pcg_init<float><<<g, 256, 0, p->st>>>(p->n, (const float *)rhs, (const float *)p->sv.Minv, (float *)p->sv.pv[0],
                                                (float *)p->sv.pv[1], (float *)p->sv.pv[2], (float *)p->sv.pv[3],
                                                (float *)p->sv.pv[5], (float *)p->sv.pv[7], p->sc, tol * tol, max_iters, p->red,
                                                p->counters + 2);
    else
        k_pcg_init<double><<<g, 256, 0, p->st>>>(p->n, (const double *)rhs, (const double *)p->sv.Minv,
                                                 (double *)p->sv.pv[0], (double *)p->sv.pv[1], (double *)p->sv.pv[2],
                                                 (double *)p->sv.pv[3], (double *)p->sv.pv[5], (double *)p->sv.pv[7], p->sc,
                                                 tol * tol, max_iters, p->red, p->counters + 2);
    ktimer_end(p, K_PCG_INIT, ev);
    p->launches += 1;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t pcg_loop_T(ba_problem *p) {
    static int blocks_per_sm = -1, n_sm = 0;
    cudaError_t e;
    if (blocks_per_sm < 0) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, k_pcg_persist<T>, 256, 0)) != cudaSuccess)
            return e;
        if (blocks_per_sm > 2) blocks_per_sm = 2;
        if (blocks_per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    }
    // enough warps for one block row each, at most what is co-resident
    int64_t want = ((int64_t)p->n * 32 + 255) / 256;
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)blocks_per_sm * n_sm);
    if ((e = cudaMemsetAsync(p->counters + 14, 0, 2 * sizeof(unsigned), p->st)) != cudaSuccess) return e;
    int n = p->n;
    const int *twp = p->tw_ptr;
    const int2 *twe = p->tw_ent;
    const T *S = (const T *)p->sv.S, *Mi = (const T *)p->sv.Minv;
    T *y = (T *)p->sv.pv[0], *r = (T *)p->sv.pv[1], *z = (T *)p->sv.pv[2], *d0 = (T *)p->sv.pv[3], *d1 = (T *)p->sv.pv[4];
    T *q = (T *)p->sv.pv[5], *r1 = (T *)p->sv.pv[6];
    DevScalars *sc = p->sc;
    double *red = p->red;
    unsigned *bar = p->counters + 14;
    long long limit = 4000000000LL;  // ~2 s of SM clock per barrier wait
    void *args[] = {&n, &twp, &twe, &S, &Mi, &y, &r, &r1, &z, &d0, &d1, &q, &sc, &red, &bar, &limit};
    return cudaLaunchCooperativeKernel((const void *)k_pcg_persist<T>, dim3(grid), dim3(256), args, 0, p->st);
}

cudaError_t launch_pcg_loop(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_LOOP, &ev);
    cudaError_t e = p->sv.f32 ? pcg_loop_T<float>(p) : pcg_loop_T<double>(p);
    ktimer_end(p, K_PCG_LOOP, ev);
    p->launches += 1;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// from_x64: r64 = b - S x64; else r64 = b (x64 = 0).
cudaError_t launch_resid64(ba_problem *p, bool from_x64) {
    cudaEvent_t ev;
    ktimer_begin(p, K_RESID64, &ev);
    if (from_x64) {
        const int gs = grid_for((int64_t)p->n * 32, 256, 152 * 8);
        if (p->fp32)
            k_spmv64<float><<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const float *)p->S, p->x64, p->q64);
        else
            k_spmv64<double><<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const double *)p->S, p->x64, p->q64);
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
    if (p->sv.f32)
        k_acc64<float><<<g, 256, 0, p->st>>>(cnt, (const float *)p->sv.pv[0], p->x64, first ? 1 : 0);
    else
        k_acc64<double><<<g, 256, 0, p->st>>>(cnt, (const double *)p->sv.pv[0], p->x64, first ? 1 : 0);
    p->launches += 1;
    return cudaGetLastError();
}

// rhs_T = (T) r64
cudaError_t launch_refine_rhs(ba_problem *p, void *rhs) {
    const int64_t cnt = (int64_t)p->n * 6;
    const int g = grid_for(cnt, 256, VEC_CAP);
    if (p->sv.f32)
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

template <typename TS>
__global__ void __launch_bounds__(256) k_spmv_f32(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                                  const TS *__restrict__ S, const float *__restrict__ x, float *y) {
    spmv_rows<TS, float, false>(n, tw_ptr, tw_ent, S, x, nullptr, nullptr, y, 0.f);
}

cudaError_t launch_spmv_f32(ba_problem *p, const float *x, float *y) {
    const int gs = grid_for((int64_t)p->n * 32, 256, 152 * 8);
    if (p->fp32)
        k_spmv_f32<float><<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const float *)p->S, x, y);
    else
        k_spmv_f32<double><<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const double *)p->S, x, y);
    p->launches += 1;
    return cudaGetLastError();
}

__global__ void k_demote(int64_t cnt, const double *__restrict__ a, float *__restrict__ o) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x)
        o[x] = (float)a[x];
}

// FP32 shadows of an FP64 problem's S and M^-1 (mixed-precision solve)
cudaError_t launch_demote(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_DEMOTE, &ev);
    const int64_t cs = p->nnzb * BW, cm = (int64_t)p->n * 36;
    k_demote<<<grid_for(cs, 256, 152 * 16), 256, 0, p->st>>>(cs, (const double *)p->S, (float *)p->S32);
    k_demote<<<grid_for(cm, 256, 152 * 4), 256, 0, p->st>>>(cm, (const double *)p->Minv, (float *)p->Minv32);
    ktimer_end(p, K_DEMOTE, ev);
    p->launches += 2;
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
