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
//
// FP32 solves instead run CG on the split-preconditioned system
// S^ = G^T S G (M^-1 = G G^T per camera, G from a Cholesky factor), which is
// block-Jacobi PCG in other variables, in the Chronopoulos-Gear arrangement:
// both dot products of an iteration come after its one SpMV, and the SpMV
// forms each neighbour's new residual r_j - alpha (w_j + beta s_j) itself, so
// an iteration is one phase and one grid all-reduce (see k_pcg_split).
#include <algorithm>
#include <vector>

#include "device_util.cuh"
#include "tma_util.cuh"

namespace ba {

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

// q = S x over BSMC without atomics: a warp per block row i walks the row's
// two-sided entry list - the stored blocks (i, j >= i), applied as S_ij x_j,
// then the blocks (j < i, i) of column i, applied as S_ji^T x_j - so q_i is
// one warp's sum: deterministic, no zeroing, no red.add.  (Fig. 13 reads each
// block once and scatters; here each off-diagonal block is read twice, from
// L2.)  A lane takes two entries at a time and issues all their loads before
// any arithmetic, so one L2 round trip covers ~64 blocks of the row.
// PCG variant: x_j = z_j + beta d_old_j, the row owner stores d_new_i, and the
// function returns this thread's share of d^T S d = sum_i d_i^T q_i.
template <typename TS, typename TV, class GX>
__device__ __forceinline__ void spmv_row(int i, int lane, const int *__restrict__ tw_ptr,
                                         const int2 *__restrict__ tw_ent, const TS *__restrict__ S, GX gx,
                                         TV (&acc)[6]) {
    const int tb = __ldg(tw_ptr + i), te = __ldg(tw_ptr + i + 1);
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] = TV(0);
    for (int t0 = tb + lane; t0 < te; t0 += 64) {
        const int t1 = t0 + 32;
        const bool has1 = t1 < te;
        const int2 ea = __ldg(tw_ent + t0);
        const int2 eb = has1 ? __ldg(tw_ent + t1) : ea;
        TV Sa[36], Sb[36], xa[6], xb[6];
        load_block<TS, TV>(S + (int64_t)(ea.x & 0x7fffffff) * BW, Sa);
        load_block<TS, TV>(S + (int64_t)(eb.x & 0x7fffffff) * BW, Sb);
        gx(ea.y, xa);
        gx(eb.y, xb);
        block_apply<TV>(Sa, xa, ea.x < 0, acc);
        if (has1) block_apply<TV>(Sb, xb, eb.x < 0, acc);
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) acc[r] = warp_sum(acc[r]);
}

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
        TV di[6];
        gather_x<TV, PCG>(xz, dold, beta, i, di);
        if (PCG) {
#pragma unroll
            for (int c = 0; c < 6; ++c)
                if (lane == c) dnew[6 * i + c] = di[c];
        }
        TV acc[6];
        spmv_row<TS, TV>(i, lane, tw_ptr, tw_ent, S,
                         [&](int j, TV(&x)[6]) { gather_x<TV, PCG>(xz, dold, beta, j, x); }, acc);
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

// The same product reading every stored block once (FP32 solves of large
// systems, where the second, transposed read of each off-diagonal block
// would come from DRAM): a warp per block row i takes the row's stored
// blocks (i, j >= i), lane l the blocks l, l + 32, ... two at a time; each
// applies S_ij d_j to the row sum and, for j > i, S_ij^T d_i to q_j with
// vector reductions; the row sum joins q_i the same way.  q must be zero on
// entry.  d^T S d is summed per block as (2 for j > i, 1 for j = i)
// d_i^T S_ij d_j, so it needs no complete q.  The order of q's terms is not
// fixed (floating-point reductions).
__device__ __forceinline__ void red_add2_f(float *a, float u, float v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(u), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add4_f(float *a, float u0, float u1, float u2, float u3) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(u0), "f"(u1), "f"(u2), "f"(u3)
                 : "memory");
}
__device__ __forceinline__ void red_add6_f(float *qj, const float (&t)[6]) {
    if ((reinterpret_cast<uintptr_t>(qj) & 15u) == 0) {
        red_add4_f(qj, t[0], t[1], t[2], t[3]);
        red_add2_f(qj + 4, t[4], t[5]);
    } else {
        red_add2_f(qj, t[0], t[1]);
        red_add4_f(qj + 2, t[2], t[3], t[4], t[5]);
    }
}
__device__ __forceinline__ double spmv_rows_once(int n, const int *__restrict__ row_ptr,
                                                 const int *__restrict__ col, const float *__restrict__ S,
                                                 const float *__restrict__ z, const float *__restrict__ dold,
                                                 float *__restrict__ dnew, float *__restrict__ q, float beta) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    float pap = 0.f;
    for (int i = warp; i < n; i += nw) {
        float di[6];
        gather_x<float, true>(z, dold, beta, i, di);
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (lane == c) dnew[6 * i + c] = di[c];
        const int tb = __ldg(row_ptr + i), te = __ldg(row_ptr + i + 1);
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int t0 = tb + lane; t0 < te; t0 += 64) {
            const int t1 = t0 + 32;
            const bool has1 = t1 < te;
            const int ja = __ldg(col + t0), jb = __ldg(col + (has1 ? t1 : t0));
            float va[36], vb[36], xa[6], xb[6];
            load_block<float, float>(S + (int64_t)t0 * BW, va);
            load_block<float, float>(S + (int64_t)(has1 ? t1 : t0) * BW, vb);
            gather_x<float, true>(z, dold, beta, ja, xa);
            gather_x<float, true>(z, dold, beta, jb, xb);
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && !has1) break;
                const float(&v)[36] = h ? vb : va;
                const float(&xj)[6] = h ? xb : xa;
                const int j = h ? jb : ja;
                float yb[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                block_apply<float>(v, xj, false, yb);
                float dy = 0.f;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    acc[c] += yb[c];
                    dy += di[c] * yb[c];
                }
                pap += j == i ? dy : 2.f * dy;
                if (j != i) {
                    float tr[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                    block_apply<float>(v, di, true, tr);
                    red_add6_f(q + 6 * (int64_t)j, tr);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum(acc[c]);
        if (lane < 6) {
            float out = acc[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) out = acc[c];
            atomicAdd(q + 6 * (int64_t)i + lane, out);
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

// q = S x to about 2^-44 relative on the FP32 pipe, for the refinement
// residual of FP32 problems (FP64 arithmetic runs at a small fraction of the
// FP32 rate on GB300).  x arrives split in FP32 pairs (xh + xl, k_split_x);
// S is FP32.  Each product is the exact s xh (FMA TwoProd) plus s xl, added
// with TwoSum (double-float).  A warp per block row over its two-sided
// entries.
__device__ __forceinline__ void split_f64(double v, float &h, float &l) {
    h = (float)v;
    l = (float)(v - (double)h);
}
__global__ void k_split_x(int64_t cnt, const double *__restrict__ x, float2 *__restrict__ xs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x) {
        float h, l;
        split_f64(x[i], h, l);
        xs[i] = make_float2(h, l);
    }
}
__global__ void __launch_bounds__(256) k_spmv_df(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                                 const float *__restrict__ S, const float2 *__restrict__ xs, double *q) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = warp; i < n; i += nw) {
        df32 acc[6];
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[r] = df32{0.f, 0.f};
        for (int t = __ldg(tw_ptr + i) + lane; t < __ldg(tw_ptr + i + 1); t += 32) {
            const int2 e = __ldg(tw_ent + t);
            const bool tr = e.x < 0;
            const float4 *s4 = reinterpret_cast<const float4 *>(S + (int64_t)(e.x & 0x7fffffff) * BW);
            float sb[36];  // the block, 16-byte loads
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float4 v = __ldg(s4 + q);
                sb[4 * q] = v.x; sb[4 * q + 1] = v.y; sb[4 * q + 2] = v.z; sb[4 * q + 3] = v.w;
            }
            float xh[6], xl[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                const float2 v = __ldcg(xs + 6 * (int64_t)e.y + c);
                xh[c] = v.x;
                xl[c] = v.y;
            }
#pragma unroll
            for (int r = 0; r < 6; ++r)
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    const float sv = tr ? sb[6 * c + r] : sb[6 * r + c];
                    const float ph = sv * xh[c];
                    const float pl = __fmaf_rn(sv, xh[c], -ph) + sv * xl[c];
                    acc[r] = df_add(acc[r], df32{ph, pl});
                }
        }
#pragma unroll
        for (int r = 0; r < 6; ++r) acc[r] = warp_sum_df(acc[r]);
#pragma unroll
        for (int r = 0; r < 6; ++r)
            if (lane == r) q[6 * (int64_t)i + r] = (double)acc[r].hi + (double)acc[r].lo;
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
// ONCE (FP32 only): the product reads each stored block once (spmv_rows_once)
// into q, which is double-buffered by iteration parity: the update phase of
// iteration k reads q_k and zeroes the buffer iteration k + 1 adds into.
template <typename T, bool ONCE>
__global__ void __launch_bounds__(256) k_pcg_persist(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                                                     const int *__restrict__ row_ptr, const int *__restrict__ col,
                                                     const T *__restrict__ S, const T *__restrict__ Minv, T *y, T *r0,
                                                     T *r1, T *z, T *d0, T *d1, T *q0, T *q1, DevScalars *sc,
                                                     double *red, unsigned *bar, long long limit_cycles) {
    __shared__ double sh[40];
    if (sc->done) return;
    double rz = sc->rz;
    const double rr0 = sc->rr0, tol2 = sc->tol2;
    const int max_iters = sc->max_iters;
    double beta = 0.0;
    int it = 0;
    unsigned gen = 0;
    const int ne = 6 * n;
    for (;;) {
        const bool odd = it & 1;
        T *dold = odd ? d1 : d0, *dnew = odd ? d0 : d1;
        T *rc = odd ? r1 : r0, *rn = odd ? r0 : r1;
        T *q = (ONCE && odd) ? q1 : q0, *qz = odd ? q0 : q1;
        // SpMV phase: d = z + beta d_old, q = S d, d^T S d
        double v1[1];
        if constexpr (ONCE)
            v1[0] = spmv_rows_once(n, row_ptr, col, S, z, dold, dnew, q, (float)beta);
        else
            v1[0] = spmv_rows<T, T, true>(n, tw_ptr, tw_ent, S, z, dold, dnew, q, (T)beta);
        block_sum<1>(v1, sh);
        if (!grid_allreduce_sym<1>(v1, red, gen++, bar, &sc->err, limit_cycles)) return;
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
            if (ONCE) qz[e] = T(0);  // the next product adds into it
            rz_p += ra * ze;
            rr_p += ra * ra;
        }
        double v2[2] = {(double)rz_p, (double)rr_p};
        block_sum<2>(v2, sh);
        if (!grid_allreduce_sym<2>(v2, red, gen++, bar, &sc->err, limit_cycles)) return;
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
            T j[JW];
            load_jrow(J + (int64_t)a * JW, j);
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
// Split-preconditioned CG for FP32 solves
// --------------------------------------------------------------------------

// Cholesky A = L L^T of a symmetric 6x6 (row-major, lower triangle read) and
// L^-1, both packed lower (index k(k+1)/2 + l).  False if A is not SPD.
__device__ bool chol6_with_inverse(const double *A, double *L, double *Li) {
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            double s = A[i * 6 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * (i + 1) / 2 + i] = sqrt(s);
            } else {
                L[i * (i + 1) / 2 + j] = s / L[j * (j + 1) / 2 + j];
            }
        }
    }
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Li[i * (i + 1) / 2 + i] = 1.0 / L[i * (i + 1) / 2 + i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            double s = 0.0;
#pragma unroll
            for (int k = j; k < i; ++k) s += L[i * (i + 1) / 2 + k] * Li[k * (k + 1) / 2 + j];
            Li[i * (i + 1) / 2 + j] = -s * Li[i * (i + 1) / 2 + i];
        }
    }
    return true;
}

// Per camera, in FP64, a factor G_i with M_i^-1 = G_i G_i^T and H_i = G_i^-T
// (H r^ gives back the residual of the original system):
//   block-Jacobi (from_minv = 0): S_ii = L L^T, G = L^-T, H = L;
//   a given M^-1 (from_minv = 1):  M^-1 = C C^T, G = C,   H = C^-T.
// Stored row-major FP32, n x 36 each.  The diagonal block of S^ = G^T S G is
// the identity for block-Jacobi (L^-1 L L^T L^-T); for a given M^-1 it is
// G_i^T S_ii G_i, written to Shd (n x 36).
template <typename T>
__global__ void __launch_bounds__(128) k_split_factor(int n, const int *__restrict__ row_ptr, const T *__restrict__ S,
                                                      const T *__restrict__ Minv, int from_minv, float *__restrict__ G,
                                                      float *__restrict__ H, float *__restrict__ Shd, DevScalars *sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T *src = from_minv ? Minv + 36 * (int64_t)i : S + (int64_t)__ldg(row_ptr + i) * BW;
    double A[36], L[21], Li[21];
#pragma unroll
    for (int k = 0; k < 36; ++k) A[k] = (double)src[k];
    float *g = G + 36 * (int64_t)i, *h = H + 36 * (int64_t)i;
    if (!chol6_with_inverse(A, L, Li)) {
        atomicExch(&sc->err, (int)BA_ERR_NOT_SPD);
#pragma unroll
        for (int k = 0; k < 36; ++k) g[k] = h[k] = (k % 7 == 0) ? 1.f : 0.f;
        return;
    }
#pragma unroll
    for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            const double low = a >= c ? L[a * (a + 1) / 2 + c] : 0.0;    // L[a][c]
            const double lit = c >= a ? Li[c * (c + 1) / 2 + a] : 0.0;   // (L^-1)^T[a][c]
            g[6 * a + c] = (float)(from_minv ? low : lit);
            h[6 * a + c] = (float)(from_minv ? lit : low);
        }
    if (from_minv) {
        // S_ii G, then G^T (S_ii G), with G = L (lower) in FP64
        const T *sd = S + (int64_t)__ldg(row_ptr + i) * BW;
        double SG[36];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                double v = 0.0;
#pragma unroll
                for (int k = c; k < 6; ++k) v += (double)sd[6 * a + k] * L[k * (k + 1) / 2 + c];
                SG[6 * a + c] = v;
            }
        float *d = Shd + 36 * (int64_t)i;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                double v = 0.0;
#pragma unroll
                for (int k = a; k < 6; ++k) v += L[k * (k + 1) / 2 + a] * SG[6 * k + c];
                d[6 * a + c] = (float)v;
            }
    }
}

// S^ in two-sided entry order without the diagonal blocks (the split CG's
// lists): entry t of block row i (column j = the entry's y) gets
// S^_ij = G_i^T S_ij G_j, with S_ij the stored block or, for the entries of
// column i, the transpose of the stored block (j, i).  Every off-diagonal
// block is thus held twice, already transposed where needed, so the entries
// of consecutive rows are one contiguous, 16-byte aligned range that a bulk
// copy moves.  A warp per block row, a lane per entry.
template <typename TS>
__global__ void __launch_bounds__(128) k_split_scale(int n, const int *__restrict__ tw_ptr,
                                                     const int2 *__restrict__ tw_ent, const TS *__restrict__ S,
                                                     const float *__restrict__ G, float *__restrict__ Sh) {
    const int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (i >= n) return;
    // G_i (the warp's row, the same for every lane) and each entry's G_j in
    // registers, 16-byte loads; the products accumulate in the order of the
    // plain loops (k ascending), row k of S_ij G_j at a time
    float gi[36];
    {
        const float4 *g4 = reinterpret_cast<const float4 *>(G + 36 * (int64_t)i);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float4 v = __ldg(g4 + q);
            gi[4 * q] = v.x; gi[4 * q + 1] = v.y; gi[4 * q + 2] = v.z; gi[4 * q + 3] = v.w;
        }
    }
    for (int t = __ldg(tw_ptr + i) + lane; t < __ldg(tw_ptr + i + 1); t += 32) {
        const int2 e = __ldg(tw_ent + t);
        const bool tr = e.x < 0;
        const TS *sb = S + (int64_t)(e.x & 0x7fffffff) * BW;
        float gj[36];
        {
            const float4 *g4 = reinterpret_cast<const float4 *>(G + 36 * (int64_t)e.y);
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                const float4 v = __ldg(g4 + q);
                gj[4 * q] = v.x; gj[4 * q + 1] = v.y; gj[4 * q + 2] = v.z; gj[4 * q + 3] = v.w;
            }
        }
        float o[36];
#pragma unroll
        for (int q = 0; q < 36; ++q) o[q] = 0.f;
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float srow[6], t1[6];  // row k of S_ij, then of S_ij G_j
#pragma unroll
            for (int m = 0; m < 6; ++m) srow[m] = (float)(tr ? sb[6 * m + k] : sb[6 * k + m]);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                float v = 0.f;
#pragma unroll
                for (int m = 0; m < 6; ++m) v = __fmaf_rn(srow[m], gj[6 * m + c], v);
                t1[c] = v;
            }
#pragma unroll
            for (int a = 0; a < 6; ++a)
#pragma unroll
                for (int c = 0; c < 6; ++c) o[6 * a + c] = __fmaf_rn(gi[6 * k + a], t1[c], o[6 * a + c]);
        }
        float4 *o4 = reinterpret_cast<float4 *>(Sh + (int64_t)t * BW);
#pragma unroll
        for (int q = 0; q < 9; ++q) o4[q] = make_float4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]);
    }
}

// Vector records of the split CG, double-buffered by iteration parity: per
// camera 20 floats [r (6), w (6), s (6), pad (2)], 80 B and 16-byte aligned,
// so a gather of a neighbour's three vectors is five float4 loads.
constexpr int SREC = 20;

__device__ __forceinline__ void load_rec(const float *rec, int j, float (&v)[20]) {
    const float4 *q = reinterpret_cast<const float4 *>(rec + (int64_t)SREC * j);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const float4 t = __ldcg(q + k);
        v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
}

// r^_0 = G^T rhs per camera into record 0, s = 0 in both records, x^ = p = 0,
// and the scalars of the solve.
__global__ void __launch_bounds__(256) k_split_init(int n, const float *__restrict__ rhs, const float *__restrict__ G,
                                                    float *rec0, float *rec1, float *x, float *p, DevScalars *sc,
                                                    double tol2, int max_iters, int prof) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float b6[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) b6[c] = rhs[6 * i + c];
        const float *g = G + 36 * (int64_t)i;
        float *q0 = rec0 + (int64_t)SREC * i, *q1 = rec1 + (int64_t)SREC * i;
#pragma unroll
        for (int a = 0; a < 6; ++a) {
            float t = 0.f;
#pragma unroll
            for (int c = 0; c < 6; ++c) t = __fmaf_rn(__ldg(g + 6 * c + a), b6[c], t);
            q0[a] = t;
            q0[12 + a] = 0.f;
            q1[12 + a] = 0.f;
            x[6 * i + a] = 0.f;
            p[6 * i + a] = 0.f;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        sc->tol2 = tol2;
        sc->max_iters = max_iters;
        sc->iters = 0;
        sc->alpha = 0.0;
        sc->beta = 0.0;
        sc->done = max_iters <= 0 ? 1 : 0;
        sc->prof_on = prof;
        for (int k = 0; k < 4; ++k) sc->ph[k] = 0.0;
        sc->ph_work_max = 0ull;
    }
}

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// The new residual of a camera from the previous iteration's vectors: the row
// owner and every row that gathers it evaluate exactly these two FMAs.
__device__ __forceinline__ float next_r(float r, float w, float s, float a, float b) {
    return __fmaf_rn(-a, __fmaf_rn(b, s, w), r);
}

// Balanced SpMV of the split CG with a shared-memory halo.  CTA c owns block
// rows [rb, re) (chosen on the host for about equal work) and their entries
// [eb, ee), cut into passes of 32 consecutive entries; warp w of the
// SPLIT_WARPS takes passes w, w + SPLIT_WARPS, ...  The cameras the CTA's
// entries reference (its halo, a few hundred at the benchmark size, with one
// CTA per SM) are gathered once per iteration from the
// previous iteration's records, each transformed once into the vector the
// SpMV applies, x_j = r_j - alpha (w_j + beta s_j), and kept in shared
// memory.  The gather of iteration k + 1 is issued (16-byte asynchronous
// copies of the 80-byte records into the halo area, transformed there in
// place) as soon as the all-reduce that ends iteration k has seen every CTA
// arrive, so its L2 round trip overlaps the partial reads, the block sum and
// the scalar update.  A pass's 32 S^ blocks (4.6 KB, contiguous in entry order) and the
// entries' packed (local row, halo index) arrive by 1-D bulk copies into one
// of the warp's SPLIT_NBUF buffers; since S^ does not change during the
// solve, each refill fetches the warp's pass SPLIT_NBUF positions ahead,
// wrapping into the next iteration.  The pass loop thus reads shared memory only.  A segmented
// shuffle scan over the pass (entries are sorted by row) leaves each row
// segment's sum in its last lane, which stores it in a slot: (q, 0) if the
// segment opens pass q, (q, 1) if it closes it, else the row's own slot.  The
// sums depend only on the entry order: deterministic.
constexpr int SPLIT_WARPS = 16;
constexpr int SPLIT_NBUF = 2;         // copy buffers (passes in flight) per warp
constexpr int SPLIT_CTAS_PER_SM = 1;  // co-resident CTAs per SM the grid is sized for
constexpr int PASS_S_BYTES = 32 * BW * 4;                        // 4608
constexpr int PASS_BYTES = PASS_S_BYTES + 32 * 4;                // + packed metadata
constexpr int SPLIT_STAGE_BYTES = SPLIT_WARPS * SPLIT_NBUF * PASS_BYTES;
constexpr int HX = 20;  // floats per halo camera: its fetched record, then x_j written over r_j

struct SplitPipe {
    float *stage;    // [warp][2][32 * 36 floats + 32 u32]
    uint64_t *mbar;  // [warp][2]
    const float *Sh;
    const uint32_t *meta;  // this CTA's packed entry metadata (16-byte aligned base)
    int eb, ee, m;   // entry range; passes of this warp
    uint32_t seq;    // passes this warp has consumed so far
};

__device__ __forceinline__ float *pass_buf(const SplitPipe &pp, uint32_t s) {
    return pp.stage + (size_t)(SPLIT_NBUF * (threadIdx.x >> 5) + s % SPLIT_NBUF) * (PASS_BYTES / 4);
}

// lane 0: refill buffer (s mod NBUF) with the warp's pass number (s mod m)
__device__ __forceinline__ void split_issue(const SplitPipe &pp, uint32_t s) {
    const int wid = threadIdx.x >> 5;
    const int q = wid + SPLIT_WARPS * (int)(s % (uint32_t)pp.m);
    const int cnt = min(32, pp.ee - pp.eb - 32 * q);
    const uint32_t sbytes = (uint32_t)cnt * BW * 4, mbytes = (uint32_t)((cnt + 3) & ~3) * 4;
    uint64_t *bar = pp.mbar + SPLIT_NBUF * wid + s % SPLIT_NBUF;
    float *buf = pass_buf(pp, s);
    mbar_expect_tx(bar, sbytes + mbytes);
    bulk_g2s(buf, pp.Sh + (int64_t)(pp.eb + 32 * q) * BW, sbytes, bar);
    bulk_g2s(buf + PASS_S_BYTES / 4, pp.meta + 32 * q, mbytes, bar);
}

// lane 0: wait (bounded) for the copies still in flight before the CTA leaves
__device__ __forceinline__ void split_drain(const SplitPipe &pp, long long limit) {
    if ((threadIdx.x & 31) != 0 || pp.m == 0) return;
    const int wid = threadIdx.x >> 5;
    for (uint32_t s = pp.seq; s < pp.seq + SPLIT_NBUF; ++s)
        mbar_wait(pp.mbar + SPLIT_NBUF * wid + s % SPLIT_NBUF, (s / SPLIT_NBUF) & 1u, limit);
}

// One sweep of the warp's passes over the halo vectors hx.  False on an
// mbarrier timeout (then the warp stops; callers agree CTA-wide with
// __syncthreads_and and leave).
__device__ __forceinline__ bool split_passes(SplitPipe &pp, int rb, const int *__restrict__ tw_ptr, const float *hx,
                                             float *slot, float *rowacc, int *err, long long limit) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int eb = pp.eb, ee = pp.ee;
    for (int k = 0; k < pp.m; ++k) {
        const int q = wid + SPLIT_WARPS * k;
        const int t = eb + 32 * q + lane;
        const bool valid = t < ee;
        const uint32_t b = pp.seq % SPLIT_NBUF;
        // every lane observes the copy's completion; the outcome is warp-uniform
        if (!__all_sync(0xffffffffu, mbar_wait(pp.mbar + SPLIT_NBUF * wid + b, (pp.seq / SPLIT_NBUF) & 1u, limit))) {
            if (lane == 0) atomicExch(err, (int)BA_ERR_TIMEOUT);
            return false;
        }
        const float *buf = pass_buf(pp, pp.seq);
        int lr = 0xFFFF;
        float y[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (valid) {
            const uint32_t md = reinterpret_cast<const uint32_t *>(buf + PASS_S_BYTES / 4)[lane];
            lr = (int)(md & 0xFFFFu);
            const float4 *x4 = reinterpret_cast<const float4 *>(hx + HX * (md >> 16));
            const float4 xa = x4[0], xb = x4[1];
            const float x[6] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y};
            const float4 *s4 = reinterpret_cast<const float4 *>(buf + lane * BW);
#pragma unroll
            for (int h = 0; h < 3; ++h) {  // two block rows (12 floats) at a time
                const float4 u0 = s4[3 * h], u1 = s4[3 * h + 1], u2 = s4[3 * h + 2];
                const float ra[6] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y};
                const float rb6[6] = {u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    y[2 * h] = __fmaf_rn(ra[c], x[c], y[2 * h]);
                    y[2 * h + 1] = __fmaf_rn(rb6[c], x[c], y[2 * h + 1]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) split_issue(pp, pp.seq + SPLIT_NBUF);  // this buffer is free again
        ++pp.seq;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int lu = __shfl_up_sync(0xffffffffu, lr, d);
            float yu[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) yu[c] = __shfl_up_sync(0xffffffffu, y[c], d);
            if (lane >= d && lu == lr)
#pragma unroll
                for (int c = 0; c < 6; ++c) y[c] += yu[c];
        }
        const int ld = __shfl_down_sync(0xffffffffu, lr, 1);
        if (valid && (lane == 31 || ld != lr)) {
            const int i = rb + lr;
            const int rs = __ldg(tw_ptr + i), rend = __ldg(tw_ptr + i + 1);
            const int ps = eb + 32 * q, pe = min(ps + 32, ee);
            float *dst = rs <= ps ? slot + 12 * q : (rend >= pe ? slot + 12 * q + 6 : rowacc + 6 * lr);
#pragma unroll
            for (int c = 0; c < 6; ++c) dst[c] = y[c];
        }
    }
    return true;
}

// Component c of the off-diagonal part of (S^ x)_i for local row lr after
// split_passes and a __syncthreads: the row's segment sums in pass order
// (zero for a row without off-diagonal entries).
__device__ __forceinline__ float split_combine(int lr, int c, int rs, int rend, int eb, int ee, const float *slot,
                                               const float *rowacc) {
    float w = 0.f;
    if (rs >= rend) return w;
    for (int q = (rs - eb) >> 5; q <= (rend - 1 - eb) >> 5; ++q) {
        const int ps = eb + 32 * q, pe = min(ps + 32, ee);
        const float *src = rs <= ps ? slot + 12 * q : (rend >= pe ? slot + 12 * q + 6 : rowacc + 6 * lr);
        w += src[c];
    }
    return w;
}

// Component c of S^_ii x_i: x_i itself for block-Jacobi (S^_ii = I), else
// row c of the stored diagonal block times x_i.
__device__ __forceinline__ float split_diag(int i, int c, const float *x6, const float *__restrict__ Shd,
                                            int ident) {
    if (ident) return x6[c];
    const float *d = Shd + 36 * (int64_t)i + 6 * c;
    float w = 0.f;
#pragma unroll
    for (int k = 0; k < 6; ++k) w = __fmaf_rn(__ldg(d + k), x6[k], w);
    return w;
}

// Halo gather: for each halo camera the vector the SpMV applies (x = r for
// the prologue, else next_r of its record), and for the CTA's own rows the
// old r, w, s (own[lr][0..17]).
__device__ __forceinline__ void split_halo_fetch(const int *__restrict__ halo_col, int hb, int H, int hj0,
                                                 const float *rec, float *hx) {
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        const int j = h == (int)threadIdx.x ? hj0 : __ldg(halo_col + hb + h);
        const float4 *q = reinterpret_cast<const float4 *>(rec + (int64_t)SREC * j);
        float4 *d = reinterpret_cast<float4 *>(hx + HX * h);
#pragma unroll
        for (int k = 0; k < 5; ++k) cp_async16(d + k, q + k);
    }
}
// Each thread transforms, in place, the records it fetched (so no barrier is
// needed between the copies and this); own rows keep their whole record.
__device__ __forceinline__ void split_halo_apply(int H, int ob, int R, bool first, float a, float b, float *hx,
                                                 float *own) {
    static_assert(HX == SREC, "the halo area holds whole records");
    cp_async_wait_all();
    for (int h = threadIdx.x; h < H; h += blockDim.x) {
        const float4 *q = reinterpret_cast<const float4 *>(hx + HX * h);
        float t[20];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const float4 v = q[k];
            t[4 * k] = v.x; t[4 * k + 1] = v.y; t[4 * k + 2] = v.z; t[4 * k + 3] = v.w;
        }
        float x[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) x[k] = first ? t[k] : next_r(t[k], t[6 + k], t[12 + k], a, b);
        float4 *o = reinterpret_cast<float4 *>(hx + HX * h);
        o[0] = make_float4(x[0], x[1], x[2], x[3]);
        o[1] = make_float4(x[4], x[5], 0.f, 0.f);
        const int lr = h - ob;
        if (lr >= 0 && lr < R) {
            float4 *w4 = reinterpret_cast<float4 *>(own + 20 * lr);
#pragma unroll
            for (int k = 0; k < 5; ++k) w4[k] = make_float4(t[4 * k], t[4 * k + 1], t[4 * k + 2], t[4 * k + 3]);
        }
    }
}

// CG on S^ x^ = r^_0 (Chronopoulos-Gear), with per iteration k
//   p = r + beta p,  s = w + beta s,  x^ += alpha p,  r -= alpha s,  w = S^ r,
//   gamma = r.r, delta = w.r, beta' = gamma'/gamma,
//   alpha' = gamma' / (delta' - beta' gamma' / alpha),
// one phase per iteration: the halo gather, the SpMV passes, then a thread
// per (row, component) of the CTA's rows combines w_i and updates the row's
// own p, s, x^, r, w (a thread's first element keeps p, x^ and its row of H
// in registers across iterations).  The stop test uses the original
// residual norm ||H r^|| (block-Jacobi: ||L r^||).  One grid all-reduce of
// (gamma, delta, ||H r||^2) ends each phase.
__global__ void __launch_bounds__(SPLIT_WARPS * 32, SPLIT_CTAS_PER_SM) k_pcg_split(const int *__restrict__ cta_rows, const int *__restrict__ tw_ptr,
                                                      const uint32_t *__restrict__ tw_meta,
                                                      const int *__restrict__ meta_off,
                                                      const int *__restrict__ halo_ptr,
                                                      const int *__restrict__ halo_col,
                                                      const int *__restrict__ own_base, int slot_floats,
                                                      const float *__restrict__ Sh, const float *__restrict__ H,
                                                      const float *__restrict__ Shd, int diag_ident,
                                                      float *x, float *p, float *rec0, float *rec1, DevScalars *sc,
                                                      double *red, unsigned *bar, long long limit_cycles) {
    extern __shared__ __align__(16) float sdyn[];
    __shared__ uint64_t mbar[SPLIT_NBUF * SPLIT_WARPS];
    if (sc->done) return;
    const int rb = __ldg(cta_rows + blockIdx.x), re = __ldg(cta_rows + blockIdx.x + 1);
    const int eb = __ldg(tw_ptr + rb), ee = __ldg(tw_ptr + re);
    const int hb = __ldg(halo_ptr + blockIdx.x), NH = __ldg(halo_ptr + blockIdx.x + 1) - hb;
    const int ob = __ldg(own_base + blockIdx.x);
    const int R = re - rb, P = (ee - eb + 31) >> 5, wid = threadIdx.x >> 5;
    // dynamic shared memory: copy buffers | slots + row sums | halo | own records
    float *slot = sdyn + SPLIT_STAGE_BYTES / 4, *rowacc = slot + 12 * P;
    float *hx = slot + slot_floats, *own = hx + HX * NH;
    const int hj0 = (int)threadIdx.x < NH ? __ldg(halo_col + hb + threadIdx.x) : 0;
    SplitPipe pp{sdyn, mbar, Sh, tw_meta + __ldg(meta_off + blockIdx.x), eb, ee,
                 wid < P ? (P - 1 - wid) / SPLIT_WARPS + 1 : 0, 0u};
    if (threadIdx.x < SPLIT_NBUF * SPLIT_WARPS) mbar_init(&mbar[threadIdx.x], 1);
    fence_proxy_async();
    __syncthreads();
    if ((threadIdx.x & 31) == 0 && pp.m > 0)
        for (uint32_t q = 0; q < (uint32_t)SPLIT_NBUF; ++q) split_issue(pp, q);
    // this thread's first (row, component): p, x^, its row of H and the row's
    // entry range stay in registers
    const int u0 = threadIdx.x;
    const bool has0 = u0 < 6 * R;
    const int lr0 = u0 / 6, c0 = u0 - 6 * lr0;
    float p0 = 0.f, x0 = 0.f, h0[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    int rs0 = 0, re0 = 0;
    if (has0) {
#pragma unroll
        for (int k = 0; k < 6; ++k) h0[k] = __ldg(H + 36 * (int64_t)(rb + lr0) + 6 * c0 + k);
        rs0 = __ldg(tw_ptr + rb + lr0);
        re0 = __ldg(tw_ptr + rb + lr0 + 1);
    }
    unsigned gen = 0;
    // The recurrence's scalars live in thread 0, which decides alpha, beta and
    // the stop after each all-reduce and publishes them here.  They are
    // double-floats (the all-reduce's totals as they come): GB300's FP64 pipe
    // is slow enough that an FP64 recurrence on this critical path cost more
    // than a microsecond per iteration; FP64 is used once, for the threshold.
    __shared__ float2 sh_df[3 * SPLIT_WARPS];
    __shared__ int s_ctl;  // 0 go on, 1 stop, 2 not SPD, 3 timeout
    __shared__ int s_arok;
    __shared__ float s_ab[2];
    df32 gamma{0.f, 0.f}, delta{0.f, 0.f}, rr{0.f, 0.f}, rr0{0.f, 0.f}, gamma_prev{0.f, 0.f}, ga_prev{0.f, 0.f};
    float thr = 0.f;  // tol^2 r0^T r0: the stop threshold on r^T r
    int it = 0;
    const double tol2 = threadIdx.x == 0 ? sc->tol2 : 0.0;
    const int max_iters = threadIdx.x == 0 ? sc->max_iters : 0;
    // alpha = gamma / (delta - gamma (gamma / (gamma_prev alpha_prev))): the
    // difference (p^T S^ p, prone to cancellation) in double-float; alpha and
    // beta, applied in FP32, as FP32 quotients of the leading parts
    auto decide = [&](bool ok, const df32(&t)[3], bool first) {
        if (!ok) {
            s_ctl = 3;
            return;
        }
        if (first) {
            rr0 = t[2];
            thr = (float)(tol2 * df_to_double(rr0));
        } else {
            gamma_prev = gamma;
            ++it;
        }
        gamma = t[0];
        delta = t[1];
        rr = t[2];
        if (rr.hi <= thr || it >= max_iters) {
            s_ctl = 1;
            return;
        }
        const df32 den = it == 0 ? delta : df_sub(delta, df_mul(gamma, df_div(gamma, ga_prev)));
        const float alpha = den.hi > 0.f ? gamma.hi / den.hi : 0.f;
        const float beta = it == 0 ? 0.f : gamma.hi / gamma_prev.hi;
        ga_prev = df_mulf(gamma, alpha);
        if (!(den.hi > 0.f) || !(alpha > 0.f) || !(alpha < 1e30f)) {  // p^T S^ p <= 0 or not finite
            s_ctl = 2;
            return;
        }
        s_ctl = 0;
        s_ab[0] = alpha;
        s_ab[1] = beta;
    };
    auto leave = [&]() {
        if (has0) x[6 * (int64_t)(rb + lr0) + c0] = x0;
        cp_async_wait_all();
        split_drain(pp, limit_cycles);
    };
    // phase timing (thread 0 of each CTA, profile >= 2): passes, combine, all-reduce
    const bool prof = sc->prof_on != 0 && threadIdx.x == 0;
    unsigned long long t_pass = 0, t_comb = 0, t_red = 0, t0 = 0, t1 = 0, t2 = 0;
    {  // prologue: w_0 = S^ r_0 and the dot products of iteration 0
        split_halo_fetch(halo_col, hb, NH, hj0, rec0, hx);
        split_halo_apply(NH, ob, R, true, 0.f, 0.f, hx, own);
        __syncthreads();
        const bool ok = __syncthreads_and(split_passes(pp, rb, tw_ptr, hx, slot, rowacc, &sc->err, limit_cycles));
        if (!ok) {
            leave();
            return;
        }
        RunSum<float> gp, dp, rp;
        for (int u = threadIdx.x; u < 6 * R; u += blockDim.x) {
            const int lr = u / 6, c = u - 6 * lr, i = rb + lr;
            const int rs = u == u0 ? rs0 : __ldg(tw_ptr + i), rend = u == u0 ? re0 : __ldg(tw_ptr + i + 1);
            const float *r6 = hx + HX * (ob + lr);
            const float wc = split_combine(lr, c, rs, rend, eb, ee, slot, rowacc) + split_diag(i, c, r6, Shd, diag_ident);
            rec0[(int64_t)SREC * i + 6 + c] = wc;
            float hr = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                hr = __fmaf_rn(u == u0 ? h0[k] : __ldg(H + 36 * (int64_t)i + 6 * c + k), r6[k], hr);
            const float rc = r6[c];
            gp.add(rc * rc);
            dp.add(wc * rc);
            rp.add(hr * hr);
        }
        df32 v[3] = {{gp.s, gp.c}, {dp.s, dp.c}, {rp.s, rp.c}};
        block_sum_df<3>(v, sh_df);
        df32 t[3];
        const bool ok2 = grid_allreduce_df<3>(v, red, gen++, bar, &sc->err, limit_cycles, t, sh_df, &s_arok,
                                              [&]() { split_halo_fetch(halo_col, hb, NH, hj0, rec0, hx); });
        if (threadIdx.x == 0) decide(ok2, t, true);
        __syncthreads();
    }
    uint32_t par = 0;  // parity of the current iteration's records
    for (;;) {
        const int ctl = s_ctl;
        if (ctl != 0) {
            if (threadIdx.x == 0) {
                if (blockIdx.x == 0 && ctl != 3) {
                    if (ctl == 2) sc->err = (int)BA_ERR_NOT_SPD;
                    sc->iters = it;
                    sc->rr = df_to_double(rr);
                    sc->rr0 = df_to_double(rr0);
                    sc->rz = df_to_double(gamma);
                    sc->done = 1;
                }
                if (prof) {
                    atomicAdd(&sc->ph[0], (double)t_pass);
                    atomicAdd(&sc->ph[1], (double)t_comb);
                    atomicAdd(&sc->ph[2], (double)t_red);
                    atomicAdd(&sc->ph[3], (double)it);
                    atomicMax(&sc->ph_work_max, t_pass + t_comb);
                }
            }
            leave();
            return;
        }
        const float a = s_ab[0], b = s_ab[1];
        float *rn = par ? rec0 : rec1;
        if (prof) t0 = global_ns();
        split_halo_apply(NH, ob, R, false, a, b, hx, own);
        __syncthreads();
        const bool ok = __syncthreads_and(split_passes(pp, rb, tw_ptr, hx, slot, rowacc, &sc->err, limit_cycles));
        if (!ok) {
            leave();
            return;
        }
        if (prof) t1 = global_ns();
        RunSum<float> gp, dp, rp;
        for (int u = threadIdx.x; u < 6 * R; u += blockDim.x) {
            const int lr = u / 6, c = u - 6 * lr, i = rb + lr, e = 6 * i + c;
            const bool first = u == u0;
            const int rs = first ? rs0 : __ldg(tw_ptr + i), rend = first ? re0 : __ldg(tw_ptr + i + 1);
            const float *rnew = hx + HX * (ob + lr);  // this row's new residual (all six components)
            const float w_e = split_combine(lr, c, rs, rend, eb, ee, slot, rowacc) + split_diag(i, c, rnew, Shd, diag_ident);
            const float *o6 = own + 20 * lr;
            const float r_e = rnew[c], rold = o6[c], wold = o6[6 + c], sold = o6[12 + c];
            const float pval = __fmaf_rn(b, first ? p0 : __ldcg(p + e), rold);
            const float sval = __fmaf_rn(b, sold, wold);
            const float xval = __fmaf_rn(a, pval, first ? x0 : __ldcg(x + e));
            if (first) {
                p0 = pval;
                x0 = xval;
            } else {
                p[e] = pval;
                x[e] = xval;
            }
            float *o = rn + (int64_t)SREC * i;
            o[c] = r_e;
            o[6 + c] = w_e;
            o[12 + c] = sval;
            float hr = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k)
                hr = __fmaf_rn(first ? h0[k] : __ldg(H + 36 * (int64_t)i + 6 * c + k), rnew[k], hr);
            gp.add(r_e * r_e);
            dp.add(w_e * r_e);
            rp.add(hr * hr);
        }
        df32 v[3] = {{gp.s, gp.c}, {dp.s, dp.c}, {rp.s, rp.c}};
        block_sum_df<3>(v, sh_df);
        if (prof) t2 = global_ns();
        df32 t[3];
        const bool ok2 = grid_allreduce_df<3>(v, red, gen++, bar, &sc->err, limit_cycles, t, sh_df, &s_arok,
                                              [&]() { split_halo_fetch(halo_col, hb, NH, hj0, rn, hx); });
        if (threadIdx.x == 0) {
            if (prof) {
                const unsigned long long t3 = global_ns();
                t_pass += t1 - t0;
                t_comb += t2 - t1;
                t_red += t3 - t2;
            }
            decide(ok2, t, false);
        }
        __syncthreads();
        par ^= 1u;
    }
}

// x64 (+)= G x^ per camera (the solution of the original system)
__global__ void k_acc64_split(int n, const float *__restrict__ G, const float *__restrict__ xh, double *x64,
                              int first) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 6 * n) return;
    const int i = e / 6, a = e - 6 * i;
    const float *g = G + 36 * (int64_t)i + 6 * a;
    float t = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) t = __fmaf_rn(__ldg(g + c), __ldcg(xh + 6 * i + c), t);
    x64[e] = (first ? 0.0 : x64[e]) + (double)t;
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

// FP32 systems whose stored blocks exceed this many bytes run the product
// that reads each block once (the second, transposed read of the two-sided
// product would come from DRAM); smaller ones keep the deterministic
// two-sided product, whose second read hits L2.
constexpr int64_t ONCE_MIN_BYTES = 64ll << 20;

template <typename T, bool ONCE>
static cudaError_t pcg_loop_T(ba_problem *p) {
    int blocks_per_sm = 0, n_sm = 0;
    cudaError_t e;
    if ((e = occupancy((const void *)k_pcg_persist<T, ONCE>, 256, 0, &blocks_per_sm, &n_sm)) != cudaSuccess) return e;
    if (blocks_per_sm > 2) blocks_per_sm = 2;
    if (blocks_per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // enough warps for one block row each, at most what is co-resident
    int64_t want = ((int64_t)p->n * 32 + 255) / 256;
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)blocks_per_sm * n_sm);
    // armed test of the timeout path: the counter starts at -1 (one arrival short)
    const long long test_limit = p->test_wait_limit;
    p->test_wait_limit = 0;
    if ((e = cudaMemsetAsync(p->counters + 14, test_limit > 0 ? 0xFF : 0, sizeof(unsigned), p->st)) != cudaSuccess)
        return e;
    if ((e = cudaMemsetAsync(p->counters + 15, 0, sizeof(unsigned), p->st)) != cudaSuccess) return e;
    int n = p->n;
    const int *twp = p->tw_ptr, *rp = p->row_ptr, *cl = p->col;
    const int2 *twe = p->tw_ent;
    const T *S = (const T *)p->sv.S, *Mi = (const T *)p->sv.Minv;
    T *y = (T *)p->sv.pv[0], *r = (T *)p->sv.pv[1], *z = (T *)p->sv.pv[2], *d0 = (T *)p->sv.pv[3], *d1 = (T *)p->sv.pv[4];
    T *q = (T *)p->sv.pv[5], *r1 = (T *)p->sv.pv[6], *q1 = (T *)p->sv.pv[7];
    DevScalars *sc = p->sc;
    double *red = p->red;
    unsigned *bar = p->counters + 14;
    long long limit = test_limit > 0 ? test_limit : 4000000000LL;  // ~2 s of SM clock per barrier wait
    void *args[] = {&n, &twp, &twe, &rp, &cl, &S, &Mi, &y, &r, &r1, &z, &d0, &d1, &q, &q1, &sc, &red, &bar, &limit};
    return cudaLaunchCooperativeKernel((const void *)k_pcg_persist<T, ONCE>, dim3(grid), dim3(256), args, 0, p->st);
}

cudaError_t launch_pcg_loop(ba_problem *p) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_LOOP, &ev);
    cudaError_t e = !p->sv.f32 ? pcg_loop_T<double, false>(p)
                    : (p->nnzb * (int64_t)BW * 4 > ONCE_MIN_BYTES ? pcg_loop_T<float, true>(p)
                                                                 : pcg_loop_T<float, false>(p));
    ktimer_end(p, K_PCG_LOOP, ev);
    p->launches += 1;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

static cudaError_t ensure_xs(ba_problem *p) {
    if (p->xs) return cudaSuccess;
    void *v = nullptr;
    const size_t bytes = (size_t)p->n * 6 * sizeof(float2);
    cudaError_t e = cudaMalloc(&v, bytes);
    if (e != cudaSuccess) return e;
    p->xs = (float2 *)v;
    p->allocs.push_back(v);
    p->dev_bytes += bytes;
    return cudaSuccess;
}

// from_x64: r64 = b - S x64; else r64 = b (x64 = 0).
cudaError_t launch_resid64(ba_problem *p, bool from_x64) {
    cudaEvent_t ev;
    ktimer_begin(p, K_RESID64, &ev);
    if (from_x64) {
        const int gs = grid_for((int64_t)p->n * 32, 256, 152 * 8);
        // FP32 problems: double-float products on the FP32 pipe; FP64
        // problems keep FP64 arithmetic (their S is FP64)
        if (p->fp32) {
            cudaError_t e = ensure_xs(p);
            if (e != cudaSuccess) return e;
            const int64_t cnt = (int64_t)p->n * 6;
            k_split_x<<<grid_for(cnt, 256, VEC_CAP), 256, 0, p->st>>>(cnt, p->x64, p->xs);
            k_spmv_df<<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const float *)p->S, p->xs, p->q64);
            p->launches += 1;
        } else {
            k_spmv64<double><<<gs, 256, 0, p->st>>>(p->n, p->tw_ptr, p->tw_ent, (const double *)p->S, p->x64, p->q64);
        }
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

static cudaError_t split_alloc(ba_problem *p) {
    cudaError_t e = cudaSuccess;
    auto al = [&](float **q, size_t cnt) {
        if (e == cudaSuccess && !*q) {
            void *v = nullptr;
            e = cudaMalloc(&v, cnt * sizeof(float));
            if (e == cudaSuccess) {
                *q = (float *)v;
                p->allocs.push_back(v);
                p->dev_bytes += cnt * sizeof(float);
            }
        }
    };
    al(&p->Gs, (size_t)p->n * 36);
    al(&p->Hs, (size_t)p->n * 36);
    al(&p->Shd, (size_t)p->n * 36);
    const size_t E = std::max<size_t>(1, (size_t)(2 * p->nnzb - 2 * p->n));  // entries without the diagonal
    al(&p->Sh, E * BW);
    al(&p->srec, (size_t)2 * SREC * p->n);
    return e;
}

cudaError_t launch_split_prepare(ba_problem *p, bool from_minv) {
    cudaError_t e = split_alloc(p);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev;
    ktimer_begin(p, K_SPLIT_PREP, &ev);
    // the factors: a thread per camera in FP64, 32 to a CTA so that the
    // cameras spread over every SM's FP64 units; S^: a warp per block row
    const int nb = (p->n + 31) / 32, ns = (int)(((int64_t)p->n * 32 + 127) / 128);
    if (p->fp32) {
        k_split_factor<float><<<nb, 32, 0, p->st>>>(p->n, p->row_ptr, (const float *)p->S, (const float *)p->Minv,
                                                     from_minv ? 1 : 0, p->Gs, p->Hs, p->Shd, p->sc);
        k_split_scale<float><<<ns, 128, 0, p->st>>>(p->n, p->tws_ptr, p->tws_ent, (const float *)p->S, p->Gs, p->Sh);
    } else {
        k_split_factor<double><<<nb, 32, 0, p->st>>>(p->n, p->row_ptr, (const double *)p->S,
                                                      (const double *)p->Minv, from_minv ? 1 : 0, p->Gs, p->Hs,
                                                      p->Shd, p->sc);
        k_split_scale<double><<<ns, 128, 0, p->st>>>(p->n, p->tws_ptr, p->tws_ent, (const double *)p->S, p->Gs, p->Sh);
    }
    ktimer_end(p, K_SPLIT_PREP, ev);
    p->launches += 2;
    return cudaGetLastError();
}

// Work partition of the split CG, made once per problem on the host: the
// grid size; each CTA's row range (contiguous rows, about equal entries + a
// fixed cost per row); its halo (the sorted distinct columns of its entries;
// its own rows are one contiguous stretch of it, starting at own_base); the
// packed metadata of every entry (local row | halo index << 16), laid out
// per CTA from a 16-byte aligned offset; and the dynamic shared memory of
// the busiest CTA (copy buffers, pass slots and row sums, halo vectors, own
// records).  Problems that need more than 200 KB in a CTA keep the standard
// recurrence (split_grid < 0).
static cudaError_t split_partition(ba_problem *p) {
    if (p->split_grid != 0) return cudaSuccess;
    cudaError_t e;
    const int n = p->n;
    std::vector<int32_t> twp0(n + 1);
    if ((e = cudaMemcpy(twp0.data(), p->tw_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    std::vector<int2> twe0(twp0[n]);
    if (twp0[n] &&
        (e = cudaMemcpy(twe0.data(), p->tw_ent, twp0[n] * sizeof(int2), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return e;
    // the split CG's entry lists: the two-sided lists without the diagonal
    // block (its product is added in the row combine: S^_ii x_i)
    std::vector<int32_t> twp(n + 1, 0);
    std::vector<int2> twe;
    twe.reserve(twp0[n]);
    for (int i = 0; i < n; ++i) {
        for (int32_t t = twp0[i]; t < twp0[i + 1]; ++t)
            if (twe0[t].y != i) twe.push_back(twe0[t]);
        twp[i + 1] = (int32_t)twe.size();
    }
    const int64_t E = twp[n];
    if (twe.empty()) twe.push_back(make_int2(0, 0));  // a valid (unused) upload
    int dev = 0, n_sm = 0, bps = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    constexpr int SMEM_MAX = 226 * 1024, ROW_COST = 8;  // 227 KB per CTA less the static part
    if ((e = cudaFuncSetAttribute(k_pcg_split, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_MAX)) != cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_pcg_split, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
    auto unavailable = [&]() {
        p->split_grid = -1;
        return cudaSuccess;
    };
    std::vector<int32_t> rows, hptr, hcol, obase;
    size_t smem = SPLIT_STAGE_BYTES;
    int slot_floats = 0, G = 0;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_pcg_split, SPLIT_WARPS * 32, smem)) != cudaSuccess) return e;
        bps = std::min(bps, SPLIT_CTAS_PER_SM);
        if (bps < 1) return unavailable();
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)bps * n_sm, (E + 255) / 256));
        if (g == G) break;
        G = g;
        rows.assign(G + 1, n);
        rows[0] = 0;
        const double total = (double)E + (double)ROW_COST * n;
        int c = 1;
        double acc = 0.0;
        for (int i = 0; i < n && c < G; ++i) {
            acc += (double)(twp[i + 1] - twp[i]) + ROW_COST;
            while (c < G && acc >= total * c / G) rows[c++] = i + 1;
        }
        // A CTA's passes are shared round-robin by its warps, so the slowest
        // warp of a CTA with 16k + 1 passes takes k + 1: cap every CTA at the
        // fewest whole rounds of passes a contiguous partition allows (the
        // greedy count decides) and move boundary rows off the CTAs above it.
        {
            const int64_t round = 32LL * SPLIT_WARPS;
            auto fits = [&](int64_t cap) {
                int cnt = 1;
                int64_t cur = 0;
                for (int i = 0; i < n; ++i) {
                    const int64_t r = twp[i + 1] - twp[i];
                    if (r > cap) return false;
                    if (cur + r > cap) {
                        ++cnt;
                        cur = 0;
                    }
                    cur += r;
                }
                return cnt <= G;
            };
            int64_t cap = std::max<int64_t>(1, (E + round * G - 1) / (round * G)) * round;
            while (cap < E && !fits(cap)) cap += round;
            auto ent = [&](int k) { return (int64_t)twp[rows[k + 1]] - twp[rows[k]]; };
            for (int sweep = 0; sweep < 4; ++sweep) {
                bool over = false;
                for (int k = 0; k + 1 < G; ++k)  // forward: last rows to the next CTA
                    while (ent(k) > cap && rows[k + 1] > rows[k] + 1) --rows[k + 1];
                for (int k = G - 1; k > 0; --k)  // backward: first rows to the previous CTA
                    while (ent(k) > cap && rows[k] < rows[k + 1] - 1) ++rows[k];
                for (int k = 0; k < G; ++k) over = over || ent(k) > cap;
                if (!over) break;
            }
        }
        // halos
        hptr.assign(G + 1, 0);
        hcol.clear();
        obase.assign(G, 0);
        int Hmax = 0, Rmax = 0;
        slot_floats = 0;
        std::vector<int32_t> cols;
        for (int k = 0; k < G; ++k) {
            cols.clear();
            for (int64_t t = twp[rows[k]]; t < twp[rows[k + 1]]; ++t) cols.push_back(twe[t].y);
            for (int i = rows[k]; i < rows[k + 1]; ++i) cols.push_back(i);  // own rows (their diagonal products)
            std::sort(cols.begin(), cols.end());
            cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
            obase[k] = (int32_t)(std::lower_bound(cols.begin(), cols.end(), rows[k]) - cols.begin());
            hcol.insert(hcol.end(), cols.begin(), cols.end());
            hptr[k + 1] = (int32_t)hcol.size();
            const int R = rows[k + 1] - rows[k];
            const int64_t P = ((int64_t)twp[rows[k + 1]] - twp[rows[k]] + 31) / 32;
            Hmax = std::max(Hmax, (int)cols.size());
            Rmax = std::max(Rmax, R);
            slot_floats = std::max(slot_floats, (int)(12 * P + 6 * R + 3) & ~3);
        }
        smem = SPLIT_STAGE_BYTES +
               ((size_t)slot_floats + (size_t)HX * Hmax + 20 * (size_t)Rmax) * sizeof(float);
        if (smem > (size_t)SMEM_MAX || Hmax > 0xFFFF || Rmax > 0xFFFE) return unavailable();
    }
    // the occupancy at the final shared-memory size must keep the grid resident
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_pcg_split, SPLIT_WARPS * 32, smem)) != cudaSuccess) return e;
    if (G < 1 || (int64_t)bps * n_sm < G) return unavailable();
    // packed entry metadata, per CTA from a 16-byte aligned offset (+ padding
    // for the rounded-up copy of a CTA's last pass)
    std::vector<int32_t> moff(G);
    int64_t mtotal = 0;
    for (int k = 0; k < G; ++k) {
        moff[k] = (int32_t)mtotal;
        mtotal += ((int64_t)twp[rows[k + 1]] - twp[rows[k]] + 3) & ~3;
    }
    mtotal += 4;
    std::vector<uint32_t> meta(mtotal, 0u);
    for (int k = 0; k < G; ++k) {
        const int32_t *hc = hcol.data() + hptr[k];
        const int H = hptr[k + 1] - hptr[k];
        for (int i = rows[k]; i < rows[k + 1]; ++i)
            for (int64_t t = twp[i]; t < twp[i + 1]; ++t) {
                const uint32_t h = (uint32_t)(std::lower_bound(hc, hc + H, twe[t].y) - hc);
                meta[moff[k] + (t - twp[rows[k]])] = (uint32_t)(i - rows[k]) | (h << 16);
            }
    }
    std::vector<std::pair<void **, std::pair<const void *, size_t>>> up = {
        {(void **)&p->tws_ptr, {twp.data(), twp.size() * sizeof(int32_t)}},
        {(void **)&p->tws_ent, {twe.data(), twe.size() * sizeof(int2)}},
        {(void **)&p->cta_rows, {rows.data(), rows.size() * sizeof(int32_t)}},
        {(void **)&p->tw_meta, {meta.data(), meta.size() * sizeof(uint32_t)}},
        {(void **)&p->meta_off, {moff.data(), moff.size() * sizeof(int32_t)}},
        {(void **)&p->halo_ptr, {hptr.data(), hptr.size() * sizeof(int32_t)}},
        {(void **)&p->halo_col, {hcol.data(), std::max<size_t>(hcol.size(), 1) * sizeof(int32_t)}},
        {(void **)&p->own_base, {obase.data(), obase.size() * sizeof(int32_t)}}};
    for (auto &u : up) {
        void *d = nullptr;
        if ((e = cudaMalloc(&d, u.second.second)) != cudaSuccess) return e;
        p->allocs.push_back(d);
        p->dev_bytes += u.second.second;
        if ((e = cudaMemcpy(d, u.second.first, u.second.second, cudaMemcpyHostToDevice)) != cudaSuccess) return e;
        *u.first = d;
    }
    p->split_slot_floats = slot_floats;
    p->split_smem = smem;
    p->split_grid = G;
    return cudaSuccess;
}

bool split_available(ba_problem *p) {
    if (split_partition(p) != cudaSuccess) {
        cudaGetLastError();
        p->split_grid = -1;
    }
    return p->split_grid > 0;
}

// vectors: pv[0] x^, pv[2] p of the active FP32 view; records in p->srec
cudaError_t launch_split_init(ba_problem *p, const float *rhs, double tol, int max_iters) {
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_INIT, &ev);
    float **v = (float **)p->sv.pv;
    float *rec0 = p->srec, *rec1 = p->srec + (size_t)SREC * p->n;
    k_split_init<<<grid_for(p->n, 256, VEC_CAP), 256, 0, p->st>>>(p->n, rhs, p->Gs, rec0, rec1, v[0], v[2], p->sc,
                                                                  tol * tol, max_iters, p->opt.profile >= 2);
    ktimer_end(p, K_PCG_INIT, ev);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_pcg_split(ba_problem *p) {
    cudaEvent_t ev;
    cudaError_t e = cudaSuccess;
    if (!p->ar_bar) {
        void *v = nullptr;
        if ((e = cudaMalloc(&v, AR_SUB * 32 * sizeof(unsigned))) != cudaSuccess) return e;
        p->ar_bar = (unsigned *)v;
        p->allocs.push_back(v);
        p->dev_bytes += AR_SUB * 32 * sizeof(unsigned);
    }
    ktimer_begin(p, K_PCG_LOOP, &ev);
    // armed test of the timeout path: every counter starts at -1, so each one
    // ends a call one arrival short of its target and the wait runs out
    const long long test_limit = p->test_wait_limit;
    p->test_wait_limit = 0;
    e = cudaMemsetAsync(p->ar_bar, test_limit > 0 ? 0xFF : 0, AR_SUB * 32 * sizeof(unsigned), p->st);
    if (e == cudaSuccess) {
        const int *cr = p->cta_rows, *twp = p->tws_ptr, *mo = p->meta_off, *hp = p->halo_ptr, *hc = p->halo_col,
                  *ob = p->own_base;
        const uint32_t *meta = p->tw_meta;
        int sf = p->split_slot_floats;
        const float *Sh = p->Sh, *H = p->Hs, *Shd = p->Shd;
        int ident = p->minv_learned ? 0 : 1;
        float **v = (float **)p->sv.pv;
        float *x = v[0], *pp = v[2];
        float *rec0 = p->srec, *rec1 = p->srec + (size_t)SREC * p->n;
        DevScalars *sc = p->sc;
        double *red = p->red;
        unsigned *bar = p->ar_bar;
        long long limit = test_limit > 0 ? test_limit : 4000000000LL;  // ~2 s of SM clock per wait
        void *args[] = {&cr, &twp, &meta, &mo, &hp, &hc, &ob, &sf, &Sh, &H, &Shd, &ident, &x, &pp, &rec0, &rec1, &sc,
                        &red, &bar, &limit};
        e = cudaLaunchCooperativeKernel((const void *)k_pcg_split, dim3(p->split_grid), dim3(SPLIT_WARPS * 32), args,
                                        p->split_smem, p->st);
    }
    ktimer_end(p, K_PCG_LOOP, ev);
    p->launches += 1;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_accumulate_split(ba_problem *p, bool first) {
    const int cnt = p->n * 6;
    k_acc64_split<<<(cnt + 255) / 256, 256, 0, p->st>>>(p->n, p->Gs, (const float *)p->sv.pv[0], p->x64,
                                                        first ? 1 : 0);
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
