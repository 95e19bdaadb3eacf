// The reduced camera system in three storage formats and a y = S x kernel
// for each, for the storage comparison of Sec. 4 (Table 1, Eqs. 8-10):
//   BSMC      the library's own: the upper-triangle 6x6 blocks with the full
//             diagonal block first in each row (Fig. 4); the product reads
//             every off-diagonal block twice, once as S_ij x_j for row i and
//             once as S_ij^T x_i for row j (the two-sided entry lists), so no
//             atomics are needed and the result is deterministic;
//   BSR_FULL  block CSR of the whole symmetric matrix: both triangles stored,
//             one column index per block (what a general block-sparse format
//             holds without exploiting symmetry);
//   CSR       scalar CSR of the whole matrix (Eq. 8): a value and a column
//             index per non-zero element, a start per scalar row.
// The full formats are built on the device from the two-sided entry lists
// (the entry order of row i: its stored blocks, then the transposed blocks
// of its column), so all three products sum each row's terms in the same
// block order.
#include <vector>

#include "device_util.cuh"

namespace ba {

// Full BSR values: entry e of the two-sided lists is its stored block, or
// that block transposed where the entry is flagged.
template <typename T>
__global__ void k_build_bsr(int64_t E, const int2 *__restrict__ tw_ent, const T *__restrict__ S, T *__restrict__ val,
                            int *__restrict__ bcol) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < E * BW; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = x / BW;
        const int q = (int)(x - e * BW), r = q / 6, c = q - 6 * r;
        const int2 en = tw_ent[e];
        const int64_t blk = en.x & 0x7fffffff;
        val[x] = en.x < 0 ? S[blk * BW + 6 * c + r] : S[blk * BW + q];
        if (q == 0) bcol[e] = en.y;
    }
}

// Scalar CSR from the full BSR: block row i with deg_i blocks gives scalar
// rows 6i + a (a = 0..5) of 6 deg_i elements each, in block order then
// column order within the block.
__global__ void k_build_csr_ptr(int n, const int *__restrict__ tw_ptr, int *__restrict__ rptr) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r > 6 * n) return;
    if (r == 6 * n) {
        rptr[r] = BW * tw_ptr[n];
        return;
    }
    const int i = r / 6, a = r - 6 * i;
    const int deg = tw_ptr[i + 1] - tw_ptr[i];
    rptr[r] = BW * tw_ptr[i] + 6 * a * deg;
}
template <typename T>
__global__ void k_build_csr(int n, int64_t E, const int *__restrict__ tw_ptr, const T *__restrict__ bval,
                            const int *__restrict__ bcol, int *__restrict__ ccol, T *__restrict__ cval) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < E * BW; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = x / BW;
        const int q = (int)(x - e * BW), a = q / 6, b = q - 6 * a;
        int lo = 0, hi = n;  // the block row of entry e: tw_ptr[i] <= e < tw_ptr[i + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tw_ptr[mid] <= e) lo = mid; else hi = mid;
        }
        const int i = lo, t0 = tw_ptr[i], deg = tw_ptr[i + 1] - t0;
        const int64_t at = (int64_t)BW * t0 + (int64_t)6 * a * deg + 6 * (e - t0) + b;
        cval[at] = bval[x];
        ccol[at] = 6 * bcol[e] + b;
    }
}

// y = S x over blocks, a warp per block row: lane l takes the row's blocks
// l, l + 32, l + 64, ... two at a time (both loads in flight together), each
// applies its 6x6 block to x_j, and a shuffle sum joins the six components.  TWO_SIDED: the BSMC entry lists
// (block index with the transpose flag, column); else the full BSR (block
// e of the row at val + e * 36, column bcol[e]).
template <typename T, bool TWO_SIDED>
__global__ void __launch_bounds__(256) k_spmv_blocks(int n, const int *__restrict__ rptr, const int2 *__restrict__ ent,
                                                     const int *__restrict__ bcol, const T *__restrict__ val,
                                                     const T *__restrict__ x, T *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n; i += nw) {
        const int tb = __ldg(rptr + i), te = __ldg(rptr + i + 1);
        T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        auto entry = [&](int t, int64_t &blk, int &j, bool &tr) {
            if (TWO_SIDED) {
                const int2 en = __ldg(ent + t);
                blk = en.x & 0x7fffffff;
                j = en.y;
                tr = en.x < 0;
            } else {
                blk = t;
                j = __ldg(bcol + t);
                tr = false;
            }
        };
        for (int t0 = tb + lane; t0 < te; t0 += 64) {
            const int t1 = t0 + 32;
            const bool has1 = t1 < te;
            int64_t ba, bb;
            int ja, jb;
            bool ta, tb1;
            entry(t0, ba, ja, ta);
            entry(has1 ? t1 : t0, bb, jb, tb1);
            T va[36], vb[36], xa[6], xb[6];
            load_block<T, T>(val + ba * BW, va);
            load_block<T, T>(val + bb * BW, vb);
            load6(x + 6 * (int64_t)ja, xa);
            load6(x + 6 * (int64_t)jb, xb);
            block_apply<T>(va, xa, ta, acc);
            if (has1) block_apply<T>(vb, xb, tb1, acc);
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum(acc[c]);
        if (lane < 6) {
            T out = acc[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) out = acc[c];
            y[6 * (int64_t)i + lane] = out;
        }
    }
}

// Vector reductions into an L2-resident result (sm_90 and later).
__device__ __forceinline__ void red_add2(float *a, float u, float v) {
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(a), "f"(u), "f"(v) : "memory");
}
__device__ __forceinline__ void red_add2(double *a, double u, double v) {
    atomicAdd(a, u);
    atomicAdd(a + 1, v);
}

// The transposed product S_ij^T x_i of a block added into y_j (6 values,
// 8-byte aligned): two vector reductions, the 16-byte one on the aligned half.
__device__ __forceinline__ void red_add4(float *a, float u0, float u1, float u2, float u3) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(a), "f"(u0), "f"(u1), "f"(u2), "f"(u3)
                 : "memory");
}
__device__ __forceinline__ void red_add6(float *yj, const float (&t)[6]) {
    if ((reinterpret_cast<uintptr_t>(yj) & 15u) == 0) {
        red_add4(yj, t[0], t[1], t[2], t[3]);
        red_add2(yj + 4, t[4], t[5]);
    } else {
        red_add2(yj, t[0], t[1]);
        red_add4(yj + 2, t[2], t[3], t[4], t[5]);
    }
}
__device__ __forceinline__ void red_add6(double *yj, const double (&t)[6]) {
#pragma unroll
    for (int c = 0; c < 6; ++c) atomicAdd(yj + c, t[c]);
}

// y += S x over BSMC reading every stored block once: a warp per block row i
// takes the row's stored blocks (i, j >= i; contiguous in memory) two at a
// time per lane, adds S_ij x_j to its row sum and, for j > i, S_ij^T x_i
// into y_j with vector reductions; the row sum joins y_i the same way (other
// rows add to it concurrently).  y must be zero on entry and 16-byte
// aligned.  The transposed product of Sec. 6.2 (Fig. 13) as the paper
// describes it: each block read once and its two results added where they
// belong.  The order in which y's terms are added is not fixed
// (floating-point reductions), so results may differ from run to run in the
// last bits.
template <typename T>
__global__ void __launch_bounds__(256) k_spmv_bsmc_once(int n, const int *__restrict__ row_ptr,
                                                        const int *__restrict__ col, const T *__restrict__ val,
                                                        const T *__restrict__ x, T *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n; i += nw) {
        const int tb = __ldg(row_ptr + i), te = __ldg(row_ptr + i + 1);
        T xi[6];
        load6(x + 6 * (int64_t)i, xi);
        T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        for (int t0 = tb + lane; t0 < te; t0 += 64) {
            const int t1 = t0 + 32;
            const bool has1 = t1 < te;
            const int ja = __ldg(col + t0), jb = __ldg(col + (has1 ? t1 : t0));
            T va[36], vb[36], xa[6], xb[6];
            load_block<T, T>(val + (int64_t)t0 * BW, va);
            load_block<T, T>(val + (int64_t)(has1 ? t1 : t0) * BW, vb);
            load6(x + 6 * (int64_t)ja, xa);
            load6(x + 6 * (int64_t)jb, xb);
            block_apply<T>(va, xa, false, acc);
            if (has1) block_apply<T>(vb, xb, false, acc);
            if (ja != i) {
                T tr[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                block_apply<T>(va, xi, true, tr);
                red_add6(y + 6 * (int64_t)ja, tr);
            }
            if (has1 && jb != i) {
                T tr[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
                block_apply<T>(vb, xi, true, tr);
                red_add6(y + 6 * (int64_t)jb, tr);
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum(acc[c]);
        if (lane < 6) {
            T out = acc[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) out = acc[c];
            atomicAdd(y + 6 * (int64_t)i + lane, out);
        }
    }
}

// y = S x over scalar CSR, a warp per scalar row (the row's values and
// column indices read coalesced), a shuffle sum per row.
template <typename T>
__global__ void __launch_bounds__(256) k_spmv_csr(int rows, const int *__restrict__ rptr, const int *__restrict__ ccol,
                                                  const T *__restrict__ cval, const T *__restrict__ x,
                                                  T *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int r = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); r < rows; r += nw) {
        const int kb = __ldg(rptr + r), ke = __ldg(rptr + r + 1);
        T acc = T(0);
        int k = kb + lane;
        for (; k + 96 < ke; k += 128) {  // four elements per lane in flight
            const int c0 = __ldg(ccol + k), c1 = __ldg(ccol + k + 32), c2 = __ldg(ccol + k + 64),
                      c3 = __ldg(ccol + k + 96);
            const T v0 = __ldg(cval + k), v1 = __ldg(cval + k + 32), v2 = __ldg(cval + k + 64),
                    v3 = __ldg(cval + k + 96);
            acc += v0 * __ldg(x + c0);
            acc += v1 * __ldg(x + c1);
            acc += v2 * __ldg(x + c2);
            acc += v3 * __ldg(x + c3);
        }
        for (; k < ke; k += 32) acc += __ldg(cval + k) * __ldg(x + __ldg(ccol + k));
        acc = warp_sum(acc);
        if (lane == 0) y[r] = acc;
    }
}

// Implicit (matrix-free) y = S x from the stored linearization, without the
// aggregated RCS (the next step the paper states for its cluster design):
//   y_i = (U_i + lambda clamp(diag U_i)) x_i
//         - sum_{a in cam i} J_c,a^T J_p,a V_k^-1 sum_{b in track k} J_p,b^T J_c,b x_cam(b)
// Phase A, a thread per point k: s_a = J_c,a x_cam(a) for its observations,
// t_k = sum_a J_p,a^T s_a, u_k = V_k^-1 t_k = L^-T L^-1 t_k (the per-point
// factor of the last RCS formation, same lambda), w_a = s_a - J_p,a u_k.
// Phase B, a warp per camera over its observations (camera-major index):
// y_i = sum_a J_c,a^T w_a + lambda clamp(diag U_i) x_i, with diag U_i =
// sum_a diag(J_c,a^T J_c,a) formed in the same pass.  Fixed orders: the
// result is deterministic.
// The vector the product applies, camera j's six entries: a plain x, or the
// PCG direction d = z + beta d_old formed on the fly.
template <typename T>
struct PlainX {
    const T *x;
    __device__ __forceinline__ void operator()(int64_t j, T (&v)[6]) const { load6(x + 6 * j, v); }
};
template <typename T>
struct PcgDir {
    const T *z, *dold;
    T beta;
    __device__ __forceinline__ void operator()(int64_t j, T (&v)[6]) const {
        T d[6];
        load6(z + 6 * j, v);
        load6(dold + 6 * j, d);
#pragma unroll
        for (int c = 0; c < 6; ++c) v[c] += beta * d[c];
    }
};

// Phase A over the grid's threads (one point each, strided).
template <typename T, class GX>
__device__ __forceinline__ void implicit_points(int64_t P, const int *__restrict__ trk_ptr,
                                                const int *__restrict__ obs_cam, const T *__restrict__ J,
                                                const T *__restrict__ Linv, GX gx, T *__restrict__ w) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < P; k += (int64_t)gridDim.x * blockDim.x) {
        const int a0 = __ldg(trk_ptr + k), a1 = __ldg(trk_ptr + k + 1);
        T t0 = T(0), t1 = T(0), t2 = T(0);
        for (int a = a0; a < a1; ++a) {
            T r[JW], xc[6];
            load_jrow(J + (int64_t)a * JW, r);
            gx(__ldg(obs_cam + a), xc);
            T s0 = T(0), s1 = T(0);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                s0 += r[c] * xc[c];
                s1 += r[6 + c] * xc[c];
            }
            t0 += r[12] * s0 + r[15] * s1;
            t1 += r[13] * s0 + r[16] * s1;
            t2 += r[14] * s0 + r[17] * s1;
            w[2 * (int64_t)a] = s0;
            w[2 * (int64_t)a + 1] = s1;
        }
        const T *m = Linv + 6 * k;  // L^-1 lower: m00 m10 m11 m20 m21 m22
        const T v0 = m[0] * t0, v1 = m[1] * t0 + m[2] * t1, v2 = m[3] * t0 + m[4] * t1 + m[5] * t2;
        const T u0 = m[0] * v0 + m[1] * v1 + m[3] * v2, u1 = m[2] * v1 + m[4] * v2, u2 = m[5] * v2;
        for (int a = a0; a < a1; ++a) {
            const T *r = J + (int64_t)a * JW;
            w[2 * (int64_t)a] -= r[12] * u0 + r[13] * u1 + r[14] * u2;
            w[2 * (int64_t)a + 1] -= r[15] * u0 + r[16] * u1 + r[17] * u2;
        }
    }
}
// Phase B over the grid's warps (one camera each, strided): out(i, c, y_ic,
// x_ic) receives each component of y_i = (S x)_i with x_i's own entry.
template <typename T, class GX, class OUT>
__device__ __forceinline__ void implicit_cams(int n, const int *__restrict__ cam_ptr, const int *__restrict__ cam_obs,
                                              const T *__restrict__ J, const T *__restrict__ w, GX gx, double lambda,
                                              OUT out) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n; i += nw) {
        T acc[6] = {T(0), T(0), T(0), T(0), T(0), T(0)}, dg[6] = {T(0), T(0), T(0), T(0), T(0), T(0)};
        for (int q = __ldg(cam_ptr + i) + lane; q < __ldg(cam_ptr + i + 1); q += 32) {
            const int64_t a = __ldg(cam_obs + q);
            T r[JW];
            load_jrow(J + a * JW, r);
            const T w0 = __ldcg(w + 2 * a), w1 = __ldcg(w + 2 * a + 1);
#pragma unroll
            for (int c = 0; c < 6; ++c) {
                acc[c] += r[c] * w0 + r[6 + c] * w1;
                dg[c] += r[c] * r[c] + r[6 + c] * r[6 + c];
            }
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            acc[c] = warp_sum(acc[c]);
            dg[c] = warp_sum(dg[c]);
        }
        T xi[6];
        gx(i, xi);
        if (lane < 6) {
            T a = acc[0], d = dg[0], xv = xi[0];
#pragma unroll
            for (int c = 1; c < 6; ++c)
                if (lane == c) {
                    a = acc[c];
                    d = dg[c];
                    xv = xi[c];
                }
            out(i, lane, a + (T)lambda * clampT(d) * xv, xv);
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_implicit_points(int64_t P, const int *__restrict__ trk_ptr,
                                                         const int *__restrict__ obs_cam, const T *__restrict__ J,
                                                         const T *__restrict__ Linv, const T *__restrict__ x,
                                                         T *__restrict__ w) {
    implicit_points<T>(P, trk_ptr, obs_cam, J, Linv, PlainX<T>{x}, w);
}
template <typename T>
__global__ void __launch_bounds__(256) k_implicit_cams(int n, const int *__restrict__ cam_ptr,
                                                       const int *__restrict__ cam_obs, const T *__restrict__ J,
                                                       const T *__restrict__ w, const T *__restrict__ x, double lambda,
                                                       T *__restrict__ y) {
    implicit_cams<T>(n, cam_ptr, cam_obs, J, w, PlainX<T>{x}, lambda,
                     [&](int i, int c, T v, T) { y[6 * (int64_t)i + c] = v; });
}

// Block-Jacobi PCG (the Sec. 3.2 recurrence, as k_pcg_persist runs it) with
// the implicit product in place of the stored RCS: per iteration phase A, a
// grid barrier, phase B (which also stores d_new and sums d^T S d), the
// all-reduce of d^T S d, the update phase, the all-reduce of r^T z and r^T r.
// The preconditioner, right-hand side and per-point factors are those of the
// last RCS formation (same lambda).  Cooperative launch; bounded waits.
template <typename T>
__global__ void __launch_bounds__(256) k_pcg_implicit(int n, int64_t P, const int *__restrict__ trk_ptr,
                                                      const int *__restrict__ obs_cam, const T *__restrict__ J,
                                                      const T *__restrict__ Linv, const int *__restrict__ cam_ptr,
                                                      const int *__restrict__ cam_obs, T *w, double lambda,
                                                      const T *__restrict__ Minv, T *y, T *r0, T *r1, T *z, T *d0,
                                                      T *d1, T *q, DevScalars *sc, double *red, unsigned *bar,
                                                      long long limit_cycles) {
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
        const PcgDir<T> dir{z, dold, (T)beta};
        implicit_points<T>(P, trk_ptr, obs_cam, J, Linv, dir, w);
        double bar1[1] = {0.0};
        block_sum<1>(bar1, sh);
        if (!grid_allreduce_sym<1>(bar1, red, gen++, bar, &sc->err, limit_cycles)) return;  // w complete
        T pap_t = T(0);
        implicit_cams<T>(n, cam_ptr, cam_obs, J, w, dir, lambda, [&](int i, int c, T v, T xv) {
            q[6 * (int64_t)i + c] = v;
            dnew[6 * (int64_t)i + c] = xv;
            pap_t += xv * v;
        });
        double v1[1] = {(double)pap_t};
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

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// One wave: at most the CTAs that fit on the GPU at once (the loops stride
// over the rest), so no partial second wave.
static int fmt_grid(const void *kern, int64_t warps, size_t smem = 0) {
    int per_sm = 0, n_sm = 0;
    if (occupancy(kern, 256, smem, &per_sm, &n_sm) != cudaSuccess) return 1;
    const int64_t resident = (int64_t)std::max(1, per_sm) * n_sm;
    const int64_t ctas = (warps * 32 + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ctas, resident));
}

cudaError_t launch_rcs_format_build(ba_problem *p, int format) {
    const int64_t E = (2 * p->nnzb - p->n);
    const int n = p->n;
    cudaError_t e;
    auto alloc = [&](void **d, size_t bytes) -> cudaError_t {
        if (*d) return cudaSuccess;
        cudaError_t r = cudaMalloc(d, std::max<size_t>(bytes, 16));
        if (r == cudaSuccess) {
            p->allocs.push_back(*d);
            p->dev_bytes += bytes;
        }
        return r;
    };
    if (format == BA_FMT_IMPLICIT) {
        // the camera-major observation index (once per problem: the pattern is
        // fixed) and the per-observation work vector
        if (!p->imp_cam_ptr) {
            const int64_t m = p->m;
            std::vector<int32_t> oc(m), ptr(n + 1, 0), idx(m);
            if ((e = cudaMemcpy(oc.data(), p->obs_cam, m * sizeof(int32_t), cudaMemcpyDeviceToHost)) != cudaSuccess)
                return e;
            for (int64_t a = 0; a < m; ++a) ptr[oc[a] + 1]++;
            for (int i = 0; i < n; ++i) ptr[i + 1] += ptr[i];
            std::vector<int32_t> fill(ptr.begin(), ptr.end() - 1);
            for (int64_t a = 0; a < m; ++a) idx[fill[oc[a]]++] = (int32_t)a;
            if ((e = alloc((void **)&p->imp_cam_ptr, (size_t)(n + 1) * sizeof(int32_t))) != cudaSuccess) return e;
            if ((e = alloc((void **)&p->imp_cam_obs, (size_t)m * sizeof(int32_t))) != cudaSuccess) return e;
            if ((e = cudaMemcpy(p->imp_cam_ptr, ptr.data(), (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return e;
            if ((e = cudaMemcpy(p->imp_cam_obs, idx.data(), m * sizeof(int32_t), cudaMemcpyHostToDevice)) !=
                cudaSuccess)
                return e;
        }
        return alloc(&p->imp_w, (size_t)p->m * 2 * p->esz);
    }
    const int gb = (int)std::max<int64_t>(1, std::min<int64_t>((E * BW + 255) / 256, 152 * 16));
    // the full BSR (also the source of the CSR)
    if (p->fmt_gen[BA_FMT_BSR_FULL] != p->rcs_gen) {
        if ((e = alloc(&p->fmt_bsr_val, (size_t)E * BW * p->esz)) != cudaSuccess) return e;
        if ((e = alloc((void **)&p->fmt_bsr_col, (size_t)E * sizeof(int))) != cudaSuccess) return e;
        if (p->fp32)
            k_build_bsr<float><<<gb, 256, 0, p->st>>>(E, p->tw_ent, (const float *)p->S, (float *)p->fmt_bsr_val,
                                                      p->fmt_bsr_col);
        else
            k_build_bsr<double><<<gb, 256, 0, p->st>>>(E, p->tw_ent, (const double *)p->S, (double *)p->fmt_bsr_val,
                                                       p->fmt_bsr_col);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        p->fmt_gen[BA_FMT_BSR_FULL] = p->rcs_gen;
    }
    if (format == BA_FMT_CSR && p->fmt_gen[BA_FMT_CSR] != p->rcs_gen) {
        if ((e = alloc((void **)&p->fmt_csr_ptr, (size_t)(6 * n + 1) * sizeof(int))) != cudaSuccess) return e;
        if ((e = alloc((void **)&p->fmt_csr_col, (size_t)E * BW * sizeof(int))) != cudaSuccess) return e;
        if ((e = alloc(&p->fmt_csr_val, (size_t)E * BW * p->esz)) != cudaSuccess) return e;
        k_build_csr_ptr<<<(6 * n + 1 + 255) / 256, 256, 0, p->st>>>(n, p->tw_ptr, p->fmt_csr_ptr);
        if (p->fp32)
            k_build_csr<float><<<gb, 256, 0, p->st>>>(n, E, p->tw_ptr, (const float *)p->fmt_bsr_val, p->fmt_bsr_col,
                                                      p->fmt_csr_col, (float *)p->fmt_csr_val);
        else
            k_build_csr<double><<<gb, 256, 0, p->st>>>(n, E, p->tw_ptr, (const double *)p->fmt_bsr_val,
                                                       p->fmt_bsr_col, p->fmt_csr_col, (double *)p->fmt_csr_val);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        p->fmt_gen[BA_FMT_CSR] = p->rcs_gen;
    }
    return cudaSuccess;
}

template <typename T>
static void spmv_format_T(ba_problem *p, int format, const T *x, T *y) {
    const int n = p->n;
    if (format == BA_FMT_IMPLICIT) {
        k_implicit_points<T><<<fmt_grid((const void *)k_implicit_points<T>, (p->P + 31) / 32), 256, 0,
                                p->st>>>(p->P, p->trk_ptr, p->obs_cam, (const T *)p->J, (const T *)p->Linv, x,
                                         (T *)p->imp_w);
        k_implicit_cams<T><<<fmt_grid((const void *)k_implicit_cams<T>, n), 256, 0, p->st>>>(
            n, p->imp_cam_ptr, p->imp_cam_obs, (const T *)p->J, (const T *)p->imp_w, x, p->rcs_lambda, y);
        return;
    }
    if (format == BA_FMT_BSMC)
        k_spmv_blocks<T, true><<<fmt_grid((const void *)k_spmv_blocks<T, true>, n), 256, 0, p->st>>>(
            n, p->tw_ptr, p->tw_ent, nullptr, (const T *)p->S, x, y);
    else if (format == BA_FMT_BSMC_ONCE) {
        cudaMemsetAsync(y, 0, (size_t)6 * n * sizeof(T), p->st);
        k_spmv_bsmc_once<T><<<fmt_grid((const void *)k_spmv_bsmc_once<T>, n), 256, 0, p->st>>>(
            n, p->row_ptr, p->col, (const T *)p->S, x, y);
    }
    else if (format == BA_FMT_BSR_FULL)
        k_spmv_blocks<T, false><<<fmt_grid((const void *)k_spmv_blocks<T, false>, n), 256, 0, p->st>>>(
            n, p->tw_ptr, nullptr, p->fmt_bsr_col, (const T *)p->fmt_bsr_val, x, y);
    else
        k_spmv_csr<T><<<fmt_grid((const void *)k_spmv_csr<T>, 6 * (int64_t)n), 256, 0, p->st>>>(
            6 * n, p->fmt_csr_ptr, p->fmt_csr_col, (const T *)p->fmt_csr_val, x, y);
}

cudaError_t launch_rcs_spmv(ba_problem *p, int format, const void *x, void *y) {
    if (p->fp32)
        spmv_format_T<float>(p, format, (const float *)x, (float *)y);
    else
        spmv_format_T<double>(p, format, (const double *)x, (double *)y);
    p->launches += format == BA_FMT_IMPLICIT ? 2 : 1;
    return cudaGetLastError();
}

template <typename T>
static cudaError_t pcg_implicit_T(ba_problem *p) {
    int per_sm = 0, n_sm = 0;
    cudaError_t e;
    if ((e = occupancy((const void *)k_pcg_implicit<T>, 256, 0, &per_sm, &n_sm)) != cudaSuccess) return e;
    // the products are gathers from the stored J: as many warps in flight as fit
    if (per_sm > 4) per_sm = 4;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // enough threads for a point each or a warp per camera, at most what is co-resident
    const int64_t want = std::max<int64_t>((p->P + 255) / 256, ((int64_t)p->n * 32 + 255) / 256);
    int grid = (int)std::min<int64_t>(std::max<int64_t>(want, 1), (int64_t)per_sm * n_sm);
    if ((e = cudaMemsetAsync(p->counters + 14, 0, 2 * sizeof(unsigned), p->st)) != cudaSuccess) return e;
    int n = p->n;
    int64_t P = p->P;
    const int *trk = p->trk_ptr, *oc = p->obs_cam, *cp = p->imp_cam_ptr, *co = p->imp_cam_obs;
    const T *J = (const T *)p->J, *Li = (const T *)p->Linv, *Mi = (const T *)p->sv.Minv;
    T *w = (T *)p->imp_w;
    double lambda = p->rcs_lambda;
    T *y = (T *)p->sv.pv[0], *r = (T *)p->sv.pv[1], *z = (T *)p->sv.pv[2], *d0 = (T *)p->sv.pv[3], *d1 = (T *)p->sv.pv[4];
    T *q = (T *)p->sv.pv[5], *r1 = (T *)p->sv.pv[6];
    DevScalars *sc = p->sc;
    double *red = p->red;
    unsigned *bar = p->counters + 14;
    long long limit = 4000000000LL;  // ~2 s of SM clock per barrier wait
    void *args[] = {&n, &P, &trk, &oc, &J, &Li, &cp, &co, &w, &lambda, &Mi, &y, &r, &r1, &z, &d0, &d1, &q, &sc, &red, &bar, &limit};
    return cudaLaunchCooperativeKernel((const void *)k_pcg_implicit<T>, dim3(grid), dim3(256), args, 0, p->st);
}

// The PCG loop on the implicit operator (state from launch_pcg_init); the
// solve vectors must be in the problem's precision.
cudaError_t launch_pcg_implicit(ba_problem *p) {
    cudaError_t e = launch_rcs_format_build(p, BA_FMT_IMPLICIT);
    if (e != cudaSuccess) return e;
    cudaEvent_t ev;
    ktimer_begin(p, K_PCG_LOOP, &ev);
    e = p->fp32 ? pcg_implicit_T<float>(p) : pcg_implicit_T<double>(p);
    ktimer_end(p, K_PCG_LOOP, ev);
    p->launches += 1;
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

int64_t rcs_format_bytes(const ba_problem *p, int format) {
    const int64_t n = p->n, E = (2 * p->nnzb - p->n), nnzb = p->nnzb;
    // implicit: what one product reads instead of S - the stored J rows (twice
    // the J_c part), L^-1 per point, the work vector (written and read) and
    // the camera-major index
    if (format == BA_FMT_IMPLICIT)
        return p->m * (int64_t)(JW + 12) * p->esz + p->P * 6 * (int64_t)p->esz + p->m * 2 * 2 * (int64_t)p->esz +
               (p->m + n + 1) * 4;
    if (format == BA_FMT_BSMC || format == BA_FMT_BSMC_ONCE) return nnzb * BW * p->esz + nnzb * 4 + (n + 1) * 4;
    if (format == BA_FMT_BSR_FULL) return E * BW * p->esz + E * 4 + (n + 1) * 4;
    return E * BW * (p->esz + 4) + (6 * n + 1) * 4;
}

}  // namespace ba
