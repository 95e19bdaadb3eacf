// Variable-size BSMC (Sec. 4, Fig. 4: block (i, j) is c_i x c_j; c = 11 with
// five interior unknowns in Sec. 4.1): storage, the two-sided product of
// Sec. 6.2 (Fig. 13) and the block-Jacobi PCG of Sec. 3.2 (Eqs. 6-7), behind
// the ba_vbsmc_* calls of ba_vbsmc.h.
//
// Device layout: the upper blocks packed in row order (block k at value
// offset boff[k], row-major c_row x c_col), a column per block, row starts,
// block sizes cdim and vector offsets off (camera i's entries are
// off[i] .. off[i] + c_i - 1).  The product runs from two-sided entry lists
// built on the host: row i lists its stored blocks, then the blocks of its
// column in the rows above it, flagged "transposed" (one 16-byte record per
// entry); so every row is summed by one warp with no atomics, in a fixed
// order.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "device_util.cuh"
#include "vbsmc_internal.h"

namespace ba {

// Warp-per-row product: lane a + 16 h (a < 16 the output component, h the
// parity of the entries it takes) sums S_ij x_j over its entries; the halves
// are joined by one shuffle.  Each two-sided entry is one 16-byte record
// (value offset lo / hi, vector offset of j, c_j << 1 | transposed), and a
// lane loads its whole block row (or column) and the c_j values of x with
// independent predicated loads before the FMAs, so an entry costs two
// dependent memory round trips, not one per column.  (Staging each block in
// shared memory with coalesced loads first measured 1.9x slower: the copy,
// the warp barrier and the shared reads chain per entry.)  gx(idx) returns x
// at vector index idx; lanes a < c_i of half 0 call out(idx, (S x)_idx).
template <typename T, class GX, class OUT>
__device__ __forceinline__ void vb_row(int i, const int *__restrict__ cdim, const int *__restrict__ off,
                                       const int *__restrict__ tw_ptr, const int4 *__restrict__ tw_info,
                                       const T *__restrict__ val, GX gx, OUT out) {
    const int lane = threadIdx.x & 31, a = lane & 15, h = lane >> 4;
    const int ci = __ldg(cdim + i);
    T acc = T(0);
    const int e1 = __ldg(tw_ptr + i + 1);
    for (int e = __ldg(tw_ptr + i) + h; e < e1; e += 2) {
        const int4 in = __ldg(tw_info + e);
        const int64_t vo = (int64_t)(uint32_t)in.x | ((int64_t)in.y << 32);
        const int oj = in.z, cj = in.w >> 1;
        const T *B = val + vo;
        // element (a, c) of this row's block: B[c * ci + a] if transposed, else B[a * cj + c]
        const int stride = (in.w & 1) ? ci : 1, base = (in.w & 1) ? a : a * cj;
        T bv[BA_VB_CMAX], xv[BA_VB_CMAX];
#pragma unroll
        for (int c = 0; c < BA_VB_CMAX; ++c) {
            const bool on = c < cj && a < ci;
            bv[c] = on ? __ldg(B + base + c * stride) : T(0);
            xv[c] = c < cj ? gx(oj + c) : T(0);
        }
#pragma unroll
        for (int c = 0; c < BA_VB_CMAX; ++c) acc += bv[c] * xv[c];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 16);
    if (h == 0 && a < ci) out(__ldg(off + i) + a, acc);
}

template <typename T>
__global__ void __launch_bounds__(256) k_vb_spmv(int n, const int *__restrict__ cdim, const int *__restrict__ off,
                                                 const int *__restrict__ tw_ptr, const int4 *__restrict__ tw_info,
                                                 const T *__restrict__ val, const T *__restrict__ x, T *__restrict__ y) {
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5); i < n; i += nw)
        vb_row<T>(i, cdim, off, tw_ptr, tw_info, val, [&](int idx) { return __ldg(x + idx); },
                  [&](int idx, T v) { y[idx] = v; });
}

// M^-1 per camera (a thread each): FP64 Cholesky of the diagonal block, then
// its inverse column by column; a block that is not positive definite sets
// BA_ERR_NOT_SPD and leaves zeros.
template <typename T>
__global__ void k_vb_minv(int n, const int *__restrict__ cdim, const int *__restrict__ row_ptr,
                          const int64_t *__restrict__ boff, const T *__restrict__ val, const int64_t *__restrict__ moff,
                          T *__restrict__ Minv, int *err) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cdim[i];
    const T *D = val + boff[row_ptr[i]];
    T *M = Minv + moff[i];
    double L[BA_VB_CMAX * BA_VB_CMAX];
    bool ok = true;
    for (int r = 0; r < c; ++r)
        for (int q = 0; q <= r; ++q) {
            double s = 0.5 * ((double)D[r * c + q] + (double)D[q * c + r]);
            for (int k = 0; k < q; ++k) s -= L[r * BA_VB_CMAX + k] * L[q * BA_VB_CMAX + k];
            if (r == q) {
                if (!(s > 0.0)) {
                    ok = false;
                    s = 1.0;
                }
                L[r * BA_VB_CMAX + r] = sqrt(s);
            } else {
                L[r * BA_VB_CMAX + q] = s / L[q * BA_VB_CMAX + q];
            }
        }
    if (!ok) {
        atomicExch(err, (int)BA_ERR_NOT_SPD);
        for (int k = 0; k < c * c; ++k) M[k] = T(0);
        return;
    }
    // column q of (L L^T)^-1: forward then backward substitution on e_q
    double w[BA_VB_CMAX];
    for (int q = 0; q < c; ++q) {
        for (int r = 0; r < c; ++r) {
            double s = (r == q) ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s -= L[r * BA_VB_CMAX + k] * w[k];
            w[r] = s / L[r * BA_VB_CMAX + r];
        }
        for (int r = c - 1; r >= 0; --r) {
            double s = w[r];
            for (int k = r + 1; k < c; ++k) s -= L[k * BA_VB_CMAX + r] * w[k];
            w[r] = s / L[r * BA_VB_CMAX + r];
        }
        for (int r = 0; r < c; ++r) M[r * c + q] = (T)w[r];
    }
}

// z_e = (M^-1_i v_i)[a] for vector entry e = off[i] + a, where v_i[c] = g(off[i] + c).
template <typename T, class G>
__device__ __forceinline__ T vb_precond_entry(int i, int a, const int *__restrict__ cdim, const int *__restrict__ off,
                                              const int64_t *__restrict__ moff, const T *__restrict__ Minv, G g) {
    const int c = __ldg(cdim + i), o = __ldg(off + i);
    const T *M = Minv + __ldg(moff + i) + (int64_t)a * c;
    T z = T(0);
    for (int k = 0; k < c; ++k) z += __ldg(M + k) * g(o + k);
    return z;
}

// The PCG of Sec. 3.2 on the variable-size system in one cooperative launch:
// the start (r = b, z = M^-1 b, y = 0) and r^T z, r^T r by one all-reduce;
// then per iteration the product phase (d = z + beta d_old formed on the fly,
// q = S d, d^T S d), its all-reduce, the update phase (y += alpha d,
// r -= alpha q, z = M^-1 r, r^T z, r^T r) and its all-reduce.  Every grid wait
// is bounded (BA_ERR_TIMEOUT).
template <typename T>
__global__ void __launch_bounds__(256) k_vb_pcg(int n, int N, const int *__restrict__ cdim, const int *__restrict__ off,
                                                const int *__restrict__ ent_cam, const int *__restrict__ tw_ptr,
                                                const int4 *__restrict__ tw_info, const T *__restrict__ val,
                                                const int64_t *__restrict__ moff,
                                                const T *__restrict__ Minv, const T *__restrict__ b, T *y, T *r0, T *r1,
                                                T *z, T *d0, T *d1, T *q, VbScalars *sc, double *red, unsigned *bar,
                                                long long limit_cycles) {
    __shared__ double sh[40];
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const double tol2 = sc->tol2;
    const int max_iters = sc->max_iters;
    unsigned gen = 0;
    double v0[2] = {0.0, 0.0};
    for (int e = tid; e < N; e += nth) {
        const int i = __ldg(ent_cam + e);
        const T ze = vb_precond_entry<T>(i, e - __ldg(off + i), cdim, off, moff, Minv, [&](int k) { return __ldg(b + k); });
        const T be = __ldg(b + e);
        r0[e] = be;
        z[e] = ze;
        y[e] = T(0);
        d0[e] = T(0);
        v0[0] += (double)(be * ze);
        v0[1] += (double)(be * be);
    }
    block_sum<2>(v0, sh);
    if (!grid_allreduce_sym<2>(v0, red, gen++, bar, &sc->err, limit_cycles)) return;
    double rz = v0[0];
    const double rr0 = v0[1];
    if (!(rr0 > 0.0) || max_iters <= 0) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            sc->rr0 = rr0;
            sc->rr = rr0;
            sc->iters = 0;
            sc->done = 1;
        }
        return;
    }
    double beta = 0.0;
    int it = 0;
    const int nw = nth >> 5;
    for (;;) {
        const bool odd = it & 1;
        T *dold = odd ? d1 : d0, *dnew = odd ? d0 : d1;
        T *rc = odd ? r1 : r0, *rn = odd ? r0 : r1;
        const T bt = (T)beta;
        auto dir = [&](int k) { return __ldcg(z + k) + bt * __ldcg(dold + k); };
        T pap_t = T(0);
        for (int i = tid >> 5; i < n; i += nw)
            vb_row<T>(i, cdim, off, tw_ptr, tw_info, val, dir, [&](int idx, T v) {
                const T dv = dir(idx);
                q[idx] = v;
                dnew[idx] = dv;
                pap_t += dv * v;
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
        double v2[2] = {0.0, 0.0};
        for (int e = tid; e < N; e += nth) {
            const int i = __ldg(ent_cam + e);
            const T ze = vb_precond_entry<T>(i, e - __ldg(off + i), cdim, off, moff, Minv,
                                             [&](int k) { return __ldcg(rc + k) - alpha * __ldcg(q + k); });
            const T ra = __ldcg(rc + e) - alpha * __ldcg(q + e);
            y[e] += alpha * __ldcg(dnew + e);
            rn[e] = ra;
            z[e] = ze;
            v2[0] += (double)(ra * ze);
            v2[1] += (double)(ra * ra);
        }
        block_sum<2>(v2, sh);
        if (!grid_allreduce_sym<2>(v2, red, gen++, bar, &sc->err, limit_cycles)) return;
        const double rz_new = v2[0], rr = v2[1];
        ++it;
        if (rr <= tol2 * rr0 || it >= max_iters) {
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                sc->iters = it;
                sc->rr = rr;
                sc->rr0 = rr0;
                sc->rz = rz_new;
                sc->done = 1;
            }
            return;
        }
        beta = rz_new / rz;
        rz = rz_new;
    }
}

}  // namespace ba

using namespace ba;

namespace ba {

ba_status vb_alloc(ba_vbsmc *h, void **d, size_t bytes) {
    bytes = bytes < 16 ? 16 : bytes;
    if (h->cap && h->dev_bytes + bytes > h->cap) return set_error(BA_ERR_OOM, "device_mem_cap reached");
    cudaError_t e = cudaMalloc(d, bytes);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(BA_ERR_OOM, "cudaMalloc failed");
    }
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    h->allocs.push_back(*d);
    h->dev_bytes += bytes;
    return BA_OK;
}

ba_status vb_cuda(ba_vbsmc *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return BA_OK;
    h->dead = true;
    return set_error(BA_ERR_CUDA, (std::string(what) + ": " + cudaGetErrorString(e)).c_str());
}

}  // namespace ba

namespace {

template <typename T>
ba_status vb_upload(ba_vbsmc *h, void *dst, const double *src, size_t cnt) {
    std::vector<T> tmp(cnt);
    for (size_t k = 0; k < cnt; ++k) tmp[k] = (T)src[k];
    return vb_cuda(h, cudaMemcpy(dst, tmp.data(), cnt * sizeof(T), cudaMemcpyHostToDevice), "upload");
}

template <typename T>
cudaError_t vb_spmv_T(ba_vbsmc *h, const T *x, T *y) {
    int per_sm = 0, n_sm = 0;
    cudaError_t e = occupancy((const void *)k_vb_spmv<T>, 256, 0, &per_sm, &n_sm);
    if (e != cudaSuccess) return e;
    const int64_t want = ((int64_t)h->n * 32 + 255) / 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)std::max(per_sm, 1) * n_sm));
    k_vb_spmv<T><<<grid, 256, 0, h->st>>>(h->n, h->cdim, h->off, h->tw_ptr, h->tw_info, (const T *)h->val, x, y);
    return cudaGetLastError();
}

template <typename T>
cudaError_t vb_pcg_T(ba_vbsmc *h) {
    int per_sm = 0, n_sm = 0;
    cudaError_t e = occupancy((const void *)k_vb_pcg<T>, 256, 0, &per_sm, &n_sm);
    if (e != cudaSuccess) return e;
    if (per_sm > 2) per_sm = 2;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int64_t want = std::max<int64_t>(((int64_t)h->n * 32 + 255) / 256, (h->N + 255) / 256);
    int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)per_sm * n_sm));
    if ((e = cudaMemsetAsync(h->bar, 0, sizeof(unsigned), h->st)) != cudaSuccess) return e;
    int n = h->n, N = (int)h->N;
    const int *cd = h->cdim, *of = h->off, *ec = h->ent_cam, *twp = h->tw_ptr;
    const int4 *twi = h->tw_info;
    const int64_t *mo = h->moff;
    const T *val = (const T *)h->val, *Mi = (const T *)h->Minv, *b = (const T *)h->b;
    T *y = (T *)h->vec[0], *r0 = (T *)h->vec[1], *r1 = (T *)h->vec[2], *z = (T *)h->vec[3], *d0 = (T *)h->vec[4],
      *d1 = (T *)h->vec[5], *q = (T *)h->vec[6];
    VbScalars *sc = h->sc;
    double *red = h->red;
    unsigned *bar = h->bar;
    long long limit = 4000000000LL;  // ~2 s of SM clock per grid wait
    void *args[] = {&n, &N, &cd, &of, &ec, &twp, &twi, &val, &mo, &Mi, &b, &y, &r0, &r1, &z, &d0, &d1, &q,
                    &sc, &red, &bar, &limit};
    return cudaLaunchCooperativeKernel((const void *)k_vb_pcg<T>, dim3(grid), dim3(256), args, 0, h->st);
}

}  // namespace

namespace ba {

ba_status vb_check_pattern(const ba_options &o, int32_t n, const int32_t *cdim, int64_t nnzb, const int32_t *row_ptr,
                           const int32_t *col, int64_t *N_out, int64_t *nval_out) {
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return set_error(BA_ERR_INVALID_ARG, "bad precision");
    if (n <= 0 || n >= (1 << 30) || nnzb < n || nnzb >= (int64_t)INT32_MAX)
        return set_error(BA_ERR_INVALID_ARG, "need 0 < n < 2^30 and n <= nnzb < 2^31");
    if (!cdim || !row_ptr || !col) return set_error(BA_ERR_INVALID_ARG, "null input array");
    if (row_ptr[0] != 0 || row_ptr[n] != nnzb) return set_error(BA_ERR_INVALID_ARG, "row_ptr must run from 0 to nnzb");
    int64_t N = 0, nval = 0;
    for (int32_t i = 0; i < n; ++i) {
        if (cdim[i] < 1 || cdim[i] > BA_VB_CMAX) return set_error(BA_ERR_INVALID_ARG, "block size out of 1..BA_VB_CMAX");
        N += cdim[i];
    }
    if (N >= (int64_t)INT32_MAX) return set_error(BA_ERR_INVALID_ARG, "too many unknowns");
    for (int32_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] <= row_ptr[i]) return set_error(BA_ERR_INVALID_ARG, "every row needs its diagonal block");
        if (col[row_ptr[i]] != i) return set_error(BA_ERR_INVALID_ARG, "the first block of a row must be its diagonal");
        for (int32_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k)
            if (col[k] <= col[k - 1] || col[k] >= n)
                return set_error(BA_ERR_INVALID_ARG, "columns must increase within a row and stay below n");
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) nval += (int64_t)cdim[i] * cdim[col[k]];
    }
    *N_out = N;
    *nval_out = nval;
    return BA_OK;
}

ba_status vb_build(const ba_options &o, int32_t n, const int32_t *cdim, int64_t nnzb, const int32_t *row_ptr,
                   const int32_t *col, ba_vbsmc **out) {
    int64_t N = 0, nval = 0, nminv = 0;
    ba_status s = vb_check_pattern(o, n, cdim, nnzb, row_ptr, col, &N, &nval);
    if (s) return s;
    // host-side layout: offsets, two-sided entry lists
    std::vector<int32_t> off(n + 1, 0), ent_cam(N), tw_ptr(n + 1, 0);
    std::vector<int64_t> boff(nnzb + 1, 0), moff(n + 1, 0);
    for (int32_t i = 0; i < n; ++i) {
        off[i + 1] = off[i] + cdim[i];
        moff[i + 1] = moff[i] + (int64_t)cdim[i] * cdim[i];
        for (int32_t a = 0; a < cdim[i]; ++a) ent_cam[off[i] + a] = i;
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) boff[k + 1] = boff[k] + (int64_t)cdim[i] * cdim[col[k]];
    }
    nminv = moff[n];
    for (int32_t i = 0; i < n; ++i) {
        tw_ptr[i + 1] += row_ptr[i + 1] - row_ptr[i];
        for (int32_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) tw_ptr[col[k] + 1] += 1;
    }
    for (int32_t i = 0; i < n; ++i) tw_ptr[i + 1] += tw_ptr[i];
    // two-sided entry records: value offset (lo, hi), vector offset of the
    // other camera j, c_j << 1 | transposed
    std::vector<int4> tw_info(tw_ptr[n]);
    {
        auto rec = [&](int32_t k, int32_t j, int tr) {
            return make_int4((int)(uint32_t)(boff[k] & 0xffffffffu), (int)(boff[k] >> 32), off[j], (cdim[j] << 1) | tr);
        };
        std::vector<int32_t> fill(tw_ptr.begin(), tw_ptr.end() - 1);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) tw_info[fill[i]++] = rec(k, col[k], 0);
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = row_ptr[i] + 1; k < row_ptr[i + 1]; ++k) tw_info[fill[col[k]]++] = rec(k, i, 1);
    }
    ba_vbsmc *h = new ba_vbsmc();
    h->n = n;
    h->nnzb = nnzb;
    h->N = N;
    h->nval = nval;
    h->nminv = nminv;
    h->fp32 = o.precision == BA_FP32;
    h->esz = h->fp32 ? 4 : 8;
    h->st = (cudaStream_t)o.cuda_stream;
    h->cap = o.device_mem_cap;
    auto up = [&](void **d, const void *src, size_t bytes) -> ba_status {
        ba_status r = vb_alloc(h, d, bytes);
        if (r) return r;
        return vb_cuda(h, cudaMemcpy(*d, src, bytes, cudaMemcpyHostToDevice), "upload");
    };
    std::vector<int32_t> brow(nnzb);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) brow[k] = i;
    if (!s) s = up((void **)&h->cdim, cdim, n * sizeof(int32_t));
    if (!s) s = up((void **)&h->off, off.data(), (n + 1) * sizeof(int32_t));
    if (!s) s = up((void **)&h->row_ptr, row_ptr, (n + 1) * sizeof(int32_t));
    if (!s) s = up((void **)&h->col, col, nnzb * sizeof(int32_t));
    if (!s) s = up((void **)&h->brow, brow.data(), nnzb * sizeof(int32_t));
    if (!s) s = up((void **)&h->ent_cam, ent_cam.data(), N * sizeof(int32_t));
    if (!s) s = up((void **)&h->tw_ptr, tw_ptr.data(), (n + 1) * sizeof(int32_t));
    if (!s) s = up((void **)&h->tw_info, tw_info.data(), tw_info.size() * sizeof(int4));
    if (!s) s = up((void **)&h->boff, boff.data(), (nnzb + 1) * sizeof(int64_t));
    if (!s) s = up((void **)&h->moff, moff.data(), (n + 1) * sizeof(int64_t));
    if (!s) s = vb_alloc(h, &h->val, nval * h->esz);
    if (!s) s = vb_alloc(h, &h->b, N * h->esz);
    if (!s) s = vb_alloc(h, &h->Minv, nminv * h->esz);
    for (auto &v : h->vec)
        if (!s) s = vb_alloc(h, &v, N * h->esz);
    if (!s) s = vb_alloc(h, (void **)&h->sc, sizeof(VbScalars));
    if (!s) s = vb_alloc(h, (void **)&h->red, (size_t)RED_SLOTS * sizeof(double));
    if (!s) s = vb_alloc(h, (void **)&h->bar, sizeof(unsigned));
    if (!s) s = vb_alloc(h, (void **)&h->err, sizeof(int));
    if (!s) s = vb_cuda(h, cudaEventCreate(&h->ev[0]), "event");
    if (!s) s = vb_cuda(h, cudaEventCreate(&h->ev[1]), "event");
    if (s) {
        ba_vbsmc_destroy(h);
        return s;
    }
    *out = h;
    return BA_OK;
}

ba_status vb_finish(ba_vbsmc *h) {
    ba_status s;
    if ((s = vb_cuda(h, cudaMemsetAsync(h->err, 0, sizeof(int), h->st), "memset"))) return s;
    const int g = (h->n + 127) / 128;
    if (h->fp32)
        k_vb_minv<float><<<g, 128, 0, h->st>>>(h->n, h->cdim, h->row_ptr, h->boff, (const float *)h->val, h->moff,
                                               (float *)h->Minv, h->err);
    else
        k_vb_minv<double><<<g, 128, 0, h->st>>>(h->n, h->cdim, h->row_ptr, h->boff, (const double *)h->val, h->moff,
                                                (double *)h->Minv, h->err);
    if ((s = vb_cuda(h, cudaGetLastError(), "k_vb_minv"))) return s;
    int err = 0;
    if ((s = vb_cuda(h, cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->st), "read flag")))
        return s;
    if ((s = vb_cuda(h, cudaStreamSynchronize(h->st), "sync"))) return s;
    if (err == BA_ERR_NOT_SPD) return set_error(BA_ERR_NOT_SPD, "a diagonal block is not positive definite");
    return BA_OK;
}

}  // namespace ba

extern "C" {

ba_status ba_vbsmc_create(const ba_options *opt, int32_t n, const int32_t *cdim, int64_t nnzb, const int32_t *row_ptr,
                          const int32_t *col, const double *val, const double *b, ba_vbsmc **out) {
    if (!out) return set_error(BA_ERR_INVALID_ARG, "null output pointer");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (!val || !b) return set_error(BA_ERR_INVALID_ARG, "null input array");
    int64_t N = 0, nval = 0;
    ba_status s = vb_check_pattern(o, n, cdim, nnzb, row_ptr, col, &N, &nval);
    if (s) return s;
    for (int64_t k = 0; k < nval; ++k)
        if (!std::isfinite(val[k])) return set_error(BA_ERR_NONFINITE, "non-finite block value");
    for (int64_t k = 0; k < N; ++k)
        if (!std::isfinite(b[k])) return set_error(BA_ERR_NONFINITE, "non-finite b");
    ba_vbsmc *h = nullptr;
    if ((s = vb_build(o, n, cdim, nnzb, row_ptr, col, &h))) return s;
    s = h->fp32 ? vb_upload<float>(h, h->val, val, nval) : vb_upload<double>(h, h->val, val, nval);
    if (!s) s = h->fp32 ? vb_upload<float>(h, h->b, b, N) : vb_upload<double>(h, h->b, b, N);
    if (!s) s = vb_finish(h);
    if (s) {
        ba_vbsmc_destroy(h);
        return s;
    }
    *out = h;
    return BA_OK;
}

ba_status ba_vbsmc_get_system(const ba_vbsmc *h, int32_t *row_ptr, int32_t *col, double *val, double *b) {
    if (!h) return set_error(BA_ERR_INVALID_ARG, "null object");
    if (h->dead) return set_error(BA_ERR_STATE, "the object is unusable after an earlier error");
    ba_vbsmc *m = const_cast<ba_vbsmc *>(h);
    ba_status s;
    if (row_ptr && (s = vb_cuda(m, cudaMemcpy(row_ptr, h->row_ptr, (h->n + 1) * sizeof(int32_t), cudaMemcpyDeviceToHost),
                                "read row_ptr")))
        return s;
    if (col && (s = vb_cuda(m, cudaMemcpy(col, h->col, h->nnzb * sizeof(int32_t), cudaMemcpyDeviceToHost), "read col")))
        return s;
    auto rd = [&](double *dst, const void *src, int64_t cnt) -> ba_status {
        std::vector<char> raw(cnt * h->esz);
        ba_status r = vb_cuda(m, cudaMemcpy(raw.data(), src, raw.size(), cudaMemcpyDeviceToHost), "read values");
        if (r) return r;
        for (int64_t k = 0; k < cnt; ++k)
            dst[k] = h->fp32 ? (double)reinterpret_cast<const float *>(raw.data())[k]
                             : reinterpret_cast<const double *>(raw.data())[k];
        return BA_OK;
    };
    if (val && (s = rd(val, h->val, h->nval))) return s;
    if (b && (s = rd(b, h->b, h->N))) return s;
    return BA_OK;
}

ba_status ba_vbsmc_spmv(ba_vbsmc *h, const void *x, void *y) {
    if (!h || !x || !y) return set_error(BA_ERR_INVALID_ARG, "null argument");
    if (h->dead) return set_error(BA_ERR_STATE, "the object is unusable after an earlier error");
    cudaError_t e = h->fp32 ? vb_spmv_T<float>(h, (const float *)x, (float *)y)
                            : vb_spmv_T<double>(h, (const double *)x, (double *)y);
    return vb_cuda(h, e, "k_vb_spmv");
}

ba_status ba_vbsmc_solve(ba_vbsmc *h, double tol, int32_t max_iters, double *x_out, int32_t *iters, double *rel_resid,
                         double *kernel_ms) {
    if (!h) return set_error(BA_ERR_INVALID_ARG, "null object");
    if (h->dead) return set_error(BA_ERR_STATE, "the object is unusable after an earlier error");
    if (!(tol > 0) || max_iters < 0) return set_error(BA_ERR_INVALID_ARG, "need tol > 0 and max_iters >= 0");
    VbScalars init{};
    init.tol2 = tol * tol;
    init.max_iters = max_iters > 0 ? max_iters : std::max(1000, 6 * h->n);
    ba_status s;
    if ((s = vb_cuda(h, cudaMemcpyAsync(h->sc, &init, sizeof(init), cudaMemcpyHostToDevice, h->st), "scalars")))
        return s;
    if ((s = vb_cuda(h, cudaEventRecord(h->ev[0], h->st), "event"))) return s;
    cudaError_t e = h->fp32 ? vb_pcg_T<float>(h) : vb_pcg_T<double>(h);
    if ((s = vb_cuda(h, e, "k_vb_pcg"))) return s;
    if ((s = vb_cuda(h, cudaEventRecord(h->ev[1], h->st), "event"))) return s;
    if ((s = vb_cuda(h, cudaMemcpyAsync(&h->host, h->sc, sizeof(VbScalars), cudaMemcpyDeviceToHost, h->st),
                     "scalars")))
        return s;
    if ((s = vb_cuda(h, cudaStreamSynchronize(h->st), "sync"))) return s;
    if (h->host.err == BA_ERR_TIMEOUT) {
        h->dead = true;
        return set_error(BA_ERR_TIMEOUT, "PCG grid wait timed out");
    }
    if (kernel_ms) {
        float ms = 0.f;
        if ((s = vb_cuda(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]), "event"))) return s;
        *kernel_ms = ms;
    }
    if (x_out) {
        std::vector<char> raw(h->N * h->esz);
        if ((s = vb_cuda(h, cudaMemcpy(raw.data(), h->vec[0], raw.size(), cudaMemcpyDeviceToHost), "read y"))) return s;
        for (int64_t k = 0; k < h->N; ++k)
            x_out[k] = h->fp32 ? (double)reinterpret_cast<const float *>(raw.data())[k]
                               : reinterpret_cast<const double *>(raw.data())[k];
    }
    const double rel = h->host.rr0 > 0 ? std::sqrt(h->host.rr / h->host.rr0) : 0.0;
    if (iters) *iters = h->host.iters;
    if (rel_resid) *rel_resid = rel;
    if (h->host.err == BA_ERR_NOT_SPD) return set_error(BA_ERR_NOT_SPD, "d^T S d <= 0 in PCG");
    if (h->host.rr0 > 0 && !(h->host.rr <= h->host.tol2 * h->host.rr0))
        return set_error(BA_ERR_NO_CONVERGENCE, "PCG reached its iteration cap");
    return BA_OK;
}

ba_status ba_vbsmc_info(const ba_vbsmc *h, int64_t *n_unknowns, int64_t *storage_bytes, int64_t *n_blocks) {
    if (!h) return set_error(BA_ERR_INVALID_ARG, "null object");
    if (n_unknowns) *n_unknowns = h->N;
    if (n_blocks) *n_blocks = h->nnzb;
    if (storage_bytes)
        *storage_bytes = h->nval * (int64_t)h->esz + h->nnzb * (4 + 8) + (int64_t)(h->n + 1) * 4 + (int64_t)h->n * 4;
    return BA_OK;
}

void ba_vbsmc_destroy(ba_vbsmc *h) {
    if (!h) return;
    if (h->st) cudaStreamSynchronize(h->st);
    else cudaDeviceSynchronize();
    for (auto &e : h->ev)
        if (e) cudaEventDestroy(e);
    for (void *d : h->allocs) cudaFree(d);
    delete h;
}

}  // extern "C"
