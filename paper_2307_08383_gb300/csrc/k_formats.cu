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

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
// One wave: at most the CTAs that fit on the GPU at once (the loops stride
// over the rest), so no partial second wave.
static int fmt_grid(const void *kern, int64_t warps, int &resident) {
    if (!resident) {
        int dev = 0, n_sm = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess)
            return 1;
        resident = std::max(1, per_sm) * n_sm;
    }
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
    static int res[3] = {0, 0, 0};  // resident CTAs per kernel (per precision: this template)
    if (format == BA_FMT_BSMC)
        k_spmv_blocks<T, true><<<fmt_grid((const void *)k_spmv_blocks<T, true>, n, res[0]), 256, 0, p->st>>>(
            n, p->tw_ptr, p->tw_ent, nullptr, (const T *)p->S, x, y);
    else if (format == BA_FMT_BSR_FULL)
        k_spmv_blocks<T, false><<<fmt_grid((const void *)k_spmv_blocks<T, false>, n, res[1]), 256, 0, p->st>>>(
            n, p->tw_ptr, nullptr, p->fmt_bsr_col, (const T *)p->fmt_bsr_val, x, y);
    else
        k_spmv_csr<T><<<fmt_grid((const void *)k_spmv_csr<T>, 6 * (int64_t)n, res[2]), 256, 0, p->st>>>(
            6 * n, p->fmt_csr_ptr, p->fmt_csr_col, (const T *)p->fmt_csr_val, x, y);
}

cudaError_t launch_rcs_spmv(ba_problem *p, int format, const void *x, void *y) {
    if (p->fp32)
        spmv_format_T<float>(p, format, (const float *)x, (float *)y);
    else
        spmv_format_T<double>(p, format, (const double *)x, (double *)y);
    p->launches += 1;
    return cudaGetLastError();
}

int64_t rcs_format_bytes(const ba_problem *p, int format) {
    const int64_t n = p->n, E = (2 * p->nnzb - p->n), nnzb = p->nnzb;
    if (format == BA_FMT_BSMC) return nnzb * BW * p->esz + nnzb * 4 + (n + 1) * 4;
    if (format == BA_FMT_BSR_FULL) return E * BW * p->esz + E * 4 + (n + 1) * 4;
    return E * BW * (p->esz + 4) + (6 * n + 1) * 4;
}

}  // namespace ba
