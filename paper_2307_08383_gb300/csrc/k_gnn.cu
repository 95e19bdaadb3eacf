// Learned block-Jacobi correction: tensor-core GEMM launcher (tcgen05) and the
// standalone GEMM entry point.
#include <algorithm>

#include <map>
#include <mutex>
#include <set>
#include "tc_gemm.cuh"

namespace ba {

// C (+)= A * B on the tensor cores; A: M x K, B: K x N through strided views.
template <typename TA, typename TB>
cudaError_t tc_gemm(cudaStream_t st, tc::View<TA> A, tc::View<TB> B, int M, int N, int K, const float *bias,
                    float *Z, int64_t z_rs, const float *mask, int64_t mask_rs, int relu, float *C, int64_t c_rs,
                    int64_t c_cs, bool accumulate, int *err) {
    if (M <= 0 || K <= 0) return cudaSuccess;
    if (N <= 0 || N > tc::kMaxN || (N % 32) != 0) return cudaErrorInvalidValue;
    // the kernel's shared-memory attribute, once per device (kernel
    // attributes belong to the device's context)
    static std::mutex attr_mu;
    static std::set<int> attr_set;
    cudaError_t e;
    {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(attr_mu);
        if (!attr_set.count(dev)) {
            if ((e = cudaFuncSetAttribute(tc::k_tc_gemm<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          tc::kSmemBytes)) != cudaSuccess)
                return e;
            attr_set.insert(dev);
        }
    }
    const int kchunk = tc::kMaxK;
    const int ksplit = (K + kchunk - 1) / kchunk;
    const int epi = (accumulate || ksplit > 1) ? tc::EPI_ATOMIC : tc::EPI_STORE;
    if (ksplit > 1 && (Z || relu || mask)) return cudaErrorInvalidValue;  // nonlinear epilogue needs full K
    dim3 grid((M + tc::kM - 1) / tc::kM, ksplit);
    tc::k_tc_gemm<TA, TB><<<grid, 128, tc::kSmemBytes, st>>>(A, B, M, N, K, kchunk, bias, Z, z_rs, mask, mask_rs, relu,
                                                             C, c_rs, c_cs, epi, err, 4000000000LL);
    return cudaGetLastError();
}

template cudaError_t tc_gemm<float, float>(cudaStream_t, tc::View<float>, tc::View<float>, int, int, int,
                                           const float *, float *, int64_t, const float *, int64_t, int, float *,
                                           int64_t, int64_t, bool, int *);
template cudaError_t tc_gemm<float, __nv_bfloat16>(cudaStream_t, tc::View<float>, tc::View<__nv_bfloat16>, int, int,
                                                   int, const float *, float *, int64_t, const float *, int64_t,
                                                   int, float *, int64_t, int64_t, bool, int *);


// ---------------------------------------------------------------------------
// learned block-Jacobi correction: graph features, message passing, the
// preconditioner M_i^-1 = L_i^-T T_i T_i^T L_i^-1, probe loss and backward
// ---------------------------------------------------------------------------
namespace gnn {

constexpr int H = 64, NF = 24, NO = 21, NOP = 32;  // hidden, features, outputs (padded)
constexpr float OUT_SCALE = 0.1f;

// packed parameter offsets (FP32): W1 (48 x 64), b1, W2 (128 x 64), b2, Wo (64 x 21), bo
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + 2 * NF * H, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + 2 * H * H,
              OFF_WO = OFF_B2 + H, OFF_BO = OFF_WO + H * NO, NPARAM = OFF_BO + NO;

// Frobenius norms of the diagonal blocks and the log-diagonal sums (for the mean).
template <typename T>
__global__ void k_diag_stats(int n, const int *__restrict__ row_ptr, const T *__restrict__ S, float *__restrict__ dn,
                             float *__restrict__ logd, double *red, unsigned *ctr, float *logd_mean) {
    double v[6] = {0, 0, 0, 0, 0, 0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const T *d = S + (int64_t)row_ptr[i] * BW;
        float s = 0.f;
#pragma unroll
        for (int q = 0; q < 36; ++q) s += (float)d[q] * (float)d[q];
        dn[i] = sqrtf(s);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float l = logf((float)d[7 * k]);
            logd[6 * i + k] = l;
            v[k] += l;
        }
    }
    grid_sum<6>(v, red, ctr, [&](double *t) {
        for (int k = 0; k < 6; ++k) logd_mean[k] = (float)(t[k] / n);
    });
}

// Coupling weight of every stored block: w_b = ||S_b||_F / sqrt(||S_ii|| ||S_jj||); warp per row.
template <typename T>
__global__ void k_block_weights(int n, const int *__restrict__ row_ptr, const int *__restrict__ col,
                                const T *__restrict__ S, const float *__restrict__ dn, float *__restrict__ wb) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = warp; i < n; i += nw)
        for (int b = row_ptr[i] + lane; b < row_ptr[i + 1]; b += 32) {
            const T *B = S + (int64_t)b * BW;
            float s = 0.f;
#pragma unroll
            for (int q = 0; q < 36; ++q) s += (float)B[q] * (float)B[q];
            wb[b] = sqrtf(s) / sqrtf(dn[i] * dn[col[b]]);
        }
}

// Node features (24) into A1[:, 0:24]: 15 correlations of S_ii, 6 centred
// log-diagonals, log(1 + degree), summed edge weight, 1.  Warp per camera.
template <typename T>
__global__ void k_features(int n, const int *__restrict__ row_ptr, const int *__restrict__ tw_ptr,
                           const int2 *__restrict__ tw_ent, const T *__restrict__ S, const float *__restrict__ logd,
                           const float *__restrict__ logd_mean, const float *__restrict__ wb, float *__restrict__ A1,
                           int lda) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = warp; i < n; i += nw) {
        const int tb = tw_ptr[i], te = tw_ptr[i + 1];
        float ws = 0.f;
        for (int t = tb + lane; t < te; t += 32) {
            const int2 e = tw_ent[t];
            if (e.y != i) ws += wb[e.x & 0x7fffffff];
        }
        ws = warp_sum(ws);
        float *x = A1 + (int64_t)i * lda;
        const T *d = S + (int64_t)row_ptr[i] * BW;
        if (lane < 15) {
            // lane -> (r, c), r < c, row by row
            int r = 0, c = lane + 1, k = lane;
            while (k >= 5 - r) { k -= 5 - r; ++r; }
            c = r + 1 + k;
            x[lane] = (float)d[6 * r + c] * rsqrtf((float)d[7 * r]) * rsqrtf((float)d[7 * c]);
        } else if (lane < 21) {
            const int k = lane - 15;
            x[lane] = logd[6 * i + k] - logd_mean[k];
        } else if (lane == 21) {
            x[21] = log1pf((float)(te - tb - 1));
        } else if (lane == 22) {
            x[22] = ws;
        } else if (lane == 23) {
            x[23] = 1.f;
        }
    }
}

// out_i = sum_{j != i, j ~ i} w_ij h_j / max(deg_i, 1)  (forward), or with
// adjoint != 0: out_i = sum_{j ~ i} w_ij h_j / max(deg_j, 1) (the transpose of
// the forward operator; the graph is symmetric).  Warp per camera, lanes over
// the K <= 64 features.  out may alias neither h nor overlap it.
__global__ void k_aggregate(int n, const int *__restrict__ tw_ptr, const int2 *__restrict__ tw_ent,
                            const float *__restrict__ wb, const float *__restrict__ h, int ldh, float *__restrict__ out,
                            int ldo, int K, int adjoint, int accumulate) {
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    for (int i = warp; i < n; i += nw) {
        const int tb = tw_ptr[i], te = tw_ptr[i + 1];
        float a0 = 0.f, a1 = 0.f;
        for (int t = tb; t < te; ++t) {
            const int2 e = tw_ent[t];
            const int j = e.y;
            if (j == i) continue;
            float w = wb[e.x & 0x7fffffff];
            if (adjoint) w /= (float)max(tw_ptr[j + 1] - tw_ptr[j] - 1, 1);
            const float *hj = h + (int64_t)j * ldh;
            if (lane < K) a0 += w * hj[lane];
            if (lane + 32 < K) a1 += w * hj[lane + 32];
        }
        if (!adjoint) {
            const float inv = 1.f / (float)max(te - tb - 1, 1);
            a0 *= inv;
            a1 *= inv;
        }
        float *o = out + (int64_t)i * ldo;
        if (lane < K) o[lane] = accumulate ? o[lane] + a0 : a0;
        if (lane + 32 < K) o[lane + 32] = accumulate ? o[lane + 32] + a1 : a1;
    }
}

// dZ = dH * (Z > 0), in place on dH
__global__ void k_relu_mask(int64_t cnt, float *__restrict__ dH, int ldd, const float *__restrict__ Z, int ldz, int K) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = x / K;
        const int c = (int)(x - r * K);
        if (!(Z[r * ldz + c] > 0.f)) dH[r * ldd + c] = 0.f;
    }
}

// g[c] += sum_r A[r, c] (column sums of an n x K matrix)
__global__ void k_colsum(int n, const float *__restrict__ A, int lda, int K, float *__restrict__ g) {
    const int c = blockIdx.x;
    float s = 0.f;
    for (int r = threadIdx.x; r < n; r += blockDim.x) s += A[(int64_t)r * lda + c];
    double v[1] = {(double)s};
    __shared__ double sh[32];
    block_sum<1>(v, sh);
    if (threadIdx.x == 0 && c < K) g[c] += (float)v[0];
}

__device__ __forceinline__ void chol6_inv(const float *A, float *Li) {
    // A = L L^T, Li = L^-1 (lower, full 6x6 row-major); assumes SPD
    float L[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) L[q] = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float s = A[6 * i + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[6 * i + k] * L[6 * j + k];
            L[6 * i + j] = (i == j) ? sqrtf(fmaxf(s, 1e-30f)) : s / L[6 * j + j];
        }
#pragma unroll
    for (int q = 0; q < 36; ++q) Li[q] = 0.f;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Li[7 * i] = 1.f / L[7 * i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            float s = 0.f;
#pragma unroll
            for (int k = j; k < i; ++k) s += L[6 * i + k] * Li[6 * k + j];
            Li[6 * i + j] = -s * Li[7 * i];
        }
    }
}

// T (lower) from the 21 outputs: T_kk = exp(a o), T_kl = a o
__device__ __forceinline__ void tri_from_out(const float *o, float *T) {
#pragma unroll
    for (int q = 0; q < 36; ++q) T[q] = 0.f;
    int q = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int l = 0; l <= k; ++l, ++q) T[6 * k + l] = (k == l) ? expf(OUT_SCALE * o[q]) : OUT_SCALE * o[q];
}

// M_i^-1 = G G^T with G = L_i^-T T_i; thread per camera.  Writes the mode precision Minv.
template <typename TM, typename T>
__global__ void k_precond(int n, const int *__restrict__ row_ptr, const T *__restrict__ S, const float *__restrict__ O,
                          TM *__restrict__ Minv) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float A[36], Li[36], Tm[36], G[36];
    const T *d = S + (int64_t)row_ptr[i] * BW;
#pragma unroll
    for (int q = 0; q < 36; ++q) A[q] = (float)d[q];
    chol6_inv(A, Li);
    tri_from_out(O + (int64_t)i * NOP, Tm);
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s += Li[6 * k + r] * Tm[6 * k + c];
            G[6 * r + c] = s;
        }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s += G[6 * r + k] * G[6 * c + k];
            Minv[36 * (int64_t)i + 6 * r + c] = (TM)s;
        }
}

// M_i^-1, G_i = L_i^-T T_i and L_i^-1 of camera i from S_ii and its outputs.
template <typename T>
__device__ __forceinline__ void precond_parts(const T *__restrict__ d, const float *__restrict__ o, float *M, float *G,
                                              float *Li, float *Tm) {
    float A[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) A[q] = (float)d[q];
    chol6_inv(A, Li);
    tri_from_out(o, Tm);
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s += Li[6 * k + r] * Tm[6 * k + c];
            G[6 * r + c] = s;
        }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s += G[6 * r + k] * G[6 * c + k];
            M[6 * r + c] = s;
        }
}

// Energy loss, stage 1: z_p = M^-1 u_p per camera; a = sum z^T u, e = sum w^T u.
template <typename T>
__global__ void k_energy_z(int n, int kp, const int *__restrict__ row_ptr, const T *__restrict__ S,
                           const float *__restrict__ O, const float *__restrict__ Wp, const float *__restrict__ Up,
                           float *__restrict__ Zp, double *red, unsigned *ctr, double *scal) {
    RunSum<float> sa, se;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float M[36], G[36], Li[36], Tm[36];
        precond_parts<T>(S + (int64_t)row_ptr[i] * BW, O + (int64_t)i * NOP, M, G, Li, Tm);
        for (int p = 0; p < kp; ++p) {
            const int64_t o6 = ((int64_t)p * n + i) * 6;
            float u[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) u[c] = Up[o6 + c];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                float z = 0.f;
#pragma unroll
                for (int c = 0; c < 6; ++c) z += M[6 * r + c] * u[c];
                Zp[o6 + r] = z;
                sa.add(z * u[r]);
                se.add(Wp[o6 + r] * u[r]);
            }
        }
    }
    double v[2] = {sa.get(), se.get()};
    grid_sum<2>(v, red, ctr, [&](double *t) {
        scal[1] = t[0];  // a
        scal[3] = t[1];  // e
    });
}

// Energy loss, stage 2: c = sum z^T (S z); loss = 1 - a^2 / (c e).
__global__ void k_energy_c(int64_t cnt, const float *__restrict__ Zp, const float *__restrict__ Vp, double *red,
                           unsigned *ctr, double *scal) {
    RunSum<float> sc;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x)
        sc.add(Zp[x] * Vp[x]);
    double v[1] = {sc.get()};
    grid_sum<1>(v, red, ctr, [&](double *t) {
        scal[2] = t[0];  // c
        scal[0] = 1.0 - scal[1] * scal[1] / (t[0] * scal[3]);
    });
}

// Energy loss, stage 3: d loss / d o per camera.
//   dz_p = (2a/(ce)) ((a/c) v_p - u_p),  dM = sum_p dz_p u_p^T,
//   dG = (dM + dM^T) G,  dT = L^-1 dG,  dO from dT.
template <typename T>
__global__ void k_energy_grad(int n, int kp, const int *__restrict__ row_ptr, const T *__restrict__ S,
                              const float *__restrict__ O, const float *__restrict__ Up, const float *__restrict__ Vp,
                              const double *__restrict__ scal, float *__restrict__ dO) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double a = scal[1], c = scal[2], e = scal[3];
    const float f1 = (float)(2.0 * a / (c * e)), f2 = (float)(a / c);
    float M[36], G[36], Li[36], Tm[36], dM[36];
    precond_parts<T>(S + (int64_t)row_ptr[i] * BW, O + (int64_t)i * NOP, M, G, Li, Tm);
#pragma unroll
    for (int q = 0; q < 36; ++q) dM[q] = 0.f;
    for (int p = 0; p < kp; ++p) {
        const int64_t o6 = ((int64_t)p * n + i) * 6;
        float u[6], dz[6];
#pragma unroll
        for (int c2 = 0; c2 < 6; ++c2) {
            u[c2] = Up[o6 + c2];
            dz[c2] = f1 * (f2 * Vp[o6 + c2] - u[c2]);
        }
#pragma unroll
        for (int r = 0; r < 6; ++r)
#pragma unroll
            for (int c2 = 0; c2 < 6; ++c2) dM[6 * r + c2] += dz[r] * u[c2];
    }
    float S2[36], dG[36], dT[36];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c2 = 0; c2 < 6; ++c2) S2[6 * r + c2] = dM[6 * r + c2] + dM[6 * c2 + r];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c2 = 0; c2 < 6; ++c2) {
            float s2 = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s2 += S2[6 * r + k] * G[6 * k + c2];
            dG[6 * r + c2] = s2;
        }
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c2 = 0; c2 < 6; ++c2) {
            float s2 = 0.f;
#pragma unroll
            for (int k = 0; k < 6; ++k) s2 += Li[6 * r + k] * dG[6 * k + c2];
            dT[6 * r + c2] = s2;
        }
    float *g = dO + (int64_t)i * NOP;
    int q = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int l2 = 0; l2 <= k; ++l2, ++q) g[q] = dT[6 * k + l2] * (k == l2 ? OUT_SCALE * Tm[7 * k] : OUT_SCALE);
#pragma unroll
    for (int q2 = NO; q2 < NOP; ++q2) g[q2] = 0.f;
}

// Rademacher probes from a counter-based hash (splitmix64 of seed, index).
__global__ void k_probes(int64_t cnt, uint64_t seed, float *__restrict__ Wp) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < cnt; x += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(x + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        Wp[x] = (z & 1ull) ? 1.f : -1.f;
    }
}

// Adam on the packed parameters (decoupled from the loss; bias-corrected).
__global__ void k_adam(int np, float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= np) return;
    const float gi = g[x];
    const float mi = b1 * m[x] + (1.f - b1) * gi, vi = b2 * v[x] + (1.f - b2) * gi * gi;
    m[x] = mi;
    v[x] = vi;
    w[x] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

}  // namespace gnn
}  // namespace ba

using namespace ba;

// C[M x N] = A[M x K] * B[K x N] (or C += ... when accumulate != 0), FP32 in
// and out, BF16 operands on the tensor cores with FP32 accumulation.  All
// pointers are device pointers; a_rs/a_cs etc. are element strides of rows and
// columns.  err_dev: a device int that receives BA_ERR_TIMEOUT if a bounded
// wait gave up (NULL: none).
extern "C" ba_status ba_tc_gemm(int32_t M, int32_t N, int32_t K, const float *A, int64_t a_rs, int64_t a_cs,
                                const float *B, int64_t b_rs, int64_t b_cs, float *C, int64_t c_rs, int64_t c_cs,
                                int32_t accumulate, int32_t *err_dev, void *cuda_stream) {
    if (M < 0 || K < 0 || N <= 0 || N > 128 || N % 32 != 0)
        return set_error(BA_ERR_INVALID_ARG, "ba_tc_gemm: need M, K >= 0 and N in {32, 64, 96, 128}");
    if ((M > 0 && K > 0) && (!A || !B || !C)) return set_error(BA_ERR_INVALID_ARG, "ba_tc_gemm: null pointer");
    // without a caller's error word, one per device (kept for the process)
    static std::mutex err_mu;
    static std::map<int, int *> err_words;
    int *err = err_dev;
    if (!err) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return set_error(BA_ERR_CUDA, "cudaGetDevice");
        std::lock_guard<std::mutex> lock(err_mu);
        int *&w = err_words[dev];
        if (!w && cudaMalloc(&w, sizeof(int)) != cudaSuccess) return set_error(BA_ERR_CUDA, "cudaMalloc");
        err = w;
    }
    tc::View<float> va{A, a_rs, a_cs, M, K};
    tc::View<float> vb{B, b_rs, b_cs, K, N};
    cudaError_t e = tc_gemm<float, float>((cudaStream_t)cuda_stream, va, vb, M, N, K, nullptr, nullptr, 0, nullptr, 0,
                                          0, C, c_rs, c_cs, accumulate != 0, err);
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    return BA_OK;
}

// ---------------------------------------------------------------------------
// host side of the learned preconditioner
// ---------------------------------------------------------------------------
struct ba_precond_net {
    float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // packed FP32 parameters
    float *wo_pad = nullptr, *bo_pad = nullptr;                    // Wo (64 x 32), bo (32) zero-padded views
    int64_t step = 0;
    cudaStream_t st = nullptr;
    int *err = nullptr;
    double *loss = nullptr;  // [loss, a, c, e] of the last training step
};

namespace ba {

struct GnnWork {
    int n = 0, kp = 0;
    float *dn = nullptr, *logd = nullptr, *logd_mean = nullptr, *wb = nullptr;
    float *A1 = nullptr, *Z1 = nullptr, *A2 = nullptr, *Z2 = nullptr, *H2 = nullptr, *O = nullptr;
    float *dO = nullptr, *dZ2 = nullptr, *dA2 = nullptr, *dZ1 = nullptr;
    float *Wp = nullptr, *Up = nullptr, *Zp = nullptr, *Vp = nullptr;
    std::vector<void *> bufs;
};

using namespace gnn;

static cudaError_t galloc(GnnWork *w, float **p, size_t cnt) {
    void *q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(cnt, 4) * sizeof(float));
    if (e != cudaSuccess) return e;
    w->bufs.push_back(q);
    *p = (float *)q;
    return cudaSuccess;
}

void gnn_free(ba_problem *p) {
    if (p->gw) {
        for (void *q : p->gw->bufs) cudaFree(q);
        delete p->gw;
        p->gw = nullptr;
    }
}

static cudaError_t ensure_work(ba_problem *p, int kp) {
    GnnWork *w = p->gw;
    if (w && w->kp >= kp) return cudaSuccess;
    if (w) gnn_free(p);
    w = new GnnWork();
    p->gw = w;
    const int64_t n = p->n;
    w->n = (int)n;
    w->kp = kp;
    cudaError_t e = cudaSuccess;
    auto A = [&](float **q, size_t c) { if (e == cudaSuccess) e = galloc(w, q, c); };
    A(&w->dn, n); A(&w->logd, 6 * n); A(&w->logd_mean, 8); A(&w->wb, p->nnzb);
    A(&w->A1, n * 2 * NF); A(&w->Z1, n * H); A(&w->A2, n * 2 * H); A(&w->Z2, n * H); A(&w->H2, n * H);
    A(&w->O, n * NOP); A(&w->dO, n * NOP); A(&w->dZ2, n * H); A(&w->dA2, n * 2 * H); A(&w->dZ1, n * H);
    if (kp > 0) {
        A(&w->Wp, (size_t)kp * n * 6); A(&w->Up, (size_t)kp * n * 6);
        A(&w->Zp, (size_t)kp * n * 6); A(&w->Vp, (size_t)kp * n * 6);
    }
    return e;
}

static inline int gridw(int64_t warps_work, int cap) {
    int64_t g = (warps_work * 32 + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, cap));
}

// forward: features, two message-passing layers, output layer -> w->O
template <typename T>
static cudaError_t forward_T(ba_problem *p, ba_precond_net *net) {
    GnnWork *w = p->gw;
    const int n = p->n;
    cudaStream_t st = p->st;
    cudaError_t e;
    const T *S = (const T *)p->S;
    const int gv = (int)std::min<int64_t>((n + 255) / 256, 152 * 4);
    k_diag_stats<T><<<gv, 256, 0, st>>>(n, p->row_ptr, S, w->dn, w->logd, p->red, p->counters + 8, w->logd_mean);
    k_block_weights<T><<<gridw(n, 152 * 8), 256, 0, st>>>(n, p->row_ptr, p->col, S, w->dn, w->wb);
    k_features<T><<<gridw(n, 152 * 8), 256, 0, st>>>(n, p->row_ptr, p->tw_ptr, p->tw_ent, S, w->logd, w->logd_mean,
                                                     w->wb, w->A1, 2 * NF);
    k_aggregate<<<gridw(n, 152 * 8), 256, 0, st>>>(n, p->tw_ptr, p->tw_ent, w->wb, w->A1, 2 * NF, w->A1 + NF, 2 * NF,
                                                   NF, 0, 0);
    p->launches += 4;
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // layer 1: Z1 = A1 W1 + b1, H1 = relu -> A2[:, 0:64]
    tc::View<float> a1{w->A1, 2 * NF, 1, n, 2 * NF}, b1{net->w + OFF_W1, H, 1, 2 * NF, H};
    if ((e = tc_gemm<float, float>(st, a1, b1, n, H, 2 * NF, net->w + OFF_B1, w->Z1, H, nullptr, 0, 1, w->A2, 2 * H,
                                   1, false, net->err)) != cudaSuccess)
        return e;
    k_aggregate<<<gridw(n, 152 * 8), 256, 0, st>>>(n, p->tw_ptr, p->tw_ent, w->wb, w->A2, 2 * H, w->A2 + H, 2 * H, H,
                                                   0, 0);
    // layer 2: Z2 = A2 W2 + b2, H2 = relu
    tc::View<float> a2{w->A2, 2 * H, 1, n, 2 * H}, b2{net->w + OFF_W2, H, 1, 2 * H, H};
    if ((e = tc_gemm<float, float>(st, a2, b2, n, H, 2 * H, net->w + OFF_B2, w->Z2, H, nullptr, 0, 1, w->H2, H, 1,
                                   false, net->err)) != cudaSuccess)
        return e;
    // output: O = H2 Wo + bo (21 of 32 columns)
    tc::View<float> a3{w->H2, H, 1, n, H}, b3{net->wo_pad, NOP, 1, H, NOP};
    if ((e = tc_gemm<float, float>(st, a3, b3, n, NOP, H, net->bo_pad, nullptr, 0, nullptr, 0, 0, w->O, NOP, 1, false,
                                   net->err)) != cudaSuccess)
        return e;
    p->launches += 4;
    return cudaGetLastError();
}

static cudaError_t forward(ba_problem *p, ba_precond_net *net) {
    return p->fp32 ? forward_T<float>(p, net) : forward_T<double>(p, net);
}

// Wo / bo zero-padded copies for the N = 32 output GEMM
__global__ void k_pad_out(const float *__restrict__ w, float *__restrict__ wo_pad, float *__restrict__ bo_pad) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < H * NOP) {
        const int r = x / NOP, c = x - r * NOP;
        wo_pad[x] = c < NO ? w[OFF_WO + r * NO + c] : 0.f;
    }
    if (x < NOP) bo_pad[x] = x < NO ? w[OFF_BO + x] : 0.f;
}
// gradient of Wo / bo from the padded gradient buffers
__global__ void k_unpad_grad(const float *__restrict__ gwo_pad, const float *__restrict__ gbo_pad, float *__restrict__ g) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x < H * NO) {
        const int r = x / NO, c = x - r * NO;
        g[OFF_WO + x] = gwo_pad[r * NOP + c];
    }
    if (x < NO) g[OFF_BO + x] = gbo_pad[x];
}

static cudaError_t refresh_pad(ba_precond_net *net) {
    k_pad_out<<<(H * NOP + 255) / 256, 256, 0, net->st>>>(net->w, net->wo_pad, net->bo_pad);
    return cudaGetLastError();
}

// loss and gradients (into net->g) on the problem's last RCS
template <typename T>
static cudaError_t loss_grad_T(ba_problem *p, ba_precond_net *net, int kp) {
    GnnWork *w = p->gw;
    const int n = p->n;
    cudaStream_t st = p->st;
    cudaError_t e;
    // U = S W, Z = M^-1 U, V = S Z for each probe; energy loss and d loss / d o
    for (int k = 0; k < kp; ++k)
        if ((e = launch_spmv_f32(p, w->Wp + (int64_t)k * n * 6, w->Up + (int64_t)k * n * 6)) != cudaSuccess) return e;
    const int gv = (int)std::min<int64_t>((n + 127) / 128, 152 * 4);
    k_energy_z<T><<<gv, 128, 0, st>>>(n, kp, p->row_ptr, (const T *)p->S, w->O, w->Wp, w->Up, w->Zp, p->red,
                                      p->counters + 9, net->loss);
    for (int k = 0; k < kp; ++k)
        if ((e = launch_spmv_f32(p, w->Zp + (int64_t)k * n * 6, w->Vp + (int64_t)k * n * 6)) != cudaSuccess) return e;
    const int64_t cnt = (int64_t)kp * n * 6;
    k_energy_c<<<(int)std::min<int64_t>((cnt + 255) / 256, 1024), 256, 0, st>>>(cnt, w->Zp, w->Vp, p->red,
                                                                                  p->counters + 10, net->loss);
    k_energy_grad<T><<<(n + 127) / 128, 128, 0, st>>>(n, kp, p->row_ptr, (const T *)p->S, w->O, w->Up, w->Vp,
                                                      net->loss, w->dO);
    if ((e = cudaMemsetAsync(net->g, 0, sizeof(float) * (NPARAM + H * NOP + NOP), st)) != cudaSuccess) return e;
    float *gwo_pad = net->g + NPARAM, *gbo_pad = gwo_pad + H * NOP;
    // output layer: dWo = H2^T dO, dbo = colsum(dO), dH2 = dO Wo^T masked by Z2 > 0 -> dZ2
    tc::View<float> h2t{w->H2, 1, H, H, n}, dov{w->dO, NOP, 1, n, NOP};
    if ((e = tc_gemm<float, float>(st, h2t, dov, H, NOP, n, nullptr, nullptr, 0, nullptr, 0, 0, gwo_pad, NOP, 1, true,
                                   net->err)) != cudaSuccess)
        return e;
    k_colsum<<<NOP, 256, 0, st>>>(n, w->dO, NOP, NOP, gbo_pad);
    tc::View<float> dov2{w->dO, NOP, 1, n, NOP}, wot{net->wo_pad, 1, NOP, NOP, H};
    if ((e = tc_gemm<float, float>(st, dov2, wot, n, H, NOP, nullptr, nullptr, 0, w->Z2, H, 0, w->dZ2, H, 1, false,
                                   net->err)) != cudaSuccess)
        return e;
    // layer 2: dW2 = A2^T dZ2, db2 = colsum(dZ2), dA2 = dZ2 W2^T
    tc::View<float> a2t{w->A2, 1, 2 * H, 2 * H, n}, dz2{w->dZ2, H, 1, n, H};
    if ((e = tc_gemm<float, float>(st, a2t, dz2, 2 * H, H, n, nullptr, nullptr, 0, nullptr, 0, 0, net->g + OFF_W2, H,
                                   1, true, net->err)) != cudaSuccess)
        return e;
    k_colsum<<<H, 256, 0, st>>>(n, w->dZ2, H, H, net->g + OFF_B2);
    tc::View<float> dz2b{w->dZ2, H, 1, n, H}, w2t{net->w + OFF_W2, 1, H, H, 2 * H};
    if ((e = tc_gemm<float, float>(st, dz2b, w2t, n, 2 * H, H, nullptr, nullptr, 0, nullptr, 0, 0, w->dA2, 2 * H, 1,
                                   false, net->err)) != cudaSuccess)
        return e;
    // dH1 = dA2[:, :64] + agg^T(dA2[:, 64:]), dZ1 = dH1 * (Z1 > 0)
    if ((e = cudaMemcpy2DAsync(w->dZ1, H * sizeof(float), w->dA2, 2 * H * sizeof(float), H * sizeof(float), n,
                               cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
        return e;
    k_aggregate<<<gridw(n, 152 * 8), 256, 0, st>>>(n, p->tw_ptr, p->tw_ent, w->wb, w->dA2 + H, 2 * H, w->dZ1, H, H, 1,
                                                   1);
    k_relu_mask<<<gridw((int64_t)n * H / 32 + 1, 152 * 8), 256, 0, st>>>((int64_t)n * H, w->dZ1, H, w->Z1, H, H);
    // layer 1: dW1 = A1^T dZ1, db1 = colsum(dZ1)
    tc::View<float> a1t{w->A1, 1, 2 * NF, 2 * NF, n}, dz1{w->dZ1, H, 1, n, H};
    if ((e = tc_gemm<float, float>(st, a1t, dz1, 2 * NF, H, n, nullptr, nullptr, 0, nullptr, 0, 0, net->g + OFF_W1, H,
                                   1, true, net->err)) != cudaSuccess)
        return e;
    k_colsum<<<H, 256, 0, st>>>(n, w->dZ1, H, H, net->g + OFF_B1);
    k_unpad_grad<<<(H * NO + 255) / 256, 256, 0, st>>>(gwo_pad, gbo_pad, net->g);
    p->launches += 8 + kp;
    return cudaGetLastError();
}

ba_status gnn_apply(ba_problem *p) {
    ba_precond_net *net = p->net;
    if (!net) return BA_OK;
    cudaError_t e = ensure_work(p, 0);
    if (e == cudaSuccess && !p->Minv_bj) {
        void *q = nullptr;
        e = cudaMalloc(&q, (size_t)p->n * 36 * p->esz);
        if (e == cudaSuccess) p->Minv_bj = q;
    }
    // keep the block-Jacobi M^-1 for the fallback (not a learned one left by
    // an earlier solve of the same RCS)
    if (e == cudaSuccess && !p->minv_learned)
        e = cudaMemcpyAsync(p->Minv_bj, p->Minv, (size_t)p->n * 36 * p->esz, cudaMemcpyDeviceToDevice, p->st);
    if (e == cudaSuccess) e = forward(p, net);
    if (e == cudaSuccess) {
        const int nb = (p->n + 127) / 128;
        if (p->fp32)
            k_precond<float, float><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (const float *)p->S, p->gw->O,
                                                           (float *)p->Minv);
        else
            k_precond<double, double><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (const double *)p->S, p->gw->O,
                                                             (double *)p->Minv);
        p->launches += 1;
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        p->dead = true;
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    }
    p->minv_learned = true;
    return BA_OK;
}

ba_status gnn_restore_block_jacobi(ba_problem *p) {
    p->minv_learned = false;
    if (!p->Minv_bj) return BA_OK;
    cudaError_t e = cudaMemcpyAsync(p->Minv, p->Minv_bj, (size_t)p->n * 36 * p->esz, cudaMemcpyDeviceToDevice, p->st);
    if (e != cudaSuccess) {
        p->dead = true;
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    }
    return BA_OK;
}

}  // namespace ba

static ba_status net_sync(ba_precond_net *net, cudaStream_t st) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    int err = 0;
    if ((e = cudaMemcpy(&err, net->err, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    if (err) return set_error((ba_status)err, "a bounded device wait gave up");
    return BA_OK;
}

extern "C" {

int32_t ba_precond_net_num_params(void) { return gnn::NPARAM; }

ba_status ba_precond_net_create(const float *params, uint64_t seed, void *cuda_stream, ba_precond_net **out) {
    if (!out) return set_error(BA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    ba_precond_net *net = new ba_precond_net();
    net->st = (cudaStream_t)cuda_stream;
    const size_t np = gnn::NPARAM, extra = gnn::H * gnn::NOP + gnn::NOP;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **q, size_t bytes) { if (e == cudaSuccess) e = cudaMalloc(q, bytes); };
    A((void **)&net->w, np * 4); A((void **)&net->g, (np + extra) * 4); A((void **)&net->m, np * 4);
    A((void **)&net->v, np * 4); A((void **)&net->wo_pad, extra * 4); A((void **)&net->err, sizeof(int));
    A((void **)&net->loss, 4 * sizeof(double));
    if (e == cudaSuccess) {
        net->bo_pad = net->wo_pad + gnn::H * gnn::NOP;
        std::vector<float> h(np, 0.f);
        if (params) {
            std::copy(params, params + np, h.begin());
        } else {
            // He-normal hidden layers from a seeded generator, zero output layer (= block-Jacobi)
            uint64_t st = seed * 0x9E3779B97F4A7C15ull + 1;
            auto next = [&]() {
                st ^= st << 13; st ^= st >> 7; st ^= st << 17;
                return ((st >> 11) + 0.5) * (1.0 / 9007199254740992.0);
            };
            auto normal = [&]() { return sqrt(-2.0 * log(next())) * cos(6.283185307179586 * next()); };
            for (int k = 0; k < 2 * gnn::NF * gnn::H; ++k) h[gnn::OFF_W1 + k] = (float)(normal() * sqrt(2.0 / (2 * gnn::NF)));
            for (int k = 0; k < 2 * gnn::H * gnn::H; ++k) h[gnn::OFF_W2 + k] = (float)(normal() * sqrt(2.0 / (2 * gnn::H)));
        }
        e = cudaMemcpy(net->w, h.data(), np * 4, cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemset(net->m, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(net->v, 0, np * 4);
    if (e == cudaSuccess) e = cudaMemset(net->err, 0, sizeof(int));
    if (e == cudaSuccess) {
        ba::k_pad_out<<<(gnn::H * gnn::NOP + 255) / 256, 256>>>(net->w, net->wo_pad, net->bo_pad);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ba_precond_net_destroy(net);
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    }
    *out = net;
    return BA_OK;
}

void ba_precond_net_destroy(ba_precond_net *net) {
    if (!net) return;
    for (void *q : {(void *)net->w, (void *)net->g, (void *)net->m, (void *)net->v, (void *)net->wo_pad,
                    (void *)net->err, (void *)net->loss})
        if (q) cudaFree(q);
    delete net;
}

ba_status ba_precond_net_get_params(const ba_precond_net *net, float *out) {
    if (!net || !out) return set_error(BA_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpy(out, net->w, gnn::NPARAM * 4, cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? BA_OK : set_error(BA_ERR_CUDA, cudaGetErrorString(e));
}

ba_status ba_precond_net_set_params(ba_precond_net *net, const float *params) {
    if (!net || !params) return set_error(BA_ERR_INVALID_ARG, "null argument");
    cudaError_t e = cudaMemcpy(net->w, params, gnn::NPARAM * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = ba::refresh_pad(net);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? BA_OK : set_error(BA_ERR_CUDA, cudaGetErrorString(e));
}

ba_status ba_set_precond_net(ba_problem *p, ba_precond_net *net) {
    if (!p) return set_error(BA_ERR_INVALID_ARG, "null problem");
    p->net = net;
    return BA_OK;
}

// Forward pass on the problem's last RCS: outputs o (n x 21) and M^-1 (n x 36),
// both may be NULL.  Host buffers.
ba_status ba_precond_net_forward(ba_precond_net *net, ba_problem *p, float *out_o, double *out_minv) {
    if (!net || !p) return set_error(BA_ERR_INVALID_ARG, "null argument");
    if (!p->rcs_formed) return set_error(BA_ERR_STATE, "no RCS formed");
    cudaError_t e = ba::ensure_work(p, 0);
    if (e == cudaSuccess) e = ba::forward(p, net);
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    ba_status s = net_sync(net, p->st);
    if (s) return s;
    const int n = p->n;
    if (out_o) {
        std::vector<float> o((size_t)n * gnn::NOP);
        if ((e = cudaMemcpy(o.data(), p->gw->O, o.size() * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
            return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
        for (int i = 0; i < n; ++i)
            for (int q = 0; q < gnn::NO; ++q) out_o[(size_t)i * gnn::NO + q] = o[(size_t)i * gnn::NOP + q];
    }
    if (out_minv) {
        float *tmp = nullptr;
        if ((e = cudaMalloc(&tmp, (size_t)n * 36 * 4)) != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
        const int nb = (n + 127) / 128;
        if (p->fp32)
            ba::gnn::k_precond<float, float><<<nb, 128, 0, p->st>>>(n, p->row_ptr, (const float *)p->S, p->gw->O, tmp);
        else
            ba::gnn::k_precond<float, double><<<nb, 128, 0, p->st>>>(n, p->row_ptr, (const double *)p->S, p->gw->O, tmp);
        std::vector<float> h((size_t)n * 36);
        e = cudaStreamSynchronize(p->st);
        if (e == cudaSuccess) e = cudaMemcpy(h.data(), tmp, h.size() * 4, cudaMemcpyDeviceToHost);
        cudaFree(tmp);
        if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
        for (size_t k = 0; k < h.size(); ++k) out_minv[k] = h[k];
    }
    return BA_OK;
}

// Probe loss and gradients on the problem's last RCS.  probes: host array
// (kp x n x 6) or NULL for Rademacher probes drawn from seed.  grads (host,
// ba_precond_net_num_params() floats) may be NULL.  If lr > 0 an Adam step
// (beta1 0.9, beta2 0.999, eps 1e-8) follows.
ba_status ba_precond_net_train_step(ba_precond_net *net, ba_problem *p, int32_t kp, const float *probes,
                                    uint64_t seed, double lr, double *loss, float *grads) {
    if (!net || !p || kp <= 0) return set_error(BA_ERR_INVALID_ARG, "bad argument");
    if (!p->rcs_formed) return set_error(BA_ERR_STATE, "no RCS formed");
    cudaError_t e = ba::ensure_work(p, kp);
    const int64_t cnt = (int64_t)kp * p->n * 6;
    if (e == cudaSuccess) {
        if (probes) e = cudaMemcpyAsync(p->gw->Wp, probes, cnt * 4, cudaMemcpyHostToDevice, p->st);
        else {
            ba::gnn::k_probes<<<(int)std::min<int64_t>((cnt + 255) / 256, 4096), 256, 0, p->st>>>(cnt, seed, p->gw->Wp);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) e = ba::forward(p, net);
    if (e == cudaSuccess) e = p->fp32 ? ba::loss_grad_T<float>(p, net, kp) : ba::loss_grad_T<double>(p, net, kp);
    if (e == cudaSuccess && lr > 0) {
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - powf(b1, (float)net->step), c2 = 1.f - powf(b2, (float)net->step);
        ba::gnn::k_adam<<<(ba::gnn::NPARAM + 255) / 256, 256, 0, p->st>>>(ba::gnn::NPARAM, net->w, net->g, net->m,
                                                                          net->v, (float)lr, b1, b2, 1e-8f, c1, c2);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            ba::k_pad_out<<<(ba::gnn::H * ba::gnn::NOP + 255) / 256, 256, 0, p->st>>>(net->w, net->wo_pad,
                                                                                             net->bo_pad);
            e = cudaGetLastError();
        }
        p->launches += 2;
    }
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    ba_status s = net_sync(net, p->st);
    if (s) return s;
    if (loss && (e = cudaMemcpy(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    if (grads && (e = cudaMemcpy(grads, net->g, ba::gnn::NPARAM * 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    return BA_OK;
}

}  // extern "C"
