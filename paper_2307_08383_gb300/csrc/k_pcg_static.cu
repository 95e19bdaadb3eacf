// Allocation-free block-Jacobi PCG on a caller-owned BSMC system (FP32).
//
// Some callers cannot call cudaMalloc: code that runs while a framework owns
// the device memory pool (a caching allocator, a fixed arena), real-time
// loops that must not take the allocator's lock or its implicit device
// synchronisation, and hosts with a hard device-memory budget.  For them
// ba_pcg_solve_static solves S x = b with the caller's device buffers for the
// inputs and the output, and keeps its own scratch (the PCG vectors r, z, d,
// q, the block-Jacobi inverses and the reduction slots) in one file-scope
// __device__ array of fixed size.  The array is created when the library is
// loaded on a device and lives until the process exits, on every GPU that
// loads the library.
//
// Every call shares the one array: calls that overlap on the GPU (two streams,
// or two host threads) race on it.  Each call clears the reduction counters
// and the product vector before use; the array otherwise keeps whatever the
// last call left.
#include <mutex>

#include "device_util.cuh"

namespace ba {

namespace {

constexpr int kStaticMaxCams = 8192;
constexpr size_t kScalOff = 0;      // StaticScalars
constexpr size_t kCtrOff = 256;     // reduction counters
constexpr size_t kRedOff = 512;     // per-CTA partial sums (4096 doubles)
constexpr size_t kVecBytes = (size_t)6 * kStaticMaxCams * sizeof(float);
constexpr size_t kVecOff = kRedOff + 4096 * sizeof(double);  // r, z, d0, d1, q
constexpr size_t kMinvOff = kVecOff + 5 * kVecBytes;
constexpr size_t kStaticBytes = kMinvOff + (size_t)36 * kStaticMaxCams * sizeof(float);
static_assert(kVecOff % 256 == 0 && kVecBytes % 256 == 0 && kMinvOff % 256 == 0, "scratch layout");

struct StaticScalars {
    double rz, pAp, rr, rr0, alpha, beta, tol2;
    int iters, done, max_iters, err;
};
static_assert(sizeof(StaticScalars) <= 256, "scalar slot");

static __device__ __align__(256) unsigned char g_pcg_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_ptr[kMaxDevices] = {};

// Block-Jacobi: M_i^-1 = inverse of the first (diagonal) block of row i.
// Row i is checked first: its blocks lie in [0, nnzb), the first is the
// diagonal block and the other columns ascend above i (the upper-triangle
// layout).  A malformed row - for instance one of a matrix stored with both
// triangles, which the two-sided product would count twice - sets
// BA_ERR_INVALID_ARG; a diagonal block that is not SPD sets BA_ERR_NOT_SPD.
// Either error stops the solve before its first iteration.
__global__ void k_static_minv(int n, int64_t nnzb, const int *__restrict__ row_ptr, const int *__restrict__ col,
                              const float *__restrict__ val, float *__restrict__ Minv, StaticScalars *sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double A[36], Ai[36];
    const int rs = row_ptr[i], re = row_ptr[i + 1];
    bool ok = rs >= 0 && re > rs && (int64_t)re <= nnzb && (i + 1 < n || (int64_t)re == nnzb) && col[rs] == i;
    for (int k = rs + 1; ok && k < re; ++k) ok = col[k] > col[k - 1] && col[k] < n;
    if (!ok) {
        atomicExch(&sc->err, (int)BA_ERR_INVALID_ARG);
#pragma unroll
        for (int q = 0; q < 36; ++q) Minv[36 * (int64_t)i + q] = 0.f;
        return;
    }
    const float *d = val + (int64_t)rs * BW;
#pragma unroll
    for (int q = 0; q < 36; ++q) A[q] = d[q];
    if (!spd_inverse6<double>(A, Ai)) {
        atomicCAS(&sc->err, 0, (int)BA_ERR_NOT_SPD);
#pragma unroll
        for (int q = 0; q < 36; ++q) Ai[q] = 0.0;
    }
#pragma unroll
    for (int q = 0; q < 36; ++q) Minv[36 * (int64_t)i + q] = (float)Ai[q];
}

__device__ __forceinline__ void minv_apply(const float *__restrict__ Minv, int i, const float *r, float *z) {
    const float *M = Minv + 36 * (int64_t)i;
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        float s = 0.f;
#pragma unroll
        for (int c = 0; c < 6; ++c) s += M[6 * a + c] * r[c];
        z[a] = s;
    }
}

// r = b, x = 0, q = 0, d_old = 0, z = M^-1 r, r^T z, r^T r
__global__ void k_static_init(int n, const float *__restrict__ b, float *x, float *r, float *z, float *dold,
                              float *q, const float *__restrict__ Minv, StaticScalars *sc, double tol2,
                              int max_iters, double *red, unsigned *ctr) {
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float ri[6], zi[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            ri[c] = b[6 * i + c];
            r[6 * i + c] = ri[c];
            x[6 * i + c] = 0.f;
            q[6 * i + c] = 0.f;
            dold[6 * i + c] = 0.f;
        }
        minv_apply(Minv, i, ri, zi);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[6 * i + c] = zi[c];
            v[0] += (double)ri[c] * zi[c];
            v[1] += (double)ri[c] * ri[c];
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
        // a malformed row or an indefinite diagonal block ends the solve here
        sc->done = (t[1] == 0.0 || max_iters <= 0 || sc->err != 0) ? 1 : 0;
    });
}

// d_new = z + beta d_old (row owner stores it), q += S d_new, d^T S d.
__global__ void __launch_bounds__(256) k_static_spmv(int n, const int *__restrict__ row_ptr, const int *__restrict__ col,
                                                     const float *__restrict__ S, const float *__restrict__ z,
                                                     const float *__restrict__ dold, float *__restrict__ dnew,
                                                     float *q, StaticScalars *sc, double *red, unsigned *ctr) {
    if (sc->done) return;
    const float beta = (float)sc->beta;
    const int lane = threadIdx.x & 31;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    double pap = 0.0;
    for (int i = warp; i < n; i += nw) {
        float di[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) di[c] = z[6 * i + c] + beta * dold[6 * i + c];
#pragma unroll
        for (int c = 0; c < 6; ++c)
            if (lane == c) dnew[6 * i + c] = di[c];
        float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int blk = row_ptr[i] + lane; blk < row_ptr[i + 1]; blk += 32) {
            const int j = col[blk];
            const float *Sb = S + (int64_t)blk * BW;
            float Sv[36], dj[6];
#pragma unroll
            for (int t = 0; t < 36; ++t) Sv[t] = Sb[t];
#pragma unroll
            for (int c = 0; c < 6; ++c) dj[c] = (j == i) ? di[c] : z[6 * j + c] + beta * dold[6 * j + c];
            double qf = 0.0;
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                float t = 0.f;
#pragma unroll
                for (int c = 0; c < 6; ++c) t += Sv[6 * r + c] * dj[c];
                acc[r] += t;
                qf += (double)di[r] * t;
            }
            if (j != i) {
                pap += 2.0 * qf;
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    float u = 0.f;
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

// x += alpha d, r -= alpha q, q = 0, z = M^-1 r, r^T z, r^T r; stop test
__global__ void __launch_bounds__(256) k_static_update(int n, const float *__restrict__ Minv, const float *__restrict__ d,
                                                       float *q, float *x, float *r, float *z, StaticScalars *sc,
                                                       double *red, unsigned *ctr) {
    if (sc->done) return;
    const float alpha = (float)sc->alpha;
    double v[2] = {0.0, 0.0};
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float ri[6], zi[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            x[6 * i + c] += alpha * d[6 * i + c];
            ri[c] = r[6 * i + c] - alpha * q[6 * i + c];
            r[6 * i + c] = ri[c];
            q[6 * i + c] = 0.f;
        }
        minv_apply(Minv, i, ri, zi);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
            z[6 * i + c] = zi[c];
            v[0] += (double)ri[c] * zi[c];
            v[1] += (double)ri[c] * ri[c];
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

// Device address of the scratch array on the current device; the first call
// on a device looks it up (cudaGetSymbolAddress) with that device current.
cudaError_t scratch_on_current_device(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_pcg_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[dev] = (unsigned char *)p;
    }
    *out = g_ptr[dev];
    return cudaSuccess;
}

}  // namespace
}  // namespace ba

using namespace ba;

extern "C" ba_status ba_pcg_solve_static(int32_t n, int64_t nnzb, const int32_t *row_ptr, const int32_t *col,
                                         const float *val, const float *b, float *x, double rel_tol,
                                         int32_t max_iters, void *cuda_stream, int32_t *iters_out,
                                         double *rel_resid_out) {
    if (n <= 0 || nnzb < n) return set_error(BA_ERR_INVALID_ARG, "ba_pcg_solve_static: need n > 0 and nnzb >= n");
    if (n > kStaticMaxCams)
        return set_error(BA_ERR_INVALID_ARG, "ba_pcg_solve_static: n exceeds the static scratch limit of 8192 cameras");
    if (!row_ptr || !col || !val || !b || !x) return set_error(BA_ERR_INVALID_ARG, "ba_pcg_solve_static: null pointer");
    if (!(rel_tol > 0) || max_iters < 0) return set_error(BA_ERR_INVALID_ARG, "ba_pcg_solve_static: bad tolerance");
    const int iters_cap = max_iters > 0 ? max_iters : (6 * n > 1000 ? 6 * n : 1000);
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char *base = nullptr;
    cudaError_t e = scratch_on_current_device(&base);
    if (e != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    StaticScalars *sc = (StaticScalars *)(base + kScalOff);
    unsigned *ctr = (unsigned *)(base + kCtrOff);
    double *red = (double *)(base + kRedOff);
    float *vec[5];
    for (int k = 0; k < 5; ++k) vec[k] = (float *)(base + kVecOff + k * kVecBytes);
    float *r = vec[0], *z = vec[1], *d[2] = {vec[2], vec[3]}, *q = vec[4];
    float *Minv = (float *)(base + kMinvOff);

    // counters and the error flag start at zero on every call
    if ((e = cudaMemsetAsync(ctr, 0, 64, st)) != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    if ((e = cudaMemsetAsync(sc, 0, sizeof(StaticScalars), st)) != cudaSuccess)
        return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    k_static_minv<<<(n + 127) / 128, 128, 0, st>>>(n, nnzb, row_ptr, col, val, Minv, sc);
    const int gv = (n + 255) / 256 < 152 * 4 ? (n + 255) / 256 : 152 * 4;
    const int gs = ((int64_t)n * 32 + 255) / 256 < 152 * 8 ? (int)(((int64_t)n * 32 + 255) / 256) : 152 * 8;
    k_static_init<<<gv, 256, 0, st>>>(n, b, x, r, z, d[0], q, Minv, sc, rel_tol * rel_tol, iters_cap, red, ctr + 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
    StaticScalars hs{};
    int it = 0;
    for (;;) {
        for (int c = 0; c < 8; ++c, ++it) {
            float *dold = d[it & 1], *dnew = d[(it + 1) & 1];
            k_static_spmv<<<gs, 256, 0, st>>>(n, row_ptr, col, val, z, dold, dnew, q, sc, red, ctr + 1);
            k_static_update<<<gv, 256, 0, st>>>(n, Minv, dnew, q, x, r, z, sc, red, ctr + 2);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
        if ((e = cudaMemcpyAsync(&hs, sc, sizeof(hs), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
            (e = cudaStreamSynchronize(st)) != cudaSuccess)
            return set_error(BA_ERR_CUDA, cudaGetErrorString(e));
        if (hs.done) break;
        if (it > iters_cap + 16) return set_error(BA_ERR_INTERNAL, "ba_pcg_solve_static: PCG did not stop");
    }
    if (iters_out) *iters_out = hs.iters;
    const double rel = hs.rr0 > 0 ? sqrt(hs.rr / hs.rr0) : 0.0;
    if (rel_resid_out) *rel_resid_out = rel;
    if (hs.err == BA_ERR_INVALID_ARG)
        return set_error(BA_ERR_INVALID_ARG,
                         "ba_pcg_solve_static: malformed BSMC pattern (row starts, diagonal block first, ascending "
                         "upper-triangle columns)");
    if (hs.err == BA_ERR_NOT_SPD) return set_error(BA_ERR_NOT_SPD, "ba_pcg_solve_static: matrix is not positive definite");
    if (!(hs.rr <= hs.tol2 * hs.rr0)) return set_error(BA_ERR_NO_CONVERGENCE, "ba_pcg_solve_static: iteration cap reached");
    return BA_OK;
}
