// Device helpers shared by the libba kernels.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "ba_internal.h"

namespace ba {

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Sum NV doubles over the CTA; the result is valid in every lane of warp 0.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[w * NV + i] = v[i];
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) v[i] = warp_sum(lane < nw ? sh[lane * NV + i] : 0.0);
    }
    __syncthreads();
}

// Deterministic grid-wide sum: every CTA stores its partial, the last CTA to
// arrive (a counter, no waiting) adds the partials in CTA order and thread 0
// runs fin(totals).  Must be the last thing a kernel does; every thread of
// every CTA must call it.
template <int NV, class Fin>
__device__ __forceinline__ void grid_sum(double (&v)[NV], double *part, unsigned *counter, Fin fin) {
    __shared__ double sh[32 * NV];
    __shared__ bool last;
    block_sum<NV>(v, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) part[blockIdx.x * NV + i] = v[i];
        __threadfence();
        const unsigned t = atomicAdd(counter, 1u);
        last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) acc[i] = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
        for (int i = 0; i < NV; ++i) acc[i] += __ldcg(part + b * NV + i);
    block_sum<NV>(acc, sh);
    if (threadIdx.x == 0) {
        fin(acc);
        *counter = 0;
        __threadfence();
    }
}

template <typename T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }
template <typename T> __device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }

__device__ __forceinline__ double clampd(double x) { return x < 1e-6 ? 1e-6 : (x > 1e32 ? 1e32 : x); }
template <typename T> __device__ __forceinline__ T clampT(T x) { return x < T(1e-6) ? T(1e-6) : (x > T(1e32) ? T(1e32) : x); }

// Per-thread running sum in the mode precision.  FP32: compensated
// (Knuth TwoSum, error-free per step), so a thread's partial keeps about
// twice FP32 precision without touching GB300's slow FP64 pipe; the
// partials are then added across threads in FP64.  FP64: plain.
template <typename T> struct RunSum;
template <> struct RunSum<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float t = s + x, z = t - s;
        c += (s - (t - z)) + (x - z);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};
template <> struct RunSum<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};

// In-place Cholesky of a symmetric 6x6 (row-major, lower triangle used) and
// the inverse A^-1 = L^-T L^-1 written full.  Returns false if not SPD.
template <typename T>
__device__ bool spd_inverse6(const T *A, T *Ainv) {
    T L[21];  // packed lower: L[i*(i+1)/2 + j]
#pragma unroll
    for (int i = 0; i < 6; ++i) {
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            T s = A[i * 6 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) s -= L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
            if (i == j) {
                if (!(s > T(0))) return false;
                L[i * (i + 1) / 2 + i] = sqrt(s);
            } else {
                L[i * (i + 1) / 2 + j] = s / L[j * (j + 1) / 2 + j];
            }
        }
    }
    // Li = L^-1 (lower)
    T Li[21];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        Li[i * (i + 1) / 2 + i] = T(1) / L[i * (i + 1) / 2 + i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = j; k < i; ++k) s += L[i * (i + 1) / 2 + k] * Li[k * (k + 1) / 2 + j];
            Li[i * (i + 1) / 2 + j] = -s * Li[i * (i + 1) / 2 + i];
        }
    }
    // A^-1 = Li^T Li
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int j = i; j < 6; ++j) {
            T s = T(0);
#pragma unroll
            for (int k = j; k < 6; ++k) s += Li[k * (k + 1) / 2 + i] * Li[k * (k + 1) / 2 + j];
            Ainv[i * 6 + j] = s;
            Ainv[j * 6 + i] = s;
        }
    return true;
}

// Quaternion (w, x, y, z) of the rotation vector v.
__device__ __forceinline__ void quat_exp(const double *v, double *q) {
    const double th2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    const double th = sqrt(th2);
    double s, c;
    if (th < 1e-8) {
        s = 0.5 - th2 / 48.0;
        c = 1.0 - th2 / 8.0;
    } else {
        s = sin(0.5 * th) / th;
        c = cos(0.5 * th);
    }
    q[0] = c;
    q[1] = s * v[0];
    q[2] = s * v[1];
    q[3] = s * v[2];
}

// Rotation vector of a unit quaternion (shortest rotation).
__device__ __forceinline__ void quat_log(const double *qin, double *v) {
    double q[4] = {qin[0], qin[1], qin[2], qin[3]};
    if (q[0] < 0) { q[0] = -q[0]; q[1] = -q[1]; q[2] = -q[2]; q[3] = -q[3]; }
    const double s = sqrt(q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double f;
    if (s < 1e-8) {
        f = 2.0 / q[0] * (1.0 - s * s / (3.0 * q[0] * q[0]));
    } else {
        f = 2.0 * atan2(s, q[0]) / s;
    }
    v[0] = f * q[1];
    v[1] = f * q[2];
    v[2] = f * q[3];
}

__device__ __forceinline__ void quat_mul(const double *a, const double *b, double *o) {
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// Row-major rotation matrix of a unit quaternion.
__device__ __forceinline__ void quat_to_R(const double *q, double *R) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

template <typename T> __device__ __forceinline__ void red_add(T *p, T v) { atomicAdd(p, v); }

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).
// bar[0] counts arrivals, bar[1] is the generation.  The wait is bounded by
// about `limit_cycles` SM clocks; on timeout it sets *err = BA_ERR_TIMEOUT and
// returns false, and the caller must leave the kernel.
__device__ __forceinline__ bool grid_barrier(unsigned *bar, int *err, long long limit_cycles) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *vgen = bar + 1;
        const unsigned g0 = *vgen;
        __threadfence();
        const unsigned arrived = atomicAdd(bar, 1u);
        int ok = 1;
        if (arrived == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*vgen == g0) {
                if (clock64() - t0 > limit_cycles || *(volatile int *)err == (int)BA_ERR_TIMEOUT) {
                    atomicExch(err, (int)BA_ERR_TIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Grid-wide all-reduce fused with a barrier (cooperative launch).  On entry
// v holds this CTA's partial in thread 0; every CTA stores it, the last CTA
// to arrive adds the partials in CTA order, publishes the totals in bcast and
// releases the others; on return every thread holds the totals.  Waits are
// bounded as in grid_barrier; returns false on timeout.
__device__ __forceinline__ unsigned atom_add_release(unsigned *p, unsigned v) {
    unsigned old;
    asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

template <int NV>
__device__ __forceinline__ bool grid_allreduce(double (&v)[NV], double *part, double *bcast, unsigned *bar, int *err,
                                               long long limit_cycles) {
    __shared__ int s_last, s_ok;
    __shared__ double s_tot[NV];
    __shared__ double s_red[32 * NV];
    unsigned g0 = 0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) part[blockIdx.x * NV + k] = v[k];
        g0 = ld_acquire(bar + 1);
        // release: the partial above is visible to whoever sees this arrival
        const unsigned arrived = atom_add_release(bar, 1u);
        s_last = (arrived == gridDim.x - 1);
        s_ok = 1;
    }
    __syncthreads();
    if (s_last) {
        if (threadIdx.x == 0) ld_acquire(bar);  // acquire: every CTA's partial is visible
        __syncthreads();
        double acc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = 0.0;
        for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __ldcg(part + b * NV + k);
        block_sum<NV>(acc, s_red);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                __stcg(bcast + k, acc[k]);
                s_tot[k] = acc[k];
            }
            atomicExch(bar, 0u);
            atom_add_release(bar + 1, 1u);  // release: totals and the reset counter
        }
    } else if (threadIdx.x == 0) {
        const long long t0 = clock64();
        while (ld_acquire(bar + 1) == g0) {
            if (clock64() - t0 > limit_cycles || *(volatile int *)err == (int)BA_ERR_TIMEOUT) {
                atomicExch(err, (int)BA_ERR_TIMEOUT);
                s_ok = 0;
                break;
            }
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) s_tot[k] = __ldcg(bcast + k);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = s_tot[k];
    const bool ok = s_ok != 0;
    __syncthreads();
    return ok;
}

__device__ __forceinline__ void red_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Symmetric deterministic grid all-reduce for persistent cooperative kernels.
// `bar` is an arrival counter that starts at 0 for the launch and only grows;
// `gen` numbers this kernel's calls 0, 1, 2, ...  Each CTA stores its NV
// partials (v, valid in warp 0 as block_sum leaves them) in half (gen & 1)
// of `part` (2 * gridDim.x * AR_NV_MAX doubles), announces itself with a release
// add and waits (bounded) until (gen + 1) * gridDim.x arrivals.  Then every
// thread loads the partials of CTAs threadIdx.x, threadIdx.x + blockDim.x, ...
// (its loads issued together: one L2 round trip) and a block sum joins them,
// an order fixed by the launch shape, so every CTA obtains the same bits
// without a broadcast round trip.  A half is written again only two calls
// later, by a CTA that has passed call gen + 1, which every CTA enters after
// reading the partials of call gen.  On return every thread holds the totals;
// false on timeout.  The shared totals are rewritten by the next call only
// after its first barrier, which every thread reaches after reading them.
constexpr int AR_NV_MAX = 4;
template <int NV>
__device__ __forceinline__ bool grid_allreduce_sym(double (&v)[NV], double *part, unsigned gen, unsigned *bar,
                                                   int *err, long long limit_cycles) {
    static_assert(NV <= AR_NV_MAX, "too many values");
    __shared__ double s_tot[NV];
    __shared__ double s_red[NV * 32];
    __shared__ int s_ok;
    double *half = part + (size_t)(gen & 1u) * gridDim.x * AR_NV_MAX;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) __stcg(half + blockIdx.x * AR_NV_MAX + k, v[k]);
        red_add_release(bar, 1u);
        const unsigned target = (gen + 1u) * gridDim.x;
        const long long t0 = clock64();
        int ok = 1;
        while (ld_acquire(bar) < target) {
            if (clock64() - t0 > limit_cycles || *(volatile int *)err == (int)BA_ERR_TIMEOUT) {
                atomicExch(err, (int)BA_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();  // thread 0's acquire orders every thread's partial reads
    const bool ok = s_ok != 0;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0.0;
    if (ok) {
        const unsigned b0 = threadIdx.x, b1 = threadIdx.x + blockDim.x;
        double t0[NV], t1[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            t0[k] = b0 < gridDim.x ? __ldcg(half + b0 * AR_NV_MAX + k) : 0.0;
            t1[k] = b1 < gridDim.x ? __ldcg(half + b1 * AR_NV_MAX + k) : 0.0;
        }
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] = t0[k] + t1[k];
        for (unsigned b = threadIdx.x + 2 * blockDim.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
            for (int k = 0; k < NV; ++k) acc[k] += __ldcg(half + b * AR_NV_MAX + k);
    }
    block_sum<NV>(acc, s_red);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) s_tot[k] = acc[k];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = s_tot[k];
    return ok;
}

// ---- 6x6 block SpMV helpers (BSMC and the full-block formats) ----

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

// One stored linearization row (JW values, 16-byte aligned, read-only) into
// registers with vector loads.
__device__ __forceinline__ void load_jrow(const float *__restrict__ s, float (&v)[JW]) {
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 4; ++q) {
        const float4 t = __ldg(s4 + q);
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}
__device__ __forceinline__ void load_jrow(const double *__restrict__ s, double (&v)[JW]) {
    const double2 *s2 = reinterpret_cast<const double2 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 2; ++q) {
        const double2 t = __ldg(s2 + q);
        v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
}

// Double-float (hi + lo, both FP32) values for reductions on the FP32 pipe:
// the sum of two is formed with an error-free TwoSum, so it is exact to about
// 2^-44 relative and, TwoSum being symmetric, a xor-butterfly gives every lane
// the same bits.
struct df32 {
    float hi, lo;
};
__device__ __forceinline__ df32 df_add(df32 a, df32 b) {
    const float s = a.hi + b.hi, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e += a.lo + b.lo;
    const float hi = s + e;
    return {hi, e - (hi - s)};
}
// Products and quotients of double-floats (Dekker's two-product by FMA, one
// Newton correction of the FP32 quotient): about 2^-44 relative, within the
// FP32 exponent range.
__device__ __forceinline__ df32 df_fast_norm(float s, float e) {
    const float hi = s + e;
    return {hi, e - (hi - s)};
}
__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df32{-b.hi, -b.lo}); }
__device__ __forceinline__ df32 df_mul(df32 a, df32 b) {
    const float p = a.hi * b.hi;
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_fast_norm(p, e);
}
__device__ __forceinline__ df32 df_mulf(df32 a, float b) {
    const float p = a.hi * b;
    const float e = __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p));
    return df_fast_norm(p, e);
}
__device__ __forceinline__ df32 df_div(df32 a, df32 b) {
    const float q1 = a.hi / b.hi;
    float r = __fmaf_rn(-q1, b.hi, a.hi);  // exact: a.hi - q1 b.hi
    r = __fmaf_rn(-q1, b.lo, r + a.lo);
    return df_fast_norm(q1, r / b.hi);
}
__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df32 warp_sum_df(df32 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const df32 u = {__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = df_add(v, u);
    }
    return v;
}

// Block sum of NV double-floats; the totals are valid in every lane of warp 0.
template <int NV>
__device__ __forceinline__ void block_sum_df(df32 (&v)[NV], float2 *sh) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = warp_sum_df(v[i]);
    if (lane == 0)
#pragma unroll
        for (int i = 0; i < NV; ++i) sh[w * NV + i] = make_float2(v[i].hi, v[i].lo);
    __syncthreads();
    if (w == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
            const float2 t = lane < nw ? sh[lane * NV + i] : make_float2(0.f, 0.f);
            v[i] = warp_sum_df(df32{t.x, t.y});
        }
    }
    __syncthreads();
}

// grid_allreduce_sym for double-floats (partials stored as float2 in the same
// slots): every CTA adds all partials itself in CTA order.  Arrivals are
// spread over AR_SUB counters, one per 128-byte line (CTA c announces itself
// on counter c % AR_SUB), so the release adds of a large grid do not queue on
// one address; lanes 0..AR_SUB-1 of warp 0 each poll one counter.  Once all
// have arrived, every thread of the CTA loads the partials of CTAs
// threadIdx.x, threadIdx.x + blockDim.x, ... (all loads of a thread issued
// before its adds, so the grid's partials cost one L2 round trip instead of
// gridDim.x / 32 dependent ones), and a block sum joins them: a fixed order
// for a given launch shape, so every CTA gets the same bits.  `bar` holds
// AR_SUB * 32 words, zero at launch; `sh` holds NV * warps float2, `s_ok` is
// shared.  Every thread of the CTA calls this (it holds __syncthreads); the
// CTA's own partial is v as left by block_sum_df (valid in warp 0).  Once
// every CTA has arrived, every thread runs after_wait() (what the grid wrote
// before arriving is visible to it) right after issuing its partial reads;
// meant for asynchronous copies that overlap the rest.  On return the
// totals are valid in thread 0 only (as double-floats); false on timeout.
constexpr int AR_SUB = 16;
template <int NV, class F>
__device__ __forceinline__ bool grid_allreduce_df(df32 (&v)[NV], double *part, unsigned gen, unsigned *bar,
                                                  int *err, long long limit_cycles, df32 (&tot)[NV], float2 *sh,
                                                  int *s_ok, F &&after_wait) {
    static_assert(NV <= AR_NV_MAX, "too many values");
    float2 *half = reinterpret_cast<float2 *>(part + (size_t)(gen & 1u) * gridDim.x * AR_NV_MAX);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) __stcg(half + blockIdx.x * AR_NV_MAX + k, make_float2(v[k].hi, v[k].lo));
        red_add_release(bar + 32 * (blockIdx.x % AR_SUB), 1u);
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int lane_ok = 1;
        if (lane < AR_SUB) {
            // CTAs that announce themselves on this lane's counter
            const unsigned per = gridDim.x / AR_SUB + ((unsigned)lane < gridDim.x % AR_SUB ? 1u : 0u);
            const unsigned target = (gen + 1u) * per;
            const long long t0 = clock64();
            while (ld_acquire(bar + 32 * lane) < target) {
                if (clock64() - t0 > limit_cycles || *(volatile int *)err == (int)BA_ERR_TIMEOUT) {
                    lane_ok = 0;
                    break;
                }
            }
        }
        const bool ok = __all_sync(0xffffffffu, lane_ok) != 0;
        if (lane == 0) {
            *s_ok = ok ? 1 : 0;
            if (!ok) atomicExch(err, (int)BA_ERR_TIMEOUT);
        }
    }
    __syncthreads();  // the pollers' acquires order every thread's partial reads
    const bool ok = *s_ok != 0;
    df32 acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = df32{0.f, 0.f};
    if (ok) {
        const unsigned b0 = threadIdx.x, b1 = threadIdx.x + blockDim.x;
        float2 t0[NV], t1[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            t0[k] = b0 < gridDim.x ? __ldcg(half + b0 * AR_NV_MAX + k) : make_float2(0.f, 0.f);
            t1[k] = b1 < gridDim.x ? __ldcg(half + b1 * AR_NV_MAX + k) : make_float2(0.f, 0.f);
        }
        after_wait();  // issued behind the partial reads, overlapping their use
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            acc[k] = df_add(df32{t0[k].x, t0[k].y}, df32{t1[k].x, t1[k].y});
        }
        for (unsigned b = threadIdx.x + 2 * blockDim.x; b < gridDim.x; b += blockDim.x)
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const float2 u = __ldcg(half + b * AR_NV_MAX + k);
                acc[k] = df_add(acc[k], df32{u.x, u.y});
            }
    }
    block_sum_df<NV>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) tot[k] = acc[k];
    return ok;
}

}  // namespace ba
