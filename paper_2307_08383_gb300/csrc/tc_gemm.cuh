// Small dense GEMMs on the 5th-generation tensor cores (tcgen05, sm_100+),
// used by the learned preconditioner's layers.
//
//   C[M x N] (+)= A[M x K] * B[K x N]   (+ bias, ReLU, mask)
//
// One CTA of 128 threads computes a 128-row tile of C for all N <= 128 columns
// and one K chunk of <= 128: it converts its A and B pieces to BF16 into shared
// memory in the canonical K-major layout without swizzle (8-row x 16-byte core
// matrices; core matrices adjacent in K are 128 B apart, adjacent 8-row groups
// (K/8)*128 B apart), one thread issues K/16 tcgen05.mma (kind::f16, BF16 x
// BF16 -> FP32) into a TMEM accumulator of 128 lanes x N columns, commits to an
// mbarrier, and the four warps read their 32 lanes back with tcgen05.ld.
// Operands are read through (row, column) strides, so transposed inputs need
// no copy; a grid.y > 1 splits K and the epilogue then adds with atomics.
#pragma once

#include <cuda_bf16.h>

#include "device_util.cuh"

namespace ba {
namespace tc {

constexpr int kM = 128;     // rows per CTA tile (TMEM lanes)
constexpr int kMaxK = 128;  // K per CTA
constexpr int kMaxN = 128;
constexpr int kSmemBytes = (kM + kMaxN) * kMaxK * 2;  // dynamic shared memory of k_tc_gemm

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor: K-major, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1u << 46;  // descriptor version for tcgen05
    return d;                 // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: D FP32, A and B BF16, both K-major, shape M x N.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int M, int N) {
    return (1u << 4)                         // D format: F32
           | (1u << 7)                       // A format: BF16
           | (1u << 10)                      // B format: BF16
           | ((uint32_t)(N >> 3) << 17)      // N / 8
           | ((uint32_t)(M >> 4) << 24);     // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
}

__device__ __forceinline__ void mbar_init1(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity, long long limit) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(ok)
            : "r"(saddr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
        if (clock64() - t0 > limit) return false;
    }
}

template <typename T> __device__ __forceinline__ float to_f(T x);
template <> __device__ __forceinline__ float to_f<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 x) { return __bfloat162float(x); }

// Operand view: element (r, c) at p[r * rs + c * cs]; rows >= rows_valid and
// columns >= cols_valid read as zero.
template <typename T>
struct View {
    const T *p;
    int64_t rs, cs;
    int rows_valid, cols_valid;
};

// Stage `rows` x K (K multiple of 16) of a K-major operand into the core-matrix
// layout: element (r, k) -> byte ((r/8)*(K/8) + k/8)*128 + (r%8)*16 + (k%8)*2.
// get(r, k) supplies the value.
template <class Get>
__device__ __forceinline__ void stage_kmajor(unsigned char *dst, int rows, int K, Get get) {
    const int kc = K / 8;
    for (int idx = threadIdx.x; idx < rows * kc; idx += blockDim.x) {
        const int r = idx / kc, c8 = idx - r * kc;
        __align__(16) __nv_bfloat16 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = __float2bfloat16_rn(get(r, c8 * 8 + t));
        *reinterpret_cast<uint4 *>(dst + ((r >> 3) * kc + c8) * 128 + (r & 7) * 16) = *reinterpret_cast<uint4 *>(v);
    }
}

enum Epi : int { EPI_STORE = 0, EPI_ATOMIC = 1 };

// C tile = A[m0:m0+128, k0:k0+Kc] * B[k0:k0+Kc, 0:N]; epilogue per row:
//   v = acc + bias[c] (if bias and blockIdx.y == 0), Z[r, c] = v (if Z),
//   v = relu(v) (if relu), v *= (mask[r, c] > 0) (if mask), C[r, c] = v or += v.
// Requirements (checked by the launcher): N in {32, 64, 96, 128}, K chunk a
// multiple of 16 and <= 128, blockDim = 128.
template <typename TA, typename TB>
__global__ void __launch_bounds__(128) k_tc_gemm(View<TA> A, View<TB> B, int M, int N, int K, int kchunk,
                                                 const float *__restrict__ bias, float *__restrict__ Z, int64_t z_rs,
                                                 const float *__restrict__ mask, int64_t mask_rs, int relu, float *C,
                                                 int64_t c_rs, int64_t c_cs, int epi, int *err, long long limit) {
    extern __shared__ __align__(128) unsigned char tc_smem[];
    unsigned char *sA = tc_smem;                    // kM x kMaxK BF16
    unsigned char *sB = tc_smem + kM * kMaxK * 2;   // kMaxN x kMaxK BF16
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    __shared__ int s_ok;
    const int m0 = blockIdx.x * kM;
    const int k0 = blockIdx.y * kchunk;
    const int kc = min(kchunk, K - k0);          // valid K of this chunk
    const int kpad = (kc + 15) & ~15;            // MMA K multiple of 16
    const uint32_t ncols = N <= 32 ? 32u : (N <= 64 ? 64u : 128u);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (warp == 0) tmem_alloc(&s_taddr, ncols);
    if (threadIdx.x == 0) {
        mbar_init1(&mbar);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // operands: A rows m0.., B^T rows 0..N-1 (K-major)
    stage_kmajor(sA, kM, kpad, [&](int r, int k) -> float {
        const int gr = m0 + r, gk = k0 + k;
        return (gr < A.rows_valid && k < kc && gk < A.cols_valid) ? to_f<TA>(A.p[gr * A.rs + gk * A.cs]) : 0.f;
    });
    stage_kmajor(sB, N, kpad, [&](int n, int k) -> float {
        const int gk = k0 + k;
        return (k < kc && gk < B.rows_valid && n < B.cols_valid) ? to_f<TB>(B.p[gk * B.rs + n * B.cs]) : 0.f;
    });
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // smem writes -> tensor core reads
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t taddr = s_taddr;
    if (threadIdx.x == 0) {
        const uint32_t idesc = instr_desc_bf16(kM, N);
        const uint32_t a0 = saddr(sA), b0 = saddr(sB);
        const uint32_t sbo = (uint32_t)(kpad / 8) * 128u;
        for (int s = 0; s < kpad / 16; ++s) {
            const uint64_t ad = smem_desc(a0 + s * 256u, 128u, sbo);
            const uint64_t bd = smem_desc(b0 + s * 256u, 128u, sbo);
            mma_bf16(taddr, ad, bd, idesc, s > 0 ? 1 : 0);
        }
        mma_commit(&mbar);
        s_ok = mbar_wait_parity(&mbar, 0, limit) ? 1 : 0;
    }
    __syncthreads();
    fence_after_sync();
    const bool ok = s_ok != 0;
    if (ok) {
        const int r = m0 + warp * 32 + lane;  // this thread's row
        const uint32_t lane_addr = taddr + ((uint32_t)(warp * 32) << 16);
        for (int c0 = 0; c0 < N; c0 += 16) {
            float v[16];
            tmem_ld16(lane_addr + (uint32_t)c0, v);
            if (r < M) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int c = c0 + t;
                    if (c >= N) break;
                    float x = v[t];
                    if (bias && blockIdx.y == 0) x += bias[c];
                    if (Z) Z[(int64_t)r * z_rs + c] = x;
                    if (relu) x = fmaxf(x, 0.f);
                    if (mask) x = mask[(int64_t)r * mask_rs + c] > 0.f ? x : 0.f;
                    float *dst = C + (int64_t)r * c_rs + (int64_t)c * c_cs;
                    if (epi == EPI_ATOMIC) atomicAdd(dst, x);
                    else *dst = x;
                }
            }
        }
    } else if (threadIdx.x == 0) {
        // the MMA may still be writing TMEM: wait once more (bounded) before freeing it
        atomicExch(err, (int)BA_ERR_TIMEOUT);
        mbar_wait_parity(&mbar, 0, limit);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        tmem_dealloc(taddr, ncols);
    }
}

}  // namespace tc
}  // namespace ba
