// Formation of the reduced camera system (Eq. 4) point group by point group
// (Sec. 5, Sec. 6.1), its aggregation into BSMC (Sec. 4) and the block-Jacobi
// preconditioner (Sec. 3.2).
//
// Per point k with observations a (camera i_a) the damped V_k = sum J_p^T J_p
// + lambda clamp(diag) is factored V_k = L L^T.  With P_a = J_p,a L^-T (2x3),
// q_k = L^-1 l_p,k and e^_a = e_a + P_a q_k the point's sub-RCS is
//   S_(i_a, i_b) -= J_c,a^T (P_a P_b^T) J_c,b          (a != b, i_a < i_b)
//   S_(i_a, i_a) += J_c,a^T (I - P_a P_a^T) J_c,a      (U and -W V^-1 W^T)
//   b_(i_a)      -= J_c,a^T e^_a                         (l_c - W V^-1 l_p)
// which is W V^-1 W^T = (J_c^T P)(J_c^T P)^T written through the 2x2 middle
// factors.  Persistent CTAs walk the point groups (whole tracks, Sec. 6.1);
// for each group a CTA copies the group's Jacobian rows and (a, b) product
// list into shared memory with TMA bulk copies - double-buffered, the next
// group's copy in flight while the current one is computed - turns J_p and e
// into P and e^ in place, then sums the products of each sub-RCS block in
// registers (work items of <= 8 products, joined by a warp-segmented shuffle
// reduction) - no atomics - and writes them as partials.  The per-point work
// of the next group runs on the threads that finish their products first,
// so one barrier per group remains.  A segmented sum over the partials of each global block
// (precomputed CSR) then forms S, adds lambda clamp(diag U) on the diagonal,
// and inverts the diagonal blocks for the preconditioner.
#include <algorithm>
#include <cstring>
#include <type_traits>

#include "device_util.cuh"
#include "tma_util.cuh"

namespace ba {

__host__ __device__ constexpr int up_idx(int r, int c) { return 6 * r - r * (r - 1) / 2 + (c - r); }

// One staged observation row (JW values, 16-byte aligned) into registers.
__device__ __forceinline__ void load_slot(const float *s, float (&v)[JW]) {
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 4; ++q) {
        const float4 t = s4[q];
        v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
    }
}
__device__ __forceinline__ void load_slot(const double *s, double (&v)[JW]) {
    const double2 *s2 = reinterpret_cast<const double2 *>(s);
#pragma unroll
    for (int q = 0; q < JW / 2; ++q) {
        const double2 t = s2[q];
        v[2 * q] = t.x; v[2 * q + 1] = t.y;
    }
}

__device__ __forceinline__ unsigned long long global_ns_rcs() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Per point of group g (points pl0, pl0 + blockDim.x, ...): V_k, its Cholesky
// factor, q_k; J_p -> P and e -> e^ in place in the staged rows `so`.
template <typename T>
__device__ __forceinline__ void rcs_points(const GroupDesc &g, T *so, int pl0, const int *__restrict__ trk_ptr,
                                           double lambda, T *__restrict__ Linv_out, T *__restrict__ lp_out,
                                           DevScalars *sc, int fp64_v) {
    for (int pl = pl0; pl < g.npts; pl += blockDim.x) {
        const int k = g.pt_begin + pl;
        const int a0 = trk_ptr[k] - g.obs_begin, a1 = trk_ptr[k + 1] - g.obs_begin;
        T v00 = 0, v01 = 0, v02 = 0, v11 = 0, v12 = 0, v22 = 0, l0 = 0, l1 = 0, l2 = 0;
        for (int a = a0; a < a1; ++a) {
            const T *s = so + a * JW;
            const T p0 = s[12], p1 = s[13], p2 = s[14], r0 = s[15], r1 = s[16], r2 = s[17], e0 = s[18], e1 = s[19];
            // one FMA per term (a sum of two products added in one
            // statement costs a multiply, an FMA and an add)
            v00 += p0 * p0; v00 += r0 * r0; v01 += p0 * p1; v01 += r0 * r1;
            v02 += p0 * p2; v02 += r0 * r2; v11 += p1 * p1; v11 += r1 * r1;
            v12 += p1 * p2; v12 += r1 * r2; v22 += p2 * p2; v22 += r2 * r2;
            l0 -= p0 * e0; l0 -= r0 * e1; l1 -= p1 * e0; l1 -= r1 * e1;
            l2 -= p2 * e0; l2 -= r2 * e1;
        }
        const T lam = (T)lambda;
        v00 += lam * clampT(v00);
        v11 += lam * clampT(v11);
        v22 += lam * clampT(v22);
        // Cholesky V = L L^T, then M = L^-1 (lower)
        T m00, m10, m11, m20, m21, m22;
        bool ok;
        {
            const T c00 = v00;
            const T d0 = sqrt(c00);
            const T c10 = v01 / d0, c20 = v02 / d0;
            const T s11 = v11 - c10 * c10;
            const T d1 = sqrt(s11);
            const T c21 = (v12 - c20 * c10) / d1;
            const T s22 = v22 - c20 * c20 - c21 * c21;
            const T d2 = sqrt(s22);
            ok = (c00 > T(0)) && (s11 > T(0)) && (s22 > T(0));
            m00 = T(1) / d0; m11 = T(1) / d1; m22 = T(1) / d2;
            m10 = -c10 * m00 * m11;
            m21 = -c21 * m11 * m22;
            m20 = -(c20 * m00 + c21 * m10) * m22;
        }
        if (fp64_v && ok) {
            // FP32 mode: refactor in FP64 when kappa~ = ||V||_F ||V^-1||_F > 1e4
            const T i00 = m00 * m00 + m10 * m10 + m20 * m20, i11 = m11 * m11 + m21 * m21, i22 = m22 * m22;
            const T i01 = m10 * m11 + m20 * m21, i02 = m20 * m22, i12 = m21 * m22;
            const T nv = v00 * v00 + v11 * v11 + v22 * v22 + 2 * (v01 * v01 + v02 * v02 + v12 * v12);
            const T ni = i00 * i00 + i11 * i11 + i22 * i22 + 2 * (i01 * i01 + i02 * i02 + i12 * i12);
            if (nv * ni > T(1e8)) {
                double w00 = 0, w01 = 0, w02 = 0, w11 = 0, w12 = 0, w22 = 0;
                for (int a = a0; a < a1; ++a) {
                    const T *s = so + a * JW;
                    const double p0 = s[12], p1 = s[13], p2 = s[14], r0 = s[15], r1 = s[16], r2 = s[17];
                    w00 += p0 * p0 + r0 * r0; w01 += p0 * p1 + r0 * r1; w02 += p0 * p2 + r0 * r2;
                    w11 += p1 * p1 + r1 * r1; w12 += p1 * p2 + r1 * r2; w22 += p2 * p2 + r2 * r2;
                }
                w00 += lambda * clampd(w00); w11 += lambda * clampd(w11); w22 += lambda * clampd(w22);
                const double d0 = sqrt(w00), c10 = w01 / d0, c20 = w02 / d0;
                const double s11 = w11 - c10 * c10, d1 = sqrt(s11), c21 = (w12 - c20 * c10) / d1;
                const double s22 = w22 - c20 * c20 - c21 * c21, d2 = sqrt(s22);
                if (w00 > 0 && s11 > 0 && s22 > 0) {
                    const double n00 = 1 / d0, n11 = 1 / d1, n22 = 1 / d2, n10 = -c10 * n00 * n11;
                    const double n21 = -c21 * n11 * n22, n20 = -(c20 * n00 + c21 * n10) * n22;
                    m00 = (T)n00; m10 = (T)n10; m11 = (T)n11; m20 = (T)n20; m21 = (T)n21; m22 = (T)n22;
                    atomicAdd(&sc->n_v64, 1ull);
                } else {
                    ok = false;
                }
            }
        }
        if (!ok) {
            atomicExch(&sc->err, (int)BA_ERR_NOT_SPD);
            m00 = m10 = m11 = m20 = m21 = m22 = T(0);
        }
        const T q0 = m00 * l0, q1 = m10 * l0 + m11 * l1, q2 = m20 * l0 + m21 * l1 + m22 * l2;
        T *lo = Linv_out + 6 * (int64_t)k;
        lo[0] = m00; lo[1] = m10; lo[2] = m11; lo[3] = m20; lo[4] = m21; lo[5] = m22;
        T *lpo = lp_out + 3 * (int64_t)k;
        lpo[0] = l0; lpo[1] = l1; lpo[2] = l2;
        for (int a = a0; a < a1; ++a) {
            T *s = so + a * JW;
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const T j0 = s[12 + 3 * r], j1 = s[13 + 3 * r], j2 = s[14 + 3 * r];
                const T P0 = j0 * m00, P1 = j0 * m10 + j1 * m11, P2 = j0 * m20 + j1 * m21 + j2 * m22;
                s[12 + 3 * r] = P0; s[13 + 3 * r] = P1; s[14 + 3 * r] = P2;
                s[18 + r] += P0 * q0 + P1 * q1 + P2 * q2;
            }
        }
    }
}

// The products of group g: its work items, from the staged rows `so` and
// product list `sc_list`, into the group's partials.
template <typename T>
__device__ __forceinline__ void rcs_products(const GroupDesc &g, const T *so, const uint32_t *sc_list,
                                             const ItemDesc *__restrict__ items, T *__restrict__ part) {
    // 3) work items: each lane sums <= ITEM_MAX products of one sub-RCS block in
    //    registers; the items of a block that share a warp are added by a
    //    segmented shuffle reduction and the run's head writes the partial.
    const ItemDesc *itg = items + g.item_begin;
    for (int base = 0; base < g.nitems; base += blockDim.x) {
        const int it = base + threadIdx.x;
        const ItemDesc d = it < g.nitems ? itg[it] : ItemDesc{0u, 0u};
        const int cb = (int)(d.x & 0xffffu), cnt = (int)((d.x >> 16) & 0xfu);
        const bool diag = (d.x >> 20) & 1u;
        const int nfollow = (int)((d.x >> 21) & 31u);
        const bool head = (d.x >> 26) & 1u;
        T acc[36];
#pragma unroll
        for (int q = 0; q < 36; ++q) acc[q] = T(0);
        if (!diag) {
            for (int c = cb; c < cb + cnt; ++c) {
                const uint32_t u = sc_list[c];
                T sa[JW], sb[JW];
                load_slot(so + (u & 0xffffu) * JW, sa);
                load_slot(so + (u >> 16) * JW, sb);
                // -P_a P_b^T (the minus sign rides on the 2x2 factor, so
                // every accumulation below is two FMAs)
                const T M00 = -sa[12] * sb[12] - sa[13] * sb[13] - sa[14] * sb[14];
                const T M01 = -sa[12] * sb[15] - sa[13] * sb[16] - sa[14] * sb[17];
                const T M10 = -sa[15] * sb[12] - sa[16] * sb[13] - sa[17] * sb[14];
                const T M11 = -sa[15] * sb[15] - sa[16] * sb[16] - sa[17] * sb[17];
                T t0[6], t1[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    t0[j] = M00 * sb[j] + M01 * sb[6 + j];
                    t1[j] = M10 * sb[j] + M11 * sb[6 + j];
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const T ai0 = sa[i], ai1 = sa[6 + i];
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        acc[6 * i + j] += ai0 * t0[j];
                        acc[6 * i + j] += ai1 * t1[j];
                    }
                }
            }
        } else {
            // packed [21 upper entries of U - W V^-1 W^T | 6 diag(J_c^T J_c) | 6 b | 3 zero]
            for (int c = cb; c < cb + cnt; ++c) {
                T sa[JW];
                load_slot(so + (sc_list[c] & 0xffffu) * JW, sa);
                const T g00 = T(1) - (sa[12] * sa[12] + sa[13] * sa[13] + sa[14] * sa[14]);
                const T g01 = -(sa[12] * sa[15] + sa[13] * sa[16] + sa[14] * sa[17]);
                const T g11 = T(1) - (sa[15] * sa[15] + sa[16] * sa[16] + sa[17] * sa[17]);
                T t0[6], t1[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    t0[j] = g00 * sa[j] + g01 * sa[6 + j];
                    t1[j] = g01 * sa[j] + g11 * sa[6 + j];
                }
#pragma unroll
                for (int i = 0; i < 6; ++i) {
                    const T ai0 = sa[i], ai1 = sa[6 + i];
#pragma unroll
                    for (int j = i; j < 6; ++j) {
                        acc[up_idx(i, j)] += ai0 * t0[j];
                        acc[up_idx(i, j)] += ai1 * t1[j];
                    }
                    acc[21 + i] += ai0 * ai0;
                    acc[21 + i] += ai1 * ai1;
                    acc[27 + i] -= ai0 * sa[18];
                    acc[27 + i] -= ai1 * sa[19];
                }
            }
        }
        const unsigned maxnf = __reduce_max_sync(0xffffffffu, (unsigned)nfollow);
        if (maxnf > 0) {
            for (unsigned off = 1; off <= maxnf; off <<= 1) {
#pragma unroll
                for (int q = 0; q < 36; ++q) {
                    const T v = __shfl_down_sync(0xffffffffu, acc[q], off);
                    if (off <= (unsigned)nfollow) acc[q] += v;
                }
            }
        }
        if (head) {
            T *out = part + (g.part_begin + d.y) * BW;
            if constexpr (sizeof(T) == 4) {
                float4 *o4 = reinterpret_cast<float4 *>(out);
#pragma unroll
                for (int q = 0; q < 9; ++q) o4[q] = make_float4(acc[4 * q], acc[4 * q + 1], acc[4 * q + 2], acc[4 * q + 3]);
            } else {
                double2 *o2 = reinterpret_cast<double2 *>(out);
#pragma unroll
                for (int q = 0; q < 18; ++q) o2[q] = make_double2(acc[2 * q], acc[2 * q + 1]);
            }
        }
    }
}

__host__ __device__ constexpr size_t form_round128(size_t b) { return (b + 127) & ~(size_t)127; }

template <typename T>
__global__ void __launch_bounds__(FORM_THREADS) k_form_rcs(const GroupDesc *__restrict__ grp, int ngroups,
                                                           const ItemDesc *__restrict__ items,
                                                           const uint32_t *__restrict__ contrib,
                                                           const int *__restrict__ trk_ptr, const T *__restrict__ J,
                                                           double lambda, T *__restrict__ part, T *__restrict__ Linv_out,
                                                           T *__restrict__ lp_out, DevScalars *sc, int fp64_v,
                                                           int o_cap, int c_cap, long long limit, int prof) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ GroupDesc sdesc[2];
    // a staging buffer: rows of up to o_cap observations, then c_cap products
    // (the largest group's), each part starting on a 128-byte boundary
    const size_t jbytes_max = form_round128((size_t)o_cap * JW * sizeof(T));
    const size_t buf_bytes = form_round128(jbytes_max + (size_t)c_cap * sizeof(uint32_t));
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_proxy_async();
    }
    __syncthreads();
    // thread 0: copy group gi's rows and product list into buffer b
    auto issue = [&](int gi, int b) {
        const GroupDesc d = grp[gi];
        sdesc[b] = d;
        unsigned char *dst = smem_raw + b * buf_bytes;
        const uint32_t jb = (uint32_t)d.nobs * JW * (uint32_t)sizeof(T);
        const uint32_t cb = (uint32_t)((d.nc + 3) & ~3) * 4u;
        fence_proxy_async();  // earlier generic writes to this buffer before the async copy
        mbar_expect_tx(&mbar[b], jb + cb);
        bulk_g2s(dst, J + (int64_t)d.obs_begin * JW, jb, &mbar[b]);
        if (cb) bulk_g2s(dst + jbytes_max, contrib + d.c_begin, cb, &mbar[b]);
    };
    auto rows = [&](int b) { return reinterpret_cast<T *>(smem_raw + b * buf_bytes); };
    auto plist = [&](int b) { return reinterpret_cast<const uint32_t *>(smem_raw + b * buf_bytes + jbytes_max); };
    // per buffer: the mbarrier phase to wait for (every thread), a copy in
    // flight (thread 0, for the drain after a timeout)
    uint32_t parity = 0u, pending = 0u;
    auto wait_buf = [&](int b) {
        if (!mbar_wait(&mbar[b], (parity >> b) & 1u, limit)) return false;
        parity ^= 1u << b;
        pending &= ~(1u << b);
        return true;
    };
    // The per-point work of a group runs on the highest threads: warp w takes
    // product chunks w, w + 8, ..., so the last warps have the fewest.
    const int pl0 = (int)blockDim.x - 1 - (int)threadIdx.x;
    // phase timing (the last thread, prof): barrier wait, products, the next
    // group's copy wait and per-point work
    const bool tm = prof && threadIdx.x == blockDim.x - 1;
    unsigned long long ta = 0, tb = 0, tc = 0, t_bar = 0, t_prod = 0, t_pts = 0, ngr = 0;
    int gi = blockIdx.x;
    if (gi >= ngroups) return;
    if (threadIdx.x == 0) {
        issue(gi, 0);
        pending = 1u;
        if (gi + (int)gridDim.x < ngroups) {
            issue(gi + gridDim.x, 1);
            pending |= 2u;
        }
    }
    bool fail = !wait_buf(0);
    if (!fail) rcs_points<T>(sdesc[0], rows(0), pl0, trk_ptr, lambda, Linv_out, lp_out, sc, fp64_v);
    // Group k (buffer k & 1): one barrier (its per-point work and the previous
    // group's products are done), then the copy of group k + 1 into the other
    // buffer (from k = 1; the first two were issued above), the products of
    // group k, and - as each thread finishes its products - the per-point
    // work of group k + 1, overlapping the slower warps' products.
    for (int k = 0;; ++k) {
        const int b = k & 1;
        if (tm) ta = global_ns_rcs();
        if (__syncthreads_or(fail)) {
            // give up: flag it, let the copies still in flight land (bounded), leave
            if (threadIdx.x == 0) {
                atomicExch(&sc->err, (int)BA_ERR_TIMEOUT);
                for (int q = 0; q < 2; ++q)
                    if ((pending >> q) & 1u) mbar_wait(&mbar[q], (parity >> q) & 1u, limit);
            }
            return;
        }
        if (tm) tb = global_ns_rcs();
        const int gn = gi + (int)gridDim.x;
        if (k >= 1 && gn < ngroups && threadIdx.x == 0) {
            issue(gn, b ^ 1);
            pending |= 1u << (b ^ 1);
        }
        rcs_products<T>(sdesc[b], rows(b), plist(b), items, part);
        if (tm) tc = global_ns_rcs();
        if (gn < ngroups) {
            fail = !wait_buf(b ^ 1);
            if (!fail) rcs_points<T>(sdesc[b ^ 1], rows(b ^ 1), pl0, trk_ptr, lambda, Linv_out, lp_out, sc, fp64_v);
        }
        if (tm) {
            t_bar += tb - ta;
            t_prod += tc - tb;
            t_pts += global_ns_rcs() - tc;
            ++ngr;
        }
        if (gn >= ngroups) break;
        gi = gn;
    }
    if (tm && ngr) {
        atomicAdd(&sc->ph_rcs[0], (double)t_bar);
        atomicAdd(&sc->ph_rcs[1], (double)t_prod);
        atomicAdd(&sc->ph_rcs[2], (double)t_pts);
        atomicAdd(&sc->ph_rcs[3], (double)ngr);
    }
}

// K3: S[block] = sum of the block's partials in list order (fixed), a thread
// per 16-byte chunk of the block (9 for FP32, 18 for FP64): the chunks of a
// partial are read by consecutive threads, and each thread keeps four
// partials' loads in flight before adding them in order.  (Writing each
// partial straight to a block-ordered slot in RCS formation made this
// reduction contiguous but cost the formation more than it saved here.)
__device__ __forceinline__ void add16(float4 &s, const float4 v) {
    s.x += v.x; s.y += v.y; s.z += v.z; s.w += v.w;
}
__device__ __forceinline__ void add16(double2 &s, const double2 v) {
    s.x += v.x; s.y += v.y;
}
template <typename T>
__global__ void __launch_bounds__(256) k_rcs_reduce(int64_t nblk, const int *__restrict__ pptr, const int *__restrict__ plist,
                                                    const T *__restrict__ part, T *__restrict__ S) {
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    constexpr int NCH = BW * (int)sizeof(T) / 16;
    const V *pv = reinterpret_cast<const V *>(part);
    V *sv = reinterpret_cast<V *>(S);
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < nblk * NCH; x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t blk = x / NCH;
        const int c = (int)(x - blk * NCH);
        const int q1 = __ldg(pptr + blk + 1);
        int q = __ldg(pptr + blk);
        V s;
        std::memset(&s, 0, sizeof(V));
        for (; q + 4 <= q1; q += 4) {
            const int i0 = __ldg(plist + q), i1 = __ldg(plist + q + 1), i2 = __ldg(plist + q + 2),
                      i3 = __ldg(plist + q + 3);
            const V v0 = pv[(int64_t)i0 * NCH + c], v1 = pv[(int64_t)i1 * NCH + c], v2 = pv[(int64_t)i2 * NCH + c],
                    v3 = pv[(int64_t)i3 * NCH + c];
            add16(s, v0);
            add16(s, v1);
            add16(s, v2);
            add16(s, v3);
        }
        for (; q < q1; ++q) add16(s, pv[(int64_t)__ldg(plist + q) * NCH + c]);
        sv[x] = s;
    }
}

// K4: unpack the diagonal blocks, damp them, extract b, invert for M^-1.
template <typename T>
__global__ void k_rcs_diag(int n, const int *__restrict__ row_ptr, T *__restrict__ S, T *__restrict__ b,
                           T *__restrict__ Minv, double lambda, DevScalars *sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T *Sd = S + (int64_t)row_ptr[i] * BW;
    T pk[36], A[36], Ai[36];
#pragma unroll
    for (int q = 0; q < 36; ++q) pk[q] = Sd[q];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int c = r; c < 6; ++c) {
            A[6 * r + c] = pk[up_idx(r, c)];
            A[6 * c + r] = pk[up_idx(r, c)];
        }
    const T lam = (T)lambda;
#pragma unroll
    for (int r = 0; r < 6; ++r) A[7 * r] += lam * clampT(pk[21 + r]);
#pragma unroll
    for (int q = 0; q < 36; ++q) Sd[q] = A[q];
#pragma unroll
    for (int r = 0; r < 6; ++r) b[6 * i + r] = pk[27 + r];
    if (!spd_inverse6<T>(A, Ai)) {
        atomicExch(&sc->err, (int)BA_ERR_NOT_SPD);
#pragma unroll
        for (int q = 0; q < 36; ++q) Ai[q] = T(0);
    }
#pragma unroll
    for (int q = 0; q < 36; ++q) Minv[36 * (int64_t)i + q] = Ai[q];
}

// Block-Jacobi only: M_i^-1 = S_ii^-1 (diagonal blocks stored full, first in each row).
template <typename T>
__global__ void k_block_jacobi(int n, const int *__restrict__ row_ptr, const T *__restrict__ S, T *__restrict__ Minv,
                               DevScalars *sc) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    T A[36], Ai[36];
    const T *d = S + (int64_t)row_ptr[i] * BW;
#pragma unroll
    for (int q = 0; q < 36; ++q) A[q] = d[q];
    if (!spd_inverse6<T>(A, Ai)) {
        atomicExch(&sc->err, (int)BA_ERR_NOT_SPD);
#pragma unroll
        for (int q = 0; q < 36; ++q) Ai[q] = T(0);
    }
#pragma unroll
    for (int q = 0; q < 36; ++q) Minv[36 * (int64_t)i + q] = Ai[q];
}

static inline int grid_for(int64_t work, int threads, int cap) {
    int64_t g = (work + threads - 1) / threads;
    return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

static int form_o_cap(const ba_problem *p) { return std::max(1, p->hs.max_nobs); }
static int form_c_cap(const ba_problem *p) { return std::max(4, (p->hs.max_nc + 3) & ~3); }

template <typename T>
static cudaError_t form_rcs_T(ba_problem *p, double lambda, size_t smem, long long limit) {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_form_rcs<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
    int ctas_per_sm = 0, n_sm = 0;
    if ((e = occupancy((const void *)k_form_rcs<T>, FORM_THREADS, smem, &ctas_per_sm, &n_sm)) != cudaSuccess) return e;
    ctas_per_sm = std::max(1, ctas_per_sm);
    const int grid = (int)std::min<int64_t>(p->ngroups, (int64_t)ctas_per_sm * n_sm);
    k_form_rcs<T><<<grid, FORM_THREADS, smem, p->st>>>(p->grp, (int)p->ngroups, p->items, p->contrib, p->trk_ptr,
                                                      (const T *)p->J, lambda, (T *)p->part, (T *)p->Linv, (T *)p->lp,
                                                      p->sc, p->fp32 ? 1 : 0, form_o_cap(p), form_c_cap(p), limit,
                                                      p->opt.profile >= 2 ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_block_jacobi(ba_problem *p) {
    const int nb = (p->n + 127) / 128;
    if (p->fp32)
        k_block_jacobi<float><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (const float *)p->S, (float *)p->Minv, p->sc);
    else
        k_block_jacobi<double><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (const double *)p->S, (double *)p->Minv, p->sc);
    p->launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_form_rcs(ba_problem *p, double lambda) {
    cudaError_t err;
    cudaEvent_t ev;
    const size_t smem =
        2 * form_round128(form_round128((size_t)form_o_cap(p) * JW * p->esz) + (size_t)form_c_cap(p) * sizeof(uint32_t));
    const long long limit = 4000000000LL;  // ~2 s of SM clock per copy wait
    // points re-factored in FP64 are counted per formation
    if ((err = cudaMemsetAsync(&p->sc->n_v64, 0, sizeof(unsigned long long), p->st)) != cudaSuccess) return err;
    ktimer_begin(p, K_FORM_RCS, &ev);
    if (p->fp32)
        err = form_rcs_T<float>(p, lambda, smem, limit);
    else
        err = form_rcs_T<double>(p, lambda, smem, limit);
    ktimer_end(p, K_FORM_RCS, ev);
    p->launches += 1;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    ktimer_begin(p, K_RCS_REDUCE, &ev);
    const int g = grid_for(p->nnzb * (int64_t)(BW * p->esz / 16), 256, 152 * 16);
    if (p->fp32)
        k_rcs_reduce<float><<<g, 256, 0, p->st>>>(p->nnzb, p->pptr, p->plist, (const float *)p->part, (float *)p->S);
    else
        k_rcs_reduce<double><<<g, 256, 0, p->st>>>(p->nnzb, p->pptr, p->plist, (const double *)p->part,
                                                   (double *)p->S);
    ktimer_end(p, K_RCS_REDUCE, ev);
    p->launches += 1;
    if ((err = cudaGetLastError()) != cudaSuccess) return err;
    ktimer_begin(p, K_RCS_DIAG, &ev);
    const int nb = (p->n + 127) / 128;
    if (p->fp32)
        k_rcs_diag<float><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (float *)p->S, (float *)p->b, (float *)p->Minv,
                                                 lambda, p->sc);
    else
        k_rcs_diag<double><<<nb, 128, 0, p->st>>>(p->n, p->row_ptr, (double *)p->S, (double *)p->b,
                                                  (double *)p->Minv, lambda, p->sc);
    ktimer_end(p, K_RCS_DIAG, ev);
    p->launches += 1;
    return cudaGetLastError();
}

}  // namespace ba
