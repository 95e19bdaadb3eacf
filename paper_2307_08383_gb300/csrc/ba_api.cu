// C ABI of libba (declared in include/ba.h) and the host side of one LM
// iteration: linearize -> form RCS (Eq. 4) -> PCG (Sec. 3.2) -> back-substitute
// (Eq. 5) -> trial evaluation -> accept / reject (Fig. 2 pipeline).  Every
// step runs on the caller's stream in the kernels of k_obs.cu, k_rcs.cu and
// k_pcg.cu; only scalars come back to the host.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <tuple>
#include <mutex>
#include <map>
#include <string>

#include "ba_internal.h"

namespace ba {
cudaError_t launch_accumulate_solution(ba_problem *p, bool first);
}

using namespace ba;

static thread_local std::string g_err;

static ba_status fail(ba_status s, const std::string &m) {
    g_err = m;
    return s;
}

#define CK(p, call)                                                                                   \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            (p)->dead = true;                                                                         \
            return fail(BA_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));            \
        }                                                                                             \
    } while (0)

#define LIVE(p)                                                                                       \
    do {                                                                                              \
        if (!(p)) return fail(BA_ERR_INVALID_ARG, "null problem");                                    \
        if ((p)->dead) return fail(BA_ERR_STATE, "problem unusable after an earlier CUDA/internal error"); \
    } while (0)

namespace ba {

ba_status set_error(ba_status s, const char *msg) { return fail(s, msg); }

cudaError_t occupancy(const void *kernel, int threads, size_t smem, int *per_sm, int *n_sm) {
    static std::mutex mu;
    static std::map<std::tuple<int, const void *, int, size_t>, std::pair<int, int>> cache;
    int dev = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    const auto key = std::make_tuple(dev, kernel, threads, smem);
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it == cache.end()) {
        int sms = 0, ps = 0;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ps, kernel, threads, smem)) != cudaSuccess) return e;
        it = cache.emplace(key, std::make_pair(ps, sms)).first;
    }
    *per_sm = it->second.first;
    *n_sm = it->second.second;
    return cudaSuccess;
}

const char *kernel_name(int k) {
    static const char *names[K_COUNT] = {"prepare_state", "linearize", "cost",    "form_rcs",
                                         "rcs_reduce",    "rcs_diag",  "pcg_init", "pcg_loop",
                                         "resid64",       "back_substitute", "trial_cameras",
                                         "demote",        "split_prepare", "step_points",
                                         "triangulate"};
    return (k >= 0 && k < K_COUNT) ? names[k] : nullptr;
}

static bool timed(const ba_problem *p, int k) {
    if (!p->opt.profile) return false;
    return true;
}

void ktimer_begin(ba_problem *p, int k, cudaEvent_t *a) {
    *a = nullptr;
    if (!timed(p, k)) return;
    if (p->ev_pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        p->ev_pool.push_back(e);
    }
    *a = p->ev_pool.back();
    p->ev_pool.pop_back();
    cudaEventRecord(*a, p->st);
}

void ktimer_end(ba_problem *p, int k, cudaEvent_t a) {
    if (!a) return;
    cudaEvent_t b;
    if (p->ev_pool.empty()) {
        if (cudaEventCreate(&b) != cudaSuccess) { p->ev_pool.push_back(a); return; }
    } else {
        b = p->ev_pool.back();
        p->ev_pool.pop_back();
    }
    cudaEventRecord(b, p->st);
    p->pending.push_back({k, a, b});
    if (p->pending.size() > 8192) ktimer_flush(p);
}

ba_status ktimer_flush(ba_problem *p) {
    if (p->pending.empty()) return BA_OK;
    if (cudaEventSynchronize(p->pending.back().b) != cudaSuccess) return fail(BA_ERR_CUDA, "event sync");
    for (auto &q : p->pending) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, q.a, q.b);
        p->klaunch[q.k] += 1;
        p->kms[q.k] += ms;
        p->ev_pool.push_back(q.a);
        p->ev_pool.push_back(q.b);
    }
    p->pending.clear();
    return BA_OK;
}

}  // namespace ba

// ----------------------------------------------------------------------------
// allocation helpers
// ----------------------------------------------------------------------------
template <typename X>
static cudaError_t dalloc(ba_problem *p, X **ptr, size_t count) {
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(X), 16);
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return e;
    p->allocs.push_back(q);
    p->dev_bytes += bytes;
    *ptr = (X *)q;
    return cudaSuccess;
}
static cudaError_t dalloc_raw(ba_problem *p, void **ptr, size_t bytes) {
    return dalloc(p, (unsigned char **)ptr, bytes);
}

template <typename X>
static cudaError_t upload(ba_problem *p, X *dst, const X *src, size_t count) {
    if (count == 0) return cudaSuccess;
    cudaError_t e = cudaMemcpyAsync(dst, src, count * sizeof(X), cudaMemcpyHostToDevice, p->st);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(p->st);
}

static void free_all(ba_problem *p) {
    for (void *q : p->allocs) cudaFree(q);
    p->allocs.clear();
    for (auto &q : p->pending) {
        cudaEventDestroy(q.a);
        cudaEventDestroy(q.b);
    }
    p->pending.clear();
    for (auto e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    for (auto &e : p->step_ev)
        if (e) {
            cudaEventDestroy(e);
            e = nullptr;
        }
    if (p->sc_host) cudaFreeHost(p->sc_host);
    p->sc_host = nullptr;
}

static bool finite_all(const double *x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

static ba_status sync_scalars(ba_problem *p) {
    CK(p, cudaMemcpyAsync(p->sc_host, p->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, p->st));
    CK(p, cudaStreamSynchronize(p->st));
    return BA_OK;
}

static void to_double(const void *src, bool fp32, double *dst, size_t cnt) {
    if (fp32) {
        for (size_t i = 0; i < cnt; ++i) dst[i] = ((const float *)src)[i];
    } else {
        std::memcpy(dst, src, cnt * 8);
    }
}

static void default_view(ba_problem *p) {
    p->sv.f32 = p->fp32;
    p->sv.S = p->S;
    p->sv.Minv = p->Minv;
    for (int k = 0; k < 8; ++k) p->sv.pv[k] = p->pv[k];
}

// device array of the mode precision -> host doubles
static ba_status fetch(ba_problem *p, const void *dev, size_t cnt, std::vector<double> &out) {
    std::vector<unsigned char> raw(cnt * p->esz);
    out.resize(cnt);
    CK(p, cudaMemcpyAsync(raw.data(), dev, cnt * p->esz, cudaMemcpyDeviceToHost, p->st));
    CK(p, cudaStreamSynchronize(p->st));
    to_double(raw.data(), p->fp32, out.data(), cnt);
    return BA_OK;
}

// ----------------------------------------------------------------------------
// C ABI
// ----------------------------------------------------------------------------
extern "C" {

void ba_options_default(ba_options *o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->precision = BA_FP64;
    o->fx = o->fy = 1000.0;
    o->cx = o->cy = 500.0;
    o->robust = BA_LOSS_PLAIN;
    o->huber_delta = 2.0;
    o->lambda0 = 1e-4;
    o->pcg_rel_tol = 1e-10;
    o->pcg_max_iters = 0;
    o->inner_rel_tol = 1e-4;
    o->refine_max = 20;
    o->preconditioner = BA_PC_BLOCK_JACOBI;
    o->cuda_stream = nullptr;
    o->device_mem_cap = 0;
    o->group_max_obs = 0;
    o->profile = 0;
    o->solve_precision = 0;
    o->pcg_variant = BA_PCG_AUTO;
}

const char *ba_last_error(void) { return g_err.c_str(); }

const char *ba_kernel_name(int32_t k) { return ba::kernel_name(k); }

ba_status ba_symbolic_pattern(int32_t n_cams, int64_t n_pts, int64_t n_obs, const int32_t *obs_cam,
                              const int64_t *obs_pt, int32_t *row_ptr, int32_t *col, int64_t *nnzb) {
    HostSetup hs;
    std::string err;
    ba_status s = symbolic_setup(n_cams, n_pts, n_obs, obs_cam, obs_pt, nullptr, OBS_MAX_DEFAULT, true, hs, err);
    if (s != BA_OK) return fail(s, err);
    if (nnzb) *nnzb = (int64_t)hs.col.size();
    if (row_ptr) std::memcpy(row_ptr, hs.row_ptr.data(), hs.row_ptr.size() * sizeof(int32_t));
    if (col) std::memcpy(col, hs.col.data(), hs.col.size() * sizeof(int32_t));
    return BA_OK;
}

ba_status ba_problem_create(const ba_options *opt, int32_t n_cams, const double *cams, int64_t n_pts,
                            const double *pts, int64_t n_obs, const int32_t *obs_cam, const int64_t *obs_pt,
                            const double *obs_uv, ba_problem **out) {
    if (!out) return fail(BA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (!cams || !pts || !obs_cam || !obs_pt || !obs_uv) return fail(BA_ERR_INVALID_ARG, "null input array");
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return fail(BA_ERR_INVALID_ARG, "precision must be BA_FP64 or BA_FP32");
    if (o.robust != BA_LOSS_PLAIN && o.robust != BA_LOSS_HUBER) return fail(BA_ERR_INVALID_ARG, "robust must be BA_LOSS_PLAIN or BA_LOSS_HUBER");
    if (o.robust == BA_LOSS_HUBER && !(o.huber_delta > 0)) return fail(BA_ERR_INVALID_ARG, "huber_delta must be > 0");
    if (!(o.lambda0 >= 0) || !(o.pcg_rel_tol > 0) || !(o.inner_rel_tol > 0) || o.pcg_max_iters < 0 || o.refine_max < 1 ||
        o.pcg_variant < BA_PCG_AUTO || o.pcg_variant > BA_PCG_IMPLICIT)
        return fail(BA_ERR_INVALID_ARG, "bad solver option");
    if (!(o.fx > 0) || !(o.fy > 0) || !std::isfinite(o.cx) || !std::isfinite(o.cy))
        return fail(BA_ERR_INVALID_ARG, "bad intrinsics");
    if (o.preconditioner != BA_PC_BLOCK_JACOBI) return fail(BA_ERR_INVALID_ARG, "only BA_PC_BLOCK_JACOBI is available");
    if (n_cams <= 0 || n_pts <= 0 || n_obs <= 0) return fail(BA_ERR_INVALID_ARG, "sizes must be positive");
    if (!finite_all(cams, (size_t)n_cams * 6) || !finite_all(pts, (size_t)n_pts * 3) ||
        !finite_all(obs_uv, (size_t)n_obs * 2))
        return fail(BA_ERR_NONFINITE, "non-finite camera, point or observation value");

    ba_problem *p = new ba_problem();
    p->opt = o;
    p->st = (cudaStream_t)o.cuda_stream;
    p->n = n_cams;
    p->P = n_pts;
    p->m = n_obs;
    p->fp32 = (o.precision == BA_FP32);
    p->esz = p->fp32 ? 4 : 8;
    p->obs_max = o.group_max_obs > 0 ? std::min(std::max(o.group_max_obs, 40), OBS_MAX_LIMIT) : OBS_MAX_DEFAULT;
    p->lambda = o.lambda0;
    p->nu = 2.0;
    std::string err;
    ba_status s = symbolic_setup(n_cams, n_pts, n_obs, obs_cam, obs_pt, pts, p->obs_max, false, p->hs, err);
    if (s != BA_OK) {
        delete p;
        return fail(s, err);
    }
    HostSetup &hs = p->hs;
    p->nnzb = (int64_t)hs.col.size();
    p->ngroups = (int64_t)hs.groups.size();
    p->npart = (int64_t)hs.lb_gblk.size();
    p->nitems = (int64_t)hs.items.size();
    const int64_t n = n_cams, P = n_pts, m = n_obs;
    const size_t E = p->esz;

    // planned device bytes (checked against the cap before any allocation)
    const size_t camc_w = p->fp32 ? CAMC32_W * 4 : 12 * 8;
    size_t plan = 2 * (n * 6 * 8 + P * 3 * 8 + n * camc_w + (p->fp32 ? P * 6 * 4 + m * 2 * 4 : 0)) +
                  m * 4 * 2 + (P + 1) * 4 + m * 16 + (p->fp32 ? m * 16 : 0) + m * JW * E + (n + 1) * 4 +
                  p->nnzb * 4 + 2 * (n + 1) * 4 + 2 * p->nnzb * 4 + (2 * p->nnzb - n) * 8 + p->nnzb * BW * E + n * 6 * E + n * 36 * E + p->ngroups * sizeof(GroupDesc) +
                  p->nitems * 8 + hs.contrib.size() * 4 + (p->nnzb + 1) * 4 + p->npart * 4 + p->npart * BW * E +
                  P * 9 * E + 8 * n * 6 * E + 3 * n * 6 * 8 + n * 6 * E + P * 3 * E + sizeof(DevScalars) +
                  RED_SLOTS * 8 + N_COUNTERS * 4;
    if (o.device_mem_cap && plan > o.device_mem_cap) {
        delete p;
        return fail(BA_ERR_OOM, "problem needs " + std::to_string(plan) + " device bytes, cap is " +
                                    std::to_string(o.device_mem_cap));
    }
#define AL(ptr, cnt)                                                                                  \
    do {                                                                                              \
        cudaError_t e_ = dalloc(p, &(ptr), (cnt));                                                    \
        if (e_ != cudaSuccess) {                                                                      \
            free_all(p);                                                                              \
            delete p;                                                                                 \
            cudaGetLastError();                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,                   \
                        std::string("cudaMalloc: ") + cudaGetErrorString(e_));                        \
        }                                                                                             \
    } while (0)
#define ALR(ptr, bytes)                                                                               \
    do {                                                                                              \
        cudaError_t e_ = dalloc_raw(p, &(ptr), (bytes));                                              \
        if (e_ != cudaSuccess) {                                                                      \
            free_all(p);                                                                              \
            delete p;                                                                                 \
            cudaGetLastError();                                                                       \
            return fail(e_ == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,                   \
                        std::string("cudaMalloc: ") + cudaGetErrorString(e_));                        \
        }                                                                                             \
    } while (0)
    for (StateBuf *sb : {&p->cur, &p->trial}) {
        AL(sb->cams, n * 6);
        AL(sb->pts, P * 3);
        ALR(sb->camc, n * camc_w);
        if (p->fp32) AL(sb->pts_hl, P * 6);
        if (p->fp32) AL(sb->e, m * 2);
    }
    AL(p->obs_cam, m);
    AL(p->obs_pt, m);
    AL(p->trk_ptr, P + 1);
    AL(p->uv64, m * 2);
    if (p->fp32) AL(p->uv32, m * 2);
    if (p->fp32) AL(p->uv_lo, m * 2);
    ALR(p->J, m * JW * E);
    AL(p->row_ptr, n + 1);
    AL(p->col, p->nnzb);
    AL(p->ct_ptr, n + 1);
    AL(p->ct_blk, p->nnzb - n);
    AL(p->ct_row, p->nnzb - n);
    AL(p->tw_ptr, n + 1);
    AL(p->tw_ent, 2 * p->nnzb - n);
    ALR(p->S, p->nnzb * BW * E);
    ALR(p->b, n * 6 * E);
    ALR(p->Minv, n * 36 * E);
    AL(p->grp, p->ngroups);
    AL(p->items, p->nitems);
    AL(p->contrib, hs.contrib.size());
    AL(p->pptr, p->nnzb + 1);
    AL(p->plist, p->npart);
    ALR(p->part, p->npart * BW * E);
    ALR(p->Linv, P * 6 * E);
    ALR(p->lp, P * 3 * E);
    for (int k = 0; k < 8; ++k) ALR(p->pv[k], n * 6 * E);
    AL(p->x64, n * 6);
    AL(p->r64, n * 6);
    AL(p->q64, n * 6);
    ALR(p->dxc, n * 6 * E);
    ALR(p->dxp, P * 3 * E);
    AL(p->sc, 1);
    AL(p->red, RED_SLOTS);
    AL(p->counters, N_COUNTERS);
#undef AL
#undef ALR
    if (cudaMallocHost((void **)&p->sc_host, sizeof(DevScalars)) != cudaSuccess) {
        free_all(p);
        delete p;
        return fail(BA_ERR_CUDA, "cudaMallocHost failed");
    }
    // uploads (internal orders)
    std::vector<double> tmp;
    cudaError_t e = cudaSuccess;
    auto up_ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    up_ok(upload(p, p->cur.cams, cams, n * 6));
    tmp.resize(P * 3);
    for (int64_t k = 0; k < P; ++k)
        for (int d = 0; d < 3; ++d) tmp[3 * k + d] = pts[3 * hs.pt_perm[k] + d];
    up_ok(upload(p, p->cur.pts, tmp.data(), P * 3));
    up_ok(upload(p, p->obs_cam, hs.obs_cam.data(), m));
    up_ok(upload(p, p->obs_pt, hs.obs_pt.data(), m));
    up_ok(upload(p, p->trk_ptr, hs.trk_ptr.data(), P + 1));
    tmp.resize(m * 2);
    for (int64_t a = 0; a < m; ++a) {
        tmp[2 * a] = obs_uv[2 * hs.obs_perm[a]];
        tmp[2 * a + 1] = obs_uv[2 * hs.obs_perm[a] + 1];
    }
    up_ok(upload(p, p->uv64, tmp.data(), m * 2));
    if (p->fp32) {
        std::vector<float> t32(m * 2);
        for (int64_t x = 0; x < m * 2; ++x) t32[x] = (float)tmp[x];
        up_ok(upload(p, p->uv32, t32.data(), m * 2));
        for (int64_t x = 0; x < m * 2; ++x) t32[x] = (float)(tmp[x] - (double)t32[x]);
        up_ok(upload(p, p->uv_lo, t32.data(), m * 2));
    }
    up_ok(upload(p, p->row_ptr, hs.row_ptr.data(), n + 1));
    up_ok(upload(p, p->col, hs.col.data(), p->nnzb));
    up_ok(upload(p, p->ct_ptr, hs.ct_ptr.data(), n + 1));
    up_ok(upload(p, p->ct_blk, hs.ct_blk.data(), p->nnzb - n));
    up_ok(upload(p, p->ct_row, hs.ct_row.data(), p->nnzb - n));
    up_ok(upload(p, p->tw_ptr, hs.tw_ptr.data(), n + 1));
    up_ok(upload(p, p->tw_ent, hs.tw_ent.data(), 2 * p->nnzb - n));
    up_ok(upload(p, p->grp, hs.groups.data(), p->ngroups));
    up_ok(upload(p, p->items, hs.items.data(), p->nitems));
    up_ok(upload(p, p->contrib, hs.contrib.data(), hs.contrib.size()));
    up_ok(upload(p, p->pptr, hs.pptr.data(), p->nnzb + 1));
    up_ok(upload(p, p->plist, hs.plist.data(), p->npart));
    up_ok(cudaMemsetAsync(p->q64, 0, n * 6 * 8, p->st));
    up_ok(cudaMemsetAsync(p->x64, 0, n * 6 * 8, p->st));
    up_ok(cudaMemsetAsync(p->sc, 0, sizeof(DevScalars), p->st));
    up_ok(cudaMemsetAsync(p->counters, 0, N_COUNTERS * 4, p->st));
    up_ok(cudaMemsetAsync(p->dxc, 0, n * 6 * E, p->st));
    up_ok(cudaMemsetAsync(p->dxp, 0, P * 3 * E, p->st));
    // drop host copies that the device now holds (keep permutations and pattern)
    std::vector<GroupDesc>().swap(hs.groups);
    std::vector<ItemDesc>().swap(hs.items);
    std::vector<int32_t>().swap(hs.lb_gblk);
    std::vector<uint32_t>().swap(hs.contrib);
    std::vector<int32_t>().swap(hs.pptr);
    std::vector<int32_t>().swap(hs.plist);
    std::vector<int32_t>().swap(hs.obs_pt);
    std::vector<int32_t>().swap(hs.trk_ptr);
    std::vector<int32_t>().swap(hs.ct_ptr);
    std::vector<int32_t>().swap(hs.ct_blk);
    std::vector<int32_t>().swap(hs.ct_row);
    std::vector<int32_t>().swap(hs.tw_ptr);
    std::vector<int2>().swap(hs.tw_ent);
    default_view(p);
    if (e == cudaSuccess) e = launch_prepare_state(p, p->cur);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) {
        free_all(p);
        delete p;
        return fail(BA_ERR_CUDA, std::string("problem upload: ") + cudaGetErrorString(e));
    }
    *out = p;
    return BA_OK;
}

ba_status ba_problem_create_rcs(const ba_options *opt, int32_t n, int64_t nnzb, const int32_t *row_ptr,
                                const int32_t *col, const double *val, const double *b, ba_problem **out) {
    if (!out) return fail(BA_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    ba_options o;
    if (opt) o = *opt; else ba_options_default(&o);
    if (n <= 0 || nnzb < n || nnzb >= (int64_t)INT32_MAX) return fail(BA_ERR_INVALID_ARG, "need 0 < n <= nnzb < 2^31");
    if (!row_ptr || !col || !val || !b) return fail(BA_ERR_INVALID_ARG, "null input array");
    if (o.precision != BA_FP64 && o.precision != BA_FP32) return fail(BA_ERR_INVALID_ARG, "bad precision");
    if (!(o.pcg_rel_tol > 0) || !(o.inner_rel_tol > 0) || o.pcg_max_iters < 0 || o.refine_max < 1 ||
        o.pcg_variant < BA_PCG_AUTO || o.pcg_variant > BA_PCG_SPLIT)
        return fail(BA_ERR_INVALID_ARG, "bad solver option");
    if (row_ptr[0] != 0 || row_ptr[n] != nnzb) return fail(BA_ERR_INVALID_ARG, "row_ptr must run from 0 to nnzb");
    for (int32_t i = 0; i < n; ++i) {
        if (row_ptr[i + 1] <= row_ptr[i]) return fail(BA_ERR_INVALID_ARG, "every row needs its diagonal block");
        if (col[row_ptr[i]] != i) return fail(BA_ERR_INVALID_ARG, "the first block of row i must be (i, i)");
        for (int32_t q = row_ptr[i] + 1; q < row_ptr[i + 1]; ++q)
            if (col[q] <= col[q - 1] || col[q] >= n) return fail(BA_ERR_INVALID_ARG, "columns must ascend within [i, n)");
    }
    if (!finite_all(val, (size_t)nnzb * 36) || !finite_all(b, (size_t)n * 6))
        return fail(BA_ERR_NONFINITE, "non-finite RCS value");
    ba_problem *p = new ba_problem();
    p->opt = o;
    p->st = (cudaStream_t)o.cuda_stream;
    p->n = n;
    p->P = 0;
    p->m = 0;
    p->fp32 = (o.precision == BA_FP32);
    p->esz = p->fp32 ? 4 : 8;
    p->rcs_only = true;
    p->nnzb = nnzb;
    p->hs.row_ptr.assign(row_ptr, row_ptr + n + 1);
    p->hs.col.assign(col, col + nnzb);
    build_twosided(p->hs, n);
    const size_t E = p->esz;
    cudaError_t e = cudaSuccess;
    auto A = [&](void **q, size_t bytes) { if (e == cudaSuccess) e = dalloc_raw(p, q, bytes); };
    A((void **)&p->row_ptr, (n + 1) * 4);
    A((void **)&p->col, nnzb * 4);
    A((void **)&p->tw_ptr, (n + 1) * 4);
    A((void **)&p->tw_ent, (2 * nnzb - n) * 8);
    A(&p->S, nnzb * BW * E);
    A(&p->b, (size_t)n * 6 * E);
    A(&p->Minv, (size_t)n * 36 * E);
    for (int k = 0; k < 8; ++k) A(&p->pv[k], (size_t)n * 6 * E);
    A((void **)&p->x64, (size_t)n * 6 * 8);
    A((void **)&p->r64, (size_t)n * 6 * 8);
    A((void **)&p->q64, (size_t)n * 6 * 8);
    A(&p->dxc, (size_t)n * 6 * E);
    A((void **)&p->sc, sizeof(DevScalars));
    A((void **)&p->red, RED_SLOTS * 8);
    A((void **)&p->counters, N_COUNTERS * 4);
    if (e == cudaSuccess && cudaMallocHost((void **)&p->sc_host, sizeof(DevScalars)) != cudaSuccess)
        e = cudaErrorMemoryAllocation;
    auto up_ok = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    up_ok(upload(p, p->row_ptr, row_ptr, n + 1));
    up_ok(upload(p, p->col, col, nnzb));
    up_ok(upload(p, p->tw_ptr, p->hs.tw_ptr.data(), n + 1));
    up_ok(upload(p, p->tw_ent, p->hs.tw_ent.data(), 2 * nnzb - n));
    if (p->fp32) {
        std::vector<float> t((size_t)nnzb * 36);
        for (size_t k = 0; k < t.size(); ++k) t[k] = (float)val[k];
        up_ok(upload(p, (float *)p->S, t.data(), t.size()));
        std::vector<float> tb((size_t)n * 6);
        for (size_t k = 0; k < tb.size(); ++k) tb[k] = (float)b[k];
        up_ok(upload(p, (float *)p->b, tb.data(), tb.size()));
    } else {
        up_ok(upload(p, (double *)p->S, val, (size_t)nnzb * 36));
        up_ok(upload(p, (double *)p->b, b, (size_t)n * 6));
    }
    up_ok(cudaMemsetAsync(p->q64, 0, (size_t)n * 6 * 8, p->st));
    up_ok(cudaMemsetAsync(p->x64, 0, (size_t)n * 6 * 8, p->st));
    up_ok(cudaMemsetAsync(p->sc, 0, sizeof(DevScalars), p->st));
    up_ok(cudaMemsetAsync(p->counters, 0, N_COUNTERS * 4, p->st));
    std::vector<int2>().swap(p->hs.tw_ent);
    std::vector<int32_t>().swap(p->hs.tw_ptr);
    if (e == cudaSuccess) e = launch_block_jacobi(p);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess) {
        free_all(p);
        delete p;
        return fail(e == cudaErrorMemoryAllocation ? BA_ERR_OOM : BA_ERR_CUDA,
                    std::string("RCS problem creation: ") + cudaGetErrorString(e));
    }
    default_view(p);
    p->rcs_formed = true;
    ++p->rcs_gen;
    p->lambda = 0.0;
    if (sync_scalars(p) == BA_OK && p->sc_host->err == BA_ERR_NOT_SPD) {
        free_all(p);
        delete p;
        return fail(BA_ERR_NOT_SPD, "a diagonal block of the RCS is not positive definite");
    }
    *out = p;
    return BA_OK;
}

void ba_problem_destroy(ba_problem *p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    else cudaDeviceSynchronize();
    gnn_free(p);
    if (p->Minv_bj) cudaFree(p->Minv_bj);
    free_all(p);
    delete p;
}

static ba_status check_err_flag(ba_problem *p) {
    if (p->sc_host->err) {
        int e = p->sc_host->err;
        CK(p, cudaMemsetAsync(&p->sc->err, 0, sizeof(int), p->st));
        if (e == BA_ERR_NOT_SPD) return fail(BA_ERR_NOT_SPD, "a V_k or RCS diagonal block is not positive definite");
        p->dead = true;
        return fail(BA_ERR_INTERNAL, "device consistency check failed");
    }
    return BA_OK;
}

static ba_status ensure_cost(ba_problem *p) {
    if (p->have_F) return BA_OK;
    CK(p, launch_cost(p, p->cur, false));
    ba_status s = sync_scalars(p);
    if (s) return s;
    p->F = p->sc_host->cost;
    p->have_F = true;
    p->last_rel_decrease = INFINITY;  // a fresh state: the next trial cost is evaluated whole
    if (!std::isfinite(p->F)) return fail(BA_ERR_NONFINITE, "non-finite cost");
    return BA_OK;
}

ba_status ba_linearize(ba_problem *p, double *cost_out) {
    LIVE(p);
    if (p->rcs_only) return fail(BA_ERR_STATE, "ba_linearize: the problem holds an RCS only");
    CK(p, launch_linearize(p));
    p->linearized = true;
    p->rcs_formed = p->solved = p->backsub = false;
    if (cost_out) {
        ba_status s = ensure_cost(p);
        if (s) return s;
        *cost_out = p->F;
    }
    return BA_OK;
}

ba_status ba_form_rcs(ba_problem *p, double lambda) {
    LIVE(p);
    if (p->rcs_only) return fail(BA_ERR_STATE, "ba_form_rcs: the problem holds an RCS only");
    if (!p->linearized) return fail(BA_ERR_STATE, "ba_form_rcs needs ba_linearize first");
    if (!(lambda >= 0) || !std::isfinite(lambda)) return fail(BA_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    CK(p, launch_form_rcs(p, lambda));
    p->minv_learned = false;
    p->rcs_formed = true;
    ++p->rcs_gen;
    p->rcs_lambda = lambda;
    p->solved = p->backsub = false;
    return BA_OK;
}

// The implicit variant: the PCG product from the stored linearization
static bool implicit_cg(const ba_problem *p) { return p->opt.pcg_variant == BA_PCG_IMPLICIT; }

static ba_status run_pcg(ba_problem *p, const void *rhs, double tol, int max_iters, int *iters) {
    CK(p, launch_pcg_init(p, rhs, tol, max_iters));
    CK(p, implicit_cg(p) ? launch_pcg_implicit(p) : launch_pcg_loop(p));
    ba_status s = sync_scalars(p);
    if (s) return s;
    if (p->sc_host->err == BA_ERR_TIMEOUT) {
        p->dead = true;
        return fail(BA_ERR_TIMEOUT, "PCG grid barrier timed out");
    }
    *iters = p->sc_host->iters;
    return BA_OK;
}

// One solve with the current M^-1 (no learned-preconditioner logic).
static ba_status ensure_shadows(ba_problem *p, bool matrix) {
    if (!p->pv32[0])
        for (int k = 0; k < 8; ++k) CK(p, dalloc_raw(p, &p->pv32[k], (size_t)p->n * 6 * 4));
    if (matrix && !p->S32) {
        CK(p, dalloc_raw(p, &p->S32, (size_t)p->nnzb * BW * 4));
        CK(p, dalloc_raw(p, &p->Minv32, (size_t)p->n * 36 * 4));
    }
    return BA_OK;
}

// FP32 solves run the split CG unless the standard recurrence is asked for
// or the problem is too large for the balanced SpMV's shared memory
static bool split_cg(ba_problem *p) {
    return p->sv.f32 && (p->opt.pcg_variant == BA_PCG_AUTO || p->opt.pcg_variant == BA_PCG_SPLIT) &&
           split_available(p);
}


static ba_status solve_once_view(ba_problem *p, ba_step_info *info);

// One solve with the current M^-1 (no learned-preconditioner logic).  An FP64
// problem with solve_precision = BA_FP32 runs the inner PCG in FP32 - on the
// split system G^T S G formed from the FP64 S, or (standard variant) on a
// demoted copy of S and M^-1 - and refines with the FP64 residual b - S x of
// the FP64 system; the FP32 copies are made inside the timed solve.
static ba_status solve_once(ba_problem *p, ba_step_info *info) {
    // the implicit operator reads J in the problem's precision: no FP32 inner solve
    const bool mixed = !p->fp32 && p->opt.solve_precision == BA_FP32 && !implicit_cg(p);
    ba_status s;
    if (mixed) {
        const bool standard = p->opt.pcg_variant == BA_PCG_STANDARD || !split_available(p);
        if ((s = ensure_shadows(p, standard))) return s;
        if (standard) CK(p, launch_demote(p));
        p->sv.f32 = true;
        p->sv.S = p->S32;
        p->sv.Minv = p->Minv32;
        for (int k = 0; k < 8; ++k) p->sv.pv[k] = p->pv32[k];
    } else {
        default_view(p);
    }
    s = solve_once_view(p, info);
    default_view(p);
    return s;
}

static ba_status solve_once_view(ba_problem *p, ba_step_info *info) {
    const int max_iters = p->opt.pcg_max_iters > 0 ? p->opt.pcg_max_iters : std::max(1000, 6 * p->n);
    const double tol = p->opt.pcg_rel_tol;
    int total = 0, refine = 0;
    bool converged = false;
    ba_status s;
    if (!p->sv.f32) {
        int it = 0;
        if ((s = run_pcg(p, p->b, tol, max_iters, &it))) return s;
        if ((s = check_err_flag(p))) return s;
        total = it;
        converged = p->sc_host->rr <= p->sc_host->tol2 * p->sc_host->rr0;
        CK(p, launch_accumulate_solution(p, true));
        CK(p, launch_resid64(p, true));
    } else {
        const bool split = split_cg(p);
        if (split) CK(p, launch_split_prepare(p, p->minv_learned));
        // FP32 inner PCG + FP64 iterative refinement on r = b - S x.  Each
        // sweep asks its inner solve for inner_rel_tol, or for just the
        // reduction still missing (tol / rho, rho = |r|/|b| now) when that
        // is looser, so a loose tolerance such as the paper's T = 0.1 stops
        // where the FP64 PCG stops (the FP32 recurrence's residual norm, a
        // double-float sum, and the true one differ by far less than the
        // steps between iterations), and a last sweep that needs a factor of
        // a few takes a few iterations rather than a full inner solve.  Each
        // sweep asks for at least a 10 % reduction (at most 0.9): one that
        // follows a first sweep ending just above T by the recurrence's
        // residual gap then stops just below T too.
        // One host synchronisation per sweep: the first sweep always runs (r = b;
        // a zero b stops its PCG at once), and a sweep's PCG, accumulation and
        // residual are queued together and read back once.
        CK(p, launch_resid64(p, false));  // r64 = b, x64 implicit 0
        bool first = true;
        for (int o = 0; o < p->opt.refine_max; ++o) {
            if (!first) {
                if (p->sc_host->rr64 <= tol * tol * p->sc_host->bb64) { converged = true; break; }
                if (p->sc_host->bb64 == 0.0) { converged = true; break; }
            }
            CK(p, launch_refine_rhs(p, p->sv.pv[1]));  // r buffer doubles as the rhs (copied by init)
            const double rho = first ? 1.0 : std::sqrt(p->sc_host->rr64 / p->sc_host->bb64);
            const double inner = std::min(0.9, std::max(p->opt.inner_rel_tol, tol / rho));
            if (split) {
                CK(p, launch_split_init(p, (const float *)p->sv.pv[1], inner, max_iters));
                CK(p, launch_pcg_split(p));
            } else {
                CK(p, launch_pcg_init(p, p->sv.pv[1], inner, max_iters));
                CK(p, implicit_cg(p) ? launch_pcg_implicit(p) : launch_pcg_loop(p));
            }
            CK(p, split ? launch_accumulate_split(p, first) : launch_accumulate_solution(p, first));
            first = false;
            CK(p, launch_resid64(p, true));
            if ((s = sync_scalars(p))) return s;
            if (split && p->opt.profile >= 2) {
                for (int k = 0; k < 4; ++k) p->ph_sum[k] += p->sc_host->ph[k];
                // busiest CTA's work per iteration, over the mean CTA's (load balance)
                const double its = p->sc_host->iters > 0 ? p->sc_host->iters : 1;
                const double cta_its = p->sc_host->ph[3] > 0 ? p->sc_host->ph[3] : 1;
                const double mean_work = (p->sc_host->ph[0] + p->sc_host->ph[1]) / cta_its;
                p->ph_imbalance = mean_work > 0 ? (double)p->sc_host->ph_work_max / its / mean_work : 0.0;
            }
            if (p->sc_host->err == BA_ERR_TIMEOUT) {
                p->dead = true;
                return fail(BA_ERR_TIMEOUT, "PCG grid wait timed out");
            }
            if ((s = check_err_flag(p))) return s;
            total += p->sc_host->iters;
            ++refine;
        }
        if (!converged) converged = p->sc_host->rr64 <= tol * tol * p->sc_host->bb64;
        CK(p, launch_solution_to_step(p));
    }
    if (!p->sv.f32) {
        CK(p, launch_solution_to_step(p));
        if ((s = sync_scalars(p))) return s;
    }
    const double bb = p->sc_host->bb64;
    p->last_true_rel = bb > 0 ? std::sqrt(p->sc_host->rr64 / bb) : 0.0;
    // a learned M^-1 is judged by the true residual, not PCG's recurrence
    if (p->net && !p->sv.f32 && p->last_true_rel > 10.0 * tol) converged = false;
    p->last_pcg_iters = total;
    p->last_refine = refine;
    p->solved = true;
    p->backsub = false;
    if (info) {
        info->pcg_iters = total;
        info->refine_steps = refine;
        info->rcs_rel_resid = p->last_true_rel;
    }
    if (!converged) return fail(BA_ERR_NO_CONVERGENCE, "PCG reached its iteration cap");
    return BA_OK;
}

ba_status ba_solve_rcs(ba_problem *p, ba_step_info *info) {
    LIVE(p);
    if (!p->rcs_formed) return fail(BA_ERR_STATE, "ba_solve_rcs needs ba_form_rcs first");
    ba_step_info loc;
    std::memset(&loc, 0, sizeof(loc));
    ba_status s;
    p->last_used_fallback = 0;
    if (p->net) {
        if ((s = gnn_apply(p))) return s;
        s = solve_once(p, &loc);
        if (s == BA_ERR_NOT_SPD || s == BA_ERR_NO_CONVERGENCE) {
            // the learned M^-1 failed: plain block-Jacobi PCG
            if ((s = gnn_restore_block_jacobi(p))) return s;
            const int it = loc.pcg_iters;
            s = solve_once(p, &loc);
            loc.pcg_iters += it;
            p->last_used_fallback = 1;
        }
    } else {
        s = solve_once(p, &loc);
    }
    loc.used_fallback = p->last_used_fallback;
    if (info) {
        info->pcg_iters = loc.pcg_iters;
        info->refine_steps = loc.refine_steps;
        info->rcs_rel_resid = loc.rcs_rel_resid;
        info->used_fallback = loc.used_fallback;
    }
    return s;
}

ba_status ba_back_substitute(ba_problem *p) {
    LIVE(p);
    if (p->rcs_only) return fail(BA_ERR_STATE, "ba_back_substitute: the problem holds an RCS only");
    if (!p->solved) return fail(BA_ERR_STATE, "ba_back_substitute needs ba_solve_rcs first");
    CK(p, launch_back_substitute(p));
    p->backsub = true;
    return BA_OK;
}

ba_status ba_lm_step(ba_problem *p, ba_step_info *info) {
    LIVE(p);
    if (p->rcs_only) return fail(BA_ERR_STATE, "ba_lm_step: the problem holds an RCS only");
    ba_step_info loc;
    std::memset(&loc, 0, sizeof(loc));
    if (!p->step_ev[0])
        for (auto &x : p->step_ev) CK(p, cudaEventCreate(&x));
    cudaEvent_t *ev = p->step_ev;
    ba_status s;
    CK(p, cudaEventRecord(ev[0], p->st));
    if ((s = ensure_cost(p))) return s;
    loc.cost_before = p->F;
    if (!p->linearized) CK(p, launch_linearize(p));
    p->linearized = true;
    CK(p, cudaEventRecord(ev[1], p->st));
    CK(p, launch_form_rcs(p, p->lambda));
    p->minv_learned = false;
    p->rcs_formed = true;
    ++p->rcs_gen;
    p->rcs_lambda = p->lambda;
    CK(p, cudaEventRecord(ev[2], p->st));
    s = ba_solve_rcs(p, &loc);
    if (s != BA_OK && s != BA_ERR_NO_CONVERGENCE) return s;
    CK(p, cudaEventRecord(ev[3], p->st));
    CK(p, launch_trial_cameras(p));
    CK(p, cudaEventRecord(ev[4], p->st));
    // FP32 mode: while accepted steps still change F by 1e-3 of it or more, the
    // trial cost is evaluated whole (double-float residuals); after that, as
    // F(x) plus its change formed from the step, accurate relative to the
    // change itself (the gain ratio compares changes of 1e-7 of F and less)
    p->step_diff = p->fp32 && p->last_rel_decrease < 1e-3;
    CK(p, launch_step_points(p));  // Eq. 5 + trial point + trial cost and model, one pass
    p->backsub = true;
    CK(p, cudaEventRecord(ev[5], p->st));
    if ((s = sync_scalars(p))) return s;
    if ((s = check_err_flag(p))) return s;
    const double F1 = p->step_diff ? p->F + p->sc_host->cost_trial : p->sc_host->cost_trial;
    const double pred = p->sc_host->model;
    const double rho = pred > 0 ? (p->F - F1) / pred : -INFINITY;
    const bool ok = pred > 0 && std::isfinite(F1) && rho > 1e-3;
    loc.cost_trial = F1;
    loc.predicted = pred;
    loc.rho = rho;
    loc.lambda = p->lambda;
    loc.accepted = ok ? 1 : 0;
    loc.n_cheirality = (int64_t)p->sc_host->n_cheir_trial;
    loc.n_v_fp64 = (int64_t)p->sc_host->n_v64;
    if (ok) {
        std::swap(p->cur, p->trial);
        p->last_rel_decrease = (p->F - F1) / p->F;
        p->F = F1;
        const double f = 1.0 - std::pow(2.0 * rho - 1.0, 3);
        p->lambda *= std::max(1.0 / 3.0, f);
        p->nu = 2.0;
        p->linearized = false;
        p->rcs_formed = p->solved = p->backsub = false;
    } else {
        p->lambda *= p->nu;
        p->nu *= 2.0;
    }
    loc.cost_after = p->F;
    float t;
    for (int k = 0; k < 5; ++k) {
        cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
        loc.ms[k] = t;
    }
    cudaEventElapsedTime(&t, ev[0], ev[5]);
    loc.ms[5] = t;
    if (info) *info = loc;
    return BA_OK;
}

ba_status ba_get_cameras(const ba_problem *p, double *out) {
    LIVE(p);
    if (!out) return fail(BA_ERR_INVALID_ARG, "null output");
    ba_problem *q = const_cast<ba_problem *>(p);
    CK(q, cudaMemcpyAsync(out, p->cur.cams, p->n * 6 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CK(q, cudaStreamSynchronize(p->st));
    return BA_OK;
}

// Staging buffer and permutation for caller-order point I/O (first use).
static ba_status ensure_point_io(ba_problem *p) {
    if (p->stage_pts) return BA_OK;
    std::vector<int32_t> perm(p->P);
    for (int64_t k = 0; k < p->P; ++k) perm[k] = (int32_t)p->hs.pt_perm[k];
    void *a = nullptr, *b = nullptr, *c = nullptr;
    CK(p, dalloc_raw(p, &a, (size_t)p->P * sizeof(int32_t)));
    CK(p, dalloc_raw(p, &b, (size_t)p->P * 3 * sizeof(double)));
    CK(p, dalloc_raw(p, &c, 256));
    CK(p, cudaMemcpyAsync(a, perm.data(), (size_t)p->P * sizeof(int32_t), cudaMemcpyHostToDevice, p->st));
    CK(p, cudaStreamSynchronize(p->st));
    p->d_perm = (int32_t *)a;
    p->io_flag = (unsigned *)c;
    p->stage_pts = (double *)b;
    return BA_OK;
}

// P x 3 internal-order values (FP64 or FP32) to the caller's order in out
static ba_status fetch_points(ba_problem *p, const void *internal, bool fp32, double *out) {
    ba_status s;
    if ((s = ensure_point_io(p))) return s;
    CK(p, launch_scatter_pts(p, internal, fp32, p->stage_pts));
    CK(p, cudaMemcpyAsync(out, p->stage_pts, p->P * 3 * sizeof(double), cudaMemcpyDeviceToHost, p->st));
    CK(p, cudaStreamSynchronize(p->st));
    return BA_OK;
}

ba_status ba_get_points(const ba_problem *p, double *out) {
    LIVE(p);
    if (!out) return fail(BA_ERR_INVALID_ARG, "null output");
    return fetch_points(const_cast<ba_problem *>(p), p->cur.pts, false, out);
}

ba_status ba_get_rcs(const ba_problem *p, int64_t *nnzb, int32_t *row_ptr, int32_t *col, double *val, double *b) {
    LIVE(p);
    ba_problem *q = const_cast<ba_problem *>(p);
    if (nnzb) *nnzb = p->nnzb;
    if (row_ptr) std::memcpy(row_ptr, p->hs.row_ptr.data(), (p->n + 1) * sizeof(int32_t));
    if (col) std::memcpy(col, p->hs.col.data(), p->nnzb * sizeof(int32_t));
    if ((val || b) && !p->rcs_formed) return fail(BA_ERR_STATE, "no RCS formed yet");
    std::vector<double> tmp;
    ba_status s;
    if (val) {
        if ((s = fetch(q, p->S, p->nnzb * BW, tmp))) return s;
        std::memcpy(val, tmp.data(), tmp.size() * 8);
    }
    if (b) {
        if ((s = fetch(q, p->b, p->n * 6, tmp))) return s;
        std::memcpy(b, tmp.data(), tmp.size() * 8);
    }
    return BA_OK;
}

ba_status ba_rcs_spmv(ba_problem *p, int32_t format, const void *x, void *y, int64_t *bytes_out) {
    LIVE(p);
    if (format < BA_FMT_BSMC || format > BA_FMT_BSMC_ONCE) return fail(BA_ERR_INVALID_ARG, "unknown RCS format");
    if (format == BA_FMT_IMPLICIT && p->rcs_only)
        return fail(BA_ERR_STATE, "the implicit product needs the linearization (not an RCS-only problem)");
    if (!x || !y) return fail(BA_ERR_INVALID_ARG, "null vector");
    if (!p->rcs_formed) return fail(BA_ERR_STATE, "no RCS formed yet");
    if (format == BA_FMT_CSR && (2 * p->nnzb - p->n) * (int64_t)BW >= (int64_t)INT32_MAX)
        return fail(BA_ERR_INVALID_ARG, "scalar CSR of this RCS needs 64-bit row starts");
    if (format != BA_FMT_BSMC && format != BA_FMT_BSMC_ONCE) {
        const cudaError_t e = launch_rcs_format_build(p, format);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(BA_ERR_OOM, "ba_rcs_spmv: no device memory for the format's arrays");
        }
        CK(p, e);
    }
    CK(p, launch_rcs_spmv(p, format, x, y));
    if (bytes_out) *bytes_out = rcs_format_bytes(p, format);
    return BA_OK;
}

ba_status ba_triangulate(ba_problem *p, int32_t gn_iters, int64_t *n_failed_out, double *cost_out) {
    LIVE(p);
    if (p->rcs_only) return fail(BA_ERR_STATE, "ba_triangulate: the problem holds an RCS only");
    if (gn_iters < 0 || gn_iters > 50) return fail(BA_ERR_INVALID_ARG, "gn_iters must be in [0, 50]");
    CK(p, launch_triangulate(p, gn_iters));
    CK(p, launch_prepare_state(p, p->cur));
    p->have_F = false;
    p->linearized = p->rcs_formed = p->solved = p->backsub = false;
    ba_status s = sync_scalars(p);
    if (s) return s;
    if (n_failed_out) *n_failed_out = (int64_t)p->sc_host->n_tri_fail;
    if (cost_out) {
        if ((s = ensure_cost(p))) return s;
        *cost_out = p->F;
    }
    return BA_OK;
}

ba_status ba_get_step(const ba_problem *p, double *dxc, double *dxp) {
    LIVE(p);
    ba_problem *q = const_cast<ba_problem *>(p);
    std::vector<double> tmp;
    ba_status s;
    if (dxc) {
        if ((s = fetch(q, p->dxc, p->n * 6, tmp))) return s;
        std::memcpy(dxc, tmp.data(), tmp.size() * 8);
    }
    if (dxp && (s = fetch_points(q, p->dxp, p->fp32, dxp))) return s;
    return BA_OK;
}

ba_status ba_get_linearization(const ba_problem *p, double *e, double *Jc, double *Jp) {
    LIVE(p);
    if (!p->linearized) return fail(BA_ERR_STATE, "not linearized");
    ba_problem *q = const_cast<ba_problem *>(p);
    std::vector<double> tmp;
    ba_status s;
    if ((s = fetch(q, p->J, p->m * JW, tmp))) return s;
    for (int64_t a = 0; a < p->m; ++a) {
        const int64_t u = p->hs.obs_perm[a];
        const double *r = tmp.data() + a * JW;
        if (Jc) std::memcpy(Jc + 12 * u, r, 12 * 8);
        if (Jp) std::memcpy(Jp + 6 * u, r + 12, 6 * 8);
        if (e) { e[2 * u] = r[18]; e[2 * u + 1] = r[19]; }
    }
    return BA_OK;
}

ba_status ba_set_state(ba_problem *p, const double *cams, const double *pts, double lambda, double nu) {
    LIVE(p);
    if (!(lambda >= 0) || !(nu > 0) || !std::isfinite(lambda) || !std::isfinite(nu))
        return fail(BA_ERR_INVALID_ARG, "bad lambda / nu");
    if (cams) {
        if (!finite_all(cams, p->n * 6)) return fail(BA_ERR_NONFINITE, "non-finite camera");
        CK(p, cudaMemcpyAsync(p->cur.cams, cams, p->n * 6 * 8, cudaMemcpyHostToDevice, p->st));
    }
    if (pts) {
        // caller's order to the staging buffer, checked there; the state
        // changes only when every value is finite
        ba_status s;
        if ((s = ensure_point_io(p))) return s;
        CK(p, cudaMemcpyAsync(p->stage_pts, pts, p->P * 3 * 8, cudaMemcpyHostToDevice, p->st));
        CK(p, cudaMemsetAsync(p->io_flag, 0, sizeof(unsigned), p->st));
        CK(p, launch_count_nonfinite(p, p->stage_pts, p->P * 3, p->io_flag));
        unsigned bad = 0;
        CK(p, cudaMemcpyAsync(&bad, p->io_flag, sizeof(unsigned), cudaMemcpyDeviceToHost, p->st));
        CK(p, cudaStreamSynchronize(p->st));
        if (bad) return fail(BA_ERR_NONFINITE, "non-finite point");
        CK(p, launch_gather_pts(p, p->stage_pts, p->cur.pts));
    }
    CK(p, launch_prepare_state(p, p->cur));
    p->lambda = lambda;
    p->nu = nu;
    p->have_F = false;
    p->linearized = p->rcs_formed = p->solved = p->backsub = false;
    return BA_OK;
}

ba_status ba_get_lm_state(const ba_problem *p, double *lambda, double *nu, double *cost) {
    LIVE(p);
    if (lambda) *lambda = p->lambda;
    if (nu) *nu = p->nu;
    if (cost) {
        ba_problem *q = const_cast<ba_problem *>(p);
        ba_status s = ensure_cost(q);
        if (s) return s;
        *cost = p->F;
    }
    return BA_OK;
}

ba_status ba_get_stats(const ba_problem *p, ba_stats *o) {
    LIVE(p);
    if (!o) return fail(BA_ERR_INVALID_ARG, "null output");
    {  // the device-side counters and phase totals
        ba_status s = sync_scalars(const_cast<ba_problem *>(p));
        if (s) return s;
    }
    o->n_cams = p->n;
    o->n_pts = p->P;
    o->n_obs = p->m;
    o->nnzb = p->nnzb;
    o->n_groups = p->ngroups;
    o->n_partials = p->npart;
    o->n_pairs = p->hs.n_pairs;
    o->device_bytes = (int64_t)p->dev_bytes;
    o->kernel_launches = p->launches;
    o->precision = p->opt.precision;
    for (int k = 0; k < 3; ++k) o->pcg_phase_us[k] = p->ph_sum[3] > 0 ? p->ph_sum[k] / p->ph_sum[3] / 1e3 : 0.0;
    for (int k = 0; k < 3; ++k)
        o->rcs_phase_us[k] = p->sc_host->ph_rcs[3] > 0 ? p->sc_host->ph_rcs[k] / p->sc_host->ph_rcs[3] / 1e3 : 0.0;
    o->pcg_work_imbalance = p->ph_imbalance;
    o->n_v_fp64 = p->rcs_only ? 0 : (int64_t)p->sc_host->n_v64;
    return BA_OK;
}

ba_status ba_debug_arm_wait_timeout(ba_problem *p, int64_t limit_cycles) {
    LIVE(p);
    if (limit_cycles <= 0 || limit_cycles > 4000000000LL)
        return fail(BA_ERR_INVALID_ARG, "ba_debug_arm_wait_timeout: limit_cycles must be in (0, 4e9]");
    p->test_wait_limit = limit_cycles;
    return BA_OK;
}

ba_status ba_get_kernel_time(ba_problem *p, int32_t k, int64_t *launches, double *total_ms) {
    LIVE(p);
    if (k < 0 || k >= K_COUNT) return fail(BA_ERR_INVALID_ARG, "kernel id out of range");
    ba_status s = ktimer_flush(p);
    if (s) return s;
    if (launches) *launches = p->klaunch[k];
    if (total_ms) *total_ms = p->kms[k];
    return BA_OK;
}

ba_status ba_reset_kernel_times(ba_problem *p) {
    LIVE(p);
    ba_status s = ktimer_flush(p);
    if (s) return s;
    for (int k = 0; k < K_COUNT; ++k) { p->klaunch[k] = 0; p->kms[k] = 0; }
    return BA_OK;
}

ba_status ba_set_profile(ba_problem *p, int32_t level) {
    LIVE(p);
    if (level < 0 || level > 2) return fail(BA_ERR_INVALID_ARG, "profile level must be 0, 1 or 2");
    ba_status s = ktimer_flush(p);  // collect the events of launches timed so far
    if (s) return s;
    p->opt.profile = level;
    return BA_OK;
}

}  // extern "C"
