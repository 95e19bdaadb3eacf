// Host-side symbolic phase of libba (runs once per problem, no GPU needed).
//
// * validation of the observation set;
// * a spatial (Morton) order of the points so that a run of points touches a
//   compact set of cameras (the paper groups points "naively" with equal
//   counts, Sec. 6.1; a spatial order makes each group's sub-RCS small);
// * observations sorted by (point, camera): the track CSR;
// * the BSMC pattern: every diagonal block plus each (i < j) whose cameras
//   share a point, rows in order, columns ascending, diagonal first (Sec. 4,
//   Fig. 4);
// * point groups (one CTA each) with their local sub-RCS blocks; each local
//   block gets its global block id by a binary search in row i of the BSMC
//   column ids (the "second operation" of Table 1, cost log2 s_i);
// * the per-global-block list of partials for the segmented reduction that
//   sums the sub-RCSs into the global RCS (Sec. 6.1 aggregation).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "ba_internal.h"

namespace ba {

static uint64_t spread3(uint64_t v) {
    // spread the low 21 bits of v so that bit k moves to bit 3k
    v &= 0x1fffffULL;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}

static void morton_order(int64_t P, const double *pts, std::vector<int64_t> &perm) {
    perm.resize(P);
    std::iota(perm.begin(), perm.end(), 0);
    if (!pts) return;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t k = 0; k < P; ++k)
        for (int d = 0; d < 3; ++d) {
            lo[d] = std::min(lo[d], pts[3 * k + d]);
            hi[d] = std::max(hi[d], pts[3 * k + d]);
        }
    // one scale for all axes: a flat scene keeps its thin axis in the low bits
    double ext = std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2], 1e-30});
    const double q = double((1 << 21) - 1) / ext;
    std::vector<std::pair<uint64_t, int64_t>> key(P);
    for (int64_t k = 0; k < P; ++k) {
        uint64_t c = 0;
        for (int d = 0; d < 3; ++d) {
            double t = (pts[3 * k + d] - lo[d]) * q;
            uint64_t u = (uint64_t)std::min(std::max(t, 0.0), double((1 << 21) - 1));
            c |= spread3(u) << d;
        }
        key[k] = {c, k};
    }
    std::sort(key.begin(), key.end());
    for (int64_t k = 0; k < P; ++k) perm[k] = key[k].second;
}

static int32_t find_block(const std::vector<int32_t> &row_ptr, const std::vector<int32_t> &col,
                          int32_t i, int32_t j) {
    // Table 1, second operation: binary search of column j in BSMC row i
    auto b = col.begin() + row_ptr[i], e = col.begin() + row_ptr[i + 1];
    auto it = std::lower_bound(b, e, j);
    if (it == e || *it != j) return -1;
    return (int32_t)(it - col.begin());
}

void build_twosided(HostSetup &hs, int32_t n) {
    // column index of the upper triangle: for every column i the off-diagonal
    //      blocks (j, i), j < i, in row order (the SpMV applies them transposed)
    hs.ct_ptr.assign(n + 1, 0);
    for (int32_t j = 0; j < n; ++j)
        for (int32_t b = hs.row_ptr[j] + 1; b < hs.row_ptr[j + 1]; ++b) hs.ct_ptr[hs.col[b] + 1]++;
    for (int32_t i = 0; i < n; ++i) hs.ct_ptr[i + 1] += hs.ct_ptr[i];
    hs.ct_blk.assign(hs.ct_ptr[n], 0);
    hs.ct_row.assign(hs.ct_ptr[n], 0);
    {
        std::vector<int32_t> fill(hs.ct_ptr.begin(), hs.ct_ptr.end() - 1);
        for (int32_t j = 0; j < n; ++j)
            for (int32_t b = hs.row_ptr[j] + 1; b < hs.row_ptr[j + 1]; ++b) {
                const int32_t at = fill[hs.col[b]]++;
                hs.ct_blk[at] = b;
                hs.ct_row[at] = j;
            }
    }
    // two-sided SpMV entries of row i: (i, j >= i) as stored, then (j < i, i) transposed
    hs.tw_ptr.assign(n + 1, 0);
    hs.tw_ent.clear();
    hs.tw_ent.reserve(2 * hs.col.size());
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t b = hs.row_ptr[i]; b < hs.row_ptr[i + 1]; ++b) hs.tw_ent.push_back(make_int2(b, hs.col[b]));
        for (int32_t q = hs.ct_ptr[i]; q < hs.ct_ptr[i + 1]; ++q)
            hs.tw_ent.push_back(make_int2((int32_t)((uint32_t)hs.ct_blk[q] | 0x80000000u), hs.ct_row[q]));
        hs.tw_ptr[i + 1] = (int32_t)hs.tw_ent.size();
    }

}

// A work item of the RCS formation: products [cbeg, cbeg + cnt) of the
// group's product list, all of local block blk (ordinal in the group's order).
struct WorkItem {
    int32_t blk, cbeg, cnt;
};

// Orders the products inside each work item for the shared-memory banks.
// The product loop of the RCS formation reads, per product, the a- and
// b-rows of two observations with 16-byte loads; rows are 80 bytes apart,
// so row r starts in 16-byte bank group (5 r) mod 8, and one such load of a
// quarter-warp (items 8m .. 8m + 7 of a group, one per lane) costs as many
// wavefronts as the largest number of distinct rows sharing a bank group.
// The order of a work item's products is free (they are summed), so at each
// step every lane takes, from its remaining products, the one that adds the
// fewest same-group rows to the step's a- and b-loads (diagonal items load
// only the a-row).  Deterministic: ties keep the stored (point) order.
void order_items_for_banks(uint32_t *cl, const WorkItem *its, int32_t nit, const std::vector<char> &is_diag,
                           const std::vector<int32_t> &ord) {
    std::vector<uint32_t> rem[8];
    int32_t rowsA[8][8], nA[8], rowsB[8][8], nB[8];
    auto seen = [](const int32_t *rows, int32_t n, int32_t r) {
        for (int32_t q = 0; q < n; ++q)
            if (rows[q] == r) return true;
        return false;
    };
    for (int32_t m0 = 0; m0 < nit; m0 += 8) {
        const int32_t m1 = std::min(nit, m0 + 8);
        int32_t T = 0;
        for (int32_t t = m0; t < m1; ++t) {
            rem[t - m0].assign(cl + its[t].cbeg, cl + its[t].cbeg + its[t].cnt);
            T = std::max(T, its[t].cnt);
        }
        for (int32_t step = 0; step < T; ++step) {
            std::fill(nA, nA + 8, 0);
            std::fill(nB, nB + 8, 0);
            for (int32_t t = m0; t < m1; ++t) {
                std::vector<uint32_t> &rl = rem[t - m0];
                if (rl.empty()) continue;
                const bool dg = is_diag[ord[its[t].blk]] != 0;
                size_t best = 0;
                int32_t best_cost = INT32_MAX;
                for (size_t q = 0; q < rl.size() && best_cost > 0; ++q) {
                    const int32_t ra = (int32_t)(rl[q] & 0xffffu), rb = (int32_t)(rl[q] >> 16);
                    const int32_t ca = (5 * ra) & 7, cb = (5 * rb) & 7;
                    int32_t cost = seen(rowsA[ca], nA[ca], ra) ? 0 : nA[ca];
                    if (!dg) cost += seen(rowsB[cb], nB[cb], rb) ? 0 : nB[cb];
                    if (cost < best_cost) {
                        best_cost = cost;
                        best = q;
                    }
                }
                const uint32_t u = rl[best];
                rl.erase(rl.begin() + (std::ptrdiff_t)best);
                cl[its[t].cbeg + step] = u;
                const int32_t ra = (int32_t)(u & 0xffffu), rb = (int32_t)(u >> 16);
                const int32_t ca = (5 * ra) & 7, cb = (5 * rb) & 7;
                if (!seen(rowsA[ca], nA[ca], ra)) rowsA[ca][nA[ca]++] = ra;
                if (!dg && !seen(rowsB[cb], nB[cb], rb)) rowsB[cb][nB[cb]++] = rb;
            }
        }
    }
}

ba_status symbolic_setup(int32_t n, int64_t P, int64_t m, const int32_t *obs_cam,
                         const int64_t *obs_pt, const double *pts, int obs_max, bool pattern_only,
                         HostSetup &hs, std::string &err) {
    if (n <= 0 || P <= 0 || m <= 0) { err = "n_cams, n_pts and n_obs must be positive"; return BA_ERR_INVALID_ARG; }
    if (m >= (int64_t)INT32_MAX || P >= (int64_t)INT32_MAX) { err = "n_obs and n_pts must be < 2^31"; return BA_ERR_INVALID_ARG; }
    if (!obs_cam || !obs_pt) { err = "null observation index array"; return BA_ERR_INVALID_ARG; }
    for (int64_t a = 0; a < m; ++a) {
        if (obs_cam[a] < 0 || obs_cam[a] >= n) { err = "obs_cam[" + std::to_string(a) + "] out of range"; return BA_ERR_INVALID_ARG; }
        if (obs_pt[a] < 0 || obs_pt[a] >= P) { err = "obs_pt[" + std::to_string(a) + "] out of range"; return BA_ERR_INVALID_ARG; }
    }
    // ---- point order and its inverse
    morton_order(P, pattern_only ? nullptr : pts, hs.pt_perm);
    std::vector<int32_t> pt_inv(P);
    for (int64_t k = 0; k < P; ++k) pt_inv[hs.pt_perm[k]] = (int32_t)k;

    // ---- track CSR: counting sort by internal point, then by camera in each track
    hs.trk_ptr.assign(P + 1, 0);
    for (int64_t a = 0; a < m; ++a) hs.trk_ptr[pt_inv[obs_pt[a]] + 1]++;
    for (int64_t k = 0; k < P; ++k) {
        if (hs.trk_ptr[k + 1] < 2) {
            err = "point " + std::to_string(hs.pt_perm[k]) + " has fewer than two observations";
            return BA_ERR_INVALID_ARG;
        }
        hs.trk_ptr[k + 1] += hs.trk_ptr[k];
    }
    hs.obs_perm.assign(m, 0);
    {
        std::vector<int32_t> fill(hs.trk_ptr.begin(), hs.trk_ptr.end() - 1);
        for (int64_t a = 0; a < m; ++a) hs.obs_perm[fill[pt_inv[obs_pt[a]]]++] = a;
    }
    hs.obs_cam.resize(m);
    hs.obs_pt.resize(m);
    for (int64_t k = 0; k < P; ++k) {
        int64_t b = hs.trk_ptr[k], e = hs.trk_ptr[k + 1];
        std::sort(hs.obs_perm.begin() + b, hs.obs_perm.begin() + e,
                  [&](int64_t x, int64_t y) { return obs_cam[x] < obs_cam[y] || (obs_cam[x] == obs_cam[y] && x < y); });
        for (int64_t a = b; a < e; ++a) {
            hs.obs_cam[a] = obs_cam[hs.obs_perm[a]];
            hs.obs_pt[a] = (int32_t)k;
            if (a > b && hs.obs_cam[a] == hs.obs_cam[a - 1]) {
                err = "duplicate observation of point " + std::to_string(hs.pt_perm[k]) + " by camera " +
                      std::to_string(hs.obs_cam[a]);
                return BA_ERR_INVALID_ARG;
            }
        }
    }
    // ---- camera -> observations
    std::vector<int64_t> cam_ptr(n + 1, 0);
    for (int64_t a = 0; a < m; ++a) cam_ptr[hs.obs_cam[a] + 1]++;
    for (int32_t i = 0; i < n; ++i) {
        if (cam_ptr[i + 1] == 0) { err = "camera " + std::to_string(i) + " has no observation"; return BA_ERR_INVALID_ARG; }
        cam_ptr[i + 1] += cam_ptr[i];
    }
    std::vector<int32_t> cam_obs(m);
    {
        std::vector<int64_t> fill(cam_ptr.begin(), cam_ptr.end() - 1);
        for (int64_t a = 0; a < m; ++a) cam_obs[fill[hs.obs_cam[a]]++] = (int32_t)a;
    }
    // ---- BSMC pattern (Sec. 4): row i = {i} U {j > i sharing a point with i}
    hs.row_ptr.assign(n + 1, 0);
    hs.col.clear();
    {
        std::vector<int32_t> stamp(n, -1), row;
        for (int32_t i = 0; i < n; ++i) {
            row.clear();
            for (int64_t q = cam_ptr[i]; q < cam_ptr[i + 1]; ++q) {
                int32_t k = hs.obs_pt[cam_obs[q]];
                for (int32_t bb = hs.trk_ptr[k]; bb < hs.trk_ptr[k + 1]; ++bb) {
                    int32_t j = hs.obs_cam[bb];
                    if (j > i && stamp[j] != i) { stamp[j] = i; row.push_back(j); }
                }
            }
            std::sort(row.begin(), row.end());
            hs.col.push_back(i);
            hs.col.insert(hs.col.end(), row.begin(), row.end());
            if (hs.col.size() >= (size_t)INT32_MAX) { err = "more than 2^31 BSMC blocks"; return BA_ERR_INVALID_ARG; }
            hs.row_ptr[i + 1] = (int32_t)hs.col.size();
        }
    }
    if (pattern_only) return BA_OK;

    build_twosided(hs, n);

    // ---- point groups with their sub-RCS blocks (Sec. 6.1)
    const int64_t nnzb = (int64_t)hs.col.size();
    std::vector<int32_t> lb_stamp(nnzb, -1), lb_local(nnzb, 0);
    std::vector<int32_t> g_gblk;                    // local block -> global block (current group)
    std::vector<std::pair<int32_t, uint32_t>> g_c;  // (local block, a | b << 16)
    std::vector<int32_t> trk_g;                     // global ids of the current track's pairs
    hs.groups.clear();
    hs.items.clear();
    hs.lb_gblk.clear();
    hs.contrib.clear();
    hs.n_pairs = 0;
    hs.max_nobs = 0;
    hs.max_nc = 0;
    GroupDesc g{};
    int32_t gid = 0;
    auto close_group = [&]() {
        if (g.npts == 0) return;
        const int32_t nlb = (int32_t)g_gblk.size();
        std::vector<int32_t> cnt(nlb, 0);
        std::vector<char> is_diag(nlb, 0);
        for (auto &c : g_c) cnt[c.first]++;
        for (int32_t b = 0; b < nlb; ++b) {
            // a block is diagonal iff it is the first block of its row
            auto it = std::upper_bound(hs.row_ptr.begin(), hs.row_ptr.end(), g_gblk[b]);
            is_diag[b] = hs.row_ptr[(it - hs.row_ptr.begin()) - 1] == g_gblk[b];
        }
        // diagonal blocks first (one code path per warp), then by product count
        // (descending) so that full items share warps; ties by global id
        std::vector<int32_t> ord(nlb);
        std::iota(ord.begin(), ord.end(), 0);
        std::sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) {
            if (is_diag[x] != is_diag[y]) return is_diag[x] > is_diag[y];
            if (cnt[x] != cnt[y]) return cnt[x] > cnt[y];
            return g_gblk[x] < g_gblk[y];
        });
        std::vector<int32_t> pos(nlb), start(nlb + 1, 0);
        for (int32_t r = 0; r < nlb; ++r) pos[ord[r]] = r;
        for (int32_t r = 0; r < nlb; ++r) start[r + 1] = start[r] + cnt[ord[r]];
        g.c_begin = (int64_t)hs.contrib.size();
        g.part_begin = (int64_t)hs.lb_gblk.size();
        g.item_begin = (int64_t)hs.items.size();
        g.nc = (int32_t)g_c.size();
        // each group's list starts on a 16-byte boundary and spans a multiple of 16 bytes (bulk copies)
        hs.contrib.resize(hs.contrib.size() + ((g_c.size() + 3) & ~(size_t)3), 0u);
        std::vector<int32_t> fill(start.begin(), start.end() - 1);
        for (auto &c : g_c) hs.contrib[g.c_begin + fill[pos[c.first]]++] = c.second;  // stable: point order
        // work items of <= ITEM_MAX products, sizes balanced within a block
        std::vector<WorkItem> its;
        for (int32_t r = 0; r < nlb; ++r) {
            const int32_t c = cnt[ord[r]];
            const int32_t k = (c + ITEM_MAX - 1) / ITEM_MAX;
            int32_t off = start[r];
            for (int32_t q = 0; q < k; ++q) {
                const int32_t sz = c / k + (q < c % k ? 1 : 0);
                its.push_back({r, off, sz});
                off += sz;
            }
        }
        const int32_t nit = (int32_t)its.size();
        order_items_for_banks(hs.contrib.data() + g.c_begin, its.data(), nit, is_diag, ord);
        // runs: consecutive items of one block inside one warp of 32
        int32_t npart = 0;
        for (int32_t q = 0; q < nit;) {
            int32_t e = q + 1;
            while (e < nit && its[e].blk == its[q].blk && (e / 32) == (q / 32)) ++e;
            for (int32_t t = q; t < e; ++t) {
                ItemDesc d;
                const bool dg = is_diag[ord[its[t].blk]];
                d.x = (uint32_t)its[t].cbeg | ((uint32_t)its[t].cnt << 16) | ((uint32_t)dg << 20) |
                      ((uint32_t)(e - 1 - t) << 21) | ((uint32_t)(t == q) << 26);
                d.y = (t == q) ? (uint32_t)npart : 0u;
                hs.items.push_back(d);
            }
            hs.lb_gblk.push_back(g_gblk[ord[its[q].blk]]);
            ++npart;
            q = e;
        }
        g.nitems = nit;
        hs.max_nobs = std::max(hs.max_nobs, g.nobs);
        hs.max_nc = std::max(hs.max_nc, g.nc);
        hs.groups.push_back(g);
        g_gblk.clear();
        g_c.clear();
        ++gid;
        g = GroupDesc{};
    };
    for (int64_t k = 0; k < P; ++k) {
        const int32_t tb = hs.trk_ptr[k], L = hs.trk_ptr[k + 1] - tb;
        const int32_t npair = L * (L + 1) / 2;
        trk_g.clear();
        int32_t fresh = 0;
        for (int32_t x = 0; x < L; ++x)
            for (int32_t y = x; y < L; ++y) {
                int32_t gb = find_block(hs.row_ptr, hs.col, hs.obs_cam[tb + x], hs.obs_cam[tb + y]);
                if (gb < 0) { err = "internal: pair missing from the BSMC pattern"; return BA_ERR_INTERNAL; }
                trk_g.push_back(gb);
                if (lb_stamp[gb] != gid) ++fresh;  // may count a repeated block twice; conservative
            }
        if (L > obs_max || npair > C_MAX || npair > LB_MAX) {
            err = "point " + std::to_string(hs.pt_perm[k]) + " has a track of " + std::to_string(L) +
                  " observations; the limit is " + std::to_string(std::min(obs_max, 90));
            return BA_ERR_INVALID_ARG;
        }
        if (g.npts > 0 && (g.nobs + L > obs_max || g.nc + npair > C_MAX || (int32_t)g_gblk.size() + fresh > LB_MAX))
            close_group();
        if (g.npts == 0) { g.obs_begin = tb; g.pt_begin = (int32_t)k; }
        int32_t q = 0;
        for (int32_t x = 0; x < L; ++x)
            for (int32_t y = x; y < L; ++y, ++q) {
                int32_t gb = trk_g[q];
                if (lb_stamp[gb] != gid) {
                    lb_stamp[gb] = gid;
                    lb_local[gb] = (int32_t)g_gblk.size();
                    g_gblk.push_back(gb);
                }
                uint32_t a = (uint32_t)(tb + x - g.obs_begin), b = (uint32_t)(tb + y - g.obs_begin);
                g_c.push_back({lb_local[gb], a | (b << 16)});
            }
        g.nobs += L;
        g.nc += npair;
        g.npts += 1;
        hs.n_pairs += npair;
    }
    close_group();
    if (hs.lb_gblk.size() >= (size_t)INT32_MAX) { err = "more than 2^31 partial blocks"; return BA_ERR_INVALID_ARG; }
    // ---- partials of each global block (segmented-reduction CSR), in group order
    hs.pptr.assign(nnzb + 1, 0);
    for (int32_t gb : hs.lb_gblk) hs.pptr[gb + 1]++;
    for (int64_t b = 0; b < nnzb; ++b) {
        if (hs.pptr[b + 1] == 0) { err = "internal: BSMC block without partial"; return BA_ERR_INTERNAL; }
        hs.pptr[b + 1] += hs.pptr[b];
    }
    hs.plist.assign(hs.lb_gblk.size(), 0);
    {
        std::vector<int32_t> fill(hs.pptr.begin(), hs.pptr.end() - 1);
        for (size_t r = 0; r < hs.lb_gblk.size(); ++r) hs.plist[fill[hs.lb_gblk[r]]++] = (int32_t)r;
    }
    return BA_OK;
}

}  // namespace ba
