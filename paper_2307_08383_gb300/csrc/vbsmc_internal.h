// Internal declarations of the variable-size BSMC (ba_vbsmc.h): the object
// and the steps shared by its two creation paths (given values, or formed on
// the device from a scene with interior parameters).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "ba_internal.h"
#include "ba_vbsmc.h"

namespace ba {

struct VbScalars {
    double rz, rr, rr0, tol2;
    int iters, done, max_iters, err;
};

}  // namespace ba

struct ba_vbsmc {
    int n = 0;
    int64_t nnzb = 0, N = 0, nval = 0, nminv = 0;
    bool fp32 = false, dead = false;
    size_t esz = 8, dev_bytes = 0, cap = 0;
    cudaStream_t st = nullptr;
    int *cdim = nullptr, *off = nullptr, *row_ptr = nullptr, *col = nullptr, *brow = nullptr, *ent_cam = nullptr,
        *tw_ptr = nullptr;
    int4 *tw_info = nullptr;
    int64_t *boff = nullptr, *moff = nullptr;
    void *val = nullptr, *Minv = nullptr, *b = nullptr, *vec[7] = {};
    ba::VbScalars *sc = nullptr;
    ba::VbScalars host{};
    double *red = nullptr;
    unsigned *bar = nullptr;
    int *err = nullptr;
    std::vector<void *> allocs;
    cudaEvent_t ev[2] = {nullptr, nullptr};
};

namespace ba {

// Validates precision, sizes and the upper-block pattern; sums c_i and the
// value count.
ba_status vb_check_pattern(const ba_options &o, int32_t n, const int32_t *cdim, int64_t nnzb, const int32_t *row_ptr,
                           const int32_t *col, int64_t *N_out, int64_t *nval_out);
// Checks the pattern, builds the layout (offsets, two-sided records) and
// allocates every device array; values and b are left for the caller.
ba_status vb_build(const ba_options &o, int32_t n, const int32_t *cdim, int64_t nnzb, const int32_t *row_ptr,
                   const int32_t *col, ba_vbsmc **out);
// Builds M^-1 from the diagonal blocks (BA_ERR_NOT_SPD if one is not).
ba_status vb_finish(ba_vbsmc *h);
ba_status vb_alloc(ba_vbsmc *h, void **d, size_t bytes);
ba_status vb_cuda(ba_vbsmc *h, cudaError_t e, const char *what);

}  // namespace ba
