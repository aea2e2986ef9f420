// Host side of the tensor-core masked-ALS half-step (lt_als_tc.cu), for slices of
// rank up to RP = 8 or 16; lt_complete calls it when the tensor-core form is chosen.
#pragma once

#include <stdint.h>

#include "lt_internal.cuh"
#include "lt_omega.cuh"

namespace ltk {

// Device arrays of one lt_complete call (scratch SCR_TC_PLAN, SCR_TC_IMG).
struct TcPlan {
    int32_t* kbr;          // [S + 1] prefix of ceil(n'_s / 32): image blocks of the U-step sources
    int32_t* kbc;          // [S + 1] prefix of ceil(m'_s / 32): image blocks of the V-step sources
    int32_t* tr;           // [S + 1] prefix of ceil(m'_s / 256): U-step tiles
    int32_t* tcn;          // [S + 1] prefix of ceil(n'_s / 256): V-step tiles
    int32_t* amax;         // [S] largest |observed value| of each slice (float bits)
    int32_t* xmax;         // [steps][S] largest |source factor component| of each half-step (float bits)
    int32_t* ctr;          // [steps] tile counter of each half-step
    unsigned char* img;    // images, img_cap blocks of Tc<RP>::IMG bytes
    int64_t img_cap;
    uint32_t* vr;          // [E] observed values as two fp16 parts (scaled), CSR positions
    uint32_t* vc;          // [E] the same at CSC positions
    int32_t* status;       // device status word (LT_ELIMIT when the images exceed img_cap)
    int RP;
};

// The float64 retry queue (lines whose float32 pivots fail the check), CSR / CSC mode.
struct TcQueue {
    int32_t* count;
    int64_t* dst;
    int64_t* slot;
    int64_t* src;
    int32_t* len;
    int32_t* grp;
    int32_t* rank;
    int64_t cap;
    int32_t* status;
};

// Allocates the plan for `steps` half-steps and computes the per-slice prefixes, the
// value scales and the split values (om needs CSR / CSC).  E is the sample capacity.
lt_status als_tc_plan(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, int64_t E, int R,
                      const int32_t* rk, int RP, int steps, TcPlan* plan);

// One half-step: the rows of U (rows_side) or the columns of V from `fin` into `fout`,
// for the slices of rank <= plan.RP.  `gram` non-null: write each line's Gram (packed
// lower triangle, r(r+1)/2 values) and right-hand side (r values) there instead of
// solving (line index: the slice-ordered row, or s C + column; stride r(r+3)/2).
lt_status als_tc_half(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, int R,
                      const int32_t* rk, bool rows_side, const float* fin, float* fout, float lam_rel,
                      const TcPlan& plan, int step, const TcQueue& q, float* gram);

}  // namespace ltk
