// The observed entries of every slice in the layouts the completions read
// (built by omega_build, defined with the ALS).
#pragma once

#include "lt_internal.cuh"

namespace ltk {

// rank of slice s: rk[s] clamped to [1, R], or R when there are no per-slice ranks
__device__ __forceinline__ int slice_rank(const int32_t* __restrict__ rk, int s, int R) {
    return rk ? min(max(rk[s], 1), R) : R;
}

// frame arguments the completions accept (slice indices fit 16 bits)
inline bool frame_ok2(const lt_frame* f) {
    return f && f->slice_off && f->S > 0 && f->S <= 1024 && f->m > 0 && f->C >= 1 && f->max_rows >= 0 &&
           f->max_rows <= 65535;
}

struct Omega {
    int32_t* rp;        // [m + S]      row pointers, slice s rows at slice_off[s] + s
    int32_t* cp;        // [S][C + 1]   column pointers
    uint16_t* cidx;     // [off[S]]     CSR column of each entry
    float* cval;        // [off[S]]
    uint16_t* ridx;     // [off[S]]     CSC row of each entry
    float* rval;        // [off[S]]
    int32_t* r2c;       // [off[S]]     CSC slot (within the slice) of each CSR entry
    float* mu;          // [S] mean observed value
    uint32_t* bm;       // row-major bitmaps
    uint32_t* bt;       // column-major bitmaps
    uint32_t* wr;       // per word of bm: set bits before it in its row
    uint32_t* wc;       // per word of bt: set bits before it in its column
    int64_t bm_stride, bt_stride;
    int64_t* line_pfx;  // [S + 1] prefix of n'_s (V-step lines)
    int32_t* rord;      // [m]          rows of each slice by decreasing entry count
    int32_t* cord;      // [S][C]       columns of each slice by decreasing entry count
    int32_t* rcls;      // [S][16]      per group-size class g: first sorted row, first warp task
    int32_t* ccls;      // [S][16]      the same for the columns
    // Sliced layout of the lane-group ALS (r <= 16), one per side: the entry streams
    // of the 32 lanes of a warp task interleaved in chunks of 4, entry kk of lane l at
    // base[s] + tb[t] + 128 (kk / 4) + 4 l + kk % 4, so that a lane reads 4 entries
    // with one 8-byte and one 16-byte load and a warp's loads are coalesced.
    int32_t* rpos;      // [m]          sorted position of each row
    int32_t* cpos;      // [S][C]       sorted position of each column
    int32_t* rtb;       // [S][tcap]    offset of each rows-side warp task in its slice's region
    int32_t* ctb;       // [S][tcap]
    int64_t* rbase;     // [S + 1]      region start of each slice, rows side ([S] = total)
    int64_t* cbase;     // [S + 1]
    uint16_t* sidx_r;   // [sell_cap]   column of each rows-side slot
    float* sval_r;
    uint16_t* sidx_c;   // [sell_cap]   row of each columns-side slot
    float* sval_c;
    int64_t sell_cap;
    int tcap;
    int lane_entries;   // class threshold (line_class)
    bool sell;          // fill the sliced layout
    bool csr;           // fill CSR / CSC (the warp-group ALS for r > 16)
};

// Builds Omega for the frame's samples (E = total entry count, known to the host):
// bitmaps, per-word prefixes, line counts, row / column pointers, sorted line orders,
// mean observed value per slice, and the sliced layout (sell) and / or CSR / CSC
// (csr), in scratch slot SCR_OMEGA.
lt_status omega_build(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int64_t E, bool sell, bool csr,
                      Omega* om);

}  // namespace ltk
