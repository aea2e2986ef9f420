// Pieces shared by the two forms of the masked-ALS half-step (the lane-group SIMT
// kernel and the tensor-core kernel): the float64 retry queue and the float32 /
// float64 Cholesky solve of one line.
#pragma once

#include <stdint.h>

namespace {

// a float factorisation is accepted when every pivot is positive and
// min pivot >= kPivotRatio * max pivot (pivots are the squared diagonal of L)
constexpr float kPivotRatio = 1e-6f;

template <int RP>
struct AlsQueue {
    int32_t* count;     // [1] lines queued by this half-step
    int64_t* dst;       // [cap] output row offset (floats) of each queued line
    int64_t* slot;      // [cap] first slot of the line's first lane stream in the sliced layout,
                        //       or (grp 0) the line's first position in CSR / CSC
    int64_t* src;       // [cap] offset (floats) in the source factors of the slice's rows
    int32_t* len;       // [cap] entries of the line
    int32_t* grp;       // [cap] lanes G of the line (entry e is entry e / G of stream e % G), or
                        //       0: the entries are contiguous in CSR (rows) / CSC (columns)
    int32_t* rank;      // [cap] rank of each queued line
    int64_t cap;
    int32_t* status;    // device status word (LT_ELIMIT when the queue overflows)
};

// Cholesky solve of (G + lam I) u = b in place (u returned in b); rows i >= r are
// identity rows with b_i = 0.  Returns false when `check` and the float pivots are
// not acceptable (a non-positive pivot or min/max pivot^2 < kPivotRatio).
template <int RP, typename T>
__device__ __forceinline__ bool chol_solve(T (&a)[RP * (RP + 1) / 2], T (&b)[RP], int r, float lam_rel, bool check) {
    T tr = T(0);
#pragma unroll
    for (int i = 0; i < RP; ++i) tr += a[i * (i + 1) / 2 + i];
    if (!(tr > T(0))) {  // no observed entry (or all-zero factors): zero factor
#pragma unroll
        for (int i = 0; i < RP; ++i) b[i] = T(0);
        return true;
    }
    const T lam = (T)lam_rel * tr / (T)r;
#pragma unroll
    for (int i = 0; i < RP; ++i) {
        if (i < r) {
            a[i * (i + 1) / 2 + i] += lam;
        } else {
#pragma unroll
            for (int j = 0; j <= i; ++j) a[i * (i + 1) / 2 + j] = (j == i) ? T(1) : T(0);
            b[i] = T(0);
        }
    }
    T dmin = T(3.0e38), dmax = T(0);
    bool ok = true;
#pragma unroll
    for (int j = 0; j < RP; ++j) {
        T d = a[j * (j + 1) / 2 + j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= a[j * (j + 1) / 2 + k] * a[j * (j + 1) / 2 + k];
        if (j < r) {
            ok &= d > T(0);
            dmin = d < dmin ? d : dmin;
            dmax = d > dmax ? d : dmax;
        }
        const T ljj = sqrt(d > T(0) ? d : T(1));
        const T inv = T(1) / ljj;
        a[j * (j + 1) / 2 + j] = ljj;
#pragma unroll
        for (int i = j + 1; i < RP; ++i) {
            T t = a[i * (i + 1) / 2 + j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= a[i * (i + 1) / 2 + k] * a[j * (j + 1) / 2 + k];
            a[i * (i + 1) / 2 + j] = t * inv;
        }
    }
    if (check && (!ok || dmin < (T)kPivotRatio * dmax)) return false;
#pragma unroll
    for (int i = 0; i < RP; ++i) {  // L y = b
        T t = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) t -= a[i * (i + 1) / 2 + k] * b[k];
        b[i] = t / a[i * (i + 1) / 2 + i];
    }
#pragma unroll
    for (int i = RP - 1; i >= 0; --i) {  // L^T x = y
        T t = b[i];
#pragma unroll
        for (int k = i + 1; k < RP; ++k) t -= a[k * (k + 1) / 2 + i] * b[k];
        b[i] = t / a[i * (i + 1) / 2 + i];
    }
    return true;
}

}  // namespace
