// Completion of the slices from their sampled entries and the factorised render.
//
//  * Omega build: per slice, the observed entries are placed through two occupancy
//    bitmaps (the position of an entry is a popcount of the bits before it, so the
//    layout is deterministic) into a sliced layout per side for the lane-group ALS
//    (lines sorted by entry count, warp tasks of 32 lanes, streams interleaved by
//    chunks of 4) and, for ranks above 16, into CSR / CSC.
//  * Masked ALS (the completion M_s ~= U_s V_s^T at rank r; Sec. 5 uses the factor
//    form M = X Y): up to rank 16 a line (a row of U or of V) belongs to a group of
//    2^g lanes sized by its entry count; each lane accumulates its part of the Gram
//    and right-hand side in registers from the slice's factor rows staged in shared
//    memory, the group reduces with shuffles and its first lane adds the ridge
//    lam_rel tr(G) / r, factors by Cholesky in float32 and solves; lines whose pivots
//    spread beyond 1e6 are solved again in float64.  The half-step kernel is
//    persistent: each CTA takes an equal share of all slices' warp tasks.  Above
//    rank 16 a warp group holds a line's Gram (built on the tensor cores) row by row.
//    The rank may differ per slice (factor rows keep the stride of the largest).
//  * Render (Sec. 3 step 5): t_s = V_s^T w, pixel = max(0, u_i . t_s).
#include <math.h>

#include <algorithm>
#include <vector>

#include "lt_internal.cuh"
#include "lt_omega.cuh"
#include "lt_als_common.cuh"
#include "lt_als_tc.cuh"

using namespace ltk;

namespace {



// Group-size classes of a line: class g gives a line of L entries G = 2^g lanes, so
// that a lane takes at most about `lane_entries` of them (g = 0..5; a tuning value).
constexpr int kClasses = 6;

__host__ __device__ inline int line_class(int len, int lane_entries) {
    int g = 0;
    while (g < kClasses - 1 && len > (lane_entries << g)) ++g;
    return g;
}

// Omega build in five passes over the whole GPU (slice = blockIdx.y):
//  1. clear the used words of both bitmaps;  2. set the bit of every entry and sum
//  the values (one partial per block, fixed order);  3. one warp per row (column):
//  popcount of each bitmap word, warp scan into the per-word prefix, line count;
//  4. one block per slice: exclusive scan of the line counts into row / column
//  pointers, mean value;  5. one thread per entry: slot = pointer + bits before.
__global__ void k_om_clear(lt_frame F, lt_samples smp, Omega om) {
    const int s = blockIdx.y;
    const int ms = F.slice_off[s + 1] - F.slice_off[s], ns = smp.ncol[s];
    const int64_t nbm = (int64_t)ms * ((ns + 31) >> 5), nbt = (int64_t)ns * ((ms + 31) >> 5);
    uint32_t* bm = om.bm + (int64_t)s * om.bm_stride;
    uint32_t* bt = om.bt + (int64_t)s * om.bt_stride;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbm; i += (int64_t)gridDim.x * blockDim.x)
        bm[i] = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nbt; i += (int64_t)gridDim.x * blockDim.x)
        bt[i] = 0u;
}

__global__ void k_om_bits(lt_frame F, lt_samples smp, Omega om, float* __restrict__ part, int32_t* status) {
    __shared__ float red[32];
    const int s = blockIdx.y;
    const int ms = F.slice_off[s + 1] - F.slice_off[s], ns = smp.ncol[s], ne = smp.cnt[s];
    const int W = (ns + 31) >> 5, WT = (ms + 31) >> 5;
    uint32_t* bm = om.bm + (int64_t)s * om.bm_stride;
    uint32_t* bt = om.bt + (int64_t)s * om.bt_stride;
    const uint32_t* key = smp.key + smp.off[s];
    const float* val = smp.val + smp.off[s];
    float sum = 0.f;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const uint32_t k = key[e];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        if (r >= ms || c >= ns) {
            latch(status, LT_EINVAL);
            continue;
        }
        atomicOr(bm + (int64_t)r * W + (c >> 5), 1u << (c & 31));
        atomicOr(bt + (int64_t)c * WT + (r >> 5), 1u << (r & 31));
        sum += val[e];
    }
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        part[(int64_t)s * gridDim.x + blockIdx.x] = t;
    }
}

// one warp per line: word prefixes of one bitmap row, the line's count into cnt_out
__device__ __forceinline__ void om_line_words(const uint32_t* __restrict__ bits, uint32_t* __restrict__ pfx,
                                              int nw, int32_t* cnt_out) {
    const int lane = threadIdx.x & 31;
    int carry = 0;
    for (int w0 = 0; w0 < nw; w0 += 32) {
        const int w = w0 + lane;
        const int c = w < nw ? __popc(bits[w]) : 0;
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (w < nw) pfx[w] = (uint32_t)(carry + incl - c);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) *cnt_out = carry;
}

__global__ void k_om_lines(lt_frame F, lt_samples smp, Omega om) {
    const int s = blockIdx.y;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0, ns = smp.ncol[s];
    const int W = (ns + 31) >> 5, WT = (ms + 31) >> 5;
    const int nwarps = gridDim.x * (blockDim.x >> 5);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (int l = gw; l < ms + ns; l += nwarps) {
        if (l < ms) {
            const int64_t o = (int64_t)s * om.bm_stride + (int64_t)l * W;
            om_line_words(om.bm + o, om.wr + o, W, om.rp + row0 + s + l + 1);
        } else {
            const int c = l - ms;
            const int64_t o = (int64_t)s * om.bt_stride + (int64_t)c * WT;
            om_line_words(om.bt + o, om.wc + o, WT, om.cp + (int64_t)s * (F.C + 1) + c + 1);
        }
    }
}

// in place: x[0] = 0, x[1..n] counts -> exclusive prefix x[0..n]
__device__ void om_scan_counts(int32_t* x, int n, int32_t* ws) {
    int carry = 0;
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int c = i < n ? x[i + 1] : 0;
        int tot;
        const int pre = block_exclusive_scan<int>(c, ws, &tot);
        if (i < n) x[i + 1] = carry + pre + c;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) x[0] = 0;
}

// ord[0..n) = lines by decreasing count (ties by index), from the counts ptr[1..n]
// before they are scanned; a block-wide bitonic sort in shared memory, or the
// identity when n exceeds kOrdMax.
constexpr int kOrdMax = 4096;

// cls[0..7): first sorted line of each class, largest class first (cls[kClasses - 1 - g]
// for class g) and cls[8..15): the first warp task of each, a class-g task covering
// 32 / 2^g lines; cls[6] and cls[14] are the totals.
__device__ void om_classes(const int32_t* __restrict__ cnt1, int n, const int32_t* __restrict__ ord, bool sorted,
                           int lane_entries, int32_t* __restrict__ cls) {
    __shared__ int32_t num[kClasses];
    if (threadIdx.x < kClasses) num[threadIdx.x] = 0;
    __syncthreads();
    if (sorted)
        for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&num[line_class(cnt1[ord[i]], lane_entries)], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!sorted) num[0] = n;  // unsorted: every line on one lane
        int line = 0, task = 0;
        for (int k = 0; k < kClasses; ++k) {  // k-th run in the order = class kClasses - 1 - k
            const int g = kClasses - 1 - k;
            cls[k] = line;
            cls[8 + k] = task;
            line += num[g];
            task += (num[g] + (32 >> g) - 1) / (32 >> g);
        }
        cls[kClasses] = line;
        cls[8 + kClasses] = task;
    }
    __syncthreads();
}

__device__ void om_order(const int32_t* __restrict__ cnt1, int n, int32_t* __restrict__ ord,
                         unsigned long long* key) {
    if (n > kOrdMax) {
        for (int i = threadIdx.x; i < n; i += blockDim.x) ord[i] = i;
        __syncthreads();
        return;
    }
    int N = 1;
    while (N < n) N <<= 1;
    for (int i = threadIdx.x; i < N; i += blockDim.x)
        key[i] = i < n ? ((unsigned long long)(0xffffffffu - (uint32_t)cnt1[i]) << 32) | (uint32_t)i : ~0ull;
    __syncthreads();
    for (int k = 2; k <= N; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < N; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = key[i], b = key[l];
                    if ((a > b) == ((i & k) == 0)) {
                        key[i] = b;
                        key[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < n; i += blockDim.x) ord[i] = (int32_t)(key[i] & 0xffffffffu);
    __syncthreads();
}

// run of the sorted order that holds position li (classes largest first)
__device__ __forceinline__ int om_run(const int32_t* cls, int li) {
    int k = 0;
    while (k + 1 < kClasses && li >= cls[k + 1]) ++k;
    return k;
}

// pos[ord[i]] = i, and the sliced layout of one side: a class-g task covers
// P = 32 / 2^g lines, its lanes hold ceil(count / 2^g) slots at most, so the task
// takes 32 x (that maximum over its lines, rounded up to 4) slots; tb[t] = the
// slots before task t (a multiple of 128).
// The region size goes to *size.
__device__ void om_tasks(const int32_t* __restrict__ cnt1, int n, const int32_t* __restrict__ ord,
                         const int32_t* __restrict__ cls, int32_t* __restrict__ pos, int32_t* __restrict__ tb,
                         int64_t* size, int32_t* ws) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) pos[ord[i]] = i;
    const int T = cls[8 + kClasses];
    int carry = 0;
    for (int t0 = 0; t0 < T; t0 += blockDim.x) {
        const int t = t0 + threadIdx.x;
        int w = 0;
        if (t < T) {
            int k = 0;
            while (k + 1 < kClasses && t >= cls[8 + k + 1]) ++k;
            const int g = kClasses - 1 - k, G = 1 << g, P = 32 >> g;
            const int li0 = cls[k] + (t - cls[8 + k]) * P, li1 = min(li0 + P, cls[k + 1]);
            int kk = 0;
            for (int li = li0; li < li1; ++li) kk = max(kk, (cnt1[ord[li]] + G - 1) >> g);
            w = 32 * ((kk + 3) & ~3);
        }
        int tot;
        const int pre = block_exclusive_scan<int>(w, ws, &tot);
        if (t < T) tb[t] = carry + pre;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *size = carry;
    __syncthreads();
}

__global__ void k_om_scan(lt_frame F, lt_samples smp, Omega om, const float* __restrict__ part, int nparts) {
    __shared__ int32_t ws[32];
    __shared__ unsigned long long key[kOrdMax];
    const int s = blockIdx.x;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0, ns = smp.ncol[s], ne = smp.cnt[s];
    const int32_t* rc1 = om.rp + row0 + s + 1;                // row counts (before the scan)
    const int32_t* cc1 = om.cp + (int64_t)s * (F.C + 1) + 1;  // column counts
    int32_t* rord = om.rord + row0;
    int32_t* cord = om.cord + (int64_t)s * F.C;
    int32_t* rcls = om.rcls + (int64_t)s * 16;
    int32_t* ccls = om.ccls + (int64_t)s * 16;
    om_order(rc1, ms, rord, key);
    om_classes(rc1, ms, rord, ms <= kOrdMax, om.lane_entries, rcls);
    om_order(cc1, ns, cord, key);
    om_classes(cc1, ns, cord, ns <= kOrdMax, om.lane_entries, ccls);
    if (om.sell) {
        om_tasks(rc1, ms, rord, rcls, om.rpos + row0, om.rtb + (int64_t)s * om.tcap, om.rbase + s + 1, ws);
        om_tasks(cc1, ns, cord, ccls, om.cpos + (int64_t)s * F.C, om.ctb + (int64_t)s * om.tcap, om.cbase + s + 1,
                 ws);
    }
    om_scan_counts(om.rp + row0 + s, ms, ws);
    om_scan_counts(om.cp + (int64_t)s * (F.C + 1), ns, ws);
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int q = 0; q < nparts; ++q) t += part[(int64_t)s * nparts + q];
        om.mu[s] = ne > 0 ? t / (float)ne : 0.f;
    }
}

// region starts of the sliced layouts: in place, x[1..S] sizes -> x[0..S] prefix;
// a total beyond the capacity latches LT_ELIMIT (the scatter then skips slots past it)
__global__ void k_om_sellpfx(int S, Omega om, int32_t* status) {
    __shared__ int64_t ws[32];
    for (int side = 0; side < 2; ++side) {
        int64_t* x = side == 0 ? om.rbase : om.cbase;
        int64_t carry = 0;
        for (int i0 = 0; i0 < S; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            const int64_t c = i < S ? x[i + 1] : 0;
            int64_t tot;
            const int64_t pre = block_exclusive_scan<int64_t>(c, ws, &tot);
            if (i < S) x[i + 1] = carry + pre + c;
            carry += tot;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            x[0] = 0;
            if (carry > om.sell_cap) latch(status, LT_ELIMIT);
        }
        __syncthreads();
    }
}

// slot, within the slice's region, of entry k of the line at sorted position li
__device__ __forceinline__ int64_t sell_slot(const int32_t* __restrict__ cls, const int32_t* __restrict__ tb, int li,
                                             int k) {
    const int run = om_run(cls, li);
    const int g = kClasses - 1 - run, P = 32 >> g;
    const int rel = li - cls[run];
    const int t = cls[8 + run] + rel / P, lane = (rel % P) * (1 << g) + (k & ((1 << g) - 1));
    const int kk = k >> g;
    return (int64_t)tb[t] + 128 * (int64_t)(kk >> 2) + 4 * lane + (kk & 3);
}

__global__ void k_om_scatter(lt_frame F, lt_samples smp, Omega om) {
    const int s = blockIdx.y;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0, ns = smp.ncol[s], ne = smp.cnt[s];
    const int W = (ns + 31) >> 5, WT = (ms + 31) >> 5;
    const uint32_t* bm = om.bm + (int64_t)s * om.bm_stride;
    const uint32_t* bt = om.bt + (int64_t)s * om.bt_stride;
    const uint32_t* wr = om.wr + (int64_t)s * om.bm_stride;
    const uint32_t* wc = om.wc + (int64_t)s * om.bt_stride;
    const int32_t* rp = om.rp + row0 + s;
    const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
    const int64_t o = smp.off[s];
    const uint32_t* key = smp.key + o;
    const float* val = smp.val + o;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const uint32_t k = key[e];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        if (r >= ms || c >= ns) continue;
        const int64_t iw = (int64_t)r * W + (c >> 5), jw = (int64_t)c * WT + (r >> 5);
        const int kr = (int)wr[iw] + __popc(bm[iw] & ((1u << (c & 31)) - 1u));  // index in its row
        const int kc = (int)wc[jw] + __popc(bt[jw] & ((1u << (r & 31)) - 1u));  // index in its column
        const float v = val[e];
        if (om.csr) {
            om.cidx[o + rp[r] + kr] = (uint16_t)c;
            om.cval[o + rp[r] + kr] = v;
            om.ridx[o + cp[c] + kc] = (uint16_t)r;
            om.rval[o + cp[c] + kc] = v;
            om.r2c[o + rp[r] + kr] = cp[c] + kc;
        }
        if (om.sell) {
            const int64_t pr = sell_slot(om.rcls + (int64_t)s * 16, om.rtb + (int64_t)s * om.tcap,
                                         om.rpos[row0 + r], kr) + om.rbase[s];
            const int64_t pc = sell_slot(om.ccls + (int64_t)s * 16, om.ctb + (int64_t)s * om.tcap,
                                         om.cpos[(int64_t)s * F.C + c], kc) + om.cbase[s];
            if (pr < om.sell_cap) {
                om.sidx_r[pr] = (uint16_t)c;
                om.sval_r[pr] = v;
            }
            if (pc < om.sell_cap) {
                om.sidx_c[pc] = (uint16_t)r;
                om.sval_c[pc] = v;
            }
        }
    }
}

__global__ void k_line_prefix(const lt_samples smp, int S, int64_t* pfx) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < S ? (int64_t)smp.ncol[s] : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < S) pfx[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) pfx[S] = carry;
}

__global__ void k_als_init(lt_frame F, lt_samples smp, Omega om, int R, const int32_t* __restrict__ rk, SeedRef sr,
                           float* __restrict__ V) {
    const int s = blockIdx.y;
    const uint64_t seed = sr.get();
    const int ns = smp.ncol[s];
    const int r = slice_rank(rk, s, R);  // the slice's rank; components r .. R-1 are 0
    const float amp = sqrtf(fmaxf(om.mu[s], 0.f) / (float)r);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns * R; i += gridDim.x * blockDim.x) {
        const int j = i / R, k = i % R;
        if (k >= r) {
            V[((int64_t)s * F.C + j) * R + k] = 0.f;
            continue;
        }
        const uint32_t w = philox((uint32_t)k, (uint32_t)j, slice_key(F.slice_id, s), kTagAlsInit, seed).x;
        V[((int64_t)s * F.C + j) * R + k] = amp * (0.5f + (float)w * 2.3283064365386963e-10f);
    }
}

// ---- Gram of one line by one warp (ranks above 16) ---------------------------
// For one line (a row of U or of V) with observed entries e and factor rows x_e,
// G = sum_e x_e x_e^T and b = sum_e a_e x_e.  Lane k accumulates row k of G (all RP
// columns; G is symmetric) and b_k.  The entries are taken 32 at a time: lane l loads
// the factor row of entry l with 16-byte loads and stages it in shared memory (the
// line's Gram buffer, 16-byte chunk c of row l at chunk c ^ (l & 7) so that the
// stores of eight lanes fill all banks), then for each staged row every lane reads
// the whole row (broadcast loads) and its own component, and adds x_e[k] x_e and
// a_e x_e[k].  The rows have stride R; components at or beyond R are zero.  At the
// end rows k of G go to Gs[RP][RP+1] (over the stage) and b to bs[RP].
template <int RP>  // RP == 32: lane k holds row k
__device__ __forceinline__ void gram_warp(int len, const uint16_t* __restrict__ idx, const float* __restrict__ val,
                                          const float* __restrict__ src, int R, float* Gs, float* bs) {
    static_assert(RP == 32, "one lane per Gram row");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool vec = (R & 3) == 0 && ((uintptr_t)src & 15) == 0;
    float4* xs4 = reinterpret_cast<float4*>(Gs);  // 32 staged rows of 8 chunks (4 KB <= the Gram buffer)
    const float* xsf = Gs;
    float g[RP];
#pragma unroll
    for (int c = 0; c < RP; ++c) g[c] = 0.f;
    float b = 0.f;
    for (int e0 = 0; e0 < len; e0 += 32) {
        const int n = min(32, len - e0);
        const bool mine = lane < n;
        const int j = mine ? (int)idx[e0 + lane] : 0;
        const float av = mine ? val[e0 + lane] : 0.f;
        const float* xr = src + (int64_t)j * R;
        float4 t[RP / 4];
#pragma unroll
        for (int c = 0; c < RP / 4; ++c) {
            t[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (mine) {
                if (vec) {
                    if (4 * c < R) t[c] = __ldg(reinterpret_cast<const float4*>(xr) + c);
                } else {
                    t[c].x = 4 * c < R ? __ldg(xr + 4 * c) : 0.f;
                    t[c].y = 4 * c + 1 < R ? __ldg(xr + 4 * c + 1) : 0.f;
                    t[c].z = 4 * c + 2 < R ? __ldg(xr + 4 * c + 2) : 0.f;
                    t[c].w = 4 * c + 3 < R ? __ldg(xr + 4 * c + 3) : 0.f;
                }
            }
        }
        __syncwarp();  // the previous chunk's rows have been read
#pragma unroll
        for (int c = 0; c < RP / 4; ++c) xs4[lane * 8 + (c ^ (lane & 7))] = t[c];
        __syncwarp();
        const int kc = lane >> 2, kw = lane & 3;
        for (int q = 0; q < n; ++q) {  // n is warp-uniform
            const float a = __shfl_sync(FULL, av, q);
            float x[RP];
#pragma unroll
            for (int c = 0; c < RP / 4; ++c) {
                const float4 u = xs4[q * 8 + (c ^ (q & 7))];
                x[4 * c] = u.x;
                x[4 * c + 1] = u.y;
                x[4 * c + 2] = u.z;
                x[4 * c + 3] = u.w;
            }
            const float xk = xsf[(q * 8 + (kc ^ (q & 7))) * 4 + kw];
            b = fmaf(a, xk, b);
#pragma unroll
            for (int c = 0; c < RP; ++c) g[c] = fmaf(xk, x[c], g[c]);
        }
    }
    __syncwarp();  // every lane is done with the staged rows
#pragma unroll
    for (int c = 0; c < RP; ++c) Gs[lane * (RP + 1) + c] = g[c];
    bs[lane] = b;
}

// A group of G lanes solves (Gram + ridge) u = b for one line: lane k holds row k of
// the Gram in acc and b_k in rhs.  Returns false when the float factorisation is not
// acceptable (a non-positive pivot, or pivots spread by more than 1/kPivotRatio).
// Column J of the in-warp Cholesky and the columns after it, unrolled at compile
// time (a loop whose inner bound depends on the outer index is not fully unrolled
// by the compiler, and acc then lives in local memory)
template <int G, typename T, int J>
__device__ __forceinline__ void chol_col(T (&acc)[G], int k, int r, bool& ok, T& dmin, T& dmax) {
    if constexpr (J < G) {
        const unsigned FULL = 0xffffffffu;
        const T djj = __shfl_sync(FULL, acc[J], J, G);
        if (J < r) {
            ok &= (djj > T(0));
            dmin = djj < dmin ? djj : dmin;
            dmax = djj > dmax ? djj : dmax;
        }
        const T dpos = djj > T(0) ? djj : T(1);
        const T ljj = sqrt(dpos);
        const T inv = T(1) / ljj;
        const T lij = (k > J) ? acc[J] * inv : (k == J ? ljj : T(0));
        acc[J] = lij;
#pragma unroll
        for (int c = J + 1; c < G; ++c) {
            const T lcj = __shfl_sync(FULL, lij, c, G);
            if (k > J) acc[c] -= lij * lcj;
        }
        chol_col<G, T, J + 1>(acc, k, r, ok, dmin, dmax);
    }
}

// Step J of the backward substitution L^T x = y and the steps before it
template <int G, typename T, int J>
__device__ __forceinline__ void back_col(const T (&acc)[G], int k, T& x) {
    if constexpr (J >= 0) {
        const unsigned FULL = 0xffffffffu;
        const T xj = __shfl_sync(FULL, x, J, G) / __shfl_sync(FULL, acc[J], J, G);
        if (k == J) x = xj;
#pragma unroll
        for (int c = 0; c < J; ++c) {
            const T ljc = __shfl_sync(FULL, acc[c], J, G);
            if (k == c) x -= ljc * xj;
        }
        back_col<G, T, J - 1>(acc, k, x);
    }
}

template <int G, typename T, bool SMEM_L>
__device__ __forceinline__ bool factor_solve_rows(T (&acc)[G], T rhs, bool live, int len, int r, float lam_rel,
                                                  int k, T* out_k, bool check, float* Lsh) {
    const unsigned FULL = 0xffffffffu;
    if (!live) len = 0;
    T tr = T(0);
#pragma unroll
    for (int c = 0; c < G; ++c)
        if (c == k) tr = acc[c];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) tr += __shfl_xor_sync(FULL, tr, o, G);
    const bool zero = !(tr > T(0)) || len == 0;
    const T lam = (T)lam_rel * tr / (T)r;
#pragma unroll
    for (int c = 0; c < G; ++c)
        if (c == k) acc[c] = (k < r) ? acc[c] + lam : T(1);
    if (k >= r) {
#pragma unroll
        for (int c = 0; c < G; ++c)
            if (c != k) acc[c] = T(0);
        rhs = T(0);
    }
    // right-looking Cholesky: lane i keeps row i; column j of L overwrites acc[j]
    T dmin = T(3.0e38), dmax = T(0);
    bool ok = true;
    chol_col<G, T, 0>(acc, k, r, ok, dmin, dmax);
    if (check && !zero && (!ok || dmin < (T)kPivotRatio * dmax)) return false;
    if (SMEM_L) {
        // triangular solves through shared memory (Lsh may alias this line's Gram:
        // every lane has read its row before any lane writes here)
        __syncwarp();
        // row k of L; the diagonal slot holds 1 / L[k][k]
        T dk = T(1);
#pragma unroll
        for (int c = 0; c < G; ++c)
            if (c == k) dk = acc[c];
#pragma unroll
        for (int c = 0; c < G; ++c) Lsh[k * G + c] = (c == k) ? (float)(T(1) / dk) : (float)acc[c];
        __syncwarp();
        T y = rhs;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const T yj = __shfl_sync(FULL, y, j, G) * (T)Lsh[j * G + j];
            if (k == j) y = yj;
            else if (k > j) y -= (T)Lsh[k * G + j] * yj;
        }
        T x = y;
#pragma unroll
        for (int j = G - 1; j >= 0; --j) {
            const T xj = __shfl_sync(FULL, x, j, G) * (T)Lsh[j * G + j];
            if (k == j) x = xj;
            else if (k < j) x -= (T)Lsh[j * G + k] * xj;
        }
        __syncwarp();
        *out_k = (zero || k >= r) ? T(0) : x;
        return true;
    }
    if (SMEM_L) return true;  // not reached
    // forward L y = b: lane k holds L[k][0..k] in acc[0..k]
    T y = rhs;
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const T yj = __shfl_sync(FULL, y, j, G) / __shfl_sync(FULL, acc[j], j, G);
        if (k == j) y = yj;
        else if (k > j) y -= acc[j] * yj;
    }
    // backward L^T x = y: x_j is final at step j; L[j][c] (c < j) comes from lane j
    T x = y;
    back_col<G, T, G - 1>(acc, k, x);
    *out_k = (zero || k >= r) ? T(0) : x;
    return true;
}

// the same with row k of the Gram and b_k read from Gs [G][G + 1] and bs
template <int G, typename T, bool SMEM_L>
__device__ __forceinline__ bool factor_solve(const float* Gs, const float* bs, bool live, int len, int r,
                                             float lam_rel, int k, T* out_k, bool check, float* Lsh) {
    T acc[G];
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = live ? (T)Gs[k * (G + 1) + c] : T(0);
    const T rhs = live ? (T)bs[k] : T(0);
    return factor_solve_rows<G, T, SMEM_L>(acc, rhs, live, len, r, lam_rel, k, out_k, check, Lsh);
}

// One half-step for ranks above 16: rows of U (rows_side) or columns of V, slice by
// slice.  CTA (p, s) takes the p-th of P equal parts of the lines of slice s; a warp
// builds the Gram of one line at a time (gram_warp, the other side's factor rows
// read from L2) and factors and solves it in the warp in float32; a line whose
// pivots fail the check goes to the float64 pass (k_als_retry).
template <int RP>
__host__ __device__ constexpr int als_warps() { return RP == 32 ? 8 : 16; }

template <int RP>
__global__ void __launch_bounds__(32 * als_warps<RP>(), 2) k_als_half(lt_frame F, lt_samples smp, Omega om, int R,
                                                                   const int32_t* __restrict__ rk,
                                                                   float lam_rel, bool rows_side,
                                                                   const float* __restrict__ Fin,
                                                                   float* __restrict__ Fout, AlsQueue<RP> aq) {
    constexpr int LPW = 32 / RP;  // lines per warp
    constexpr int NW = als_warps<RP>();
    __shared__ __align__(16) float Gs_all[NW][LPW][RP * (RP + 1)];
    __shared__ float bs_all[NW][LPW][RP];
    const int s = blockIdx.y, P = gridDim.x, p = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / RP, k = lane % RP;
    const int r = slice_rank(rk, s, R);  // the slice's rank (factor rows have stride R)
    if (rk && r <= 16) return;           // per-slice ranks: the lane-group kernel has these slices
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0;
    const int ns = smp.ncol[s];
    const int nlines = rows_side ? ms : ns;
    const int l0 = (int)((int64_t)nlines * p / P), l1 = (int)((int64_t)nlines * (p + 1) / P);
    if (l0 >= l1) return;
    const float* src = rows_side ? Fin + (int64_t)s * F.C * R : Fin + (int64_t)row0 * R;
    const int64_t o = smp.off[s];
    for (int base = l0 + wid * LPW; base < l1; base += NW * LPW) {
        int my_len = 0;
        int64_t my_dst = 0, my_pos = 0;
#pragma unroll
        for (int q = 0; q < LPW; ++q) {
            const int line = base + q;
            if (line >= l1) break;  // warp-uniform
            int len, b;
            const uint16_t* idx;
            const float* vv;
            int64_t dst;
            if (rows_side) {
                const int32_t* rp = om.rp + row0 + s;
                b = rp[line];
                len = rp[line + 1] - b;
                idx = om.cidx + o + b;
                vv = om.cval + o + b;
                dst = (int64_t)(row0 + line) * R;           // U row
            } else {
                const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
                b = cp[line];
                len = cp[line + 1] - b;
                idx = om.ridx + o + b;
                vv = om.rval + o + b;
                dst = ((int64_t)s * F.C + line) * R;        // V row
            }
            gram_warp<RP>(len, idx, vv, src, R, &Gs_all[wid][q][0], &bs_all[wid][q][0]);
            if (grp == q) {
                my_len = len;
                my_dst = dst;
                my_pos = o + b;
            }
        }
        __syncwarp();
        const bool live = base + grp < l1;
        const float* Gs = &Gs_all[wid][grp][0];
        const float* bs = &bs_all[wid][grp][0];
        float xf = 0.f;
        const bool okf = factor_solve<RP, float, true>(Gs, bs, live, my_len, r, lam_rel, k, &xf, true,
                                                 &Gs_all[wid][grp][0]);
        if (live && k < R) Fout[my_dst + k] = (okf && k < r) ? xf : 0.f;
        if (live && !okf && k == 0) {
            // rare: the float pivots were not acceptable; the line goes to the float64
            // pass (k_als_retry), which forms its Gram again in float64 from the factor
            // rows (a Gram summed in float32 would carry its rounding into the solve)
            const int qs = atomicAdd(aq.count, 1);
            if (qs < aq.cap) {
                aq.dst[qs] = my_dst;
                aq.slot[qs] = my_pos;
                aq.src[qs] = src - Fin;
                aq.len[qs] = my_len;
                aq.grp[qs] = 0;  // contiguous in CSR / CSC
                aq.rank[qs] = r;
            } else {
                latch(aq.status, LT_ELIMIT);
            }
        }
        __syncwarp();
    }
}

// ---- rank <= 16: Gram on the tensor cores, then one thread per line ------------
// The in-warp Cholesky of the line solve costs as many warp instructions as the
// whole tensor-core Gram; a 16 x 16 Cholesky fits one thread's registers instead.
// ---- Masked ALS, one thread per line (r <= 16) --------------------------------
// A line is a row of U_s (U-step, its entries in CSR) or a column of V_s (V-step,
// CSC).  The thread gathers the factor row x_j of each observed entry from the
// slice's factor rows staged in shared memory and accumulates the lower triangle of
// G = sum x_j x_j^T and b = sum a_j x_j in registers (RP(RP+1)/2 + RP values),
// adds the ridge lam_rel tr(G)/r, factors G by Cholesky in float32 and solves.
// Lines whose pivots fail the check go to a queue; a second kernel forms their
// Gram again in float64 (products of the float32 factors are exact in float64) and
// solves it in float64, so an ill-conditioned line carries no float32 rounding.
// A staged factor row is RP floats (RP/4 16-byte slots).  Slot q of row j is stored
// at slot q ^ h(j) so that the rows read by one quarter-warp (random j) spread over
// all eight 16-byte bank groups of a 128-byte shared-memory wavefront.
template <int RP>
__device__ __forceinline__ int stage_slot(int j, int q) {
    constexpr int NQ = RP / 4, RPB = 8 / NQ;  // slots per row, rows per wavefront
    return j * NQ + (q ^ ((j / RPB) % NQ));
}

// Adds x_e x_e^T (lower triangle) and a_e x_e for the nk entries of one lane's
// stream (chunks of 4 at idx4[32 c], vv4[32 c]) to a and bb, in stream order.
template <int RP>
__device__ __forceinline__ void stream_gram(int nk, const uint2* __restrict__ idx4, const float4* __restrict__ vv4,
                                            int r, int R, const float* __restrict__ src, bool staged,
                                            const float4* stage4, float (&a)[RP * (RP + 1) / 2], float (&bb)[RP]) {
    constexpr int NQ = RP / 4;
    const int nc = (nk + 3) >> 2;
    // the next two chunks' loads are in flight during this chunk's four entries
    uint2 ic = nc > 0 ? idx4[0] : make_uint2(0u, 0u), in = nc > 1 ? idx4[32] : ic;
    float4 vc = nc > 0 ? vv4[0] : make_float4(0.f, 0.f, 0.f, 0.f), vn = nc > 1 ? vv4[32] : vc;
    for (int c = 0; c < nc; ++c) {
        uint2 in2 = in;
        float4 vn2 = vn;
        if (c + 2 < nc) {
            in2 = idx4[32 * (c + 2)];
            vn2 = vv4[32 * (c + 2)];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (4 * c + q < nk) {
                const uint32_t w = q < 2 ? ic.x : ic.y;
                const int j = (int)((w >> (16 * (q & 1))) & 0xffffu);
                const float av = q == 0 ? vc.x : q == 1 ? vc.y : q == 2 ? vc.z : vc.w;
                float x[RP];
                if (staged) {
#pragma unroll
                    for (int c4 = 0; c4 < NQ; ++c4) {
                        const float4 t = stage4[stage_slot<RP>(j, c4)];
                        x[4 * c4] = t.x;
                        x[4 * c4 + 1] = t.y;
                        x[4 * c4 + 2] = t.z;
                        x[4 * c4 + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int cc = 0; cc < RP; ++cc) x[cc] = cc < r ? __ldg(src + (int64_t)j * R + cc) : 0.f;
                }
#pragma unroll
                for (int i = 0; i < RP; ++i) {
                    bb[i] = fmaf(av, x[i], bb[i]);
#pragma unroll
                    for (int k = 0; k <= i; ++k)
                        a[i * (i + 1) / 2 + k] = fmaf(x[i], x[k], a[i * (i + 1) / 2 + k]);
                }
            }
        }
        ic = in;
        vc = vn;
        in = in2;
        vn = vn2;
    }
}

// One lane of a warp task: `line` (or -1) is its line, `sub` its rank among the G
// lanes of the line, `slot` the first slot of its stream (task base + 4 lane).
template <int RP>
__device__ __forceinline__ void als_line(const lt_frame& F, const Omega& om, int r, int R, bool rows_side,
                                         const float* __restrict__ src_base, const float* __restrict__ src,
                                         bool staged, const float4* stage4,
                                         float* __restrict__ Fout, float lam_rel, const AlsQueue<RP>& q, int s,
                                         int line, int sub, int G, int64_t slot) {
    constexpr int NA = RP * (RP + 1) / 2;
    const int row0 = F.slice_off[s];
    int len = 0;
    if (line >= 0) {
        if (rows_side) {
            const int32_t* rp = om.rp + row0 + s;
            len = rp[line + 1] - rp[line];
        } else {
            const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
            len = cp[line + 1] - cp[line];
        }
    }
    const uint16_t* sidx = rows_side ? om.sidx_r : om.sidx_c;
    const float* sval = rows_side ? om.sval_r : om.sval_c;
    float a[NA], bb[RP];
#pragma unroll
    for (int i = 0; i < NA; ++i) a[i] = 0.f;
#pragma unroll
    for (int i = 0; i < RP; ++i) bb[i] = 0.f;
    const int nk = sub < len ? (len - sub + G - 1) / G : 0;
    stream_gram<RP>(nk, reinterpret_cast<const uint2*>(sidx + slot), reinterpret_cast<const float4*>(sval + slot), r,
                    R, src, staged, stage4, a, bb);
    if (G > 1) {  // the group's partial sums into its first lane (G is warp-uniform)
        for (int m = G >> 1; m > 0; m >>= 1) {
#pragma unroll
            for (int i = 0; i < NA; ++i) a[i] += __shfl_down_sync(0xffffffffu, a[i], m, G);
#pragma unroll
            for (int i = 0; i < RP; ++i) bb[i] += __shfl_down_sync(0xffffffffu, bb[i], m, G);
        }
    }
    if (line < 0 || sub != 0) return;
    const int64_t dst = rows_side ? (int64_t)(row0 + line) * R : ((int64_t)s * F.C + line) * R;
    for (int i = r; i < R; ++i) Fout[dst + i] = 0.f;  // components beyond the slice's rank
    if (chol_solve<RP, float>(a, bb, r, lam_rel, true)) {
#pragma unroll
        for (int i = 0; i < RP; ++i)
            if (i < r) Fout[dst + i] = bb[i];
        return;
    }
    // rare: queue the line for the float64 pass (k_als_retry)
    const int qs = atomicAdd(q.count, 1);
    if (qs >= q.cap) {
        latch(q.status, LT_ELIMIT);
        return;
    }
    q.dst[qs] = dst;
    q.slot[qs] = slot;
    q.src[qs] = src - src_base;
    q.len[qs] = len;
    q.grp[qs] = G;
    q.rank[qs] = r;
}

// stage the slice's source factor rows (nsrc rows of stride R, the first r values,
// zero-padded to RP) in shared memory
template <int RP>
__device__ __forceinline__ void stage_factors(const float* __restrict__ src, int nsrc, int r, int R, float4* stage4) {
    constexpr int NQ = RP / 4;
    if (r == RP && R == RP) {
        const float4* src4 = reinterpret_cast<const float4*>(src);
        for (int i = threadIdx.x; i < nsrc * NQ; i += blockDim.x)
            stage4[stage_slot<RP>(i / NQ, i % NQ)] = __ldg(src4 + i);
    } else {
        for (int i = threadIdx.x; i < nsrc * NQ; i += blockDim.x) {
            const int row = i / NQ, q4 = i % NQ;
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) v[c] = 4 * q4 + c < r ? __ldg(src + (int64_t)row * R + 4 * q4 + c) : 0.f;
            stage4[stage_slot<RP>(row, q4)] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
}

// Persistent half-step: one CTA per SM.  CTA c owns the warp tasks (all slices, in
// slice order) whose first slot lies in its equal share [lo, hi) of all the slots
// of the side; for each slice it touches it stages the source factor rows once and
// its warps take that slice's tasks from a shared counter.
template <int RP>
__global__ void __launch_bounds__(256, 1) k_als_line(lt_frame F, lt_samples smp, Omega om, int R,
                                                    const int32_t* __restrict__ rk, bool rows_side,
                                                    const float* __restrict__ Fin, float* __restrict__ Fout,
                                                    float lam_rel, AlsQueue<RP> q, int stage_rows) {
    extern __shared__ float4 stage4[];
    __shared__ int s_next, s_t0, s_t1, s_slice;
    const int S = F.S;
    const int64_t* base = rows_side ? om.rbase : om.cbase;
    const int64_t total = base[S];
    // a layout over its capacity was latched as LT_ELIMIT and not written: read nothing
    if (total > om.sell_cap) return;
    const int64_t lo = total * blockIdx.x / gridDim.x;
    const int64_t hi = blockIdx.x + 1 == gridDim.x ? INT64_MAX : total * (blockIdx.x + 1) / gridDim.x;
    const int lane = threadIdx.x & 31;
    int s = -1, t = 0;  // next task to consider (thread 0's view, shared through s_*)
    if (threadIdx.x == 0) {
        // Task starts are non-decreasing in (slice, task) order and every task of slice
        // s starts at or before base[s + 1]: the first slice with base[s + 1] >= lo holds
        // the first task at or after lo, if it has one, else a later slice does.
        int x = 0, y = S;
        while (x < y) {
            const int m = (x + y) >> 1;
            if (base[m + 1] < lo) x = m + 1; else y = m;
        }
        s = x;
        t = 0;
        if (s < S) {
            const int32_t* cls = (rows_side ? om.rcls : om.ccls) + (int64_t)s * 16;
            const int32_t* tb = (rows_side ? om.rtb : om.ctb) + (int64_t)s * om.tcap;
            int a = 0, b = cls[8 + kClasses];
            while (a < b) {
                const int m = (a + b) >> 1;
                if (base[s] + tb[m] < lo) a = m + 1; else b = m;
            }
            t = a;
        }
    }
    for (;;) {
        if (threadIdx.x == 0) {
            // the next slice segment of this CTA: tasks [t, t1) of slice s starting before hi
            int seg = -1, t0 = 0, t1 = 0;
            while (s < S) {
                const int32_t* cls = (rows_side ? om.rcls : om.ccls) + (int64_t)s * 16;
                const int32_t* tb = (rows_side ? om.rtb : om.ctb) + (int64_t)s * om.tcap;
                const int T = cls[8 + kClasses];
                if (t < T && base[s] + tb[t] < hi) {
                    int x = t, y = T;  // first task at or after hi
                    while (x < y) {
                        const int m = (x + y) >> 1;
                        if (base[s] + tb[m] < hi) x = m + 1; else y = m;
                    }
                    seg = s;
                    t0 = t;
                    t1 = x;
                    if (x < T) {
                        s = S;  // the share ends inside this slice
                    } else {
                        ++s;
                        t = 0;
                    }
                    break;
                }
                if (t < T) {  // the next task of this slice is past hi: done
                    s = S;
                    break;
                }
                ++s;
                t = 0;
            }
            s_slice = seg;
            s_t0 = t0;
            s_t1 = t1;
            s_next = t0;
        }
        __syncthreads();
        const int sl = s_slice;
        if (sl < 0) break;
        const int row0 = F.slice_off[sl], ms = F.slice_off[sl + 1] - row0, ns = smp.ncol[sl];
        const int r = slice_rank(rk, sl, R);  // the slice's rank (factor rows have stride R)
        const bool mine = r <= RP;      // per-slice ranks above RP are the warp-group kernel's
        const float* src = rows_side ? Fin + (int64_t)sl * F.C * R : Fin + (int64_t)row0 * R;
        const int nsrc = rows_side ? ns : ms;
        const bool staged = nsrc <= stage_rows;
        if (staged && mine) stage_factors<RP>(src, nsrc, r, R, stage4);
        __syncthreads();
        const int32_t* ord = rows_side ? om.rord + row0 : om.cord + (int64_t)sl * F.C;
        const int32_t* cls = (rows_side ? om.rcls : om.ccls) + (int64_t)sl * 16;
        const int32_t* tb = (rows_side ? om.rtb : om.ctb) + (int64_t)sl * om.tcap;
        const int t1 = mine ? s_t1 : 0;
        for (;;) {
            int tk = 0;
            if (lane == 0) tk = atomicAdd(&s_next, 1);
            tk = __shfl_sync(0xffffffffu, tk, 0);
            if (tk >= t1) break;
            int k = 0;
            while (k + 1 < kClasses && tk >= cls[8 + k + 1]) ++k;
            const int g = kClasses - 1 - k, G = 1 << g;
            const int li = cls[k] + (tk - cls[8 + k]) * (32 >> g) + (lane >> g);
            const bool live = li < cls[k + 1];
            als_line<RP>(F, om, r, R, rows_side, Fin, src, staged, stage4, Fout, lam_rel, q, sl, live ? ord[li] : -1,
                         lane & (G - 1), G, base[sl] + tb[tk] + 4 * lane);
        }
        __syncthreads();  // the stage is reused by the next segment
    }
}

// float64 solve of the queued lines: one warp per line.  The warp walks the line's
// entries in chunks of 32 (lane l gathers entry e0 + l: its factor row and value into
// shared memory), and each lane accumulates its share of the Gram lower triangle and
// right-hand side elements (element lane + 32 p) in float64 over the chunk; the
// first lane then factors and solves in float64.
template <int RP>
__global__ void __launch_bounds__(128) k_als_retry(AlsQueue<RP> q, Omega om, bool rows_side,
                                                   const float* __restrict__ Fin, int R, float lam_rel,
                                                   float* __restrict__ Fout, int32_t* __restrict__ n_fp64) {
    constexpr int NA = RP * (RP + 1) / 2, NV = NA + RP, PER = (NV + 31) / 32;
    __shared__ float xs[4][32][RP + 1];
    __shared__ float av[4][32];
    __shared__ double gs[4][NV];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int ei[PER], ek[PER];  // owned element: Gram (ei, ek) with ek <= ei, or b_ei (ek = -1); ei = -1 for none
#pragma unroll
    for (int p = 0; p < PER; ++p) {
        const int e = lane + 32 * p;
        ei[p] = -1;
        ek[p] = -1;
        if (e < NA) {
            int i = 0;
            while ((i + 1) * (i + 2) / 2 <= e) ++i;
            ei[p] = i;
            ek[p] = e - i * (i + 1) / 2;
        } else if (e < NV) {
            ei[p] = e - NA;
        }
    }
    const uint16_t* sidx = rows_side ? om.sidx_r : om.sidx_c;
    const float* sval = rows_side ? om.sval_r : om.sval_c;
    const int n = (int)min((int64_t)*q.count, q.cap);
    for (int t = blockIdx.x * 4 + w; t < n; t += gridDim.x * 4) {
        const int len = q.len[t], G = q.grp[t], r = q.rank[t];
        const int64_t slot = q.slot[t];
        const float* src = Fin + q.src[t];
        double acc[PER];
#pragma unroll
        for (int p = 0; p < PER; ++p) acc[p] = 0.0;
        for (int e0 = 0; e0 < len; e0 += 32) {
            const int e = e0 + lane;
            if (e < len) {
                int j;
                if (G > 0) {  // sliced layout
                    const int u = e % G, kk = e / G;
                    const int64_t pos = slot + 4 * u + 128 * (kk >> 2) + (kk & 3);
                    j = sidx[pos];
                    av[w][lane] = sval[pos];
                } else {      // CSR / CSC
                    j = (rows_side ? om.cidx : om.ridx)[slot + e];
                    av[w][lane] = (rows_side ? om.cval : om.rval)[slot + e];
                }
#pragma unroll
                for (int c = 0; c < RP; ++c) xs[w][lane][c] = c < r ? src[(int64_t)j * R + c] : 0.f;
            }
            __syncwarp();
            const int ne = min(32, len - e0);
            for (int k2 = 0; k2 < ne; ++k2) {
#pragma unroll
                for (int p = 0; p < PER; ++p) {
                    if (ei[p] >= 0) {
                        const double xi = (double)xs[w][k2][ei[p]];
                        const double xk = ek[p] >= 0 ? (double)xs[w][k2][ek[p]] : (double)av[w][k2];
                        acc[p] = fma(xi, xk, acc[p]);
                    }
                }
            }
            __syncwarp();
        }
#pragma unroll
        for (int p = 0; p < PER; ++p)
            if (lane + 32 * p < NV) gs[w][lane + 32 * p] = acc[p];
        __syncwarp();
        if constexpr (RP == 32) {
            // rank above 16: the warp factors and solves (lane k holds row k), the
            // Cholesky of one lane would not fit its registers
            double row[32];
#pragma unroll
            for (int c = 0; c < 32; ++c)
                row[c] = c <= lane ? gs[w][lane * (lane + 1) / 2 + c] : gs[w][c * (c + 1) / 2 + lane];
            double xd = 0.0;
            factor_solve_rows<32, double, false>(row, gs[w][NA + lane], true, len, r, lam_rel, lane, &xd, false,
                                                 nullptr);
            if (lane < r) Fout[q.dst[t] + lane] = (float)xd;
            if (lane == 0) atomicAdd(n_fp64, 1);
        } else if (lane == 0) {
            double a[NA], b[RP];
            for (int i = 0; i < NA; ++i) a[i] = gs[w][i];
            for (int i = 0; i < RP; ++i) b[i] = gs[w][NA + i];
            chol_solve<RP, double>(a, b, r, lam_rel, false);
            float* d = Fout + q.dst[t];
            for (int i = 0; i < RP; ++i)
                if (i < r) d[i] = (float)b[i];
            atomicAdd(n_fp64, 1);
        }
        __syncwarp();
    }
}

// Image of slice s (Sec. 3): t_s = V_s^T w, then img[perm[i]] = max(0, u_i . t_s).
// blockIdx.y is the slice; each CTA forms t_s itself (the slice's V rows are read once
// from DRAM and then from L2): thread x owns component x % r of the columns
// x / r + c (blockDim / r), c = 0, 1, ... (consecutive threads read consecutive floats),
// and the partial sums are added in a fixed order.  The CTAs of a slice then split
// its rows, a thread per row (16-byte loads of u_i when r is a multiple of 4 and U
// 16-byte aligned).
__global__ void __launch_bounds__(512) k_render(lt_frame F, lt_samples smp, const float* __restrict__ U,
                                                const float* __restrict__ V, int r, const float* __restrict__ w,
                                                const int32_t* __restrict__ perm, float* __restrict__ img) {
    __shared__ float part[512];
    __shared__ float t[32];
    const int s = blockIdx.y;
    const int ns = smp.ncol[s];
    const int cpp = (int)blockDim.x / r;  // columns per pass
    const int col = (int)threadIdx.x / r, k = (int)threadIdx.x - col * r;
    float acc = 0.f;
    if (col < cpp) {
        const float* Vs = V + (int64_t)s * F.C * r;
        const float* ws = w ? w + (int64_t)s * F.C : nullptr;
        for (int j = col; j < ns; j += cpp) acc = fmaf(Vs[(int64_t)j * r + k], ws ? ws[j] : 1.f, acc);
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    if ((int)threadIdx.x < r) {
        float a = 0.f;
        for (int c = 0; c < cpp; ++c) a += part[c * r + threadIdx.x];
        t[threadIdx.x] = a;
    }
    __syncthreads();
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0;
    const bool vec = (r & 3) == 0 && ((uintptr_t)U & 15) == 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ms; i += gridDim.x * blockDim.x) {
        const float* u = U + (int64_t)(row0 + i) * r;
        float v = 0.f;
        if (vec) {
            const float4* u4 = reinterpret_cast<const float4*>(u);
            for (int q = 0; q < (r >> 2); ++q) {
                const float4 x = __ldg(u4 + q);
                v = fmaf(x.x, t[4 * q], v);
                v = fmaf(x.y, t[4 * q + 1], v);
                v = fmaf(x.z, t[4 * q + 2], v);
                v = fmaf(x.w, t[4 * q + 3], v);
            }
        } else {
            for (int q = 0; q < r; ++q) v = fmaf(__ldg(u + q), t[q], v);
        }
        img[perm[row0 + i]] = fmaxf(v, 0.f);
    }
}

// r_s = min(R, max(8, 8 ceil(n'_s / cols))): a multiple of 8 growing with the coarsened cut
__global__ void k_slice_ranks(lt_samples smp, int S, int R, int cols, int32_t* __restrict__ rank) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        const int n = smp.ncol[s];
        rank[s] = min(R, max(8, 8 * ((n + cols - 1) / cols)));
    }
}

}  // namespace

namespace ltk {

lt_status omega_build(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int64_t E, bool sell, bool csr,
                      Omega* omp) {
    const int S = f->S, C = f->C;
    constexpr int kOmParts = 8;
    const int64_t mr = std::max(f->max_rows, 1);
    Omega& om = *omp;
    om.bm_stride = mr * ((C + 31) / 32);
    om.bt_stride = (int64_t)C * ((mr + 31) / 32);
    om.sell = sell;
    om.csr = csr;
    // Sliced layout capacity, le = lane_entries.  Per slice and side, for lines sorted
    // by count, the padding of a task is at most the entries of the task before it
    // (the first task of class g < 5 adds at most 32 le slots, of class 5 at most
    // L_max), rounding to a multiple of 4 adds at most 128 slots per task, and there
    // are at most n / 32 + 2 E_s / (32 le) + 6 tasks (a class g > 0 line has more than
    // le 2^(g-1) entries): at most E_s (1 + 8 / le) + 4 n + L_max + 160 le + 768 slots.
    // Beyond the capacity the scatter latches LT_ELIMIT.
    const int64_t nmax = std::max<int64_t>(mr, C);
    om.lane_entries = ctx->tune.als_lane_entries;
    const int64_t le = om.lane_entries;
    om.sell_cap = om.sell ? E + (8 * E + le - 1) / le + E / 32 + (int64_t)S * (5 * nmax + 160 * le + 1024) : 0;
    om.tcap = (int)nmax + 8;
    const size_t e_csr = om.csr ? (size_t)E : 0, e_sell = (size_t)om.sell_cap;
    const size_t t_sell = om.sell ? (size_t)S * om.tcap : 0;
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_OMEGA,
                                (size_t)(f->m + S) * 4 + (size_t)S * (C + 1) * 4 + e_csr * 16 + e_sell * 12 + S * 8 +
                                    (size_t)S * (om.bm_stride + om.bt_stride) * 8 + (S + 1) * 8 + (size_t)f->m * 8 +
                                    (size_t)S * C * 8 + (size_t)S * 128 + t_sell * 8 + (size_t)(S + 1) * 16 +
                                    (size_t)S * kOmParts * 4 + 34 * 256,
                                &st);
    if (!p) return st;
    auto take = [&](size_t nbytes) {
        char* q = p;
        p += (nbytes + 255) & ~(size_t)255;
        return q;
    };
    om.rp = (int32_t*)take((f->m + S) * 4);
    om.cp = (int32_t*)take((size_t)S * (C + 1) * 4);
    om.cidx = (uint16_t*)take(e_csr * 2);
    om.cval = (float*)take(e_csr * 4);
    om.ridx = (uint16_t*)take(e_csr * 2);
    om.rval = (float*)take(e_csr * 4);
    om.r2c = (int32_t*)take(e_csr * 4);
    om.mu = (float*)take(S * 4);
    om.bm = (uint32_t*)take((size_t)S * om.bm_stride * 4);
    om.bt = (uint32_t*)take((size_t)S * om.bt_stride * 4);
    om.wr = (uint32_t*)take((size_t)S * om.bm_stride * 4);
    om.wc = (uint32_t*)take((size_t)S * om.bt_stride * 4);
    om.line_pfx = (int64_t*)take((S + 1) * 8);
    om.rord = (int32_t*)take((size_t)f->m * 4);
    om.cord = (int32_t*)take((size_t)S * C * 4);
    om.rcls = (int32_t*)take((size_t)S * 16 * 4);
    om.ccls = (int32_t*)take((size_t)S * 16 * 4);
    om.rpos = (int32_t*)take((size_t)f->m * 4);
    om.cpos = (int32_t*)take((size_t)S * C * 4);
    om.rtb = (int32_t*)take(t_sell * 4);
    om.ctb = (int32_t*)take(t_sell * 4);
    om.rbase = (int64_t*)take((size_t)(S + 1) * 8);
    om.cbase = (int64_t*)take((size_t)(S + 1) * 8);
    om.sidx_r = (uint16_t*)take(e_sell * 2);
    om.sval_r = (float*)take(e_sell * 4);
    om.sidx_c = (uint16_t*)take(e_sell * 2);
    om.sval_c = (float*)take(e_sell * 4);
    float* part = (float*)take((size_t)S * kOmParts * 4);  // partial sums of the observed values
    if ((size_t)(p - (char*)ctx->scr[SCR_OMEGA]) > ctx->scr_size[SCR_OMEGA])
        return lt_fail(ctx, LT_ENOMEM, "omega_build: layout overflow");
    const int nsm = ctx->num_sms;
    k_om_clear<<<dim3(std::max(1, 2 * nsm / S), S), 256, 0, ctx->stream>>>(*f, *smp, om);
    LT_LAUNCH_CHECK(ctx, "k_om_clear");
    k_om_bits<<<dim3(kOmParts, S), 256, 0, ctx->stream>>>(*f, *smp, om, part, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_om_bits");
    k_om_lines<<<dim3(std::max(1, 4 * nsm / S), S), 256, 0, ctx->stream>>>(*f, *smp, om);
    LT_LAUNCH_CHECK(ctx, "k_om_lines");
    k_om_scan<<<S, 1024, 0, ctx->stream>>>(*f, *smp, om, part, kOmParts);
    LT_LAUNCH_CHECK(ctx, "k_om_scan");
    if (om.sell) {
        k_om_sellpfx<<<1, 1024, 0, ctx->stream>>>(S, om, ctx->d_status);
        LT_LAUNCH_CHECK(ctx, "k_om_sellpfx");
    }
    k_om_scatter<<<dim3(std::max(1, 4 * nsm / S), S), 256, 0, ctx->stream>>>(*f, *smp, om);
    LT_LAUNCH_CHECK(ctx, "k_om_scatter");
    k_line_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, S, om.line_pfx);
    LT_LAUNCH_CHECK(ctx, "k_line_prefix");
    return LT_OK;
}

}  // namespace ltk

namespace {

// The previous frame's columns and factors that start a frame's completion
struct WarmStart {
    const int32_t* col_node;   // [S][C] tree node of each previous column
    const int32_t* ncol;       // [S]    previous columns per slice
    const float* V;            // [S][C][R] previous V rows
};

// Temporal coherence: column c of slice s whose node was a column i of the previous
// frame's slice s starts from the previous V row i (components below the slice's
// rank; the previous rows are zero beyond their own rank), the others keep the
// seeded start.  One CTA per slice; the previous node list is staged in shared memory
// and searched linearly (the cut is not sorted by node id).
__global__ void __launch_bounds__(256) k_als_warm(lt_frame F, lt_samples smp, int R, const int32_t* __restrict__ rk,
                                                  WarmStart w, float* __restrict__ V) {
    extern __shared__ int32_t pn[];
    const int s = blockIdx.x;
    const int np = min(w.ncol[s], F.C), ns = smp.ncol[s];
    for (int i = threadIdx.x; i < np; i += blockDim.x) pn[i] = w.col_node[(int64_t)s * F.C + i];
    __syncthreads();
    const int r = slice_rank(rk, s, R);
    for (int c = threadIdx.x; c < ns; c += blockDim.x) {
        const int node = smp.col_node[(int64_t)s * F.C + c];
        int hit = -1;
        for (int i = 0; i < np; ++i)
            if (pn[i] == node) {
                hit = i;
                break;
            }
        if (hit < 0) continue;
        const float* src = w.V + ((int64_t)s * F.C + hit) * R;
        float* dst = V + ((int64_t)s * F.C + c) * R;
        for (int k = 0; k < R; ++k) dst[k] = k < r ? src[k] : 0.f;
    }
}

lt_status complete_impl(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters, float lam_rel,
                        uint64_t seed, lt_factors* uv, const WarmStart* warm) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->key || !smp->val || !smp->off || !smp->cnt || !smp->ncol || !uv ||
        !uv->U || !uv->V || uv->r < 1 || uv->r > 32 || iters < 0 || !(lam_rel >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_complete: bad arguments");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C;
    // The sampling capacity sizes the scratch; a captured frame reuses the recorded value.
    int64_t E = 0;
    if (ctx->use_plan) {
        E = ctx->plan.entries;
    } else {
        LT_CUDA(ctx, cudaMemcpyAsync(&E, smp->off + S, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->plan.entries = E;
    }
    const int64_t mr = std::max(f->max_rows, 1);
    const int R = uv->r;            // stride of the factor rows, the largest rank
    const int32_t* rk = uv->rank;   // per-slice ranks (NULL: R for every slice)
    // Slices of rank <= 16 go to the tensor-core form (CSR / CSC) or the lane-group
    // SIMT kernel (sliced layout), as tuned; the warp-group ALS takes the others
    // (CSR / CSC); with per-slice ranks above 16 two of them run.
    const bool low = R <= 16 || rk != nullptr;
    const bool tc = low && ctx->tune.als_form == 1;
    Omega om;
    lt_status st = omega_build(ctx, f, smp, E, low && !tc, R > 16 || tc, &om);
    if (st != LT_OK) return st;
    const int RP = R <= 8 ? 8 : 16;  // the low-rank kernels cover ranks up to RP
    // per half-step retry counters (one set for ranks <= 16, one above) and the
    // float64 count
    const bool high = R > 16;
    const int nq = std::max(1, 2 * iters);
    char* sp = (char*)lt_scratch(ctx, SCR_ALS, (size_t)(2 * nq + 64) * 4 + 256, &st);
    if (!sp) return st;
    int32_t* n64 = (int32_t*)sp;
    int32_t* qcount = n64 + 64;
    int32_t* qcount_hi = qcount + nq;
    LT_CUDA(ctx, cudaMemsetAsync(n64, 0, (size_t)(2 * nq + 64) * 4, ctx->stream));
    const int nsm = ctx->num_sms;
    k_als_init<<<dim3(8, S), 256, 0, ctx->stream>>>(*f, *smp, om, R, rk, seed_ref(ctx, seed), uv->V);
    LT_LAUNCH_CHECK(ctx, "k_als_init");
    if (warm) {
        const size_t shm = (size_t)C * 4;
        if (shm > 48 * 1024)
            LT_CUDA(ctx, cudaFuncSetAttribute(k_als_warm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
        k_als_warm<<<S, 256, shm, ctx->stream>>>(*f, *smp, R, rk, *warm, uv->V);
        LT_LAUNCH_CHECK(ctx, "k_als_warm");
    }
    // lane-group kernel: one thread (group) per line; one 256-thread CTA per SM stages
    // the slice's factor rows (up to 110 KB) and leaves the rest of the SM to L1
    const size_t row_bytes = (size_t)RP * 4;
    const int stage_rows = (int)std::min<int64_t>((110 * 1024) / row_bytes, std::max<int64_t>(mr, C));
    const size_t dyn = (size_t)stage_rows * row_bytes;
    const int64_t cap = std::min<int64_t>(std::max<int64_t>(f->m, (int64_t)S * C), 1 << 18);
    int64_t *qdst = nullptr, *qslot = nullptr, *qsrc = nullptr;
    int32_t *qlen = nullptr, *qgrp = nullptr, *qrank = nullptr;
    AlsQueue<32> qhi{};
    if (low || high) {
        const size_t a8 = ((size_t)cap * 8 + 255) & ~(size_t)255, a4 = ((size_t)cap * 4 + 255) & ~(size_t)255;
        const size_t set = 3 * a8 + 3 * a4;
        char* qp = (char*)lt_scratch(ctx, SCR_GRAM, 2 * set, &st);
        if (!qp) return st;
        char* hp = qp + set;  // the queue of the lines above rank 16
        qhi = AlsQueue<32>{nullptr, (int64_t*)hp, (int64_t*)(hp + a8), (int64_t*)(hp + 2 * a8),
                           (int32_t*)(hp + 3 * a8), (int32_t*)(hp + 3 * a8 + a4), (int32_t*)(hp + 3 * a8 + 2 * a4),
                           cap, ctx->d_status};
        qdst = (int64_t*)qp;
        qslot = (int64_t*)(qp + a8);
        qsrc = (int64_t*)(qp + 2 * a8);
        qlen = (int32_t*)(qp + 3 * a8);
        qgrp = (int32_t*)(qp + 3 * a8 + a4);
        qrank = (int32_t*)(qp + 3 * a8 + 2 * a4);
    }
    if (om.sell) {
        if (RP == 8)
            LT_CUDA(ctx, cudaFuncSetAttribute(k_als_line<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
        else
            LT_CUDA(ctx, cudaFuncSetAttribute(k_als_line<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    }
    // warp-per-line kernel for ranks above 16: each slice's lines split over P CTAs
    // (about 16 CTAs per SM in all, so that uneven slices balance)
    const int P = std::max(1, (16 * ctx->num_sms + S - 1) / S);
    TcPlan tcp{};
    if (tc) {
        st = als_tc_plan(ctx, f, smp, om, E, R, rk, RP, 2 * iters, &tcp);
        if (st != LT_OK) return st;
    }
    for (int it = 0; it < iters; ++it) {
        for (int side = 0; side < 2; ++side) {
            const bool rows = side == 0;
            const float* fin = rows ? uv->V : uv->U;
            float* fout = rows ? uv->U : uv->V;
            int32_t* cnt = qcount + 2 * it + side;
            if (tc) {
                TcQueue tq{cnt, qdst, qslot, qsrc, qlen, qgrp, qrank, cap, ctx->d_status};
                st = als_tc_half(ctx, f, smp, om, R, rk, rows, fin, fout, lam_rel, tcp, 2 * it + side, tq, nullptr);
                if (st != LT_OK) return st;
                if (RP == 8) {
                    AlsQueue<8> q{cnt, qdst, qslot, qsrc, qlen, qgrp, qrank, cap, ctx->d_status};
                    k_als_retry<8><<<nsm, 128, 0, ctx->stream>>>(q, om, rows, fin, R, lam_rel, fout, n64);
                } else {
                    AlsQueue<16> q{cnt, qdst, qslot, qsrc, qlen, qgrp, qrank, cap, ctx->d_status};
                    k_als_retry<16><<<nsm, 128, 0, ctx->stream>>>(q, om, rows, fin, R, lam_rel, fout, n64);
                }
                LT_LAUNCH_CHECK(ctx, "k_als_retry");
            } else if (om.sell && RP == 8) {
                AlsQueue<8> q{cnt, qdst, qslot, qsrc, qlen, qgrp, qrank, cap, ctx->d_status};
                k_als_line<8><<<nsm, 256, dyn, ctx->stream>>>(*f, *smp, om, R, rk, rows, fin, fout, lam_rel, q,
                                                              stage_rows);
                LT_LAUNCH_CHECK(ctx, "k_als_line");
                k_als_retry<8><<<nsm, 128, 0, ctx->stream>>>(q, om, rows, fin, R, lam_rel, fout, n64);
                LT_LAUNCH_CHECK(ctx, "k_als_retry");
            } else if (om.sell) {
                AlsQueue<16> q{cnt, qdst, qslot, qsrc, qlen, qgrp, qrank, cap, ctx->d_status};
                k_als_line<16><<<nsm, 256, dyn, ctx->stream>>>(*f, *smp, om, R, rk, rows, fin, fout, lam_rel, q,
                                                               stage_rows);
                LT_LAUNCH_CHECK(ctx, "k_als_line");
                k_als_retry<16><<<nsm, 128, 0, ctx->stream>>>(q, om, rows, fin, R, lam_rel, fout, n64);
                LT_LAUNCH_CHECK(ctx, "k_als_retry");
            }
            if (high) {
                AlsQueue<32> q = qhi;
                q.count = qcount_hi + 2 * it + side;
                k_als_half<32><<<dim3(P, S), 32 * als_warps<32>(), 0, ctx->stream>>>(
                    *f, *smp, om, R, rk, lam_rel, rows, fin, fout, q);
                LT_LAUNCH_CHECK(ctx, "k_als_half");
                k_als_retry<32><<<nsm, 128, 0, ctx->stream>>>(q, om, rows, fin, R, lam_rel, fout, n64);
                LT_LAUNCH_CHECK(ctx, "k_als_retry");
            }
        }
    }
    return LT_OK;
}

}  // namespace

extern "C" lt_status lt_complete(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                                 float lam_rel, uint64_t seed, lt_factors* uv) {
    return complete_impl(ctx, f, smp, iters, lam_rel, seed, uv, nullptr);
}

extern "C" lt_status lt_complete_warm(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                                      float lam_rel, uint64_t seed, const int32_t* prev_col_node,
                                      const int32_t* prev_ncol, const float* prev_V, lt_factors* uv) {
    if (!prev_col_node || !prev_ncol || !prev_V || (uv && prev_V == uv->V))
        return lt_fail(ctx, LT_EINVAL, "lt_complete_warm: bad arguments");
    const WarmStart w{prev_col_node, prev_ncol, prev_V};
    return complete_impl(ctx, f, smp, iters, lam_rel, seed, uv, &w);
}

extern "C" lt_status lt_als_gram(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_factors* uv,
                                 int32_t side, float* gram) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->key || !smp->val || !smp->off || !smp->cnt || !smp->ncol || !uv ||
        !uv->U || !uv->V || uv->r < 1 || uv->r > 16 || uv->rank || (side != 0 && side != 1) || !gram)
        return lt_fail(ctx, LT_EINVAL, "lt_als_gram: bad arguments");
    cudaSetDevice(ctx->device);
    int64_t E = 0;
    LT_CUDA(ctx, cudaMemcpyAsync(&E, smp->off + f->S, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    Omega om;
    lt_status st = omega_build(ctx, f, smp, E, false, true, &om);
    if (st != LT_OK) return st;
    const int R = uv->r, RP = R <= 8 ? 8 : 16;
    TcPlan tcp{};
    st = als_tc_plan(ctx, f, smp, om, E, R, nullptr, RP, 1, &tcp);
    if (st != LT_OK) return st;
    const TcQueue none{};
    return als_tc_half(ctx, f, smp, om, R, nullptr, side == 0, side == 0 ? uv->V : uv->U, nullptr, 0.f, tcp, 0, none,
                       gram);
}

extern "C" lt_status lt_complete_fp64_lines(lt_ctx* ctx, int64_t* count_host) {
    if (!ctx || !count_host) return lt_fail(ctx, LT_EINVAL, "lt_complete_fp64_lines: bad arguments");
    *count_host = 0;
    if (!ctx->scr[SCR_ALS]) return LT_OK;  // no lt_complete ran on this context yet
    cudaSetDevice(ctx->device);
    int32_t v = 0;  // word 0 of the ALS scratch: the float64 count of the last lt_complete
    LT_CUDA(ctx, cudaMemcpyAsync(&v, ctx->scr[SCR_ALS], sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *count_host = v;
    return LT_OK;
}

extern "C" lt_status lt_slice_ranks(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t R, int32_t cols,
                                    int32_t* rank) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->ncol || !rank || R < 1 || R > 32 || cols < 1)
        return lt_fail(ctx, LT_EINVAL, "lt_slice_ranks: bad arguments");
    cudaSetDevice(ctx->device);
    k_slice_ranks<<<(f->S + 255) / 256, 256, 0, ctx->stream>>>(*smp, f->S, R, cols, rank);
    LT_LAUNCH_CHECK(ctx, "k_slice_ranks");
    return LT_OK;
}

extern "C" lt_status lt_render(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_factors* uv,
                               const float* w, const int32_t* row_perm, float* img) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->ncol || !uv || !uv->U || !uv->V || uv->r < 1 || uv->r > 32 ||
        !row_perm || !img)
        return lt_fail(ctx, LT_EINVAL, "lt_render: bad arguments");
    cudaSetDevice(ctx->device);
    const int per = std::max(1, std::min(64, (int)((f->max_rows + 511) / 512)));
    k_render<<<dim3(per, f->S), 512, 0, ctx->stream>>>(*f, *smp, uv->U, uv->V, uv->r, w, row_perm, img);
    LT_LAUNCH_CHECK(ctx, "k_render");
    return LT_OK;
}
