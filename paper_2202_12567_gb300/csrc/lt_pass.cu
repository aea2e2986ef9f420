// Sampling passes of the sparse renderer.
//
//  * Pass 1 and light coarsening (Sec. 4, Eq. 2): the cut nodes of every slice draw
//    their k_c rows and evaluate them (one kernel over all slices), then the cut's
//    ancestor forest is walked level by level with a few kernels per level over all
//    slices: sibling pairs are laid out as the union zeta_f = zeta_a U zeta_b (one
//    thread per small pair, one CTA per big pair), the entries missing from either
//    child are queued and evaluated one shadow ray per thread, and each pair merges
//    when cost = eps + cost(q) < tau * S_hat, eps = max |V_q - V_p I_q / I_p| (in a dark
//    slice, S_hat = 0, when the cost is exactly zero).
//  * Pass 2 (Sec. 5, Eq. 3): per slice one cluster of eight CTAs draws (column from
//    the integer CDF of g or of given weights, row uniform) in rounds, keeps the
//    first occurrence of every new entry in draw order, and stops at
//    ceil(rate m' n') entries.
//  * Entry evaluation: one thread per pass-2 entry (one shadow ray), the column side
//    read from per-frame column records (k_col_records).
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr int kP1Threads = 512;
constexpr int kMaxRowsPerNode = 64;
constexpr int kMaxDraws = 1 << 16;
constexpr int kMaxCut = 16384;
constexpr int kStNot = 0, kStAlive = 1, kStDead = 2, kStRejected = 3;

struct P1Plan {
    int32_t* k;        // [S][C]   rows per cut node
    int32_t* cap;      // [S][NF]  storage capacity per forest node
    int32_t* off;      // [S][NF]  storage offset inside the slice's region
    int32_t* cnt;      // [S][NF]  current |zeta|
    int32_t* state;    // [S][NF]
    float* cost;       // [S][NF]
    int32_t* pfx;      // [S][C+1] prefix of k
    int32_t* colx;     // [S][C]   forest node of each output column
    int32_t* eoff;     // [S][C]   output offset of each column
    int64_t* total;    // [S]      storage slots of the slice
    int64_t* base;     // [S]      start of the slice's storage
};

__device__ __forceinline__ float node_scale(const lt_tree& T, const float4* __restrict__ vpls, int64_t n, int node) {
    const int r = T.rep[node];
    const float flux = __ldg(&vpls[2 * n + r].w);
    const float alb = __ldg(&vpls[r].w);
    return __fdiv_rn(T.I[node], __fmul_rn(flux, alb));
}

// Chunked exclusive scan over an array in global memory; returns the total.
__device__ int block_scan_array(const int32_t* in, int32_t* out, int count, int32_t* warp_sums) {
    int carry = 0;
    for (int c0 = 0; c0 < count; c0 += blockDim.x) {
        const int i = c0 + threadIdx.x;
        const int x = i < count ? in[i] : 0;
        int tot;
        const int pre = block_exclusive_scan<int>(x, warp_sums, &tot);
        if (i < count) out[i] = carry + pre;
        carry += tot;
    }
    return carry;
}

// ------------------------------------------------------------------ pass 1: plan
__global__ void __launch_bounds__(kP1Threads) k_pass1_plan(lt_frame F, float rate1, P1Plan pl) {
    __shared__ int32_t ws[32];
    const int s = blockIdx.x;
    const int C = F.C, NF = 2 * C - 1;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    int32_t* k = pl.k + (int64_t)s * C;
    int32_t* cap = pl.cap + (int64_t)s * NF;
    int32_t* off = pl.off + (int64_t)s * NF;
    int32_t* pfx = pl.pfx + (int64_t)s * (C + 1);
    const float kappa = fmaxf(2.0f, __fmul_rn(rate1, (float)ms));
    const float Iroot = F.tree.I[0];
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int node = F.forest[8 * c];
        const float x = __fmul_rn(__fmul_rn(kappa, (float)C), __fdiv_rn(F.tree.I[node], Iroot));
        int kc = (int)floorf(__fadd_rn(x, 0.5f));
        kc = min(max(kc, 2), kMaxRowsPerNode);
        kc = min(kc, ms);
        k[c] = kc;
    }
    __syncthreads();
    const int K = block_scan_array(k, pfx, C, ws);
    if (threadIdx.x == 0) pfx[C] = K;
    __syncthreads();
    for (int x = threadIdx.x; x < NF; x += blockDim.x) {
        const int* fx = F.forest + 8 * x;
        cap[x] = x < C ? k[x] : min(ms, pfx[fx[5] + 1] - pfx[fx[4]]);
    }
    __syncthreads();
    const int tot = block_scan_array(cap, off, NF, ws);
    if (threadIdx.x == 0) pl.total[s] = tot;
}

// ------------------------------------------------------------------ pass 1: flat kernels
// Every step below runs over all slices at once.  Per forest level: setup lays out
// the union of each testable sibling pair and queues the entries it lacks (small
// pairs by a thread, big ones by a CTA), rays evaluates the queue (one shadow ray
// per thread), decide reduces eps, applies Eq. 2 and merges or rejects.  The levels
// run either as separate launches per step (the default: on the 256x256, 16K-VPL
// frame 2.07 ms) or inside one persistent cooperative launch with grid-wide
// barriers between the steps (k_p1_walk, 2.52 ms there: the steps are chains of
// dependent loads, and a grid barrier costs more than a launch inside a graph).

struct P1Store {
    int32_t* rows;     // [total] row of each storage slot
    float* v0;         // [total]  (V_a, or V_f after a merge)
    float* v1;         // [total]  (V_b), == v0 + total
    float* v2;         // [total]  V_a kept at a merge (coarsening to a target size), else null
    int64_t total;
};

struct P1Work {
    int64_t* kpfx;     // [S+1] prefix over slices of the initial entry counts
    float* leafmean;   // [S][C] mean of each cut node's initial entries
    float* thr;        // [S] tau * S_hat (-1 in a dark slice, S_hat = 0)
    int64_t* mcount;   // [Hmax] queued missing entries per level
    int64_t* bcount;   // [Hmax] big pairs per level
    int64_t* mdst;     // [mcap] flat value index (v0 or v1) of a missing entry
    int32_t* mpt;      // [mcap] slice-ordered point of the entry
    int32_t* mnode;    // [mcap] tree node of the entry's column
    int64_t* big;      // [bcap] flat pair index of a big pair
    unsigned* bar;     // arrival counter of the persistent walk's grid barriers
    int64_t mcap, bcap;
};

// -- draws of the cut nodes and state of every forest node
__global__ void k_p1_draws(lt_frame F, SeedRef sr, P1Plan pl, P1Store st, int32_t* status) {
    const int C = F.C, NF = 2 * C - 1;
    const uint64_t seed = sr.get();
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)F.S * NF;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx / NF), x = (int)(idx % NF);
        const int ms = F.slice_off[s + 1] - F.slice_off[s];
        int32_t* cnt = pl.cnt + (int64_t)s * NF;
        int32_t* state = pl.state + (int64_t)s * NF;
        float* cost = pl.cost + (int64_t)s * NF;
        cost[x] = 0.f;
        if (x >= C) {
            cnt[x] = 0;
            state[x] = kStNot;
            continue;
        }
        const int k = pl.k[(int64_t)s * C + x];
        int32_t* r = st.rows + pl.base[s] + pl.off[(int64_t)s * NF + x];
        int got = 0;
        if (k >= ms) {
            for (int t = 0; t < ms; ++t) r[t] = t;
            got = ms;
        } else {
            for (int t = 0; got < k && t < kMaxDraws; ++t) {
                const int v = (int)uniform_index(philox((uint32_t)t, (uint32_t)x, slice_key(F.slice_id, s), kTagPass1, seed).x,
                                                 (uint32_t)ms);
                bool dup = false;
                for (int q = 0; q < got; ++q) dup |= (r[q] == v);
                if (!dup) r[got++] = v;
            }
            if (got < k) latch(status, LT_ELIMIT);
            for (int a = 1; a < got; ++a) {  // insertion sort, got <= 64
                const int v = r[a];
                int b = a - 1;
                while (b >= 0 && r[b] > v) {
                    r[b + 1] = r[b];
                    --b;
                }
                r[b + 1] = v;
            }
        }
        cnt[x] = got;
        state[x] = ms > 0 ? kStAlive : kStNot;
    }
}

// -- first row slot of every slice: exclusive prefix of the per-slice totals
__global__ void k_p1_base(int S, P1Plan pl) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < S ? pl.total[s] : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < S) pl.base[s] = carry + pre;
        carry += tot;
    }
}

__global__ void k_p1_kpfx(lt_frame F, P1Plan pl, int64_t* kpfx) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < F.S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < F.S ? (int64_t)pl.pfx[(int64_t)s * (F.C + 1) + F.C] : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < F.S) kpfx[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) kpfx[F.S] = carry;
}

// -- initial entries of every cut node of every slice (one shadow ray per thread)
__global__ void __launch_bounds__(128) k_p1_initial(lt_frame F, Grid g, float dmin2, P1Plan pl, P1Store st,
                                                    const int64_t* __restrict__ kpfx, int32_t* status) {
    const float4* pts = reinterpret_cast<const float4*>(F.pts);
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    const int C = F.C, NF = 2 * C - 1;
    const int64_t total = kpfx[F.S];
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = F.S;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (kpfx[mid] <= idx) lo = mid;
            else hi = mid;
        }
        const int s = lo;
        const int e = (int)(idx - kpfx[s]);
        const int32_t* pf = pl.pfx + (int64_t)s * (C + 1);
        int a = 0, b = C;  // largest c with pf[c] <= e
        while (b - a > 1) {
            const int mid = (a + b) >> 1;
            if (pf[mid] <= e) a = mid;
            else b = mid;
        }
        const int c = a, t = e - pf[c];
        const int64_t slot = pl.base[s] + pl.off[(int64_t)s * NF + c] + t;
        const int node = F.forest[8 * c];
        const PointRec P = load_rec(pts, F.m, F.slice_off[s] + st.rows[slot]);
        const PointRec L = load_rec(vpls, F.n, F.tree.rep[node]);
        const float v = entry_value(P, L, node_scale(F.tree, vpls, F.n, node), dmin2, g);
        if (!isfinite(v)) latch(status, LT_ENUMERIC);  // a non-finite input (flux, albedo, position)
        st.v0[slot] = v;
    }
}

__global__ void k_p1_leafmean(lt_frame F, P1Plan pl, P1Store st, float* leafmean) {
    const int C = F.C, NF = 2 * C - 1;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < (int64_t)F.S * C;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int s = (int)(idx / C), c = (int)(idx % C);
        const int n = pl.cnt[(int64_t)s * NF + c];
        const float* v = st.v0 + pl.base[s] + pl.off[(int64_t)s * NF + c];
        float sum = 0.f;
        for (int t = 0; t < n; ++t) sum += v[t];
        leafmean[idx] = n > 0 ? sum / (float)n : 0.f;
    }
}

// tau * S_hat per slice, S_hat = sum_c mean(V_c) (fixed reduction order).  A dark
// slice (S_hat = 0: every pass-1 entry is zero) gets -1: its relative bound is zero,
// and it is read as met by a pair whose cost is exactly zero (the samples cannot
// tell the two lights apart), so such a slice coarsens as far as its entries agree.
__global__ void k_p1_thr(lt_frame F, const float* __restrict__ leafmean, float tau, float* thr) {
    __shared__ float red[32];
    const int s = blockIdx.x;
    float sum = 0.f;
    for (int c = threadIdx.x; c < F.C; c += blockDim.x) sum += leafmean[(int64_t)s * F.C + c];
    sum = warp_sum(sum);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = sum;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        thr[s] = t > 0.f ? tau * t : -1.f;
    }
}

// -- coarsening to a target cut size (Sec. 4): every pair is tested (threshold +inf,
// so all merge and every internal node gets its cost); then per slice the C - target
// pairs of smallest effective cost eff(f) = max(cost(f), eff(a), eff(b)) (ties: lower
// height, lower id) are the merged ones.  Merging by least cost among the testable
// pairs, one at a time, merges exactly those: a pair becomes testable only after its
// children merged, and the effective cost is the cost at which the greedy order
// reaches it.
__global__ void k_p1_thr_inf(int S, float* thr) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) thr[s] = INFINITY;
}

__device__ __forceinline__ unsigned long long eff_key(const lt_frame& F, const float* eff, int f) {
    return (unsigned long long)__float_as_uint(eff[f]) << 32 | (unsigned long long)F.forest[8 * f + 6] << 20 |
           (unsigned long long)(f - F.C);
}

__global__ void __launch_bounds__(1024) k_p1_target(lt_frame F, P1Plan pl, float* __restrict__ effs, int target) {
    __shared__ int32_t hist[256];
    __shared__ unsigned long long sel[2];
    __shared__ int32_t krem;
    const int s = blockIdx.x;
    const int C = F.C, NF = 2 * C - 1;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    if (ms == 0) return;
    const float* cost = pl.cost + (int64_t)s * NF;
    int32_t* state = pl.state + (int64_t)s * NF;
    float* eff = effs + (int64_t)s * NF;
    for (int x = threadIdx.x; x < C; x += blockDim.x) eff[x] = 0.f;
    __syncthreads();
    for (int h = 1; h <= F.H; ++h) {
        for (int i = F.level_off[h] + threadIdx.x; i < F.level_off[h + 1]; i += blockDim.x) {
            const int f = F.level_nodes[i];
            eff[f] = fmaxf(cost[f], fmaxf(eff[F.forest[8 * f + 1]], eff[F.forest[8 * f + 2]]));
        }
        __syncthreads();
    }
    const int K = max(0, min(C - target, C - 1));
    if (threadIdx.x == 0) {
        sel[0] = sel[1] = 0ull;
        krem = K - 1;
    }
    __syncthreads();
    for (int pass = 7; pass >= 0 && K > 0; --pass) {  // radix select of the K-th smallest key
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned long long prefix = sel[0], mask = sel[1];
        for (int f = C + threadIdx.x; f < NF; f += blockDim.x) {
            const unsigned long long key = eff_key(F, eff, f);
            if ((key & mask) == prefix) atomicAdd(&hist[(key >> (8 * pass)) & 255], 1);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int k = krem, digit = 255;
            for (int b = 0; b < 256; ++b) {
                if (k < hist[b]) {
                    digit = b;
                    break;
                }
                k -= hist[b];
            }
            krem = k;
            sel[0] = prefix | ((unsigned long long)digit << (8 * pass));
            sel[1] = mask | (255ull << (8 * pass));
        }
        __syncthreads();
    }
    const unsigned long long pivot = sel[0];
    auto merged = [&](int x) { return x >= C && K > 0 && eff_key(F, eff, x) <= pivot; };
    for (int x = threadIdx.x; x < NF; x += blockDim.x) {
        const bool chosen = x < C || merged(x);
        const int par = F.forest[8 * x + 3];
        int stt;
        if (chosen) {
            stt = (par >= 0 && merged(par)) ? kStDead : kStAlive;
        } else {
            const int a = F.forest[8 * x + 1], b = F.forest[8 * x + 2];
            const bool ca = a < C || merged(a), cb = b < C || merged(b);
            stt = (ca && cb) ? kStRejected : kStNot;
        }
        state[x] = stt;
    }
}

struct PairCtx {
    int s, f, a, b, na, nb, row0;
    int64_t base;
    const int32_t* ra;
    const int32_t* rb;
    int64_t ia, ib, iff;   // storage offsets of a, b, f inside the slice's region
};

__device__ __forceinline__ bool load_pair(const lt_frame& F, const P1Plan& pl, const P1Store& st, int h, int64_t t,
                                          PairCtx& pc) {
    const int l0 = F.level_off[h], np = F.level_off[h + 1] - l0;
    const int NF = 2 * F.C - 1;
    pc.s = (int)(t / np);
    pc.f = F.level_nodes[l0 + (int)(t % np)];
    pc.a = F.forest[8 * pc.f + 1];
    pc.b = F.forest[8 * pc.f + 2];
    const int32_t* state = pl.state + (int64_t)pc.s * NF;
    if (state[pc.a] != kStAlive || state[pc.b] != kStAlive) return false;
    const int32_t* cnt = pl.cnt + (int64_t)pc.s * NF;
    const int32_t* off = pl.off + (int64_t)pc.s * NF;
    pc.na = cnt[pc.a];
    pc.nb = cnt[pc.b];
    pc.base = pl.base[pc.s];
    pc.ia = pc.base + off[pc.a];
    pc.ib = pc.base + off[pc.b];
    pc.iff = pc.base + off[pc.f];
    pc.ra = st.rows + pc.ia;
    pc.rb = st.rows + pc.ib;
    pc.row0 = F.slice_off[pc.s];
    return true;
}

// Reserve n queue slots for each lane of the warp with one atomic per warp; returns
// this lane's first slot.  Every lane of the warp must call it.
__device__ __forceinline__ long long warp_reserve(unsigned long long* counter, int n) {
    const int lane = threadIdx.x & 31;
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total > 0) base = atomicAdd(counter, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return (long long)base + (incl - n);
}

__device__ __forceinline__ void put_missing(const P1Work& w, long long q, int64_t dst, int pt, int node,
                                            int32_t* status) {
    if (q < w.mcap) {
        w.mdst[q] = dst;
        w.mpt[q] = pt;
        w.mnode[q] = node;
    } else {
        latch(status, LT_ELIMIT);
    }
}

// -- level h, step 1: union layout of every testable pair, queue of missing entries.
// A pair of at most kThreadPair rows is laid out by one thread (a serial merge of
// the two sorted lists, once to count the rows that only one list holds and once to
// write), a bigger one by a CTA (queued as big).
constexpr int kThreadPair = 64;

__device__ __forceinline__ bool pair_big(const PairCtx& pc) { return pc.na + pc.nb > kThreadPair; }

__device__ __forceinline__ int serial_missing(const PairCtx& pc) {
    int i = 0, j = 0, nmiss = 0;
    while (i < pc.na || j < pc.nb) {
        const int xa = i < pc.na ? pc.ra[i] : 0x7fffffff, xb = j < pc.nb ? pc.rb[j] : 0x7fffffff;
        if (xa < xb) ++i, ++nmiss;
        else if (xb < xa) ++j, ++nmiss;
        else ++i, ++j;
    }
    return nmiss;
}

__device__ __forceinline__ void serial_write(const lt_frame& F, const P1Plan& pl, const P1Store& st, const P1Work& w,
                                             const PairCtx& pc, long long q, int32_t* status) {
    const int ta = F.forest[8 * pc.a], tb = F.forest[8 * pc.b];
    int32_t* rf = st.rows + pc.iff;
    float* fa = st.v0 + pc.iff;
    float* fb = st.v1 + pc.iff;
    int i = 0, j = 0, n = 0;
    while (i < pc.na || j < pc.nb) {
        const int xa = i < pc.na ? pc.ra[i] : 0x7fffffff, xb = j < pc.nb ? pc.rb[j] : 0x7fffffff;
        if (xa < xb) {
            rf[n] = xa;
            fa[n] = st.v0[pc.ia + i++];
            put_missing(w, q++, st.total + pc.iff + n, pc.row0 + xa, tb, status);   // V_b(xa)
        } else if (xb < xa) {
            rf[n] = xb;
            fb[n] = st.v0[pc.ib + j++];
            put_missing(w, q++, pc.iff + n, pc.row0 + xb, ta, status);              // V_a(xb)
        } else {
            rf[n] = xa;
            fa[n] = st.v0[pc.ia + i++];
            fb[n] = st.v0[pc.ib + j++];
        }
        ++n;
    }
    pl.cnt[(int64_t)pc.s * (2 * F.C - 1) + pc.f] = n;
}

__device__ __forceinline__ void p1_setup_body(const lt_frame& F, const P1Plan& pl, const P1Store& st, const P1Work& w,
                                              int h, int32_t* status) {
    const int np = F.level_off[h + 1] - F.level_off[h];
    const int64_t npairs = (int64_t)F.S * np;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // warp-uniform trip count so that every lane takes part in the reservations
    for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x; t0 < npairs; t0 += stride) {
        const int64_t t = t0 + threadIdx.x;
        PairCtx pc;
        const bool active = t < npairs && load_pair(F, pl, st, h, t, pc);
        const bool big = active && pair_big(pc);
        const long long qb = warp_reserve((unsigned long long*)&w.bcount[h], big ? 1 : 0);
        if (big) {
            if (qb < w.bcap) w.big[qb] = t;
            else latch(status, LT_ELIMIT);
        }
        const bool mine = active && !big;
        const long long q = warp_reserve((unsigned long long*)&w.mcount[h], mine ? serial_missing(pc) : 0);
        if (mine) serial_write(F, pl, st, w, pc, q, status);
    }
}

// big pairs, one CTA per pair: both sorted row lists staged in shared memory (global
// reads beyond kBigStage rows), the slot of a row from its rank in the other list
// (binary search) and a block scan of the "in both" flags
constexpr int kBigStage = 4096;

__device__ __forceinline__ void p1_setup_big_body(const lt_frame& F, const P1Plan& pl, const P1Store& st,
                                                  const P1Work& w, int h, int32_t* status) {
    __shared__ int32_t sa[kBigStage], sb[kBigStage];
    __shared__ int32_t ws[32];
    const int NF = 2 * F.C - 1;
    const int64_t nbig = min(w.bcount[h], w.bcap);
    for (int64_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        PairCtx pc;
        if (!load_pair(F, pl, st, h, w.big[q], pc)) continue;  // uniform in the block
        const int ta = F.forest[8 * pc.a], tb = F.forest[8 * pc.b];
        const bool staged = pc.na <= kBigStage && pc.nb <= kBigStage;
        __syncthreads();  // the previous pair is done with the stage
        if (staged) {
            for (int i = threadIdx.x; i < pc.na; i += blockDim.x) sa[i] = pc.ra[i];
            for (int j = threadIdx.x; j < pc.nb; j += blockDim.x) sb[j] = pc.rb[j];
        }
        __syncthreads();
        const int32_t* A = staged ? sa : pc.ra;
        const int32_t* B = staged ? sb : pc.rb;
        int32_t* rf = st.rows + pc.iff;
        float* fa = st.v0 + pc.iff;
        float* fb = st.v1 + pc.iff;
        int common = 0;
        for (int i0 = 0; i0 < pc.na; i0 += blockDim.x) {
            const int i = i0 + threadIdx.x;
            int x = 0, pb = 0;
            bool both = false;
            if (i < pc.na) {
                x = A[i];
                pb = lower_bound<int32_t>(B, pc.nb, x);
                both = pb < pc.nb && B[pb] == x;
            }
            int tot;
            const int pre = block_exclusive_scan<int>(both ? 1 : 0, ws, &tot);
            const long long m = warp_reserve((unsigned long long*)&w.mcount[h], (i < pc.na && !both) ? 1 : 0);
            if (i < pc.na) {
                const int slot = i + pb - (common + pre);
                rf[slot] = x;
                fa[slot] = st.v0[pc.ia + i];
                if (both) fb[slot] = st.v0[pc.ib + pb];
                else put_missing(w, m, st.total + pc.iff + slot, pc.row0 + x, tb, status);   // V_b(x)
            }
            common += tot;
        }
        int seen = 0;
        for (int j0 = 0; j0 < pc.nb; j0 += blockDim.x) {
            const int j = j0 + threadIdx.x;
            int y = 0, pa = 0;
            bool both = false;
            if (j < pc.nb) {
                y = B[j];
                pa = lower_bound<int32_t>(A, pc.na, y);
                both = pa < pc.na && A[pa] == y;
            }
            int tot;
            const int pre = block_exclusive_scan<int>(both ? 1 : 0, ws, &tot);
            const long long m = warp_reserve((unsigned long long*)&w.mcount[h], (j < pc.nb && !both) ? 1 : 0);
            if (j < pc.nb && !both) {
                const int slot = j + pa - (seen + pre);
                rf[slot] = y;
                fb[slot] = st.v0[pc.ib + j];
                put_missing(w, m, pc.iff + slot, pc.row0 + y, ta, status);   // V_a(y)
            }
            seen += tot;
        }
        if (threadIdx.x == 0) pl.cnt[(int64_t)pc.s * NF + pc.f] = pc.na + pc.nb - common;
    }
}

// -- level h, step 2: the queued entries, one shadow ray per thread
__device__ __forceinline__ void p1_rays_body(const lt_frame& F, const Grid& g, float dmin2, const P1Store& st,
                                             const P1Work& w, int h, int32_t* status) {
    const float4* pts = reinterpret_cast<const float4*>(F.pts);
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    const int64_t n = min(w.mcount[h], w.mcap);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        const int node = w.mnode[q];
        const PointRec P = load_rec(pts, F.m, w.mpt[q]);
        const PointRec L = load_rec(vpls, F.n, F.tree.rep[node]);
        const float v = entry_value(P, L, node_scale(F.tree, vpls, F.n, node), dmin2, g);
        if (!isfinite(v)) latch(status, LT_ENUMERIC);
        st.v0[w.mdst[q]] = v;
    }
}

// -- level h, step 3: eps (Sec. 4), cost (Eq. 2), merge or reject
__device__ __forceinline__ void decide_pair(const lt_frame& F, const P1Plan& pl, const P1Store& st, const float* thr,
                                            const PairCtx& pc, float e_max, int first, int step, bool writer) {
    const int NF = 2 * F.C - 1;
    const int ta = F.forest[8 * pc.a], tb = F.forest[8 * pc.b], tf = F.forest[8 * pc.f];
    const float Ia = F.tree.I[ta], Ib = F.tree.I[tb], If = F.tree.I[tf];
    const bool p_is_a = Ia >= Ib;
    float* cost = pl.cost + (int64_t)pc.s * NF;
    int32_t* state = pl.state + (int64_t)pc.s * NF;
    const int q = p_is_a ? pc.b : pc.a;
    const float cf = e_max + cost[q];
    const float th = thr[pc.s];
    const bool merge = th < 0.f ? cf == 0.f : cf < th;  // th < 0: a dark slice
    const int nf = pl.cnt[(int64_t)pc.s * NF + pc.f];
    if (merge) {
        const float rfp = __fdiv_rn(If, p_is_a ? Ia : Ib);
        float* fa = st.v0 + pc.iff;
        const float* fb = st.v1 + pc.iff;
        float* keep = st.v2 ? st.v2 + pc.iff : nullptr;
        for (int t = first; t < nf; t += step) {
            if (keep) keep[t] = fa[t];
            fa[t] = (p_is_a ? fa[t] : fb[t]) * rfp;
        }
    }
    if (writer) {
        cost[pc.f] = cf;
        state[pc.f] = merge ? kStAlive : kStRejected;
        if (merge) {
            state[pc.a] = kStDead;
            state[pc.b] = kStDead;
        }
    }
}

__device__ __forceinline__ float pair_eps(const lt_frame& F, const P1Store& st, const PairCtx& pc, int nf, int lane,
                                          int step) {
    const int ta = F.forest[8 * pc.a], tb = F.forest[8 * pc.b];
    const float Ia = F.tree.I[ta], Ib = F.tree.I[tb];
    const bool p_is_a = Ia >= Ib;
    const float rq = p_is_a ? __fdiv_rn(Ib, Ia) : __fdiv_rn(Ia, Ib);
    const float* fa = st.v0 + pc.iff;
    const float* fb = st.v1 + pc.iff;
    float e = 0.f;
    for (int t = lane; t < nf; t += step) {
        const float vp = p_is_a ? fa[t] : fb[t];
        const float vq = p_is_a ? fb[t] : fa[t];
        e = fmaxf(e, fabsf(vq - vp * rq));
    }
    return e;
}

// pairs that are not big, one thread per pair
__device__ __forceinline__ void p1_decide_body(const lt_frame& F, const P1Plan& pl, const P1Store& st,
                                               const P1Work& w, int h) {
    const int np = F.level_off[h + 1] - F.level_off[h];
    const int NF = 2 * F.C - 1;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)F.S * np;
         t += (int64_t)gridDim.x * blockDim.x) {
        PairCtx pc;
        if (!load_pair(F, pl, st, h, t, pc)) continue;
        if (pair_big(pc)) continue;
        const int nf = pl.cnt[(int64_t)pc.s * NF + pc.f];
        decide_pair(F, pl, st, w.thr, pc, pair_eps(F, st, pc, nf, 0, 1), 0, 1, true);
    }
}

// big pairs, one CTA per pair
__device__ __forceinline__ void p1_decide_big_body(const lt_frame& F, const P1Plan& pl, const P1Store& st,
                                                   const P1Work& w, int h) {
    __shared__ float red[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int NF = 2 * F.C - 1;
    const int64_t nbig = min(w.bcount[h], w.bcap);
    for (int64_t q = blockIdx.x; q < nbig; q += gridDim.x) {
        PairCtx pc;
        if (!load_pair(F, pl, st, h, w.big[q], pc)) continue;  // uniform in the block
        const int nf = pl.cnt[(int64_t)pc.s * NF + pc.f];
        const float e = warp_max(pair_eps(F, st, pc, nf, threadIdx.x, blockDim.x));
        __syncthreads();  // red is free
        if (lane == 0) red[wid] = e;
        __syncthreads();
        float em = 0.f;
        for (int k = 0; k < nw; ++k) em = fmaxf(em, red[k]);
        decide_pair(F, pl, st, w.thr, pc, em, threadIdx.x, blockDim.x, threadIdx.x == 0);
    }
}

// Per-level form: each step of each level is its own launch.
__global__ void __launch_bounds__(128) k_p1_setup(lt_frame F, P1Plan pl, P1Store st, P1Work w, int h,
                                                  int32_t* status) {
    p1_setup_body(F, pl, st, w, h, status);
}
__global__ void __launch_bounds__(256) k_p1_setup_big(lt_frame F, P1Plan pl, P1Store st, P1Work w, int h,
                                                      int32_t* status) {
    p1_setup_big_body(F, pl, st, w, h, status);
}
__global__ void __launch_bounds__(128) k_p1_rays(lt_frame F, Grid g, float dmin2, P1Store st, P1Work w, int h,
                                                 int32_t* status) {
    p1_rays_body(F, g, dmin2, st, w, h, status);
}
__global__ void __launch_bounds__(128) k_p1_decide(lt_frame F, P1Plan pl, P1Store st, P1Work w, int h) {
    p1_decide_body(F, pl, st, w, h);
}
__global__ void __launch_bounds__(256) k_p1_decide_big(lt_frame F, P1Plan pl, P1Store st, P1Work w, int h) {
    p1_decide_big_body(F, pl, st, w, h);
}

// Persistent form: one cooperative launch walks every level, the four steps of a level
// separated by grid-wide barriers.  `bar` counts block arrivals (zeroed before the
// launch); barrier k is passed when it reaches k * gridDim.x.  Every wait is bounded:
// past the limit the block latches LT_ELIMIT and leaves the walk (so do the others at
// their next barrier, also bounded).
constexpr unsigned kBarSpins = 1u << 21;

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& k, int32_t* status, int* s_ok) {
    __syncthreads();
    ++k;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = k * gridDim.x;
        int ok = 1;
        for (unsigned it = 0; ld_acquire_gpu(bar) < target; ++it) {
            if (it >= kBarSpins) {
                ok = 0;
                latch(status, LT_ELIMIT);
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

__global__ void __launch_bounds__(256, 3) k_p1_walk(lt_frame F, Grid g, float dmin2, P1Plan pl, P1Store st, P1Work w,
                                                 int32_t* status) {
    __shared__ int s_ok;
    unsigned k = 0;
    for (int h = 1; h <= F.H; ++h) {
        if (F.level_off[h + 1] == F.level_off[h]) continue;  // uniform over the grid
        p1_setup_body(F, pl, st, w, h, status);
        if (!grid_barrier(w.bar, k, status, &s_ok)) return;
        p1_setup_big_body(F, pl, st, w, h, status);
        if (!grid_barrier(w.bar, k, status, &s_ok)) return;
        p1_rays_body(F, g, dmin2, st, w, h, status);
        if (!grid_barrier(w.bar, k, status, &s_ok)) return;
        p1_decide_body(F, pl, st, w, h);
        p1_decide_big_body(F, pl, st, w, h);
        if (!grid_barrier(w.bar, k, status, &s_ok)) return;
    }
}

// -- the coarsened cut of every slice in leaf order and its observed entries
__global__ void __launch_bounds__(kP1Threads) k_p1_output(lt_frame F, P1Plan pl, P1Store st, lt_samples smp,
                                                          int32_t* status) {
    extern __shared__ int32_t mark[];  // [C] forest node whose first leaf is c, else -1
    __shared__ int32_t ws[32];
    __shared__ float red[32];
    const int s = blockIdx.x;
    const int C = F.C, NF = 2 * C - 1;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int32_t* off = pl.off + (int64_t)s * NF;
    const int32_t* cnt = pl.cnt + (int64_t)s * NF;
    const int32_t* state = pl.state + (int64_t)s * NF;
    const int64_t base = pl.base[s];
    const int32_t* rows = st.rows + base;
    const float* v0 = st.v0 + base;
    const float* v1 = st.v1 + base;
    if (ms == 0) {
        if (threadIdx.x == 0) {
            smp.ncol[s] = 0;
            smp.n1[s] = 0;
            smp.cnt[s] = 0;
        }
        return;
    }
    for (int c = threadIdx.x; c < C; c += blockDim.x) mark[c] = -1;
    __syncthreads();
    for (int x = threadIdx.x; x < NF; x += blockDim.x)
        if (state[x] == kStAlive) mark[F.forest[8 * x + 4]] = x;
    __syncthreads();
    int32_t* colx = pl.colx + (int64_t)s * C;
    int32_t* eoff = pl.eoff + (int64_t)s * C;
    int ncol = 0;
    for (int c0 = 0; c0 < C; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        const int x = c < C ? mark[c] : -1;
        int tot;
        const int pre = block_exclusive_scan<int>(x >= 0 ? 1 : 0, ws, &tot);
        if (x >= 0) {
            const int j = ncol + pre;
            colx[j] = x;
            const int par = F.forest[8 * x + 3];
            const bool from_par = par >= 0 && state[par] == kStRejected;
            eoff[j] = from_par ? cnt[par] : cnt[x];
            smp.col_node[(int64_t)s * C + j] = F.forest[8 * x];
        }
        ncol += tot;
    }
    __syncthreads();
    int n1 = 0;
    for (int c0 = 0; c0 < ncol; c0 += blockDim.x) {
        const int j = c0 + threadIdx.x;
        const int x = j < ncol ? eoff[j] : 0;
        int tot;
        const int pre = block_exclusive_scan<int>(x, ws, &tot);
        if (j < ncol) eoff[j] = n1 + pre;
        n1 += tot;
    }
    __syncthreads();
    const int64_t capacity = smp.off[s + 1] - smp.off[s];
    const bool over = (int64_t)n1 > capacity;
    if (over && threadIdx.x == 0) latch(status, LT_ELIMIT);
    uint32_t* key = smp.key + smp.off[s];
    float* val = smp.val + smp.off[s];
    float* gs = smp.g + (int64_t)s * C;
    for (int j = wid; j < ncol; j += nw) {
        const int x = colx[j];
        const int par = F.forest[8 * x + 3];
        const bool from_par = par >= 0 && state[par] == kStRejected;
        const int src = from_par ? par : x;
        const int n = cnt[src];
        const int32_t* rr = rows + off[src];
        const float* vv = (from_par && F.forest[8 * par + 2] == x) ? v1 + off[src]
                          : (from_par && st.v2)                   ? st.v2 + base + off[src]
                                                                  : v0 + off[src];
        float mx = -3.0e38f, mn = 3.0e38f;
        const int dst = (int)(eoff[j]);
        for (int t = lane; t < n; t += 32) {
            const float v = vv[t];
            mx = fmaxf(mx, v);
            mn = fminf(mn, v);
            if (!over) {
                key[dst + t] = ((uint32_t)rr[t] << 16) | (uint32_t)j;
                val[dst + t] = v;
            }
        }
        mx = warp_max(mx);
        mn = warp_min(mn);
        if (lane == 0) gs[j] = n >= 2 ? mx - mn : -1.f;
    }
    __syncthreads();
    float gm = -1.f;
    for (int j = threadIdx.x; j < ncol; j += blockDim.x) gm = fmaxf(gm, gs[j]);
    gm = warp_max(gm);
    if (lane == 0) red[wid] = gm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = -1.f;
        for (int w = 0; w < nw; ++w) m = fmaxf(m, red[w]);
        red[0] = m;
    }
    __syncthreads();
    const float gfill = red[0] >= 0.f ? red[0] : 0.f;
    for (int j = threadIdx.x; j < ncol; j += blockDim.x)
        if (gs[j] < 0.f) gs[j] = gfill;
    if (threadIdx.x == 0) {
        smp.ncol[s] = ncol;
        const int stored = over ? 0 : n1;
        smp.n1[s] = stored;
        smp.cnt[s] = stored;
    }
}

// ------------------------------------------------------------------ pass 2
__device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}

constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kP2Cluster = 8;    // CTAs per slice (one thread-block cluster)
constexpr int kP2Block = 512;    // threads per CTA
constexpr int kP2Draws = 4;      // draws per thread per round
constexpr int kGuide = 2048;     // buckets of the CDF guide table

// Per slice (one CTA each): the inclusive integer CDF of the quantised column
// weights (q = max(1, floor(w / w_max * 2^24)), 0 for w <= 0) and the bitmap of the
// pass-1 entries.
__global__ void __launch_bounds__(1024) k_p2_prep(lt_frame F, const float* __restrict__ weights, lt_samples smp,
                                                  unsigned long long* __restrict__ cdf_all,
                                                  unsigned long long* __restrict__ total_all, uint32_t* bitmap_all,
                                                  int64_t bitmap_stride) {
    __shared__ unsigned long long wsum[32];
    __shared__ float red[32];
    const int s = blockIdx.x;
    const int C = F.C;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    const int ns = smp.ncol[s];
    const int n1 = smp.n1[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float* w = (weights ? weights : smp.g) + (int64_t)s * C;
    float wm = 0.f;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) wm = fmaxf(wm, w[j]);
    wm = warp_max(wm);
    if (lane == 0) red[wid] = wm;
    __syncthreads();
    float wmax = 0.f;
    for (int i = 0; i < nw; ++i) wmax = fmaxf(wmax, red[i]);
    unsigned long long* cdf = cdf_all + (int64_t)s * C;
    unsigned long long carry = 0;
    for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
        const int j = c0 + threadIdx.x;
        unsigned long long q = 0;
        if (j < ns) {
            if (!(wmax > 0.f)) {
                q = 1;
            } else {
                const float wj = w[j];
                if (wj > 0.f) {
                    const float r = __fmul_rn(__fdiv_rn(wj, wmax), 16777216.0f);
                    q = (unsigned long long)floorf(r);
                    if (q < 1) q = 1;
                }
            }
        }
        unsigned long long tot;
        const unsigned long long pre = block_exclusive_scan<unsigned long long>(q, wsum, &tot);
        if (j < ns) cdf[j] = carry + pre + q;
        carry += tot;
    }
    if (threadIdx.x == 0) total_all[s] = carry;
    const int W = (ns + 31) >> 5;
    uint32_t* bm = bitmap_all + (int64_t)s * bitmap_stride;
    for (int64_t i = threadIdx.x; i < (int64_t)ms * W; i += blockDim.x) bm[i] = 0u;
    __syncthreads();
    const uint32_t* key1 = smp.key + smp.off[s];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const uint32_t k = key1[i];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        if (r < ms && c < ns) atomicOr(bm + (int64_t)r * W + (c >> 5), 1u << (c & 31));
    }
}

// One cluster of kP2Cluster CTAs per slice.  A round takes the next
// kP2Cluster x kP2Block x kP2Draws draws in order (CTA k the k-th block of them,
// thread i of a CTA kP2Draws consecutive ones), keeps those whose (row, col) is
// not observed yet (bitmap) and is the first of its key in the round (a hash table
// spread over the cluster's shared memory: a key lives in the part of CTA
// hash & (kP2Cluster - 1) and keeps the smallest draw index), and accepts them in
// draw order (a prefix over the CTAs' counts) up to the target.  Every CTA of the
// cluster computes the same accepted count, so all take the same cluster barriers.
__global__ void __cluster_dims__(kP2Cluster, 1, 1) __launch_bounds__(kP2Block, 2)
    k_pass2(lt_frame F, float rate, SeedRef sr, lt_samples smp, const unsigned long long* __restrict__ cdf_all,
            const unsigned long long* __restrict__ total_all, uint32_t* bitmap_all, int64_t bitmap_stride, int hpart,
            int32_t* status) {
    namespace cg = cooperative_groups;
    // dynamic shared memory: cdf[C] (u64), hkey[hpart] (u32), htid[hpart] (int32: the
    // smallest draw index of the key in the round), guide[kGuide + 1] (int32)
    extern __shared__ unsigned long long p2sm[];
    unsigned long long* scdf = p2sm;
    uint32_t* hkey = reinterpret_cast<uint32_t*>(p2sm + F.C);
    int32_t* htid = reinterpret_cast<int32_t*>(hkey + hpart);
    int32_t* guide = htid + hpart;
    __shared__ int32_t ws[32];
    __shared__ int32_t s_cnt;
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int s = blockIdx.x / kP2Cluster;
    const int C = F.C;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    const int ns = smp.ncol[s];
    const int n1 = smp.n1[s];
    const uint64_t seed = sr.get();
    if (ms == 0 || ns == 0) {
        if (rank == 0 && threadIdx.x == 0) smp.cnt[s] = n1;
        return;
    }
    const int64_t T = (int64_t)ceil((double)rate * (double)ms * (double)ns);
    int64_t need = T - n1;
    if (need <= 0) {
        if (rank == 0 && threadIdx.x == 0) smp.cnt[s] = n1;
        return;
    }
    const int64_t capacity = smp.off[s + 1] - smp.off[s];
    if (n1 + need > capacity) {
        if (rank == 0 && threadIdx.x == 0) latch(status, LT_ELIMIT);
        need = capacity - n1;
    }
    const unsigned long long total = total_all[s];
    const uint32_t th = (uint32_t)(total >> 32), tl = (uint32_t)total;
    const int W = (ns + 31) >> 5;
    uint32_t* bm = bitmap_all + (int64_t)s * bitmap_stride;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) scdf[j] = cdf_all[(int64_t)s * C + j];
    for (int i = threadIdx.x; i < hpart; i += blockDim.x) {
        hkey[i] = kEmpty;
        htid[i] = 0x7fffffff;
    }
    __syncthreads();
    // guide table: guide[k] = first c with cdf[c] > floor(k total / kGuide); a draw u in
    // bucket k = floor(u kGuide / total) has its column in [guide[k], guide[k + 1]]
    for (int k = threadIdx.x; k <= kGuide; k += blockDim.x) {
        const unsigned long long v = (unsigned long long)k * total / kGuide;
        int a = 0, b = ns - 1;  // cdf[ns - 1] = total > v for k < kGuide
        while (a < b) {
            const int m = (a + b) >> 1;
            if (scdf[m] > v) b = m;
            else a = m + 1;
        }
        guide[k] = a;
    }
    cl.sync();
    const int64_t cap_draws = 64 * T + 64;
    uint32_t* keyout = smp.key + smp.off[s] + n1;
    const int64_t per_cta = (int64_t)blockDim.x * kP2Draws, per_round = per_cta * kP2Cluster;
    int64_t accepted = 0;
    for (int64_t t0 = 0; accepted < need && t0 < cap_draws; t0 += per_round) {
        uint32_t rc[kP2Draws];
        int home[kP2Draws], slot[kP2Draws], tr[kP2Draws];
        int64_t tt[kP2Draws];
        unsigned long long u[kP2Draws];
        uint32_t wrow[kP2Draws];
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d) {  // draw and column search, all draws at once
            tt[d] = t0 + rank * per_cta + (int64_t)threadIdx.x * kP2Draws + d;
            const U4 x = philox((uint32_t)tt[d], 0u, slice_key(F.slice_id, s), kTagPass2, seed);
            u[d] = (unsigned long long)x.x * th + (((unsigned long long)x.x * tl) >> 32);
            wrow[d] = x.y;
            home[d] = -1;
        }
        int lo[kP2Draws];
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d) {  // first c with cdf[c] > u, from its guide bucket
            const int k = (int)(u[d] * kGuide / total);
            int a = guide[k], b = guide[k + 1];
            while (a < b) {
                const int m = (a + b) >> 1;
                if (scdf[m] > u[d]) b = m;
                else a = m + 1;
            }
            lo[d] = a;
        }
        uint32_t word[kP2Draws];
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d) {
            const int c = lo[d], r = (int)uniform_index(wrow[d], (uint32_t)ms);
            rc[d] = ((uint32_t)r << 16) | (uint32_t)c;
            // L2 reads: other CTAs of the cluster set bits in earlier rounds (L1 is not coherent)
            word[d] = tt[d] < cap_draws ? __ldcg(bm + (int64_t)r * W + (c >> 5)) : 0xffffffffu;
        }
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d) {
            const int r = (int)(rc[d] >> 16), c = (int)(rc[d] & 0xffffu);
            if ((word[d] >> (c & 31)) & 1u) continue;  // observed (or past the draw cap)
            const uint32_t key = (uint32_t)r * (uint32_t)ns + (uint32_t)c;
            const uint32_t h = hash32(key);
            const int k = (int)(h & (kP2Cluster - 1));
            uint32_t* rk = cl.map_shared_rank(hkey, k);
            int32_t* rt = cl.map_shared_rank(htid, k);
            uint32_t p = (h >> 3) & (uint32_t)(hpart - 1);
            tr[d] = (int)(tt[d] - t0);
            for (int probe = 0; probe < hpart; ++probe) {
                const uint32_t prev = atomicCAS(&rk[p], kEmpty, key);
                if (prev == kEmpty || prev == key) {
                    atomicMin(&rt[p], tr[d]);
                    home[d] = k;
                    slot[d] = (int)p;
                    break;
                }
                p = (p + 1) & (uint32_t)(hpart - 1);
            }
            if (home[d] < 0) latch(status, LT_ELIMIT);  // a full table part: not expected at load 1/2
        }
        cl.sync();
        int mine = 0;
        uint32_t firstmask = 0;
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d)
            if (home[d] >= 0 && cl.map_shared_rank(htid, home[d])[slot[d]] == tr[d]) {
                firstmask |= 1u << d;
                ++mine;
            }
        int tot;
        int pos = block_exclusive_scan<int>(mine, ws, &tot);
        if (threadIdx.x == 0) s_cnt = tot;
        cl.sync();
        int before = 0, round_total = 0;
        for (int k = 0; k < kP2Cluster; ++k) {
            const int ck = *cl.map_shared_rank(&s_cnt, k);
            if (k < rank) before += ck;
            round_total += ck;
        }
#pragma unroll
        for (int d = 0; d < kP2Draws; ++d)
            if (firstmask & (1u << d)) {
                const int64_t g = accepted + before + pos;
                if (g < need) {
                    keyout[g] = rc[d];
                    const int r = (int)(rc[d] >> 16), c = (int)(rc[d] & 0xffffu);
                    atomicOr(bm + (int64_t)r * W + (c >> 5), 1u << (c & 31));
                }
                ++pos;
            }
        accepted += min((int64_t)round_total, need - accepted);
        for (int i = threadIdx.x; i < hpart; i += blockDim.x) {
            hkey[i] = kEmpty;
            htid[i] = 0x7fffffff;
        }
        __threadfence();  // this round's bitmap bits before the next round's reads
        cl.sync();
    }
    if (rank == 0 && threadIdx.x == 0) smp.cnt[s] = n1 + (int)accepted;
}

// ------------------------------------------------------------------ entry evaluation
__global__ void k_count_prefix(const lt_samples smp, int S, int64_t* pfx) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < S ? (int64_t)(smp.cnt[s] - smp.n1[s]) : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < S) pfx[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) pfx[S] = carry;
}

// Column records of a frame: for every (slice, coarsened column) the representative
// VPL's three record planes and the node's scale I_c / (flux albedo) of its
// representative, 64 B each ([S][C][4] float4), so that an entry gathers its column
// with one contiguous load (a slice's few hundred columns stay in L1) instead of the
// node, its representative, the three VPL planes and three scale terms.
__global__ void k_col_records(lt_frame F, lt_samples smp, float4* __restrict__ tab) {
    const int s = blockIdx.y;
    const int ns = smp.ncol[s];
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ns; c += gridDim.x * blockDim.x) {
        const int node = smp.col_node[(int64_t)s * F.C + c];
        const PointRec L = load_rec(vpls, F.n, F.tree.rep[node]);
        float4* t = tab + ((int64_t)s * F.C + c) * 4;
        t[0] = L.a;
        t[1] = L.b;
        t[2] = L.c;
        t[3] = make_float4(node_scale(F.tree, vpls, F.n, node), 0.f, 0.f, 0.f);
    }
}

template <bool COUNT>
__global__ void __launch_bounds__(128) k_eval_entries(lt_frame F, Grid g, float dmin2, lt_samples smp,
                                                      const int64_t* __restrict__ pfx,
                                                      const float4* __restrict__ coltab,
                                                      unsigned long long* __restrict__ stats, int32_t* status) {
    extern __shared__ int64_t spfx[];
    const int S = F.S;
    for (int i = threadIdx.x; i <= S; i += blockDim.x) spfx[i] = pfx[i];
    __syncthreads();
    const int64_t total = spfx[S];
    const float4* pts = reinterpret_cast<const float4*>(F.pts);
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    WorkCount wc;
    int rays = 0, entries = 0;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        int lo = 0, hi = S;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (spfx[mid] <= idx) lo = mid;
            else hi = mid;
        }
        const int s = lo;
        const int64_t e = smp.off[s] + smp.n1[s] + (idx - spfx[s]);
        const uint32_t k = smp.key[e];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        const PointRec P = load_rec(pts, F.m, F.slice_off[s] + r);
        PointRec L;
        float scale;
        if (coltab) {  // the frame's column records
            const float4* t = coltab + ((int64_t)s * F.C + c) * 4;
            L.a = __ldg(t);
            L.b = __ldg(t + 1);
            L.c = __ldg(t + 2);
            scale = __ldg(t + 3).x;
        } else {
            const int node = smp.col_node[(int64_t)s * F.C + c];
            L = load_rec(vpls, F.n, F.tree.rep[node]);
            scale = node_scale(F.tree, vpls, F.n, node);
        }
        const float v = entry_value<COUNT>(P, L, scale, dmin2, g, &wc, &rays);
        if (COUNT) {
            ++entries;
        } else {
            if (!isfinite(v)) latch(status, LT_ENUMERIC);
            smp.val[e] = v;
        }
    }
    if (COUNT) {
        atomicAdd(stats + 0, (unsigned long long)entries);
        atomicAdd(stats + 1, (unsigned long long)rays);
        atomicAdd(stats + 2, (unsigned long long)wc.cells);
        atomicAdd(stats + 3, (unsigned long long)wc.boxes);
    }
}

bool frame_ok(const lt_frame* f) {
    return f && f->pts && f->vpls && f->slice_off && f->S > 0 && f->m > 0 && f->n > 0 && f->C >= 1 &&
           f->C <= kMaxCut && f->forest && f->max_rows >= 0 && f->max_rows <= 65535 && f->tree.I &&
           f->tree.rep && (((uintptr_t)f->pts & 15) == 0) && (((uintptr_t)f->vpls & 15) == 0) &&
           (f->C == 1 || (f->level_off && f->level_nodes)) && f->H >= 0;
}

bool samples_ok(const lt_samples* s) {
    return s && s->ncol && s->col_node && s->g && s->off && s->key && s->val && s->n1 && s->cnt;
}

}  // namespace

namespace {

lt_status sample_pass1(lt_ctx* ctx, const lt_frame* f, float rate1, float tau, int32_t target, float d_min,
                       uint64_t seed, lt_samples* smp) {
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_sample_pass1: no scene uploaded");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C, NF = 2 * C - 1;
    lt_status st;
    const size_t n_k = (size_t)S * C, n_f = (size_t)S * NF, n_p = (size_t)S * (C + 1);
    const size_t bytes = (n_k * 3 + n_f * 5 + n_p) * sizeof(int32_t) + 2 * S * sizeof(int64_t) + 16 * 256;
    char* p = (char*)lt_scratch(ctx, SCR_P1_PLAN, bytes, &st);
    if (!p) return st;
    P1Plan pl;
    auto take = [&](size_t nbytes) {
        char* q = p;
        p += (nbytes + 255) & ~(size_t)255;
        return q;
    };
    pl.total = (int64_t*)take(S * sizeof(int64_t));
    pl.base = (int64_t*)take(S * sizeof(int64_t));
    pl.k = (int32_t*)take(n_k * 4);
    pl.colx = (int32_t*)take(n_k * 4);
    pl.eoff = (int32_t*)take(n_k * 4);
    pl.cap = (int32_t*)take(n_f * 4);
    pl.off = (int32_t*)take(n_f * 4);
    pl.cnt = (int32_t*)take(n_f * 4);
    pl.state = (int32_t*)take(n_f * 4);
    pl.cost = (float*)take(n_f * 4);
    pl.pfx = (int32_t*)take(n_p * 4);
    if ((size_t)(p - (char*)ctx->scr[SCR_P1_PLAN]) > ctx->scr_size[SCR_P1_PLAN])
        return lt_fail(ctx, LT_ENOMEM, "lt_sample_pass1: plan layout overflow");
    k_pass1_plan<<<S, kP1Threads, 0, ctx->stream>>>(*f, rate1, pl);
    LT_LAUNCH_CHECK(ctx, "k_pass1_plan");
    k_p1_base<<<1, 1024, 0, ctx->stream>>>(S, pl);
    LT_LAUNCH_CHECK(ctx, "k_p1_base");
    // The row-slot total sizes the scratch below; it follows from the setup alone
    // (cut, forest, slices, rate1), so a captured frame reuses the recorded value.
    int64_t acc = 0;
    if (ctx->use_plan) {
        acc = ctx->plan.p1_total;
    } else {
        std::vector<int64_t> tot(S);
        LT_CUDA(ctx, cudaMemcpyAsync(tot.data(), pl.total, S * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        for (int s = 0; s < S; ++s) acc += tot[s];
        ctx->plan.p1_total = acc;
    }
    // storage: rows, then v0 and v1 back to back (a flat value index addresses both);
    // then the work arrays of the flat kernels
    const int Hn = f->H + 2;
    const int64_t mcap = std::max<int64_t>(acc, 1024), bcap = std::max<int64_t>((int64_t)S * C, 1024);
    const size_t store_bytes = (size_t)std::max<int64_t>(acc, 1) * (target > 0 ? 16 : 12) + 1024;
    const size_t eff_bytes = target > 0 ? (size_t)S * NF * 4 : 0;
    const size_t work_bytes = (size_t)(S + 1) * 8 + (size_t)S * C * 4 + (size_t)S * 4 + (size_t)Hn * 16 +
                              (size_t)mcap * 16 + (size_t)bcap * 8 + eff_bytes + 17 * 256;
    char* q = (char*)lt_scratch(ctx, SCR_P1_STORE, store_bytes + work_bytes, &st);
    if (!q) return st;
    P1Store store;
    store.total = acc;
    store.rows = (int32_t*)q;
    store.v0 = (float*)(q + ((acc * 4 + 255) & ~255LL));
    store.v1 = store.v0 + acc;
    store.v2 = target > 0 ? store.v1 + acc : nullptr;
    char* wp = q + ((store_bytes + 255) & ~(size_t)255);
    auto wtake = [&](size_t nbytes) {
        char* r = wp;
        wp += (nbytes + 255) & ~(size_t)255;
        return r;
    };
    P1Work w;
    w.kpfx = (int64_t*)wtake((size_t)(S + 1) * 8);
    w.leafmean = (float*)wtake((size_t)S * C * 4);
    w.thr = (float*)wtake((size_t)S * 4);
    w.mcount = (int64_t*)wtake((size_t)Hn * 8 + 8);
    w.bcount = (int64_t*)wtake((size_t)Hn * 8);
    w.mdst = (int64_t*)wtake((size_t)mcap * 8);
    w.mpt = (int32_t*)wtake((size_t)mcap * 4);
    w.mnode = (int32_t*)wtake((size_t)mcap * 4);
    w.big = (int64_t*)wtake((size_t)bcap * 8);
    w.bar = (unsigned*)(w.mcount + Hn);  // shares the zeroing of the level counters
    w.mcap = mcap;
    w.bcap = bcap;
    float* effs = target > 0 ? (float*)wtake(eff_bytes) : nullptr;
    if ((size_t)(wp - q) > ctx->scr_size[SCR_P1_STORE])
        return lt_fail(ctx, LT_ENOMEM, "lt_sample_pass1: work layout overflow");
    LT_CUDA(ctx, cudaMemsetAsync(w.mcount, 0, (size_t)Hn * 8 + 8, ctx->stream));
    LT_CUDA(ctx, cudaMemsetAsync(w.bcount, 0, (size_t)Hn * 8, ctx->stream));
    const int nsm = ctx->num_sms;
    const float dmin2 = d_min * d_min;
    auto grid_for = [&](int64_t items, int threads) {
        return (unsigned)std::max<int64_t>(1, std::min<int64_t>((items + threads - 1) / threads, 32 * (int64_t)nsm));
    };
    k_p1_draws<<<grid_for((int64_t)S * NF, 256), 256, 0, ctx->stream>>>(*f, seed_ref(ctx, seed), pl, store,
                                                                        ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_p1_draws");
    k_p1_kpfx<<<1, 1024, 0, ctx->stream>>>(*f, pl, w.kpfx);
    LT_LAUNCH_CHECK(ctx, "k_p1_kpfx");
    const int ray_grid = ctx->tune.ray_ctas_per_sm * nsm;
    k_p1_initial<<<ray_grid, 128, 0, ctx->stream>>>(*f, ctx->grid, dmin2, pl, store, w.kpfx, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_p1_initial");
    k_p1_leafmean<<<grid_for((int64_t)S * C, 256), 256, 0, ctx->stream>>>(*f, pl, store, w.leafmean);
    LT_LAUNCH_CHECK(ctx, "k_p1_leafmean");
    if (target > 0) {
        k_p1_thr_inf<<<(S + 255) / 256, 256, 0, ctx->stream>>>(S, w.thr);
        LT_LAUNCH_CHECK(ctx, "k_p1_thr_inf");
    } else {
        k_p1_thr<<<S, 256, 0, ctx->stream>>>(*f, w.leafmean, tau, w.thr);
        LT_LAUNCH_CHECK(ctx, "k_p1_thr");
    }
    std::vector<int32_t> loff(f->H + 2, 0);
    if (ctx->use_plan) {
        if ((int)ctx->plan.level_off.size() != f->H + 2)
            return lt_fail(ctx, LT_EINVAL, "lt_sample_pass1: recorded frame plan does not match the forest");
        loff = ctx->plan.level_off;
    } else {
        if (f->H > 0)
            LT_CUDA(ctx, cudaMemcpyAsync(loff.data(), f->level_off, (f->H + 2) * 4, cudaMemcpyDeviceToHost,
                                         ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->plan.level_off = loff;
    }
    const bool walk = ctx->tune.p1_form == 1 && f->H > 0;
    if (walk) {
        if (ctx->p1_walk_blocks == 0) {
            int nb = 0;
            LT_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_p1_walk, 256, 0));
            ctx->p1_walk_blocks = std::max(1, std::min(nb, 8));
        }
        // every block resident at once (the cooperative launch checks it)
        cudaLaunchConfig_t lc = {};
        lc.gridDim = dim3((unsigned)(ctx->p1_walk_blocks * nsm));
        lc.blockDim = dim3(256);
        lc.dynamicSmemBytes = 0;
        lc.stream = ctx->stream;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        LT_CUDA(ctx, cudaLaunchKernelEx(&lc, k_p1_walk, *f, ctx->grid, dmin2, pl, store, w, ctx->d_status));
        LT_LAUNCH_CHECK(ctx, "k_p1_walk");
    }
    for (int h = 1; h <= f->H && !walk; ++h) {
        const int64_t npairs = (int64_t)S * (loff[h + 1] - loff[h]);
        if (npairs == 0) continue;
        k_p1_setup<<<grid_for(npairs, 128), 128, 0, ctx->stream>>>(*f, pl, store, w, h, ctx->d_status);
        LT_LAUNCH_CHECK(ctx, "k_p1_setup");
        k_p1_setup_big<<<4 * nsm, 256, 0, ctx->stream>>>(*f, pl, store, w, h, ctx->d_status);
        LT_LAUNCH_CHECK(ctx, "k_p1_setup_big");
        k_p1_rays<<<ray_grid, 128, 0, ctx->stream>>>(*f, ctx->grid, dmin2, store, w, h, ctx->d_status);
        LT_LAUNCH_CHECK(ctx, "k_p1_rays");
        k_p1_decide<<<grid_for(npairs, 128), 128, 0, ctx->stream>>>(*f, pl, store, w, h);
        LT_LAUNCH_CHECK(ctx, "k_p1_decide");
        k_p1_decide_big<<<4 * nsm, 256, 0, ctx->stream>>>(*f, pl, store, w, h);
        LT_LAUNCH_CHECK(ctx, "k_p1_decide_big");
    }
    if (target > 0) {
        k_p1_target<<<S, 1024, 0, ctx->stream>>>(*f, pl, effs, target);
        LT_LAUNCH_CHECK(ctx, "k_p1_target");
    }
    const size_t shm = (size_t)C * 4;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_p1_output, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_p1_output<<<S, kP1Threads, shm, ctx->stream>>>(*f, pl, store, *smp, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_p1_output");
    return LT_OK;
}

}  // namespace

extern "C" lt_status lt_sample_pass1(lt_ctx* ctx, const lt_frame* f, float rate1, float tau, float d_min,
                                     uint64_t seed, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp) || !(rate1 >= 0.f) || !(tau >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_sample_pass1: bad arguments");
    return sample_pass1(ctx, f, rate1, tau, 0, d_min, seed, smp);
}

extern "C" lt_status lt_sample_pass1_target(lt_ctx* ctx, const lt_frame* f, float rate1, int32_t target,
                                            float d_min, uint64_t seed, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp) || !(rate1 >= 0.f) || target < 1)
        return lt_fail(ctx, LT_EINVAL, "lt_sample_pass1_target: bad arguments");
    return sample_pass1(ctx, f, rate1, 0.f, target, d_min, seed, smp);
}

extern "C" lt_status lt_sample_pass2(lt_ctx* ctx, const lt_frame* f, const float* weights, float rate,
                                     uint64_t seed, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp) || !(rate >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_sample_pass2: bad arguments");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C;
    const int64_t stride = (int64_t)std::max(f->max_rows, 1) * ((C + 31) / 32);
    lt_status st;
    uint32_t* bm = (uint32_t*)lt_scratch(ctx, SCR_BITMAP, (size_t)S * stride * 4, &st);
    if (!bm) return st;
    unsigned long long* cdf_all = (unsigned long long*)lt_scratch(ctx, SCR_P2_CDF, ((size_t)S * C + S + 64) * 8, &st);
    if (!cdf_all) return st;
    unsigned long long* total_all = cdf_all + (size_t)S * C;
    k_p2_prep<<<S, 1024, 0, ctx->stream>>>(*f, weights, *smp, cdf_all, total_all, bm, stride);
    LT_LAUNCH_CHECK(ctx, "k_p2_prep");
    // each CTA's part of the round's hash table: 2 slots per draw of the CTA
    const int hpart = 2 * kP2Block * kP2Draws;
    const size_t shm = (size_t)C * 8 + (size_t)hpart * 8 + (size_t)(kGuide + 2) * 4;
    if (shm > (size_t)220 * 1024)
        return lt_fail(ctx, LT_EINVAL, "lt_sample_pass2: global cut too large for the pass-2 CDF in shared memory");
    LT_CUDA(ctx, cudaFuncSetAttribute(k_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_pass2<<<S * kP2Cluster, kP2Block, shm, ctx->stream>>>(*f, rate, seed_ref(ctx, seed), *smp, cdf_all, total_all, bm,
                                                            stride, hpart, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_pass2");
    return LT_OK;
}

extern "C" lt_status lt_eval_entries(lt_ctx* ctx, const lt_frame* f, float d_min, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp)) return lt_fail(ctx, LT_EINVAL, "lt_eval_entries: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_eval_entries: no scene uploaded");
    cudaSetDevice(ctx->device);
    lt_status st;
    const size_t apfx = ((size_t)(f->S + 1) * 8 + 255) & ~(size_t)255;
    char* p = (char*)lt_scratch(ctx, SCR_MISC, apfx + (size_t)f->S * f->C * 64, &st);
    if (!p) return st;
    int64_t* pfx = (int64_t*)p;
    float4* tab = (float4*)(p + apfx);
    k_count_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, f->S, pfx);
    LT_LAUNCH_CHECK(ctx, "k_count_prefix");
    k_col_records<<<dim3((unsigned)std::min(16, (f->C + 255) / 256), f->S), 256, 0, ctx->stream>>>(*f, *smp, tab);
    LT_LAUNCH_CHECK(ctx, "k_col_records");
    const size_t shm = (size_t)(f->S + 1) * 8;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_eval_entries<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shm));
    k_eval_entries<false><<<ctx->num_sms * ctx->tune.eval_ctas_per_sm, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, *smp, pfx,
                                                                        tab, nullptr, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_eval_entries");
    return LT_OK;
}

// ------------------------------------------------------------------ allocation-free variant
// lt_eval_entries keeps its per-slice prefix in context scratch, which it grows
// with cudaMalloc.  Some hosts cannot allow that: an application that owns the
// whole device-memory budget and hands the library only its inputs and outputs
// (for example a renderer plugin running inside a frame loop), where a cudaMalloc
// could fail against the fixed budget or stall the device in the middle of a frame.
// For them the prefix lives in this fixed device array instead.  It is part of the
// module image, so every GPU that loads the library holds its 32 KB until exit.
constexpr int kNoAllocMaxSlices = 4096;
static __device__ __align__(256) int64_t g_noalloc_prefix[kNoAllocMaxSlices + 1];

namespace {
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
int64_t* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_prefix on the context's device.  In host code the
// symbol names a host-side stand-in, so the real address is looked up with that
// device current.  It is looked up again on every call (cheap, and it allocates
// nothing), so a module reloaded after a device reset is found where it now is; the
// last address seen per device is kept only for calls made while the context's
// stream is being captured, where the lookup is not attempted.
lt_status noalloc_prefix(lt_ctx* ctx, int64_t** out) {
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return lt_fail(ctx, LT_EINVAL, "lt_eval_entries_noalloc: device index out of range");
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    LT_CUDA(ctx, cudaStreamIsCapturing(ctx->stream, &cap));
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (cap != cudaStreamCaptureStatusNone) {
        if (!g_noalloc_addr[ctx->device])
            return lt_fail(ctx, LT_EINVAL,
                           "lt_eval_entries_noalloc: make one call on this device before capturing a stream");
        *out = g_noalloc_addr[ctx->device];
        return LT_OK;
    }
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_prefix);
    if (e != cudaSuccess) return lt_cuda_check(ctx, e, "cudaGetSymbolAddress(g_noalloc_prefix)");
    g_noalloc_addr[ctx->device] = (int64_t*)p;
    *out = (int64_t*)p;
    return LT_OK;
}
}  // namespace

extern "C" lt_status lt_eval_entries_noalloc(lt_ctx* ctx, const lt_frame* f, float d_min, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp))
        return lt_fail(ctx, LT_EINVAL, "lt_eval_entries_noalloc: bad arguments");
    if (f->S > kNoAllocMaxSlices)
        return lt_fail(ctx, LT_EINVAL,
                       "lt_eval_entries_noalloc: at most " + std::to_string(kNoAllocMaxSlices) + " slices");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_eval_entries_noalloc: no scene uploaded");
    LT_CUDA(ctx, cudaSetDevice(ctx->device));
    int64_t* pfx = nullptr;
    const lt_status st = noalloc_prefix(ctx, &pfx);
    if (st != LT_OK) return st;
    // every entry of the prefix that the evaluation reads is rewritten here first
    k_count_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, f->S, pfx);
    LT_LAUNCH_CHECK(ctx, "k_count_prefix");
    const size_t shm = (size_t)(f->S + 1) * 8;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_eval_entries<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shm));
    k_eval_entries<false><<<ctx->num_sms * ctx->tune.eval_ctas_per_sm, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, *smp, pfx,
                                                                        nullptr, nullptr, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_eval_entries");
    return LT_OK;
}

extern "C" lt_status lt_eval_stats(lt_ctx* ctx, const lt_frame* f, float d_min, const lt_samples* smp,
                                   int64_t* stats_host) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp) || !stats_host)
        return lt_fail(ctx, LT_EINVAL, "lt_eval_stats: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_eval_stats: no scene uploaded");
    cudaSetDevice(ctx->device);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_MISC, (size_t)(f->S + 1) * 8 + 512, &st);
    if (!p) return st;
    int64_t* pfx = (int64_t*)p;
    unsigned long long* stats = (unsigned long long*)(p + (((f->S + 1) * 8 + 255) & ~255));
    LT_CUDA(ctx, cudaMemsetAsync(stats, 0, 4 * 8, ctx->stream));
    k_count_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, f->S, pfx);
    LT_LAUNCH_CHECK(ctx, "k_count_prefix");
    const size_t shm = (size_t)(f->S + 1) * 8;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_eval_entries<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shm));
    lt_samples copy = *smp;
    k_eval_entries<true><<<ctx->num_sms * ctx->tune.eval_ctas_per_sm, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, copy, pfx,
                                                                       nullptr, stats, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_eval_entries<count>");
    unsigned long long h[4];
    LT_CUDA(ctx, cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 4; ++i) stats_host[i] = (int64_t)h[i];
    return LT_OK;
}
