// Sampling passes of the sparse renderer.
//
//  * Pass 1 and light coarsening (Sec. 4, Eq. 2): one CTA per slice draws k_c rows
//    for every global-cut node, evaluates them, then walks the cut's ancestor
//    forest level by level.  A warp tests one sibling pair: it merges the two
//    sorted row sets (zeta_f = zeta_a U zeta_b), evaluates the missing entries,
//    reduces eps = max |V_q - V_p I_q / I_p| and merges when
//    cost = eps + cost(q) < tau * S_hat.
//  * Pass 2 (Sec. 5, Eq. 3): one CTA per slice draws (column from the integer CDF
//    of g, row uniform) in blocks of blockDim draws, keeps the first occurrence of
//    every new entry in draw order, and stops at ceil(rate m' n') entries.
//  * Entry evaluation: one thread per pass-2 entry (one shadow ray).
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr int kP1Threads = 512;
constexpr int kPairLanes = 8;   // lanes per sibling-pair test
constexpr int kP2Threads = 1024;
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

// ------------------------------------------------------------------ pass 1: main
struct P1Store {
    int32_t* rows;
    float* v0;
    float* v1;
};

__global__ void __launch_bounds__(kP1Threads) k_pass1(lt_frame F, Grid g, float rate, float tau, float dmin2,
                                                      uint64_t seed, P1Plan pl, P1Store st, lt_samples smp,
                                                      int32_t* status) {
    extern __shared__ int32_t sh[];                 // [C+1] prefix of k
    __shared__ int32_t ws[32];
    __shared__ float red[32];
    __shared__ float s_thr;
    const int s = blockIdx.x;
    const int C = F.C, NF = 2 * C - 1;
    const int row0 = F.slice_off[s];
    const int ms = F.slice_off[s + 1] - row0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const float4* pts = reinterpret_cast<const float4*>(F.pts);
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    const int32_t* kk = pl.k + (int64_t)s * C;
    const int32_t* off = pl.off + (int64_t)s * NF;
    int32_t* cnt = pl.cnt + (int64_t)s * NF;
    int32_t* state = pl.state + (int64_t)s * NF;
    float* cost = pl.cost + (int64_t)s * NF;
    const int64_t base = pl.base[s];
    int32_t* rows = st.rows + base;
    float* v0 = st.v0 + base;
    float* v1 = st.v1 + base;
    if (ms == 0) {
        if (threadIdx.x == 0) {
            smp.ncol[s] = 0;
            smp.n1[s] = 0;
            smp.cnt[s] = 0;
        }
        return;
    }
    for (int i = threadIdx.x; i <= C; i += blockDim.x) sh[i] = pl.pfx[(int64_t)s * (C + 1) + i];

    // -- A: rows per cut node, first k distinct Philox draws, sorted ascending
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        const int k = kk[c];
        int32_t* r = rows + off[c];
        int got = 0;
        if (k >= ms) {
            for (int t = 0; t < ms; ++t) r[t] = t;
            got = ms;
        } else {
            for (int t = 0; got < k && t < kMaxDraws; ++t) {
                const int x = (int)uniform_index(philox((uint32_t)t, (uint32_t)c, (uint32_t)s, kTagPass1, seed).x,
                                                 (uint32_t)ms);
                bool dup = false;
                for (int q = 0; q < got; ++q) dup |= (r[q] == x);
                if (!dup) r[got++] = x;
            }
            if (got < k) latch(status, LT_ELIMIT);
            for (int a = 1; a < got; ++a) {  // insertion sort, got <= 64
                const int x = r[a];
                int b = a - 1;
                while (b >= 0 && r[b] > x) {
                    r[b + 1] = r[b];
                    --b;
                }
                r[b + 1] = x;
            }
        }
        cnt[c] = got;
        state[c] = kStAlive;
        cost[c] = 0.f;
    }
    for (int x = C + threadIdx.x; x < NF; x += blockDim.x) {
        cnt[x] = 0;
        state[x] = kStNot;
        cost[x] = 0.f;
    }
    __syncthreads();

    // -- B: initial entries of every cut node; S_hat = sum_c mean(V_c)
    const int K = sh[C];
    float part = 0.f;
    for (int idx = threadIdx.x; idx < K; idx += blockDim.x) {
        int lo = 0, hi = C;  // largest c with sh[c] <= idx
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (sh[mid] <= idx) lo = mid;
            else hi = mid;
        }
        const int c = lo, t = idx - sh[c];
        const int node = F.forest[8 * c];
        const int r = rows[off[c] + t];
        const PointRec P = load_rec(pts, F.m, row0 + r);
        const PointRec L = load_rec(vpls, F.n, F.tree.rep[node]);
        const float v = entry_value(P, L, node_scale(F.tree, vpls, F.n, node), dmin2, g);
        v0[off[c] + t] = v;
        part += v / (float)kk[c];
    }
    part = warp_sum(part);
    if (lane == 0) red[wid] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        float shat = 0.f;
        for (int w = 0; w < nw; ++w) shat += red[w];
        s_thr = tau * shat;
    }
    __syncthreads();
    const float thr = s_thr;

    // -- C: coarsening, one forest level per round, one group of kPairLanes lanes per
    //       sibling pair (most pairs union only a few rows)
    {
        constexpr int GS = kPairLanes;
        const int grp = lane / GS, gl = lane % GS;
        const unsigned gmask = ((GS == 32) ? 0xffffffffu : ((1u << GS) - 1u)) << (grp * GS);
        const unsigned lt_mask = (1u << gl) - 1u;
        const int ngroups = nw * (32 / GS), gid = wid * (32 / GS) + grp;
        for (int h = 1; h <= F.H; ++h) {
            const int l0 = F.level_off[h], l1 = F.level_off[h + 1];
            for (int li = l0 + gid; li < l1; li += ngroups) {
                const int f = F.level_nodes[li];
                const int* fx = F.forest + 8 * f;
                const int a = fx[1], b = fx[2];
                if (state[a] != kStAlive || state[b] != kStAlive) continue;  // uniform in the group
                const int ta = F.forest[8 * a], tb = F.forest[8 * b], tf = fx[0];
                const float Ia = F.tree.I[ta], Ib = F.tree.I[tb], If = F.tree.I[tf];
                const bool p_is_a = Ia >= Ib;
                const int na = cnt[a], nb = cnt[b];
                const int32_t* ra = rows + off[a];
                const int32_t* rb = rows + off[b];
                const float* va = v0 + off[a];
                const float* vb = v0 + off[b];
                int32_t* rf = rows + off[f];
                float* fa = v0 + off[f];
                float* fb = v1 + off[f];
                const float sa = node_scale(F.tree, vpls, F.n, ta), sb = node_scale(F.tree, vpls, F.n, tb);
                const PointRec La = load_rec(vpls, F.n, F.tree.rep[ta]);
                const PointRec Lb = load_rec(vpls, F.n, F.tree.rep[tb]);
                // Union of two sorted row sets: the slot of a row is the number of
                // distinct rows below it, i.e. (rows of a below) + (rows of b below) -
                // (rows in both below); the last term is a running ballot count.
                int common = 0;
                for (int i0 = 0; i0 < na; i0 += GS) {
                    const int i = i0 + gl;
                    int x = 0, pb = 0;
                    bool both = false;
                    if (i < na) {
                        x = ra[i];
                        pb = lower_bound<int32_t>(rb, nb, x);
                        both = pb < nb && rb[pb] == x;
                    }
                    const unsigned bal = (__ballot_sync(gmask, both) >> (grp * GS)) & (gmask >> (grp * GS));
                    if (i < na) {
                        const int slot = i + pb - (common + __popc(bal & lt_mask));
                        float xb;
                        if (both) {
                            xb = vb[pb];
                        } else {
                            const PointRec P = load_rec(pts, F.m, row0 + x);
                            xb = entry_value(P, Lb, sb, dmin2, g);
                        }
                        rf[slot] = x;
                        fa[slot] = va[i];
                        fb[slot] = xb;
                    }
                    common += __popc(bal);
                }
                int seen = 0;  // rows of b (so far) that are also in a
                for (int j0 = 0; j0 < nb; j0 += GS) {
                    const int j = j0 + gl;
                    int y = 0, pa = 0;
                    bool both = false;
                    if (j < nb) {
                        y = rb[j];
                        pa = lower_bound<int32_t>(ra, na, y);
                        both = pa < na && ra[pa] == y;
                    }
                    const unsigned bal = (__ballot_sync(gmask, both) >> (grp * GS)) & (gmask >> (grp * GS));
                    if (j < nb && !both) {
                        const int slot = j + pa - (seen + __popc(bal & lt_mask));
                        const PointRec P = load_rec(pts, F.m, row0 + y);
                        rf[slot] = y;
                        fa[slot] = entry_value(P, La, sa, dmin2, g);
                        fb[slot] = vb[j];
                    }
                    seen += __popc(bal);
                }
                const int nf = na + nb - common;
                __syncwarp(gmask);
                const float rq = p_is_a ? __fdiv_rn(Ib, Ia) : __fdiv_rn(Ia, Ib);
                float e = 0.f;
                for (int i = gl; i < nf; i += GS) {
                    const float vp = p_is_a ? fa[i] : fb[i];
                    const float vq = p_is_a ? fb[i] : fa[i];
                    e = fmaxf(e, fabsf(vq - vp * rq));
                }
#pragma unroll
                for (int o = GS / 2; o > 0; o >>= 1) e = fmaxf(e, __shfl_xor_sync(gmask, e, o, GS));
                const int q = p_is_a ? b : a;
                const float cf = e + cost[q];
                const bool merge = cf < thr;
                if (merge) {
                    const float rfp = __fdiv_rn(If, p_is_a ? Ia : Ib);
                    for (int i = gl; i < nf; i += GS) fa[i] = (p_is_a ? fa[i] : fb[i]) * rfp;
                }
                if (gl == 0) {
                    cnt[f] = nf;
                    cost[f] = cf;
                    state[f] = merge ? kStAlive : kStRejected;
                    if (merge) {
                        state[a] = kStDead;
                        state[b] = kStDead;
                    }
                }
                __syncwarp(gmask);
            }
            __syncthreads();
        }
    }

    // -- D: the coarsened cut in leaf order and its observed entries
    int32_t* mark = sh;  // reuse: [C] forest node whose first leaf is c, else -1
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
    // entry counts -> offsets (in place)
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
        const float* vv = (from_par && F.forest[8 * par + 2] == x) ? v1 + off[src] : v0 + off[src];
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

constexpr int kHashSize = 2 * kP2Threads;
constexpr uint32_t kEmpty = 0xffffffffu;

__global__ void __launch_bounds__(kP2Threads) k_pass2(lt_frame F, const float* __restrict__ weights, float rate,
                                                      uint64_t seed, lt_samples smp, uint32_t* bitmap_all,
                                                      int64_t bitmap_stride, int32_t* status) {
    extern __shared__ unsigned long long cdf[];  // [C]
    __shared__ uint32_t hkey[kHashSize];
    __shared__ int32_t htid[kHashSize];
    __shared__ int32_t ws[32];
    __shared__ float red[32];
    __shared__ unsigned long long s_total;
    const int s = blockIdx.x;
    const int C = F.C;
    const int ms = F.slice_off[s + 1] - F.slice_off[s];
    const int ns = smp.ncol[s];
    const int n1 = smp.n1[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (ms == 0 || ns == 0) {
        if (threadIdx.x == 0) smp.cnt[s] = n1;
        return;
    }
    const int64_t T = (int64_t)ceil((double)rate * (double)ms * (double)ns);
    int64_t need = T - n1;
    if (need <= 0) {
        if (threadIdx.x == 0) smp.cnt[s] = n1;
        return;
    }
    const int64_t capacity = smp.off[s + 1] - smp.off[s];
    if (n1 + need > capacity) {
        if (threadIdx.x == 0) latch(status, LT_ELIMIT);
        need = capacity - n1;
    }
    const float* w = (weights ? weights : smp.g) + (int64_t)s * C;
    // quantised weights -> inclusive integer CDF
    float wm = 0.f;
    for (int j = threadIdx.x; j < ns; j += blockDim.x) wm = fmaxf(wm, w[j]);
    wm = warp_max(wm);
    if (lane == 0) red[wid] = wm;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int i = 0; i < nw; ++i) m = fmaxf(m, red[i]);
        red[0] = m;
    }
    __syncthreads();
    const float wmax = red[0];
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
        const unsigned long long pre = block_exclusive_scan<unsigned long long>(q, (unsigned long long*)hkey, &tot);
        if (j < ns) cdf[j] = carry + pre + q;
        carry += tot;
    }
    if (threadIdx.x == 0) s_total = carry;
    // bitmap of the observed entries: row-major, W words per row
    const int W = (ns + 31) >> 5;
    uint32_t* bm = bitmap_all + (int64_t)s * bitmap_stride;
    for (int64_t i = threadIdx.x; i < (int64_t)ms * W; i += blockDim.x) bm[i] = 0u;
    __syncthreads();
    const uint32_t* key1 = smp.key + smp.off[s];
    for (int i = threadIdx.x; i < n1; i += blockDim.x) {
        const uint32_t k = key1[i];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        atomicOr(bm + (int64_t)r * W + (c >> 5), 1u << (c & 31));
    }
    for (int i = threadIdx.x; i < kHashSize; i += blockDim.x) {
        hkey[i] = kEmpty;
        htid[i] = 0x7fffffff;
    }
    __syncthreads();
    const unsigned long long total = s_total;
    const uint32_t th = (uint32_t)(total >> 32), tl = (uint32_t)total;
    const int64_t cap_draws = 64 * T + 64;
    uint32_t* keyout = smp.key + smp.off[s] + n1;
    int64_t accepted = 0;
    for (int64_t t0 = 0; accepted < need && t0 < cap_draws; t0 += blockDim.x) {
        const int64_t t = t0 + threadIdx.x;
        bool cand = false;
        uint32_t key = 0;
        int hslot = -1;
        int r = 0, c = 0;
        if (t < cap_draws) {
            const U4 x = philox((uint32_t)t, 0u, (uint32_t)s, kTagPass2, seed);
            const unsigned long long u =
                (unsigned long long)x.x * th + (((unsigned long long)x.x * tl) >> 32);
            int lo = 0, hi = ns;  // first c with cdf[c] > u
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (cdf[mid] > u) hi = mid;
                else lo = mid + 1;
            }
            c = lo;
            r = (int)uniform_index(x.y, (uint32_t)ms);
            const bool seen = (bm[(int64_t)r * W + (c >> 5)] >> (c & 31)) & 1u;
            if (!seen) {
                key = (uint32_t)r * (uint32_t)ns + (uint32_t)c;
                uint32_t h = hash32(key) & (kHashSize - 1);
                for (int probe = 0; probe < kHashSize; ++probe) {
                    const uint32_t prev = atomicCAS(&hkey[h], kEmpty, key);
                    if (prev == kEmpty || prev == key) {
                        atomicMin(&htid[h], (int)threadIdx.x);
                        hslot = (int)h;
                        break;
                    }
                    h = (h + 1) & (kHashSize - 1);
                }
                cand = hslot >= 0;
            }
        }
        __syncthreads();
        const bool first = cand && htid[hslot] == (int)threadIdx.x;
        int tot;
        const int rank = block_exclusive_scan<int>(first ? 1 : 0, ws, &tot);
        if (first && accepted + rank < need) {
            keyout[accepted + rank] = ((uint32_t)r << 16) | (uint32_t)c;
            atomicOr(bm + (int64_t)r * W + (c >> 5), 1u << (c & 31));
        }
        accepted += min((int64_t)tot, need - accepted);
        for (int i = threadIdx.x; i < kHashSize; i += blockDim.x) {
            hkey[i] = kEmpty;
            htid[i] = 0x7fffffff;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) smp.cnt[s] = n1 + (int)accepted;
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

template <bool COUNT>
__global__ void __launch_bounds__(128) k_eval_entries(lt_frame F, Grid g, float dmin2, lt_samples smp,
                                                      const int64_t* __restrict__ pfx,
                                                      unsigned long long* __restrict__ stats) {
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
        const int node = smp.col_node[(int64_t)s * F.C + c];
        const PointRec P = load_rec(pts, F.m, F.slice_off[s] + r);
        const PointRec L = load_rec(vpls, F.n, F.tree.rep[node]);
        const float v = entry_value<COUNT>(P, L, node_scale(F.tree, vpls, F.n, node), dmin2, g, &wc, &rays);
        if (COUNT) ++entries;
        else smp.val[e] = v;
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

extern "C" lt_status lt_sample_pass1(lt_ctx* ctx, const lt_frame* f, float rate1, float tau, float d_min,
                                     uint64_t seed, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp) || !(rate1 >= 0.f) || !(tau >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_sample_pass1: bad arguments");
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
    std::vector<int64_t> tot(S), basev(S);
    LT_CUDA(ctx, cudaMemcpyAsync(tot.data(), pl.total, S * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int64_t acc = 0;
    for (int s = 0; s < S; ++s) {
        basev[s] = acc;
        acc += tot[s];
    }
    LT_CUDA(ctx, cudaMemcpyAsync(pl.base, basev.data(), S * sizeof(int64_t), cudaMemcpyHostToDevice, ctx->stream));
    char* q = (char*)lt_scratch(ctx, SCR_P1_STORE, (size_t)std::max<int64_t>(acc, 1) * 12 + 1024, &st);
    if (!q) return st;
    P1Store store;
    store.rows = (int32_t*)q;
    store.v0 = (float*)(q + ((acc * 4 + 255) & ~255LL));
    store.v1 = (float*)(q + 2 * ((acc * 4 + 255) & ~255LL));
    const size_t shm = (size_t)(C + 1) * sizeof(int32_t);
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_pass1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_pass1<<<S, kP1Threads, shm, ctx->stream>>>(*f, ctx->grid, rate1, tau, d_min * d_min, seed, pl, store, *smp,
                                                 ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_pass1");
    // memory stays referenced by the stream: the host vectors were consumed by the
    // synchronous copy above and the async upload below must finish before return
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LT_OK;
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
    const size_t shm = (size_t)C * 8;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_pass2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_pass2<<<S, kP2Threads, shm, ctx->stream>>>(*f, weights, rate, seed, *smp, bm, stride, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_pass2");
    return LT_OK;
}

extern "C" lt_status lt_eval_entries(lt_ctx* ctx, const lt_frame* f, float d_min, lt_samples* smp) {
    if (!ctx || !frame_ok(f) || !samples_ok(smp)) return lt_fail(ctx, LT_EINVAL, "lt_eval_entries: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_eval_entries: no scene uploaded");
    cudaSetDevice(ctx->device);
    lt_status st;
    int64_t* pfx = (int64_t*)lt_scratch(ctx, SCR_MISC, (size_t)(f->S + 1) * 8, &st);
    if (!pfx) return st;
    k_count_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, f->S, pfx);
    LT_LAUNCH_CHECK(ctx, "k_count_prefix");
    const size_t shm = (size_t)(f->S + 1) * 8;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_eval_entries<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)shm));
    k_eval_entries<false><<<ctx->num_sms * 16, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, *smp, pfx,
                                                                        nullptr);
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
// symbol names a host-side stand-in, so the real address is looked up once per
// device (with that device current) and cached.
lt_status noalloc_prefix(lt_ctx* ctx, int64_t** out) {
    if (ctx->device < 0 || ctx->device >= kNoAllocMaxDevices)
        return lt_fail(ctx, LT_EINVAL, "lt_eval_entries_noalloc: device index out of range");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[ctx->device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_prefix);
        if (e != cudaSuccess) return lt_cuda_check(ctx, e, "cudaGetSymbolAddress(g_noalloc_prefix)");
        g_noalloc_addr[ctx->device] = (int64_t*)p;
    }
    *out = g_noalloc_addr[ctx->device];
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
    k_eval_entries<false><<<ctx->num_sms * 16, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, *smp, pfx,
                                                                        nullptr);
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
    k_eval_entries<true><<<ctx->num_sms * 16, 128, shm, ctx->stream>>>(*f, ctx->grid, d_min * d_min, copy, pfx,
                                                                       stats);
    LT_LAUNCH_CHECK(ctx, "k_eval_entries<count>");
    unsigned long long h[4];
    LT_CUDA(ctx, cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 4; ++i) stats_host[i] = (int64_t)h[i];
    return LT_OK;
}
