// Nonnegative completion of the slices by the alternating direction method (App. A).
//
// The appendix iterates on a dense Z (m' x n'), equal to M on Omega and to X Y
// elsewhere.  Here Z is never formed: with S = P_Omega(M - X Y) (nonzero on Omega
// only), Z_k = X_k Y_k + S_k, and the two factor steps become
//
//   X_{k+1} = X_k + (S_k Y_k^T + alpha (U_k - X_k) - Lambda_k) (Y_k Y_k^T + alpha I)^-1
//   Y_{k+1} = (B + beta I)^-1 (C Y_k + X_{k+1}^T S_k + beta V_k - Pi_k),
//             B = X_{k+1}^T X_{k+1},  C = X_{k+1}^T X_k,
//
// which are the appendix's X and Y steps rewritten exactly (the first uses
// X_k (A + alpha I) - alpha X_k = X_k A).  The entries of S_k are formed in the X step,
// where x_i (of X_k) and y_j (of Y_k) are at hand, and stored per observed entry for
// the Y step, so the state per slice is X (two buffers: the Y step needs X_k and
// X_{k+1}), U, Lambda, Y, V, Pi and the |Omega| residuals.
//
// One cluster of K CTAs (K = 2, 4 or 8, so that the whole grid is resident at
// two CTAs per SM where possible) completes one slice and runs all iterations in
// one launch.  Per iteration: (1) the X step, a group of G lanes per row of the CTA's
// rows (G a power of two sized by the slice's mean row length; the lanes split the
// row's entries two at a time, reduce with shuffles and split the r output
// components), with the U and Lambda updates fused and no barrier between rows;
// then the CTA's part of B and C from its rows staged through shared memory;
// cluster barrier; (2) every CTA sums the K partial Gram matrices from distributed
// shared memory in rank order (so every CTA holds the same bits), inverts
// B + beta I by Gauss-Jordan in one warp and forms D = (B + beta I)^-1 C; the Y step
// per column of the CTA's columns (residual through the CSC -> CSR slot map, row of
// X_{k+1}) with the V and Pi updates fused, and the CTA's part of the next Y Y^T;
// cluster barrier; (3) the next (Y Y^T + alpha I)^-1 and the slice's Y staged in
// shared memory for the next X step.  All reads of data written in the launch by
// other CTAs go to L2 (ld.global.cg): L1 is not coherent across SMs.
#include <cooperative_groups.h>
#include <math.h>

#include <algorithm>

#include "lt_internal.cuh"
#include "lt_omega.cuh"

using namespace ltk;
namespace cg = cooperative_groups;

namespace {

constexpr int kAdmMaxK = 8;                  // CTAs per slice (one cluster), at most
constexpr int kAdmThreads = 256;
constexpr int kAdmChunk = 128;               // rows per chunk of a Gram pass
constexpr size_t kAdmStageBytes = 96 * 1024; // Y staged in shared memory up to this size

struct AdmArgs {
    float* X0;   // [m][R]  X_k / X_{k+1} alternate between X0 (the output) and X1
    float* X1;
    float* Up;   // [m][R]  U of App. A (the projected copy of X)
    float* Lam;  // [m][R]  Lambda
    float* Y;    // [S][C][R]  Y^T (the output)
    float* Vp;   // [S][C][R]  V^T
    float* Pi;   // [S][C][R]  Pi^T
    float* S;    // [E]  residual m_ij - x_i . y_j of each observed entry (CSR order)
    const int32_t* ordr;  // [m]        rows of each slice ordered by class (k_adm_order)
    const int32_t* ordc;  // [S][C]     columns of each slice ordered by class
    const int32_t* ncls;  // [S][2][8]  lines per class, rows then columns
    int R;
    const int32_t* rk;
    int iters;
    float alpha_rel, gamma;
    int stage_cap;   // factor rows the shared buffer holds: Y (X) is staged when n'_s (m'_s) fits
};

// a factor row of stride R into RP registers (zeros beyond R), from L2
template <int RP>
__device__ __forceinline__ void load_row_cg(const float* __restrict__ p, int R, float (&v)[RP]) {
    if (R == RP) {
#pragma unroll
        for (int c = 0; c < RP; c += 4) {
            const float4 q = __ldcg(reinterpret_cast<const float4*>(p + c));
            v[c] = q.x, v[c + 1] = q.y, v[c + 2] = q.z, v[c + 3] = q.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < RP; ++c) v[c] = c < R ? __ldcg(p + c) : 0.f;
    }
}


// Group-size class of a line of `len` entries: the line gets G = 2^g lanes, the
// smallest with at most kAdmLaneEntries entries per lane (g <= 5).
constexpr int kAdmLaneEntries = 32;
constexpr int kAdmClasses = 6;

__device__ __forceinline__ int adm_class(int len) {
    int g = 0;
    while (g < kAdmClasses - 1 && len > (kAdmLaneEntries << g)) ++g;
    return g;
}

// Lines of every slice and side ordered by class, largest class first and by line
// index within a class (a stable counting sort, so the order is deterministic), and
// the count of each class.  Block (s, side): side 0 the rows, 1 the columns.
__global__ void k_adm_order(lt_frame F, lt_samples smp, Omega om, int32_t* __restrict__ ordr,
                            int32_t* __restrict__ ordc, int32_t* __restrict__ ncls) {
    __shared__ int32_t ws[32];
    __shared__ int32_t cnt[kAdmClasses], base[kAdmClasses];
    const int s = blockIdx.x, side = blockIdx.y;
    const int row0 = F.slice_off[s];
    const int n = side ? smp.ncol[s] : F.slice_off[s + 1] - row0;
    const int32_t* ptr = side ? om.cp + (int64_t)s * (F.C + 1) : om.rp + row0 + s;
    int32_t* ord = side ? ordc + (int64_t)s * F.C : ordr + row0;
    if (threadIdx.x < kAdmClasses) cnt[threadIdx.x] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&cnt[adm_class(ptr[i + 1] - ptr[i])], 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        int P = 0;
        for (int g = kAdmClasses - 1; g >= 0; --g) {
            base[g] = P;
            P += cnt[g];
            ncls[((int64_t)s * 2 + side) * 8 + g] = cnt[g];
        }
    }
    __syncthreads();
    for (int i0 = 0; i0 < n; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const int g = i < n ? adm_class(ptr[i + 1] - ptr[i]) : -1;
        for (int c = kAdmClasses - 1; c >= 0; --c) {
            int32_t tot;
            const int32_t before = block_exclusive_scan<int32_t>(g == c ? 1 : 0, ws, &tot);
            if (g == c) ord[base[c] + before] = i;
            __syncthreads();
            if (threadIdx.x == 0) base[c] += tot;
            __syncthreads();
        }
    }
}

// The lines of one side that a CTA (rank k of K) takes: the class-g lines at sorted
// positions pos0[g] + k + K q, q < n[g], in warp tasks of 32 / 2^g lines, tasks of
// the largest class first.
struct AdmSched {
    int n[kAdmClasses], pos0[kAdmClasses], t0[kAdmClasses], tend[kAdmClasses];
    int lines, tasks;
};

__device__ __forceinline__ void make_sched(const int32_t* __restrict__ cnt, int k, int K, AdmSched& sc) {
    int P = 0, T = 0, L = 0;
    for (int g = kAdmClasses - 1; g >= 0; --g) {
        const int c = cnt[g];
        sc.pos0[g] = P;
        P += c;
        sc.n[g] = c > k ? (c - k + K - 1) / K : 0;
        L += sc.n[g];
        sc.t0[g] = T;
        T += (sc.n[g] + (32 >> g) - 1) >> (5 - g);
        sc.tend[g] = T;
    }
    sc.lines = L;
    sc.tasks = T;
}

// sorted position of the CTA's local line l (0 <= l < sc.lines; classes in task order)
__device__ __forceinline__ int sched_pos(const AdmSched& sc, int l, int k, int K) {
    int g = kAdmClasses - 1;
    while (l >= sc.n[g]) l -= sc.n[g--];
    return sc.pos0[g] + k + K * l;
}

// Offset in shared memory of float4 chunk q of staged factor row j: the chunk index
// is XOR-swizzled by the row's place in its 128-byte bank line, so that a warp
// gathering chunk q of random rows spreads over all banks.
template <int RP>
__device__ __forceinline__ int sy_chunk(int j, int q) {
    constexpr int CPR = RP / 4, RPL = CPR >= 8 ? 1 : 8 / CPR;
    return j * RP + 4 * (q ^ ((j / RPL) % CPR));
}

// Inverse of the symmetric positive definite M + add I (RP x RP, row-major in shared
// memory) by Gauss-Jordan elimination without pivoting in one warp: lane l holds
// columns l and l + 32 of [M + add I | I].
template <int RP>
__device__ void gj_inverse(const float* __restrict__ M, float add, float* __restrict__ inv, int lane) {
    constexpr int NC = 2 * RP, CPL = (NC + 31) / 32;
    float col[CPL][RP];
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lane + 32 * q;
#pragma unroll
        for (int i = 0; i < RP; ++i) {
            float v = 0.f;
            if (c < RP)
                v = M[i * RP + c] + (i == c ? add : 0.f);
            else if (c < NC)
                v = (i == c - RP) ? 1.f : 0.f;
            col[q][i] = v;
        }
    }
#pragma unroll
    for (int k = 0; k < RP; ++k) {
        const float p = __shfl_sync(0xffffffffu, col[0][k], k);  // pivot, column k (lane k)
        float f[RP];
#pragma unroll
        for (int i = 0; i < RP; ++i) f[i] = __shfl_sync(0xffffffffu, col[0][i], k);
        const float ip = 1.f / p;
#pragma unroll
        for (int q = 0; q < CPL; ++q) {
            const float rk = col[q][k] * ip;
            col[q][k] = rk;
#pragma unroll
            for (int i = 0; i < RP; ++i)
                if (i != k) col[q][i] = fmaf(-f[i], rk, col[q][i]);
        }
    }
#pragma unroll
    for (int q = 0; q < CPL; ++q) {
        const int c = lane + 32 * q;
        if (c >= RP && c < NC) {
#pragma unroll
            for (int i = 0; i < RP; ++i) inv[i * RP + (c - RP)] = col[q][i];
        }
    }
}

// sum over the cluster's CTAs, in rank order, of the partial matrices at `part`
// (n floats each) into `out` (this CTA's shared memory)
__device__ __forceinline__ void cluster_sum(cg::cluster_group& cl, int K, float* part, float* out, int n) {
    for (int e = threadIdx.x; e < n; e += blockDim.x) {
        float t = 0.f;
        for (int q = 0; q < K; ++q) t += cl.map_shared_rank(part, q)[e];
        out[e] = t;
    }
}

// Gram partials over a tile of `nt` rows: g += N^T N, or N^T O when O is given
template <int RP, int NE>
__device__ __forceinline__ void tile_gram(const float* __restrict__ N, const float* __restrict__ O, int nt,
                                          float (&g)[NE]) {
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = threadIdx.x + kAdmThreads * q;
        if (e < RP * RP) {
            const int a = e / RP, b = e % RP;
            float t = g[q];
            for (int i = 0; i < nt; ++i) t = fmaf(N[i * RP + a], (O ? O : N)[i * RP + b], t);
            g[q] = t;
        }
    }
}

// g1 += N^T N and, when O is given, g2 += N^T O over n factor rows of stride R (row
// l at N + line(l) R), staged through `buf` (2 kAdmChunk RP floats of shared memory)
// in chunks; every thread of the CTA calls it
template <int RP, int NE, class Line>
__device__ void gram_rows(const float* N, const float* O, int n, int R, Line line, float* __restrict__ buf,
                          float (&g1)[NE], float (&g2)[NE]) {
    float* bn = buf;
    float* bo = buf + kAdmChunk * RP;
    for (int base = 0; base < n; base += kAdmChunk) {
        const int nt = min(kAdmChunk, n - base);
        for (int e = threadIdx.x; e < nt * RP; e += kAdmThreads) {
            const int i = e / RP, c = e % RP;
            const int64_t at = (int64_t)line(base + i) * R + c;
            bn[e] = c < R ? __ldcg(N + at) : 0.f;
            if (O) bo[e] = c < R ? __ldcg(O + at) : 0.f;
        }
        __syncthreads();
        tile_gram<RP, NE>(bn, nullptr, nt, g1);
        if (O) tile_gram<RP, NE>(bn, bo, nt, g2);
        __syncthreads();
    }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = threadIdx.x < kAdmThreads / 32 ? red[threadIdx.x] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;  // valid in warp 0
}

template <int RP, int NE>
__device__ __forceinline__ void store_part(float* part, const float (&g)[NE]) {
#pragma unroll
    for (int q = 0; q < NE; ++q) {
        const int e = threadIdx.x + kAdmThreads * q;
        if (e < RP * RP) part[e] = g[q];
    }
}

// butterfly sum of acc over the G lanes of a group (every lane gets the same bits)
template <int RP>
__device__ __forceinline__ void group_reduce(float (&acc)[RP], int G, unsigned gmask) {
    for (int off = G >> 1; off > 0; off >>= 1) {
#pragma unroll
        for (int c = 0; c < RP; ++c) acc[c] += __shfl_xor_sync(gmask, acc[c], off);
    }
}

// stage n factor rows of stride R into shared memory, swizzled
template <int RP>
__device__ __forceinline__ void stage_rows(float* sm, const float* src, int n, int R) {
    for (int e = threadIdx.x; e < n * RP; e += kAdmThreads) {
        const int j = e / RP, c = e % RP;
        sm[sy_chunk<RP>(j, c >> 2) + (c & 3)] = c < R ? src[(int64_t)j * R + c] : 0.f;
    }
}

// a factor row from the staged copy or from global memory (plain loads: every
// reader is ordered after the writer by a cluster or CTA barrier)
template <int RP>
__device__ __forceinline__ void load_f(bool staged, const float* sm, const float* src, int j, int R,
                                       float (&y)[RP]) {
    if (staged) {
#pragma unroll
        for (int q = 0; q < RP / 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(sm + sy_chunk<RP>(j, q));
            y[4 * q] = t.x, y[4 * q + 1] = t.y, y[4 * q + 2] = t.z, y[4 * q + 3] = t.w;
        }
    } else if (R == RP) {
#pragma unroll
        for (int q = 0; q < RP / 4; ++q) {
            const float4 t = *reinterpret_cast<const float4*>(src + (int64_t)j * R + 4 * q);
            y[4 * q] = t.x, y[4 * q + 1] = t.y, y[4 * q + 2] = t.z, y[4 * q + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int c = 0; c < RP; ++c) y[c] = c < R ? src[(int64_t)j * R + c] : 0.f;
    }
}

constexpr int kAdmBatch = 8;  // entries whose indices a lane loads at once

template <int RP>
__global__ void __launch_bounds__(kAdmThreads, 2) k_adm(lt_frame F, lt_samples smp, Omega om, AdmArgs a, SeedRef sr) {
    constexpr int NE = (RP * RP + kAdmThreads - 1) / kAdmThreads;
    __shared__ __align__(16) float sInv[RP * RP];   // (A + alpha I)^-1, then (B + beta I)^-1
    __shared__ __align__(16) float sD[RP * RP];     // (B + beta I)^-1 C
    __shared__ __align__(16) float sM[2 * RP * RP]; // reduced A, or B and C
    __shared__ __align__(16) float sPartA[RP * RP + 1];
    __shared__ __align__(16) float sPartBC[2 * RP * RP];
    __shared__ float sRed[32];
    __shared__ float sAB[2];                        // alpha, beta
    // the slice's Y^T [n'][RP] during the X step; Gram staging otherwise
    extern __shared__ __align__(16) float sY[];

    cg::cluster_group cl = cg::this_cluster();
    const int K = (int)cl.dim_blocks().x;
    const int k = (int)cl.block_rank();
    const int s = blockIdx.x / K;
    const int tid = threadIdx.x;
    const int R = a.R;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0;
    const int ns = smp.ncol[s], ne = smp.cnt[s];
    const int64_t o = smp.off[s];
    const int r = slice_rank(a.rk, s, R);
    const float mu = om.mu[s];
    const int rlo = (int)((int64_t)k * ms / K), rhi = (int)((int64_t)(k + 1) * ms / K);
    const int clo = (int)((int64_t)k * ns / K), chi = (int)((int64_t)(k + 1) * ns / K);
    float* Yb = a.Y + (int64_t)s * F.C * R;
    float* Vb = a.Vp + (int64_t)s * F.C * R;
    float* Pb = a.Pi + (int64_t)s * F.C * R;
    float* Sr = a.S + o;  // residual of each observed entry, CSC order
    const int32_t* rp = om.rp + row0 + s;
    const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
    const uint16_t* cidx = om.cidx + o;
    const float* cval = om.cval + o;
    const uint16_t* ridx = om.ridx + o;
    const int32_t* r2c = om.r2c + o;

    if (ne == 0 || !(mu > 0.f)) {
        // nothing observed, or an all-zero slice: the zero factors fit
        for (int64_t e = tid; e < (int64_t)(rhi - rlo) * R; e += kAdmThreads)
            a.X0[(int64_t)(row0 + rlo) * R + e] = 0.f;
        for (int64_t e = tid; e < (int64_t)(chi - clo) * R; e += kAdmThreads) Yb[(int64_t)clo * R + e] = 0.f;
        cl.sync();
        return;
    }
    const uint64_t seed = sr.get();
    const float amp = sqrtf(mu / (float)r);
    const bool staged = ns <= a.stage_cap, staged_x = ms <= a.stage_cap;

    // ---- start: Y0 as the ALS start (Philox (k, j, slice, 3)), X0 from (k, i, slice, 6);
    // U0 = X0, V0 = Y0, Lambda0 = Pi0 = 0; the CTA's parts of Y0 Y0^T and ||X0||^2
    for (int64_t e = tid; e < (int64_t)(chi - clo) * R; e += kAdmThreads) {
        const int j = clo + (int)(e / R), c = (int)(e % R);
        float v = 0.f;
        if (c < r) {
            const uint32_t w = philox((uint32_t)c, (uint32_t)j, slice_key(F.slice_id, s), kTagAlsInit, seed).x;
            v = amp * (0.5f + (float)w * 2.3283064365386963e-10f);
        }
        const int64_t at = (int64_t)j * R + c;
        Yb[at] = v;
        Vb[at] = v;
        Pb[at] = 0.f;
    }
    float ssx = 0.f;
    for (int64_t e = tid; e < (int64_t)(rhi - rlo) * R; e += kAdmThreads) {
        const int i = rlo + (int)(e / R), c = (int)(e % R);
        float v = 0.f;
        if (c < r) {
            const uint32_t w = philox((uint32_t)c, (uint32_t)i, slice_key(F.slice_id, s), kTagAdmInit, seed).x;
            v = amp * (0.5f + (float)w * 2.3283064365386963e-10f);
        }
        const int64_t at = (int64_t)(row0 + i) * R + c;
        a.X0[at] = v;
        a.Up[at] = v;
        a.Lam[at] = 0.f;
        ssx = fmaf(v, v, ssx);
    }
    ssx = block_sum(ssx, sRed);  // its barriers also order the Y0 writes before the Gram
    float gA[NE], gB[NE], gC[NE];
#pragma unroll
    for (int q = 0; q < NE; ++q) gA[q] = 0.f;
    gram_rows<RP, NE>(Yb, nullptr, chi - clo, R, [&](int l) { return clo + l; }, sY, gA, gA);
    store_part<RP, NE>(sPartA, gA);
    if (tid == 0) sPartA[RP * RP] = ssx;
    __threadfence();
    cl.sync();
    cluster_sum(cl, K, sPartA, sM, RP * RP + 1);
    __syncthreads();
    if (tid == 0) {
        float tr = 0.f;
        for (int c = 0; c < RP; ++c) tr += sM[c * RP + c];
        sAB[0] = a.alpha_rel * tr / (float)r;            // alpha = alpha_rel ||Y0||^2 / r
        sAB[1] = a.alpha_rel * sM[RP * RP] / (float)r;   // beta = alpha_rel ||X0||^2 / r
    }
    __syncthreads();
    const float alpha = sAB[0], beta = sAB[1], gamma = a.gamma;
    if (tid < 32) gj_inverse<RP>(sM, alpha, sInv, tid);
    if (staged) stage_rows<RP>(sY, Yb, ns, R);
    __syncthreads();

    __shared__ AdmSched shr, shc;  // the CTA's rows and columns
    if (tid == 0) {
        make_sched(a.ncls + (int64_t)s * 16, k, K, shr);
        make_sched(a.ncls + (int64_t)s * 16 + 8, k, K, shc);
    }
    __syncthreads();
    const int32_t* ordr = a.ordr + row0;
    const int32_t* ordc = a.ordc + (int64_t)s * F.C;
    const int warp = tid >> 5, lane32 = tid & 31;
    for (int it = 0; it < a.iters; ++it) {
        const float* Xc = (it & 1) ? a.X1 : a.X0;  // X_k
        float* Xn = (it & 1) ? a.X0 : a.X1;        // X_{k+1}
        // ---- X step: a warp task = 32 / G rows of one class, G lanes per row -----------
        for (int tau = warp; tau < shr.tasks; tau += kAdmThreads / 32) {
            int g = kAdmClasses - 1;
            while (tau >= shr.tend[g]) --g;
            const int G = 1 << g, lane = lane32 & (G - 1);
            const int q = (tau - shr.t0[g]) * (32 >> g) + (lane32 >> g);
            if (q >= shr.n[g]) continue;  // a whole group leaves together
            const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane32 & ~(G - 1)));
            const int i = ordr[shr.pos0[g] + k + K * q];
            const int64_t row = (int64_t)(row0 + i) * R;
            float xo[RP], acc[RP];
            load_row_cg<RP>(Xc + row, R, xo);
#pragma unroll
            for (int c = 0; c < RP; ++c) acc[c] = 0.f;
            const int e1 = rp[i + 1];
            for (int e0 = rp[i] + lane; e0 < e1; e0 += kAdmBatch * G) {
                int jj[kAdmBatch], ss[kAdmBatch];
                float mm[kAdmBatch];
#pragma unroll
                for (int u = 0; u < kAdmBatch; ++u) {
                    const int e = e0 + u * G;
                    jj[u] = e < e1 ? cidx[e] : -1;
                    mm[u] = e < e1 ? cval[e] : 0.f;
                    ss[u] = e < e1 ? r2c[e] : 0;
                }
#pragma unroll
                for (int u = 0; u < kAdmBatch; ++u) {
                    if (jj[u] < 0) break;
                    float y[RP];
                    load_f<RP>(staged, sY, Yb, jj[u], R, y);
                    float d = mm[u];
#pragma unroll
                    for (int c = 0; c < RP; ++c) d = fmaf(-xo[c], y[c], d);
                    Sr[ss[u]] = d;
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(d, y[c], acc[c]);
                }
            }
            if (lane == 0) {  // alpha (U_k - X_k) - Lambda_k, once per row
                float u[RP], lm[RP];
                load_row_cg<RP>(a.Up + row, R, u);
                load_row_cg<RP>(a.Lam + row, R, lm);
#pragma unroll
                for (int c = 0; c < RP; ++c) acc[c] += fmaf(alpha, u[c] - xo[c], -lm[c]);
            }
            group_reduce<RP>(acc, G, gmask);
            for (int c = lane; c < R; c += G) {
                float v = __ldcg(Xc + row + c);
#pragma unroll
                for (int q2 = 0; q2 < RP; ++q2) v = fmaf(acc[q2], sInv[q2 * RP + c], v);
                const float lam = __ldcg(a.Lam + row + c);
                const float u = fmaxf(0.f, v + lam / alpha);
                Xn[row + c] = v;
                a.Up[row + c] = u;
                a.Lam[row + c] = lam + gamma * alpha * (v - u);
            }
        }
        __syncthreads();  // the CTA's new rows are written; sY is free
        {
#pragma unroll
            for (int q = 0; q < NE; ++q) gB[q] = gC[q] = 0.f;
            auto line = [&](int l) { return row0 + ordr[sched_pos(shr, l, k, K)]; };
            gram_rows<RP, NE>(Xn, Xc, shr.lines, R, line, sY, gB, gC);
            store_part<RP, NE>(sPartBC, gB);
            store_part<RP, NE>(sPartBC + RP * RP, gC);
        }
        __threadfence();
        cl.sync();
        // ---- (B + beta I)^-1 and D = (B + beta I)^-1 C ----------------------------
        cluster_sum(cl, K, sPartBC, sM, 2 * RP * RP);
        __syncthreads();
        if (tid < 32) gj_inverse<RP>(sM, beta, sInv, tid);
        __syncthreads();
        for (int e = tid; e < RP * RP; e += kAdmThreads) {
            const int c = e / RP, b = e % RP;
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < RP; ++q) t = fmaf(sInv[c * RP + q], sM[RP * RP + q * RP + b], t);
            sD[e] = t;
        }
        __syncthreads();
        if (staged_x) stage_rows<RP>(sY, Xn + (int64_t)row0 * R, ms, R);
        __syncthreads();
        // ---- Y step: a warp task = 32 / G columns of one class --------------------------
        for (int tau = warp; tau < shc.tasks; tau += kAdmThreads / 32) {
            int g = kAdmClasses - 1;
            while (tau >= shc.tend[g]) --g;
            const int G = 1 << g, lane = lane32 & (G - 1);
            const int q = (tau - shc.t0[g]) * (32 >> g) + (lane32 >> g);
            if (q >= shc.n[g]) continue;
            const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane32 & ~(G - 1)));
            const int j = ordc[shc.pos0[g] + k + K * q];
            const int64_t col = (int64_t)j * R;
            float yo[RP], acc[RP];
            load_row_cg<RP>(Yb + col, R, yo);
#pragma unroll
            for (int c = 0; c < RP; ++c) acc[c] = 0.f;
            const int e1 = cp[j + 1];
            const float* Xs = Xn + (int64_t)row0 * R;
            for (int e0 = cp[j] + lane; e0 < e1; e0 += kAdmBatch * G) {
                int ii[kAdmBatch];
                float sv[kAdmBatch];
#pragma unroll
                for (int u = 0; u < kAdmBatch; ++u) {
                    const int e = e0 + u * G;
                    ii[u] = e < e1 ? ridx[e] : -1;
                    sv[u] = e < e1 ? Sr[e] : 0.f;
                }
#pragma unroll
                for (int u = 0; u < kAdmBatch; ++u) {
                    if (ii[u] < 0) break;
                    float x[RP];
                    load_f<RP>(staged_x, sY, Xs, ii[u], R, x);
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(sv[u], x[c], acc[c]);
                }
            }
            if (lane == 0) {  // beta V_k - Pi_k, once per column
                float v[RP], pv[RP];
                load_row_cg<RP>(Vb + col, R, v);
                load_row_cg<RP>(Pb + col, R, pv);
#pragma unroll
                for (int c = 0; c < RP; ++c) acc[c] += fmaf(beta, v[c], -pv[c]);
            }
            group_reduce<RP>(acc, G, gmask);
            for (int c = lane; c < R; c += G) {
                float v = 0.f;
#pragma unroll
                for (int q2 = 0; q2 < RP; ++q2) v = fmaf(sD[c * RP + q2], yo[q2], v);
#pragma unroll
                for (int q2 = 0; q2 < RP; ++q2) v = fmaf(sInv[c * RP + q2], acc[q2], v);
                const float pi = __ldcg(Pb + col + c);
                const float vv = fmaxf(0.f, v + pi / beta);
                Yb[col + c] = v;
                Vb[col + c] = vv;
                Pb[col + c] = pi + gamma * beta * (v - vv);
            }
        }
        __syncthreads();
        {
#pragma unroll
            for (int q = 0; q < NE; ++q) gA[q] = 0.f;
            auto line = [&](int l) { return ordc[sched_pos(shc, l, k, K)]; };
            gram_rows<RP, NE>(Yb, nullptr, shc.lines, R, line, sY, gA, gA);
            store_part<RP, NE>(sPartA, gA);
        }
        __threadfence();
        cl.sync();
        if (it + 1 < a.iters) {
            // ---- next (A + alpha I)^-1 and the staged Y ------------------------------
            cluster_sum(cl, K, sPartA, sM, RP * RP);
            __syncthreads();
            if (tid < 32) gj_inverse<RP>(sM, alpha, sInv, tid);
            if (staged) stage_rows<RP>(sY, Yb, ns, R);
            __syncthreads();
        }
    }
    // X_iters sits in X1 after an odd count: copy the CTA's rows to the output
    if (a.iters & 1)
        for (int64_t e = tid; e < (int64_t)(rhi - rlo) * R; e += kAdmThreads) {
            const int64_t at = (int64_t)(row0 + rlo) * R + e;
            a.X0[at] = __ldcg(a.X1 + at);
        }
    cl.sync();  // no CTA leaves while another may still read its shared memory
}

template <int RP>
lt_status launch_adm(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, const AdmArgs& a,
                     SeedRef sr) {
    const size_t dyn = (size_t)std::max(2 * kAdmChunk, a.stage_cap) * RP * 4;
    LT_CUDA(ctx, cudaFuncSetAttribute(k_adm<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    // the largest cluster (8, 4 or 2 CTAs) with which all slices fit at two CTAs per SM
    int K = kAdmMaxK;
    while (K > 2 && (int64_t)f->S * K > 2 * (int64_t)ctx->num_sms) K >>= 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(f->S * K));
    cfg.blockDim = dim3(kAdmThreads);
    cfg.dynamicSmemBytes = dyn;
    cfg.stream = ctx->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)K;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    LT_CUDA(ctx, cudaLaunchKernelEx(&cfg, k_adm<RP>, *f, *smp, om, a, sr));
    LT_LAUNCH_CHECK(ctx, "k_adm");
    return LT_OK;
}

}  // namespace

extern "C" lt_status lt_complete_adm(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                                     float alpha_rel, float gamma, uint64_t seed, lt_factors* uv) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->key || !smp->val || !smp->off || !smp->cnt || !smp->ncol || !uv ||
        !uv->U || !uv->V || uv->r < 1 || uv->r > 32 || iters < 0 || !(alpha_rel > 0.f) || !(gamma > 0.f) ||
        !(gamma < 1.618f))
        return lt_fail(ctx, LT_EINVAL, "lt_complete_adm: bad arguments");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C, R = uv->r;
    int64_t E = 0;
    if (ctx->use_plan) {
        E = ctx->plan.entries;
    } else {
        LT_CUDA(ctx, cudaMemcpyAsync(&E, smp->off + S, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        ctx->plan.entries = E;
    }
    Omega om;
    lt_status st = omega_build(ctx, f, smp, E, false, true, &om);
    if (st != LT_OK) return st;
    const size_t nx = (size_t)f->m * R, ny = (size_t)S * C * R;
    auto up = [](size_t n) { return (n * 4 + 255) & ~(size_t)255; };
    char* p = (char*)lt_scratch(ctx, SCR_ADM,
                                3 * up(nx) + 2 * up(ny) + up((size_t)E) + up((size_t)f->m) + up((size_t)S * C) +
                                    up((size_t)S * 16),
                                &st);
    if (!p) return st;
    AdmArgs a;
    a.X0 = uv->U;
    a.X1 = (float*)p;
    a.Up = (float*)(p + up(nx));
    a.Lam = (float*)(p + 2 * up(nx));
    a.Y = uv->V;
    a.Vp = (float*)(p + 3 * up(nx));
    a.Pi = (float*)(p + 3 * up(nx) + up(ny));
    a.S = (float*)(p + 3 * up(nx) + 2 * up(ny));
    int32_t* ordr = (int32_t*)(p + 3 * up(nx) + 2 * up(ny) + up((size_t)E));
    int32_t* ordc = (int32_t*)((char*)ordr + up((size_t)f->m));
    int32_t* ncls = (int32_t*)((char*)ordc + up((size_t)S * C));
    a.ordr = ordr;
    a.ordc = ordc;
    a.ncls = ncls;
    k_adm_order<<<dim3(S, 2), 1024, 0, ctx->stream>>>(*f, *smp, om, ordr, ordc, ncls);
    LT_LAUNCH_CHECK(ctx, "k_adm_order");
    a.R = R;
    a.rk = uv->rank;
    a.iters = iters;
    a.alpha_rel = alpha_rel;
    a.gamma = gamma;
    const int RP = R <= 8 ? 8 : R <= 16 ? 16 : 32;
    a.stage_cap = (int)(kAdmStageBytes / ((size_t)RP * 4));
    const SeedRef sr = seed_ref(ctx, seed);
    if (RP == 8) return launch_adm<8>(ctx, f, smp, om, a, sr);
    if (RP == 16) return launch_adm<16>(ctx, f, smp, om, a, sr);
    return launch_adm<32>(ctx, f, smp, om, a, sr);
}
