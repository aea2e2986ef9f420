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
    int R;
    const int32_t* rk;
    int iters;
    float alpha_rel, gamma;
    int stage_cols;  // Y is staged in shared memory when n'_s <= stage_cols
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

template <int RP>
__device__ __forceinline__ void load_row_smem(const float* __restrict__ p, float (&v)[RP]) {
#pragma unroll
    for (int c = 0; c < RP; c += 4) {
        const float4 q = *reinterpret_cast<const float4*>(p + c);
        v[c] = q.x, v[c + 1] = q.y, v[c + 2] = q.z, v[c + 3] = q.w;
    }
}

// group size for lines of mean length L: the smallest power of two in [2, 32] with
// at most about 6 entries per lane
__device__ __forceinline__ int group_size(int64_t entries, int lines) {
    const int64_t L = lines > 0 ? (entries + lines - 1) / lines : 0;
    int G = 2;
    while (G < 32 && (int64_t)G * 6 < L) G <<= 1;
    return G;
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

// g1 += N^T N and, when O is given, g2 += N^T O over the n factor rows of stride R
// that start at N and O, staged through `buf` (2 kAdmChunk RP floats of shared
// memory) in chunks; every thread of the CTA calls it
template <int RP, int NE>
__device__ void gram_rows(const float* N, const float* O, int n, int R, float* __restrict__ buf, float (&g1)[NE],
                          float (&g2)[NE]) {
    float* bn = buf;
    float* bo = buf + kAdmChunk * RP;
    for (int base = 0; base < n; base += kAdmChunk) {
        const int nt = min(kAdmChunk, n - base);
        for (int e = threadIdx.x; e < nt * RP; e += kAdmThreads) {
            const int i = e / RP, c = e % RP;
            const int64_t at = (int64_t)(base + i) * R + c;
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

template <int RP>
__device__ __forceinline__ void load_y(bool staged, const float* sY, const float* Yb, int j, int R, float (&y)[RP]) {
    if (staged)
        load_row_smem<RP>(sY + j * RP, y);
    else
        load_row_cg<RP>(Yb + (int64_t)j * R, R, y);
}

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
    float* Sr = a.S + o;  // residual of each observed entry, CSR order
    const int32_t* rp = om.rp + row0 + s;
    const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
    const uint16_t* cidx = om.cidx + o;
    const float* cval = om.cval + o;
    const uint16_t* ridx = om.ridx + o;
    const int32_t* c2r = om.c2r + o;

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
    const bool staged = ns <= a.stage_cols;

    // ---- start: Y0 as the ALS start (Philox (k, j, slice, 3)), X0 from (k, i, slice, 6);
    // U0 = X0, V0 = Y0, Lambda0 = Pi0 = 0; the CTA's parts of Y0 Y0^T and ||X0||^2
    for (int64_t e = tid; e < (int64_t)(chi - clo) * R; e += kAdmThreads) {
        const int j = clo + (int)(e / R), c = (int)(e % R);
        float v = 0.f;
        if (c < r) {
            const uint32_t w = philox((uint32_t)c, (uint32_t)j, (uint32_t)s, kTagAlsInit, seed).x;
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
            const uint32_t w = philox((uint32_t)c, (uint32_t)i, (uint32_t)s, kTagAdmInit, seed).x;
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
    gram_rows<RP, NE>(Yb + (int64_t)clo * R, nullptr, chi - clo, R, sY, gA, gA);
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
    if (staged)
        for (int e = tid; e < ns * RP; e += kAdmThreads) {
            const int j = e / RP, c = e % RP;
            sY[e] = c < R ? __ldcg(Yb + (int64_t)j * R + c) : 0.f;
        }
    __syncthreads();

    const int Gx = group_size(ne, ms), Gy = group_size(ne, ns);
    for (int it = 0; it < a.iters; ++it) {
        const float* Xc = (it & 1) ? a.X1 : a.X0;  // X_k
        float* Xn = (it & 1) ? a.X0 : a.X1;        // X_{k+1}
        // ---- X step: a group of Gx lanes per row, no barrier between rows ----------
        {
            const int G = Gx, ng = kAdmThreads / G, lane = tid % G;
            const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
            for (int i = rlo + tid / G; i < rhi; i += ng) {
                const int64_t row = (int64_t)(row0 + i) * R;
                float xo[RP], acc[RP];
                load_row_cg<RP>(Xc + row, R, xo);
#pragma unroll
                for (int c = 0; c < RP; ++c) acc[c] = 0.f;
                const int e1 = rp[i + 1];
                int e = rp[i] + lane;
                for (; e + G < e1; e += 2 * G) {  // two entries in flight
                    const int j0 = cidx[e], j1 = cidx[e + G];
                    float d0 = cval[e], d1 = cval[e + G];
                    float y0[RP], y1[RP];
                    load_y<RP>(staged, sY, Yb, j0, R, y0);
                    load_y<RP>(staged, sY, Yb, j1, R, y1);
#pragma unroll
                    for (int c = 0; c < RP; ++c) {
                        d0 = fmaf(-xo[c], y0[c], d0);
                        d1 = fmaf(-xo[c], y1[c], d1);
                    }
                    Sr[e] = d0;
                    Sr[e + G] = d1;
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(d1, y1[c], fmaf(d0, y0[c], acc[c]));
                }
                if (e < e1) {
                    float y0[RP];
                    load_y<RP>(staged, sY, Yb, cidx[e], R, y0);
                    float d0 = cval[e];
#pragma unroll
                    for (int c = 0; c < RP; ++c) d0 = fmaf(-xo[c], y0[c], d0);
                    Sr[e] = d0;
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(d0, y0[c], acc[c]);
                }
                // the lane that owns component c adds alpha (u_c - x_c) - lambda_c
#pragma unroll
                for (int c = 0; c < RP; ++c)
                    if (c < R && (c & (G - 1)) == lane)
                        acc[c] += fmaf(alpha, __ldcg(a.Up + row + c) - xo[c], -__ldcg(a.Lam + row + c));
                group_reduce<RP>(acc, G, gmask);
                for (int c = lane; c < R; c += G) {
                    float v = __ldcg(Xc + row + c);
#pragma unroll
                    for (int q = 0; q < RP; ++q) v = fmaf(acc[q], sInv[q * RP + c], v);
                    const float lam = __ldcg(a.Lam + row + c);
                    const float u = fmaxf(0.f, v + lam / alpha);
                    Xn[row + c] = v;
                    a.Up[row + c] = u;
                    a.Lam[row + c] = lam + gamma * alpha * (v - u);
                }
            }
            __syncthreads();  // the CTA's new rows are written; sY is free
#pragma unroll
            for (int q = 0; q < NE; ++q) gB[q] = gC[q] = 0.f;
            gram_rows<RP, NE>(Xn + (int64_t)(row0 + rlo) * R, Xc + (int64_t)(row0 + rlo) * R, rhi - rlo, R, sY, gB,
                              gC);
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
        // ---- Y step: a group of Gy lanes per column -----------------------------------
        {
            const int G = Gy, ng = kAdmThreads / G, lane = tid % G;
            const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
            for (int j = clo + tid / G; j < chi; j += ng) {
                const int64_t col = (int64_t)j * R;
                float yo[RP], acc[RP];
                load_row_cg<RP>(Yb + col, R, yo);
#pragma unroll
                for (int c = 0; c < RP; ++c) acc[c] = 0.f;
                const int e1 = cp[j + 1];
                int e = cp[j] + lane;
                for (; e + G < e1; e += 2 * G) {
                    const int i0 = ridx[e], i1 = ridx[e + G];
                    const float s0 = __ldcg(Sr + c2r[e]), s1 = __ldcg(Sr + c2r[e + G]);
                    float x0[RP], x1[RP];
                    load_row_cg<RP>(Xn + (int64_t)(row0 + i0) * R, R, x0);
                    load_row_cg<RP>(Xn + (int64_t)(row0 + i1) * R, R, x1);
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(s1, x1[c], fmaf(s0, x0[c], acc[c]));
                }
                if (e < e1) {
                    const float s0 = __ldcg(Sr + c2r[e]);
                    float x0[RP];
                    load_row_cg<RP>(Xn + (int64_t)(row0 + ridx[e]) * R, R, x0);
#pragma unroll
                    for (int c = 0; c < RP; ++c) acc[c] = fmaf(s0, x0[c], acc[c]);
                }
                // the lane that owns component c adds beta v_c - pi_c
#pragma unroll
                for (int c = 0; c < RP; ++c)
                    if (c < R && (c & (G - 1)) == lane)
                        acc[c] += fmaf(beta, __ldcg(Vb + col + c), -__ldcg(Pb + col + c));
                group_reduce<RP>(acc, G, gmask);
                for (int c = lane; c < R; c += G) {
                    float v = 0.f;
#pragma unroll
                    for (int q = 0; q < RP; ++q) v = fmaf(sD[c * RP + q], yo[q], v);
#pragma unroll
                    for (int q = 0; q < RP; ++q) v = fmaf(sInv[c * RP + q], acc[q], v);
                    const float pi = __ldcg(Pb + col + c);
                    const float vv = fmaxf(0.f, v + pi / beta);
                    Yb[col + c] = v;
                    Vb[col + c] = vv;
                    Pb[col + c] = pi + gamma * beta * (v - vv);
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < NE; ++q) gA[q] = 0.f;
            gram_rows<RP, NE>(Yb + (int64_t)clo * R, nullptr, chi - clo, R, sY, gA, gA);
            store_part<RP, NE>(sPartA, gA);
        }
        __threadfence();
        cl.sync();
        if (it + 1 < a.iters) {
            // ---- next (A + alpha I)^-1 and the staged Y ------------------------------
            cluster_sum(cl, K, sPartA, sM, RP * RP);
            __syncthreads();
            if (tid < 32) gj_inverse<RP>(sM, alpha, sInv, tid);
            if (staged)
                for (int e = tid; e < ns * RP; e += kAdmThreads) {
                    const int j = e / RP, c = e % RP;
                    sY[e] = c < R ? __ldcg(Yb + (int64_t)j * R + c) : 0.f;
                }
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
    const size_t dyn = (size_t)std::max(2 * kAdmChunk, a.stage_cols) * RP * 4;
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
    char* p = (char*)lt_scratch(ctx, SCR_ADM, 3 * up(nx) + 2 * up(ny) + up((size_t)E), &st);
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
    a.R = R;
    a.rk = uv->rank;
    a.iters = iters;
    a.alpha_rel = alpha_rel;
    a.gamma = gamma;
    const int RP = R <= 8 ? 8 : R <= 16 ? 16 : 32;
    a.stage_cols = (int)std::min<size_t>((size_t)C, kAdmStageBytes / ((size_t)RP * 4));
    const SeedRef sr = seed_ref(ctx, seed);
    if (RP == 8) return launch_adm<8>(ctx, f, smp, om, a, sr);
    if (RP == 16) return launch_adm<16>(ctx, f, smp, om, a, sr);
    return launch_adm<32>(ctx, f, smp, om, a, sr);
}
