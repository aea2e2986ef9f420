// Completion of the slices from their sampled entries and the factorised render.
//
//  * Omega build: per slice, the observed entries are placed in row-major (CSR) and
//    column-major (CSC) order through two occupancy bitmaps; the position of an entry
//    is a popcount of the bits before it, so the layout is deterministic.
//  * Masked ALS (the completion M_s ~= U_s V_s^T at rank r; Sec. 5 uses the factor
//    form M = X Y): one group of G lanes (G = 8, 16 or 32 >= r) solves one row (or
//    column).  Lane k owns row k of the r x r Gram matrix in registers; the factor
//    row of every observed entry is broadcast with shuffles.  The ridge-regularised
//    Gram is factored by an in-register Cholesky; when the float32 pivots spread
//    beyond 1e6 the group repeats the row in float64.
//  * Render (Sec. 3 step 5): t_s = V_s^T w, pixel = max(0, u_i . t_s).
#include <math.h>

#include <algorithm>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr float kPivotRatio = 1e-6f;

struct Omega {
    int32_t* rp;        // [m + S]      row pointers, slice s rows at slice_off[s] + s
    int32_t* cp;        // [S][C + 1]   column pointers
    uint16_t* cidx;     // [off[S]]     CSR column of each entry
    float* cval;        // [off[S]]
    uint16_t* ridx;     // [off[S]]     CSC row of each entry
    float* rval;        // [off[S]]
    float* mu;          // [S] mean observed value
    uint32_t* bm;       // row-major bitmaps
    uint32_t* bt;       // column-major bitmaps
    int64_t bm_stride, bt_stride;
    int64_t* line_pfx;  // [S + 1] prefix of n'_s (V-step lines)
};

__device__ __forceinline__ int popc_prefix(const uint32_t* words, int bit) {
    int c = 0;
    const int w = bit >> 5;
    for (int i = 0; i < w; ++i) c += __popc(words[i]);
    const uint32_t mask = (bit & 31) ? ((1u << (bit & 31)) - 1u) : 0u;
    return c + __popc(words[w] & mask);
}

__global__ void __launch_bounds__(1024) k_omega(lt_frame F, lt_samples smp, Omega om, int32_t* status) {
    __shared__ int32_t ws[32];
    __shared__ float red[32];
    const int s = blockIdx.x;
    const int C = F.C;
    const int row0 = F.slice_off[s];
    const int ms = F.slice_off[s + 1] - row0;
    const int ns = smp.ncol[s];
    const int ne = smp.cnt[s];
    const int W = (ns + 31) >> 5, WT = (ms + 31) >> 5;
    uint32_t* bm = om.bm + (int64_t)s * om.bm_stride;
    uint32_t* bt = om.bt + (int64_t)s * om.bt_stride;
    const uint32_t* key = smp.key + smp.off[s];
    const float* val = smp.val + smp.off[s];
    for (int64_t i = threadIdx.x; i < (int64_t)ms * W; i += blockDim.x) bm[i] = 0u;
    for (int64_t i = threadIdx.x; i < (int64_t)ns * WT; i += blockDim.x) bt[i] = 0u;
    __syncthreads();
    float sum = 0.f;
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
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
        om.mu[s] = ne > 0 ? t / (float)ne : 0.f;
    }
    // row and column pointers
    int32_t* rp = om.rp + row0 + s;
    int carry = 0;
    for (int r0 = 0; r0 < ms; r0 += blockDim.x) {
        const int r = r0 + threadIdx.x;
        int c = 0;
        if (r < ms)
            for (int w = 0; w < W; ++w) c += __popc(bm[(int64_t)r * W + w]);
        int tot;
        const int pre = block_exclusive_scan<int>(c, ws, &tot);
        if (r < ms) rp[r] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) rp[ms] = carry;
    int32_t* cp = om.cp + (int64_t)s * (C + 1);
    carry = 0;
    for (int c0 = 0; c0 < ns; c0 += blockDim.x) {
        const int c = c0 + threadIdx.x;
        int n = 0;
        if (c < ns)
            for (int w = 0; w < WT; ++w) n += __popc(bt[(int64_t)c * WT + w]);
        int tot;
        const int pre = block_exclusive_scan<int>(n, ws, &tot);
        if (c < ns) cp[c] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) cp[ns] = carry;
    __syncthreads();
    const int64_t o = smp.off[s];
    for (int e = threadIdx.x; e < ne; e += blockDim.x) {
        const uint32_t k = key[e];
        const int r = (int)(k >> 16), c = (int)(k & 0xffffu);
        if (r >= ms || c >= ns) continue;
        const int pr = rp[r] + popc_prefix(bm + (int64_t)r * W, c);
        const int pc = cp[c] + popc_prefix(bt + (int64_t)c * WT, r);
        om.cidx[o + pr] = (uint16_t)c;
        om.cval[o + pr] = val[e];
        om.ridx[o + pc] = (uint16_t)r;
        om.rval[o + pc] = val[e];
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

__global__ void k_als_init(lt_frame F, lt_samples smp, Omega om, int r, uint64_t seed, float* __restrict__ V) {
    const int s = blockIdx.y;
    const int ns = smp.ncol[s];
    const float amp = sqrtf(fmaxf(om.mu[s], 0.f) / (float)r);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns * r; i += gridDim.x * blockDim.x) {
        const int j = i / r, k = i % r;
        const uint32_t w = philox((uint32_t)k, (uint32_t)j, (uint32_t)s, kTagAlsInit, seed).x;
        V[((int64_t)s * F.C + j) * r + k] = amp * (0.5f + (float)w * 2.3283064365386963e-10f);
    }
}

// Solve one line in scalar type T.  Returns false when the factorisation is not
// acceptable in float (non-positive or badly spread pivots).
template <int G, typename T>
__device__ __forceinline__ bool solve_line(int len, const uint16_t* __restrict__ idx, const float* __restrict__ val,
                                           const float* __restrict__ Fb, int r, float lam_rel, int k, T* Lsh,
                                           T* out_k, bool check) {
    const unsigned FULL = 0xffffffffu;
    T acc[G];
#pragma unroll
    for (int c = 0; c < G; ++c) acc[c] = T(0);
    T rhs = T(0);
    // warp-uniform trip count: every group of the warp runs max(len) steps
    int lmax = len;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmax = max(lmax, __shfl_xor_sync(FULL, lmax, o));
    for (int e = 0; e < lmax; ++e) {
        T fk = T(0), a = T(0);
        if (e < len) {
            const int j = idx[e];
            a = (T)val[e];
            if (k < r) fk = (T)__ldg(Fb + (int64_t)j * r + k);
        }
#pragma unroll
        for (int c = 0; c < G; ++c) {
            const T fc = __shfl_sync(FULL, fk, c, G);
            acc[c] += fk * fc;
        }
        rhs += a * fk;
    }
    // trace and ridge
    T tr = acc[0] * T(0);
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
#pragma unroll
    for (int j = 0; j < G; ++j) {
        T djj = __shfl_sync(FULL, acc[j], j, G);
        if (j < r) {
            ok &= (djj > T(0));
            dmin = djj < dmin ? djj : dmin;
            dmax = djj > dmax ? djj : dmax;
        }
        const T ljj = sqrt(djj > T(0) ? djj : T(1));
        const T lij = (k > j) ? acc[j] / ljj : (k == j ? ljj : T(0));
        acc[j] = lij;
#pragma unroll
        for (int c = j + 1; c < G; ++c) {
            const T lcj = __shfl_sync(FULL, lij, c, G);
            if (k > j) acc[c] -= lij * lcj;
        }
    }
    if (check && !zero && (!ok || dmin < (T)kPivotRatio * dmax)) return false;
    // triangular solves through shared memory (row k of L)
#pragma unroll
    for (int c = 0; c < G; ++c) Lsh[k * G + c] = acc[c];
    __syncwarp();
    // forward: L y = b (lane k holds b_k)
    T y = rhs;
    for (int j = 0; j < G; ++j) {
        const T yj = __shfl_sync(FULL, y, j, G) / Lsh[j * G + j];
        if (k == j) y = yj;
        else if (k > j) y -= Lsh[k * G + j] * yj;
    }
    // backward: L^T x = y
    T x = y;
    for (int j = G - 1; j >= 0; --j) {
        const T xj = __shfl_sync(FULL, x, j, G) / Lsh[j * G + j];
        if (k == j) x = xj;
        else if (k < j) x -= Lsh[j * G + k] * xj;
    }
    __syncwarp();
    *out_k = (zero || k >= r) ? T(0) : x;
    return true;
}

// One half-step: lines are slice rows (U-step, rows_side = true) or slice columns.
template <int G>
constexpr int als_warps() { return G == 32 ? 4 : 8; }

template <int G>
__global__ void __launch_bounds__(32 * als_warps<G>()) k_als_half(lt_frame F, lt_samples smp, Omega om, int r,
                                                                  float lam_rel, bool rows_side,
                                                                  const float* __restrict__ Fin,
                                                                  float* __restrict__ Fout, int32_t* n_fp64) {
    __shared__ double Lsh_all[als_warps<G>()][32 / G][G * G];
    __shared__ int64_t spfx[1025];
    const int S = F.S;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int grp = lane / G, k = lane % G;
    const int gpw = 32 / G;
    int64_t nlines;
    if (rows_side) {
        for (int i = threadIdx.x; i <= S; i += blockDim.x) spfx[i] = F.slice_off[i];
        nlines = F.m;
    } else {
        for (int i = threadIdx.x; i <= S; i += blockDim.x) spfx[i] = om.line_pfx[i];
        __syncthreads();
        nlines = spfx[S];
    }
    __syncthreads();
    const int64_t warps_total = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t wglobal = (int64_t)blockIdx.x * (blockDim.x >> 5) + wid;
    for (int64_t base = wglobal * gpw; base < nlines; base += warps_total * gpw) {
        const int64_t line = base + grp;
        const bool live = line < nlines;
        int s = 0, len = 0;
        const uint16_t* idx = nullptr;
        const float* vv = nullptr;
        const float* Fb = Fin;
        float* dst = nullptr;
        if (live) {
            int lo = 0, hi = S;
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (spfx[mid] <= line) lo = mid;
                else hi = mid;
            }
            s = lo;
            const int64_t o = smp.off[s];
            if (rows_side) {
                const int rloc = (int)(line - F.slice_off[s]);
                const int32_t* rp = om.rp + F.slice_off[s] + s;
                const int b = rp[rloc];
                len = rp[rloc + 1] - b;
                idx = om.cidx + o + b;
                vv = om.cval + o + b;
                Fb = Fin + (int64_t)s * F.C * r;                 // V of the slice
                dst = Fout + line * r;                            // U row
            } else {
                const int c = (int)(line - spfx[s]);
                const int32_t* cp = om.cp + (int64_t)s * (F.C + 1);
                const int b = cp[c];
                len = cp[c + 1] - b;
                idx = om.ridx + o + b;
                vv = om.rval + o + b;
                Fb = Fin + (int64_t)F.slice_off[s] * r;          // U rows of the slice
                dst = Fout + ((int64_t)s * F.C + c) * r;          // V row
            }
        }
        float* Lf = reinterpret_cast<float*>(&Lsh_all[wid][grp][0]);
        float xf;
        const bool okf = solve_line<G, float>(len, idx, vv, Fb, r, lam_rel, k, Lf, &xf, true);
        const unsigned bad = __ballot_sync(0xffffffffu, live && !okf);
        if (bad) {
            double xd;
            solve_line<G, double>(len, idx, vv, Fb, r, lam_rel, k, &Lsh_all[wid][grp][0], &xd, false);
            if (live && !okf) {
                xf = (float)xd;
                if (k == 0) atomicAdd(n_fp64, 1);
            }
        }
        if (live && k < r) dst[k] = xf;
    }
}

__global__ void k_render(lt_frame F, lt_samples smp, const float* __restrict__ U, const float* __restrict__ V,
                         int r, const float* __restrict__ w, const int32_t* __restrict__ perm,
                         float* __restrict__ img) {
    __shared__ float t[32];
    __shared__ float part[8][32];
    const int s = blockIdx.y;
    const int ns = smp.ncol[s];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // t_s = V_s^T w: warp wid sums columns wid, wid+8, ...; lane k owns component k
    float acc = 0.f;
    if (lane < r)
        for (int j = wid; j < ns; j += blockDim.x >> 5)
            acc += V[((int64_t)s * F.C + j) * r + lane] * (w ? w[(int64_t)s * F.C + j] : 1.f);
    part[wid][lane] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float a = 0.f;
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) a += part[i][threadIdx.x];
        t[threadIdx.x] = a;
    }
    __syncthreads();
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ms; i += gridDim.x * blockDim.x) {
        const float* u = U + (int64_t)(row0 + i) * r;
        float v = 0.f;
        for (int k = 0; k < r; ++k) v += u[k] * t[k];
        img[perm[row0 + i]] = fmaxf(v, 0.f);
    }
}

bool frame_ok2(const lt_frame* f) {
    return f && f->slice_off && f->S > 0 && f->S <= 1024 && f->m > 0 && f->C >= 1 && f->max_rows >= 0 &&
           f->max_rows <= 65535;
}

}  // namespace

extern "C" lt_status lt_complete(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, int32_t iters,
                                 float lam_rel, uint64_t seed, lt_factors* uv) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->key || !smp->val || !smp->off || !smp->cnt || !smp->ncol || !uv ||
        !uv->U || !uv->V || uv->r < 1 || uv->r > 32 || iters < 0 || !(lam_rel >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_complete: bad arguments");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C;
    std::vector<int64_t> off(S + 1);
    LT_CUDA(ctx, cudaMemcpyAsync(off.data(), smp->off, (S + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const int64_t E = off[S];
    const int64_t mr = std::max(f->max_rows, 1);
    Omega om;
    om.bm_stride = mr * ((C + 31) / 32);
    om.bt_stride = (int64_t)C * ((mr + 31) / 32);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_OMEGA,
                                (size_t)(f->m + S) * 4 + (size_t)S * (C + 1) * 4 + (size_t)E * 12 + S * 8 +
                                    (size_t)S * (om.bm_stride + om.bt_stride) * 4 + (S + 1) * 8 + 16 * 256,
                                &st);
    if (!p) return st;
    auto take = [&](size_t nbytes) {
        char* q = p;
        p += (nbytes + 255) & ~(size_t)255;
        return q;
    };
    om.rp = (int32_t*)take((f->m + S) * 4);
    om.cp = (int32_t*)take((size_t)S * (C + 1) * 4);
    om.cidx = (uint16_t*)take(E * 2);
    om.cval = (float*)take(E * 4);
    om.ridx = (uint16_t*)take(E * 2);
    om.rval = (float*)take(E * 4);
    om.mu = (float*)take(S * 4);
    om.bm = (uint32_t*)take((size_t)S * om.bm_stride * 4);
    om.bt = (uint32_t*)take((size_t)S * om.bt_stride * 4);
    om.line_pfx = (int64_t*)take((S + 1) * 8);
    int32_t* n64 = (int32_t*)lt_scratch(ctx, SCR_ALS, 256, &st);
    if (!n64) return st;
    LT_CUDA(ctx, cudaMemsetAsync(n64, 0, 4, ctx->stream));
    k_omega<<<S, 1024, 0, ctx->stream>>>(*f, *smp, om, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_omega");
    k_line_prefix<<<1, 1024, 0, ctx->stream>>>(*smp, S, om.line_pfx);
    LT_LAUNCH_CHECK(ctx, "k_line_prefix");
    const int r = uv->r;
    k_als_init<<<dim3(8, S), 256, 0, ctx->stream>>>(*f, *smp, om, r, seed, uv->V);
    LT_LAUNCH_CHECK(ctx, "k_als_init");
    const int blocks = ctx->num_sms * 4;
    for (int it = 0; it < iters; ++it) {
        for (int side = 0; side < 2; ++side) {
            const bool rows = side == 0;
            const float* fin = rows ? uv->V : uv->U;
            float* fout = rows ? uv->U : uv->V;
            if (r <= 8)
                k_als_half<8><<<blocks, 32 * als_warps<8>(), 0, ctx->stream>>>(*f, *smp, om, r, lam_rel, rows, fin,
                                                                                fout, n64);
            else if (r <= 16)
                k_als_half<16><<<blocks, 32 * als_warps<16>(), 0, ctx->stream>>>(*f, *smp, om, r, lam_rel, rows, fin,
                                                                                  fout, n64);
            else
                k_als_half<32><<<2 * blocks, 32 * als_warps<32>(), 0, ctx->stream>>>(*f, *smp, om, r, lam_rel, rows,
                                                                                      fin, fout, n64);
            LT_LAUNCH_CHECK(ctx, "k_als_half");
        }
    }
    return LT_OK;
}

extern "C" lt_status lt_render(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_factors* uv,
                               const float* w, const int32_t* row_perm, float* img) {
    if (!ctx || !frame_ok2(f) || !smp || !smp->ncol || !uv || !uv->U || !uv->V || uv->r < 1 || uv->r > 32 ||
        !row_perm || !img)
        return lt_fail(ctx, LT_EINVAL, "lt_render: bad arguments");
    cudaSetDevice(ctx->device);
    const int per = std::max(1, std::min(64, (int)((f->max_rows + 255) / 256)));
    k_render<<<dim3(per, f->S), 256, 0, ctx->stream>>>(*f, *smp, uv->U, uv->V, uv->r, w, row_perm, img);
    LT_LAUNCH_CHECK(ctx, "k_render");
    return LT_OK;
}
