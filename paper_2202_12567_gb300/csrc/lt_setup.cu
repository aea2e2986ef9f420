// Setup of a frame: light tree and conservative global cut (Sec. 3 step 1, the
// splitting test parallel over the nodes of a level, Sec. 6), the cut's ancestor
// forest used by the coarsening, and the slicing of the matrix rows by k-means on
// position and normal (Sec. 3 step 2).
//
// Tree: Morton codes (float32 decisions, orientation class above the code), a
// bitonic sort of the unique 64-bit keys, Karras's parallel radix-tree
// construction and a bottom-up pass with one atomic counter per internal node.
#include <math.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

// ------------------------------------------------------------------ bitonic sort
__global__ void k_bitonic_step(unsigned long long* keys, int64_t n, int64_t j, int64_t k) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = i ^ j;
        if (l > i) {
            const unsigned long long a = keys[i], b = keys[l];
            const bool up = (i & k) == 0;
            if ((a > b) == up) {
                keys[i] = b;
                keys[l] = a;
            }
        }
    }
}

lt_status bitonic_sort(lt_ctx* ctx, unsigned long long* keys, int64_t npow2) {
    const int blocks = (int)std::min<int64_t>((npow2 + 255) / 256, 8 * (int64_t)ctx->num_sms);
    for (int64_t k = 2; k <= npow2; k <<= 1)
        for (int64_t j = k >> 1; j > 0; j >>= 1) {
            k_bitonic_step<<<blocks, 256, 0, ctx->stream>>>(keys, npow2, j, k);
            LT_LAUNCH_CHECK(ctx, "k_bitonic_step");
        }
    return LT_OK;
}

int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// ------------------------------------------------------------------ Morton keys
__device__ __forceinline__ uint32_t expand10(uint32_t v) {
    uint32_t out = 0;
    for (int b = 0; b < 10; ++b) out |= ((v >> b) & 1u) << (3 * b);
    return out;
}

__device__ __forceinline__ uint32_t morton3(float3 p, const float* lo, const float* ext) {
    const float pa[3] = {p.x, p.y, p.z};
    uint32_t q[3];
    for (int a = 0; a < 3; ++a) {
        const float x = __fdiv_rn(__fsub_rn(pa[a], lo[a]), ext[a]);
        int v = (int)floorf(__fmul_rn(x, 1024.0f));
        v = v < 0 ? 0 : (v > 1023 ? 1023 : v);
        q[a] = (uint32_t)v;
    }
    return (expand10(q[0]) << 2) | (expand10(q[1]) << 1) | expand10(q[2]);
}

// Single-block bounding box of a float4 plane (xyz of plane 0).
__global__ void k_bbox(const float4* __restrict__ pl, int64_t n, float* out6) {
    __shared__ float red[6][32];
    float lo[3] = {3e38f, 3e38f, 3e38f}, hi[3] = {-3e38f, -3e38f, -3e38f};
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float4 p = pl[i];
        lo[0] = fminf(lo[0], p.x);
        lo[1] = fminf(lo[1], p.y);
        lo[2] = fminf(lo[2], p.z);
        hi[0] = fmaxf(hi[0], p.x);
        hi[1] = fmaxf(hi[1], p.y);
        hi[2] = fmaxf(hi[2], p.z);
    }
    for (int a = 0; a < 3; ++a) {
        lo[a] = warp_min(lo[a]);
        hi[a] = warp_max(hi[a]);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
        for (int a = 0; a < 3; ++a) {
            red[a][wid] = lo[a];
            red[3 + a][wid] = hi[a];
        }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int a = 0; a < 3; ++a) {
            float l = 3e38f, h = -3e38f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
                l = fminf(l, red[a][w]);
                h = fmaxf(h, red[3 + a][w]);
            }
            out6[a] = l;
            const float e = __fsub_rn(h, l);
            out6[3 + a] = e > 0.f ? e : 1.0f;  // extent
        }
    }
}

__global__ void k_vpl_keys(const float4* __restrict__ vpls, int64_t n, const float* __restrict__ box,
                           int64_t npad, unsigned long long* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= n) {
            keys[i] = ~0ull;
            continue;
        }
        const float4 p = vpls[i], nr = vpls[n + i];
        const uint32_t code = morton3(make_float3(p.x, p.y, p.z), box, box + 3);
        int ax = 0;
        float best = fabsf(nr.x);
        if (fabsf(nr.y) > best) {
            ax = 1;
            best = fabsf(nr.y);
        }
        if (fabsf(nr.z) > best) ax = 2;
        const float comp = ax == 0 ? nr.x : (ax == 1 ? nr.y : nr.z);
        const uint32_t cls = 2u * ax + (comp > 0.f ? 1u : 0u);
        const unsigned long long hi = ((unsigned long long)cls << 30) | code;
        keys[i] = (hi << 32) | (unsigned long long)i;
    }
}

__device__ __forceinline__ int delta(const unsigned long long* k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j > n - 1) return -1;
    return __clzll(k[i] ^ k[j]);
}

// Karras (HPG 2012): internal node i finds its key range and its split.
__global__ void k_karras(const unsigned long long* __restrict__ keys, int64_t n, lt_tree T) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n - 1; i += (int64_t)gridDim.x * blockDim.x) {
        const int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) > 0 ? 1 : -1;
        const int dmin = delta(keys, n, i, i - d);
        int64_t lmax = 2;
        while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
        int64_t l = 0;
        for (int64_t t = lmax / 2; t >= 1; t /= 2)
            if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
        const int64_t j = i + l * d;
        const int dnode = delta(keys, n, i, j);
        int64_t s = 0;
        for (int64_t div = 2;; div *= 2) {
            const int64_t t = (l + div - 1) / div;
            if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
            if (t <= 1) break;
        }
        const int64_t gamma = i + s * d + min(d, 0);
        const int64_t a = min(i, j), b = max(i, j);
        const int64_t left = (a == gamma) ? (n - 1 + gamma) : gamma;
        const int64_t right = (b == gamma + 1) ? (n - 1 + gamma + 1) : gamma + 1;
        T.child[2 * i] = (int32_t)left;
        T.child[2 * i + 1] = (int32_t)right;
        T.parent[left] = (int32_t)i;
        T.parent[right] = (int32_t)i;
        T.range[2 * i] = (int32_t)a;
        T.range[2 * i + 1] = (int32_t)b;
    }
}

__global__ void k_tree_leaves(const unsigned long long* __restrict__ keys, const float4* __restrict__ vpls, int64_t n,
                              lt_tree T, int32_t* flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int v = (int)(keys[j] & 0xffffffffu);
        const int64_t node = n - 1 + j;
        const float4 p = vpls[v], nr = vpls[n + v], L = vpls[2 * n + v];
        T.order[j] = v;
        T.child[2 * node] = -1;
        T.child[2 * node + 1] = -1;
        T.range[2 * node] = (int32_t)j;
        T.range[2 * node + 1] = (int32_t)j;
        T.rep[node] = v;
        T.I[node] = __fmul_rn(L.w, p.w);
        const float e = nr.w;
        T.B[node] = e > 0.f ? 0.5f * kInvPi + 0.5f * (e + 2.f) * (0.5f * kInvPi) : kInvPi;
        float* bb = T.aabb + 6 * node;
        bb[0] = p.x;
        bb[1] = p.y;
        bb[2] = p.z;
        bb[3] = p.x;
        bb[4] = p.y;
        bb[5] = p.z;
        if (j < n - 1) flags[j] = 0;
    }
    if (n == 1 && blockIdx.x == 0 && threadIdx.x == 0) T.parent[0] = -1;
}

// Bottom-up records: the second thread to reach a node combines its children.
__global__ void k_tree_up(int64_t n, lt_tree T, int32_t* flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t node = n - 1 + j;
        for (int guard = 0; guard < 128 && node > 0; ++guard) {
            const int p = T.parent[node];
            __threadfence();
            if (atomicAdd(&flags[p], 1) == 0) break;
            __threadfence();
            const int a = T.child[2 * p], b = T.child[2 * p + 1];
            const float Ia = *(volatile float*)&T.I[a], Ib = *(volatile float*)&T.I[b];
            T.I[p] = __fadd_rn(Ia, Ib);
            T.B[p] = fmaxf(*(volatile float*)&T.B[a], *(volatile float*)&T.B[b]);
            T.rep[p] = Ia >= Ib ? *(volatile int*)&T.rep[a] : *(volatile int*)&T.rep[b];
            for (int q = 0; q < 3; ++q) {
                T.aabb[6 * p + q] = fminf(*(volatile float*)&T.aabb[6 * a + q], *(volatile float*)&T.aabb[6 * b + q]);
                T.aabb[6 * p + 3 + q] =
                    fmaxf(*(volatile float*)&T.aabb[6 * a + 3 + q], *(volatile float*)&T.aabb[6 * b + 3 + q]);
            }
            node = p;
        }
    }
}

// ------------------------------------------------------------------ global cut
__device__ __forceinline__ float brdf_max(float alb, float gloss) {
    return gloss > 0.f ? 0.5f * alb * kInvPi + 0.5f * alb * (gloss + 2.f) * (0.5f * kInvPi) : alb * kInvPi;
}

// estimate(x) = sum over cut nodes of the unoccluded A(x, c); one warp per test row.
__global__ void k_cut_estimate(const float4* __restrict__ pts, int64_t m, const float4* __restrict__ vpls, int64_t n,
                               lt_tree T, const int32_t* __restrict__ rows, int64_t nr,
                               const int32_t* __restrict__ cut, int C, float dmin2, float* est) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t x = w; x < nr; x += nw) {
        const PointRec P = load_rec(pts, m, rows[x]);
        float acc = 0.f;
        for (int c = lane; c < C; c += 32) {
            const int node = cut[c];
            const int r = T.rep[node];
            const PointRec L = load_rec(vpls, n, r);
            const float sc = __fdiv_rn(T.I[node], __fmul_rn(L.c.w, L.a.w));
            acc += unoccluded(P, L, dmin2) * sc;
        }
        acc = warp_sum(acc);
        if (lane == 0) est[x] = acc;
    }
}

// error(c) = max over rows of bound(x, c) / estimate(x); one warp per cut node.
__global__ void k_cut_error(const float4* __restrict__ pts, int64_t m, lt_tree T, const int32_t* __restrict__ rows,
                            int64_t nr, const int32_t* __restrict__ cut, int C, const float* __restrict__ est,
                            float dmin2, float* err) {
    const int lane = threadIdx.x & 31;
    const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t ci = w; ci < C; ci += nw) {
        const int node = cut[ci];
        const float* bb = T.aabb + 6 * node;
        const float IB = T.I[node] * T.B[node];
        float e = 0.f;
        for (int64_t x = lane; x < nr; x += 32) {
            const PointRec P = load_rec(pts, m, rows[x]);
            const float gx = fmaxf(0.f, fmaxf(bb[0] - P.a.x, P.a.x - bb[3]));
            const float gy = fmaxf(0.f, fmaxf(bb[1] - P.a.y, P.a.y - bb[4]));
            const float gz = fmaxf(0.f, fmaxf(bb[2] - P.a.z, P.a.z - bb[5]));
            const float d2 = gx * gx + gy * gy + gz * gz;
            const float b = IB * brdf_max(P.a.w, P.b.w) / fmaxf(d2, dmin2);
            const float ex = est[x];
            const float ratio = ex > 0.f ? b / ex : (b > 0.f ? INFINITY : 0.f);
            e = fmaxf(e, ratio);
        }
        e = warp_max(e);
        if (lane == 0) err[ci] = e;
    }
}

// ------------------------------------------------------------------ k-means
__global__ void k_point_keys(const float4* __restrict__ pts, int64_t m, const float* __restrict__ box, int64_t npad,
                             unsigned long long* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= m) {
            keys[i] = ~0ull;
            continue;
        }
        const float4 p = pts[i];
        keys[i] = ((unsigned long long)morton3(make_float3(p.x, p.y, p.z), box, box + 3) << 32) |
                  (unsigned long long)i;
    }
}

__device__ __forceinline__ void feature(const float4* pts, int64_t m, int64_t i, float w, float* f) {
    const float4 p = pts[i], nr = pts[m + i];
    f[0] = p.x;
    f[1] = p.y;
    f[2] = p.z;
    f[3] = w * nr.x;
    f[4] = w * nr.y;
    f[5] = w * nr.z;
}

__global__ void k_kmeans_seed(const float4* __restrict__ pts, int64_t m, const unsigned long long* __restrict__ keys,
                              int S, float w, float* cen) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
        const int64_t rank = (2 * (int64_t)k + 1) * m / (2 * (int64_t)S);
        const int64_t i = (int64_t)(keys[rank] & 0xffffffffu);
        feature(pts, m, i, w, cen + 6 * k);
    }
}

__global__ void k_kmeans_assign(const float4* __restrict__ pts, int64_t m, int S, float w,
                                const float* __restrict__ cen, int32_t* __restrict__ lab, double* sums) {
    extern __shared__ float sc[];  // [S][6]
    for (int i = threadIdx.x; i < 6 * S; i += blockDim.x) sc[i] = cen[i];
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        float f[6];
        feature(pts, m, i, w, f);
        int best = 0;
        float bd = 3e38f;
        for (int k = 0; k < S; ++k) {
            float d = 0.f;
            for (int a = 0; a < 6; ++a) {
                const float t = f[a] - sc[6 * k + a];
                d += t * t;
            }
            if (d < bd) {
                bd = d;
                best = k;
            }
        }
        lab[i] = best;
        if (sums) {
            double* sk = sums + 7 * best;
            for (int a = 0; a < 6; ++a) atomicAdd(sk + a, (double)f[a]);
            atomicAdd(sk + 6, 1.0);
        }
    }
}

__global__ void k_kmeans_update(int S, const double* __restrict__ sums, float* cen) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < S; k += gridDim.x * blockDim.x) {
        const double cnt = sums[7 * k + 6];
        if (cnt > 0)
            for (int a = 0; a < 6; ++a) cen[6 * k + a] = (float)(sums[7 * k + a] / cnt);
    }
}

__global__ void k_label_keys(const int32_t* __restrict__ lab, int64_t m, int64_t npad, unsigned long long* keys,
                             int32_t* counts) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= m) {
            keys[i] = ~0ull;
            continue;
        }
        keys[i] = ((unsigned long long)lab[i] << 32) | (unsigned long long)i;
        atomicAdd(&counts[lab[i]], 1);
    }
}

__global__ void k_perm_from_keys(const unsigned long long* __restrict__ keys, int64_t m, int32_t* perm) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        perm[i] = (int32_t)(keys[i] & 0xffffffffu);
}

bool tree_ok(const lt_tree* t) {
    return t && t->n >= 1 && t->order && t->child && t->parent && t->range && t->rep && t->I && t->B && t->aabb;
}

// ------------------------------------------------------------------ triangle BVH
// Linear BVH over triangles (the paper casts its shadow rays through a BVH, Sec. 6):
// Morton codes of the centroids in the centroids' box, sorted with the triangle index
// below them, the Karras topology, leaf boxes and a bottom-up refit.
__global__ void k_tri_prep(const float* __restrict__ tris, int64_t nt, float4* __restrict__ cen,
                           float4* __restrict__ rec) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt; i += (int64_t)gridDim.x * blockDim.x) {
        const float* t = tris + 9 * i;
        const float3 a = make_float3(t[0], t[1], t[2]), b = make_float3(t[3], t[4], t[5]),
                     c = make_float3(t[6], t[7], t[8]);
        cen[i] = make_float4((a.x + b.x + c.x) * (1.f / 3.f), (a.y + b.y + c.y) * (1.f / 3.f),
                             (a.z + b.z + c.z) * (1.f / 3.f), 0.f);
        rec[3 * i] = make_float4(a.x, a.y, a.z, 0.f);
        rec[3 * i + 1] = make_float4(b.x - a.x, b.y - a.y, b.z - a.z, 0.f);
        rec[3 * i + 2] = make_float4(c.x - a.x, c.y - a.y, c.z - a.z, 0.f);
    }
}

__global__ void k_tri_keys(const float4* __restrict__ cen, int64_t nt, const float* __restrict__ box, int64_t npad,
                           unsigned long long* keys) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npad; i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= nt) {
            keys[i] = ~0ull;
            continue;
        }
        const float4 c = cen[i];
        keys[i] = ((unsigned long long)morton3(make_float3(c.x, c.y, c.z), box, box + 3) << 32) |
                  (unsigned long long)i;
    }
}

__global__ void k_bvh_leaves(const unsigned long long* __restrict__ keys, const float* __restrict__ tris, int64_t nt,
                             int32_t* __restrict__ leaf_tri, float* __restrict__ aabb, int32_t* __restrict__ parent,
                             int32_t* __restrict__ flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nt; j += (int64_t)gridDim.x * blockDim.x) {
        const int t = (int)(keys[j] & 0xffffffffu);
        leaf_tri[j] = t;
        const float* v = tris + 9 * (int64_t)t;
        float* bb = aabb + 6 * (nt - 1 + j);
        for (int a = 0; a < 3; ++a) {
            bb[a] = fminf(v[a], fminf(v[3 + a], v[6 + a]));
            bb[3 + a] = fmaxf(v[a], fmaxf(v[3 + a], v[6 + a]));
        }
        if (j < nt - 1) flags[j] = 0;
    }
    if (nt == 1 && blockIdx.x == 0 && threadIdx.x == 0) parent[0] = -1;
}

// bottom-up boxes: the second thread to reach a node combines its children
__global__ void k_bvh_up(int64_t nt, const int32_t* __restrict__ child, const int32_t* __restrict__ parent,
                         float* aabb, int32_t* flags) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < nt; j += (int64_t)gridDim.x * blockDim.x) {
        int64_t node = nt - 1 + j;
        for (int guard = 0; guard < 128 && node > 0; ++guard) {
            const int p = parent[node];
            __threadfence();
            if (atomicAdd(&flags[p], 1) == 0) break;
            __threadfence();
            const int a = child[2 * p], b = child[2 * p + 1];
            for (int q = 0; q < 3; ++q) {
                aabb[6 * p + q] = fminf(*(volatile float*)&aabb[6 * a + q], *(volatile float*)&aabb[6 * b + q]);
                aabb[6 * p + 3 + q] =
                    fmaxf(*(volatile float*)&aabb[6 * a + 3 + q], *(volatile float*)&aabb[6 * b + 3 + q]);
            }
            node = p;
        }
    }
}

}  // namespace

// ------------------------------------------------------------------ tree
extern "C" lt_status lt_build_tree(lt_ctx* ctx, const float* vpls, int64_t n, lt_tree* tree) {
    if (!ctx || !vpls || n < 1 || n > (1 << 28) || !tree_ok(tree) || tree->n != n || ((uintptr_t)vpls & 15))
        return lt_fail(ctx, LT_EINVAL, "lt_build_tree: bad arguments");
    cudaSetDevice(ctx->device);
    const int64_t npad = next_pow2(n);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_SORT, (size_t)npad * 8 + (size_t)n * 4 + 1024, &st);
    if (!p) return st;
    unsigned long long* keys = (unsigned long long*)p;
    int32_t* flags = (int32_t*)(p + npad * 8);
    float* box = (float*)lt_scratch(ctx, SCR_MISC, 64, &st);
    if (!box) return st;
    const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 16 * (int64_t)ctx->num_sms);
    k_bbox<<<1, 1024, 0, ctx->stream>>>((const float4*)vpls, n, box);
    LT_LAUNCH_CHECK(ctx, "k_bbox");
    k_vpl_keys<<<blocks, 256, 0, ctx->stream>>>((const float4*)vpls, n, box, npad, keys);
    LT_LAUNCH_CHECK(ctx, "k_vpl_keys");
    if ((st = bitonic_sort(ctx, keys, npad)) != LT_OK) return st;
    k_karras<<<blocks, 256, 0, ctx->stream>>>(keys, n, *tree);
    LT_LAUNCH_CHECK(ctx, "k_karras");
    k_tree_leaves<<<blocks, 256, 0, ctx->stream>>>(keys, (const float4*)vpls, n, *tree, flags);
    LT_LAUNCH_CHECK(ctx, "k_tree_leaves");
    if (n > 1) {
        LT_CUDA(ctx, cudaMemsetAsync(tree->parent, 0xff, sizeof(int32_t), ctx->stream));  // root has no parent
        k_tree_up<<<blocks, 256, 0, ctx->stream>>>(n, *tree, flags);
        LT_LAUNCH_CHECK(ctx, "k_tree_up");
    }
    return LT_OK;
}

// ------------------------------------------------------------------ global cut
namespace {
// est[nr] and err[C] of the cut (device arrays); the refinement's per-round errors.
lt_status cut_errors(lt_ctx* ctx, const lt_tree* tree, const float* pts, int64_t m, const float* vpls,
                     const int32_t* rows, int64_t nr, const int32_t* cut, int C, float d_min, float* est, float* err) {
    const int blocks = std::max(1, 8 * ctx->num_sms);
    k_cut_estimate<<<blocks, 256, 0, ctx->stream>>>((const float4*)pts, m, (const float4*)vpls, tree->n, *tree, rows,
                                                   nr, cut, C, d_min * d_min, est);
    LT_LAUNCH_CHECK(ctx, "k_cut_estimate");
    k_cut_error<<<blocks, 256, 0, ctx->stream>>>((const float4*)pts, m, *tree, rows, nr, cut, C, est, d_min * d_min,
                                                err);
    LT_LAUNCH_CHECK(ctx, "k_cut_error");
    return LT_OK;
}
}  // namespace

extern "C" lt_status lt_cut_errors(lt_ctx* ctx, const lt_tree* tree, const float* pts, int64_t m, const float* vpls,
                                   const int32_t* rows, int64_t nr, const int32_t* cut, int32_t C, float d_min,
                                   float* err) {
    if (!ctx || !tree_ok(tree) || !pts || !vpls || !rows || nr < 1 || m < 1 || !cut || C < 1 || !err)
        return lt_fail(ctx, LT_EINVAL, "lt_cut_errors: bad arguments");
    cudaSetDevice(ctx->device);
    lt_status st;
    float* est = (float*)lt_scratch(ctx, SCR_CUT, (size_t)nr * 4 + 256, &st);
    if (!est) return st;
    return cut_errors(ctx, tree, pts, m, vpls, rows, nr, cut, C, d_min, est, err);
}

extern "C" lt_status lt_build_global_cut(lt_ctx* ctx, const lt_tree* tree, const float* pts, int64_t m,
                                         const float* vpls, const int32_t* rows, int64_t nr, float eps,
                                         int32_t max_cut, float growth, float d_min, int32_t* cut,
                                         int32_t* cut_size_host) {
    if (!ctx || !tree_ok(tree) || !pts || !vpls || !rows || nr < 1 || m < 1 || max_cut < 1 || !cut ||
        !cut_size_host || !(growth > 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_build_global_cut: bad arguments");
    cudaSetDevice(ctx->device);
    const int64_t n = tree->n, NN = 2 * n - 1;
    std::vector<int32_t> child(2 * NN), range(2 * NN);
    LT_CUDA(ctx, cudaMemcpyAsync(child.data(), tree->child, child.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(range.data(), tree->range, range.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_CUT, (size_t)nr * 4 + (size_t)max_cut * 8 + 1024, &st);
    if (!p) return st;
    float* est = (float*)p;
    float* err = (float*)(p + ((nr * 4 + 255) & ~255LL));
    std::vector<int32_t> cur = {0};
    std::vector<float> herr;
    for (int round = 0; round < 4096; ++round) {
        const int C = (int)cur.size();
        LT_CUDA(ctx, cudaMemcpyAsync(cut, cur.data(), C * 4, cudaMemcpyHostToDevice, ctx->stream));
        st = cut_errors(ctx, tree, pts, m, vpls, rows, nr, cut, C, d_min, est, err);
        if (st != LT_OK) return st;
        herr.resize(C);
        LT_CUDA(ctx, cudaMemcpyAsync(herr.data(), err, C * 4, cudaMemcpyDeviceToHost, ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::vector<int> cand;
        for (int i = 0; i < C; ++i)
            if (cur[i] < n - 1 && herr[i] > eps) cand.push_back(i);
        if (cand.empty()) break;
        int64_t room = (int64_t)max_cut - C;
        room = std::min<int64_t>(room, std::max<int64_t>(1, (int64_t)(growth * C)));
        bool stop = false;
        if ((int64_t)cand.size() > room) {
            std::stable_sort(cand.begin(), cand.end(), [&](int x, int y) {
                if (herr[x] != herr[y]) return herr[x] > herr[y];
                return cur[x] < cur[y];
            });
            cand.resize((size_t)std::max<int64_t>(0, room));
            stop = C + (int64_t)cand.size() >= max_cut;
        }
        if (cand.empty()) break;
        std::vector<char> split(C, 0);
        for (int i : cand) split[i] = 1;
        std::vector<int32_t> nxt;
        nxt.reserve(C + cand.size());
        for (int i = 0; i < C; ++i) {
            if (split[i]) {
                nxt.push_back(child[2 * cur[i]]);
                nxt.push_back(child[2 * cur[i] + 1]);
            } else {
                nxt.push_back(cur[i]);
            }
        }
        cur.swap(nxt);
        if (stop) break;
    }
    std::stable_sort(cur.begin(), cur.end(), [&](int a, int b) { return range[2 * a] < range[2 * b]; });
    LT_CUDA(ctx, cudaMemcpyAsync(cut, cur.data(), cur.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *cut_size_host = (int32_t)cur.size();
    return LT_OK;
}

// ------------------------------------------------------------------ forest of the cut
extern "C" lt_status lt_cut_forest(lt_ctx* ctx, const lt_tree* tree, const int32_t* cut, int32_t C, int32_t* forest,
                                   int32_t* level_off, int32_t max_levels, int32_t* level_nodes,
                                   int32_t* height_host) {
    if (!ctx || !tree_ok(tree) || !cut || C < 1 || !forest || !level_off || max_levels < 1 || !height_host ||
        (C > 1 && !level_nodes))
        return lt_fail(ctx, LT_EINVAL, "lt_cut_forest: bad arguments");
    cudaSetDevice(ctx->device);
    const int64_t n = tree->n, NN = 2 * n - 1;
    std::vector<int32_t> child(2 * NN), parent(NN), hc(C);
    LT_CUDA(ctx, cudaMemcpyAsync(child.data(), tree->child, child.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(parent.data(), tree->parent, parent.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(hc.data(), cut, C * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    std::vector<int32_t> local(NN, -1);
    for (int c = 0; c < C; ++c) {
        if (hc[c] < 0 || hc[c] >= NN || local[hc[c]] >= 0)
            return lt_fail(ctx, LT_EINVAL, "lt_cut_forest: cut nodes out of range or repeated");
        local[hc[c]] = c;
    }
    std::vector<char> anc(NN, 0);
    for (int c = 0; c < C; ++c)
        for (int x = parent[hc[c]]; x >= 0 && !anc[x]; x = parent[x]) anc[x] = 1;
    std::vector<int32_t> inner;
    for (int64_t x = 0; x < NN; ++x)
        if (anc[x]) inner.push_back((int32_t)x);
    if ((int64_t)inner.size() != C - 1) return lt_fail(ctx, LT_EINVAL, "lt_cut_forest: the cut is not a partition");
    for (size_t i = 0; i < inner.size(); ++i) local[inner[i]] = C + (int32_t)i;
    const int NF = 2 * C - 1;
    std::vector<int32_t> fo((size_t)NF * 8, 0);
    for (int c = 0; c < C; ++c) {
        fo[8 * c + 0] = hc[c];
        fo[8 * c + 1] = -1;
        fo[8 * c + 2] = -1;
        fo[8 * c + 3] = -1;
        fo[8 * c + 4] = c;
        fo[8 * c + 5] = c;
        fo[8 * c + 6] = 0;
    }
    for (int x = C; x < NF; ++x) fo[8 * x + 3] = -1;
    for (size_t i = 0; i < inner.size(); ++i) {
        const int x = C + (int)i, t = inner[i];
        const int a = local[child[2 * t]], b = local[child[2 * t + 1]];
        if (a < 0 || b < 0) return lt_fail(ctx, LT_EINVAL, "lt_cut_forest: the cut is not a partition");
        fo[8 * x + 0] = t;
        fo[8 * x + 1] = a;
        fo[8 * x + 2] = b;
        fo[8 * a + 3] = x;  // a parent may come before or after its children in tree-id order
        fo[8 * b + 3] = x;
    }
    // leaf ranges and heights, children before parents (ancestors have smaller tree ids
    // in a radix tree only along a path, so iterate to a fixed point by height order)
    std::vector<int> order(NF);
    std::iota(order.begin(), order.end(), 0);
    std::vector<int> depth(NF, 0);
    for (int x = 0; x < NF; ++x) {
        int d = 0;
        for (int y = fo[8 * x + 3]; y >= 0; y = fo[8 * y + 3]) ++d;
        depth[x] = d;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return depth[a] > depth[b]; });
    int H = 0;
    for (int x : order) {
        if (x < C) continue;
        const int a = fo[8 * x + 1], b = fo[8 * x + 2];
        fo[8 * x + 4] = std::min(fo[8 * a + 4], fo[8 * b + 4]);
        fo[8 * x + 5] = std::max(fo[8 * a + 5], fo[8 * b + 5]);
        fo[8 * x + 6] = 1 + std::max(fo[8 * a + 6], fo[8 * b + 6]);
        H = std::max(H, fo[8 * x + 6]);
    }
    if (H + 2 > max_levels + 2 || H > max_levels) return lt_fail(ctx, LT_EINVAL, "lt_cut_forest: max_levels too small");
    std::vector<int32_t> loff(H + 2, 0), lnodes;
    for (int h = 1; h <= H; ++h) {
        loff[h] = (int32_t)lnodes.size();
        for (int x = C; x < NF; ++x)
            if (fo[8 * x + 6] == h) lnodes.push_back(x);
    }
    loff[0] = 0;
    loff[H + 1] = (int32_t)lnodes.size();
    LT_CUDA(ctx, cudaMemcpyAsync(forest, fo.data(), fo.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(level_off, loff.data(), loff.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    if (!lnodes.empty())
        LT_CUDA(ctx, cudaMemcpyAsync(level_nodes, lnodes.data(), lnodes.size() * 4, cudaMemcpyHostToDevice,
                                     ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *height_host = H;
    return LT_OK;
}

// ------------------------------------------------------------------ slicing
extern "C" lt_status lt_make_slices(lt_ctx* ctx, const float* pts, int64_t m, int32_t S, int32_t iters,
                                    float normal_weight, int32_t* row_perm, int32_t* slice_off) {
    if (!ctx || !pts || m < 1 || S < 1 || S > 4096 || S > m || iters < 0 || !row_perm || !slice_off ||
        ((uintptr_t)pts & 15))
        return lt_fail(ctx, LT_EINVAL, "lt_make_slices: bad arguments");
    cudaSetDevice(ctx->device);
    const int64_t npad = next_pow2(m);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_SORT,
                                (size_t)npad * 8 + (size_t)m * 4 + (size_t)S * 7 * 8 + (size_t)S * 6 * 4 + S * 4 + 4096,
                                &st);
    if (!p) return st;
    unsigned long long* keys = (unsigned long long*)p;
    int32_t* lab = (int32_t*)(p + npad * 8);
    double* sums = (double*)(p + npad * 8 + ((m * 4 + 255) & ~255LL));
    float* cen = (float*)((char*)sums + ((S * 7 * 8 + 255) & ~255LL));
    int32_t* counts = (int32_t*)((char*)cen + ((S * 6 * 4 + 255) & ~255LL));
    float* box = (float*)lt_scratch(ctx, SCR_MISC, 64, &st);
    if (!box) return st;
    const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 16 * (int64_t)ctx->num_sms);
    k_bbox<<<1, 1024, 0, ctx->stream>>>((const float4*)pts, m, box);
    LT_LAUNCH_CHECK(ctx, "k_bbox");
    k_point_keys<<<blocks, 256, 0, ctx->stream>>>((const float4*)pts, m, box, npad, keys);
    LT_LAUNCH_CHECK(ctx, "k_point_keys");
    if ((st = bitonic_sort(ctx, keys, npad)) != LT_OK) return st;
    k_kmeans_seed<<<(S + 255) / 256, 256, 0, ctx->stream>>>((const float4*)pts, m, keys, S, normal_weight, cen);
    LT_LAUNCH_CHECK(ctx, "k_kmeans_seed");
    const size_t shm = (size_t)S * 6 * 4;
    if (shm > 16 * 1024)
        LT_CUDA(ctx, cudaFuncSetAttribute(k_kmeans_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const int ablocks = (int)std::min<int64_t>((m + 255) / 256, 4 * (int64_t)ctx->num_sms);
    for (int it = 0; it < iters; ++it) {
        LT_CUDA(ctx, cudaMemsetAsync(sums, 0, (size_t)S * 7 * 8, ctx->stream));
        k_kmeans_assign<<<ablocks, 256, shm, ctx->stream>>>((const float4*)pts, m, S, normal_weight, cen, lab, sums);
        LT_LAUNCH_CHECK(ctx, "k_kmeans_assign");
        k_kmeans_update<<<(S + 255) / 256, 256, 0, ctx->stream>>>(S, sums, cen);
        LT_LAUNCH_CHECK(ctx, "k_kmeans_update");
    }
    k_kmeans_assign<<<ablocks, 256, shm, ctx->stream>>>((const float4*)pts, m, S, normal_weight, cen, lab, nullptr);
    LT_LAUNCH_CHECK(ctx, "k_kmeans_assign");
    LT_CUDA(ctx, cudaMemsetAsync(counts, 0, (size_t)S * 4, ctx->stream));
    k_label_keys<<<blocks, 256, 0, ctx->stream>>>(lab, m, npad, keys, counts);
    LT_LAUNCH_CHECK(ctx, "k_label_keys");
    if ((st = bitonic_sort(ctx, keys, npad)) != LT_OK) return st;
    k_perm_from_keys<<<blocks, 256, 0, ctx->stream>>>(keys, m, row_perm);
    LT_LAUNCH_CHECK(ctx, "k_perm_from_keys");
    std::vector<int32_t> hc(S), off(S + 1, 0);
    LT_CUDA(ctx, cudaMemcpyAsync(hc.data(), counts, S * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < S; ++s) off[s + 1] = off[s] + hc[s];
    LT_CUDA(ctx, cudaMemcpyAsync(slice_off, off.data(), (S + 1) * 4, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LT_OK;
}

extern "C" lt_status lt_mesh_upload(lt_ctx* ctx, const float* tris, int64_t nt) {
    if (!ctx || nt < 0 || (nt > 0 && !tris) || nt > (1 << 26))
        return lt_fail(ctx, LT_EINVAL, "lt_mesh_upload: bad arguments");
    if (ctx->graphs > 0)
        return lt_fail(ctx, LT_EINVAL, "lt_mesh_upload: live frame graphs reference the current scene");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_mesh_upload: upload the boxes first");
    cudaSetDevice(ctx->device);
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_mesh);
    ctx->d_mesh = nullptr;
    Grid& g = ctx->grid;
    g.nt = 0;
    g.tri = nullptr;
    g.bvh_aabb = nullptr;
    g.bvh_child = nullptr;
    g.bvh_tri = nullptr;
    if (nt == 0) return LT_OK;
    const int64_t nn = 2 * nt - 1;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t b_rec = up((size_t)nt * 48), b_aabb = up((size_t)nn * 24), b_child = up((size_t)nn * 8),
                 b_par = up((size_t)nn * 4), b_range = up((size_t)nn * 8), b_leaf = up((size_t)nt * 4);
    char* m = nullptr;
    LT_CUDA(ctx, cudaMalloc(&m, b_rec + b_aabb + b_child + b_par + b_range + b_leaf));
    ctx->d_mesh = m;
    float4* rec = (float4*)m;
    float* aabb = (float*)(m + b_rec);
    int32_t* child = (int32_t*)(m + b_rec + b_aabb);
    int32_t* parent = (int32_t*)(m + b_rec + b_aabb + b_child);
    int32_t* range = (int32_t*)(m + b_rec + b_aabb + b_child + b_par);
    int32_t* leaf = (int32_t*)(m + b_rec + b_aabb + b_child + b_par + b_range);
    const int64_t npad = next_pow2(nt);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_SORT, (size_t)npad * 8 + (size_t)nt * 4 + (size_t)nt * 16 + 1024, &st);
    if (!p) return st;
    unsigned long long* keys = (unsigned long long*)p;
    int32_t* flags = (int32_t*)(p + npad * 8);
    float4* cen = (float4*)(p + up(npad * 8 + (size_t)nt * 4));
    float* box = (float*)lt_scratch(ctx, SCR_MISC, 64, &st);
    if (!box) return st;
    const int blocks = (int)std::min<int64_t>((npad + 255) / 256, 16 * (int64_t)ctx->num_sms);
    k_tri_prep<<<blocks, 256, 0, ctx->stream>>>(tris, nt, cen, rec);
    LT_LAUNCH_CHECK(ctx, "k_tri_prep");
    k_bbox<<<1, 1024, 0, ctx->stream>>>(cen, nt, box);
    LT_LAUNCH_CHECK(ctx, "k_bbox");
    k_tri_keys<<<blocks, 256, 0, ctx->stream>>>(cen, nt, box, npad, keys);
    LT_LAUNCH_CHECK(ctx, "k_tri_keys");
    if ((st = bitonic_sort(ctx, keys, npad)) != LT_OK) return st;
    lt_tree view{};
    view.n = nt;
    view.child = child;
    view.parent = parent;
    view.range = range;
    k_karras<<<blocks, 256, 0, ctx->stream>>>(keys, nt, view);
    LT_LAUNCH_CHECK(ctx, "k_karras");
    k_bvh_leaves<<<blocks, 256, 0, ctx->stream>>>(keys, tris, nt, leaf, aabb, parent, flags);
    LT_LAUNCH_CHECK(ctx, "k_bvh_leaves");
    if (nt > 1) {
        LT_CUDA(ctx, cudaMemsetAsync(parent, 0xff, sizeof(int32_t), ctx->stream));  // the root
        k_bvh_up<<<blocks, 256, 0, ctx->stream>>>(nt, child, parent, aabb, flags);
        LT_LAUNCH_CHECK(ctx, "k_bvh_up");
    }
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    g.nt = (int)nt;
    g.tri = rec;
    g.bvh_aabb = aabb;
    g.bvh_child = child;
    g.bvh_tri = leaf;
    return LT_OK;
}

extern "C" lt_status lt_mesh_bvh(const lt_ctx* ctx, float* aabb, int32_t* child, int32_t* leaf_tri) {
    if (!ctx || ctx->grid.nt < 1 || !aabb || !child || !leaf_tri) return LT_EINVAL;
    cudaSetDevice(ctx->device);
    const Grid& g = ctx->grid;
    const int64_t nt = g.nt, nn = 2 * nt - 1;
    if (cudaMemcpy(aabb, g.bvh_aabb, (size_t)nn * 24, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(child, g.bvh_child, (size_t)(nt - 1) * 8, cudaMemcpyDeviceToDevice) != cudaSuccess ||
        cudaMemcpy(leaf_tri, g.bvh_tri, (size_t)nt * 4, cudaMemcpyDeviceToDevice) != cudaSuccess)
        return LT_ECUDA;
    return LT_OK;
}
