// Internal device code shared by the translation units of liblt (sm_103a).
//
// Philox4x32-10 (Salmon et al., SC'11), the uniform-grid shadow-ray test, the
// entry model A(i, j) of the lighting matrix (Sec. 3; the shading formula is the
// reading documented in include/lt.h), block-wide scans and the context struct.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/lt.h"

namespace ltk {

constexpr float kRayOffset = 1e-4f;
constexpr float kTMin = 1e-4f;
constexpr float kTMax = 1.0f - 1e-4f;
constexpr float kInvPi = 0.318309886183790672f;
constexpr uint32_t kTagPass1 = 1, kTagPass2 = 2, kTagAlsInit = 3, kTagAdmInit = 6;

// The seed of a frame: passed by value, or read from a device word so that one
// captured graph replays every seed.
struct SeedRef {
    uint64_t value;
    const uint64_t* dev;
    __device__ __forceinline__ uint64_t get() const { return dev ? *dev : value; }
};

// ----------------------------------------------------------------- Philox4x32-10
struct U4 {
    uint32_t x, y, z, w;
};

__host__ __device__ inline U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t seed) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
#else
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
#endif
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        if (r < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
    return {c0, c1, c2, c3};
}

// The slice index a random counter uses: the slice's index in the whole frame.
__device__ __forceinline__ uint32_t slice_key(const int32_t* slice_id, int s) {
    return slice_id ? (uint32_t)slice_id[s] : (uint32_t)s;
}

// floor(w * size / 2^32)
__host__ __device__ inline uint32_t uniform_index(uint32_t w, uint32_t size) {
    return (uint32_t)(((uint64_t)w * (uint64_t)size) >> 32);
}

// ----------------------------------------------------------------- small vector helpers
__device__ __forceinline__ float3 f3(float4 a) { return make_float3(a.x, a.y, a.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return make_float3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return make_float3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// ----------------------------------------------------------------- occluder grid
// Uniform grid of R^3 cells over the boxes' bounds; cell c lists the boxes that
// overlap it (expanded by a small margin so that rounding at cell faces cannot hide
// a box from a ray that the exact test would block).
struct Grid {
    const float* box;        // [nb][6]
    const int32_t* cell_off; // [R^3 + 1]
    const int32_t* cell_box; // [cell_off[R^3]]
    int nb;
    int R;
    int nlist;               // entries of cell_box
    float lo[3];
    float cell[3];
    float inv_cell[3];
    // triangle occluders (lt_mesh_upload): a linear BVH over nt triangles, internal
    // nodes 0..nt-2 (root 0), leaf j = node nt-1+j holding triangle bvh_tri[j]
    const float4* tri;       // [nt][3] v0, e1 = v1 - v0, e2 = v2 - v0 (w unused)
    const float* bvh_aabb;   // [2nt-1][6] lo xyz, hi xyz
    const int32_t* bvh_child;// [nt-1][2]
    const int32_t* bvh_tri;  // [nt]
    int nt;
};

// Closed-box slab test of o + t D over t in [kTMin, kTMax].
__device__ __forceinline__ bool slab_hit(const float* __restrict__ b, float3 o, float3 inv, int par) {
    float tn = kTMin, tf = kTMax;
    const float2 b01 = reinterpret_cast<const float2*>(b)[0];
    const float2 b23 = reinterpret_cast<const float2*>(b)[1];
    const float2 b45 = reinterpret_cast<const float2*>(b)[2];
    const float lo0 = b01.x, lo1 = b01.y, lo2 = b23.x, hi0 = b23.y, hi1 = b45.x, hi2 = b45.y;
    if (par & 1) {
        if (o.x < lo0 || o.x > hi0) return false;
    } else {
        const float ta = (lo0 - o.x) * inv.x, tb = (hi0 - o.x) * inv.x;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    if (par & 2) {
        if (o.y < lo1 || o.y > hi1) return false;
    } else {
        const float ta = (lo1 - o.y) * inv.y, tb = (hi1 - o.y) * inv.y;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    if (par & 4) {
        if (o.z < lo2 || o.z > hi2) return false;
    } else {
        const float ta = (lo2 - o.z) * inv.z, tb = (hi2 - o.z) * inv.z;
        tn = fmaxf(tn, fminf(ta, tb));
        tf = fminf(tf, fmaxf(ta, tb));
    }
    return tn <= tf;
}

// Work done by the traversal (instrumentation of the ALU roofline).
struct WorkCount {
    int cells = 0;
    int boxes = 0;
};

// Any-hit test of the segment o -> e (t in (kTMin, kTMax)) against the boxes by a 3-D
// DDA walk.  The walk is bounded by the number of cells a straight segment can cross.
template <bool COUNT = false>
__device__ inline bool grid_blocked(const Grid& g, float3 o, float3 e, WorkCount* wc = nullptr) {
    const float3 D = e - o;
    const int par = (D.x == 0.f ? 1 : 0) | (D.y == 0.f ? 2 : 0) | (D.z == 0.f ? 4 : 0);
    const float3 inv = make_float3((par & 1) ? 0.f : 1.f / D.x, (par & 2) ? 0.f : 1.f / D.y,
                                   (par & 4) ? 0.f : 1.f / D.z);
    const int R = g.R;
    float t0 = kTMin, t1 = kTMax;
    const float oa[3] = {o.x, o.y, o.z};
    const float ia[3] = {inv.x, inv.y, inv.z};
    const float da[3] = {D.x, D.y, D.z};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = g.lo[a], hi = g.lo[a] + R * g.cell[a];
        if (par & (1 << a)) {
            if (oa[a] < lo || oa[a] > hi) return false;
        } else {
            const float ta = (lo - oa[a]) * ia[a], tb = (hi - oa[a]) * ia[a];
            t0 = fmaxf(t0, fminf(ta, tb));
            t1 = fminf(t1, fmaxf(ta, tb));
        }
    }
    if (t0 > t1) return false;
    int c[3], st[3];
    float tn[3], td[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float x = oa[a] + t0 * da[a];
        int ci = (int)floorf((x - g.lo[a]) * g.inv_cell[a]);
        ci = ci < 0 ? 0 : (ci >= R ? R - 1 : ci);
        c[a] = ci;
        if (par & (1 << a)) {
            st[a] = 0;
            tn[a] = 3.0e38f;
            td[a] = 3.0e38f;
        } else {
            st[a] = da[a] > 0.f ? 1 : -1;
            const float bnd = g.lo[a] + (float)(ci + (st[a] > 0 ? 1 : 0)) * g.cell[a];
            tn[a] = (bnd - oa[a]) * ia[a];
            td[a] = g.cell[a] * fabsf(ia[a]);
        }
    }
    const int max_steps = 3 * R + 3;
    for (int it = 0; it < max_steps; ++it) {
        const int cell = (c[2] * R + c[1]) * R + c[0];
        const int b0 = g.cell_off[cell], b1 = g.cell_off[cell + 1];
        if (COUNT) ++wc->cells;
        for (int k = b0; k < b1; ++k) {
            const int bi = g.cell_box[k];
            if (COUNT) ++wc->boxes;
            if (slab_hit(g.box + 6 * bi, o, inv, par)) return true;
        }
        int a = 0;
        if (tn[1] < tn[a]) a = 1;
        if (tn[2] < tn[a]) a = 2;
        if (tn[a] > t1) break;
        c[a] += st[a];
        if (c[a] < 0 || c[a] >= R) break;
        tn[a] += td[a];
    }
    return false;
}

// Closed triangle (v0, v0 + e1, v0 + e2) against o + t D, t in (kTMin, kTMax)
// (Moller-Trumbore; a segment in the triangle's plane does not hit).
__device__ __forceinline__ bool tri_hit(const float4* __restrict__ t3, float3 o, float3 D) {
    const float4 a = t3[0], b = t3[1], c = t3[2];
    const float3 v0 = make_float3(a.x, a.y, a.z), e1 = make_float3(b.x, b.y, b.z), e2 = make_float3(c.x, c.y, c.z);
    const float3 p = make_float3(D.y * e2.z - D.z * e2.y, D.z * e2.x - D.x * e2.z, D.x * e2.y - D.y * e2.x);
    const float det = dot3(e1, p);
    if (det == 0.f) return false;
    const float inv = 1.f / det;
    const float3 sv = o - v0;
    const float u = dot3(sv, p) * inv;
    if (u < 0.f || u > 1.f) return false;
    const float3 q = make_float3(sv.y * e1.z - sv.z * e1.y, sv.z * e1.x - sv.x * e1.z, sv.x * e1.y - sv.y * e1.x);
    const float v = dot3(D, q) * inv;
    if (v < 0.f || u + v > 1.f) return false;
    const float t = dot3(e2, q) * inv;
    return t > kTMin && t < kTMax;
}

// Any-hit test of the segment against the triangles: depth-first walk of the BVH
// with an explicit stack.  The tree's keys are 64-bit and distinct, so it is at
// most 64 levels deep and the stack (one entry pushed per level) cannot overflow;
// the walk visits each node at most once, which bounds the loop.
__device__ inline bool bvh_blocked(const Grid& g, float3 o, float3 e) {
    const float3 D = e - o;
    const int par = (D.x == 0.f ? 1 : 0) | (D.y == 0.f ? 2 : 0) | (D.z == 0.f ? 4 : 0);
    const float3 inv = make_float3((par & 1) ? 0.f : 1.f / D.x, (par & 2) ? 0.f : 1.f / D.y,
                                   (par & 4) ? 0.f : 1.f / D.z);
    const int nt = g.nt, nl = nt - 1;  // leaves start at node nl
    if (!slab_hit(g.bvh_aabb, o, inv, par)) return false;
    int stack[64];
    int sp = 0;
    int node = 0;
    for (int it = 0; it < 2 * nt; ++it) {
        if (node >= nl) {  // leaf
            if (tri_hit(g.tri + 3 * g.bvh_tri[node - nl], o, D)) return true;
            if (sp == 0) break;
            node = stack[--sp];
            continue;
        }
        const int a = g.bvh_child[2 * node], b = g.bvh_child[2 * node + 1];
        const bool ha = slab_hit(g.bvh_aabb + 6 * a, o, inv, par);
        const bool hb = slab_hit(g.bvh_aabb + 6 * b, o, inv, par);
        if (ha && hb) {
            if (sp < 64) stack[sp++] = b;
            node = a;
        } else if (ha || hb) {
            node = ha ? a : b;
        } else {
            if (sp == 0) break;
            node = stack[--sp];
        }
    }
    return false;
}

// Any-hit test of the segment o -> e against every occluder (boxes, then triangles).
template <bool COUNT = false>
__device__ inline bool seg_blocked(const Grid& g, float3 o, float3 e, WorkCount* wc = nullptr) {
    if (g.nb > 0 && grid_blocked<COUNT>(g, o, e, wc)) return true;
    return g.nt > 0 && bvh_blocked(g, o, e);
}

// ----------------------------------------------------------------- entry model
// Float pairs (hi, lo) holding a value as an unevaluated sum, from the error-free
// transformations of Knuth (two-sum: the exact rounding error of a + b) and Dekker
// (two-product: the exact rounding error of a b, here by one fma).
struct F2 {
    float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ F2 two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// a . b of float3 as a float pair (error of order 2^-46 |a||b|)
__device__ __forceinline__ F2 dot3_f2(float3 a, float3 b) {
    const F2 p0 = two_prod(a.x, b.x), p1 = two_prod(a.y, b.y), p2 = two_prod(a.z, b.z);
    const F2 s1 = two_sum(p0.hi, p1.hi);
    const F2 s2 = two_sum(s1.hi, p2.hi);
    return {s2.hi, __fadd_rn(__fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, s1.lo)), s2.lo)};
}

// Phong lobe: cos a = R(wi) . wo with R(wi) = 2 (n.wi) n - wi the mirrored incident
// direction, so cos a - 1 = 2 (n.wi)(n.wo) - wi.wo - 1.  The lobe raises cos a to the
// exponent e (up to 100), which multiplies the error of cos a - 1 by e, and near the
// peak the terms cancel: they are carried as float pairs, so the cancellation is
// exact and cos a - 1 is as accurate as a float can hold it.  The power is taken as
// exp(e log1p(cos a - 1)).
__device__ __forceinline__ float brdf(float alb, float gloss, float3 n, float3 wi, float3 wo) {
    if (!(gloss > 0.f)) return alb * kInvPi;
    const F2 ni = dot3_f2(n, wi), no = dot3_f2(n, wo), io = dot3_f2(wi, wo);
    const F2 pp = two_prod(ni.hi, no.hi);  // (ni no) as a pair
    const float plo = __fadd_rn(pp.lo, __fadd_rn(__fmul_rn(ni.hi, no.lo), __fmul_rn(ni.lo, no.hi)));
    const F2 d1 = two_sum(__fmul_rn(2.f, pp.hi), -io.hi);                 // 2 ni no - io
    const float l1 = __fadd_rn(d1.lo, __fsub_rn(__fmul_rn(2.f, plo), io.lo));
    const F2 d2 = two_sum(d1.hi, -1.f);                                   // - 1
    const float cm1 = __fadd_rn(d2.hi, __fadd_rn(d2.lo, l1));
    const float lobe = cm1 > -1.f ? expf(gloss * log1pf(cm1)) : 0.f;
    return 0.5f * alb * kInvPi + 0.5f * alb * (gloss + 2.f) * (0.5f * kInvPi) * lobe;
}

struct PointRec {
    float4 a, b, c;   // [p albedo] [n gloss] [wo 0]
};

__device__ __forceinline__ PointRec load_rec(const float4* __restrict__ planes, int64_t count, int64_t i) {
    PointRec r;
    r.a = __ldg(planes + i);
    r.b = __ldg(planes + count + i);
    r.c = __ldg(planes + 2 * count + i);
    return r;
}

// The same from a generic (global or shared) pointer.
__device__ __forceinline__ PointRec load_rec_any(const float4* planes, int64_t count, int64_t i) {
    PointRec r;
    r.a = planes[i];
    r.b = planes[count + i];
    r.c = planes[2 * count + i];
    return r;
}

// Unoccluded part flux * f_p * f_q * G (0 when a cosine is not positive).
__device__ __forceinline__ float unoccluded(const PointRec& P, const PointRec& L, float dmin2) {
    const float3 d = f3(L.a) - f3(P.a);
    const float dist2 = dot3(d, d);
    const float inv = 1.f / sqrtf(fmaxf(dist2, 1e-30f));
    const float3 w = inv * d;
    const float cp = dot3(f3(P.b), w);
    const float cq = -dot3(f3(L.b), w);
    if (!(cp > 0.f && cq > 0.f)) return 0.f;
    const float G = cp * cq / fmaxf(dist2, dmin2);
    const float fp = brdf(P.a.w, P.b.w, f3(P.b), w, f3(P.c));
    const float fq = brdf(L.a.w, L.b.w, f3(L.b), f3(L.c), make_float3(-w.x, -w.y, -w.z));
    return L.c.w * fp * fq * G;
}

// scale * A(i, j): the unoccluded value, then the shadow ray where it is positive.
template <bool COUNT = false>
__device__ __forceinline__ float entry_value(const PointRec& P, const PointRec& L, float scale, float dmin2,
                                             const Grid& g, WorkCount* wc = nullptr, int* rays = nullptr) {
    float v = unoccluded(P, L, dmin2) * scale;
    if (v > 0.f) {
        const float3 o = f3(P.a) + kRayOffset * f3(P.b);
        const float3 e = f3(L.a) + kRayOffset * f3(L.b);
        if (COUNT) ++*rays;
        if (seg_blocked<COUNT>(g, o, e, wc)) v = 0.f;
    }
    return v;
}

// ----------------------------------------------------------------- block scans
// Exclusive prefix sum over the block (blockDim.x a multiple of 32, <= 1024).
// `warp_sums` must hold 32 ints of shared memory.  Returns the prefix; *total gets
// the block sum.  Every thread of the block must call it.
template <typename T>
__device__ inline T block_exclusive_scan(T x, T* warp_sums, T* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
    }
    if (lane == 31) warp_sums[wid] = v;
    __syncthreads();
    if (wid == 0) {
        T s = lane < nw ? warp_sums[lane] : T(0);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const T y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const T before = (wid > 0 ? warp_sums[wid - 1] : T(0)) + v - x;
    *total = warp_sums[nw - 1];
    __syncthreads();
    return before;
}

template <typename T>
__device__ inline T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ inline float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ inline float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Latch the first error code into the status word.
__device__ inline void latch(int32_t* status, int32_t code) { atomicCAS(status, 0, code); }

// First index in [0, n) with a[idx] >= x (a ascending).
template <typename T>
__device__ __forceinline__ int lower_bound(const T* a, int n, T x) {
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

}  // namespace ltk

// ----------------------------------------------------------------- context
enum ScratchSlot {
    SCR_P1_PLAN = 0,    // per slice per forest node: k, cap, off, cnt, cost, state
    SCR_P1_STORE,       // node storage (rows, v0, v1)
    SCR_BITMAP,         // per slice observed-entry bitmaps (row-major and column-major)
    SCR_OMEGA,          // CSR / CSC of the observed entries
    SCR_ALS,            // per-slice statistics for ALS
    SCR_MISC,           // small reductions
    SCR_SORT,           // sort keys
    SCR_CUT,            // global-cut work arrays
    SCR_GRAM,           // per-line Gram matrices of an ALS half-step
    SCR_PROPOSAL,       // per-slice feature statistics
    SCR_PROPOSAL_T,     // Gram matrices and subspace bases of the targets
    SCR_PROPOSAL_G,     // logits, their gradient and per-CTA weight gradients
    SCR_FRAME_PROP,     // features, groups, logits and weights of a frame's proposal
    SCR_P2_CDF,         // pass-2 integer CDF of every slice
    SCR_ADM,            // second X buffer, U, Lambda, V and Pi of the ADM completion
    SCR_TC_PLAN,        // tensor-core ALS: per-slice prefixes, scales and tile counters
    SCR_TC_IMG,         // tensor-core ALS: W / X images of the source factor rows
    SCR_NSLOTS
};

struct lt_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t* d_status = nullptr;
    int32_t* h_status = nullptr;
    std::string err;
    // occluder grid
    float* d_boxes = nullptr;
    int32_t* d_cell_off = nullptr;
    int32_t* d_cell_box = nullptr;
    void* d_mesh = nullptr;      // triangles and their BVH (lt_mesh_upload), one allocation
    ltk::Grid grid{};
    // scratch
    void* scr[SCR_NSLOTS] = {};
    size_t scr_size[SCR_NSLOTS] = {};
    int num_sms = 0;
    int64_t launches = 0;   // kernels launched through this context
    // Sizes that the frame calls read back from the device.  They depend on the
    // frame's setup (cut, forest, slices, sampling capacity), never on the seed, so a
    // replayed frame (graph capture) takes them from here instead of synchronising.
    struct Plan {
        int64_t p1_total = 0;              // pass-1 row slots of all slices
        std::vector<int32_t> level_off;    // forest level offsets [H + 2]
        int64_t entries = 0;               // sampling capacity off[S]
    } plan;
    bool use_plan = false;                 // set while a frame is captured
    const uint64_t* seed_dev = nullptr;    // device seed word of the graph being captured
    std::vector<void*> retired;            // scratch that live graphs may still reference
    int graphs = 0;                        // graphs alive on this context
    lt_tuning tune{16, 16, 96, 0, 0};         // launch tuning (lt_set_tuning)
    int p1_walk_blocks = 0;                // resident blocks per SM of the persistent pass-1 walk
    int64_t scratch_limit = 0;             // bytes of scratch the context may hold (0: no limit)
};

inline ltk::SeedRef seed_ref(const lt_ctx* ctx, uint64_t seed) { return ltk::SeedRef{seed, ctx->seed_dev}; }

// Helpers implemented in lt_api.cu.
lt_status lt_fail(lt_ctx* ctx, lt_status code, const std::string& msg);
lt_status lt_cuda_check(lt_ctx* ctx, cudaError_t e, const char* what);
void* lt_scratch(lt_ctx* ctx, int slot, size_t bytes, lt_status* st);

#define LT_CUDA(ctx, call)                                           \
    do {                                                             \
        cudaError_t e__ = (call);                                    \
        if (e__ != cudaSuccess) return lt_cuda_check(ctx, e__, #call); \
    } while (0)

#define LT_LAUNCH_CHECK(ctx, name)                                         \
    do {                                                                   \
        ++(ctx)->launches;                                                 \
        cudaError_t e__ = cudaGetLastError();                              \
        if (e__ != cudaSuccess) return lt_cuda_check(ctx, e__, name);      \
    } while (0)
