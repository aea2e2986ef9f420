// The paper's own slicing (Sec. 6 step 2): the 6-D vectors (p, w n) of the shading
// points are split recursively into a binary tree until a node holds at most
// `target` points (slices of about 800 pixels in Sec. 3).  A node of n points splits
// along its feature dimension of largest extent at the median: the floor(n/2) points
// smallest in (feature value, pixel index) go left in their current order, the rest
// go right.  The node sizes depend on m and target only, so the host lays out every
// level; one launch per level splits all of its nodes, one CTA per node: min/max
// reduction of the six features, an eight-pass radix select of the median over the
// 64-bit keys (sortable feature bits << 32 | pixel), and a stable partition by block
// scans.
#include <math.h>

#include <algorithm>
#include <array>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr int kSplitThreads = 1024;

__device__ __forceinline__ void feature6(const float4* __restrict__ pts, int64_t m, int32_t i, float w, float* f) {
    const float4 a = pts[i], b = pts[m + i];
    f[0] = a.x, f[1] = a.y, f[2] = a.z;
    f[3] = __fmul_rn(w, b.x), f[4] = __fmul_rn(w, b.y), f[5] = __fmul_rn(w, b.z);
}

// order-preserving map of a float (with -0 taken as +0) to 32 bits, above it the pixel
__device__ __forceinline__ unsigned long long split_key(const float4* __restrict__ pts, int64_t m, int32_t i,
                                                        float w, int d) {
    const float4 a = pts[i], b = pts[m + i];
    const float v = d == 0 ? a.x : d == 1 ? a.y : d == 2 ? a.z : __fmul_rn(w, d == 3 ? b.x : d == 4 ? b.y : b.z);
    const uint32_t u = __float_as_uint(__fadd_rn(v, 0.f));
    const uint32_t s = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return (unsigned long long)s << 32 | (uint32_t)i;
}

__global__ void __launch_bounds__(kSplitThreads) k_split_level(const float4* __restrict__ pts, int64_t m, float w,
                                                               const int2* __restrict__ nodes,
                                                               const int32_t* __restrict__ in,
                                                               int32_t* __restrict__ out) {
    __shared__ float red[2][6][32];
    __shared__ int dstar;
    __shared__ int32_t hist[256];
    __shared__ unsigned long long sel[2];  // prefix, mask
    __shared__ int32_t krem;
    __shared__ int32_t ws[32];
    const int2 nd = nodes[blockIdx.x];
    const int start = nd.x, n = nd.y;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    // 1. extents of the six features
    float lo[6], hi[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) lo[d] = INFINITY, hi[d] = -INFINITY;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
        float f[6];
        feature6(pts, m, in[start + t], w, f);
#pragma unroll
        for (int d = 0; d < 6; ++d) lo[d] = fminf(lo[d], f[d]), hi[d] = fmaxf(hi[d], f[d]);
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[d] = fminf(lo[d], __shfl_xor_sync(0xffffffffu, lo[d], o));
            hi[d] = fmaxf(hi[d], __shfl_xor_sync(0xffffffffu, hi[d], o));
        }
        if (lane == 0) red[0][d][wid] = lo[d], red[1][d][wid] = hi[d];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int best = 0;
        float be = -INFINITY;
        for (int d = 0; d < 6; ++d) {
            float l = INFINITY, h = -INFINITY;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) l = fminf(l, red[0][d][q]), h = fmaxf(h, red[1][d][q]);
            const float e = __fsub_rn(h, l);
            if (e > be) be = e, best = d;
        }
        dstar = best;
        sel[0] = sel[1] = 0ull;
        krem = n / 2;
    }
    __syncthreads();
    const int d = dstar;
    // 2. radix select of the (n/2)-th smallest key, eight bits at a time
    for (int pass = 7; pass >= 0; --pass) {
        for (int b = threadIdx.x; b < 256; b += blockDim.x) hist[b] = 0;
        __syncthreads();
        const unsigned long long prefix = sel[0], mask = sel[1];
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const unsigned long long key = split_key(pts, m, in[start + t], w, d);
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
    const int half = n / 2;
    // 3. stable partition: keys below the pivot to the left half
    int carry = 0;  // left entries before the chunk
    for (int c0 = 0; c0 < n; c0 += blockDim.x) {
        const int t = c0 + threadIdx.x;
        int32_t i = 0;
        int left = 0;
        if (t < n) {
            i = in[start + t];
            left = split_key(pts, m, i, w, d) < pivot ? 1 : 0;
        }
        int32_t tot;
        const int32_t before = block_exclusive_scan<int32_t>(left, ws, &tot);
        if (t < n) out[start + (left ? carry + before : half + (t - carry - before))] = i;
        carry += tot;
    }
}

__global__ void k_iota(int32_t* p, int64_t m) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (int32_t)i;
}

void split_plan(int64_t start, int64_t n, int64_t target, int depth, std::vector<std::vector<int2>>& levels,
                std::vector<int32_t>& sizes) {
    if (n <= target) {
        sizes.push_back((int32_t)n);
        return;
    }
    if ((int)levels.size() <= depth) levels.resize(depth + 1);
    levels[depth].push_back(make_int2((int)start, (int)n));
    split_plan(start, n / 2, target, depth + 1, levels, sizes);
    split_plan(start + n / 2, n - n / 2, target, depth + 1, levels, sizes);
}

}  // namespace

extern "C" int32_t lt_split_slice_count(int64_t m, int32_t target) {
    if (m < 1 || target < 1 || m > INT32_MAX) return -1;
    std::vector<std::vector<int2>> levels;
    std::vector<int32_t> sizes;
    split_plan(0, m, target, 0, levels, sizes);
    return (int32_t)sizes.size();
}

extern "C" lt_status lt_make_slices_split(lt_ctx* ctx, const float* pts, int64_t m, int32_t target,
                                          float normal_weight, int32_t* row_perm, int32_t* slice_off) {
    if (!ctx || !pts || m < 1 || m > INT32_MAX || target < 1 || !row_perm || !slice_off || !(normal_weight >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_make_slices_split: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<std::vector<int2>> levels;
    std::vector<int32_t> sizes;
    split_plan(0, m, target, 0, levels, sizes);
    std::vector<int32_t> off(sizes.size() + 1, 0);
    for (size_t s = 0; s < sizes.size(); ++s) off[s + 1] = off[s] + sizes[s];
    size_t nn = 0;
    for (auto& l : levels) nn += l.size();
    std::vector<int2> all;
    all.reserve(nn);
    for (auto& l : levels) all.insert(all.end(), l.begin(), l.end());
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_SORT, (size_t)m * 4 + nn * 8 + 512, &st);
    if (!p) return st;
    int32_t* pong = (int32_t*)p;
    int2* dnodes = (int2*)(p + (((size_t)m * 4 + 255) & ~(size_t)255));
    if (nn) LT_CUDA(ctx, cudaMemcpyAsync(dnodes, all.data(), nn * 8, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(slice_off, off.data(), off.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    k_iota<<<4 * ctx->num_sms, 256, 0, ctx->stream>>>(row_perm, m);
    LT_LAUNCH_CHECK(ctx, "k_iota");
    int32_t* in = row_perm;
    int32_t* out = pong;
    size_t at = 0;
    for (auto& l : levels) {
        LT_CUDA(ctx, cudaMemcpyAsync(out, in, (size_t)m * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        k_split_level<<<(unsigned)l.size(), kSplitThreads, 0, ctx->stream>>>(
            reinterpret_cast<const float4*>(pts), m, normal_weight, dnodes + at, in, out);
        LT_LAUNCH_CHECK(ctx, "k_split_level");
        at += l.size();
        std::swap(in, out);
    }
    if (in != row_perm)
        LT_CUDA(ctx, cudaMemcpyAsync(row_perm, in, (size_t)m * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    // the host vectors feed asynchronous copies: wait for them before returning
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return LT_OK;
}

// ------------------------------------------------------------------ slice bounds
// Slices held between min_rows and max_rows rows (the uneven slices of the batched
// workloads): while a slice has fewer than min_rows rows and more than one slice is
// left, the smallest such slice (ties: the lowest index) joins the slice whose
// centroid is nearest to its own (float64 means of the float32 features summed in
// ascending pixel order, squared Euclidean distance, ties to the lowest index); then
// every slice of more than max_rows rows is split by the recursive 6-D median split
// above (k_split_level over its range of row_perm), its parts taking its place.  The
// merges run on the host (a few slices), the splits on the GPU.
extern "C" lt_status lt_bound_slices(lt_ctx* ctx, const float* pts, int64_t m, const int32_t* row_perm_in,
                                     const int32_t* slice_off_in, int32_t S, int32_t min_rows, int32_t max_rows,
                                     float normal_weight, int32_t max_slices, int32_t* row_perm,
                                     int32_t* slice_off, int32_t* S_out) {
    if (!ctx || !pts || m < 1 || m > INT32_MAX || !row_perm_in || !slice_off_in || S < 1 || min_rows < 1 ||
        max_rows < min_rows || max_slices < 1 || !row_perm || !slice_off || !S_out || !(normal_weight >= 0.f) ||
        ((uintptr_t)pts & 15) != 0)
        return lt_fail(ctx, LT_EINVAL, "lt_bound_slices: bad arguments");
    cudaSetDevice(ctx->device);
    std::vector<int32_t> perm((size_t)m), off((size_t)S + 1);
    std::vector<float4> planes((size_t)2 * m);
    LT_CUDA(ctx, cudaMemcpyAsync(perm.data(), row_perm_in, (size_t)m * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(off.data(), slice_off_in, ((size_t)S + 1) * 4, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(planes.data(), pts, (size_t)2 * m * 16, cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (off[0] != 0 || off[S] != m) return lt_fail(ctx, LT_EINVAL, "lt_bound_slices: slice_off does not cover m");
    for (int s = 0; s < S; ++s)
        if (off[s + 1] < off[s]) return lt_fail(ctx, LT_EINVAL, "lt_bound_slices: slice_off decreases");
    auto feat = [&](int32_t i, int d) -> float {
        const float4 a = planes[(size_t)i], b = planes[(size_t)m + i];
        switch (d) {
            case 0: return a.x;
            case 1: return a.y;
            case 2: return a.z;
            case 3: return normal_weight * b.x;
            case 4: return normal_weight * b.y;
            default: return normal_weight * b.z;
        }
    };
    std::vector<std::vector<int32_t>> sl((size_t)S);
    for (int s = 0; s < S; ++s) {
        sl[s].assign(perm.begin() + off[s], perm.begin() + off[s + 1]);
        std::sort(sl[s].begin(), sl[s].end());
        for (int32_t i : sl[s])
            if (i < 0 || i >= m) return lt_fail(ctx, LT_EINVAL, "lt_bound_slices: row index out of range");
    }
    auto centroid = [&](const std::vector<int32_t>& a, double* c) {
        for (int d = 0; d < 6; ++d) {
            double t = 0.0;
            for (int32_t i : a) t += (double)feat(i, d);
            c[d] = a.empty() ? 0.0 : t / (double)a.size();
        }
    };
    std::vector<std::array<double, 6>> cen((size_t)S);
    for (int s = 0; s < S; ++s) centroid(sl[s], cen[s].data());
    while (sl.size() > 1) {
        int small = -1;
        for (int s = 0; s < (int)sl.size(); ++s)
            if ((int64_t)sl[s].size() < min_rows && (small < 0 || sl[s].size() < sl[small].size())) small = s;
        if (small < 0) break;
        int best = -1;
        double bd = INFINITY;
        for (int t = 0; t < (int)sl.size(); ++t) {
            if (t == small) continue;
            double d2 = 0.0;
            for (int d = 0; d < 6; ++d) {
                const double v = cen[small][d] - cen[t][d];
                d2 = d2 + v * v;
            }
            if (d2 < bd) best = t, bd = d2;
        }
        sl[best].insert(sl[best].end(), sl[small].begin(), sl[small].end());
        std::sort(sl[best].begin(), sl[best].end());
        centroid(sl[best], cen[best].data());
        sl.erase(sl.begin() + small);
        cen.erase(cen.begin() + small);
    }
    // merged layout, then the split plan of every slice above max_rows
    std::vector<int32_t> merged;
    merged.reserve((size_t)m);
    std::vector<std::vector<int2>> levels;
    std::vector<int32_t> sizes;
    for (auto& a : sl) {
        const int64_t start = (int64_t)merged.size();
        merged.insert(merged.end(), a.begin(), a.end());
        split_plan(start, (int64_t)a.size(), max_rows, 0, levels, sizes);
    }
    if ((int64_t)sizes.size() > max_slices) return lt_fail(ctx, LT_EINVAL, "lt_bound_slices: max_slices too small");
    std::vector<int32_t> noff(sizes.size() + 1, 0);
    for (size_t s = 0; s < sizes.size(); ++s) noff[s + 1] = noff[s] + sizes[s];
    size_t nn = 0;
    for (auto& l : levels) nn += l.size();
    std::vector<int2> all;
    all.reserve(nn);
    for (auto& l : levels) all.insert(all.end(), l.begin(), l.end());
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_SORT, (size_t)m * 4 + nn * 8 + 512, &st);
    if (!p) return st;
    int32_t* pong = (int32_t*)p;
    int2* dnodes = (int2*)(p + (((size_t)m * 4 + 255) & ~(size_t)255));
    if (nn) LT_CUDA(ctx, cudaMemcpyAsync(dnodes, all.data(), nn * 8, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(row_perm, merged.data(), (size_t)m * 4, cudaMemcpyHostToDevice, ctx->stream));
    LT_CUDA(ctx, cudaMemcpyAsync(slice_off, noff.data(), noff.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    int32_t* in = row_perm;
    int32_t* out = pong;
    size_t at = 0;
    for (auto& l : levels) {
        LT_CUDA(ctx, cudaMemcpyAsync(out, in, (size_t)m * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        k_split_level<<<(unsigned)l.size(), kSplitThreads, 0, ctx->stream>>>(
            reinterpret_cast<const float4*>(pts), m, normal_weight, dnodes + at, in, out);
        LT_LAUNCH_CHECK(ctx, "k_split_level");
        at += l.size();
        std::swap(in, out);
    }
    if (in != row_perm)
        LT_CUDA(ctx, cudaMemcpyAsync(row_perm, in, (size_t)m * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // the host vectors feed asynchronous copies
    *S_out = (int32_t)sizes.size();
    return LT_OK;
}
