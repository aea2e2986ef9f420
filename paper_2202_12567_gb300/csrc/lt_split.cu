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
