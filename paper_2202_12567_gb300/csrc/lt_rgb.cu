// Colour: three channels stacked as rows of each slice (one V shared by them).
//
// With the shading of the scalar frame, an entry factors as A(i, c) = rho_p(i) I_c
// K(i, rep(c)): the point's albedo, the node's intensity and a kernel of geometry,
// BRDF shape and visibility that does not depend on colour.  Channel k replaces the
// albedo and the intensity by their channel, so A_k(i, c) = A(i, c) (rho_p,k(i) /
// rho_p(i)) (I_c,k / I_c): the sampled scalar entries give all three channels with
// no further shadow ray.  lt_rgb_setup forms the two ratio tables (per slice-ordered
// row and per tree node) and the stacked row layout; lt_expand_rgb turns every
// sampled entry (i, c) of slice s into entries (3i + k, c) of the stacked slice.
#include <algorithm>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

// pt_ratio[r][k] = albedo_k(pixel row_perm[r]) / rho_p(r) (the frame's scalar albedo)
__global__ void k_rgb_points(lt_frame F, const float4* __restrict__ pt_albedo, const int32_t* __restrict__ perm,
                             float4* __restrict__ pt_ratio) {
    const float4* p0 = reinterpret_cast<const float4*>(F.pts);  // plane 0: position, albedo
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < F.m; r += (int64_t)gridDim.x * blockDim.x) {
        const float a = p0[r].w;
        const float4 c = pt_albedo[perm[r]];
        const float inv = a > 0.f ? 1.f / a : 0.f;
        pt_ratio[r] = make_float4(c.x * inv, c.y * inv, c.z * inv, 0.f);
    }
}

// node_ratio[v][k] = I_v,k / I_v with I_v,k the sum of vpl_power_k over the node's
// leaves (one warp per node)
__global__ void k_rgb_nodes(lt_tree T, const float4* __restrict__ vpl_power, float4* __restrict__ node_ratio) {
    const int lane = threadIdx.x & 31;
    const int64_t nn = 2 * T.n - 1;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = w0; v < nn; v += nw) {
        const int first = T.range[2 * v], last = T.range[2 * v + 1];
        float x = 0.f, y = 0.f, z = 0.f;
        for (int j = first + lane; j <= last; j += 32) {
            const float4 p = vpl_power[T.order[j]];
            x += p.x, y += p.y, z += p.z;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
            z += __shfl_xor_sync(0xffffffffu, z, o);
        }
        if (lane == 0) {
            const float I = T.I[v];
            const float inv = I > 0.f ? 1.f / I : 0.f;
            node_ratio[v] = make_float4(x * inv, y * inv, z * inv, 0.f);
        }
    }
}

// stacked layout: slice_off3 = 3 slice_off, row_perm3[3r + k] = 3 row_perm[r] + k
__global__ void k_rgb_layout(lt_frame F, const int32_t* __restrict__ perm, int32_t* __restrict__ slice_off3,
                             int32_t* __restrict__ perm3) {
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nt = (int64_t)gridDim.x * blockDim.x;
    for (int64_t s = t0; s <= F.S; s += nt) slice_off3[s] = 3 * F.slice_off[s];
    for (int64_t r = t0; r < F.m; r += nt) {
        const int32_t p = perm[r];
        perm3[3 * r] = 3 * p;
        perm3[3 * r + 1] = 3 * p + 1;
        perm3[3 * r + 2] = 3 * p + 2;
    }
}

// entry e of slice s -> entries 3e .. 3e + 2 of the stacked slice
__global__ void k_expand_rgb(lt_frame F, lt_samples smp, const float4* __restrict__ pt_ratio,
                             const float4* __restrict__ node_ratio, lt_samples out, int32_t* status) {
    const int s = blockIdx.y;
    int ne = smp.cnt[s];
    if (3 * (int64_t)ne > out.off[s + 1] - out.off[s]) {  // the stacked slice's capacity
        if (blockIdx.x == 0 && threadIdx.x == 0) latch(status, LT_ELIMIT);
        ne = (int)((out.off[s + 1] - out.off[s]) / 3);
    }
    const int row0 = F.slice_off[s];
    const uint32_t* key = smp.key + smp.off[s];
    const float* val = smp.val + smp.off[s];
    uint32_t* key3 = out.key + out.off[s];
    float* val3 = out.val + out.off[s];
    const int32_t* cn = smp.col_node + (int64_t)s * F.C;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out.cnt[s] = 3 * ne;
        out.n1[s] = 3 * smp.n1[s];
        out.ncol[s] = smp.ncol[s];
    }
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
        const uint32_t kk = key[e];
        const uint32_t i = kk >> 16, c = kk & 0xffffu;
        const float v = val[e];
        const float4 pr = pt_ratio[row0 + i];
        const float4 nr = node_ratio[cn[c]];
        const uint32_t base = (3u * i) << 16 | c;
        key3[3 * e] = base;
        key3[3 * e + 1] = base + (1u << 16);
        key3[3 * e + 2] = base + (2u << 16);
        val3[3 * e] = v * pr.x * nr.x;
        val3[3 * e + 1] = v * pr.y * nr.y;
        val3[3 * e + 2] = v * pr.z * nr.z;
    }
}

}  // namespace

extern "C" lt_status lt_rgb_setup(lt_ctx* ctx, const lt_frame* f, const float* pt_albedo, const float* vpl_power,
                                  const int32_t* row_perm, lt_rgb* out) {
    if (!ctx || !f || !f->pts || f->m < 1 || f->S < 1 || !f->slice_off || !f->tree.range || !f->tree.order ||
        !f->tree.I || f->tree.n < 1 || !pt_albedo || !vpl_power || !row_perm || !out || !out->pt_ratio ||
        !out->node_ratio || !out->slice_off3 || !out->row_perm3 || 3 * (int64_t)f->max_rows > 65535)
        return lt_fail(ctx, LT_EINVAL, "lt_rgb_setup: bad arguments");
    cudaSetDevice(ctx->device);
    const int nsm = ctx->num_sms;
    k_rgb_points<<<4 * nsm, 256, 0, ctx->stream>>>(*f, reinterpret_cast<const float4*>(pt_albedo), row_perm,
                                                   reinterpret_cast<float4*>(out->pt_ratio));
    LT_LAUNCH_CHECK(ctx, "k_rgb_points");
    k_rgb_nodes<<<4 * nsm, 256, 0, ctx->stream>>>(f->tree, reinterpret_cast<const float4*>(vpl_power),
                                                  reinterpret_cast<float4*>(out->node_ratio));
    LT_LAUNCH_CHECK(ctx, "k_rgb_nodes");
    k_rgb_layout<<<4 * nsm, 256, 0, ctx->stream>>>(*f, row_perm, out->slice_off3, out->row_perm3);
    LT_LAUNCH_CHECK(ctx, "k_rgb_layout");
    return LT_OK;
}

extern "C" lt_status lt_expand_rgb(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const lt_rgb* c,
                                   lt_samples* smp3) {
    if (!ctx || !f || f->S < 1 || !f->slice_off || !smp || !smp->key || !smp->val || !smp->off || !smp->cnt ||
        !smp->n1 || !smp->ncol || !smp->col_node || !c || !c->pt_ratio || !c->node_ratio || !smp3 || !smp3->key ||
        !smp3->val || !smp3->off || !smp3->cnt || !smp3->n1 || !smp3->ncol || 3 * (int64_t)f->max_rows > 65535)
        return lt_fail(ctx, LT_EINVAL, "lt_expand_rgb: bad arguments");
    cudaSetDevice(ctx->device);
    const int per = std::max(1, 2 * ctx->num_sms / f->S);
    k_expand_rgb<<<dim3(per, f->S), 256, 0, ctx->stream>>>(*f, *smp, reinterpret_cast<const float4*>(c->pt_ratio),
                                                           reinterpret_cast<const float4*>(c->node_ratio), *smp3,
                                                           ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_expand_rgb");
    return LT_OK;
}
