// Context, status handling, occluder grid, shadow test, pair evaluation and the
// brute-force column sum (Sec. 3: the image is the sum of the columns of A).
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <vector>

#include "lt_internal.cuh"

using namespace ltk;

// ------------------------------------------------------------------ status / context
extern "C" const char* lt_status_str(lt_status s) {
    switch (s) {
        case LT_OK: return "ok";
        case LT_EINVAL: return "invalid argument";
        case LT_ENOMEM: return "out of device memory";
        case LT_ECUDA: return "CUDA runtime error";
        case LT_ELIMIT: return "device loop bound or capacity reached";
        case LT_ENUMERIC: return "non-finite value";
        default: return "unknown status";
    }
}

extern "C" const char* lt_last_error(const lt_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

lt_status lt_fail(lt_ctx* ctx, lt_status code, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return code;
}

lt_status lt_cuda_check(lt_ctx* ctx, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return lt_fail(ctx, e == cudaErrorMemoryAllocation ? LT_ENOMEM : LT_ECUDA, msg);
}

void* lt_scratch(lt_ctx* ctx, int slot, size_t bytes, lt_status* st) {
    *st = LT_OK;
    if (bytes == 0) bytes = 256;
    if (ctx->scr_size[slot] >= bytes) return ctx->scr[slot];
    if (ctx->use_plan) {  // a captured frame must find the scratch its warm run sized
        *st = lt_fail(ctx, LT_EINVAL, "scratch growth while a frame is being captured");
        return nullptr;
    }
    if (ctx->scr[slot]) {
        if (ctx->graphs > 0) {
            ctx->retired.push_back(ctx->scr[slot]);  // a live graph may still use it
        } else {
            cudaStreamSynchronize(ctx->stream);
            cudaFree(ctx->scr[slot]);
        }
        ctx->scr[slot] = nullptr;
        ctx->scr_size[slot] = 0;
    }
    size_t want = bytes + bytes / 4;
    if (ctx->scratch_limit > 0) {  // a caller's device-memory budget for this context
        size_t held = 0;
        for (int k = 0; k < SCR_NSLOTS; ++k) held += ctx->scr_size[k];
        if ((int64_t)(held + bytes) > ctx->scratch_limit) {
            *st = lt_fail(ctx, LT_ENOMEM, "scratch limit of " + std::to_string(ctx->scratch_limit) +
                                              " bytes reached (" + std::to_string(held + bytes) + " needed)");
            return nullptr;
        }
        if ((int64_t)(held + want) > ctx->scratch_limit) want = bytes;
    }
    cudaError_t e = cudaMalloc(&ctx->scr[slot], want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *st = lt_fail(ctx, LT_ENOMEM, "scratch allocation of " + std::to_string(want) + " bytes failed");
        return nullptr;
    }
    ctx->scr_size[slot] = want;
    return ctx->scr[slot];
}

extern "C" lt_status lt_create(lt_ctx** out, int device, void* stream) {
    if (!out) return LT_EINVAL;
    *out = nullptr;
    lt_ctx* ctx = new lt_ctx();
    ctx->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e != cudaSuccess) {
        lt_status s = lt_cuda_check(ctx, e, "cudaSetDevice");
        delete ctx;
        return s;
    }
    ctx->stream = (cudaStream_t)stream;  // NULL: the CUDA default stream
    ctx->own_stream = false;
    if (cudaMalloc(&ctx->d_status, sizeof(int32_t)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_status, sizeof(int32_t)) != cudaSuccess) {
        delete ctx;
        return LT_ENOMEM;
    }
    cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    *out = ctx;
    return LT_OK;
}

extern "C" lt_status lt_destroy(lt_ctx* ctx) {
    if (!ctx) return LT_EINVAL;
    if (ctx->graphs > 0) return lt_fail(ctx, LT_EINVAL, "lt_destroy: destroy the context's frame graphs first");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (int i = 0; i < SCR_NSLOTS; ++i)
        if (ctx->scr[i]) cudaFree(ctx->scr[i]);
    for (void* q : ctx->retired) cudaFree(q);
    cudaFree(ctx->d_boxes);
    cudaFree(ctx->d_cell_off);
    cudaFree(ctx->d_cell_box);
    cudaFree(ctx->d_mesh);
    cudaFree(ctx->d_status);
    cudaFreeHost(ctx->h_status);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
    return LT_OK;
}

extern "C" int32_t* lt_status_word(lt_ctx* ctx) { return ctx ? ctx->d_status : nullptr; }

extern "C" lt_status lt_get_tuning(const lt_ctx* ctx, lt_tuning* t) {
    if (!ctx || !t) return LT_EINVAL;
    *t = ctx->tune;
    return LT_OK;
}

extern "C" lt_status lt_set_tuning(lt_ctx* ctx, const lt_tuning* t) {
    if (!ctx || !t) return LT_EINVAL;
    if (t->eval_ctas_per_sm < 1 || t->eval_ctas_per_sm > 64 || t->ray_ctas_per_sm < 1 || t->ray_ctas_per_sm > 64 ||
        t->als_lane_entries < 16 || t->als_lane_entries > 1024 || t->als_form < 0 || t->als_form > 1 ||
        t->p1_form < 0 || t->p1_form > 1)
        return lt_fail(ctx, LT_EINVAL, "lt_set_tuning: value out of range");
    ctx->tune = *t;
    return LT_OK;
}

extern "C" int64_t lt_launch_count(const lt_ctx* ctx) { return ctx ? ctx->launches : 0; }

extern "C" lt_status lt_set_scratch_limit(lt_ctx* ctx, int64_t bytes) {
    if (!ctx || bytes < 0) return lt_fail(ctx, LT_EINVAL, "lt_set_scratch_limit: bad arguments");
    ctx->scratch_limit = bytes;
    return LT_OK;
}

extern "C" lt_status lt_debug_scratch(lt_ctx* ctx, int32_t slot, void** ptr, int64_t* bytes) {
    if (!ctx || slot < 0 || slot >= SCR_NSLOTS || !ptr || !bytes) return LT_EINVAL;
    *ptr = ctx->scr[slot];
    *bytes = (int64_t)ctx->scr_size[slot];
    return LT_OK;
}

extern "C" lt_status lt_sync(lt_ctx* ctx) {
    if (!ctx) return LT_EINVAL;
    LT_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int32_t s = *ctx->h_status;
    if (s != 0) {
        LT_CUDA(ctx, cudaMemsetAsync(ctx->d_status, 0, sizeof(int32_t), ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return lt_fail(ctx, s, std::string("device status: ") + lt_status_str(s));
    }
    return LT_OK;
}

// ------------------------------------------------------------------ occluder grid
extern "C" lt_status lt_scene_upload(lt_ctx* ctx, const float* boxes, int64_t nb, int32_t grid_res) {
    if (!ctx || nb < 0 || (nb > 0 && !boxes) || grid_res < 0 || grid_res > 128 || nb > (1 << 24))
        return lt_fail(ctx, LT_EINVAL, "lt_scene_upload: bad arguments");
    if (ctx->graphs > 0)
        return lt_fail(ctx, LT_EINVAL, "lt_scene_upload: live frame graphs reference the current scene");
    cudaSetDevice(ctx->device);
    std::vector<float> hb((size_t)nb * 6);
    if (nb) {
        LT_CUDA(ctx, cudaMemcpyAsync(hb.data(), boxes, hb.size() * sizeof(float), cudaMemcpyDeviceToHost,
                                     ctx->stream));
        LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    }
    int R = grid_res;
    if (R == 0) R = std::max(1, std::min(64, (int)ceil(2.5 * cbrt((double)std::max<int64_t>(nb, 1)))));
    const float margin = 1e-4f;
    float lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    if (nb) {
        for (int a = 0; a < 3; ++a) {
            lo[a] = 3e38f;
            hi[a] = -3e38f;
        }
        for (int64_t b = 0; b < nb; ++b)
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], hb[b * 6 + a]);
                hi[a] = std::max(hi[a], hb[b * 6 + 3 + a]);
            }
        for (int a = 0; a < 3; ++a) {
            lo[a] -= 2 * margin;
            hi[a] += 2 * margin;
        }
    }
    float cell[3], inv[3];
    for (int a = 0; a < 3; ++a) {
        cell[a] = (hi[a] - lo[a]) / R;
        if (!(cell[a] > 0)) cell[a] = 1.f;
        inv[a] = 1.f / cell[a];
    }
    const int64_t ncell = (int64_t)R * R * R;
    std::vector<int32_t> count(ncell + 1, 0);
    auto cell_range = [&](int64_t b, int a, int& c0, int& c1) {
        c0 = (int)floorf((hb[b * 6 + a] - margin - lo[a]) * inv[a]);
        c1 = (int)floorf((hb[b * 6 + 3 + a] + margin - lo[a]) * inv[a]);
        c0 = std::max(0, std::min(R - 1, c0));
        c1 = std::max(0, std::min(R - 1, c1));
    };
    for (int pass = 0; pass < 2; ++pass) {
        std::vector<int32_t> cursor;
        std::vector<int32_t> list;
        if (pass == 1) {
            for (int64_t c = 0; c < ncell; ++c) count[c + 1] += count[c];
            cursor.assign(count.begin(), count.end() - 1);
            list.assign(count[ncell], 0);
        }
        for (int64_t b = 0; b < nb; ++b) {
            int r[3][2];
            for (int a = 0; a < 3; ++a) cell_range(b, a, r[a][0], r[a][1]);
            for (int z = r[2][0]; z <= r[2][1]; ++z)
                for (int y = r[1][0]; y <= r[1][1]; ++y)
                    for (int x = r[0][0]; x <= r[0][1]; ++x) {
                        const int64_t c = ((int64_t)z * R + y) * R + x;
                        if (pass == 0) count[c + 1]++;
                        else list[cursor[c]++] = (int32_t)b;
                    }
        }
        if (pass == 1) {
            cudaFree(ctx->d_boxes);
            cudaFree(ctx->d_cell_off);
            cudaFree(ctx->d_cell_box);
            ctx->d_boxes = nullptr;
            ctx->d_cell_off = nullptr;
            ctx->d_cell_box = nullptr;
            LT_CUDA(ctx, cudaMalloc(&ctx->d_boxes, std::max<size_t>(1, hb.size()) * sizeof(float)));
            LT_CUDA(ctx, cudaMalloc(&ctx->d_cell_off, (ncell + 1) * sizeof(int32_t)));
            LT_CUDA(ctx, cudaMalloc(&ctx->d_cell_box, std::max<size_t>(1, list.size()) * sizeof(int32_t)));
            if (nb)
                LT_CUDA(ctx, cudaMemcpy(ctx->d_boxes, hb.data(), hb.size() * sizeof(float), cudaMemcpyHostToDevice));
            LT_CUDA(ctx, cudaMemcpy(ctx->d_cell_off, count.data(), (ncell + 1) * sizeof(int32_t),
                                    cudaMemcpyHostToDevice));
            if (!list.empty())
                LT_CUDA(ctx, cudaMemcpy(ctx->d_cell_box, list.data(), list.size() * sizeof(int32_t),
                                        cudaMemcpyHostToDevice));
        }
    }
    // a new scene has no triangles until lt_mesh_upload (no kernel of the stream may
    // still read the old ones)
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->d_mesh);
    ctx->d_mesh = nullptr;
    Grid& g = ctx->grid;
    g.nt = 0;
    g.tri = nullptr;
    g.bvh_aabb = nullptr;
    g.bvh_child = nullptr;
    g.bvh_tri = nullptr;
    g.box = ctx->d_boxes;
    g.cell_off = ctx->d_cell_off;
    g.cell_box = ctx->d_cell_box;
    g.nb = (int)nb;
    g.R = R;
    g.nlist = (int)(count[ncell]);
    for (int a = 0; a < 3; ++a) {
        g.lo[a] = lo[a];
        g.cell[a] = cell[a];
        g.inv_cell[a] = inv[a];
    }
    return LT_OK;
}

// ------------------------------------------------------------------ shadow test
__global__ void k_shadow_test(Grid g, const float* __restrict__ org, const float* __restrict__ end, int64_t k,
                              uint8_t* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < k; i += (int64_t)gridDim.x * blockDim.x) {
        const float3 o = make_float3(org[3 * i], org[3 * i + 1], org[3 * i + 2]);
        const float3 e = make_float3(end[3 * i], end[3 * i + 1], end[3 * i + 2]);
        out[i] = seg_blocked(g, o, e) ? 1 : 0;
    }
}

extern "C" lt_status lt_shadow_test(lt_ctx* ctx, const float* org, const float* end, int64_t k, uint8_t* blocked) {
    if (!ctx || k < 0 || (k > 0 && (!org || !end || !blocked))) return lt_fail(ctx, LT_EINVAL, "lt_shadow_test");
    if (k == 0) return LT_OK;
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_shadow_test: no scene uploaded");
    const int blocks = (int)std::min<int64_t>((k + 255) / 256, 32 * (int64_t)ctx->num_sms);
    k_shadow_test<<<blocks, 256, 0, ctx->stream>>>(ctx->grid, org, end, k, blocked);
    LT_LAUNCH_CHECK(ctx, "k_shadow_test");
    return LT_OK;
}

// ------------------------------------------------------------------ pair evaluation
__global__ void k_eval_pairs(Grid g, const float4* __restrict__ pts, int64_t m, const float4* __restrict__ vpls,
                             int64_t n, const int32_t* __restrict__ rows, const int32_t* __restrict__ vpl,
                             const float* __restrict__ scale, int64_t count, float dmin2, float* __restrict__ out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const PointRec P = load_rec(pts, m, rows[k]);
        const PointRec L = load_rec(vpls, n, vpl[k]);
        out[k] = entry_value(P, L, scale ? scale[k] : 1.f, dmin2, g);
    }
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

extern "C" lt_status lt_eval_pairs(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                                   const int32_t* rows, const int32_t* vpl, const float* scale, int64_t count,
                                   float d_min, float* out) {
    if (!ctx || count < 0 || m <= 0 || n <= 0 || !pts || !vpls || !aligned16(pts) || !aligned16(vpls) ||
        (count > 0 && (!rows || !vpl || !out)))
        return lt_fail(ctx, LT_EINVAL, "lt_eval_pairs: bad arguments");
    if (count == 0) return LT_OK;
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_eval_pairs: no scene uploaded");
    const int blocks = (int)std::min<int64_t>((count + 127) / 128, 64 * (int64_t)ctx->num_sms);
    k_eval_pairs<<<blocks, 128, 0, ctx->stream>>>(ctx->grid, (const float4*)pts, m, (const float4*)vpls, n, rows,
                                                  vpl, scale, count, d_min * d_min, out);
    LT_LAUNCH_CHECK(ctx, "k_eval_pairs");
    return LT_OK;
}

// ------------------------------------------------------------------ brute force
// One thread per shading point; the VPLs stream through shared memory in tiles.
constexpr int kBfThreads = 128;
constexpr int kBfTile = 128;

template <bool COUNT>
__global__ void __launch_bounds__(kBfThreads) k_bruteforce(Grid g, const float4* __restrict__ pts, int64_t m,
                                                           const float4* __restrict__ vpls, int64_t n, float dmin2,
                                                           float* __restrict__ img,
                                                           unsigned long long* __restrict__ stats) {
    __shared__ float4 tile[3][kBfTile];
    const int64_t i = blockIdx.x * (int64_t)kBfThreads + threadIdx.x;
    const bool live = i < m;
    PointRec P;
    if (live) P = load_rec(pts, m, i);
    float acc = 0.f;
    WorkCount wc;
    int rays = 0;
    for (int64_t j0 = 0; j0 < n; j0 += kBfTile) {
        const int cnt = (int)((n - j0) < kBfTile ? (n - j0) : kBfTile);
        __syncthreads();
        for (int t = threadIdx.x; t < cnt; t += kBfThreads) {
            tile[0][t] = __ldg(vpls + j0 + t);
            tile[1][t] = __ldg(vpls + n + j0 + t);
            tile[2][t] = __ldg(vpls + 2 * n + j0 + t);
        }
        __syncthreads();
        if (live) {
            for (int t = 0; t < cnt; ++t) {
                PointRec L;
                L.a = tile[0][t];
                L.b = tile[1][t];
                L.c = tile[2][t];
                acc += entry_value<COUNT>(P, L, 1.f, dmin2, g, &wc, &rays);
            }
        }
    }
    if (COUNT) {
        if (live) {
            atomicAdd(stats + 0, (unsigned long long)n);
            atomicAdd(stats + 1, (unsigned long long)rays);
            atomicAdd(stats + 2, (unsigned long long)wc.cells);
            atomicAdd(stats + 3, (unsigned long long)wc.boxes);
        }
    } else if (live) {
        img[i] = acc;
    }
}

extern "C" lt_status lt_bruteforce(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                                   float d_min, float* img) {
    if (!ctx || m <= 0 || n <= 0 || !pts || !vpls || !img || !aligned16(pts) || !aligned16(vpls))
        return lt_fail(ctx, LT_EINVAL, "lt_bruteforce: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_bruteforce: no scene uploaded");
    const int64_t blocks = (m + kBfThreads - 1) / kBfThreads;
    k_bruteforce<false><<<(unsigned)blocks, kBfThreads, 0, ctx->stream>>>(
        ctx->grid, (const float4*)pts, m, (const float4*)vpls, n, d_min * d_min, img, nullptr);
    LT_LAUNCH_CHECK(ctx, "k_bruteforce");
    return LT_OK;
}

extern "C" lt_status lt_bruteforce_stats(lt_ctx* ctx, const float* pts, int64_t m, const float* vpls, int64_t n,
                                         float d_min, int64_t* stats_host) {
    if (!ctx || m <= 0 || n <= 0 || !pts || !vpls || !stats_host || !aligned16(pts) || !aligned16(vpls))
        return lt_fail(ctx, LT_EINVAL, "lt_bruteforce_stats: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_bruteforce_stats: no scene uploaded");
    cudaSetDevice(ctx->device);
    lt_status st;
    unsigned long long* stats = (unsigned long long*)lt_scratch(ctx, SCR_MISC, 256, &st);
    if (!stats) return st;
    LT_CUDA(ctx, cudaMemsetAsync(stats, 0, 4 * 8, ctx->stream));
    const int64_t blocks = (m + kBfThreads - 1) / kBfThreads;
    k_bruteforce<true><<<(unsigned)blocks, kBfThreads, 0, ctx->stream>>>(
        ctx->grid, (const float4*)pts, m, (const float4*)vpls, n, d_min * d_min, nullptr, stats);
    LT_LAUNCH_CHECK(ctx, "k_bruteforce<count>");
    unsigned long long h[4];
    LT_CUDA(ctx, cudaMemcpyAsync(h, stats, sizeof(h), cudaMemcpyDeviceToHost, ctx->stream));
    LT_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    for (int i = 0; i < 4; ++i) stats_host[i] = (int64_t)h[i];
    return LT_OK;
}

// ------------------------------------------------------------------ permute points
__global__ void k_permute(const float4* __restrict__ in, int64_t m, const int32_t* __restrict__ perm,
                          float4* __restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = perm[i];
        out[i] = __ldg(in + s);
        out[m + i] = __ldg(in + m + s);
        out[2 * m + i] = __ldg(in + 2 * m + s);
    }
}

extern "C" lt_status lt_permute_points(lt_ctx* ctx, const float* pts, int64_t m, const int32_t* row_perm,
                                       float* pts_out) {
    if (!ctx || m <= 0 || !pts || !row_perm || !pts_out || !aligned16(pts) || !aligned16(pts_out))
        return lt_fail(ctx, LT_EINVAL, "lt_permute_points: bad arguments");
    const int blocks = (int)std::min<int64_t>((m + 255) / 256, 16 * (int64_t)ctx->num_sms);
    k_permute<<<blocks, 256, 0, ctx->stream>>>((const float4*)pts, m, row_perm, (float4*)pts_out);
    LT_LAUNCH_CHECK(ctx, "k_permute");
    return LT_OK;
}
