// The whole frame: the plain sequence of launches and its captured CUDA graph.
//
// A frame is Sec. 3 steps 3-5: pass 1 with coarsening (Sec. 4), pass 2 (Sec. 5),
// evaluation of the new entries, completion and the factorised render.  Every call
// of the sequence is sync-free except two read-backs of sizes that depend on the
// setup only (pass-1 row slots and forest levels; the sampling capacity).  The
// graph form records them in a warm run, then captures the frame on a private
// stream with those sizes fixed and the seed read from a device word, so one
// instantiated graph replays any seed with a single launch.
#include "lt_internal.cuh"

using namespace ltk;

struct lt_graph {
    lt_ctx* ctx = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t* d_seed = nullptr;
    int64_t kernels = 0;
};

namespace {

__global__ void k_set_seed(uint64_t* dst, uint64_t seed) { *dst = seed; }

bool params_ok(const lt_params* p) {
    return p && p->rate1 >= 0.f && p->tau >= 0.f && p->d_min >= 0.f && p->rate >= 0.f && p->als_iters >= 0 &&
           p->lam_rel >= 0.f && (!p->proposal || (p->mix >= 0.f && p->mix <= 1.f)) && p->rank_cols >= 0 &&
           (p->completion == LT_COMPLETE_ALS ||
            (p->completion == LT_COMPLETE_ADM && p->adm_iters >= 0 && p->adm_alpha_rel > 0.f &&
             p->adm_gamma > 0.f && p->adm_gamma < 1.618f)) &&
           p->target_cut >= 0;
}

lt_status run_frame(lt_ctx* ctx, const lt_frame* f, const lt_params* p, uint64_t seed, lt_samples* smp,
                    lt_factors* uv, const int32_t* row_perm, float* img) {
    lt_status st = p->target_cut > 0 ? lt_sample_pass1_target(ctx, f, p->rate1, p->target_cut, p->d_min, seed, smp)
                                     : lt_sample_pass1(ctx, f, p->rate1, p->tau, p->d_min, seed, smp);
    if (st != LT_OK) return st;
    if (p->rank_cols > 0) {  // per-slice ranks from the coarsened cut
        st = lt_slice_ranks(ctx, f, smp, uv->r, p->rank_cols, uv->rank);
        if (st != LT_OK) return st;
    }
    const float* w = p->weights;
    if (!w && p->proposal) {
        // learned proposal: features -> logits -> mixed weights, all on the stream
        const size_t rows = (size_t)f->S * f->C;
        char* q = (char*)lt_scratch(ctx, SCR_FRAME_PROP, rows * (LT_MLP_FEATURES + 2) * 4 + (f->S + 1) * 4 + 4 * 256,
                                    &st);
        if (!q) return st;
        float* feat = (float*)q;
        float* z = feat + rows * LT_MLP_FEATURES;
        float* wts = z + rows;
        int32_t* goff = (int32_t*)((char*)(wts + rows) + 256 - (((size_t)(wts + rows)) & 255));
        st = lt_proposal_features(ctx, f, smp, feat, goff);
        if (st != LT_OK) return st;
        st = lt_proposal_forward(ctx, p->proposal, feat, (int64_t)rows, goff + f->S, z);
        if (st != LT_OK) return st;
        st = lt_proposal_weights(ctx, f, smp, goff, z, p->mix, wts);
        if (st != LT_OK) return st;
        w = wts;
    }
    st = lt_sample_pass2(ctx, f, w, p->rate, seed, smp);
    if (st != LT_OK) return st;
    st = lt_eval_entries(ctx, f, p->d_min, smp);
    if (st != LT_OK) return st;
    st = p->completion == LT_COMPLETE_ADM
             ? lt_complete_adm(ctx, f, smp, p->adm_iters, p->adm_alpha_rel, p->adm_gamma, seed, uv)
             : lt_complete(ctx, f, smp, p->als_iters, p->lam_rel, seed, uv);
    if (st != LT_OK) return st;
    return lt_render(ctx, f, smp, uv, nullptr, row_perm, img);
}

}  // namespace

extern "C" lt_status lt_render_frame(lt_ctx* ctx, const lt_frame* f, const lt_params* p, uint64_t seed,
                                     lt_samples* smp, lt_factors* uv, const int32_t* row_perm, float* img) {
    if (!ctx || !f || !params_ok(p) || !smp || !uv || !row_perm || !img || (p->rank_cols > 0 && !uv->rank))
        return lt_fail(ctx, LT_EINVAL, "lt_render_frame: bad arguments");
    return run_frame(ctx, f, p, seed, smp, uv, row_perm, img);
}

extern "C" lt_status lt_frame_graph_capture(lt_ctx* ctx, const lt_frame* f, const lt_params* p, lt_samples* smp,
                                            lt_factors* uv, const int32_t* row_perm, float* img, lt_graph** out) {
    if (!ctx || !f || !params_ok(p) || !smp || !uv || !row_perm || !img || !out || (p->rank_cols > 0 && !uv->rank))
        return lt_fail(ctx, LT_EINVAL, "lt_frame_graph_capture: bad arguments");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    // warm run: records the setup-dependent sizes and grows the scratch to them
    lt_status st = run_frame(ctx, f, p, 0, smp, uv, row_perm, img);
    if (st != LT_OK) return st;
    st = lt_sync(ctx);
    if (st != LT_OK) return st;
    lt_graph* g = new lt_graph();
    g->ctx = ctx;
    cudaError_t e = cudaMalloc(&g->d_seed, sizeof(uint64_t));
    if (e != cudaSuccess) {
        delete g;
        return lt_cuda_check(ctx, e, "cudaMalloc(seed)");
    }
    cudaStream_t cap = nullptr;
    e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(g->d_seed);
        delete g;
        return lt_cuda_check(ctx, e, "cudaStreamCreateWithFlags");
    }
    cudaStream_t orig = ctx->stream;
    const int64_t n0 = ctx->launches;
    ctx->stream = cap;
    ctx->use_plan = true;
    ctx->seed_dev = g->d_seed;
    cudaGraph_t graph = nullptr;
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        st = run_frame(ctx, f, p, 0, smp, uv, row_perm, img);
        const cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (st == LT_OK && e2 != cudaSuccess) st = lt_cuda_check(ctx, e2, "cudaStreamEndCapture");
    } else {
        st = lt_cuda_check(ctx, e, "cudaStreamBeginCapture");
    }
    ctx->stream = orig;
    ctx->use_plan = false;
    ctx->seed_dev = nullptr;
    g->kernels = ctx->launches - n0;
    ctx->launches = n0;
    cudaStreamDestroy(cap);
    if (st == LT_OK) {
        e = cudaGraphInstantiate(&g->exec, graph, 0);
        if (e != cudaSuccess) st = lt_cuda_check(ctx, e, "cudaGraphInstantiate");
    }
    if (graph) cudaGraphDestroy(graph);
    if (st != LT_OK) {
        cudaGetLastError();
        if (g->exec) cudaGraphExecDestroy(g->exec);
        cudaFree(g->d_seed);
        delete g;
        return st;
    }
    ctx->graphs++;
    *out = g;
    return LT_OK;
}

extern "C" lt_status lt_frame_graph_launch(lt_graph* g, uint64_t seed) {
    if (!g || !g->ctx || !g->exec) return LT_EINVAL;
    lt_ctx* ctx = g->ctx;
    cudaSetDevice(ctx->device);
    k_set_seed<<<1, 1, 0, ctx->stream>>>(g->d_seed, seed);
    LT_LAUNCH_CHECK(ctx, "k_set_seed");
    LT_CUDA(ctx, cudaGraphLaunch(g->exec, ctx->stream));
    ctx->launches += g->kernels;
    return LT_OK;
}

extern "C" int64_t lt_frame_graph_kernels(const lt_graph* g) { return g ? g->kernels : 0; }

extern "C" lt_status lt_frame_graph_destroy(lt_graph* g) {
    if (!g) return LT_EINVAL;
    lt_ctx* ctx = g->ctx;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    cudaFree(g->d_seed);
    ctx->graphs--;
    if (ctx->graphs == 0) {
        for (void* q : ctx->retired) cudaFree(q);
        ctx->retired.clear();
    }
    delete g;
    return LT_OK;
}
