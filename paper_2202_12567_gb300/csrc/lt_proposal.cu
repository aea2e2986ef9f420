// Learned pass-2 proposal: per-(slice, column) features after pass 1, a bfloat16
// MLP (32 -> 64 -> 64 -> 64 -> 1, SiLU) on the tensor cores (mma.sync m16n8k16,
// float32 accumulate), the slice softmax mixed with the pass-1 estimate g (Sec. 5)
// into pass-2 weights, and the training side: full slice matrices, leverage targets
// by subspace iteration, forward + backward + Adam.  The paper names a learned
// importance only as future work; every choice here is ours (layout of the features
// and of the parameters in include/lt.h).
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "lt_internal.cuh"

using namespace ltk;

namespace {

constexpr int NF = LT_MLP_FEATURES, NH = LT_MLP_HIDDEN, NPAR = LT_MLP_PARAMS;
constexpr int OW1 = 0, OB1 = OW1 + NH * NF, OW2 = OB1 + NH, OB2 = OW2 + NH * NH, OW3 = OB2 + NH,
              OB3 = OW3 + NH * NH, OW4 = OB3 + NH, OB4 = OW4 + NH;
static_assert(OB4 + 1 == NPAR, "parameter layout");
constexpr uint32_t kTagLeverage = 4, kTagInit = 5;
constexpr int TM = 64;            // rows per tile (4 warps x 16)
constexpr int L1 = NF + 8;        // bf16 row stride of 32-wide operands (conflict-free fragments)
constexpr int L2 = NH + 8;        // of 64-wide operands

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ float silu(float h) { return h / (1.f + expf(-h)); }
__device__ __forceinline__ float dsilu(float h) {
    const float s = 1.f / (1.f + expf(-h));
    return s * (1.f + h * (1.f - s));
}
__device__ __forceinline__ float rbf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t ld2(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }

// One warp: C[16][8 NT] += A[16][K] B^T with A row-major (stride lda) and Bt = B^T
// row-major [8 NT][K] (stride ldb), K a multiple of 16.  Fragment layout of
// m16n8k16: g = lane / 4, t = lane % 4; A regs (g, 2t) (g+8, 2t) (g, 2t+8)
// (g+8, 2t+8); B regs (k 2t, n g) (k 2t+8, n g); C (g, 2t) (g, 2t+1) (g+8, 2t) (g+8, 2t+1).
template <int NT>
__device__ __forceinline__ void warp_gemm(const bf16* A, int lda, const bf16* Bt, int ldb, int K, float (&c)[NT][4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    for (int k0 = 0; k0 < K; k0 += 16) {
        const uint32_t a0 = ld2(A + g * lda + k0 + 2 * t), a1 = ld2(A + (g + 8) * lda + k0 + 2 * t);
        const uint32_t a2 = ld2(A + g * lda + k0 + 8 + 2 * t), a3 = ld2(A + (g + 8) * lda + k0 + 8 + 2 * t);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const bf16* b = Bt + (8 * nt + g) * ldb + k0 + 2 * t;
            mma_bf16(c[nt], a0, a1, a2, a3, ld2(b), ld2(b + 8));
        }
    }
}

template <int NT>
__device__ __forceinline__ void zero(float (&c)[NT][4]) {
#pragma unroll
    for (int i = 0; i < NT; ++i) c[i][0] = c[i][1] = c[i][2] = c[i][3] = 0.f;
}

// ---------------------------------------------------------------- parameters
struct MlpSmem {
    bf16 X[TM * L1];      // input tile, rows x 32
    bf16 W1[NH * L1];     // [out][in]
    bf16 W2[NH * L2];
    bf16 W3[NH * L2];
    bf16 A1[TM * L2];     // activations, rows x 64
    bf16 A2[TM * L2];
    bf16 A3[TM * L2];
    float b1[NH], b2[NH], b3[NH], w4[NH], b4;
    float z[TM];
};

__device__ void load_params(const float* __restrict__ th, MlpSmem& s) {
    for (int i = threadIdx.x; i < NH * NF; i += blockDim.x) s.W1[(i / NF) * L1 + i % NF] = __float2bfloat16_rn(th[OW1 + i]);
    for (int i = threadIdx.x; i < NH * NH; i += blockDim.x) {
        s.W2[(i / NH) * L2 + i % NH] = __float2bfloat16_rn(th[OW2 + i]);
        s.W3[(i / NH) * L2 + i % NH] = __float2bfloat16_rn(th[OW3 + i]);
    }
    for (int i = threadIdx.x; i < NH; i += blockDim.x) {
        s.b1[i] = th[OB1 + i];
        s.b2[i] = th[OB2 + i];
        s.b3[i] = th[OB3 + i];
        s.w4[i] = rbf(th[OW4 + i]);
    }
    if (threadIdx.x == 0) s.b4 = th[OB4];
}

// rows [r0, r0 + TM) of feat into s.X (rows >= n are zero)
__device__ void load_tile(const float* __restrict__ feat, int64_t r0, int64_t n, MlpSmem& s) {
    for (int i = threadIdx.x; i < TM * NF; i += blockDim.x) {
        const int row = i / NF, c = i % NF;
        const float v = r0 + row < n ? feat[(r0 + row) * NF + c] : 0.f;
        s.X[row * L1 + c] = __float2bfloat16_rn(v);
    }
}

// one hidden layer for the warp's 16 rows: H = A W^T + b, out = bf16(silu(H)); the
// pre-activations go to Hs (float [TM][NH]) when it is given
template <int K>
__device__ __forceinline__ void layer(const bf16* Ain, int lda, const bf16* W, int ldw, const float* b, bf16* Aout,
                                      float* Hs) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    float c[8][4];
    zero(c);
    warp_gemm<8>(Ain + 16 * w * lda, lda, W, ldw, K, c);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = 16 * w + g + (q >= 2 ? 8 : 0), col = 8 * nt + 2 * t + (q & 1);
            const float h = c[nt][q] + b[col];
            if (Hs) Hs[row * NH + col] = h;
            Aout[row * L2 + col] = __float2bfloat16_rn(silu(h));
        }
}

// forward of the tile in s.X: logits into s.z (each warp its 16 rows)
__device__ void forward_tile(MlpSmem& s, float* H1, float* H2, float* H3) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    layer<NF>(s.X, L1, s.W1, L1, s.b1, s.A1, H1);
    __syncwarp();
    layer<NH>(s.A1, L2, s.W2, L2, s.b2, s.A2, H2);
    __syncwarp();
    layer<NH>(s.A2, L2, s.W3, L2, s.b3, s.A3, H3);
    __syncwarp();
    if (lane < 16) {
        const int row = 16 * w + lane;
        float z = s.b4;
        for (int j = 0; j < NH; ++j) z = fmaf(__bfloat162float(s.A3[row * L2 + j]), s.w4[j], z);
        s.z[row] = z;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(128) k_mlp_forward(const float* __restrict__ theta, const float* __restrict__ feat,
                                                     int64_t n_max, const int32_t* __restrict__ n_dev,
                                                     float* __restrict__ z) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlpSmem& s = *reinterpret_cast<MlpSmem*>(smem_raw);
    const int64_t n = n_dev ? min((int64_t)*n_dev, n_max) : n_max;
    load_params(theta, s);
    for (int64_t r0 = (int64_t)blockIdx.x * TM; r0 < n; r0 += (int64_t)gridDim.x * TM) {
        __syncthreads();
        load_tile(feat, r0, n, s);
        __syncthreads();
        forward_tile(s, nullptr, nullptr, nullptr);
        __syncthreads();
        for (int i = threadIdx.x; i < TM; i += blockDim.x)
            if (r0 + i < n) z[r0 + i] = s.z[i];
    }
}

// ---------------------------------------------------------------- training
struct BwdSmem {
    MlpSmem f;
    bf16 XT[NF * L2];      // [in][rows]
    bf16 A1T[NH * L2];     // [in][rows]
    bf16 A2T[NH * L2];
    bf16 W2T[NH * L2];     // [in][out]
    bf16 W3T[NH * L2];
    bf16 D[TM * L2];       // dH of the current layer, [rows][out]
    bf16 DT[NH * L2];      // [out][rows]
    float H1[TM * NH], H2[TM * NH], H3[TM * NH];  // pre-activations, then dH in float
    float dz[TM];
    float grad[NPAR];      // this CTA's gradient, accumulated over its tiles
};

// transpose a [rows][cols] bf16 tile (stride ls) into [cols][rows] (stride lt)
__device__ void transpose(const bf16* S, int ls, bf16* T, int lt, int rows, int cols) {
    for (int i = threadIdx.x; i < rows * cols; i += blockDim.x) {
        const int r = i / cols, c = i % cols;
        T[c * lt + r] = S[r * ls + c];
    }
}

// dW[out][in] += DT[out][rows] (X^T)[in][rows]^T for the tile: warp w owns outputs 16w..
template <int NT>
__device__ void weight_grad(const bf16* DT, const bf16* XT, int K_in, float* gW) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    float c[NT][4];
    zero(c);
    warp_gemm<NT>(DT + 16 * w * L2, L2, XT, L2, TM, c);
#pragma unroll
    for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int o = 16 * w + g + (q >= 2 ? 8 : 0), i = 8 * nt + 2 * t + (q & 1);
            gW[o * K_in + i] += c[nt][q];
        }
}

// Hf [rows][NH] float holds dA of the layer on entry; turns it into dH = dA silu'(H)
// (H the pre-activations in Hpre), fills D / DT (bf16) and adds the bias gradient.
__device__ void act_grad(float* Hf, const float* Hpre, BwdSmem& s, float* gb, int nrows) {
    for (int i = threadIdx.x; i < TM * NH; i += blockDim.x) {
        const int r = i / NH, c = i % NH;
        const float d = r < nrows ? Hf[i] * dsilu(Hpre[i]) : 0.f;
        Hf[i] = d;
        const bf16 b = __float2bfloat16_rn(d);
        s.D[r * L2 + c] = b;
        s.DT[c * L2 + r] = b;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < NH; c += blockDim.x) {
        float a = 0.f;
        for (int r = 0; r < TM; ++r) a += Hf[r * NH + c];
        gb[c] += a;
    }
}

// dA_prev[rows][in] = D[rows][out] W[out][in] (Wt = W^T as [in][out]) into Hf
__device__ void input_grad(const BwdSmem& s, const bf16* Wt, float* Hf) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, w = threadIdx.x >> 5;
    float c[8][4];
    zero(c);
    warp_gemm<8>(s.D + 16 * w * L2, L2, Wt, L2, NH, c);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int row = 16 * w + g + (q >= 2 ? 8 : 0), col = 8 * nt + 2 * t + (q & 1);
            Hf[row * NH + col] = c[nt][q];
        }
}

// Gradient of loss = sum_rows dz * z over rows [0, n); per CTA into part[blockIdx][NPAR].
__global__ void __launch_bounds__(128) k_mlp_backward(const float* __restrict__ theta, const float* __restrict__ feat,
                                                      const float* __restrict__ dz, int64_t n,
                                                      float* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    BwdSmem& s = *reinterpret_cast<BwdSmem*>(smem_raw);
    load_params(theta, s.f);
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) s.grad[i] = 0.f;
    __syncthreads();
    transpose(s.f.W2, L2, s.W2T, L2, NH, NH);
    transpose(s.f.W3, L2, s.W3T, L2, NH, NH);
    for (int64_t r0 = (int64_t)blockIdx.x * TM; r0 < n; r0 += (int64_t)gridDim.x * TM) {
        const int nrows = (int)min((int64_t)TM, n - r0);
        __syncthreads();
        load_tile(feat, r0, n, s.f);
        for (int i = threadIdx.x; i < TM; i += blockDim.x) s.dz[i] = i < nrows ? dz[r0 + i] : 0.f;
        __syncthreads();
        forward_tile(s.f, s.H1, s.H2, s.H3);
        __syncthreads();
        // output layer: z = w4 . a3 + b4
        for (int j = threadIdx.x; j < NH; j += blockDim.x) {
            float a = 0.f;
            for (int r = 0; r < TM; ++r) a += s.dz[r] * __bfloat162float(s.f.A3[r * L2 + j]);
            s.grad[OW4 + j] += a;
        }
        if (threadIdx.x == 0) {
            float a = 0.f;
            for (int r = 0; r < TM; ++r) a += s.dz[r];
            s.grad[OB4] += a;
        }
        // dH3 = dz w4 silu'(H3), in place of the pre-activations
        for (int i = threadIdx.x; i < TM * NH; i += blockDim.x) {
            const int r = i / NH, c = i % NH;
            s.H3[i] = r < nrows ? s.dz[r] * s.f.w4[c] * dsilu(s.H3[i]) : 0.f;
        }
        __syncthreads();
        for (int i = threadIdx.x; i < TM * NH; i += blockDim.x) {
            const int r = i / NH, c = i % NH;
            const bf16 b = __float2bfloat16_rn(s.H3[i]);
            s.D[r * L2 + c] = b;
            s.DT[c * L2 + r] = b;
        }
        transpose(s.f.A2, L2, s.A2T, L2, TM, NH);
        transpose(s.f.A1, L2, s.A1T, L2, TM, NH);
        transpose(s.f.X, L1, s.XT, L2, TM, NF);
        __syncthreads();
        for (int c = threadIdx.x; c < NH; c += blockDim.x) {
            float a = 0.f;
            for (int r = 0; r < TM; ++r) a += s.H3[r * NH + c];
            s.grad[OB3 + c] += a;
        }
        weight_grad<8>(s.DT, s.A2T, NH, s.grad + OW3);
        __syncthreads();
        // layer 2
        input_grad(s, s.W3T, s.H3);  // dA2 into H3's storage
        __syncthreads();
        act_grad(s.H3, s.H2, s, s.grad + OB2, nrows);
        __syncthreads();
        weight_grad<8>(s.DT, s.A1T, NH, s.grad + OW2);
        __syncthreads();
        // layer 1
        input_grad(s, s.W2T, s.H3);  // dA1
        __syncthreads();
        act_grad(s.H3, s.H1, s, s.grad + OB1, nrows);
        __syncthreads();
        weight_grad<4>(s.DT, s.XT, NF, s.grad + OW1);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NPAR; i += blockDim.x) part[(int64_t)blockIdx.x * NPAR + i] = s.grad[i];
}

// softmax over each group's rows, dz = (softmax - target) / G, loss per group
__global__ void k_group_softmax(const float* __restrict__ z, const float* __restrict__ target,
                                const int32_t* __restrict__ goff, int G, float* __restrict__ dz,
                                float* __restrict__ gloss) {
    const int lane = threadIdx.x & 31;
    for (int gi = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < G; gi += gridDim.x * (blockDim.x >> 5)) {
        const int a = goff[gi], b = goff[gi + 1];
        float mx = -3.0e38f;
        for (int i = a + lane; i < b; i += 32) mx = fmaxf(mx, z[i]);
        mx = warp_max(mx);
        float se = 0.f;
        for (int i = a + lane; i < b; i += 32) se += expf(z[i] - mx);
        se = warp_sum(se);
        const float lse = logf(se);
        float l = 0.f;
        for (int i = a + lane; i < b; i += 32) {
            const float lp = z[i] - mx - lse;
            dz[i] = (expf(lp) - target[i]) / (float)G;
            l -= target[i] * lp;
        }
        l = warp_sum(l);
        if (lane == 0) gloss[gi] = l;
    }
}

// grad[p] = sum over the CTA partials in order; loss = sum of the group losses / G
__global__ void k_grad_reduce(const float* __restrict__ part, int nparts, float* __restrict__ grad,
                              const float* __restrict__ gloss, int G, float* __restrict__ loss) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPAR; p += gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int q = 0; q < nparts; ++q) a += part[(int64_t)q * NPAR + p];
        grad[p] = a;
    }
    if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
        float a = 0.f;
        for (int g = 0; g < G; ++g) a += gloss[g];
        *loss = a / (float)G;
    }
}

__global__ void k_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ grad, int step, float lr) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPAR; p += gridDim.x * blockDim.x) {
        const float g = grad[p];
        const float mm = b1 * m[p] + (1.f - b1) * g;
        const float vv = b2 * v[p] + (1.f - b2) * g * g;
        m[p] = mm;
        v[p] = vv;
        theta[p] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
    }
}

__global__ void k_mlp_init(uint64_t seed, float* __restrict__ theta) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < NPAR; p += gridDim.x * blockDim.x) {
        float v = 0.f;
        const bool w = p < OB1 || (p >= OW2 && p < OB2) || (p >= OW3 && p < OB3) || (p >= OW4 && p < OB4);
        if (w) {
            const float fan = p < OB1 ? (float)NF : (float)NH;
            const float u = (float)((double)philox((uint32_t)p, 0u, 0u, kTagInit, seed).x * 2.3283064365386963e-10 - 0.5);
            v = 2.f * u / sqrtf(fan);
        }
        theta[p] = v;
    }
}

// ---------------------------------------------------------------- features
// per slice: mean position and normal, AABB, mean pass-1 value, m', n'
constexpr int kSliceStats = 16;

__global__ void k_feat_slice(lt_frame F, lt_samples smp, float* __restrict__ st) {
    __shared__ float red[16][32];
    const int s = blockIdx.x;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0;
    const float4* P0 = reinterpret_cast<const float4*>(F.pts);
    const float4* P1 = P0 + F.m;
    float acc[13];
    for (int k = 0; k < 6; ++k) acc[k] = 0.f;
    for (int k = 6; k < 9; ++k) acc[k] = 3.0e38f;
    for (int k = 9; k < 12; ++k) acc[k] = -3.0e38f;
    acc[12] = 0.f;
    for (int i = threadIdx.x; i < ms; i += blockDim.x) {
        const float4 p = P0[row0 + i], nn = P1[row0 + i];
        acc[0] += p.x;
        acc[1] += p.y;
        acc[2] += p.z;
        acc[3] += nn.x;
        acc[4] += nn.y;
        acc[5] += nn.z;
        acc[6] = fminf(acc[6], p.x);
        acc[7] = fminf(acc[7], p.y);
        acc[8] = fminf(acc[8], p.z);
        acc[9] = fmaxf(acc[9], p.x);
        acc[10] = fmaxf(acc[10], p.y);
        acc[11] = fmaxf(acc[11], p.z);
    }
    const int n1 = smp.n1[s];
    const float* val = smp.val + smp.off[s];
    for (int e = threadIdx.x; e < n1; e += blockDim.x) acc[12] += val[e];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int k = 0; k < 13; ++k) {
        float v = acc[k];
        v = (k >= 6 && k < 9) ? warp_min(v) : (k >= 9 && k < 12) ? warp_max(v) : warp_sum(v);
        if (lane == 0) red[k][w] = v;
    }
    __syncthreads();
    if (threadIdx.x < 13) {
        const int k = threadIdx.x;
        float v = red[k][0];
        for (int q = 1; q < nw; ++q) v = (k >= 6 && k < 9) ? fminf(v, red[k][q]) : (k >= 9 && k < 12) ? fmaxf(v, red[k][q]) : v + red[k][q];
        float* o = st + (int64_t)s * kSliceStats;
        if (k < 6) o[k] = ms > 0 ? v / (float)ms : 0.f;
        else if (k < 12) o[k] = ms > 0 ? v : 0.f;
        else {
            const float mu = n1 > 0 ? v / (float)n1 : 0.f;
            o[12] = mu > 0.f ? mu : 1.f;
            o[13] = logf((float)max(ms, 1)) / 10.f;
            o[14] = logf((float)max(smp.ncol[s], 1)) / 10.f;
        }
    }
}

__global__ void k_group_prefix(const int32_t* __restrict__ ncol, int S, int32_t* __restrict__ goff) {
    __shared__ int32_t ws[32];
    int carry = 0;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int x = s < S ? ncol[s] : 0;
        int tot;
        const int pre = block_exclusive_scan<int>(x, ws, &tot);
        if (s < S) goff[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) goff[S] = carry;
}

// first pass-1 entry of the slice (keys grouped by column, ascending) whose column >= j
__device__ __forceinline__ int first_col_at_least(const uint32_t* key, int n1, int j) {
    int a = 0, b = n1;
    while (a < b) {
        const int m = (a + b) >> 1;
        if ((int)(key[m] & 0xffffu) < j) a = m + 1; else b = m;
    }
    return a;
}

// one warp per (slice, column): the 32 features into feat[goff[s] + j]
__global__ void k_feat_cols(lt_frame F, lt_samples smp, const float* __restrict__ st,
                            const int32_t* __restrict__ goff, float* __restrict__ feat) {
    const int lane = threadIdx.x & 31;
    const int S = F.S, C = F.C;
    const float4* V0 = reinterpret_cast<const float4*>(F.vpls);
    const float4* V1 = V0 + F.n;
    const float iroot = F.tree.I[0];
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t x = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); x < (int64_t)S * C; x += nwarps) {
        const int s = (int)(x / C), j = (int)(x % C);
        const int ns = smp.ncol[s];
        if (j >= ns) continue;
        const uint32_t* key = smp.key + smp.off[s];
        const float* val = smp.val + smp.off[s];
        const int n1 = smp.n1[s];
        const int lo = first_col_at_least(key, n1, j), hi = first_col_at_least(key, n1, j + 1);
        const int cnt = hi - lo;
        float sum = 0.f, mn = 3.0e38f, mx = -3.0e38f;
        for (int e = lo + lane; e < hi; e += 32) {
            const float v = val[e];
            sum += v;
            mn = fminf(mn, v);
            mx = fmaxf(mx, v);
        }
        sum = warp_sum(sum);
        mn = warp_min(mn);
        mx = warp_max(mx);
        const float mean = cnt > 0 ? sum / (float)cnt : 0.f;
        float sq = 0.f;
        for (int e = lo + lane; e < hi; e += 32) {
            const float d = val[e] - mean;
            sq += d * d;
        }
        sq = warp_sum(sq);
        const float* ss = st + (int64_t)s * kSliceStats;
        const float mu = ss[12];
        const int node = smp.col_node[(int64_t)s * C + j];
        const int rep = F.tree.rep[node];
        float v = 0.f;
        if (lane < 12) v = ss[lane];
        else if (lane < 18) v = F.tree.aabb[(int64_t)node * 6 + (lane - 12)];
        else if (lane < 24) {
            const float4 p = lane < 21 ? V0[rep] : V1[rep];
            const int k = (lane - 18) % 3;
            v = k == 0 ? p.x : k == 1 ? p.y : p.z;
        } else if (lane == 24) v = logf(F.tree.I[node] / iroot);
        else if (lane == 25) v = mean / mu;
        else if (lane == 26) v = cnt > 0 ? sqrtf(sq / (float)cnt) / mu : 0.f;
        else if (lane == 27) v = log1pf((float)cnt);
        else if (lane == 28) v = cnt > 0 ? mn / mu : 0.f;
        else if (lane == 29) v = cnt > 0 ? mx / mu : 0.f;
        else if (lane == 30) v = ss[13];
        else v = ss[14];
        feat[((int64_t)goff[s] + j) * NF + lane] = v;
    }
}

// pass-2 weights w[s][j] = mix softmax_s(z)_j + (1 - mix) g_j / sum g (one warp per slice)
__global__ void k_mix_weights(lt_frame F, lt_samples smp, const int32_t* __restrict__ goff,
                              const float* __restrict__ z, float mix, float* __restrict__ w) {
    const int lane = threadIdx.x & 31;
    for (int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); s < F.S; s += gridDim.x * (blockDim.x >> 5)) {
        const int ns = smp.ncol[s];
        const float* zz = z + goff[s];
        const float* g = smp.g + (int64_t)s * F.C;
        float mx = -3.0e38f, gs = 0.f;
        for (int j = lane; j < ns; j += 32) {
            mx = fmaxf(mx, zz[j]);
            gs += fmaxf(g[j], 0.f);
        }
        mx = warp_max(mx);
        gs = warp_sum(gs);
        float se = 0.f;
        for (int j = lane; j < ns; j += 32) se += expf(zz[j] - mx);
        se = warp_sum(se);
        for (int j = lane; j < ns; j += 32) {
            const float pg = gs > 0.f ? fmaxf(g[j], 0.f) / gs : 1.f / (float)ns;
            w[(int64_t)s * F.C + j] = mix * (expf(zz[j] - mx) / se) + (1.f - mix) * pg;
        }
    }
}

// ---------------------------------------------------------------- targets
// M_s[i][c] = A(row0 + i, column c) for every slice, at M + moff[s]
__global__ void k_moff(lt_frame F, lt_samples smp, int64_t* __restrict__ moff) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < F.S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < F.S ? (int64_t)(F.slice_off[s + 1] - F.slice_off[s]) * smp.ncol[s] : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < F.S) moff[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) moff[F.S] = carry;
}

__global__ void __launch_bounds__(256) k_slice_matrix(lt_frame F, lt_samples smp, Grid g, float dmin2,
                                                      const int64_t* __restrict__ moff, int64_t cap,
                                                      float* __restrict__ M, int32_t* status) {
    const float4* pts = reinterpret_cast<const float4*>(F.pts);
    const float4* vpls = reinterpret_cast<const float4*>(F.vpls);
    if (moff[F.S] > cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) latch(status, LT_ELIMIT);
        return;
    }
    const int s = blockIdx.y;
    const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0, ns = smp.ncol[s];
    float* out = M + moff[s];
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)ms * ns;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(e / ns), c = (int)(e % ns);
        const int node = smp.col_node[(int64_t)s * F.C + c];
        const int rep = F.tree.rep[node];
        const PointRec P = load_rec(pts, F.m, row0 + i);
        const PointRec L = load_rec(vpls, F.n, rep);
        // I_c / I_rep(c), I = flux * albedo, rounded as in the sampling passes
        const float scale = __fdiv_rn(F.tree.I[node], __fmul_rn(L.c.w, L.a.w));
        out[e] = entry_value(P, L, scale, dmin2, g);
    }
}

// G_s = M_s^T M_s (n' x n', float) at G + goff2[s] with goff2 the prefix of n'^2
__global__ void k_goff(lt_samples smp, int S, int64_t* __restrict__ goff2) {
    __shared__ int64_t ws[32];
    int64_t carry = 0;
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        const int64_t x = s < S ? (int64_t)smp.ncol[s] * smp.ncol[s] : 0;
        int64_t tot;
        const int64_t pre = block_exclusive_scan<int64_t>(x, ws, &tot);
        if (s < S) goff2[s] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) goff2[S] = carry;
}

// 32 x 32 output tiles, rows of M streamed through shared memory in steps of 32
__global__ void __launch_bounds__(256) k_gram(lt_frame F, lt_samples smp, const float* __restrict__ M,
                                              const int64_t* __restrict__ moff, const int64_t* __restrict__ goff2,
                                              int64_t gcap, float* __restrict__ G) {
    __shared__ float A[32][33], B[32][33];
    if (goff2[F.S] > gcap) return;
    const int s = blockIdx.z;
    const int ms = F.slice_off[s + 1] - F.slice_off[s], ns = smp.ncol[s];
    const int ti = blockIdx.y * 32, tj = blockIdx.x * 32;
    if (ti >= ns || tj >= ns) return;
    const float* Ms = M + moff[s];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 4 outputs per thread
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r0 = 0; r0 < ms; r0 += 32) {
        for (int q = ty; q < 32; q += 8) {
            const int r = r0 + q;
            A[q][tx] = (r < ms && ti + tx < ns) ? Ms[(int64_t)r * ns + ti + tx] : 0.f;
            B[q][tx] = (r < ms && tj + tx < ns) ? Ms[(int64_t)r * ns + tj + tx] : 0.f;
        }
        __syncthreads();
        for (int k = 0; k < 32; ++k) {
            const float b = B[k][tx];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fmaf(A[k][ty + 8 * u], b, acc[u]);
        }
        __syncthreads();
    }
    float* Gs = G + goff2[s];
    for (int u = 0; u < 4; ++u) {
        const int i = ti + ty + 8 * u, j = tj + tx;
        if (i < ns && j < ns) Gs[(int64_t)i * ns + j] = acc[u];
    }
}

// Subspace iteration per slice (one CTA): Q (n' x r, float, in global scratch) from
// Philox, `iters` rounds of Q <- mgs(G Q), then p_c = (|Q_c|^2 + 1/n') / (r' + 1) with
// r' the columns kept.  Modified Gram-Schmidt column by column, block reductions in a
// fixed order.
__device__ float block_sum(float v, float* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    float t = 0.f;
    for (int q = 0; q < nw; ++q) t += red[q];
    return t;
}

__device__ void mgs_cols(float* Q, int n, int r, float* red) {
    for (int k = 0; k < r; ++k) {
        for (int j = 0; j < k; ++j) {
            float d = 0.f;
            for (int i = threadIdx.x; i < n; i += blockDim.x) d += Q[(int64_t)i * r + j] * Q[(int64_t)i * r + k];
            d = block_sum(d, red);
            for (int i = threadIdx.x; i < n; i += blockDim.x) Q[(int64_t)i * r + k] -= d * Q[(int64_t)i * r + j];
            __syncthreads();
        }
        float q2 = 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) q2 += Q[(int64_t)i * r + k] * Q[(int64_t)i * r + k];
        q2 = block_sum(q2, red);
        const float inv = q2 > 0.f ? 1.f / sqrtf(q2) : 0.f;
        for (int i = threadIdx.x; i < n; i += blockDim.x) Q[(int64_t)i * r + k] *= inv;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(512) k_leverage(lt_samples smp, const int32_t* __restrict__ slice_id, int S, int C,
                                                  const float* __restrict__ G,
                                                  const int64_t* __restrict__ goff2, int64_t gcap, int r, int iters,
                                                  uint64_t seed, float* __restrict__ Qall, float* __restrict__ Yall,
                                                  const int32_t* __restrict__ goff, float* __restrict__ target) {
    __shared__ float red[32];
    if (goff2[S] > gcap) return;
    const int s = blockIdx.x;
    const int ns = smp.ncol[s];
    if (ns == 0) return;
    const int rr = min(r, ns);
    float* Q = Qall + (int64_t)s * C * r;
    float* Y = Yall + (int64_t)s * C * r;
    const float* Gs = G + goff2[s];
    for (int e = threadIdx.x; e < ns * rr; e += blockDim.x) {
        const int c = e / rr, k = e % rr;
        Q[e] = (float)((double)philox((uint32_t)k, (uint32_t)c, slice_key(slice_id, s), kTagLeverage, seed).x *
                           2.3283064365386963e-10 - 0.5);
    }
    __syncthreads();
    mgs_cols(Q, ns, rr, red);
    for (int it = 0; it < iters; ++it) {
        for (int e = threadIdx.x; e < ns * rr; e += blockDim.x) {
            const int i = e / rr, k = e % rr;
            const float* gi = Gs + (int64_t)i * ns;
            float a = 0.f;
            for (int j = 0; j < ns; ++j) a = fmaf(gi[j], Q[(int64_t)j * rr + k], a);
            Y[e] = a;
        }
        __syncthreads();
        for (int e = threadIdx.x; e < ns * rr; e += blockDim.x) Q[e] = Y[e];
        __syncthreads();
        mgs_cols(Q, ns, rr, red);
    }
    float tot = 0.f;
    for (int c = threadIdx.x; c < ns; c += blockDim.x) {
        float l = 0.f;
        for (int k = 0; k < rr; ++k) l += Q[(int64_t)c * rr + k] * Q[(int64_t)c * rr + k];
        Y[c] = l + 1.f / (float)ns;
        tot += Y[c];
    }
    tot = block_sum(tot, red);
    for (int c = threadIdx.x; c < ns; c += blockDim.x) target[goff[s] + c] = Y[c] / tot;
}

bool frame_ok3(const lt_frame* f) { return f && f->slice_off && f->S > 0 && f->S <= 1024 && f->C >= 1 && f->pts; }

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" lt_status lt_proposal_features(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, float* feat,
                                          int32_t* group_off) {
    if (!ctx || !frame_ok3(f) || !smp || !smp->ncol || !smp->key || !smp->val || !smp->n1 || !smp->col_node || !feat ||
        !group_off)
        return lt_fail(ctx, LT_EINVAL, "lt_proposal_features: bad arguments");
    cudaSetDevice(ctx->device);
    lt_status st;
    float* stats = (float*)lt_scratch(ctx, SCR_PROPOSAL, (size_t)f->S * kSliceStats * 4, &st);
    if (!stats) return st;
    k_feat_slice<<<f->S, 256, 0, ctx->stream>>>(*f, *smp, stats);
    LT_LAUNCH_CHECK(ctx, "k_feat_slice");
    k_group_prefix<<<1, 1024, 0, ctx->stream>>>(smp->ncol, f->S, group_off);
    LT_LAUNCH_CHECK(ctx, "k_group_prefix");
    const int64_t warps = (int64_t)f->S * f->C;
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((warps + 7) / 8, 16 * ctx->num_sms));
    k_feat_cols<<<grid, 256, 0, ctx->stream>>>(*f, *smp, stats, group_off, feat);
    LT_LAUNCH_CHECK(ctx, "k_feat_cols");
    return LT_OK;
}

extern "C" lt_status lt_proposal_forward(lt_ctx* ctx, const float* theta, const float* feat, int64_t n_max,
                                         const int32_t* n_dev, float* z) {
    if (!ctx || !theta || !feat || !z || n_max < 0) return lt_fail(ctx, LT_EINVAL, "lt_proposal_forward: bad arguments");
    if (n_max == 0) return LT_OK;
    cudaSetDevice(ctx->device);
    const size_t shm = sizeof(MlpSmem);
    LT_CUDA(ctx, cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_max + TM - 1) / TM, 4 * ctx->num_sms));
    k_mlp_forward<<<grid, 128, shm, ctx->stream>>>(theta, feat, n_max, n_dev, z);
    LT_LAUNCH_CHECK(ctx, "k_mlp_forward");
    return LT_OK;
}

extern "C" lt_status lt_proposal_weights(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp,
                                         const int32_t* group_off, const float* z, float mix, float* w) {
    if (!ctx || !frame_ok3(f) || !smp || !smp->ncol || !smp->g || !group_off || !z || !w || !(mix >= 0.f && mix <= 1.f))
        return lt_fail(ctx, LT_EINVAL, "lt_proposal_weights: bad arguments");
    cudaSetDevice(ctx->device);
    k_mix_weights<<<(f->S + 7) / 8, 256, 0, ctx->stream>>>(*f, *smp, group_off, z, mix, w);
    LT_LAUNCH_CHECK(ctx, "k_mix_weights");
    return LT_OK;
}

extern "C" lt_status lt_slice_matrices(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, float d_min, float* M,
                                       int64_t cap, int64_t* moff) {
    if (!ctx || !frame_ok3(f) || !smp || !smp->ncol || !smp->col_node || !M || !moff || cap < 0)
        return lt_fail(ctx, LT_EINVAL, "lt_slice_matrices: bad arguments");
    if (!ctx->d_cell_off) return lt_fail(ctx, LT_EINVAL, "lt_slice_matrices: no scene uploaded");
    cudaSetDevice(ctx->device);
    k_moff<<<1, 1024, 0, ctx->stream>>>(*f, *smp, moff);
    LT_LAUNCH_CHECK(ctx, "k_moff");
    k_slice_matrix<<<dim3(std::max(1, 4 * ctx->num_sms / f->S), f->S), 256, 0, ctx->stream>>>(
        *f, *smp, ctx->grid, d_min * d_min, moff, cap, M, ctx->d_status);
    LT_LAUNCH_CHECK(ctx, "k_slice_matrix");
    return LT_OK;
}

extern "C" lt_status lt_leverage_targets(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const float* M,
                                         const int64_t* moff, const int32_t* group_off, int32_t r, int32_t iters,
                                         uint64_t seed, float* target) {
    if (!ctx || !frame_ok3(f) || !smp || !smp->ncol || !M || !moff || !group_off || !target || r < 1 || r > 64 ||
        iters < 0)
        return lt_fail(ctx, LT_EINVAL, "lt_leverage_targets: bad arguments");
    cudaSetDevice(ctx->device);
    const int S = f->S, C = f->C;
    // Gram capacity: sum of n'^2 <= S * min(C, 4096)^2 floats is bounded by the
    // largest coarsened cut the slices can have; slices beyond it are skipped
    const int64_t nmax = std::min<int64_t>(C, 4096);
    const int64_t gcap = (int64_t)S * nmax * nmax;
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_PROPOSAL_T,
                                (size_t)gcap * 4 + (size_t)2 * S * C * r * 4 + (size_t)(S + 1) * 8 + 4 * 256, &st);
    if (!p) return st;
    float* G = (float*)p;
    float* Q = (float*)(p + (((size_t)gcap * 4 + 255) & ~(size_t)255));
    float* Y = Q + (size_t)S * C * r;
    int64_t* goff2 = (int64_t*)((char*)Y + (((size_t)S * C * r * 4 + 255) & ~(size_t)255));
    k_goff<<<1, 1024, 0, ctx->stream>>>(*smp, S, goff2);
    LT_LAUNCH_CHECK(ctx, "k_goff");
    const unsigned tiles = (unsigned)((nmax + 31) / 32);
    k_gram<<<dim3(tiles, tiles, S), 256, 0, ctx->stream>>>(*f, *smp, M, moff, goff2, gcap, G);
    LT_LAUNCH_CHECK(ctx, "k_gram");
    k_leverage<<<S, 512, 0, ctx->stream>>>(*smp, f->slice_id, S, C, G, goff2, gcap, r, iters, seed, Q, Y, group_off,
                                           target);
    LT_LAUNCH_CHECK(ctx, "k_leverage");
    return LT_OK;
}

extern "C" lt_status lt_proposal_init(lt_ctx* ctx, uint64_t seed, float* theta) {
    if (!ctx || !theta) return lt_fail(ctx, LT_EINVAL, "lt_proposal_init: bad arguments");
    cudaSetDevice(ctx->device);
    k_mlp_init<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(seed, theta);
    LT_LAUNCH_CHECK(ctx, "k_mlp_init");
    return LT_OK;
}

extern "C" lt_status lt_proposal_grad(lt_ctx* ctx, const float* theta, const float* feat, const float* target,
                                      const int32_t* group_off, int32_t ngroups, int64_t n, float* grad, float* loss) {
    if (!ctx || !theta || !feat || !target || !group_off || !grad || ngroups < 1 || n < 1)
        return lt_fail(ctx, LT_EINVAL, "lt_proposal_grad: bad arguments");
    cudaSetDevice(ctx->device);
    const int nparts = (int)std::min<int64_t>((n + TM - 1) / TM, ctx->num_sms);
    lt_status st;
    char* p = (char*)lt_scratch(ctx, SCR_PROPOSAL_G,
                                (size_t)n * 8 + (size_t)ngroups * 4 + (size_t)nparts * NPAR * 4 + 4 * 256, &st);
    if (!p) return st;
    float* z = (float*)p;
    float* dz = z + n;
    float* gloss = (float*)((char*)p + (((size_t)n * 8 + 255) & ~(size_t)255));
    float* part = (float*)((char*)gloss + (((size_t)ngroups * 4 + 255) & ~(size_t)255));
    lt_status s1 = lt_proposal_forward(ctx, theta, feat, n, nullptr, z);
    if (s1 != LT_OK) return s1;
    k_group_softmax<<<(ngroups + 7) / 8, 256, 0, ctx->stream>>>(z, target, group_off, ngroups, dz, gloss);
    LT_LAUNCH_CHECK(ctx, "k_group_softmax");
    const size_t shm = sizeof(BwdSmem);
    LT_CUDA(ctx, cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    k_mlp_backward<<<nparts, 128, shm, ctx->stream>>>(theta, feat, dz, n, part);
    LT_LAUNCH_CHECK(ctx, "k_mlp_backward");
    k_grad_reduce<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(part, nparts, grad, gloss, ngroups, loss);
    LT_LAUNCH_CHECK(ctx, "k_grad_reduce");
    return LT_OK;
}

extern "C" lt_status lt_proposal_adam(lt_ctx* ctx, float* theta, float* m, float* v, const float* grad, int32_t step,
                                      float lr) {
    if (!ctx || !theta || !m || !v || !grad || step < 1 || !(lr >= 0.f))
        return lt_fail(ctx, LT_EINVAL, "lt_proposal_adam: bad arguments");
    cudaSetDevice(ctx->device);
    k_adam<<<(NPAR + 255) / 256, 256, 0, ctx->stream>>>(theta, m, v, grad, step, lr);
    LT_LAUNCH_CHECK(ctx, "k_adam");
    return LT_OK;
}
