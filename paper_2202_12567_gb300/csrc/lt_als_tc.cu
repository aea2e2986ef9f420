// Masked-ALS half-step on the tensor cores (tcgen05, TMEM) for ranks up to 16.
//
// The completion of Sec. 5 alternates least-squares solves for the rows of U_s and
// of V_s.  For one slice and one side, line i (a row of U for the U-step, a column
// of V for the V-step) needs
//     G_i = sum_j B_ij x_j x_j^T      and      b_i = sum_j A_ij x_j,
// where x_j are the other side's factor rows, B is the slice's 0/1 observation mask
// and A its observed values.  With w_j = the lower triangle of x_j x_j^T packed in
// the order of chol_solve (element (a, c), c <= a, at a (a + 1) / 2 + c), the Grams
// of a tile of lines are the rows of one product  B_tile (lines x K) W (K x NT)
// over the K source lines of the slice, and the right-hand sides the rows of
// A_tile (lines x K) X (K x r): dense contractions with a 0/1 (and a sparse) left
// operand, which the tensor cores run at many times the FP32 FMA rate even though
// most of B is zero at the method's sampling rates.
//
// Precision: fp16 operands, fp32 accumulation.  The mask is exact in fp16.  W, X and
// A are scaled per slice by powers of two into fp16's range and split into two fp16
// parts (v = hi + lo, 22 significant bits), so that
//     B W = B W_hi + B W_lo,     A X = A_hi X_hi + A_hi X_lo + A_lo X_hi
// keep float32-level accuracy (the dropped A_lo X_lo is 2^-22 of a product).
//
// Per lt_complete: k_tc_prefix (tile and block prefixes), k_tc_amax (the value scale
// of each slice), k_tc_vsplit (every observed value as its two fp16 parts, in CSR and
// in CSC order).  Per half-step:
//  * k_tc_xmax: the per-slice largest magnitude of the source factor rows (their scale);
//  * k_tc_image: for every block of 32 source lines, W_hi, W_lo, X_hi and X_lo laid
//    out as the tensor cores read them from shared memory (K-major 8 x 8 core
//    matrices, no swizzle), one contiguous image per block;
//  * k_als_tc: persistent, one CTA per SM: eight builder warps and one MMA warp.  A
//    tile is 256 lines, two M = 128 halves that share each block's image.  For each
//    block of 32 source lines the builders write their lines' rows of the mask and
//    value tiles (from the occupancy bitmap and the split values, loaded ahead) and
//    arrive on the stage's mbarrier; the MMA thread bulk-copies the images two
//    blocks ahead (cp.async.bulk), issues the block's MMAs (tcgen05.mma, accumulators
//    in TMEM) and commits them to the stages' mbarriers, so building, copying and
//    multiplying overlap without a block-wide barrier.  At the end of a tile each
//    builder thread reads its line's Gram and right-hand side from its TMEM lane,
//    adds the ridge lam_rel tr(G) / r, factors by Cholesky in float32 and solves;
//    lines whose pivots fail the check are queued for the float64 pass.
// Every wait is bounded: past the limit the kernel latches LT_ELIMIT, stops issuing,
// waits (bounded) for its copies and MMAs in flight, frees its TMEM and returns.

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "lt_internal.cuh"
#include "lt_omega.cuh"
#include "lt_als_common.cuh"
#include "lt_als_tc.cuh"

using namespace ltk;

namespace {

constexpr int kTcK = 32;                          // source lines per K block
constexpr int kTcM = 128;                         // MMA M (= TMEM lanes)
constexpr int kTcL = 256;                         // lines per tile: two MMA row halves
constexpr int kTcBuild = kTcL / 32;               // builder warps (one thread per line)
constexpr int kTcThreads = kTcL + 32;             // the builders and the MMA warp
constexpr int kTcNA = 2;                          // mask / value stages
constexpr int kTcNI = 4;                          // image stages
constexpr int kTcAhead = 2;                       // image copies run this many blocks ahead
constexpr long long kTcWaitCycles = 4000000000LL; // bound of every wait (about 2 s)

template <int RP>
struct Tc {
    static constexpr int NT = RP * (RP + 1) / 2;          // packed Gram values
    static constexpr int NG = (NT + 15) / 16 * 16;        // MMA N of the Gram (48, 144)
    static constexpr int NB = 16;                         // MMA N of the right-hand side
    static constexpr int BCOL = (NG + 31) / 32 * 32;      // TMEM column of b in a half (64, 160)
    static constexpr int HCOLS = RP == 16 ? 256 : 128;    // TMEM columns of one row half
    static constexpr int TCOLS = 2 * HCOLS;               // TMEM columns allocated
    static constexpr int ATILE = kTcL * kTcK * 2;         // one 256 x 32 fp16 tile (16 KB)
    static constexpr int AHALF = kTcM / 8 * 512;          // byte offset of row 128 in a tile
    static constexpr int ASTAGE = 3 * ATILE;              // mask, value hi, value lo
    static constexpr int WTILE = NG * kTcK * 2;           // one W part
    static constexpr int XTILE = NB * kTcK * 2;           // one X part (1 KB)
    static constexpr int IMG = 2 * WTILE + 2 * XTILE;     // image of one K block
    static constexpr size_t DYN = (size_t)kTcNA * ASTAGE + (size_t)kTcNI * IMG + 1024;
    static_assert(BCOL + NB <= HCOLS, "TMEM allocation too small");
    static_assert(ASTAGE % 1024 == 0 && IMG % 1024 == 0, "stages keep 1 KB alignment");
};

// Byte offset of element (row, k) of a rows x 32 fp16 tile, K-major without swizzle:
// 8 x 8 core matrices of 128 B; the four cores of a row group lie contiguous along K
// (leading byte offset 128) and row groups are 512 B apart (stride byte offset).
__host__ __device__ constexpr int tc_off(int row, int k) {
    return (row >> 3) * 512 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2;
}

// shared-memory matrix descriptor of a tile at shared address `saddr` (no swizzle,
// LBO 128 B, SBO 512 B, descriptor version 1)
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(512 >> 4) << 32) |
           ((uint64_t)1 << 46);
}

// instruction descriptor of kind::f16: fp32 accumulator, fp16 A and B, both K-major,
// M = 128, N = N
template <int N>
__host__ __device__ constexpr uint32_t tc_idesc() {
    static_assert(N % 16 == 0 && N >= 16 && N <= 256, "MMA N for M = 128");
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, int count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the completion of the phase of parity `parity`; false when the bound ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
    const long long t0 = clock64();
    while (!mbar_test(b, parity))
        if (clock64() - t0 > kTcWaitCycles) return false;
    return true;
}

// The same for a whole warp: lane 0 polls, the others wait at the warp barrier.
__device__ __forceinline__ bool mbar_wait_warp(uint64_t* b, uint32_t parity) {
    int ok = 1;
    if ((threadIdx.x & 31) == 0) ok = mbar_wait(b, parity);
    return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// global -> shared bulk copy (sizes and addresses multiples of 16 B), completion
// counted in bytes on `bar`
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

// whole warp: allocate `ncols` TMEM columns, the address goes to *dst
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// whole warp (the allocating one)
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D (TMEM) = A B + (acc ? D : 0), A and B from shared memory (one thread issues)
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

// the mbarrier completes a phase once every MMA this thread issued before has finished
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 16 consecutive 32-bit columns of this thread's TMEM lane (valid after tmem_ld_wait)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// keeps the compiler from moving uses of a loaded register above tmem_ld_wait
__device__ __forceinline__ void reg_pin(uint32_t& x) { asm volatile("" : "+r"(x)::"memory"); }

// v = hi + lo in fp16 (v is in fp16 range after the slice's scaling)
__device__ __forceinline__ void split_half(float v, __half& hi, __half& lo) {
    hi = __float2half_rn(v);
    lo = __float2half_rn(v - __half2float(hi));
}

// 2^e as a float (|e| < 127)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// exponent e with m * 2^e < 2^14 for the largest magnitude m (0 when m = 0)
__device__ __forceinline__ int tc_exp(float m) {
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);  // m = f 2^e, f in [0.5, 1)
    return 14 - e;
}

// -------------------------------------------------------------------- per lt_complete
// One block: the four per-slice prefixes (slices of rank above RP get no tiles and
// no image blocks: the warp-group kernel has them).
__global__ void __launch_bounds__(1024) k_tc_prefix(lt_frame F, lt_samples smp, int R, const int32_t* rk, int RP,
                                                    TcPlan P) {
    __shared__ int32_t ws[32];
    const int S = F.S;
    int32_t carry[4] = {0, 0, 0, 0};
    for (int c0 = 0; c0 < S; c0 += blockDim.x) {
        const int s = c0 + threadIdx.x;
        int32_t v[4] = {0, 0, 0, 0};
        if (s < S && slice_rank(rk, s, R) <= RP) {
            const int ms = F.slice_off[s + 1] - F.slice_off[s], ns = smp.ncol[s];
            v[0] = (ns + kTcK - 1) / kTcK;
            v[1] = (ms + kTcK - 1) / kTcK;
            v[2] = (ms + kTcL - 1) / kTcL;
            v[3] = (ns + kTcL - 1) / kTcL;
        }
        int32_t* out[4] = {P.kbr, P.kbc, P.tr, P.tcn};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            int32_t tot;
            const int32_t pre = block_exclusive_scan<int32_t>(v[k], ws, &tot);
            if (s < S) out[k][s] = carry[k] + pre;
            carry[k] += tot;
        }
    }
    if (threadIdx.x == 0) {
        P.kbr[S] = carry[0];
        P.kbc[S] = carry[1];
        P.tr[S] = carry[2];
        P.tcn[S] = carry[3];
    }
}

// The largest magnitude of each slice's observed values (float bits, atomicMax on
// non-negative floats orders like the values): blockIdx.y = slice.
__global__ void __launch_bounds__(256) k_tc_amax(lt_samples smp, int32_t* __restrict__ amax) {
    __shared__ float red[8];
    const int s = blockIdx.y;
    const float* v = smp.val + smp.off[s];
    const int n = smp.cnt[s];
    float m = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmaxf(m, fabsf(v[i]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
        if (m > 0.f) atomicMax(amax + s, __float_as_int(m));
    }
}

// Every observed value v of slice s as its two fp16 parts of v 2^ea (hi in the low
// half-word, lo in the high one), at its CSR position (vr) and its CSC position (vc).
__global__ void __launch_bounds__(256) k_tc_vsplit(lt_samples smp, Omega om, const int32_t* __restrict__ amax,
                                                   uint32_t* __restrict__ vr, uint32_t* __restrict__ vc) {
    const int s = blockIdx.y;
    const int64_t o = smp.off[s];
    const int n = smp.cnt[s];
    const float sa = pow2f(tc_exp(__int_as_float(amax[s])));
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        __half h, l;
        split_half(om.cval[o + i] * sa, h, l);
        vr[o + i] = (uint32_t)__half_as_ushort(h) | ((uint32_t)__half_as_ushort(l) << 16);
        split_half(om.rval[o + i] * sa, h, l);
        vc[o + i] = (uint32_t)__half_as_ushort(h) | ((uint32_t)__half_as_ushort(l) << 16);
    }
}

// ---------------------------------------------------------------------- per half-step
// The largest magnitude of each slice's source factor rows (the first r components),
// as float bits into xmax[s]: blockIdx.y = slice.
__global__ void __launch_bounds__(256) k_tc_xmax(lt_frame F, lt_samples smp, int R, const int32_t* rk, int RP,
                                                 bool rows_side, const float* __restrict__ Fin,
                                                 int32_t* __restrict__ xmax) {
    __shared__ float red[8];
    const int s = blockIdx.y;
    const int r = slice_rank(rk, s, R);
    const int row0 = F.slice_off[s];
    const int nsrc = rows_side ? smp.ncol[s] : F.slice_off[s + 1] - row0;
    const float* src = rows_side ? Fin + (int64_t)s * F.C * R : Fin + (int64_t)row0 * R;
    float m = 0.f;
    if (r <= RP)
        for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nsrc; j += gridDim.x * blockDim.x)
            for (int c = 0; c < r; ++c) m = fmaxf(m, fabsf(src[(int64_t)j * R + c]));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 0; w < 8; ++w) m = fmaxf(m, red[w]);
        if (m > 0.f) atomicMax(xmax + s, __float_as_int(m));
    }
}

// Packed lower-triangle position n -> (a, c), c <= a, n = a (a + 1) / 2 + c.
__device__ __forceinline__ void tri_pos(int n, int& a, int& c) {
    a = 0;
    while ((a + 1) * (a + 2) / 2 <= n) ++a;
    c = n - a * (a + 1) / 2;
}

// Images of the source factor rows: per block of 32 source lines of a slice, the
// tiles W_hi, W_lo (NG x 32: row n = packed (a, c), value x_a x_c 2^ew) and X_hi,
// X_lo (16 x 32: row c, value x_c 2^ex), each in the core-matrix layout of tc_off.
// A thread writes whole 8 x 8 cores (16 B a row); lines past the slice are zero.
template <int RP>
__global__ void __launch_bounds__(128) k_tc_image(lt_frame F, lt_samples smp, int R, const int32_t* rk,
                                                  bool rows_side, const float* __restrict__ Fin, TcPlan P,
                                                  const int32_t* __restrict__ xmax) {
    using T = Tc<RP>;
    __shared__ float xs[kTcK][RP + 1];
    const int S = F.S;
    const int32_t* kp = rows_side ? P.kbr : P.kbc;
    const int total = kp[S];
    if ((int64_t)total > P.img_cap) {  // images beyond the scratch: nothing is written or read
        if (blockIdx.x == 0 && threadIdx.x == 0) latch(P.status, LT_ELIMIT);
        return;
    }
    constexpr int WCORES = T::NG / 8 * 4, XCORES = T::NB / 8 * 4;
    for (int blk = blockIdx.x; blk < total; blk += gridDim.x) {
        int lo = 0, hi = S;  // the slice s with kp[s] <= blk < kp[s + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (kp[mid] <= blk) lo = mid; else hi = mid;
        }
        const int s = lo, kb = blk - kp[s];
        const int r = slice_rank(rk, s, R);
        const int row0 = F.slice_off[s];
        const int nsrc = rows_side ? smp.ncol[s] : F.slice_off[s + 1] - row0;
        const float* src = rows_side ? Fin + (int64_t)s * F.C * R : Fin + (int64_t)row0 * R;
        __syncthreads();  // the previous block is done with xs
        for (int i = threadIdx.x; i < kTcK * RP; i += blockDim.x) {
            const int k = i / RP, c = i % RP, j = kb * kTcK + k;
            xs[k][c] = (j < nsrc && c < r) ? src[(int64_t)j * R + c] : 0.f;
        }
        __syncthreads();
        const float xm = __int_as_float(xmax[s]);
        const float sw = pow2f(tc_exp(xm * xm)), sx = pow2f(tc_exp(xm));
        unsigned char* out = P.img + (int64_t)blk * T::IMG;
        for (int q = threadIdx.x; q < WCORES + XCORES; q += blockDim.x) {
            const bool w = q < WCORES;
            const int qq = w ? q : q - WCORES;
            const int rg = qq >> 2, kc = qq & 3;
            unsigned char* thi = out + (w ? 0 : 2 * T::WTILE);
            unsigned char* tlo = thi + (w ? T::WTILE : T::XTILE);
#pragma unroll 1
            for (int rr = 0; rr < 8; ++rr) {
                const int n = rg * 8 + rr;
                int a = 0, c = 0;
                bool on;
                if (w) {
                    on = n < T::NT;
                    if (on) tri_pos(n, a, c);
                } else {
                    on = n < RP;
                    a = n;
                }
                __align__(16) __half h[8], l[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const int k = kc * 8 + e;
                    float v = 0.f;
                    if (on) v = w ? xs[k][a] * xs[k][c] * sw : xs[k][a] * sx;
                    split_half(v, h[e], l[e]);
                }
                const int o = tc_off(n, kc * 8);
                *reinterpret_cast<uint4*>(thi + o) = *reinterpret_cast<const uint4*>(h);
                *reinterpret_cast<uint4*>(tlo + o) = *reinterpret_cast<const uint4*>(l);
            }
        }
    }
}

// ------------------------------------------------------------------- the half-step
// Persistent, one CTA per SM: eight builder warps (256 threads) and one MMA warp.
// Tiles of 256 lines (all slices, U-step rows or V-step columns) come from a
// counter.  Builder thread t owns line t of the tile, row t of the mask and value
// tiles and TMEM lane 32 (w mod 4) + (t mod 32) of row half h = w / 4 (w = t / 32):
// the two halves are two M = 128 MMAs per K step that share the block's image.
// Shared memory: kTcNA stages of [mask | value hi | value lo] (256 x 32 fp16 each)
// and kTcNI image stages.  mbarriers: a_full[i] (the builder warps wrote stage i),
// a_free[i] and img_free[j] (the MMAs that read the stage are done: tcgen05.commit),
// img_full[j] (the image copy landed).
template <int RP>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_als_tc(lt_frame F, lt_samples smp, Omega om, int R, const int32_t* __restrict__ rk, bool rows_side,
             const float* __restrict__ Fin, float* __restrict__ Fout, float lam_rel, TcPlan P,
             const int32_t* __restrict__ xmax, int32_t* __restrict__ tile_ctr, TcQueue q, float* __restrict__ gram) {
    using T = Tc<RP>;
    extern __shared__ unsigned char tc_dyn[];
    __shared__ __align__(8) uint64_t a_full[kTcNA], a_free[kTcNA], img_full[kTcNI], img_free[kTcNI];
    __shared__ uint32_t s_tmem;
    __shared__ int s_tile, s_abort;
    __shared__ uint4 s_mask8[256];  // byte b -> eight fp16: 1.0 (0x3C00) where bit k of b is set
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool builder = warp < kTcBuild;
    const bool mma_thread = warp == kTcBuild && lane == 0;
    volatile int* abort_flag = &s_abort;
    unsigned char* sm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(tc_dyn) + 1023) & ~(uintptr_t)1023);
    unsigned char* simg = sm + kTcNA * T::ASTAGE;
    const int S = F.S;
    const int32_t* tp = rows_side ? P.tr : P.tcn;
    const int32_t* kp = rows_side ? P.kbr : P.kbc;
    const int ntiles = tp[S];
    if (tid == 0) {
        for (int i = 0; i < kTcNA; ++i) {
            mbar_init(&a_full[i], kTcBuild);
            mbar_init(&a_free[i], 1);
        }
        for (int i = 0; i < kTcNI; ++i) {
            mbar_init(&img_full[i], 1);
            mbar_init(&img_free[i], 1);
        }
        s_abort = (int64_t)kp[S] > P.img_cap;  // no images were written (latched by k_tc_image)
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        fence_async_smem();
    }
    for (int b = tid; b < 256; b += kTcThreads) {
        uint32_t w4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h)
            w4[h] = (((b >> (2 * h)) & 1) ? 0x3C00u : 0u) | (((b >> (2 * h + 1)) & 1) ? 0x3C000000u : 0u);
        s_mask8[b] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
    if (warp == kTcBuild) tmem_alloc(&s_tmem, T::TCOLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = s_tmem;
    const int rowoff = tc_off(tid & (kTcL - 1), 0);
    // Blocks of this CTA so far (the builders and the MMA thread count alike: block g
    // uses mask stage g % kTcNA and image stage g % kTcNI).  The MMA thread also counts
    // the copies it issued, the copies it saw land and the blocks it committed.
    uint32_t g = 0;
    uint32_t copies = 0, fulls = 0, commits = 0;
    auto issue_copy = [&](const unsigned char* img, int kb, uint32_t gi) {  // MMA thread
        const uint32_t is = gi % kTcNI, iu = gi / kTcNI;
        if (iu > 0 && !mbar_wait(&img_free[is], (iu - 1) & 1u)) {
            latch(P.status, LT_ELIMIT);
            *abort_flag = 1;
            return;
        }
        mbar_expect_tx(&img_full[is], (uint32_t)T::IMG);
        bulk_g2s(simg + is * T::IMG, img + (int64_t)kb * T::IMG, (uint32_t)T::IMG, &img_full[is]);
        ++copies;
    };
    for (;;) {
        if (tid == 0) s_tile = *abort_flag ? ntiles : atomicAdd(tile_ctr, 1);
        __syncthreads();
        const int tile = s_tile;
        if (tile >= ntiles) break;
        int lo = 0, hi = S;  // the slice s with tp[s] <= tile < tp[s + 1]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (tp[mid] <= tile) lo = mid; else hi = mid;
        }
        const int s = lo;
        const int row0 = F.slice_off[s], ms = F.slice_off[s + 1] - row0, ns = smp.ncol[s];
        const int nlines = rows_side ? ms : ns, nsrc = rows_side ? ns : ms;
        const int nkb = (nsrc + kTcK - 1) / kTcK;
        const unsigned char* img = P.img + (int64_t)kp[s] * T::IMG;
        const int l = (tile - tp[s]) * kTcL + (tid & (kTcL - 1));
        const bool live = builder && l < nlines;
        if (builder) {
            // The line's occupancy bits: word kb holds its entries among source lines
            // [32 kb, 32 kb + 32), whose split values are the next popc(word) of its CSR /
            // CSC run (both in source-line order).  Words are loaded two blocks ahead,
            // values (up to 8) one block ahead.
            int p = 0;
            const uint32_t* wrow = nullptr;
            if (live) {
                p = rows_side ? om.rp[row0 + s + l] : om.cp[(int64_t)s * (F.C + 1) + l];
                wrow = rows_side ? om.bm + (int64_t)s * om.bm_stride + (int64_t)l * nkb
                                 : om.bt + (int64_t)s * om.bt_stride + (int64_t)l * nkb;
            }
            const uint32_t* vs = (rows_side ? P.vr : P.vc) + smp.off[s];
            uint32_t wcur = (live && nkb > 0) ? __ldg(wrow) : 0u;
            uint32_t wnext = (live && nkb > 1) ? __ldg(wrow + 1) : 0u;
            uint32_t pv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) pv[i] = i < __popc(wcur) ? __ldg(vs + p + i) : 0u;
            for (int kb = 0; kb < nkb; ++kb) {
                if (*abort_flag) break;
                const uint32_t as = g % kTcNA, au = g / kTcNA;
                unsigned char* am = sm + as * T::ASTAGE;
                unsigned char* ah = am + T::ATILE;
                unsigned char* al = am + 2 * T::ATILE;
                const uint32_t w = wcur;
                const int cnt = __popc(w);
                uint32_t v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) v[i] = pv[i];
                wcur = wnext;  // prefetch: the values of block kb + 1, the word of block kb + 2
                wnext = (live && kb + 2 < nkb) ? __ldg(wrow + kb + 2) : 0u;
                {
                    const int cn = __popc(wcur);
#pragma unroll
                    for (int i = 0; i < 8; ++i) pv[i] = i < cn ? __ldg(vs + p + cnt + i) : 0u;
                }
                // the stage is free once the MMAs of its previous use are done
                if (au > 0 && !mbar_wait_warp(&a_free[as], (au - 1) & 1u)) {
                    latch(P.status, LT_ELIMIT);
                    *abort_flag = 1;
                    break;
                }
#pragma unroll
                for (int kc = 0; kc < 4; ++kc) {  // mask: fp16 1.0 where the bit is set; values: 0
                    *reinterpret_cast<uint4*>(am + rowoff + kc * 128) = s_mask8[(w >> (8 * kc)) & 255u];
                    *reinterpret_cast<uint4*>(ah + rowoff + kc * 128) = make_uint4(0u, 0u, 0u, 0u);
                    *reinterpret_cast<uint4*>(al + rowoff + kc * 128) = make_uint4(0u, 0u, 0u, 0u);
                }
                uint32_t ww = w;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (i < cnt) {
                        const int k = __ffs(ww) - 1;
                        ww &= ww - 1u;
                        const int off = rowoff + (k >> 3) * 128 + (k & 7) * 2;
                        *reinterpret_cast<uint16_t*>(ah + off) = (uint16_t)(v[i] & 0xffffu);
                        *reinterpret_cast<uint16_t*>(al + off) = (uint16_t)(v[i] >> 16);
                    }
                }
                for (int i = 8; i < cnt; ++i) {  // a block with more than 8 entries of the line
                    const int k = __ffs(ww) - 1;
                    ww &= ww - 1u;
                    const uint32_t x = __ldg(vs + p + i);
                    const int off = rowoff + (k >> 3) * 128 + (k & 7) * 2;
                    *reinterpret_cast<uint16_t*>(ah + off) = (uint16_t)(x & 0xffffu);
                    *reinterpret_cast<uint16_t*>(al + off) = (uint16_t)(x >> 16);
                }
                p += cnt;
                fence_async_smem();  // the rows written by the threads, for the tensor cores
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[as]);
                ++g;
            }
        } else if (mma_thread) {
            for (int k = 0; k < kTcAhead && k < nkb; ++k) issue_copy(img, k, g + k);
            for (int kb = 0; kb < nkb; ++kb) {
                if (*abort_flag) break;
                const uint32_t as = g % kTcNA, au = g / kTcNA, is = g % kTcNI, iu = g / kTcNI;
                if (!mbar_wait(&a_full[as], au & 1u)) {
                    latch(P.status, LT_ELIMIT);
                    *abort_flag = 1;
                    break;
                }
                if (!mbar_wait(&img_full[is], iu & 1u)) {
                    latch(P.status, LT_ELIMIT);
                    *abort_flag = 1;
                    break;
                }
                ++fulls;
                tc_fence_after();
                const uint32_t sa = smem_u32(sm + as * T::ASTAGE), sw = smem_u32(simg + is * T::IMG);
#pragma unroll
                for (int ks = 0; ks < kTcK / 16; ++ks) {
                    const uint32_t ko = ks * 256;  // 16 K = two core matrices
                    const uint32_t acc = (kb > 0 || ks > 0) ? 1u : 0u;
                    const uint64_t wh = tc_desc(sw + ko), wl = tc_desc(sw + T::WTILE + ko);
                    const uint64_t xh = tc_desc(sw + 2 * T::WTILE + ko), xl = tc_desc(sw + 2 * T::WTILE + T::XTILE + ko);
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint32_t ho = h * T::AHALF + ko, d = tm + h * T::HCOLS;
                        const uint64_t am = tc_desc(sa + ho), ah = tc_desc(sa + T::ATILE + ho),
                                       al = tc_desc(sa + 2 * T::ATILE + ho);
                        tc_mma(d, am, wh, tc_idesc<T::NG>(), acc);
                        tc_mma(d, am, wl, tc_idesc<T::NG>(), 1u);
                        tc_mma(d + T::BCOL, ah, xh, tc_idesc<T::NB>(), acc);
                        tc_mma(d + T::BCOL, ah, xl, tc_idesc<T::NB>(), 1u);
                        tc_mma(d + T::BCOL, al, xh, tc_idesc<T::NB>(), 1u);
                    }
                }
                tc_commit(&a_free[as]);
                tc_commit(&img_free[is]);
                ++commits;
                if (kb + kTcAhead < nkb) issue_copy(img, kb + kTcAhead, g + kTcAhead);
                ++g;
            }
        }
        __syncthreads();  // both roles are through the tile's blocks (or stopped)
        if (*abort_flag) break;
        // ---- epilogue (builders): this line's Gram and right-hand side from TMEM, the solve
        if (builder) {
            const int half = warp >> 2;
            const uint32_t tl = tm + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * T::HCOLS);
            uint32_t rg[T::NG / 16][16], rb[16];
            if (nkb > 0) {
                const uint32_t last = g - 1;  // its commit covers every MMA of the tile
                if (!mbar_wait_warp(&a_free[last % kTcNA], (last / kTcNA) & 1u)) {
                    latch(P.status, LT_ELIMIT);
                    *abort_flag = 1;
                }
                tc_fence_after();
#pragma unroll
                for (int c = 0; c < T::NG / 16; ++c) tmem_ld16(tl + c * 16, rg[c]);
                tmem_ld16(tl + T::BCOL, rb);
                tmem_ld_wait();
#pragma unroll
                for (int c = 0; c < T::NG / 16; ++c)
#pragma unroll
                    for (int i = 0; i < 16; ++i) reg_pin(rg[c][i]);
#pragma unroll
                for (int i = 0; i < 16; ++i) reg_pin(rb[i]);
            } else {
#pragma unroll
                for (int c = 0; c < T::NG / 16; ++c)
#pragma unroll
                    for (int i = 0; i < 16; ++i) rg[c][i] = 0u;
#pragma unroll
                for (int i = 0; i < 16; ++i) rb[i] = 0u;
            }
            if (live && !*abort_flag) {
                const int r = slice_rank(rk, s, R);
                const float xm = __int_as_float(xmax[s]), am_ = __int_as_float(P.amax[s]);
                const float uw = pow2f(-tc_exp(xm * xm)), ub = pow2f(-tc_exp(xm) - tc_exp(am_));
                const int64_t line = rows_side ? (int64_t)(row0 + l) : (int64_t)s * F.C + l;
                float a[T::NT], b[RP];
#pragma unroll
                for (int i = 0; i < T::NT; ++i) a[i] = __uint_as_float(rg[i / 16][i % 16]) * uw;
#pragma unroll
                for (int i = 0; i < RP; ++i) b[i] = __uint_as_float(rb[i]) * ub;
                if (gram) {  // the contraction alone, for checks: packed Gram of rank R, then b
                    const int nt = R * (R + 1) / 2;
                    float* d = gram + line * (nt + R);
#pragma unroll
                    for (int i = 0; i < T::NT; ++i)
                        if (i < nt) d[i] = a[i];
#pragma unroll
                    for (int i = 0; i < RP; ++i)
                        if (i < R) d[nt + i] = b[i];
                } else {
                    const int64_t dst = line * R;
                    for (int i = r; i < R; ++i) Fout[dst + i] = 0.f;  // components beyond the slice's rank
                    if (chol_solve<RP, float>(a, b, r, lam_rel, true)) {
#pragma unroll
                        for (int i = 0; i < RP; ++i)
                            if (i < r) Fout[dst + i] = b[i];
                    } else {  // rare: the float64 pass solves it again from the CSR / CSC entries
                        const int qs = atomicAdd(q.count, 1);
                        if (qs >= q.cap) {
                            latch(q.status, LT_ELIMIT);
                        } else {
                            const int32_t* ptr = rows_side ? om.rp + row0 + s : om.cp + (int64_t)s * (F.C + 1);
                            const int pb = ptr[l], pe = ptr[l + 1];
                            q.dst[qs] = dst;
                            q.slot[qs] = smp.off[s] + pb;
                            q.src[qs] = rows_side ? (int64_t)s * F.C * R : (int64_t)row0 * R;
                            q.len[qs] = pe - pb;
                            q.grp[qs] = 0;
                            q.rank[qs] = r;
                        }
                    }
                }
            }
        }
        tc_fence_before();
        __syncthreads();  // every warp has read TMEM before the next tile's MMAs
    }
    // ---- teardown: nothing of this CTA may be in flight when its TMEM is freed
    if (mma_thread) {
        for (uint32_t k = fulls; k < copies; ++k) mbar_wait(&img_full[k % kTcNI], (k / kTcNI) & 1u);
        if (commits > 0) mbar_wait(&a_free[(commits - 1) % kTcNA], ((commits - 1) / kTcNA) & 1u);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kTcBuild) tmem_free(tm, T::TCOLS);
}

}  // namespace

namespace ltk {

lt_status als_tc_plan(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, int64_t E, int R,
                      const int32_t* rk, int RP, int steps, TcPlan* P) {
    const int S = f->S;
    lt_status st;
    const int ns = std::max(steps, 1);
    const size_t n32 = (size_t)4 * (S + 1) + (size_t)S + (size_t)ns * S + (size_t)ns;
    int32_t* pp = (int32_t*)lt_scratch(ctx, SCR_TC_PLAN, n32 * 4 + 256, &st);
    if (!pp) return st;
    P->kbr = pp;
    P->kbc = P->kbr + (S + 1);
    P->tr = P->kbc + (S + 1);
    P->tcn = P->tr + (S + 1);
    P->amax = P->tcn + (S + 1);
    P->xmax = P->amax + S;
    P->ctr = P->xmax + (size_t)ns * S;
    P->RP = RP;
    P->status = ctx->d_status;
    // image blocks: U-step sources are the n'_s <= C columns of each slice, V-step
    // sources the rows (sum over slices of ceil(m'_s / 32) <= m / 32 + S)
    const int64_t cap = std::max<int64_t>((int64_t)S * ((f->C + kTcK - 1) / kTcK), (f->m + kTcK - 1) / kTcK + S);
    const int64_t img_bytes = RP == 8 ? Tc<8>::IMG : Tc<16>::IMG;
    // one scratch slot: the images, then the split values in CSR and in CSC order
    const size_t img_total = ((size_t)(cap * img_bytes) + 255) & ~(size_t)255;
    const size_t v_total = ((size_t)std::max<int64_t>(E, 1) * 4 + 255) & ~(size_t)255;
    P->img = (unsigned char*)lt_scratch(ctx, SCR_TC_IMG, img_total + 2 * v_total, &st);
    if (!P->img) return st;
    P->img_cap = cap;
    P->vr = (uint32_t*)(P->img + img_total);
    P->vc = (uint32_t*)(P->img + img_total + v_total);
    // amax, xmax and the tile counters start at zero
    LT_CUDA(ctx, cudaMemsetAsync(P->amax, 0, ((size_t)S + (size_t)ns * S + ns) * 4, ctx->stream));
    k_tc_prefix<<<1, 1024, 0, ctx->stream>>>(*f, *smp, R, rk, RP, *P);
    LT_LAUNCH_CHECK(ctx, "k_tc_prefix");
    k_tc_amax<<<dim3(16, S), 256, 0, ctx->stream>>>(*smp, P->amax);
    LT_LAUNCH_CHECK(ctx, "k_tc_amax");
    k_tc_vsplit<<<dim3(16, S), 256, 0, ctx->stream>>>(*smp, om, P->amax, P->vr, P->vc);
    LT_LAUNCH_CHECK(ctx, "k_tc_vsplit");
    return LT_OK;
}

template <int RP>
static lt_status tc_half(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, int R,
                         const int32_t* rk, bool rows_side, const float* fin, float* fout, float lam_rel,
                         const TcPlan& P, int step, const TcQueue& q, float* gram) {
    const int nsm = ctx->num_sms;
    int32_t* xmax = P.xmax + (size_t)step * f->S;
    k_tc_xmax<<<dim3(8, f->S), 256, 0, ctx->stream>>>(*f, *smp, R, rk, RP, rows_side, fin, xmax);
    LT_LAUNCH_CHECK(ctx, "k_tc_xmax");
    k_tc_image<RP><<<4 * nsm, 128, 0, ctx->stream>>>(*f, *smp, R, rk, rows_side, fin, P, xmax);
    LT_LAUNCH_CHECK(ctx, "k_tc_image");
    const size_t dyn = Tc<RP>::DYN;
    LT_CUDA(ctx, cudaFuncSetAttribute(k_als_tc<RP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    k_als_tc<RP><<<nsm, kTcThreads, dyn, ctx->stream>>>(*f, *smp, om, R, rk, rows_side, fin, fout, lam_rel, P,
                                                           xmax, P.ctr + step, q, gram);
    LT_LAUNCH_CHECK(ctx, "k_als_tc");
    return LT_OK;
}

lt_status als_tc_half(lt_ctx* ctx, const lt_frame* f, const lt_samples* smp, const Omega& om, int R,
                      const int32_t* rk, bool rows_side, const float* fin, float* fout, float lam_rel,
                      const TcPlan& plan, int step, const TcQueue& q, float* gram) {
    if (plan.RP == 8) return tc_half<8>(ctx, f, smp, om, R, rk, rows_side, fin, fout, lam_rel, plan, step, q, gram);
    return tc_half<16>(ctx, f, smp, om, R, rk, rows_side, fin, fout, lam_rel, plan, step, q, gram);
}

}  // namespace ltk
