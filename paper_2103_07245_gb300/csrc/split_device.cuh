// Operand splitting shared by the tcgen05 paths (kernels_tc.cu, kernels_tc_list.cu).
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace pbq {

// ---------------------------------------------------------------------------
// Operand preparation: hi/lo splits (row-major and transposed) into BF16
// (hi = RN_bf16(x), lo = RN_bf16(x - hi)) or TF32 held in FP32
// (hi = RN_tf32(x), lo = RN_tf32(x - hi), rounding by cvt.rna.tf32).
// ---------------------------------------------------------------------------
// Splits are formed in the input's own precision: for x in FP32, hi = RN(x)
// and x - hi are exact in FP32 (no FP64 work, which GB300 runs at a small
// fraction of the FP32 rate); an FP64 input (the panels, or an FP64 A) is
// split in FP64 so that hi = RN(x) is the correctly rounded value of x.
struct SplitBf16 {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ T rn(float x) { return __float2bfloat16_rn(x); }
    static __device__ __forceinline__ T rn(double x) { return __double2bfloat16(x); }
    static __device__ __forceinline__ float back(T h) { return __bfloat162float(h); }
    static __device__ __forceinline__ T zero() { return __float2bfloat16_rn(0.f); }
};
struct SplitTf32 {
    using T = float;
    static __device__ __forceinline__ T rn(float x) {
        uint32_t r;
        asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
        return __uint_as_float(r);
    }
    // hi = RNA_tf32(RN_fp32(x)): the split needs hi + lo to carry x to about
    // 2^-22 relative, which this two-step rounding provides
    static __device__ __forceinline__ T rn(double x) { return rn((float)x); }
    static __device__ __forceinline__ float back(T h) { return h; }
    static __device__ __forceinline__ T zero() { return 0.f; }
};

// One 64 x 64 tile (rows r0.., columns c0..) of A into hi / lo (row-major, ld
// ldh) and, when thi is set, A^T into thi / tlo (ld ldt), by 256 threads.  A
// whole tile with vec_ok: a thread converts 16 consecutive elements of a row
// (16-byte vector loads and stores) and writes 16 consecutive elements of a
// transposed row from shared memory.  Otherwise (a partial tile, or pointers
// or leading dimensions that are not 16-byte multiples) lanes run along the
// columns, then along the rows for the transposed write, with scalar
// accesses that stay coalesced (shared memory then viewed with row stride
// 65, free of bank conflicts both ways).  Ends with the block synchronised,
// so the shared arrays can take the next tile.
template <typename Tin, typename SP>
__device__ __forceinline__ void split_tile64(int64_t r0, int64_t c0, int64_t m, int64_t n, const Tin* __restrict__ A,
                                             int64_t lda, typename SP::T* __restrict__ hi,
                                             typename SP::T* __restrict__ lo, int64_t ldh,
                                             typename SP::T* __restrict__ thi, typename SP::T* __restrict__ tlo,
                                             int64_t ldt, int vec_ok, typename SP::T (*sh)[64 + 16 / sizeof(typename SP::T)],
                                             typename SP::T (*sl)[64 + 16 / sizeof(typename SP::T)]) {
    using T = typename SP::T;
    const int tid = threadIdx.x, rr = tid >> 2, cq = (tid & 3) * 16;
    const bool full = vec_ok && r0 + 64 <= m && c0 + 64 <= n;
    if (!full) {
        T* shs = &sh[0][0];   // [64][65] views of the same storage (64 x 65 <= 64 x (64 + PAD))
        T* sls = &sl[0][0];
        const int cc = tid & 63, rq = tid >> 6;   // lane along the columns; 4 groups of 16 rows
        const int64_t c = c0 + cc;
        const Tin* ap = A + (r0 + rq) * lda + c;
        const int64_t ho = (r0 + rq) * ldh + c;
        Tin xs[16];   // all 16 loads in flight before any use
#pragma unroll
        for (int k = 0; k < 16; ++k) xs[k] = (r0 + rq + 4 * k < m && c < n) ? ap[(int64_t)(4 * k) * lda] : (Tin)0;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int rl = rq + 4 * k;
            const bool in = r0 + rl < m && c < n;
            const Tin xv = xs[k];
            const T hv = SP::rn(xv);
            const T lv = SP::rn(xv - (Tin)SP::back(hv));
            if (in) {
                hi[ho + (int64_t)(4 * k) * ldh] = hv;
                if (lo) lo[ho + (int64_t)(4 * k) * ldh] = lv;
            }
            if (thi) {
                shs[cc * 65 + rl] = hv;
                sls[cc * 65 + rl] = lv;
            }
        }
        if (!thi) return;   // uniform over the block: no shared memory was used
        __syncthreads();
        // transposed: rows c0 + rq + 4k of A^T, column r0 + cc (the lane)
        const int64_t rt = r0 + cc;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int cl = rq + 4 * k;
            const int64_t ct = c0 + cl;
            if (ct < n && rt < m) {
                thi[ct * ldt + rt] = shs[cl * 65 + cc];
                if (tlo) tlo[ct * ldt + rt] = sls[cl * 65 + cc];
            }
        }
        __syncthreads();
        return;
    }
    const int64_t r = r0 + rr;
    __align__(16) T h[16];
    __align__(16) T lw[16];
    Tin x[16];
    {
        const Tin* src = A + r * lda + c0 + cq;
        if (sizeof(Tin) == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float4 v = ((const float4*)src)[q];
                x[4 * q] = (Tin)v.x; x[4 * q + 1] = (Tin)v.y; x[4 * q + 2] = (Tin)v.z; x[4 * q + 3] = (Tin)v.w;
            }
        } else {
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const double2 v = ((const double2*)src)[q];
                x[2 * q] = v.x; x[2 * q + 1] = v.y;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        h[k] = SP::rn(x[k]);
        lw[k] = SP::rn(x[k] - (Tin)SP::back(h[k]));
    }
    constexpr int NV = 16 * (int)sizeof(T) / 16;   // 16-byte vectors per 16 elements
    {
        uint4* dh = (uint4*)(hi + r * ldh + c0 + cq);
#pragma unroll
        for (int q = 0; q < NV; ++q) dh[q] = ((const uint4*)h)[q];
        if (lo) {
            uint4* dl = (uint4*)(lo + r * ldh + c0 + cq);
#pragma unroll
            for (int q = 0; q < NV; ++q) dl[q] = ((const uint4*)lw)[q];
        }
    }
    if (!thi) return;   // uniform over the block: no shared memory was used
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        sh[cq + k][rr] = h[k];
        sl[cq + k][rr] = lw[k];
    }
    __syncthreads();
    // transposed: row c0 + rr of A^T, columns r0 + cq .. r0 + cq + 15
    const int64_t ct = c0 + rr;
    {
        uint4* dh = (uint4*)(thi + ct * ldt + r0 + cq);
#pragma unroll
        for (int q = 0; q < NV; ++q) dh[q] = ((const uint4*)&sh[rr][cq])[q];
        if (tlo) {
            uint4* dl = (uint4*)(tlo + ct * ldt + r0 + cq);
#pragma unroll
            for (int q = 0; q < NV; ++q) dl[q] = ((const uint4*)&sl[rr][cq])[q];
        }
    }
    __syncthreads();
}

}  // namespace pbq
