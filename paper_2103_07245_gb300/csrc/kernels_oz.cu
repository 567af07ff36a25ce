// FP64-accurate products on the BF16 tensor cores by exact integer digits
// (the error-free splitting of Ozaki, Ogita, Oishi & Rump, Numer. Algorithms
// 2012, with eight balanced base-128 digits held in BF16 and exact FP32 sums).
// They serve the products of Algorithm 3 that must carry FP64 accuracy: the
// Grams of CholeskyQR (the orth of Eq. 4), R = Q^T D (Eq. 6) and, in the
// emulated-FP64 mode, the products with A and A^T (Eqs. 3 and 5).
//
// Digits.  Row i of an operand X (R x K) gets the exponent e_i with
// |X[i][k]| < 2^(e_i - 1) for every k.  F = X[i][k] 2^(56 - e_i), rounded to
// the nearest integer (|F| < 2^55), is written in balanced base 128,
// F = sum_{s<8} x_s 128^(7-s) with |x_s| <= 64: each digit is an integer that
// BF16 holds exactly, and X[i][k] = 2^(e_i - 56) F up to 2^(e_i - 57).  A row
// that holds Inf or NaN has the exponent field 2047 and yields NaN products.
//
// Product.  C[i][j] = sum_k X[i][k] Y[j][k] = 2^(e_i + f_j - 112)
// sum_{s,t} 128^(14 - s - t) I_st with I_st = sum_k x_s[i][k] y_t[j][k].
// The digit products with s + t <= 7 are kept (36 of 64; the rest weigh
// below 2^-55 of 2^(e_i + f_j) per term).  Level lam = s + t gathers its
// digit products in one TMEM accumulator (48 columns); over one 128-deep
// window |I_lam| <= 8 * 128 * 64^2 = 2^22, so the tensor pipe's FP32 sums
// are exact integers whatever its rounding.  After every window the epilogue
// adds the eight level sums into two 64-bit accumulators per element,
// hi = sum_{lam<4} I_lam 128^(3-lam) and lo = sum_{lam>=4} I_lam 128^(7-lam),
// and at the end of a segment writes the FP64 partial
// (2^28 hi + lo) 2^(e_i + f_j - 63), rounded once to FP64 with integer
// operations.  A CTA that ran the whole contraction of a tile writes C;
// otherwise each epilogue warp adds its 32 x 16 slice of exact int64 sums
// into the tile's accumulator with 64-bit integer reductions and counts in on
// a per-slice counter, and the last contributor reads the accumulator once
// (the sum is exact, so the result does not depend on the split or the
// order), writes C, and clears the accumulator and the counter.
//
// MMAs.  The eight Y digit tiles of a stage sit one after the other in shared
// memory, so X digit s times Y digits t0 .. t0 + c - 1 is one MMA of N = 48 c
// that lands in the TMEM columns of levels s + t0 .. s + t0 + c - 1: 11 MMAs
// (N <= 240) per 16-deep k-step instead of 36.
//
// Kernel roles (448 threads, one CTA per SM): warp 0 issues the TMA loads of
// a stage (the 8 digit tiles of X and of Y, 32 deep, 64-byte swizzle), warp 1
// allocates TMEM and issues the MMAs; warps 2-13 (16 columns each) drain the
// eight levels after each window, and the next window's MMAs wait for that
// drain.  Every wait is bounded by a globaltimer deadline (status bit and
// abort flag on expiry).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "internal.h"
#include "oz_internal.h"
#include "tc_device.cuh"
#include "oz_convert.cuh"

namespace pbq {

using namespace tcdev;

namespace {

constexpr int kOzThreads = 448;                                    // 2 + 12 warps
constexpr int kOzEpiThreads = 384;
constexpr int kOzStages = 2;
constexpr uint32_t kOzRowBytes = kOzBK * 2;                        // 64 bytes: one swizzle row
constexpr uint32_t kOzXTile = kOzBM * kOzRowBytes;                 // one digit of X: 8 KB
constexpr uint32_t kOzYTile = kOzBN * kOzRowBytes;                 // one digit of Y: 3 KB
constexpr uint32_t kOzStageBytes = kOzDigits * (kOzXTile + kOzYTile);   // 88 KB
constexpr int kOzWindow = 4;                                       // stages (32-deep) per exact window
constexpr uint32_t kOzTmemCols = 512;                              // >= kOzDigits * kOzBN = 384, a power of two
constexpr int kOzMagic = 0x4B400000;                               // bits of 1.5 * 2^23

// K-major tile with 64-byte rows and the 64-byte swizzle (8-row groups 512 B apart).
__device__ __forceinline__ uint64_t sdesc_k_sw64(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                      // leading byte offset (unused for this layout)
    d |= (uint64_t)(512u >> 4) << 32;            // stride byte offset: 8 rows x 64 B
    d |= (uint64_t)1 << 46;                      // descriptor version
    d |= (uint64_t)4 << 61;                      // 64-byte swizzle
    return d;
}

__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0, int c1, int c2,
                                            int c3) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5, %6}], "
        "[%2];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
        : "memory");
}

// Element (digit s, row r, k) of the k-chunked digit layout (rows x Kp per digit).
__device__ __forceinline__ int64_t oz_idx(int s, int64_t r, int64_t k, int64_t rows, int64_t Kp) {
    return (int64_t)s * rows * Kp + (k >> 5) * rows * 32 + r * 32 + (k & 31);
}

__device__ __forceinline__ uint64_t mad_wide_u(uint32_t a, uint32_t b, uint64_t c) {
    uint64_t d;
    asm("mad.wide.u32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
    return d;
}

// Tile t -> (row tile, column tile); with `upper` only the column tiles
// nt >= 128 mt / 48 (the 128 x 48 tiles that touch the upper triangle) are
// enumerated.
__host__ __device__ inline int64_t oz_first_col_tile(int64_t m) { return (m * kOzBM) / kOzBN; }
__host__ __device__ inline void oz_tile(int64_t t, int NT, int upper, int64_t* mt, int* nt) {
    if (!upper) {
        *mt = t / NT;
        *nt = (int)(t - *mt * NT);
        return;
    }
    int64_t m = 0;
    for (;;) {
        const int64_t first = oz_first_col_tile(m);
        const int64_t cnt = NT - first;
        if (cnt <= 0) { *mt = m; *nt = NT; return; }   // past the end (not reached for t < tiles)
        if (t < cnt) { *mt = m; *nt = (int)(first + t); return; }
        t -= cnt;
        ++m;
    }
}

// Virtual tile v of CTA blockIdx.x -> (row tile, column tile) and the tile's own
// index: with lock > 1 the virtual tiles are the row tiles and the CTA's column
// tile is blockIdx.x % lock.
template <bool kLock>
__device__ __forceinline__ int64_t oz_vtile(int64_t v, int NT, int upper, int lock, int64_t* mt, int* nt) {
    if (kLock) {
        const int j = (int)(blockIdx.x % (unsigned)lock);
        *mt = v;
        *nt = j;
        return v * NT + j;
    }
    oz_tile(v, NT, upper, mt, nt);
    return v;
}

// CTA whose stream-K range holds iteration it.
__device__ __forceinline__ int64_t sk_owner(int64_t it, int64_t T, int64_t G) {
    int64_t c = (it * G) / T;
    while (c + 1 < G && sk_begin(c + 1, T, G) <= it) ++c;
    while (c > 0 && sk_begin(c, T, G) > it) --c;
    return c;
}

// BF16 bits of a small integer d (|d| < 2^22): exact through FP32.
__device__ __forceinline__ uint16_t digit_bf16(int d) {
    const float f = __int_as_float(kOzMagic + d) - 12582912.0f;
    return (uint16_t)(__float_as_uint(f) >> 16);
}

// Biased exponent field of x (0 for zero and subnormals).
__device__ __forceinline__ int exp_field(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7FF); }

// The 8 balanced base-128 digits of round(x 2^(56 - e)), |x| < 2^(e - 1).
__device__ __forceinline__ void digits8(double x, int e, int* d) {
    const long long bits = __double_as_longlong(x);
    int eb = (int)((bits >> 52) & 0x7FF);
    long long mant = bits & 0xFFFFFFFFFFFFFLL;
    if (eb) mant |= 1LL << 52;
    else eb = 1;
    const int sh = eb - 1075 + 56 - e;   // x = mant 2^(eb - 1075); sh <= 2 by the choice of e
    long long F;
    if (sh >= 0) F = mant << sh;
    else if (sh > -62) F = (mant + (1LL << (-sh - 1))) >> (-sh);
    else F = 0;
    if (bits < 0) F = -F;
#pragma unroll
    for (int s = 0; s < 7; ++s) {
        const int w = 7 * (7 - s);
        const long long q = (F + (1LL << (w - 1))) >> w;
        d[s] = (int)q;
        F -= q * (1LL << w);
    }
    d[7] = (int)F;
}

// The MMAs of one stage (two 16-deep k-steps): X digit sx times the Y digits
// t0 .. t0 + c - 1 (c <= 5) into the TMEM columns of levels sx + t0 ..;
// `fresh` starts new level sums (the first stage of a window).
__device__ __forceinline__ void oz_stage_mmas(uint32_t tmem_base, uint32_t xa, bool fresh) {
    const uint64_t dX = sdesc_k_sw64(xa), dY = sdesc_k_sw64(xa + kOzDigits * kOzXTile);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
        for (int sx = 0; sx < kOzDigits; ++sx) {
#pragma unroll
            for (int t0 = 0; t0 < kOzDigits - sx; t0 += 5) {
                const int cnt = (kOzDigits - sx - t0) < 5 ? (kOzDigits - sx - t0) : 5;
                const uint64_t a = dX + (uint64_t)((sx * kOzXTile + kk * 32) >> 4);
                const uint64_t b = dY + (uint64_t)((t0 * kOzYTile + kk * 32) >> 4);
                const uint32_t idesc = idesc_bf16_f32(kOzBM, cnt * kOzBN);
                tc_mma_bf16(tmem_base + (uint32_t)((sx + t0) * kOzBN), a, b, idesc,
                            (fresh && kk == 0 && sx == 0) ? 0u : 1u);
            }
        }
    }
}

// Adds the eight level sums of one window (this thread's row: TMEM lane
// quarter q; columns 16 g .. 16 g + 15) into the two 64-bit accumulators.
// The FP32 level value v (an integer, |v| <= 2^22) is read as the bits of
// v + 1.5 * 2^23, i.e. kOzMagic + v; oz_unbias removes that bias per segment.
__device__ __forceinline__ void oz_drain(uint32_t tmem_base, int q, int g, uint64_t (&hi)[16], uint64_t (&lo)[16]) {
#pragma unroll
    for (int lam = 0; lam < kOzDigits; ++lam) {
        const uint32_t wgt = 1u << (7 * ((lam < 4 ? 3 : 7) - lam));
        float v[16];
        tmem_ld16(tmem_base + (uint32_t)(lam * kOzBN + g * 16) + ((uint32_t)(q * 32) << 16), v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint32_t bv = __float_as_uint(v[j] + 12582912.0f);
            if (lam < 4) hi[j] = mad_wide_u(bv, wgt, hi[j]);
            else lo[j] = mad_wide_u(bv, wgt, lo[j]);
        }
    }
}

// Removes the bias of nwin drained windows: kOzMagic (2^21 + 2^14 + 2^7 + 1)
// was added per window to each of hi and lo (unsigned arithmetic wraps exactly).
__device__ __forceinline__ void oz_unbias(int nwin, uint64_t (&hi)[16], uint64_t (&lo)[16]) {
    const uint64_t bias = (uint64_t)nwin * (uint64_t)kOzMagic * (uint64_t)((1u << 21) + (1u << 14) + (1u << 7) + 1u);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        hi[j] -= bias;
        lo[j] -= bias;
    }
}

// ncol (<= 16) elements of a row of C from the exact sums (units of
// 2^(e_i + f_j - 63), biased exponent fields exr and ey[j]); a row or column
// holding Inf or NaN (exponent field 2047) gives NaN.
__device__ __forceinline__ void oz_store(double* crow, int ncol, int exr, const int* __restrict__ ey,
                                         const uint64_t (&hi)[16], const uint64_t (&lo)[16]) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j < ncol) {
            const int eyr = ey[j];
            crow[j] = (exr >= 2047 || eyr >= 2047)
                          ? __longlong_as_double(0x7FF8000000000000LL)
                          : oz_to_double_fast((int64_t)hi[j], (int64_t)lo[j], exr + eyr - 2 * 1021 - 63);
        }
    }
}

// ---------------------------------------------------------------------------
// The product kernel
// ---------------------------------------------------------------------------
// 448 threads are allocated registers as 16 warps: at most 65536 / 512 = 128 each.
template <bool kLock>
__global__ void __maxnreg__(128)
k_oz_gemm(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, int64_t T, int NT,
          int upper, int lock_, int64_t G, int KI, int tilewise, int64_t Rx, int64_t Ry, const int* __restrict__ ex_raw,
          const int* __restrict__ ey_raw, double* __restrict__ part, int* __restrict__ cnt, double* __restrict__ Cout,
          int64_t ldc, uint32_t* __restrict__ status, uint64_t timeout_ns, const int* __restrict__ cond) {
    if (cond && *cond == 0) return;

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[kOzStages], empty_bar[kOzStages], accf_bar, acce_bar, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int issued_sh, consumed_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Stream-K over T = (virtual tiles) x KI iterations on G = gridDim / lock
    // virtual CTAs.  lock > 1: CTAs lock c .. lock c + lock - 1 run column tiles
    // 0 .. NT - 1 of the same row tiles over the same k-chunks at the same time,
    // so X's digits come from DRAM once and from L2 for the other column tiles;
    // the virtual tiles are then the row tiles.
    const int lock = kLock ? lock_ : 1;
    const int64_t c = kLock ? blockIdx.x / lock : blockIdx.x;
    // tilewise: whole tiles per CTA (short contractions: no partials, no fix-up)
    const int64_t it_begin = tilewise ? sk_begin(c, T / KI, G) * KI : sk_begin(c, T, G);
    const int64_t it_end = tilewise ? sk_begin(c + 1, T / KI, G) * KI : sk_begin(c + 1, T, G);
    const uint64_t deadline = globaltimer() + timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&accf_bar, 1);
        mbar_init(&acce_bar, kOzEpiThreads);
        mbar_init(&drain_bar, 1);
        abort_sh = 0;
        issued_sh = 0;
        consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == 0) {
        // ---------------- TMA producer: one stage = 8 X digit tiles + 8 Y digit tiles
        if (lane == 0) {
            int li = 0;
            for (int64_t it = it_begin; it < it_end; ++it, ++li) {
                const int s = li % kOzStages;
                if (li >= kOzStages) {
                    if (!mbar_wait(&empty_bar[s], (uint32_t)((li / kOzStages - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        break;
                    }
                }
                const int64_t tile = it / KI;
                const int kc = (int)(it - tile * KI);
                int64_t mt;
                int nt;
                oz_vtile<kLock>(tile, NT, upper, lock, &mt, &nt);
                unsigned char* st = smem + (size_t)s * kOzStageBytes;
                mbar_expect_tx(&full_bar[s], kOzStageBytes);
                tma_load_4d(st, &tmX, &full_bar[s], 0, (int)(mt * kOzBM), kc, 0);
                tma_load_4d(st + kOzDigits * kOzXTile, &tmY, &full_bar[s], 0, nt * kOzBN, kc, 0);
                issued_sh = li + 1;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer.  A window is the stages of one tile with
        // k-chunks kOzWindow w .. kOzWindow w + 3 (clipped to the CTA's range).
        if (lane == 0) {
            int li = 0, win = -1;
            bool ok = true;
            for (int64_t it = it_begin; ok && it < it_end; ++it, ++li) {
                const int kc = (int)(it % KI);
                const bool wfirst = (it == it_begin) || (kc % kOzWindow == 0);
                const bool wlast = (it + 1 == it_end) || (kc % kOzWindow == kOzWindow - 1) || (kc + 1 == KI);
                const int s = li % kOzStages;
                if (!mbar_wait(&full_bar[s], (uint32_t)((li / kOzStages) & 1), deadline, &abort_sh)) {
                    abort_sh = 1;
                    ok = false;
                    break;
                }
                if (wfirst) {
                    ++win;
                    // the epilogue has read the previous window's levels out of TMEM
                    if (win > 0 && !mbar_wait(&acce_bar, (uint32_t)((win - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                }
                tc_fence_after();
                oz_stage_mmas(tmem_base, smem_u32(smem + (size_t)s * kOzStageBytes), wfirst);
                tc_commit(&empty_bar[s]);
                if (wlast) tc_commit(&accf_bar);
                consumed_sh = li + 1;
            }
            // all MMAs issued by this thread complete before TMEM is released
            tc_commit(&drain_bar);
            const uint64_t dl = globaltimer() + timeout_ns;
            uint32_t spin = 0;
            while (!mbar_test(&drain_bar, 0)) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) { abort_sh = 1; break; }
            }
        }
    } else {
        // ---------------- epilogue: exact level sums -> (hi, lo) -> C or int64 partials
        const int q = warp & 3;                 // TMEM lane quarter of this warp
        const int g = (warp - 2) >> 2;          // which 16 of the 48 columns
        const int rloc = q * 32 + lane;
        uint64_t hi[16], lo[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
        const int n_it = (int)(it_end - it_begin);
        int kc = (int)(it_begin % KI), tl = 0;  // k-chunk within the tile; tile relative to the first one
        int win = -1, nwin = 0;
        bool ok = true;
        for (int li = 0; ok && li < n_it; ++li) {
            const bool wfirst = (li == 0) || (kc % kOzWindow == 0);
            const bool tile_end = (li + 1 == n_it) || (kc + 1 == KI);
            const bool wlast = tile_end || (kc % kOzWindow == kOzWindow - 1);
            if (wfirst) ++win;
            if (wlast) {
                ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar, (uint32_t)(win & 1), deadline, &abort_sh));
                if (!ok) {
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                oz_drain(tmem_base, q, g, hi, lo);
                tc_fence_before();
                mbar_arrive(&acce_bar);
                ++nwin;
            }
            if (tile_end) {
                const int64_t tile = it_begin / KI + tl;
                int64_t mt;
                int nt;
                const int64_t rtile = oz_vtile<kLock>(tile, NT, upper, lock, &mt, &nt);
                const int64_t row = mt * kOzBM + rloc;
                const int exr = row < Rx ? ex_raw[row] : 0;
                oz_unbias(nwin, hi, lo);   // exact integer sums of this segment, in units of 2^(e_i + f_j - 63)
                const int64_t it0 = tile * KI, it1 = it0 + KI - 1;
                const int64_t col0 = (int64_t)nt * kOzBN + g * 16;
                double* crow = Cout + row * ldc + col0;
                const int ncol = (int)min((int64_t)16, Ry - col0);
                if (it_begin <= it0 && it_end > it1) {
                    // the whole contraction of this tile ran here
                    if (row < Rx) oz_store(crow, ncol, exr, ey_raw + col0, hi, lo);
                } else {
                    // stream-K fix-up per 32 x 16 slice: every contributor adds its integer
                    // sums into the tile's accumulator (64-bit integer reductions: exact
                    // and order-free, modulo 2^64 like the sums themselves), and the one
                    // that completes the slice reads it once, writes C and clears it
                    unsigned long long* acc = (unsigned long long*)part + (size_t)rtile * (size_t)(2 * kOzBM * kOzBN);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        atomicAdd(acc + (size_t)(g * 16 + j) * kOzBM + rloc, (unsigned long long)hi[j]);
                        atomicAdd(acc + (size_t)(kOzBM * kOzBN) + (size_t)(g * 16 + j) * kOzBM + rloc,
                                  (unsigned long long)lo[j]);
                    }
                    __threadfence();
                    __syncwarp();
                    int* ctr = cnt + rtile * 12 + q * 3 + g;
                    int old = 0;
                    if (lane == 0) old = atomicAdd(ctr, 1);
                    old = __shfl_sync(0xffffffffu, old, 0);
                    const int64_t cf = sk_owner(it0, T, G), cl = sk_owner(it1, T, G);
                    if (old == (int)(cl - cf)) {
                        __threadfence();
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            unsigned long long* ph = acc + (size_t)(g * 16 + j) * kOzBM + rloc;
                            unsigned long long* pl = ph + (size_t)(kOzBM * kOzBN);
                            hi[j] = __ldcg(ph);
                            lo[j] = __ldcg(pl);
                            *ph = 0ull;   // ready for the next product
                            *pl = 0ull;
                        }
                        if (row < Rx) oz_store(crow, ncol, exr, ey_raw + col0, hi, lo);
                        if (lane == 0) *ctr = 0;
                    }
                }
#pragma unroll
                for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
                nwin = 0;
                ++tl;
                kc = 0;
            } else {
                ++kc;
            }
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        // wait (bounded) for TMA copies that were issued but never consumed
        const uint64_t dl = globaltimer() + timeout_ns;
        for (int li = consumed_sh; li < issued_sh; ++li) {
            const int s = li % kOzStages;
            uint32_t spin = 0;
            while (!mbar_test(&full_bar[s], (uint32_t)((li / kOzStages) & 1))) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) break;
            }
        }
        if (abort_sh) atomicOr(status, kStTimeout);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kOzTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// The grouped product kernel: the same roles, stages and windows as k_oz_gemm,
// over a list of whole-contraction tiles of many products.  CTA c runs units
// c, c + G, ...; stage, window and level counters run on across units.
// ---------------------------------------------------------------------------
__global__ void __maxnreg__(128)
k_oz_list(const CUtensorMap* __restrict__ maps, const OzListUnit* __restrict__ units, int nunits,
          uint32_t* __restrict__ status, uint64_t timeout_ns) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[kOzStages], empty_bar[kOzStages], accf_bar, acce_bar, drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int issued_sh, consumed_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, c = blockIdx.x;
    const uint64_t deadline = globaltimer() + timeout_ns;
    // a unit whose condition is off is skipped by all three roles alike
    auto skipped = [&](const OzListUnit& U) { return U.cond && *U.cond == 0; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < kOzStages; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        mbar_init(&accf_bar, 1);
        mbar_init(&acce_bar, kOzEpiThreads);
        mbar_init(&drain_bar, 1);
        abort_sh = 0;
        issued_sh = 0;
        consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(kOzTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int li = 0;
            bool ok = true;
            for (int u = c; ok && u < nunits; u += G) {
                const OzListUnit U = units[u];
                if (skipped(U)) continue;
                for (int kc = 0; kc < U.KI; ++kc, ++li) {
                    const int s = li % kOzStages;
                    if (li >= kOzStages &&
                        !mbar_wait(&empty_bar[s], (uint32_t)((li / kOzStages - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    unsigned char* st = smem + (size_t)s * kOzStageBytes;
                    mbar_expect_tx(&full_bar[s], kOzStageBytes);
                    tma_load_4d(st, &maps[U.mapx], &full_bar[s], 0, U.m0, kc, 0);
                    tma_load_4d(st + kOzDigits * kOzXTile, &maps[U.mapy], &full_bar[s], 0, U.n0, kc, 0);
                    issued_sh = li + 1;
                }
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer: windows of kOzWindow stages within a unit
        if (lane == 0) {
            int li = 0, win = -1;
            bool ok = true;
            for (int u = c; ok && u < nunits; u += G) {
                const OzListUnit U = units[u];
                if (skipped(U)) continue;
                for (int kc = 0; kc < U.KI; ++kc, ++li) {
                    const bool wfirst = kc % kOzWindow == 0;
                    const bool wlast = (kc % kOzWindow == kOzWindow - 1) || (kc + 1 == U.KI);
                    const int s = li % kOzStages;
                    if (!mbar_wait(&full_bar[s], (uint32_t)((li / kOzStages) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    if (wfirst) {
                        ++win;
                        if (win > 0 && !mbar_wait(&acce_bar, (uint32_t)((win - 1) & 1), deadline, &abort_sh)) {
                            abort_sh = 1;
                            ok = false;
                            break;
                        }
                    }
                    tc_fence_after();
                    oz_stage_mmas(tmem_base, smem_u32(smem + (size_t)s * kOzStageBytes), wfirst);
                    tc_commit(&empty_bar[s]);
                    if (wlast) tc_commit(&accf_bar);
                    consumed_sh = li + 1;
                }
            }
            tc_commit(&drain_bar);
            const uint64_t dl = globaltimer() + timeout_ns;
            uint32_t spin = 0;
            while (!mbar_test(&drain_bar, 0)) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) { abort_sh = 1; break; }
            }
        }
    } else {
        // ---------------- epilogue: per unit, level sums -> (hi, lo) -> C
        const int q = warp & 3;
        const int g = (warp - 2) >> 2;
        const int rloc = q * 32 + lane;
        uint64_t hi[16], lo[16];
        int win = -1;
        bool ok = true;
        for (int u = c; ok && u < nunits; u += G) {
            const OzListUnit U = units[u];
            if (skipped(U)) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) { hi[j] = 0; lo[j] = 0; }
            int nwin = 0;
            for (int kc = 0; kc < U.KI; ++kc) {
                if (kc % kOzWindow == 0) ++win;
                if ((kc % kOzWindow == kOzWindow - 1) || (kc + 1 == U.KI)) {
                    ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar, (uint32_t)(win & 1), deadline, &abort_sh));
                    if (!ok) {
                        abort_sh = 1;
                        break;
                    }
                    tc_fence_after();
                    oz_drain(tmem_base, q, g, hi, lo);
                    tc_fence_before();
                    mbar_arrive(&acce_bar);
                    ++nwin;
                }
            }
            if (!ok) break;
            oz_unbias(nwin, hi, lo);
            const int row = U.m0 + rloc, col0 = U.n0 + g * 16;
            if (row < U.Rx && col0 < U.Ry)
                oz_store(U.C + (int64_t)row * U.ldc + col0, min(16, U.Ry - col0), U.ex[row], U.ey + col0, hi, lo);
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        // wait (bounded) for TMA copies that were issued but never consumed
        const uint64_t dl = globaltimer() + timeout_ns;
        for (int li = consumed_sh; li < issued_sh; ++li) {
            const int s = li % kOzStages;
            uint32_t spin = 0;
            while (!mbar_test(&full_bar[s], (uint32_t)((li / kOzStages) & 1))) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) break;
            }
        }
        if (abort_sh) atomicOr(status, kStTimeout);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(kOzTmemCols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// Digit preparation
// ---------------------------------------------------------------------------
// Column exponents of a rows x N panel: eraw[j] = max over rows of the biased exponent.
__global__ void k_oz_panel_exp(int64_t rows, int N, const double* __restrict__ P, int64_t ldp, int* __restrict__ eraw,
                               const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    const int j = blockIdx.y * 256 + threadIdx.x;
    if (j >= N) return;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int64_t r1 = r0 + 64 < rows ? r0 + 64 : rows;
    int mx = 0;
    for (int64_t r = r0; r < r1; ++r) mx = max(mx, exp_field(P[r * ldp + j]));
    if (mx > 0) atomicMax(&eraw[j], mx);
}

// Digits of P^T (rows N, contraction over the panel rows, zero digits up to
// the padded contraction length) with the column scales eraw[j].
__global__ void k_oz_panel_slice(int64_t rows, int N, const double* __restrict__ P, int64_t ldp,
                                 const int* __restrict__ eraw, uint16_t* __restrict__ S, const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    __shared__ uint16_t sd[kOzDigits][32][33];
    const int64_t Kp = oz_kpad(rows);
    const int64_t r0 = (int64_t)blockIdx.y * 32;
    const int j0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;   // 32 x 8
    const int j = j0 + tx;
    const int e = j < N ? eraw[j] - 1021 : 0;
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t r = r0 + rr;
        const double x = (r < rows && j < N) ? P[r * ldp + j] : 0.0;
        int d[kOzDigits];
        digits8(x, e, d);
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) sd[s][tx][rr] = digit_bf16(d[s]);
    }
    __syncthreads();
    const int64_t r = r0 + tx;   // < Kp: the grid covers the padded contraction exactly
    for (int jj = ty; jj < 32; jj += 8) {
        const int jc = j0 + jj;
        if (jc >= N) break;
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) S[oz_idx(s, jc, r, N, Kp)] = sd[s][jj][tx];
    }
}

template <typename Tin>
__device__ __forceinline__ double load_a(const Tin* A, int64_t i) {
    return (double)A[i];
}

// Row and column exponents of A: tiles of 64 rows x 512 columns, one column
// per thread; row maxima by warp reductions and shared memory, then one
// atomicMax per row and per column for the tile (maxima are order-free, so
// the result is deterministic).
template <typename Tin>
__global__ void __launch_bounds__(512)
k_oz_a_exp(int64_t m, int64_t n, const Tin* __restrict__ A, int64_t lda, int* __restrict__ er, int* __restrict__ ec,
           const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    __shared__ int rmax[16][64];
    const int64_t r0 = (int64_t)blockIdx.y * 64, c = (int64_t)blockIdx.x * 512 + threadIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int cm = 0;
    for (int rr = 0; rr < 64; ++rr) {
        const int64_t r = r0 + rr;
        const int eb = (r < m && c < n) ? exp_field(load_a(A, r * lda + c)) : 0;
        cm = max(cm, eb);
        const int w = __reduce_max_sync(0xffffffffu, eb);
        if (lane == 0) rmax[warp][rr] = w;
    }
    if (c < n && cm > 0) atomicMax(&ec[c], cm);
    __syncthreads();
    if (threadIdx.x < 64) {
        int v = 0;
#pragma unroll
        for (int w = 0; w < 16; ++w) v = max(v, rmax[w][threadIdx.x]);
        const int64_t r = r0 + threadIdx.x;
        if (r < m && v > 0) atomicMax(&er[r], v);
    }
}

// Digits of A (row scales; rows m, contraction n) and of A^T (column scales;
// rows n, contraction m) from one read of a 32 x 32 tile; the grid covers
// both padded contraction lengths, whose digits are zero.
template <typename Tin>
__global__ void k_oz_a_slice(int64_t m, int64_t n, const Tin* __restrict__ A, int64_t lda, const int* __restrict__ er,
                             const int* __restrict__ ec, uint16_t* __restrict__ Srow, uint16_t* __restrict__ Scol,
                             const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    __shared__ uint16_t sd[kOzDigits][32][33];
    const int64_t mp = oz_kpad(m), np = oz_kpad(n);
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t cc = c0 + tx;
    const int ecol = cc < n ? ec[cc] - 1021 : 0;
    for (int rr = ty; rr < 32; rr += 8) {
        const int64_t r = r0 + rr;
        const bool in = r < m && cc < n;
        const double x = in ? load_a(A, r * lda + cc) : 0.0;
        int d[kOzDigits];
        if (Srow && r < m) {
            digits8(x, er[r] - 1021, d);
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s) Srow[oz_idx(s, r, cc, m, np)] = digit_bf16(d[s]);
        }
        if (Scol) {
            digits8(x, ecol, d);
#pragma unroll
            for (int s = 0; s < kOzDigits; ++s) sd[s][tx][rr] = digit_bf16(d[s]);
        }
    }
    if (!Scol) return;
    __syncthreads();
    const int64_t r = r0 + tx;   // < mp
    for (int jj = ty; jj < 32; jj += 8) {
        const int64_t jc = c0 + jj;
        if (jc >= n) break;
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) Scol[oz_idx(s, jc, r, n, mp)] = sd[s][jj][tx];
    }
}

// Digits of row r of a row-major matrix P (rows x K, ld ldp; K up to a few
// thousand) in one pass by one warp: the row's largest exponent field (warp
// max), then the row's digits, zero up to the padded K.
__device__ __forceinline__ void oz_row_digits(int64_t r, int64_t rows, int64_t K, const double* __restrict__ P,
                                              int64_t ldp, int* __restrict__ er, uint16_t* __restrict__ S) {
    const int lane = threadIdx.x & 31;
    const double* pr = P + r * ldp;
    const int64_t Kp = oz_kpad(K);
    int mx = 0;
    for (int64_t k = lane; k < K; k += 32) mx = max(mx, exp_field(pr[k]));
    mx = __reduce_max_sync(0xffffffffu, mx);
    if (lane == 0) er[r] = mx;
    const int e = mx - 1021;
    for (int64_t k = lane; k < Kp; k += 32) {
        const double x = k < K ? pr[k] : 0.0;
        int d[kOzDigits];
        digits8(x, e, d);
#pragma unroll
        for (int s = 0; s < kOzDigits; ++s) S[oz_idx(s, r, k, rows, Kp)] = digit_bf16(d[s]);
    }
}

__global__ void __launch_bounds__(512)
k_oz_rows(int64_t rows, int64_t K, const double* __restrict__ P, int64_t ldp, int* __restrict__ er,
          uint16_t* __restrict__ S, const int* __restrict__ cond) {
    if (cond && *cond == 0) return;
    const int64_t r = (int64_t)blockIdx.x * 16 + (threadIdx.x >> 5);
    if (r < rows) oz_row_digits(r, rows, K, P, ldp, er, S);
}

// Row digits of the units: unit b covers rows r0 .. r0 + 15 of its matrix.
__global__ void __launch_bounds__(512) k_oz_rows_list(const OzPanelUnit* __restrict__ units) {
    const OzPanelUnit& U = units[blockIdx.x];
    if (U.cond && *U.cond == 0) return;
    const int64_t r = U.r0 + (threadIdx.x >> 5);
    if (r < U.rows) oz_row_digits(r, U.rows, U.N, U.P, U.ldp, U.eraw, (uint16_t*)U.S);
}

// Column exponents of the panel units: unit b covers rows r0 .. r0 + 127 of
// its panel; thread (tx, ty) scans columns tx + 32 cg over rows ty, ty + 8, ..
// and the column maxima go out with one atomicMax each (order-free).
__global__ void __launch_bounds__(256)
k_oz_panel_exp_list(const OzPanelUnit* __restrict__ units) {
    const OzPanelUnit U = units[blockIdx.x];
    if (U.cond && *U.cond == 0) return;
    __shared__ int sm[8][256];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int64_t r1 = U.r0 + kOzPanelRows < U.rows ? U.r0 + kOzPanelRows : U.rows;
    for (int j = tx; j < U.N; j += 32) {
        int mx = 0;
        for (int64_t r = U.r0 + ty; r < r1; r += 8) mx = max(mx, exp_field(U.P[r * U.ldp + j]));
        sm[ty][j] = mx;
    }
    __syncthreads();
    for (int j = ty * 32 + tx; j < U.N; j += 256) {
        int mx = 0;
#pragma unroll
        for (int t = 0; t < 8; ++t) mx = max(mx, sm[t][j]);
        if (mx > 0) atomicMax(&U.eraw[j], mx);
    }
}

// Digits of the panel units (P^T: rows N, contraction over the panel rows):
// each 32 x 32 block is sliced into shared memory and written transposed,
// zero digits past the panel rows up to the padded contraction length.
__global__ void __launch_bounds__(256)
k_oz_panel_slice_list(const OzPanelUnit* __restrict__ units) {
    const OzPanelUnit U = units[blockIdx.x];
    if (U.cond && *U.cond == 0) return;
    __shared__ uint16_t sd[kOzDigits][32][33];
    const int64_t Kp = oz_kpad(U.rows);
    const int tx = threadIdx.x, ty = threadIdx.y;
    uint16_t* S = (uint16_t*)U.S;
    for (int64_t rb = U.r0; rb < U.r0 + kOzPanelRows && rb < Kp; rb += 32) {
        for (int j0 = 0; j0 < U.N; j0 += 32) {
            const int j = j0 + tx;
            const int e = j < U.N ? U.eraw[j] - 1021 : 0;
            for (int rr = ty; rr < 32; rr += 8) {
                const int64_t r = rb + rr;
                const double x = (r < U.rows && j < U.N) ? U.P[r * U.ldp + j] : 0.0;
                int d[kOzDigits];
                digits8(x, e, d);
#pragma unroll
                for (int s = 0; s < kOzDigits; ++s) sd[s][tx][rr] = digit_bf16(d[s]);
            }
            __syncthreads();
            for (int jj = ty; jj < 32; jj += 8) {
                const int jc = j0 + jj;
                if (jc >= U.N) break;
#pragma unroll
                for (int s = 0; s < kOzDigits; ++s) S[oz_idx(s, jc, rb + tx, U.N, Kp)] = sd[s][jj][tx];
            }
            __syncthreads();
        }
    }
}

typedef CUresult (*PFN_encodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

PFN_encodeTiled encode_fn() {
    static PFN_encodeTiled fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_encodeTiled)p;
    }
    return fn;
}

// 4-D map over the k-chunked digits of an operand: {32, rows, chunks, digit},
// box {32, box_rows, 1, 7} (one stage: a 32-deep block of box_rows rows, all digits).
bool make_map_oz(CUtensorMap* map, const OzOperand& op, int box_rows) {
    PFN_encodeTiled fn = encode_fn();
    if (!fn || !op.S || op.rows < 1 || op.K < 1) return false;
    const int64_t Kp = oz_kpad(op.K);
    cuuint64_t dims[4] = {32, (cuuint64_t)op.rows, (cuuint64_t)(Kp / 32), (cuuint64_t)kOzDigits};
    cuuint64_t strides[3] = {64, (cuuint64_t)op.rows * 64, (cuuint64_t)op.rows * Kp * 2};
    cuuint32_t box[4] = {(cuuint32_t)kOzBK, (cuuint32_t)box_rows, 1, (cuuint32_t)kOzDigits};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(op.S), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

OzGeom oz_geometry(int64_t Mrows, int N, int64_t K, bool upper, int num_sms) {
    OzGeom g;
    const int64_t MT = (Mrows + kOzBM - 1) / kOzBM;
    g.NT = (N + kOzBN - 1) / kOzBN;
    g.upper = upper ? 1 : 0;
    if (upper) {
        g.tiles = 0;
        for (int64_t m = 0; m < MT; ++m) g.tiles += (g.NT - oz_first_col_tile(m) > 0) ? g.NT - oz_first_col_tile(m) : 0;
    } else {
        g.tiles = MT * g.NT;
    }
    g.KI = (int)((K + kOzBK - 1) / kOzBK);
    // the column tiles of a row tile run in lockstep on NT CTAs (X read from
    // DRAM once) for full rectangles of 2 .. 8 column tiles
    g.lock = (!upper && g.NT >= 2 && g.NT <= 8 && num_sms >= g.NT) ? g.NT : 1;
    const int64_t T = (g.lock > 1 ? MT : g.tiles) * g.KI;
    const int sms = num_sms / g.lock;
    // at least min_it iterations (32-deep chunks) per CTA: small products use
    // fewer CTAs.  Short contractions (the CholeskyQR solve and Qb, K = l) and
    // the Grams (a few tiles over a long K, split over many CTAs) take 4; the
    // passes over A take 16 (8 measured the same).
    const int64_t min_it = (g.KI <= 8 || upper) ? 4 : 16;
    const int64_t want = (T + min_it - 1) / min_it;
    int Gv = (int)(want < sms ? want : sms);
    // short contractions (K <= 256) run whole tiles on each CTA: splitting them
    // gains no parallelism worth its fix-up (measured: the fix-up of a 4-chunk
    // split took as long as the MMAs)
    g.tilewise = g.KI <= 8 ? 1 : 0;
    if (g.tilewise) {
        const int64_t vt = T / g.KI;
        Gv = (int)(vt < sms ? vt : sms);
    }
    if (Gv < 1) Gv = 1;
    g.G = Gv * g.lock;
    g.part_doubles = g.tiles * 2 * kOzBM * kOzBN;   // a tile's two int64 accumulators per element
    return g;
}

cudaError_t launch_oz_product(const OzOperand& X, const OzOperand& Y, const OzGeom& g, double* part, int* cnt,
                              double* C, int64_t ldc, uint32_t* status, const int* cond, cudaStream_t s,
                              cudaEvent_t after_gemm) {
    if (g.tiles < 1 || Y.rows > (int64_t)g.NT * kOzBN || !X.eraw || !Y.eraw || X.K != Y.K || !cnt)
        return cudaErrorInvalidValue;
    CUtensorMap mx, my;
    if (!make_map_oz(&mx, X, kOzBM)) return PBQ_DBG(cudaErrorInvalidValue);   // tensor map of X refused
    if (!make_map_oz(&my, Y, kOzBN)) return PBQ_DBG(cudaErrorInvalidValue);   // tensor map of Y refused
    const size_t smem = (size_t)kOzStages * kOzStageBytes + 1024;
    const void* fn = g.lock > 1 ? (const void*)k_oz_gemm<true> : (const void*)k_oz_gemm<false>;
    cudaError_t e = PBQ_DBG(func_smem_attr(fn, smem));
    if (e != cudaSuccess) return e;
    if (g.lock < 1 || g.G % g.lock != 0 || (g.lock > 1 && (g.upper || g.lock != g.NT))) return cudaErrorInvalidValue;
    const int64_t T = (g.lock > 1 ? g.tiles / g.NT : g.tiles) * (int64_t)g.KI;
    if (g.lock > 1)
        k_oz_gemm<true><<<g.G, kOzThreads, smem, s>>>(mx, my, T, g.NT, g.upper, g.lock, (int64_t)(g.G / g.lock), g.KI,
                                                      g.tilewise, X.rows, Y.rows, X.eraw, Y.eraw, part, cnt, C, ldc, status,
                                                      2000000000ull, cond);
    else
        k_oz_gemm<false><<<g.G, kOzThreads, smem, s>>>(mx, my, T, g.NT, g.upper, 1, (int64_t)g.G, g.KI, g.tilewise, X.rows,
                                                       Y.rows, X.eraw, Y.eraw, part, cnt, C, ldc, status,
                                                       2000000000ull, cond);
    count_launches(1);
    if ((e = PBQ_DBG(cudaGetLastError())) != cudaSuccess) {
        const char* v = std::getenv("PBPQLP_DEBUG");
        cudaFuncAttributes fa;
        if (v && v[0] == '1' && cudaFuncGetAttributes(&fa, fn) == cudaSuccess)
            std::fprintf(stderr, "pbpqlp: k_oz_gemm regs %d, max threads %d, static smem %zu, max dyn smem %d, local %zu, "
                         "launch %d x %d with %zu bytes\n", fa.numRegs, fa.maxThreadsPerBlock, fa.sharedSizeBytes,
                         fa.maxDynamicSharedSizeBytes, fa.localSizeBytes, g.G, kOzThreads, smem);
        return e;
    }
    if (after_gemm && (e = cudaEventRecord(after_gemm, s)) != cudaSuccess) return e;
    return cudaSuccess;
}

cudaError_t launch_oz_panel(int64_t rows, int N, const double* P, int64_t ldp, int* eraw, void* S, const int* cond,
                            cudaStream_t s) {
    if (rows < 1 || N < 1) return cudaErrorInvalidValue;
    cudaError_t e = cudaMemsetAsync(eraw, 0, sizeof(int) * (size_t)N, s);
    if (e != cudaSuccess) return e;
    k_oz_panel_exp<<<dim3((unsigned)((rows + 63) / 64), (unsigned)((N + 255) / 256)), 256, 0, s>>>(rows, N, P, ldp,
                                                                                                   eraw, cond);
    dim3 grid((unsigned)((N + 31) / 32), (unsigned)((rows + 31) / 32)), block(32, 8);
    k_oz_panel_slice<<<grid, block, 0, s>>>(rows, N, P, ldp, eraw, (uint16_t*)S, cond);
    count_launches(2);
    return cudaGetLastError();
}

cudaError_t launch_oz_rows(int64_t rows, int64_t K, const double* P, int64_t ldp, int* er, void* S, const int* cond,
                           cudaStream_t s) {
    if (rows < 1 || K < 1) return cudaErrorInvalidValue;
    k_oz_rows<<<(unsigned)((rows + 15) / 16), 512, 0, s>>>(rows, K, P, ldp, er, (uint16_t*)S, cond);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_oz_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, int* er, int* ec, void* Srow,
                        void* Scol, cudaStream_t s, const int* cond) {
    cudaError_t e = cudaMemsetAsync(er, 0, sizeof(int) * (size_t)m, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ec, 0, sizeof(int) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((n + 31) / 32), (unsigned)((m + 31) / 32)), block(32, 8);
    dim3 egrid((unsigned)((n + 511) / 512), (unsigned)((m + 63) / 64));
    if (a_f32) {
        k_oz_a_exp<float><<<egrid, 512, 0, s>>>(m, n, (const float*)A, lda, er, ec, cond);
        k_oz_a_slice<float><<<grid, block, 0, s>>>(m, n, (const float*)A, lda, er, ec, (uint16_t*)Srow,
                                                   (uint16_t*)Scol, cond);
    } else {
        k_oz_a_exp<double><<<egrid, 512, 0, s>>>(m, n, (const double*)A, lda, er, ec, cond);
        k_oz_a_slice<double><<<grid, block, 0, s>>>(m, n, (const double*)A, lda, er, ec, (uint16_t*)Srow,
                                                    (uint16_t*)Scol, cond);
    }
    count_launches(2);
    return cudaGetLastError();
}

bool make_oz_map(void* map128, const void* S, int64_t rows, int64_t K, int box_rows) {
    OzOperand op;
    op.S = S;
    op.rows = rows;
    op.K = K;
    return make_map_oz((CUtensorMap*)map128, op, box_rows);
}

cudaError_t launch_oz_list(const void* maps, const OzListUnit* units, int n, int G, uint32_t* status, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    if (!maps || !units || !status || G < 1) return cudaErrorInvalidValue;
    const size_t smem = (size_t)kOzStages * kOzStageBytes + 1024;
    cudaError_t e = PBQ_DBG(func_smem_attr((const void*)k_oz_list, smem));
    if (e != cudaSuccess) return e;
    k_oz_list<<<G < n ? G : n, kOzThreads, smem, s>>>((const CUtensorMap*)maps, units, n, status, 2000000000ull);
    count_launches(1);
    return PBQ_DBG(cudaGetLastError());
}

cudaError_t launch_oz_panel_exp_list(const OzPanelUnit* units, int n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_oz_panel_exp_list<<<n, dim3(32, 8), 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_oz_rows_list(const OzPanelUnit* units, int n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_oz_rows_list<<<n, 512, 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_oz_panel_slice_list(const OzPanelUnit* units, int n, cudaStream_t s) {
    if (n < 1) return cudaSuccess;
    k_oz_panel_slice_list<<<n, dim3(32, 8), 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq
