// Tensor-core (tcgen05 / TMEM / TMA) products with A and A^T for the mixed
// precision modes of Algorithm 3 (the sketch C = A^T Phi, the power-iteration
// products and the projection D = A Pbar; Eqs. 3 and 5).
//
// C[i][j] = sum_k Aop[i][k] * Bt[j][k]: both operands are K-major BF16 in
// global memory (A pre-split into row-major and transposed copies, the
// panels transposed), moved by TMA with the 128-byte swizzle into a ring of
// shared-memory stages and multiplied by tcgen05.mma (kind::f16, FP32
// accumulation in TMEM).  The split mode issues three MMAs per k-step,
// hi*hi + lo*hi + hi*lo, into the same accumulator.
//
// Work split: static stream-K over the (row tile, k-block) iterations, so the
// 152 SMs get equal shares; each contiguous run of k-blocks of one tile is a
// "segment" whose FP32 partial goes to a partial buffer, and a second kernel
// adds the partials of each tile in CTA order (deterministic) into the FP64
// output panel.
//
// Accumulation: the tensor pipe's FP32 accumulation drifts toward zero by an
// amount that grows with the depth of the sum, so each segment is cut into
// chunks of kTcKC k-blocks; a chunk accumulates in TMEM and is then added
// (round-to-nearest, CUDA cores) into FP32 registers of the epilogue warps.
//
// Roles (320 threads): warp 0 issues TMA, warp 1 allocates TMEM and issues
// MMAs, warps 2-9 drain the double-buffered TMEM chunk accumulator (two warps
// per TMEM lane quarter, each owning half of the tile's columns).  Every wait on
// an mbarrier is bounded by a globaltimer deadline; on expiry the CTA sets a
// status bit, raises a shared abort flag, drains what it issued and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cstdint>

#include "internal.h"
#include "tc_internal.h"
#include "split_device.cuh"
#include "tc_device.cuh"

namespace pbq {

using namespace tcdev;

constexpr int kTcBM = 128;   // rows per tile (one TMEM lane per row)
constexpr int kTcRowBytes = 128;   // one k-block = one 128-byte swizzle row: 64 BF16 or 32 TF32 elements
constexpr int kTcKC = 16;    // k-blocks per TMEM accumulation chunk (1024-deep BF16, 512-deep TF32 sums)
__host__ __device__ constexpr int tc_bk(bool tf32) { return tf32 ? 32 : 64; }
constexpr int kTcThreads = 320;

template <int NPROD, int BN, int STAGES, bool TF32>
__global__ void __launch_bounds__(kTcThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
          const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, int64_t tiles,
          int KI, int smax, float* __restrict__ part, uint32_t* __restrict__ status, uint64_t timeout_ns,
          int stall) {
    constexpr int BK = tc_bk(TF32);
    constexpr uint32_t A_BYTES = kTcBM * kTcRowBytes;
    constexpr uint32_t B_BYTES = BN * kTcRowBytes;
    constexpr uint32_t STAGE_BYTES = (A_BYTES + B_BYTES) * (NPROD == 3 ? 2 : 1);
    constexpr uint32_t ACC_COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    constexpr uint32_t IDESC = TF32 ? idesc_tf32_f32(kTcBM, BN) : idesc_bf16_f32(kTcBM, BN);

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int issued_sh, consumed_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t G = gridDim.x, c = blockIdx.x;
    const int64_t T = tiles * (int64_t)KI;
    const int64_t it_begin = sk_begin(c, T, G), it_end = sk_begin(c + 1, T, G);
    const uint64_t deadline = globaltimer() + timeout_ns;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) { mbar_init(&full_bar[s], 1); mbar_init(&empty_bar[s], 1); }
        for (int b = 0; b < 2; ++b) { mbar_init(&accf_bar[b], 1); mbar_init(&acce_bar[b], 256); }
        mbar_init(&drain_bar, 1);
        abort_sh = 0;
        issued_sh = 0;
        consumed_sh = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base_sh)),
                     "r"(2 * ACC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = tmem_base_sh;

    auto stage_ptr = [&](int s, int which) -> unsigned char* {
        // which: 0 = A hi, 1 = B hi, 2 = A lo, 3 = B lo
        unsigned char* base = smem + (size_t)s * STAGE_BYTES;
        switch (which) {
            case 0: return base;
            case 1: return base + A_BYTES;
            case 2: return base + A_BYTES + B_BYTES;
            default: return base + 2 * A_BYTES + B_BYTES;
        }
    };

    if (warp == 0) {
        // ---------------- TMA producer (stall: a host-requested test of the
        // bounded waits; nothing is issued and the consumers time out)
        if (lane == 0 && !stall) {
            int li = 0;
            for (int64_t it = it_begin; it < it_end; ++it, ++li) {
                const int s = li % STAGES;
                if (li >= STAGES) {
                    if (!mbar_wait(&empty_bar[s], (uint32_t)((li / STAGES - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        break;
                    }
                }
                const int64_t tile = it / KI;
                const int k0 = (int)(it - tile * KI) * BK;
                const int m0 = (int)(tile * kTcBM);
                mbar_expect_tx(&full_bar[s], STAGE_BYTES);
                tma_load_2d(stage_ptr(s, 0), &tmAhi, &full_bar[s], k0, m0);
                tma_load_2d(stage_ptr(s, 1), &tmBhi, &full_bar[s], k0, 0);
                if (NPROD == 3) {
                    tma_load_2d(stage_ptr(s, 2), &tmAlo, &full_bar[s], k0, m0);
                    tma_load_2d(stage_ptr(s, 3), &tmBlo, &full_bar[s], k0, 0);
                }
                issued_sh = li + 1;
            }
        }
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int li = 0, chunk = 0;
            bool ok = true;
            int64_t it = it_begin;
            while (ok && it < it_end) {
                const int64_t tile = it / KI;
                const int64_t seg_end = ((tile + 1) * KI < it_end) ? (tile + 1) * KI : it_end;
                while (ok && it < seg_end) {
                    const int64_t ch_end = (it + kTcKC < seg_end) ? it + kTcKC : seg_end;
                    const int b = chunk & 1;
                    if (chunk >= 2 &&
                        !mbar_wait(&acce_bar[b], (uint32_t)((chunk / 2 - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)b * ACC_COLS;
                    bool first = true;
                    for (; it < ch_end; ++it, ++li) {
                        const int s = li % STAGES;
                        if (!mbar_wait(&full_bar[s], (uint32_t)((li / STAGES) & 1), deadline, &abort_sh)) {
                            abort_sh = 1;
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t ahi = smem_u32(stage_ptr(s, 0)), bhi = smem_u32(stage_ptr(s, 1));
                        const uint32_t alo = smem_u32(stage_ptr(s, 2)), blo = smem_u32(stage_ptr(s, 3));
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            // one MMA k-step = 32 bytes of the swizzled row (16 BF16 or 8 TF32)
                            const uint32_t off = kk * 32;
                            auto mma = [&](uint32_t a, uint32_t b, uint32_t acc) {
                                if (TF32) tc_mma_tf32(dt, sdesc_k_sw128(a + off), sdesc_k_sw128(b + off), IDESC, acc);
                                else tc_mma_bf16(dt, sdesc_k_sw128(a + off), sdesc_k_sw128(b + off), IDESC, acc);
                            };
                            mma(ahi, bhi, (first && kk == 0) ? 0u : 1u);
                            if (NPROD == 3) {
                                mma(alo, bhi, 1u);
                                mma(ahi, blo, 1u);
                            }
                        }
                        first = false;
                        tc_commit(&empty_bar[s]);
                        consumed_sh = li + 1;
                    }
                    if (!ok) break;
                    tc_commit(&accf_bar[b]);
                    ++chunk;
                }
            }
            // all MMAs issued by this thread complete before TMEM is released;
            // this wait ignores the abort flag (bounded by the deadline only)
            tc_commit(&drain_bar);
            const uint64_t dl = globaltimer() + timeout_ns;
            uint32_t spin = 0;
            while (!mbar_test(&drain_bar, 0)) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) { abort_sh = 1; break; }
            }
        }
    } else {
        // ---------------- epilogue: TMEM chunks -> FP32 registers -> FP32 partials
        constexpr int NCH = BN / 16;              // 16-column groups of the tile
        constexpr int HCH = (NCH + 1) / 2;        // groups owned by one of the two warps of a quarter
        const int q = warp & 3;                   // TMEM lane quarter this warp may access
        const int h = (warp - 2) >> 2;            // which half of the column groups
        const int row = q * 32 + lane;
        float acc[HCH][16];
        int chunk = 0;
        int64_t it = it_begin;
        const int64_t first_tile = it_begin / KI;
        bool ok = true;
        while (ok && it < it_end) {
            const int64_t tile = it / KI;
            const int64_t seg_end = ((tile + 1) * KI < it_end) ? (tile + 1) * KI : it_end;
#pragma unroll
            for (int g = 0; g < HCH; ++g)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[g][i] = 0.f;
            while (it < seg_end) {
                const int64_t ch_end = (it + kTcKC < seg_end) ? it + kTcKC : seg_end;
                const int b = chunk & 1;
                // warp-uniform decision: the TMEM loads below are .sync.aligned
                ok = __all_sync(0xffffffffu, mbar_wait(&accf_bar[b], (uint32_t)((chunk / 2) & 1), deadline, &abort_sh));
                if (!ok) {
                    abort_sh = 1;
                    break;
                }
                tc_fence_after();
                const uint32_t taddr = tmem_base + (uint32_t)b * ACC_COLS + ((uint32_t)(q * 32) << 16);
#pragma unroll
                for (int g = 0; g < HCH; ++g) {
                    const int grp = h * HCH + g;
                    if (grp < NCH) {
                        float v[16];
                        tmem_ld16(taddr + grp * 16, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[g][i] += v[i];
                    }
                }
                tc_fence_before();
                mbar_arrive(&acce_bar[b]);
                it = ch_end;
                ++chunk;
            }
            if (!ok) break;
            float* slot = part + ((size_t)c * smax + (size_t)(tile - first_tile)) * (size_t)kTcBM * BN;
#pragma unroll
            for (int g = 0; g < HCH; ++g) {
                const int grp = h * HCH + g;
                if (grp < NCH) {
                    float4* dst = (float4*)(slot + ((size_t)grp * kTcBM + row) * 16);
                    dst[0] = make_float4(acc[g][0], acc[g][1], acc[g][2], acc[g][3]);
                    dst[1] = make_float4(acc[g][4], acc[g][5], acc[g][6], acc[g][7]);
                    dst[2] = make_float4(acc[g][8], acc[g][9], acc[g][10], acc[g][11]);
                    dst[3] = make_float4(acc[g][12], acc[g][13], acc[g][14], acc[g][15]);
                }
            }
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
        // wait (bounded) for TMA copies that were issued but never consumed
        const uint64_t dl = globaltimer() + timeout_ns;
        for (int li = consumed_sh; li < issued_sh; ++li) {
            const int s = li % STAGES;
            uint32_t spin = 0;
            while (!mbar_test(&full_bar[s], (uint32_t)((li / STAGES) & 1))) {
                if ((++spin & 255u) == 0 && globaltimer() > dl) break;
            }
        }
        if (abort_sh) atomicOr(status, kStTimeout);
    }
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(2 * ACC_COLS)
                     : "memory");
    }
}

// Sum the stream-K partials of each tile in CTA order into C (FP64, rows x N, ldc).
__global__ void k_tc_reduce(int64_t rows, int N, int BN, int64_t tiles, int KI, int64_t G, int smax,
                            const float* __restrict__ part, double* __restrict__ C, int64_t ldc) {
    const int64_t T = tiles * (int64_t)KI;
    const int64_t total = rows * (int64_t)N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / N;
        const int j = (int)(e - i * N);
        const int64_t tile = i / kTcBM;
        const int r = (int)(i - tile * kTcBM);
        const int64_t it0 = tile * KI, it1 = it0 + KI - 1;
        int64_t c = (it0 * G) / T;
        while (c + 1 < G && sk_begin(c + 1, T, G) <= it0) ++c;
        while (c > 0 && sk_begin(c, T, G) > it0) --c;
        double acc = 0.0;
        for (; c < G && sk_begin(c, T, G) <= it1; ++c) {
            const int64_t b = sk_begin(c, T, G), en = sk_begin(c + 1, T, G);
            if (en <= it0) continue;
            const int64_t ft = b / KI;
            const float* slot = part + ((size_t)c * smax + (size_t)(tile - ft)) * (size_t)kTcBM * BN;
            acc += (double)slot[((size_t)(j >> 4) * kTcBM + r) * 16 + (j & 15)];
        }
        C[i * ldc + j] = acc;
    }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

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

// 2-D tensor map over a rows x cols row-major matrix (ld elements) of BF16 or
// FP32 (TF32 operands), box {one 128-byte row of k, box_rows}.
bool make_map(CUtensorMap* map, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows, bool tf32) {
    PFN_encodeTiled fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * (tf32 ? 4 : 2)};
    cuuint32_t box[2] = {(cuuint32_t)tc_bk(tf32), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base),
              dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NPROD, int BN, bool TF32>
cudaError_t launch_tc_bn(const CUtensorMap* m, int64_t tiles, int KI, int G, int smax, float* part, uint32_t* status,
                         uint64_t timeout_ns, cudaStream_t s, int stall) {
    constexpr uint32_t A_BYTES = kTcBM * kTcRowBytes, B_BYTES = BN * kTcRowBytes;
    constexpr uint32_t STAGE = (A_BYTES + B_BYTES) * (NPROD == 3 ? 2 : 1);
    constexpr int STAGES = (int)((220u * 1024u) / STAGE) > 8 ? 8 : (int)((220u * 1024u) / STAGE);
    static_assert(STAGES >= 2, "stage ring too small");
    const size_t smem = (size_t)STAGES * STAGE + 1024;
    auto kern = k_tc_gemm<NPROD, BN, STAGES, TF32>;
    cudaError_t e = func_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<G, kTcThreads, smem, s>>>(m[0], m[1], m[2], m[3], tiles, KI, smax, part, status, timeout_ns, stall);
    count_launches(1);
    return cudaGetLastError();
}

template <int NPROD, bool TF32>
cudaError_t launch_tc_nprod(int BN, const CUtensorMap* m, int64_t tiles, int KI, int G, int smax, float* part,
                            uint32_t* status, uint64_t to, cudaStream_t s, int stall) {
    switch (BN) {
#define PBQ_BN(X) case X: return launch_tc_bn<NPROD, X, TF32>(m, tiles, KI, G, smax, part, status, to, s, stall);
        PBQ_BN(16) PBQ_BN(32) PBQ_BN(48) PBQ_BN(64) PBQ_BN(80) PBQ_BN(96) PBQ_BN(112) PBQ_BN(128)
        PBQ_BN(144) PBQ_BN(160) PBQ_BN(176) PBQ_BN(192) PBQ_BN(208) PBQ_BN(224)
#undef PBQ_BN
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

TcGeom tc_geometry(int64_t rows, int64_t K, int N, int num_sms, bool tf32) {
    TcGeom g;
    g.BN = (int)round_up(N, 16);
    g.tiles = (rows + kTcBM - 1) / kTcBM;
    g.KI = (int)((K + tc_bk(tf32) - 1) / tc_bk(tf32));
    const int64_t T = g.tiles * g.KI;
    g.G = (int)(T < num_sms ? T : num_sms);
    if (g.G < 1) g.G = 1;
    // most segments a CTA can touch: its share spans at most ceil(share / KI) + 1 tiles
    const int64_t share = (T + g.G - 1) / g.G;
    g.smax = (int)((share + g.KI - 1) / g.KI + 1);
    g.part_floats = (int64_t)g.G * g.smax * kTcBM * g.BN;
    return g;
}

int64_t tc_ld(int64_t K, bool tf32) { return round_up(K, tc_bk(tf32)); }

cudaError_t launch_tc_product(int nprod, const TcOperands& op, const TcGeom& g, float* part, double* C, int64_t ldc,
                              uint32_t* status, cudaStream_t s, cudaEvent_t after_gemm, int stall) {
    if (op.N < 1 || op.N > kMaxEll || (nprod != 1 && nprod != 3)) return cudaErrorInvalidValue;
    CUtensorMap maps[4];
    const bool t = op.tf32 != 0;
    if (!make_map(&maps[0], op.Ahi, op.rows, op.K, op.lda, kTcBM, t)) return cudaErrorInvalidValue;
    if (!make_map(&maps[1], op.Alo ? op.Alo : op.Ahi, op.rows, op.K, op.lda, kTcBM, t)) return cudaErrorInvalidValue;
    if (!make_map(&maps[2], op.Bhi, op.N, op.K, op.ldb, g.BN, t)) return cudaErrorInvalidValue;
    if (!make_map(&maps[3], op.Blo ? op.Blo : op.Bhi, op.N, op.K, op.ldb, g.BN, t)) return cudaErrorInvalidValue;
    // a stalled test launch gives up after 50 ms; real launches after 2 s
    const uint64_t timeout_ns = stall ? 50000000ull : 2000000000ull;
    cudaError_t e;
    if (t) e = nprod == 3 ? launch_tc_nprod<3, true>(g.BN, maps, g.tiles, g.KI, g.G, g.smax, part, status, timeout_ns, s, stall)
                          : launch_tc_nprod<1, true>(g.BN, maps, g.tiles, g.KI, g.G, g.smax, part, status, timeout_ns, s, stall);
    else e = nprod == 3 ? launch_tc_nprod<3, false>(g.BN, maps, g.tiles, g.KI, g.G, g.smax, part, status, timeout_ns, s, stall)
                        : launch_tc_nprod<1, false>(g.BN, maps, g.tiles, g.KI, g.G, g.smax, part, status, timeout_ns, s, stall);
    if (e != cudaSuccess) return e;
    if (after_gemm && (e = cudaEventRecord(after_gemm, s)) != cudaSuccess) return e;
    const int64_t total = op.rows * (int64_t)op.N;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_tc_reduce<<<(unsigned)blocks, 256, 0, s>>>(op.rows, op.N, g.BN, g.tiles, g.KI, g.G, g.smax, part, C, ldc);
    count_launches(1);
    return cudaGetLastError();
}

// 64 x 64 tiles of A, one per CTA (split_tile64).
template <typename Tin, typename SP>
__global__ void __launch_bounds__(256)
k_split_a(int64_t m, int64_t n, const Tin* __restrict__ A, int64_t lda, typename SP::T* __restrict__ hi,
          typename SP::T* __restrict__ lo, int64_t ldh, typename SP::T* __restrict__ thi,
          typename SP::T* __restrict__ tlo, int64_t ldt, int vec_ok) {
    using T = typename SP::T;
    constexpr int PAD = 16 / (int)sizeof(T);
    __shared__ __align__(16) T sh[64][64 + PAD];
    __shared__ __align__(16) T sl[64][64 + PAD];
    split_tile64<Tin, SP>((int64_t)blockIdx.y * 64, (int64_t)blockIdx.x * 64, m, n, A, lda, hi, lo, ldh, thi, tlo, ldt,
                          vec_ok, sh, sl);
}

template <typename SP>
static void split_a_t(dim3 grid, dim3 block, int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, void* hi,
                      void* lo, int64_t ldh, void* thi, void* tlo, int64_t ldt, cudaStream_t s) {
    using T = typename SP::T;
    auto al16 = [](const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; };
    const int vec_ok = al16(A) && al16(hi) && al16(lo) && al16(thi) && al16(tlo) &&
                       ((lda * (a_f32 ? 4 : 8)) % 16 == 0) && ((ldh * (int64_t)sizeof(T)) % 16 == 0) &&
                       ((ldt * (int64_t)sizeof(T)) % 16 == 0);
    if (a_f32)
        k_split_a<float, SP><<<grid, block, 0, s>>>(m, n, (const float*)A, lda, (T*)hi, (T*)lo, ldh, (T*)thi, (T*)tlo,
                                                   ldt, vec_ok);
    else
        k_split_a<double, SP><<<grid, block, 0, s>>>(m, n, (const double*)A, lda, (T*)hi, (T*)lo, ldh, (T*)thi,
                                                    (T*)tlo, ldt, vec_ok);
}

cudaError_t launch_split_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, void* hi, void* lo, int64_t ldh,
                           void* thi, void* tlo, int64_t ldt, cudaStream_t s, bool tf32) {
    dim3 grid((unsigned)((n + 63) / 64), (unsigned)((m + 63) / 64)), block(256);
    if (tf32) split_a_t<SplitTf32>(grid, block, m, n, A, a_f32, lda, hi, lo, ldh, thi, tlo, ldt, s);
    else split_a_t<SplitBf16>(grid, block, m, n, A, a_f32, lda, hi, lo, ldh, thi, tlo, ldt, s);
    count_launches(1);
    return cudaGetLastError();
}

// Panel P (rows x N FP64, ld ldp) -> transposed hi/lo (N x rows, ld ldt).
template <typename SP>
__global__ void k_split_panel_t(int64_t rows, int N, const double* __restrict__ P, int64_t ldp,
                                typename SP::T* __restrict__ thi, typename SP::T* __restrict__ tlo, int64_t ldt) {
    const int64_t total = rows * (int64_t)N;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / rows);
        const int64_t r = e - (int64_t)j * rows;
        const double x = P[r * ldp + j];
        const typename SP::T h = SP::rn(x);
        thi[(int64_t)j * ldt + r] = h;
        if (tlo) tlo[(int64_t)j * ldt + r] = SP::rn(x - (double)SP::back(h));
    }
}

cudaError_t launch_split_panel_t(int64_t rows, int N, const double* P, int64_t ldp, void* thi, void* tlo, int64_t ldt,
                                 cudaStream_t s, bool tf32) {
    const int64_t total = rows * (int64_t)N;
    int64_t blocks = (total + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    if (tf32) k_split_panel_t<SplitTf32><<<(unsigned)blocks, 256, 0, s>>>(rows, N, P, ldp, (float*)thi, (float*)tlo, ldt);
    else k_split_panel_t<SplitBf16><<<(unsigned)blocks, 256, 0, s>>>(rows, N, P, ldp, (__nv_bfloat16*)thi,
                                                                    (__nv_bfloat16*)tlo, ldt);
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq
