// Grouped tcgen05 products (kind::tf32) for the batched path: many matrices'
// products C_i = op(A_i) Y_i in one launch.  Each unit is one 128-row tile of
// one matrix over its full contraction, so every output element is produced
// by exactly one CTA (deterministic, no partials).  Persistent CTAs (one per
// SM) take units c, c + G, ... of a host-sorted list.  Operands are split
// TF32 hi/lo (hi = RN_tf32(x), lo = RN_tf32(x - hi)); the split mode issues
// hi*hi + lo*hi + hi*lo per k-step.  TMEM accumulation is cut into chunks of
// kTcKC k-blocks added round-to-nearest into FP32 registers, as in
// kernels_tc.cu.  Every wait is bounded.
#include <cuda.h>
#include <cstdint>

#include "internal.h"
#include "split_device.cuh"
#include "tc_device.cuh"
#include "tc_internal.h"

namespace pbq {

using namespace tcdev;

namespace {
constexpr int kLBM = 128;        // tile rows
constexpr int kLBK = 32;         // FP32 elements per k-block (one 128-byte swizzle row)
constexpr int kLKC = 16;         // k-blocks per TMEM chunk (512-deep sums)
constexpr int kLThreads = 320;
}  // namespace

template <int NPROD, int STAGES>
__global__ void __launch_bounds__(kLThreads, 1)
k_tc_list(const CUtensorMap* __restrict__ maps, const TcUnit* __restrict__ units, int nunits,
          uint32_t* __restrict__ status, uint64_t timeout_ns) {
    constexpr int BNMAX = kTcListBNMax;
    constexpr uint32_t A_BYTES = kLBM * kLBK * 4;
    constexpr uint32_t B_BYTES = BNMAX * kLBK * 4;
    constexpr uint32_t STAGE_BYTES = (A_BYTES + B_BYTES) * (NPROD == 3 ? 2 : 1);
    constexpr uint32_t ACC_COLS = BNMAX;   // 128 columns per accumulator buffer

    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    __shared__ uint64_t full_bar[STAGES], empty_bar[STAGES], accf_bar[2], acce_bar[2], drain_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ volatile int abort_sh;
    __shared__ int issued_sh, consumed_sh;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int G = gridDim.x, c = blockIdx.x;
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
        unsigned char* base = smem + (size_t)s * STAGE_BYTES;
        switch (which) {
            case 0: return base;                               // A hi
            case 1: return base + A_BYTES;                     // B hi
            case 2: return base + A_BYTES + B_BYTES;           // A lo
            default: return base + 2 * A_BYTES + B_BYTES;      // B lo
        }
    };

    if (warp == 0) {
        if (lane == 0) {
            int li = 0;
            bool ok = true;
            for (int u = c; ok && u < nunits; u += G) {
                const TcUnit U = units[u];
                const uint32_t tx = (A_BYTES + (uint32_t)U.npad * kLBK * 4) * (NPROD == 3 ? 2 : 1);
                for (int kb = 0; kb < U.KI; ++kb, ++li) {
                    const int s = li % STAGES;
                    if (li >= STAGES && !mbar_wait(&empty_bar[s], (uint32_t)((li / STAGES - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    const int k0 = kb * kLBK;
                    mbar_expect_tx(&full_bar[s], tx);
                    tma_load_2d(stage_ptr(s, 0), &maps[U.amap_hi], &full_bar[s], k0, U.m0);
                    tma_load_2d(stage_ptr(s, 1), &maps[U.bmap_hi], &full_bar[s], k0, 0);
                    if (NPROD == 3) {
                        tma_load_2d(stage_ptr(s, 2), &maps[U.amap_lo], &full_bar[s], k0, U.m0);
                        tma_load_2d(stage_ptr(s, 3), &maps[U.bmap_lo], &full_bar[s], k0, 0);
                    }
                    issued_sh = li + 1;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int li = 0, chunk = 0;
            bool ok = true;
            for (int u = c; ok && u < nunits; u += G) {
                const TcUnit U = units[u];
                const uint32_t idesc = idesc_tf32_f32(kLBM, U.npad);
                for (int kb0 = 0; ok && kb0 < U.KI; kb0 += kLKC) {
                    const int kb1 = (kb0 + kLKC < U.KI) ? kb0 + kLKC : U.KI;
                    const int b = chunk & 1;
                    if (chunk >= 2 && !mbar_wait(&acce_bar[b], (uint32_t)((chunk / 2 - 1) & 1), deadline, &abort_sh)) {
                        abort_sh = 1;
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t dt = tmem_base + (uint32_t)b * ACC_COLS;
                    for (int kb = kb0; kb < kb1; ++kb, ++li) {
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
                            const uint32_t off = kk * 32;   // 8 TF32 = 32 bytes along the swizzled row
                            tc_mma_tf32(dt, sdesc_k_sw128(ahi + off), sdesc_k_sw128(bhi + off), idesc,
                                        (kb == kb0 && kk == 0) ? 0u : 1u);
                            if (NPROD == 3) {
                                tc_mma_tf32(dt, sdesc_k_sw128(alo + off), sdesc_k_sw128(bhi + off), idesc, 1u);
                                tc_mma_tf32(dt, sdesc_k_sw128(ahi + off), sdesc_k_sw128(blo + off), idesc, 1u);
                            }
                        }
                        tc_commit(&empty_bar[s]);
                        consumed_sh = li + 1;
                    }
                    if (!ok) break;
                    tc_commit(&accf_bar[b]);
                    ++chunk;
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
        constexpr int NCH = BNMAX / 16;
        constexpr int HCH = (NCH + 1) / 2;
        const int q = warp & 3;
        const int h = (warp - 2) >> 2;
        const int row = q * 32 + lane;
        float acc[HCH][16];
        int chunk = 0;
        bool ok = true;
        for (int u = c; ok && u < nunits; u += G) {
            const TcUnit U = units[u];
            const int ng = U.npad / 16;
#pragma unroll
            for (int g = 0; g < HCH; ++g)
#pragma unroll
                for (int i = 0; i < 16; ++i) acc[g][i] = 0.f;
            for (int kb0 = 0; kb0 < U.KI; kb0 += kLKC) {
                const int b = chunk & 1;
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
                    if (grp < ng) {
                        float v[16];
                        tmem_ld16(taddr + grp * 16, v);
#pragma unroll
                        for (int i = 0; i < 16; ++i) acc[g][i] += v[i];
                    }
                }
                tc_fence_before();
                mbar_arrive(&acce_bar[b]);
                ++chunk;
            }
            if (!ok) break;
            const int64_t gr = (int64_t)U.m0 + row;
            if (gr < U.rows) {
                double* dst = U.C + gr * U.ldc;
#pragma unroll
                for (int g = 0; g < HCH; ++g) {
                    const int grp = h * HCH + g;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const int col = grp * 16 + i;
                        if (grp < ng && col < U.N) dst[col] = (double)acc[g][i];
                    }
                }
            }
        }
    }

    __syncthreads();
    if (threadIdx.x == 0) {
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

template <int NPROD>
static cudaError_t launch_tc_list_n(const void* maps, const TcUnit* units, int nunits, int G, uint32_t* status,
                                    cudaStream_t s) {
    constexpr uint32_t A_BYTES = kLBM * kLBK * 4, B_BYTES = kTcListBNMax * kLBK * 4;
    constexpr uint32_t STAGE = (A_BYTES + B_BYTES) * (NPROD == 3 ? 2 : 1);
    constexpr int STAGES = (int)((216u * 1024u) / STAGE) > 8 ? 8 : (int)((216u * 1024u) / STAGE);
    static_assert(STAGES >= 2, "stage ring too small");
    const size_t smem = (size_t)STAGES * STAGE + 1024;
    auto kern = k_tc_list<NPROD, STAGES>;
    cudaError_t e = func_smem_attr((const void*)kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<G, kLThreads, smem, s>>>((const CUtensorMap*)maps, units, nunits, status, 2000000000ull);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_tc_list(int nprod, const void* maps, const TcUnit* units, int nunits, int num_sms, uint32_t* status,
                           cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    const int G = nunits < num_sms ? nunits : num_sms;
    if (nprod == 3) return launch_tc_list_n<3>(maps, units, nunits, G, status, s);
    if (nprod == 1) return launch_tc_list_n<1>(maps, units, nunits, G, status, s);
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// TF32 splits.  hi = RN_tf32(x) (cvt.rna), lo = RN_tf32(x - hi).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// Unit: rows r0 .. r0 + 63 of one matrix; CTA (unit, y) takes its 64 x 64
// tile y (split_tile64), CTAs past the matrix's width exit at once.
template <typename Tin>
__global__ void __launch_bounds__(256) k_split_tf32_list(const SplitUnit* __restrict__ units) {
    __shared__ __align__(16) float sh[64][68];
    __shared__ __align__(16) float sl[64][68];
    const SplitUnit& u = units[blockIdx.x];
    const int64_t c0 = (int64_t)blockIdx.y * 64;
    if (c0 >= u.n) return;
    split_tile64<Tin, SplitTf32>(u.r0, c0, u.m, u.n, (const Tin*)u.A, u.lda, u.hi, u.lo, u.ldh, u.thi, u.tlo, u.ldt,
                                 u.vec_ok, sh, sl);
}

cudaError_t launch_split_tf32_list(const SplitUnit* units, int nunits, int col_tiles, int a_f32, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    if (col_tiles < 1 || col_tiles > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)nunits, (unsigned)col_tiles);
    if (a_f32) k_split_tf32_list<float><<<grid, 256, 0, s>>>(units);
    else k_split_tf32_list<double><<<grid, 256, 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_split_panel_tf32_list(const PanelUnit* __restrict__ units) {
    const PanelUnit u = units[blockIdx.x];
    // panel rows [r0, r0 + rows) (u.Y, u.thi, u.tlo point at row 0 of the panel)
    const int64_t total = u.rows * (int64_t)u.N;
    for (int64_t e = threadIdx.x; e < total; e += blockDim.x) {
        const int j = (int)(e / u.rows);
        const int64_t r = u.r0 + (e - (int64_t)j * u.rows);
        const double x = u.Y[r * u.ldy + j];
        const float h = to_tf32((float)x);
        u.thi[(int64_t)j * u.ldt + r] = h;
        if (u.tlo) u.tlo[(int64_t)j * u.ldt + r] = to_tf32((float)(x - (double)h));
    }
}

cudaError_t launch_split_panel_tf32_list(const PanelUnit* units, int nunits, cudaStream_t s) {
    if (nunits <= 0) return cudaSuccess;
    k_split_panel_tf32_list<<<nunits, 256, 0, s>>>(units);
    count_launches(1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
typedef CUresult (*PFN_encodeTiledF)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                     const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

bool make_map_f32(void* map128, const void* base, int64_t rows, int64_t cols, int64_t ld, int box_rows) {
    static PFN_encodeTiledF fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return false;
        fn = (PFN_encodeTiledF)p;
    }
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
    cuuint32_t box[2] = {(cuuint32_t)kLBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn((CUtensorMap*)map128, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides, box,
              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace pbq
