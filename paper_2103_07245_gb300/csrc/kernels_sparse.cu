// Products with a sparse A (Section III-C: for z nonzeros the products with A
// and A^T cost O(z d) instead of O(m n d)).  A arrives in CSR form (rowptr,
// colind, values); A^T is built once per call as a second CSR (the CSC of A)
// whose entries keep, within each column, the order of A's CSR (ascending
// original position, i.e. by row), so both products are deterministic.
//
// Every kernel that indexes with the caller's structure runs only after the
// structure was checked on the device: rowptr[0] = 0, rowptr[m] = nnz,
// nondecreasing, and 0 <= colind < n.  A violation sets kStBadInput in the
// status word and the later kernels write zeros instead of reading through it.
#include <cstdint>

#include "internal.h"

namespace pbq {

namespace {

__device__ __forceinline__ bool bad_input(const uint32_t* status) {
    return (*(volatile const uint32_t*)status & kStBadInput) != 0;
}

// rowptr: first entry 0, last entry nnz, nondecreasing (entries 0 .. m).
__global__ void k_csr_check_rows(int64_t m, int64_t nnz, const int64_t* __restrict__ rowptr,
                                 uint32_t* __restrict__ status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= m; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rowptr[i];
        const bool bad = a < 0 || a > nnz || (i == 0 && a != 0) || (i == m && a != nnz) || (i > 0 && rowptr[i - 1] > a);
        if (bad) atomicOr(status, kStBadInput);
    }
}

// Column counts of A (the row counts of A^T); colind out of range is flagged.
// Reads only colind[0 .. nnz), whatever rowptr holds.
__global__ void k_csr_count_cols(int64_t nnz, int64_t n, const int32_t* __restrict__ colind, int* __restrict__ cnt,
                                 uint32_t* __restrict__ status) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = colind[e];
        if (c < 0 || (int64_t)c >= n) atomicOr(status, kStBadInput);
        else atomicAdd(&cnt[c], 1);
    }
}

// colptr[0 .. n] = exclusive prefix sums of cnt[0 .. n), by one CTA of 1024
// threads: contiguous chunks per thread, a shared-memory scan of the chunk
// sums, then each chunk written from its offset.
__global__ void __launch_bounds__(1024) k_csr_scan(int64_t n, const int* __restrict__ cnt, int64_t* __restrict__ colptr) {
    __shared__ int64_t part[1024];
    const int t = threadIdx.x;
    const int64_t chunk = (n + 1023) / 1024;
    const int64_t a = (int64_t)t * chunk, b = a + chunk < n ? a + chunk : n;
    int64_t s = 0;
    for (int64_t i = a; i < b; ++i) s += cnt[i];
    part[t] = s;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {   // inclusive Hillis-Steele scan
        const int64_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - s;   // exclusive offset of this chunk
    for (int64_t i = a; i < b; ++i) {
        colptr[i] = run;
        run += cnt[i];
    }
    if (t == 1023) colptr[n] = part[1023];
}

// Scatter: each entry e of row i gets a slot in its column's segment (slot
// order within a column is arbitrary here; k_csr_order_cols fixes it).
__global__ void k_csr_scatter(int64_t m, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ colind,
                              const int64_t* __restrict__ colptr, int* __restrict__ cursor, int32_t* __restrict__ srow,
                              int64_t* __restrict__ sorig, const uint32_t* __restrict__ status) {
    if (bad_input(status)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < m; i += nw) {
        for (int64_t e = rowptr[i] + lane; e < rowptr[i + 1]; e += 32) {
            const int32_t c = colind[e];
            const int64_t slot = colptr[c] + atomicAdd(&cursor[c], 1);
            srow[slot] = (int32_t)i;
            sorig[slot] = e;
        }
    }
}

// Within each column segment, entries in ascending original position: entry
// j's rank is the number of entries of the segment with a smaller original
// index (the indices are distinct).  One warp per column.
__global__ void k_csr_order_cols(int64_t n, const int64_t* __restrict__ colptr, const int32_t* __restrict__ srow,
                                 const int64_t* __restrict__ sorig, const double* __restrict__ values,
                                 int32_t* __restrict__ trow, double* __restrict__ tval,
                                 const uint32_t* __restrict__ status) {
    if (bad_input(status)) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < n; c += nw) {
        const int64_t s0 = colptr[c], s1 = colptr[c + 1];
        for (int64_t j = s0 + lane; j < s1; j += 32) {
            const int64_t key = sorig[j];
            int64_t rank = 0;
            for (int64_t x = s0; x < s1; ++x) rank += sorig[x] < key;
            trow[s0 + rank] = srow[j];
            tval[s0 + rank] = values[key];
        }
    }
}

// C (rows x l, ld ldc) = S X for a CSR S (ptr, idx, val) and a row-major X
// (ld ldx): one warp per row, lanes over the l columns in T chunks of 32.  A
// row's nonzeros are taken 32 at a time (one coalesced load per lane, then
// broadcast by shuffles).  The last chunk holds only r = l - 32 (T - 1)
// columns; with P = 2 (r <= 16) or 4 (r <= 8) it serves P nonzeros per
// instruction, lane group g = lane / (32 / P) taking the nonzeros j = g mod P
// (GB300 has 2 FP64 lanes per SM per clock, and a masked lane costs the same
// as a busy one).  Every output sums in CSR order, except that the last
// chunk's P interleaved partial sums are added at the end: deterministic.
template <int T, int P>
__global__ void __launch_bounds__(256)
k_csr_spmm(int64_t rows, const int64_t* __restrict__ ptr, const int32_t* __restrict__ idx,
           const double* __restrict__ val, const double* __restrict__ X, int64_t ldx, int l, double* __restrict__ C,
           int64_t ldc, const uint32_t* __restrict__ status) {
    constexpr int GW = 32 / P;   // lanes per nonzero in the last chunk
    const bool bad = bad_input(status);
    const int lane = threadIdx.x & 31;
    const int grp = lane / GW, glane = lane % GW;
    const int lastcol = 32 * (T - 1) + (P == 1 ? lane : glane);
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = w0; r < rows; r += nw) {
        double acc[T];
#pragma unroll
        for (int t = 0; t < T; ++t) acc[t] = 0.0;
        if (!bad) {
            const int64_t e1 = ptr[r + 1];
            for (int64_t e0 = ptr[r]; e0 < e1; e0 += 32) {
                const int64_t e = e0 + lane;
                int32_t cl = 0;
                double vl = 0.0;
                if (e < e1) {
                    cl = idx[e];
                    vl = val[e];
                }
                const int cntj = e1 - e0 < 32 ? (int)(e1 - e0) : 32;
                for (int j = 0; j < cntj; j += P) {
#pragma unroll
                    for (int u = 0; u < P; ++u) {   // full chunks: one nonzero at a time
                        if (T > 1 && j + u < cntj) {
                            const int32_t cj = __shfl_sync(0xffffffffu, cl, j + u);
                            const double vj = __shfl_sync(0xffffffffu, vl, j + u);
                            const double* xr = X + (int64_t)cj * ldx;
#pragma unroll
                            for (int t = 0; t < T - 1; ++t) acc[t] = fma(vj, xr[lane + 32 * t], acc[t]);
                        }
                    }
                    // last chunk: nonzero j + grp for this lane group
                    const int jj = j + grp;
                    const int32_t cj = __shfl_sync(0xffffffffu, cl, jj & 31);
                    const double vj = __shfl_sync(0xffffffffu, vl, jj & 31);
                    if (jj < cntj && lastcol < l) acc[T - 1] = fma(vj, X[(int64_t)cj * ldx + lastcol], acc[T - 1]);
                }
            }
            // add the last chunk's interleaved partial sums (group 0 keeps the total)
#pragma unroll
            for (int off = GW; off < 32; off <<= 1) acc[T - 1] += __shfl_xor_sync(0xffffffffu, acc[T - 1], off);
        }
        double* cr = C + r * ldc;
#pragma unroll
        for (int t = 0; t < T - 1; ++t) cr[lane + 32 * t] = acc[t];
        if (grp == 0 && lastcol < l) cr[lastcol] = acc[T - 1];
    }
}

unsigned grid_for(int64_t items, int per_block, int num_sms) {
    int64_t b = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)num_sms * 16;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

size_t csr_transpose_bytes(int64_t n, int64_t nnz) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    return al(sizeof(int) * (size_t)n) + al(sizeof(int64_t) * (size_t)(n + 1)) + al(sizeof(int32_t) * (size_t)nnz) +
           al(sizeof(int64_t) * (size_t)nnz) + al(sizeof(int32_t) * (size_t)nnz) + al(sizeof(double) * (size_t)nnz);
}

cudaError_t launch_csr_transpose(int64_t m, int64_t n, int64_t nnz, const int64_t* rowptr, const int32_t* colind,
                                 const double* values, void* scratch, CsrT* out, uint32_t* status, int num_sms,
                                 cudaStream_t s) {
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    char* b = (char*)scratch;
    int* cnt = (int*)b;
    b += al(sizeof(int) * (size_t)n);
    int64_t* colptr = (int64_t*)b;
    b += al(sizeof(int64_t) * (size_t)(n + 1));
    int32_t* srow = (int32_t*)b;
    b += al(sizeof(int32_t) * (size_t)nnz);
    int64_t* sorig = (int64_t*)b;
    b += al(sizeof(int64_t) * (size_t)nnz);
    int32_t* trow = (int32_t*)b;
    b += al(sizeof(int32_t) * (size_t)nnz);
    double* tval = (double*)b;
    out->ptr = colptr;
    out->idx = trow;
    out->val = tval;
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    k_csr_check_rows<<<grid_for(m + 1, 256, num_sms), 256, 0, s>>>(m, nnz, rowptr, status);
    if (nnz > 0) k_csr_count_cols<<<grid_for(nnz, 256, num_sms), 256, 0, s>>>(nnz, n, colind, cnt, status);
    k_csr_scan<<<1, 1024, 0, s>>>(n, cnt, colptr);
    if ((e = cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)n, s)) != cudaSuccess) return e;   // now the cursors
    k_csr_scatter<<<grid_for(m * 32, 256, num_sms), 256, 0, s>>>(m, rowptr, colind, colptr, cnt, srow, sorig, status);
    k_csr_order_cols<<<grid_for(n * 32, 256, num_sms), 256, 0, s>>>(n, colptr, srow, sorig, values, trow, tval, status);
    count_launches(nnz > 0 ? 5 : 4);
    return cudaGetLastError();
}

cudaError_t launch_csr_spmm(int64_t rows, const int64_t* ptr, const int32_t* idx, const double* val, const double* X,
                            int64_t ldx, int l, double* C, int64_t ldc, const uint32_t* status, int num_sms,
                            cudaStream_t s) {
    if (l < 1 || l > kMaxEll) return cudaErrorInvalidValue;
    const unsigned grid = grid_for(rows * 32, 256, num_sms);
    const int T = (l + 31) / 32, rem = l - 32 * (T - 1);
    const int P = rem <= 8 ? 4 : (rem <= 16 ? 2 : 1);
    switch (T * 8 + P) {
#define PBQ_S(TT, PP) case TT * 8 + PP: \
        k_csr_spmm<TT, PP><<<grid, 256, 0, s>>>(rows, ptr, idx, val, X, ldx, l, C, ldc, status); break;
        PBQ_S(1, 1) PBQ_S(1, 2) PBQ_S(1, 4) PBQ_S(2, 1) PBQ_S(2, 2) PBQ_S(2, 4) PBQ_S(3, 1) PBQ_S(3, 2) PBQ_S(3, 4)
        PBQ_S(4, 1) PBQ_S(4, 2) PBQ_S(4, 4) PBQ_S(5, 1) PBQ_S(5, 2) PBQ_S(5, 4) PBQ_S(6, 1) PBQ_S(6, 2) PBQ_S(6, 4)
        PBQ_S(7, 1) PBQ_S(7, 2) PBQ_S(7, 4)
#undef PBQ_S
        default: return cudaErrorInvalidValue;
    }
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pbq
