// Internal interface of the FP64-accurate tensor-core products (kernels_oz.cu).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace pbq {

constexpr int kOzDigits = 8;    // balanced base-128 digits per element (56 bits)
constexpr int kOzBM = 128;      // output rows per tile (one TMEM lane per row)
constexpr int kOzBN = 48;       // output columns per tile
constexpr int kOzBK = 32;       // contraction depth of one shared-memory stage

// One operand in digit form: kOzDigits BF16 matrices of `rows` x K and the
// per-row maximum biased FP64 exponent eraw[rows] (the row scale is
// 2^(eraw - 1021)).  Layout ("k-chunked"): digit s, row r, contraction index
// k at S[s * rows * Kp + (k / 32) * rows * 32 + r * 32 + k % 32], Kp = K
// rounded up to 32 with zero digits, so the 32-deep block of a row tile that
// one stage loads is a single contiguous run per digit.
struct OzOperand {
    const void* S = nullptr;
    int64_t rows = 0, K = 0;
    const int* eraw = nullptr;
};
__host__ __device__ inline int64_t oz_kpad(int64_t K) { return (K + 31) / 32 * 32; }
// Bytes of the digits of a rows x K operand.
inline size_t oz_digit_bytes(int64_t rows, int64_t K) { return 2 * (size_t)kOzDigits * (size_t)rows * oz_kpad(K); }

// Work split of one product C (Mrows x N) = X Y^T over K: 128 x 48 tiles
// (with `upper`, only the tiles that touch the upper triangle), stream-K over
// (tile, 32-deep chunk) iterations; a tile split between CTAs is summed in
// its own pair of int64 accumulators per element (part_doubles in all).
struct OzGeom {
    int64_t tiles = 0;
    int NT = 1, KI = 1, G = 1, upper = 0;
    int lock = 1;   // > 1: the NT column tiles of a row tile on NT CTAs in lockstep
    int tilewise = 0;   // 1: whole tiles per CTA (no split, no fix-up)
    int64_t part_doubles = 0;
};
OzGeom oz_geometry(int64_t Mrows, int N, int64_t K, bool upper, int num_sms);

// C[i*ldc + j] = sum_k X[i][k] Y[j][k] (FP64), i < X.rows, j < Y.rows, in one
// launch.  X.K == Y.K is the contraction length.  part: >= g.part_doubles
// doubles (int64 accumulators); part and cnt (>= 12 g.tiles ints) zero on
// entry and left zero (a call that timed out may leave them nonzero: clear
// them before the next one).
// cond (device, optional): nothing runs when *cond == 0.
cudaError_t launch_oz_product(const OzOperand& X, const OzOperand& Y, const OzGeom& g, double* part, int* cnt,
                              double* C, int64_t ldc, uint32_t* status, const int* cond, cudaStream_t s,
                              cudaEvent_t after_gemm = nullptr);

// Panel P (rows x N FP64, ld ldp) as the operand P^T (N rows, contraction
// over the panel rows): column exponents into eraw[N] and digits into S, laid
// out as an OzOperand {S, N, rows}.
cudaError_t launch_oz_panel(int64_t rows, int N, const double* P, int64_t ldp, int* eraw, void* S, const int* cond,
                            cudaStream_t s);

// A row-major FP64 matrix P (rows x K, ld ldp) as the operand {S, rows, K}
// with row exponents er[rows], in one kernel (one warp per row).
cudaError_t launch_oz_rows(int64_t rows, int64_t K, const double* P, int64_t ldp, int* er, void* S, const int* cond,
                           cudaStream_t s);

// A (m x n, FP64 or FP32, lda) as both operands: A itself (OzOperand {Srow,
// m, n}, row exponents er) and A^T ({Scol, n, m}, column exponents ec).
// Either digit set may be null (its exponents are still formed).
// cond (device, optional): nothing runs when *cond == 0.
cudaError_t launch_oz_a(int64_t m, int64_t n, const void* A, int a_f32, int64_t lda, int* er, int* ec, void* Srow,
                        void* Scol, cudaStream_t s, const int* cond = nullptr);

// ---------------------------------------------------------------------------
// Grouped form (many independent products per launch, for the batched path)
// ---------------------------------------------------------------------------
// Tensor map (128 bytes at map128) over the digits of the operand {S, rows, K}
// for tiles of box_rows rows: kOzBM for the X side, kOzBN for the Y side.
bool make_oz_map(void* map128, const void* S, int64_t rows, int64_t K, int box_rows);

// One 128 x 48 tile C[m0 .. m0 + 127][n0 .. n0 + 47] (clipped to Rx x Ry) of
// one product C = X Y^T, over the whole contraction (KI chunks of 32) in one
// CTA, written once: no partials, deterministic.
struct OzListUnit {
    int mapx, mapy;        // maps (in the table passed to the launch) of X (box kOzBM) and Y (box kOzBN)
    int m0, n0;
    int KI;
    int Rx, Ry;
    int pad_;
    const int* ex;         // biased row exponents of X (Rx) and of Y (Ry)
    const int* ey;
    double* C;
    int64_t ldc;
    const int* cond;       // skip when *cond == 0 (null: always run)
};

// Persistent launch of min(G, n) CTAs; CTA c runs units c, c + G, ... (the
// host sorts them longest first).  status: kStTimeout on a wait that expired.
cudaError_t launch_oz_list(const void* maps, const OzListUnit* units, int n, int G, uint32_t* status, cudaStream_t s);

// kOzPanelRows rows of one panel P (rows x N FP64, ld ldp, N <= 256) seen as
// the operand P^T = {S, N, rows}.
constexpr int kOzPanelRows = 128;
struct OzPanelUnit {
    const double* P;
    int64_t ldp, rows, r0;
    int N;
    int pad_;
    int* eraw;             // column exponents (N)
    void* S;
    const int* cond;
};
// Column exponents: atomicMax of each unit's column maxima into eraw, which
// must be zero before the launch.
cudaError_t launch_oz_panel_exp_list(const OzPanelUnit* units, int n, cudaStream_t s);
// Digits of every unit's rows, up to the padded contraction length (the
// units must cover oz_kpad(rows)), from the final eraw.
cudaError_t launch_oz_panel_slice_list(const OzPanelUnit* units, int n, cudaStream_t s);
// Row form: rows r0 .. r0 + 15 of a row-major P (rows x N, ld ldp) as the
// operand {S, rows, N}, row exponents into eraw (one warp per row, no zeroing needed).
constexpr int kOzRowsPerUnit = 16;
cudaError_t launch_oz_rows_list(const OzPanelUnit* units, int n, cudaStream_t s);

}  // namespace pbq
