// C ABI and host driver of the PbP-QLP library (Algorithm 3 of Kaloorazi &
// Chen).  The plan holds sizes, split-K choices and the workspace layout; all
// device memory comes from the caller.  Every step of the factorization runs
// in this library's kernels on the plan's stream.
#include <climits>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <new>
#include <utility>
#include <vector>

#include "../../include/pbpqlp.h"
#include "internal.h"
#include "tc_internal.h"
#include "oz_internal.h"

using namespace pbq;

constexpr int kTimeClasses = 6;   // PBPQLP_TIME_PASS .. PBPQLP_TIME_OTHER

struct pbpqlp_plan_s {
    int64_t m = 0, n = 0;
    int k = 0, p = 0, q = 0, l = 0;
    uint64_t seed = 0;
    int mode = 0;
    cudaStream_t stream = nullptr;
    int64_t ldp = 0;      // leading dimension of the internal panels
    int num_sms = 152;
    // split-K choices: A passes (NN: M=m, K=n; TN: M=n, K=m) and Grams (K = m or n)
    int S_nn = 1, S_tn = 1, S_gm = 1, S_gn = 1;
    int64_t kc_nn = 0, kc_tn = 0, kc_gm = 0, kc_gn = 0;
    // workspace layout (byte offsets)
    size_t off_status = 0, off_ctl = 0, off_scal = 0, off_Xm = 0, off_Ym = 0, off_Dm = 0, off_Xn = 0, off_Yn = 0;
    size_t off_part = 0, off_G = 0, off_Rp = 0, off_R = 0, off_Pt = 0, off_work = 0, off_red = 0, total = 0;
    // mixed modes: BF16 copies of A and A^T, transposed panels, stream-K partials
    int nprod = 0;                      // 1 (BF16) or 3 (split BF16); 0 in FP64 mode
    int fault_stall = 0;                // PBPQLP_FAULT=tc_stall at plan creation (failure-detection test)
    bool tf32 = false;                  // TF32 operands (modes TF32, TF32X3) instead of BF16
    bool cluster_chol = false;          // Cholesky on an 8-CTA cluster (l > 128)
    bool cluster_qr = false;            // small QR on an 8-CTA cluster (l > 64)
    bool blocked = false;               // l > kMaxEll: blocked Cholesky and QR, products in column chunks
    int cw = 0;                         // column chunk of the products with A (<= kMaxEll)
    bool stream_a = false;              // PBPQLP_STREAM_A: A split / digitised per row block in every pass
    int64_t srows = 0;                  // rows per block of the streamed passes
    size_t off_acc = 0;                 // n x ldp FP64: partial sums of the streamed A^T passes
    size_t off_blk = 0;                 // work area of the blocked Cholesky / QR
    TcGeom g_nn, g_tn;                  // C = A Pbar (rows m, K n) and C = A^T Y (rows n, K m)
    int64_t ldk_n = 0, ldk_m = 0;       // leading dims of the BF16 copies (K rounded to 64)
    size_t off_Ahi = 0, off_Alo = 0, off_Athi = 0, off_Atlo = 0;
    size_t off_Bnhi = 0, off_Bnlo = 0, off_Bmhi = 0, off_Bmlo = 0, off_tcpart = 0;
    // FP64-accurate tensor-core products (digit form): Grams and R = Q^T D in
    // every mode (oz_gram), the products with A and A^T in MODE_FP64_EMU (emu)
    bool oz_gram = false, emu = false;
    OzGeom og_gm, og_gn, og_nn, og_tn;  // Grams over m / n rows; C = A Y; C = A^T Y
    size_t off_ozE1 = 0, off_ozE2 = 0, off_ozS1 = 0, off_ozS2 = 0, off_ozpart = 0, off_ozEb = 0, off_ozEs = 0;
    size_t off_ozcnt = 0, ozcnt_bytes = 0;   // stream-K fix-up counters (12 per tile), cleared per call
    size_t ozpart_bytes = 0;                 // stream-K fix-up accumulators (int64), cleared per call
    OzGeom og_qb;                       // Qb = Pbar Ptil (n rows, K = l)
    bool chol_inv = false;              // cluster Cholesky with T = R^{-T}; CholeskyQR solve as a digit product
    OzGeom og_tr_m, og_tr_n;            // Q = C T^T over m or n rows (K = l)
    size_t off_T = 0;
    size_t off_ozEr = 0, off_ozEc = 0, off_ozArow = 0, off_ozAcol = 0;
    void* last_ws = nullptr;
    // launch-sequence replay: after two pbpqlp_factor / _from calls in a row with the
    // same arguments the sequence is recorded once into a CUDA graph (on a private
    // stream) and replayed on the plan's stream while the arguments stay the same
    struct GraphKey {
        const void* A = nullptr; int64_t lda = 0; int a_dtype = 0; void* ws = nullptr;
        const double *omega = nullptr, *pbar0 = nullptr; int64_t ld0 = 0;
        double *pbar_out = nullptr, *Qa = nullptr, *L = nullptr, *Qb = nullptr;
        cudaStream_t stream = nullptr;
        bool operator==(const GraphKey& o) const {
            return A == o.A && lda == o.lda && a_dtype == o.a_dtype && ws == o.ws && omega == o.omega &&
                   pbar0 == o.pbar0 && ld0 == o.ld0 && pbar_out == o.pbar_out && Qa == o.Qa && L == o.L &&
                   Qb == o.Qb && stream == o.stream;
        }
    };
    bool graphs = true;                 // PBPQLP_NO_GRAPH=1 at plan creation: always launch eagerly
    bool seen = false;
    GraphKey last_key, graph_key;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    int64_t glaunches = 0;              // kernels in the recorded sequence (for the launch counter)
    // observability: CUDA event pairs around the launches of each timing
    // class (PBPQLP_TIME_*): bit c of timing_mask enables class c
    unsigned timing_mask = 0;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[kTimeClasses];
    size_t ev_used[kTimeClasses] = {};
    ~pbpqlp_plan_s() {
        for (auto& v : ev)
            for (auto& e : v) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
        if (gexec) cudaGraphExecDestroy(gexec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
    }
};

namespace {

struct Ws {
    uint32_t* status;
    int* ctl;
    double* scal;
    double *Xm, *Ym, *Dm, *Xn, *Yn, *part, *G, *Rp, *R, *Pt, *work, *red, *T;
    void* blk;
    void *Ahi, *Alo, *Athi, *Atlo, *Bnhi, *Bnlo, *Bmhi, *Bmlo;
    float* tcpart;
    double* acc;
    int *ozE1, *ozE2, *ozEr, *ozEc, *ozEb, *ozEs, *ozcnt;
    void *ozS1, *ozS2, *ozArow, *ozAcol;
    double* ozpart;
};

Ws carve(const pbpqlp_plan_s* P, void* base) {
    char* b = (char*)base;
    Ws w;
    w.status = (uint32_t*)(b + P->off_status);
    w.ctl = (int*)(b + P->off_ctl);
    w.scal = (double*)(b + P->off_scal);
    w.Xm = (double*)(b + P->off_Xm);
    w.Ym = (double*)(b + P->off_Ym);
    w.Dm = (double*)(b + P->off_Dm);
    w.Xn = (double*)(b + P->off_Xn);
    w.Yn = (double*)(b + P->off_Yn);
    w.part = (double*)(b + P->off_part);
    w.G = (double*)(b + P->off_G);
    w.Rp = (double*)(b + P->off_Rp);
    w.R = (double*)(b + P->off_R);
    w.Pt = (double*)(b + P->off_Pt);
    w.work = (double*)(b + P->off_work);
    w.red = (double*)(b + P->off_red);
    w.T = P->chol_inv ? (double*)(b + P->off_T) : nullptr;
    w.blk = P->blocked ? (void*)(b + P->off_blk) : nullptr;
    const bool mixed = P->nprod > 0, split = P->nprod == 3;
    w.Ahi = mixed ? (void*)(b + P->off_Ahi) : nullptr;
    w.Alo = split ? (void*)(b + P->off_Alo) : nullptr;
    w.Athi = mixed ? (void*)(b + P->off_Athi) : nullptr;
    w.Atlo = split ? (void*)(b + P->off_Atlo) : nullptr;
    w.Bnhi = mixed ? (void*)(b + P->off_Bnhi) : nullptr;
    w.Bnlo = split ? (void*)(b + P->off_Bnlo) : nullptr;
    w.Bmhi = mixed ? (void*)(b + P->off_Bmhi) : nullptr;
    w.Bmlo = split ? (void*)(b + P->off_Bmlo) : nullptr;
    w.tcpart = mixed ? (float*)(b + P->off_tcpart) : nullptr;
    w.acc = P->stream_a ? (double*)(b + P->off_acc) : nullptr;
    const bool oz = P->oz_gram || P->emu;
    w.ozE1 = oz ? (int*)(b + P->off_ozE1) : nullptr;
    w.ozE2 = oz ? (int*)(b + P->off_ozE2) : nullptr;
    w.ozS1 = oz ? (void*)(b + P->off_ozS1) : nullptr;
    w.ozS2 = oz ? (void*)(b + P->off_ozS2) : nullptr;
    w.ozpart = oz ? (double*)(b + P->off_ozpart) : nullptr;
    w.ozEb = oz ? (int*)(b + P->off_ozEb) : nullptr;
    w.ozEs = oz ? (int*)(b + P->off_ozEs) : nullptr;
    w.ozcnt = oz ? (int*)(b + P->off_ozcnt) : nullptr;
    w.ozEr = P->emu ? (int*)(b + P->off_ozEr) : nullptr;
    w.ozEc = P->emu ? (int*)(b + P->off_ozEc) : nullptr;
    w.ozArow = P->emu ? (void*)(b + P->off_ozArow) : nullptr;
    w.ozAcol = P->emu ? (void*)(b + P->off_ozAcol) : nullptr;
    return w;
}

// Split-K count for Mtiles output tiles over a contraction of K: the S that
// best fills whole waves of `slots` resident CTAs with chunks of >= min_chunk rows.
void choose_split(int64_t Mtiles, int64_t K, int64_t slots, int* S_out, int64_t* kc_out, int64_t min_chunk = 64) {
    int bestS = 1;
    double best = -1.0;
    const int64_t maxS = K / min_chunk > 1 ? K / min_chunk : 1;
    for (int64_t S = 1; S <= maxS && S <= 512; ++S) {
        const int64_t kc = round_up((K + S - 1) / S, kGemmBK);
        const int64_t Seff = (K + kc - 1) / kc;
        const int64_t ctas = Mtiles * Seff;
        const int64_t waves = (ctas + slots - 1) / slots;
        // efficiency: useful work over occupied slot-time, with per-CTA time ~ kc
        const double eff = (double)K * Mtiles / ((double)waves * slots * kc);
        if (eff > best + 1e-9) { best = eff; bestS = (int)Seff; }
        if (waves >= 8) break;
    }
    const int64_t kc = round_up((K + bestS - 1) / bestS, kGemmBK);
    *S_out = (int)((K + kc - 1) / kc);
    *kc_out = kc;
}

int cuda_err(cudaError_t e) { return e == cudaSuccess ? PBPQLP_OK : PBPQLP_ECUDA; }

#define PBQ_TRY(expr) do { cudaError_t e_ = PBQ_DBG(expr); if (e_ != cudaSuccess) return PBPQLP_ECUDA; } while (0)

// Event pair for the next timed launch group of class cls (nullptr pair when
// that class is not timed).
std::pair<cudaEvent_t, cudaEvent_t> next_events(pbpqlp_plan_s* P, int cls = PBPQLP_TIME_PASS) {
    if (!(P->timing_mask & (1u << cls))) return {nullptr, nullptr};
    auto& v = P->ev[cls];
    if (P->ev_used[cls] == v.size()) {
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return {nullptr, nullptr};
        v.emplace_back(a, b);
    }
    return v[P->ev_used[cls]++];
}

// Brackets the launches of one timing class between construction and end().
struct TimedGroup {
    cudaEvent_t b = nullptr;
    cudaStream_t s;
    TimedGroup(pbpqlp_plan_s* P, int cls) : s(P->stream) {
        const auto ev = next_events(P, cls);
        if (ev.first && cudaEventRecord(ev.first, s) == cudaSuccess) b = ev.second;
    }
    void end() {
        if (b) cudaEventRecord(b, s);
        b = nullptr;
    }
    ~TimedGroup() { end(); }
};

// C (M x l) = op(A) B through the split-K partial buffer when S > 1.  With
// `timed`, the GEMM kernel launch is bracketed by a plan event pair.
// Widths beyond kMaxEll run as column chunks of at most kMaxEll (each
// chunk one pass over A), all inside the one timed group.
int gemm_pass(pbpqlp_plan_s* P, const Ws& w, bool transA, int64_t M, int64_t K, const double* A, int64_t lda,
              const double* B, int64_t ldb, double* C, int64_t ldc, int N, int S, int64_t kc, bool timed = false) {
    cudaStream_t s = P->stream;
    const auto ev = timed ? next_events(P) : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
    const int nch = (N + kMaxEll - 1) / kMaxEll, cw = (N + nch - 1) / nch;
    const int64_t ps = M * P->ldp;
    for (int c0 = 0; c0 < N; c0 += cw) {
        const int nc = N - c0 < cw ? N - c0 : cw;
        if (S <= 1) {
            PBQ_TRY(launch_dgemm_skinny(transA, M, nc, K, A, lda, B + c0, ldb, C + c0, ldc, 1, K, 0, nullptr, s));
        } else {
            PBQ_TRY(launch_dgemm_skinny(transA, M, nc, K, A, lda, B + c0, ldb, w.part + c0, P->ldp, S, kc, ps, nullptr,
                                        s));
            PBQ_TRY(launch_reduce_partials(M, nc, S, w.part + c0, ps, P->ldp, C + c0, ldc, nullptr, s));
        }
    }
    if (ev.second) PBQ_TRY(cudaEventRecord(ev.second, s));
    return PBPQLP_OK;
}

// Mixed-mode product with A (transA = false: C = A Y, Y n x N) or A^T
// (C = A^T Y, Y m x N): the FP64 panel Y is split into the transposed BF16
// operand, then one tcgen05 product + deterministic stream-K reduction.
int tc_pass(pbpqlp_plan_s* P, const Ws& w, bool transA, const double* Y, int64_t ldy, int N, double* C, int64_t ldc,
            bool timed = false) {
    cudaStream_t s = P->stream;
    const auto ev = timed ? next_events(P) : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    // widths beyond kMaxEll: column chunks of the plan's chunk width; the
    // timed group starts at the first product (after its panel split)
    const int nch = (N + kMaxEll - 1) / kMaxEll, cw = (N + nch - 1) / nch;
    for (int c0 = 0; c0 < N; c0 += cw) {
        const int nc = N - c0 < cw ? N - c0 : cw;
        TcOperands op;
        const TcGeom* g;
        if (!transA) {
            PBQ_TRY(launch_split_panel_t(P->n, nc, Y + c0, ldy, w.Bnhi, w.Bnlo, P->ldk_n, s, P->tf32));
            op.Ahi = w.Ahi; op.Alo = w.Alo; op.rows = P->m; op.K = P->n; op.lda = P->ldk_n;
            op.Bhi = w.Bnhi; op.Blo = w.Bnlo; op.ldb = P->ldk_n;
            g = &P->g_nn;
        } else {
            PBQ_TRY(launch_split_panel_t(P->m, nc, Y + c0, ldy, w.Bmhi, w.Bmlo, P->ldk_m, s, P->tf32));
            op.Ahi = w.Athi; op.Alo = w.Atlo; op.rows = P->n; op.K = P->m; op.lda = P->ldk_m;
            op.Bhi = w.Bmhi; op.Blo = w.Bmlo; op.ldb = P->ldk_m;
            g = &P->g_tn;
        }
        op.N = nc;
        op.tf32 = P->tf32 ? 1 : 0;
        TcGeom gg = *g;
        if (nc != P->cw) gg = tc_geometry(op.rows, op.K, nc, P->num_sms, P->tf32);
        if (gg.part_floats > g->part_floats || gg.BN > g->BN) return PBPQLP_EINVAL;
        const bool last = c0 + nc >= N;
        if (c0 == 0 && ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
        PBQ_TRY(launch_tc_product(P->nprod, op, gg, w.tcpart, C + c0, ldc, w.status, s, last ? ev.second : nullptr,
                                  P->fault_stall));
    }
    return PBPQLP_OK;
}

// Split A once per factorization into the BF16 operands of both orientations.
int tc_prepare_a(const pbpqlp_plan_s* P, const Ws& w, const void* A, int a_f32, int64_t lda) {
    PBQ_TRY(launch_split_a(P->m, P->n, A, a_f32, lda, w.Ahi, w.Alo, P->ldk_n, w.Athi, w.Atlo, P->ldk_m, P->stream,
                           P->tf32));
    return PBPQLP_OK;
}

// Digit-form operand of a panel transposed: N rows (its columns), contraction over its `rows` rows.
OzOperand panel_digits(void* S, const int* E, int N, int64_t rows) {
    OzOperand op;
    op.S = S;
    op.rows = N;
    op.K = rows;
    op.eraw = E;
    return op;
}

// Emulated-FP64 product with A (transA = false: C = A Y, Y n x N) or A^T
// (C = A^T Y, Y m x N): digits of the panel, one tensor-core product over the
// digits of A prepared by emu_prepare_a, deterministic reduction.
int emu_pass(pbpqlp_plan_s* P, const Ws& w, bool transA, const double* Y, int64_t ldy, int N, double* C, int64_t ldc,
             bool timed = false) {
    cudaStream_t s = P->stream;
    const int64_t K = transA ? P->m : P->n;
    OzOperand X;
    X.S = transA ? w.ozAcol : w.ozArow;
    X.rows = transA ? P->n : P->m;
    X.K = K;
    X.eraw = transA ? w.ozEc : w.ozEr;
    const OzOperand Yd = panel_digits(w.ozS2, w.ozE2, N, K);
    PBQ_TRY(launch_oz_panel(K, N, Y, ldy, w.ozE2, w.ozS2, nullptr, s));
    OzGeom g = transA ? P->og_tn : P->og_nn;
    if (N != P->l) g = oz_geometry(X.rows, N, K, false, P->num_sms);
    const int64_t cap = transA ? P->og_tn.part_doubles : P->og_nn.part_doubles;
    if (g.part_doubles > cap) return PBPQLP_EINVAL;
    const auto ev = timed ? next_events(P) : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
    PBQ_TRY(launch_oz_product(X, Yd, g, w.ozpart, w.ozcnt, C, ldc, w.status, nullptr, s, ev.second));
    return PBPQLP_OK;
}

// Digits of A (row scales) and of A^T (column scales), once per factorization.
int emu_prepare_a(const pbpqlp_plan_s* P, const Ws& w, const void* A, int a_f32, int64_t lda) {
    PBQ_TRY(launch_oz_a(P->m, P->n, A, a_f32, lda, w.ozEr, w.ozEc, w.ozArow, w.ozAcol, P->stream));
    return PBPQLP_OK;
}

// Streamed products with A (PBPQLP_STREAM_A, the paper's pass-efficient
// remark of Section III-C: A stored where the device can read but not hold
// it): A is split (mixed modes) or digitised (MODE_FP64_EMU) one row block
// of srows rows at a time inside every pass.  C = A Y writes each block's rows
// of C; C = A^T Y = sum_b A_b^T Y_b adds the blocks' FP64 partial sums in
// block order (deterministic).
const char* row_block(const void* A, int a_f32, int64_t lda, int64_t r0) {
    return (const char*)A + (size_t)r0 * (size_t)lda * (a_f32 ? 4 : 8);
}

int tc_pass_stream(pbpqlp_plan_s* P, const Ws& w, bool transA, const void* A, int a_f32, int64_t lda,
                   const double* Y, int64_t ldy, int N, double* C, int64_t ldc, bool timed) {
    cudaStream_t s = P->stream;
    const auto ev = timed ? next_events(P) : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
    const int64_t m = P->m, n = P->n, R = P->srows;
    const int nch = (N + kMaxEll - 1) / kMaxEll, cw = (N + nch - 1) / nch;
    for (int c0 = 0; c0 < N; c0 += cw) {
        const int nc = N - c0 < cw ? N - c0 : cw;
        if (!transA) PBQ_TRY(launch_split_panel_t(n, nc, Y + c0, ldy, w.Bnhi, w.Bnlo, P->ldk_n, s, P->tf32));
        for (int64_t r0 = 0; r0 < m; r0 += R) {
            const int64_t rb = m - r0 < R ? m - r0 : R;
            TcOperands op;
            op.N = nc;
            op.tf32 = P->tf32 ? 1 : 0;
            double* dst;
            int64_t lddst;
            if (!transA) {
                PBQ_TRY(launch_split_a(rb, n, row_block(A, a_f32, lda, r0), a_f32, lda, w.Ahi, w.Alo, P->ldk_n,
                                       nullptr, nullptr, 0, s, P->tf32));
                op.Ahi = w.Ahi; op.Alo = w.Alo; op.rows = rb; op.K = n; op.lda = P->ldk_n;
                op.Bhi = w.Bnhi; op.Blo = w.Bnlo; op.ldb = P->ldk_n;
                dst = C + r0 * ldc + c0;
                lddst = ldc;
            } else {
                PBQ_TRY(launch_split_a(rb, n, row_block(A, a_f32, lda, r0), a_f32, lda, w.Ahi, w.Alo, P->ldk_n,
                                       w.Athi, w.Atlo, P->ldk_m, s, P->tf32));
                PBQ_TRY(launch_split_panel_t(rb, nc, Y + r0 * ldy + c0, ldy, w.Bmhi, w.Bmlo, P->ldk_m, s, P->tf32));
                op.Ahi = w.Athi; op.Alo = w.Atlo; op.rows = n; op.K = rb; op.lda = P->ldk_m;
                op.Bhi = w.Bmhi; op.Blo = w.Bmlo; op.ldb = P->ldk_m;
                dst = r0 == 0 ? C + c0 : w.acc;
                lddst = r0 == 0 ? ldc : P->ldp;
            }
            const TcGeom* g = transA ? &P->g_tn : &P->g_nn;
            const TcGeom gg = tc_geometry(op.rows, op.K, nc, P->num_sms, P->tf32);
            if (gg.part_floats > g->part_floats || gg.BN > g->BN) return PBPQLP_EINVAL;
            PBQ_TRY(launch_tc_product(P->nprod, op, gg, w.tcpart, dst, lddst, w.status, s, nullptr, P->fault_stall));
            if (transA && r0 > 0) PBQ_TRY(launch_add2d(n, nc, w.acc, P->ldp, C + c0, ldc, s));
        }
    }
    if (ev.second) PBQ_TRY(cudaEventRecord(ev.second, s));
    return PBPQLP_OK;
}

int emu_pass_stream(pbpqlp_plan_s* P, const Ws& w, bool transA, const void* A, int a_f32, int64_t lda,
                    const double* Y, int64_t ldy, int N, double* C, int64_t ldc, bool timed) {
    cudaStream_t s = P->stream;
    const auto ev = timed ? next_events(P) : std::pair<cudaEvent_t, cudaEvent_t>{nullptr, nullptr};
    if (ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
    const int64_t m = P->m, n = P->n, R = P->srows;
    if (!transA) PBQ_TRY(launch_oz_panel(n, N, Y, ldy, w.ozE2, w.ozS2, nullptr, s));
    for (int64_t r0 = 0; r0 < m; r0 += R) {
        const int64_t rb = m - r0 < R ? m - r0 : R;
        OzOperand X;
        double* dst;
        int64_t lddst;
        OzGeom g;
        if (!transA) {
            // the block's rows with their own row scales: the same digits as the whole A's rows
            PBQ_TRY(launch_oz_a(rb, n, row_block(A, a_f32, lda, r0), a_f32, lda, w.ozEr, w.ozEc, w.ozArow, nullptr, s));
            X.S = w.ozArow; X.rows = rb; X.K = n; X.eraw = w.ozEr;
            g = oz_geometry(rb, N, n, false, P->num_sms);
            dst = C + r0 * ldc;
            lddst = ldc;
        } else {
            // the block's transpose with column scales of the block
            PBQ_TRY(launch_oz_a(rb, n, row_block(A, a_f32, lda, r0), a_f32, lda, w.ozEr, w.ozEc, nullptr, w.ozAcol, s));
            PBQ_TRY(launch_oz_panel(rb, N, Y + r0 * ldy, ldy, w.ozE2, w.ozS2, nullptr, s));
            X.S = w.ozAcol; X.rows = n; X.K = rb; X.eraw = w.ozEc;
            g = oz_geometry(n, N, rb, false, P->num_sms);
            dst = r0 == 0 ? C : w.acc;
            lddst = r0 == 0 ? ldc : P->ldp;
        }
        const OzOperand Yd = panel_digits(w.ozS2, w.ozE2, N, transA ? rb : n);
        const int64_t cap = transA ? P->og_tn.part_doubles : P->og_nn.part_doubles;
        if (g.part_doubles > cap) return PBPQLP_EINVAL;
        PBQ_TRY(launch_oz_product(X, Yd, g, w.ozpart, w.ozcnt, dst, lddst, w.status, nullptr, s));
        if (transA && r0 > 0) PBQ_TRY(launch_add2d(n, N, w.acc, P->ldp, C, ldc, s));
    }
    if (ev.second) PBQ_TRY(cudaEventRecord(ev.second, s));
    return PBPQLP_OK;
}

// Orthonormalise X (rows x l, ld ldp) in place: CholeskyQR in pass pairs
// (X -> Y -> X).  Pair 1 is CholeskyQR2; pairs 2 and 3 run on the device
// only if a pass of the previous pair needed the shifted retry.
int orth(pbpqlp_plan_s* P, const Ws& w, int64_t rows, double* X, double* Y, int Sg, int64_t kcg) {
    cudaStream_t s = P->stream;
    const int l = P->l;
    const int64_t ldp = P->ldp;
    PBQ_TRY(cudaMemsetAsync(w.ctl, 0, 16 * sizeof(int), s));
    for (int pass = 1; pass <= 6; ++pass) {
        const double* src = (pass & 1) ? X : Y;
        double* dst = (pass & 1) ? Y : X;
        const int* cond = pass <= 2 ? nullptr : w.ctl + 8 + (pass + 1) / 2;
        const int64_t ps = (int64_t)l * ldp;
        // the Cholesky reads only the upper triangle of the Gram
        TimedGroup tg(P, PBPQLP_TIME_GRAM);
        if (P->oz_gram) {
            const OzOperand op = panel_digits(w.ozS1, w.ozE1, l, rows);
            PBQ_TRY(launch_oz_panel(rows, l, src, ldp, w.ozE1, w.ozS1, cond, s));
            PBQ_TRY(launch_oz_product(op, op, rows == P->m ? P->og_gm : P->og_gn, w.ozpart, w.ozcnt, w.G, l, w.status, cond,
                                      s));
        } else {
            PBQ_TRY(launch_upper_product(l, rows, src, src, ldp, w.part, ps, Sg, kcg, cond, s));
            PBQ_TRY(launch_reduce_partials(l, l, Sg, w.part, ps, ldp, w.G, l, cond, s, true));
        }
        tg.end();
        if (P->chol_inv) {
            // dst = src R^{-1} = src T^T as an FP64-accurate digit product
            TimedGroup tc(P, PBPQLP_TIME_CHOL);
            if (P->blocked) PBQ_TRY(launch_chol_inv_blocked(l, rows, w.G, w.T, w.blk, w.status, w.ctl, pass, s));
            else PBQ_TRY(launch_chol_inv(l, rows, w.G, w.Rp, w.T, w.status, w.ctl, pass, s));
            tc.end();
            TimedGroup ts(P, PBPQLP_TIME_SOLVE);
            OzOperand xd, yd;
            xd.S = w.ozS1; xd.rows = rows; xd.K = l; xd.eraw = w.ozEb;
            yd.S = w.ozS2; yd.rows = l; yd.K = l; yd.eraw = w.ozE2;
            PBQ_TRY(launch_oz_rows(rows, l, src, ldp, w.ozEb, w.ozS1, cond, s));
            PBQ_TRY(launch_oz_rows(l, l, w.T, l, w.ozE2, w.ozS2, cond, s));
            PBQ_TRY(launch_oz_product(xd, yd, rows == P->m ? P->og_tr_m : P->og_tr_n, w.ozpart, w.ozcnt, dst, ldp, w.status,
                                      cond, s));
            continue;
        }
        TimedGroup tc(P, PBPQLP_TIME_CHOL);
        if (P->cluster_chol) PBQ_TRY(launch_cholesky_cluster(l, rows, w.G, w.Rp, w.status, w.ctl, pass, s));
        else PBQ_TRY(launch_cholesky(l, rows, w.G, w.Rp, w.status, w.ctl, pass, s));
        tc.end();
        TimedGroup ts(P, PBPQLP_TIME_SOLVE);
        PBQ_TRY(launch_trsm_rows(rows, l, w.Rp, src, ldp, dst, ldp, cond, s, P->nprod > 0));
    }
    return PBPQLP_OK;
}

// A must be addressable by the device at the given address: device or managed
// memory, or pinned host memory mapped at the same address (out-of-core A).
// Anything else (pageable host memory) is rejected before any launch.
int check_device_addressable(const void* p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return PBPQLP_EINVAL;
    }
    if (at.type == cudaMemoryTypeUnregistered) return PBPQLP_EINVAL;
    if (at.type == cudaMemoryTypeHost && at.devicePointer != p) return PBPQLP_EINVAL;
    return PBPQLP_OK;
}

// Y (m x r, ld ldy) = Qa[:, :r] L[:r, :r] (both ld l).
cudaError_t qa_times_l(int64_t m, int r, const double* Qa, const double* L, int l, double* Y, int64_t ldy,
                       cudaStream_t s) {
    if (r <= kMaxEll) return launch_dgemm_skinny(false, m, r, r, Qa, l, L, l, Y, ldy, 1, r, 0, nullptr, s);
    return launch_dgemm_gen(false, false, m, r, r, 1.0, Qa, l, L, l, 0.0, Y, ldy, false, nullptr, 0, s);
}

int check_ws(pbpqlp_plan_t P, void* ws, size_t ws_bytes) {
    if (!ws || ws_bytes < P->total || ((uintptr_t)ws & 255u) != 0) return PBPQLP_EWORKSPACE;
    return PBPQLP_OK;
}

}  // namespace

extern "C" {

int pbpqlp_version(void) { return 1 * 10000 + 0 * 100 + 0; }

const char* pbpqlp_strerror(int st) {
    switch (st) {
        case PBPQLP_OK: return "ok";
        case PBPQLP_EINVAL: return "invalid argument";
        case PBPQLP_ENOMEM: return "host allocation failed";
        case PBPQLP_ECUDA: return "CUDA runtime error";
        case PBPQLP_ENONFINITE: return "non-finite value in input or intermediate panel";
        case PBPQLP_EBREAKDOWN: return "orthonormalisation broke down after shifted retries";
        case PBPQLP_ETIMEOUT: return "bounded device wait timed out";
        case PBPQLP_EUNSUPPORTED: return "mode or size not supported";
        case PBPQLP_EWORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

int pbpqlp_plan(pbpqlp_plan_t* out, int64_t m, int64_t n, int k, int p, int q, uint64_t seed, int mode,
                void* stream) {
    if (!out) return PBPQLP_EINVAL;
    *out = nullptr;
    const bool stream_a = (mode & PBPQLP_STREAM_A) != 0;
    mode &= ~PBPQLP_STREAM_A;
    const int64_t l64 = (int64_t)k + (int64_t)p;
    if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0 || q > 64) return PBPQLP_EINVAL;
    if (l64 > m || l64 > n || l64 > kMaxEllBlocked) return PBPQLP_EINVAL;
    if (mode < PBPQLP_MODE_FP64 || mode > PBPQLP_MODE_FP64_EMU) return PBPQLP_EINVAL;
    if (l64 > kMaxEll) {
        // the blocked l x l steps need the digit-form Grams and solve and the cluster kernels
        const char* nc = std::getenv("PBPQLP_NO_CLUSTER");
        const char* no = std::getenv("PBPQLP_NO_OZ_GRAM");
        if ((nc && nc[0] == '1') || (no && no[0] == '1') || !qr_blocked_fits((int)l64)) return PBPQLP_EUNSUPPORTED;
    }
    pbpqlp_plan_s* P = new (std::nothrow) pbpqlp_plan_s();
    if (!P) return PBPQLP_ENOMEM;
    P->m = m; P->n = n; P->k = k; P->p = p; P->q = q; P->l = (int)l64;
    P->seed = seed; P->mode = mode; P->stream = (cudaStream_t)stream;
    P->ldp = round_up(P->l, 8);
    P->blocked = P->l > kMaxEll;
    P->stream_a = stream_a && mode != PBPQLP_MODE_FP64;   // the FP64 passes read A in place already
    if (P->stream_a) {
        // rows per block: about 512 MB of staging (operand copies or digits of one block in both
        // orientations), a multiple of 128; PBPQLP_STREAM_ROWS overrides (tests use small blocks)
        const int64_t per_row = 32 * (n + 64);
        int64_t r = round_up((int64_t)(512ll << 20) / per_row, 128);
        const char* sr = std::getenv("PBPQLP_STREAM_ROWS");
        if (sr && std::atoll(sr) > 0) r = round_up(std::atoll(sr), 32);
        P->srows = r < m ? r : m;
    }
    {
        const int nch = (P->l + kMaxEll - 1) / kMaxEll;
        P->cw = (P->l + nch - 1) / nch;
    }
    {
        const char* nc = std::getenv("PBPQLP_NO_CLUSTER");
        P->cluster_chol = cholesky_cluster_fits(P->l) && !(nc && nc[0] == '1');
        P->cluster_qr = small_qr_cluster_fits(P->l) && !(nc && nc[0] == '1');
        const char* no = std::getenv("PBPQLP_NO_OZ_GRAM");
        P->oz_gram = !(no && no[0] == '1');
        const char* ng = std::getenv("PBPQLP_NO_GRAPH");
        P->graphs = !(ng && ng[0] == '1');
        P->emu = mode == PBPQLP_MODE_FP64_EMU;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            P->num_sms = sms;
    }
    const int64_t slots = (int64_t)P->num_sms * dgemm_skinny_occupancy(P->cw);
    const int64_t mt = (m + kGemmBM - 1) / kGemmBM, nt = (n + kGemmBM - 1) / kGemmBM;
    const int64_t lt = (P->l + kGemmBM - 1) / kGemmBM;
    choose_split(mt, n, slots, &P->S_nn, &P->kc_nn);
    choose_split(nt, m, slots, &P->S_tn, &P->kc_tn);
    // Grams and R = Q^T D are launched one 64-row tile at a time (upper triangle)
    (void)lt;
    choose_split(1, m, slots, &P->S_gm, &P->kc_gm, 32);
    choose_split(1, n, slots, &P->S_gn, &P->kc_gn, 32);

    const int64_t ldp = P->ldp, l = P->l;
    int64_t part = (int64_t)P->S_nn * m * ldp;
    part = part > (int64_t)P->S_tn * n * ldp ? part : (int64_t)P->S_tn * n * ldp;
    // FP64 FMA Grams and R = Q^T D (split-K partials), only without the digit form
    const int64_t pg = P->oz_gram ? 0 : (int64_t)(P->S_gm > P->S_gn ? P->S_gm : P->S_gn) * l * ldp;
    part = part > pg ? part : pg;
    const int64_t tiles = ((m + 63) / 64) * ((n + 63) / 64);   // residual partials of pbpqlp_error
    part = part > tiles ? part : tiles;
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = (size_t)round_up((int64_t)(off + bytes), 256); return o; };
    P->off_status = take(256);
    P->off_ctl = take(256);
    P->off_scal = take(256);
    P->off_Xm = take(sizeof(double) * m * ldp);
    P->off_Ym = take(sizeof(double) * m * ldp);
    P->off_Dm = take(sizeof(double) * m * ldp);
    P->off_Xn = take(sizeof(double) * n * ldp);
    P->off_Yn = take(sizeof(double) * n * ldp);
    P->off_part = take(sizeof(double) * (size_t)part);
    P->off_G = take(sizeof(double) * l * l);
    P->off_Rp = take(sizeof(double) * (packed_tri((int)l) + l));
    P->off_R = take(sizeof(double) * l * ldp);
    P->off_Pt = take(sizeof(double) * l * ldp);
    P->off_work = take(sizeof(double) * (2 * l * l + 2 * l));
    P->off_red = take(sizeof(double) * 2048);
    if (P->oz_gram || P->emu) {
        P->og_gm = oz_geometry(l, (int)l, m, true, P->num_sms);
        P->og_gn = oz_geometry(l, (int)l, n, true, P->num_sms);
        P->og_qb = oz_geometry(n, (int)l, l, false, P->num_sms);
        int64_t pd = P->og_gm.part_doubles > P->og_gn.part_doubles ? P->og_gm.part_doubles : P->og_gn.part_doubles;
        pd = pd > P->og_qb.part_doubles ? pd : P->og_qb.part_doubles;
        {
            const char* nc = std::getenv("PBPQLP_NO_CLUSTER");
            P->chol_inv = P->oz_gram && (P->blocked || chol_inv_fits(P->l)) && !(nc && nc[0] == '1');
        }
        if (P->chol_inv) {
            P->og_tr_m = oz_geometry(m, (int)l, l, false, P->num_sms);
            P->og_tr_n = oz_geometry(n, (int)l, l, false, P->num_sms);
            pd = pd > P->og_tr_m.part_doubles ? pd : P->og_tr_m.part_doubles;
            pd = pd > P->og_tr_n.part_doubles ? pd : P->og_tr_n.part_doubles;
            P->off_T = take(sizeof(double) * l * l);
        }
        if (P->emu) {
            const int64_t ra = P->stream_a ? P->srows : m;   // rows of A in one product
            P->og_nn = oz_geometry(ra, (int)l, n, false, P->num_sms);
            P->og_tn = oz_geometry(n, (int)l, ra, false, P->num_sms);
            // every column width a pass uses (l, or the chunk width and the last chunk)
            // and every row block (the last streamed block may be shorter) may split
            // differently: room for the largest
            const int widths[3] = {(int)l, P->cw, (int)(l % P->cw)};
            const int64_t rows[2] = {ra, P->stream_a ? m % ra : 0};
            for (int wd : widths)
                for (int64_t r : rows) {
                    if (wd < 1 || r < 1) continue;
                    const OzGeom a = oz_geometry(r, wd, n, false, P->num_sms);
                    const OzGeom b = oz_geometry(n, wd, r, false, P->num_sms);
                    if (a.part_doubles > P->og_nn.part_doubles) P->og_nn.part_doubles = a.part_doubles;
                    if (b.part_doubles > P->og_tn.part_doubles) P->og_tn.part_doubles = b.part_doubles;
                }
            pd = pd > P->og_nn.part_doubles ? pd : P->og_nn.part_doubles;
            pd = pd > P->og_tn.part_doubles ? pd : P->og_tn.part_doubles;
        }
        const size_t ne = (size_t)(l > 256 ? l : 256);   // per-column exponents of an l-column panel
        P->off_ozE1 = take(sizeof(int) * ne);
        P->off_ozE2 = take(sizeof(int) * ne);
        // a panel as the transposed operand (l rows, K = m or n) or as rows (n rows, K = l)
        const int64_t mx = m > n ? m : n;
        const size_t sz = oz_digit_bytes(l, mx) > oz_digit_bytes(mx, l) ? oz_digit_bytes(l, mx) : oz_digit_bytes(mx, l);
        P->off_ozS1 = take(sz);
        P->off_ozS2 = take(sz);
        P->off_ozEb = take(sizeof(int) * (size_t)mx);
        P->off_ozEs = take(sizeof(int) * ne);
        P->ozpart_bytes = sizeof(double) * (size_t)pd;
        P->off_ozpart = take(P->ozpart_bytes);
        {
            int64_t mt = 0;
            for (const OzGeom* g : {&P->og_gm, &P->og_gn, &P->og_qb, &P->og_nn, &P->og_tn, &P->og_tr_m, &P->og_tr_n})
                mt = mt > g->tiles ? mt : g->tiles;
            P->ozcnt_bytes = sizeof(int) * 12 * (size_t)mt;
            P->off_ozcnt = take(P->ozcnt_bytes);
        }
        if (P->emu && !P->stream_a) {
            P->off_ozEr = take(sizeof(int) * (size_t)m);
            P->off_ozEc = take(sizeof(int) * (size_t)n);
            P->off_ozArow = take(oz_digit_bytes(m, n));
            P->off_ozAcol = take(oz_digit_bytes(n, m));
        } else if (P->emu) {
            // one block's digits, in the orientation the pass needs (never both at once)
            const int64_t R = P->srows;
            P->off_ozEr = take(sizeof(int) * (size_t)R);
            P->off_ozEc = take(sizeof(int) * (size_t)n);
            const size_t a = oz_digit_bytes(R, n), b = oz_digit_bytes(n, R);
            P->off_ozArow = take(a > b ? a : b);
            P->off_ozAcol = P->off_ozArow;
        }
    }
    if (mode != PBPQLP_MODE_FP64 && mode != PBPQLP_MODE_FP64_EMU) {
        P->tf32 = (mode == PBPQLP_MODE_TF32 || mode == PBPQLP_MODE_TF32X3);
        P->nprod = (mode == PBPQLP_MODE_BF16X3 || mode == PBPQLP_MODE_TF32X3) ? 3 : 1;
        const char* fault = std::getenv("PBPQLP_FAULT");
        P->fault_stall = (fault && std::strcmp(fault, "tc_stall") == 0) ? 1 : 0;
        // streamed: copies of one row block (R rows; its transpose has ld tc_ld(R)) in place of A's
        const int64_t ra = P->stream_a ? P->srows : m;
        P->ldk_n = tc_ld(n, P->tf32);
        P->ldk_m = tc_ld(ra, P->tf32);
        P->g_nn = tc_geometry(ra, n, P->cw, P->num_sms, P->tf32);
        P->g_tn = tc_geometry(n, ra, P->cw, P->num_sms, P->tf32);
        if (P->stream_a && m % ra) {
            const TcGeom a = tc_geometry(m % ra, n, P->cw, P->num_sms, P->tf32);
            const TcGeom b = tc_geometry(n, m % ra, P->cw, P->num_sms, P->tf32);
            if (a.part_floats > P->g_nn.part_floats) P->g_nn.part_floats = a.part_floats;
            if (b.part_floats > P->g_tn.part_floats) P->g_tn.part_floats = b.part_floats;
        }
        const int64_t BN = P->g_nn.BN;
        const bool split = P->nprod == 3;
        const size_t es = P->tf32 ? 4 : 2;   // bytes per operand element
        P->off_Ahi = take(es * (size_t)ra * P->ldk_n);
        if (split) P->off_Alo = take(es * (size_t)ra * P->ldk_n);
        P->off_Athi = take(es * (size_t)n * P->ldk_m);
        if (split) P->off_Atlo = take(es * (size_t)n * P->ldk_m);
        P->off_Bnhi = take(es * (size_t)BN * P->ldk_n);
        if (split) P->off_Bnlo = take(es * (size_t)BN * P->ldk_n);
        P->off_Bmhi = take(es * (size_t)BN * P->ldk_m);
        if (split) P->off_Bmlo = take(es * (size_t)BN * P->ldk_m);
        const int64_t pf = P->g_nn.part_floats > P->g_tn.part_floats ? P->g_nn.part_floats : P->g_tn.part_floats;
        P->off_tcpart = take(sizeof(float) * (size_t)pf);
    }
    if (P->stream_a) P->off_acc = take(sizeof(double) * (size_t)n * ldp);
    if (P->blocked) {
        const size_t a = chol_inv_blocked_work_bytes(P->l), b = qr_blocked_work_bytes(P->l);
        P->off_blk = take(a > b ? a : b);
    }
    P->total = off;
    *out = P;
    return PBPQLP_OK;
}

int pbpqlp_plan_destroy(pbpqlp_plan_t plan) {
    delete plan;
    return PBPQLP_OK;
}

size_t pbpqlp_workspace_bytes(pbpqlp_plan_t plan) { return plan ? plan->total : 0; }

int pbpqlp_generate_omega(pbpqlp_plan_t P, double* omega) {
    if (!P || !omega) return PBPQLP_EINVAL;
    return cuda_err(launch_gaussian(P->seed, P->m, P->l, omega, P->l, P->stream));
}

}  // extern "C"

namespace {

// Algorithm 3 on the plan's workspace, with `product(transA, Y, C)` forming
// C = A Y (transA false, m rows) or C = A^T Y (n rows) for the plan's A.
// With pbar0 the run starts from that n x l basis (leading dimension ld0)
// in place of Phi, Eq. 3 and the first orth; pbar_out (optional) receives the
// basis after the power iterations; with Qa, L and Qb all null the run stops
// there (no projection pass).
template <class Product>
int run_factor(pbpqlp_plan_s* P, const Ws& w, Product&& product, const double* omega, double* Qa, double* L,
               double* Qb, const double* pbar0 = nullptr, int64_t ld0 = 0, double* pbar_out = nullptr) {
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n, ldp = P->ldp;
    const int l = P->l;
    int rc = PBPQLP_OK;
    if (pbar0) {
        PBQ_TRY(copy2d(pbar0, ld0, w.Xn, ldp, n, l, s));
    } else {
        // Phi (m x l)
        if (omega) PBQ_TRY(copy2d(omega, l, w.Xm, ldp, m, l, s));
        else PBQ_TRY(launch_gaussian(P->seed, m, l, w.Xm, ldp, s));
        // C = A^T Phi (Eq. 3); Pbar = orth(C) (Eq. 4)
        if ((rc = product(true, w.Xm, w.Xn))) return rc;
        if ((rc = orth(P, w, n, w.Xn, w.Yn, P->S_gn, P->kc_gn))) return rc;
    }
    // power iterations with an orth after every product (Section III-B)
    for (int it = 0; it < P->q; ++it) {
        if ((rc = product(false, w.Xn, w.Xm))) return rc;
        if ((rc = orth(P, w, m, w.Xm, w.Ym, P->S_gm, P->kc_gm))) return rc;
        if ((rc = product(true, w.Xm, w.Xn))) return rc;
        if ((rc = orth(P, w, n, w.Xn, w.Yn, P->S_gn, P->kc_gn))) return rc;
    }
    if (pbar_out) PBQ_TRY(copy2d(w.Xn, ldp, pbar_out, l, n, l, s));
    if (!Qa && !L && !Qb) return PBPQLP_OK;
    // D = A Pbar (Eq. 5); [Q, R] = qr(D) (Eq. 6) with R = Q^T D
    if ((rc = product(false, w.Xn, w.Dm))) return rc;
    PBQ_TRY(copy2d(w.Dm, ldp, w.Xm, ldp, m, l, s));
    if ((rc = orth(P, w, m, w.Xm, w.Ym, P->S_gm, P->kc_gm))) return rc;
    TimedGroup tr(P, PBPQLP_TIME_OTHER);
    if (P->oz_gram) {
        const OzOperand qd = panel_digits(w.ozS1, w.ozE1, l, m), dd = panel_digits(w.ozS2, w.ozE2, l, m);
        PBQ_TRY(launch_oz_panel(m, l, w.Xm, ldp, w.ozE1, w.ozS1, nullptr, s));
        PBQ_TRY(launch_oz_panel(m, l, w.Dm, ldp, w.ozE2, w.ozS2, nullptr, s));
        PBQ_TRY(launch_oz_product(qd, dd, P->og_gm, w.ozpart, w.ozcnt, w.R, l, w.status, nullptr, s));
    } else {
        const int64_t ps = (int64_t)l * ldp;
        PBQ_TRY(launch_upper_product(l, m, w.Xm, w.Dm, ldp, w.part, ps, P->S_gm, P->kc_gm, nullptr, s));
        PBQ_TRY(launch_reduce_partials(l, l, P->S_gm, w.part, ps, ldp, w.R, l, nullptr, s, true));
    }
    tr.end();
    // [Ptil, Rtil] = qr(R^T), L = Rtil^T (Eq. 7); Qb = Pbar Ptil (Eq. 8)
    TimedGroup tq(P, PBPQLP_TIME_SMALLQR);
    if (P->blocked) PBQ_TRY(launch_qr_blocked(l, w.R, L, w.Pt, w.blk, s));
    else if (P->cluster_qr) PBQ_TRY(launch_small_qr_cluster(l, w.R, L, w.Pt, s));
    else PBQ_TRY(launch_small_qr(l, w.R, L, w.Pt, w.work, s));
    tq.end();
    TimedGroup tb(P, PBPQLP_TIME_OTHER);
    if (P->oz_gram) {
        // Qb[i][j] = sum_k Pbar[i][k] Ptil[k][j]: Pbar by rows, Ptil^T by rows
        OzOperand xd, yd;
        xd.S = w.ozS1; xd.rows = n; xd.K = l; xd.eraw = w.ozEb;
        yd = panel_digits(w.ozS2, w.ozE2, l, l);
        PBQ_TRY(launch_oz_rows(n, l, w.Xn, ldp, w.ozEb, w.ozS1, nullptr, s));
        PBQ_TRY(launch_oz_panel(l, l, w.Pt, l, w.ozE2, w.ozS2, nullptr, s));
        PBQ_TRY(launch_oz_product(xd, yd, P->og_qb, w.ozpart, w.ozcnt, Qb, l, w.status, nullptr, s));
    } else {
        PBQ_TRY(launch_dgemm_skinny(false, n, l, l, w.Xn, ldp, w.Pt, l, Qb, l, 1, l, 0, nullptr, s));
    }
    PBQ_TRY(copy2d(w.Xm, ldp, Qa, l, m, l, s));
    return PBPQLP_OK;
}

}  // namespace

extern "C" {

static int enqueue_factor(pbpqlp_plan_t P, const void* Av, int64_t lda, int a_dtype, void* workspace,
                          const double* omega, const double* pbar0, int64_t ld0, double* pbar_out, double* Qa,
                          double* L, double* Qb);

static int factor_impl(pbpqlp_plan_t P, const void* Av, int64_t lda, int a_dtype, void* workspace, size_t ws_bytes,
                       const double* omega, const double* pbar0, int64_t ld0, double* pbar_out, double* Qa, double* L,
                       double* Qb) {
    const bool outs = Qa || L || Qb;
    if (!P || !Av || lda < P->n) return PBPQLP_EINVAL;
    if (outs ? !(Qa && L && Qb) : !pbar_out) return PBPQLP_EINVAL;
    if (pbar0 && ld0 < P->l) return PBPQLP_EINVAL;
    const bool mixed = P->nprod > 0;
    if ((mixed || P->emu) ? (a_dtype != PBPQLP_F64 && a_dtype != PBPQLP_F32) : a_dtype != PBPQLP_F64)
        return PBPQLP_EUNSUPPORTED;
    int rc = check_ws(P, workspace, ws_bytes);
    if (rc) return rc;
    if ((rc = check_device_addressable(Av))) return rc;
    P->last_ws = workspace;
    // eager launches while timing, and on a stream that is itself being captured
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (!P->graphs || P->timing_mask || cudaStreamIsCapturing(P->stream, &cs) != cudaSuccess ||
        cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    }
    pbpqlp_plan_s::GraphKey key;
    key.A = Av; key.lda = lda; key.a_dtype = a_dtype; key.ws = workspace; key.omega = omega; key.pbar0 = pbar0;
    key.ld0 = ld0; key.pbar_out = pbar_out; key.Qa = Qa; key.L = L; key.Qb = Qb; key.stream = P->stream;
    if (P->gexec && P->graph_key == key) {
        if (cudaGraphLaunch(P->gexec, P->stream) != cudaSuccess) return PBPQLP_ECUDA;
        count_launches(P->glaunches);
        return PBPQLP_OK;
    }
    if (!(P->seen && P->last_key == key)) {
        P->seen = true;
        P->last_key = key;
        return enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    }
    // the same arguments twice in a row: record the sequence once, replay it from now on
    cudaStream_t user = P->stream;
    if (!P->cap_stream && cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        P->cap_stream = nullptr;
        P->graphs = false;
        return enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        P->graphs = false;
        return enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    }
    P->stream = P->cap_stream;
    const int64_t n0 = launch_count();
    rc = enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    const int64_t nk = launch_count() - n0;
    const cudaError_t ec = cudaStreamEndCapture(P->cap_stream, &g);
    P->stream = user;
    cudaGraphExec_t ex = nullptr;
    if (rc != PBPQLP_OK || ec != cudaSuccess || !g || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        P->graphs = false;   // launch eagerly from now on (a real argument error repeats there)
        return enqueue_factor(P, Av, lda, a_dtype, workspace, omega, pbar0, ld0, pbar_out, Qa, L, Qb);
    }
    cudaGraphDestroy(g);
    if (P->gexec) cudaGraphExecDestroy(P->gexec);
    P->gexec = ex;
    P->graph_key = key;
    P->glaunches = nk;
    return cudaGraphLaunch(P->gexec, user) == cudaSuccess ? PBPQLP_OK : PBPQLP_ECUDA;
}

// The launch sequence of one factorization on the plan's stream (arguments checked).
static int enqueue_factor(pbpqlp_plan_t P, const void* Av, int64_t lda, int a_dtype, void* workspace,
                          const double* omega, const double* pbar0, int64_t ld0, double* pbar_out, double* Qa,
                          double* L, double* Qb) {
    int rc = PBPQLP_OK;
    const bool mixed = P->nprod > 0;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    const double* A = (const double*)Av;
    const int64_t m = P->m, n = P->n, ldp = P->ldp;
    const int l = P->l;
    PBQ_TRY(cudaMemsetAsync(w.status, 0, 256, s));
    if (w.ozcnt) PBQ_TRY(cudaMemsetAsync(w.ozcnt, 0, P->ozcnt_bytes, s));
    if (w.ozpart) PBQ_TRY(cudaMemsetAsync(w.ozpart, 0, P->ozpart_bytes, s));
    const int a_f32 = a_dtype == PBPQLP_F32;
    if (!P->stream_a && mixed && (rc = tc_prepare_a(P, w, Av, a_f32, lda))) return rc;
    if (!P->stream_a && P->emu && (rc = emu_prepare_a(P, w, Av, a_f32, lda))) return rc;
    // one product with A (transA = false: C = A Y) or A^T, in the plan's mode
    auto product = [&](bool transA, const double* Y, double* C) -> int {
        if (P->stream_a && mixed) return tc_pass_stream(P, w, transA, Av, a_f32, lda, Y, ldp, l, C, ldp, true);
        if (P->stream_a) return emu_pass_stream(P, w, transA, Av, a_f32, lda, Y, ldp, l, C, ldp, true);
        if (mixed) return tc_pass(P, w, transA, Y, ldp, l, C, ldp, true);
        if (P->emu) return emu_pass(P, w, transA, Y, ldp, l, C, ldp, true);
        return transA ? gemm_pass(P, w, true, n, m, A, lda, Y, ldp, C, ldp, l, P->S_tn, P->kc_tn, true)
                      : gemm_pass(P, w, false, m, n, A, lda, Y, ldp, C, ldp, l, P->S_nn, P->kc_nn, true);
    };
    return run_factor(P, w, product, omega, Qa, L, Qb, pbar0, ld0, pbar_out);
}

int pbpqlp_factor(pbpqlp_plan_t P, const void* Av, int64_t lda, int a_dtype, void* workspace, size_t ws_bytes,
                  const double* omega, double* Qa, double* L, double* Qb) {
    if (!Qa || !L || !Qb) return PBPQLP_EINVAL;
    return factor_impl(P, Av, lda, a_dtype, workspace, ws_bytes, omega, nullptr, 0, nullptr, Qa, L, Qb);
}

int pbpqlp_factor_from(pbpqlp_plan_t P, const void* A, int64_t lda, int a_dtype, void* workspace, size_t ws_bytes,
                       const double* pbar0, int64_t ld_pbar0, double* pbar_out, double* Qa, double* L, double* Qb) {
    return factor_impl(P, A, lda, a_dtype, workspace, ws_bytes, nullptr, pbar0, ld_pbar0, pbar_out, Qa, L, Qb);
}

size_t pbpqlp_csr_workspace_bytes(pbpqlp_plan_t P, int64_t nnz) {
    if (!P || nnz < 0) return 0;
    return (P->total + 255) / 256 * 256 + csr_transpose_bytes(P->n, nnz);
}

int pbpqlp_factor_csr(pbpqlp_plan_t P, const int64_t* rowptr, const int32_t* colind, const double* values,
                      int64_t nnz, void* workspace, size_t ws_bytes, const double* omega, double* Qa, double* L,
                      double* Qb) {
    if (!P || !rowptr || !Qa || !L || !Qb || nnz < 0 || (nnz > 0 && (!colind || !values))) return PBPQLP_EINVAL;
    if (P->n > INT32_MAX) return PBPQLP_EUNSUPPORTED;   // column indices are int32
    if (P->nprod > 0 || P->emu) return PBPQLP_EUNSUPPORTED;   // sparse products run in FP64
    if (!workspace || ((uintptr_t)workspace & 255u) || ws_bytes < pbpqlp_csr_workspace_bytes(P, nnz))
        return PBPQLP_EWORKSPACE;
    int rc = check_device_addressable(rowptr);
    if (!rc && nnz > 0) rc = check_device_addressable(colind);
    if (!rc && nnz > 0) rc = check_device_addressable(values);
    if (rc) return rc;
    P->last_ws = workspace;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    const int64_t m = P->m, n = P->n, ldp = P->ldp;
    const int l = P->l;
    PBQ_TRY(cudaMemsetAsync(w.status, 0, 256, s));
    if (w.ozcnt) PBQ_TRY(cudaMemsetAsync(w.ozcnt, 0, P->ozcnt_bytes, s));
    if (w.ozpart) PBQ_TRY(cudaMemsetAsync(w.ozpart, 0, P->ozpart_bytes, s));
    // A^T as a CSR (checks the structure first), once per call
    CsrT at;
    void* scratch = (char*)workspace + (P->total + 255) / 256 * 256;
    PBQ_TRY(launch_csr_transpose(m, n, nnz, rowptr, colind, values, scratch, &at, w.status, P->num_sms, s));
    auto product = [&](bool transA, const double* Y, double* C) -> int {
        const auto ev = next_events(P);
        if (ev.first) PBQ_TRY(cudaEventRecord(ev.first, s));
        for (int c0 = 0; c0 < l; c0 += P->cw) {
            const int nc = l - c0 < P->cw ? l - c0 : P->cw;
            if (transA)
                PBQ_TRY(launch_csr_spmm(n, at.ptr, at.idx, at.val, Y + c0, ldp, nc, C + c0, ldp, w.status, P->num_sms, s));
            else
                PBQ_TRY(launch_csr_spmm(m, rowptr, colind, values, Y + c0, ldp, nc, C + c0, ldp, w.status, P->num_sms, s));
        }
        if (ev.second) PBQ_TRY(cudaEventRecord(ev.second, s));
        return PBPQLP_OK;
    };
    return run_factor(P, w, product, omega, Qa, L, Qb);
}

int pbpqlp_sketch(pbpqlp_plan_t P, const void* A, int64_t lda, int a_dtype, int trans, const double* Y, int64_t ldy,
                  int ncols, double* C, int64_t ldc, void* workspace, size_t ws_bytes) {
    if (!P || !A || !Y || !C || ncols < 1 || ncols > P->l || lda < P->n) return PBPQLP_EINVAL;
    const int64_t rowsY = trans ? P->m : P->n, rowsC = trans ? P->n : P->m;
    if (ldy < ncols || ldc < ncols) return PBPQLP_EINVAL;
    const bool mixed = P->nprod > 0;
    if ((mixed || P->emu) ? (a_dtype != PBPQLP_F64 && a_dtype != PBPQLP_F32) : a_dtype != PBPQLP_F64)
        return PBPQLP_EUNSUPPORTED;
    int rc = check_ws(P, workspace, ws_bytes);
    if (rc) return rc;
    if ((rc = check_device_addressable(A))) return rc;
    P->last_ws = workspace;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    PBQ_TRY(cudaMemsetAsync(w.status, 0, 256, s));
    if (w.ozcnt) PBQ_TRY(cudaMemsetAsync(w.ozcnt, 0, P->ozcnt_bytes, s));
    if (w.ozpart) PBQ_TRY(cudaMemsetAsync(w.ozpart, 0, P->ozpart_bytes, s));
    (void)rowsY;
    if (P->stream_a && mixed) return tc_pass_stream(P, w, trans != 0, A, a_dtype == PBPQLP_F32, lda, Y, ldy, ncols, C, ldc, false);
    if (P->stream_a) return emu_pass_stream(P, w, trans != 0, A, a_dtype == PBPQLP_F32, lda, Y, ldy, ncols, C, ldc, false);
    if (P->emu) {
        if ((rc = emu_prepare_a(P, w, A, a_dtype == PBPQLP_F32, lda))) return rc;
        return emu_pass(P, w, trans != 0, Y, ldy, ncols, C, ldc);
    }
    if (mixed) {
        if ((rc = tc_prepare_a(P, w, A, a_dtype == PBPQLP_F32, lda))) return rc;
        return tc_pass(P, w, trans != 0, Y, ldy, ncols, C, ldc);
    }
    return trans ? gemm_pass(P, w, true, rowsC, P->m, (const double*)A, lda, Y, ldy, C, ldc, ncols, P->S_tn, P->kc_tn)
                 : gemm_pass(P, w, false, rowsC, P->n, (const double*)A, lda, Y, ldy, C, ldc, ncols, P->S_nn, P->kc_nn);
}

int pbpqlp_reconstruct(pbpqlp_plan_t P, const double* Qa, const double* L, const double* Qb, int r, double* Ahat,
                       int64_t ldh, void* workspace, size_t ws_bytes) {
    if (!P || !Qa || !L || !Qb || !Ahat || r < 1 || r > P->l || ldh < P->n) return PBPQLP_EINVAL;
    int rc = check_ws(P, workspace, ws_bytes);
    if (rc) return rc;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    const int l = P->l;
    // T = Qa_r L_r (m x r), then Ahat = T Qb_r^T
    PBQ_TRY(qa_times_l(P->m, r, Qa, L, l, w.Ym, P->ldp, s));
    PBQ_TRY(launch_dgemm_nt(P->m, P->n, r, w.Ym, P->ldp, Qb, l, Ahat, ldh, nullptr, 0, 0, nullptr, nullptr, s));
    return PBPQLP_OK;
}

int pbpqlp_sync_status(pbpqlp_plan_t P, uint32_t* flags_host) {
    if (!P) return PBPQLP_EINVAL;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return PBPQLP_ECUDA;
    uint32_t st = 0;
    if (P->last_ws) {
        if (cudaMemcpy(&st, (char*)P->last_ws + P->off_status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess)
            return PBPQLP_ECUDA;
    }
    if (flags_host) *flags_host = st;
    if (st & kStBadInput) return PBPQLP_EINVAL;
    if (st & kStNonFinite) return PBPQLP_ENONFINITE;
    if (st & kStTimeout) return PBPQLP_ETIMEOUT;
    if (st & kStBreakdown) return PBPQLP_EBREAKDOWN;
    return PBPQLP_OK;
}

int pbpqlp_error(pbpqlp_plan_t P, const void* A, int64_t lda, int a_dtype, const double* Qa, const double* L,
                 const double* Qb, int r, int method, int nprobes, uint64_t probe_seed, void* workspace,
                 size_t ws_bytes, double* rel_err) {
    if (!P || !A || !Qa || !L || !Qb || !rel_err || r < 1 || r > P->l || lda < P->n) return PBPQLP_EINVAL;
    if (a_dtype != PBPQLP_F64 && a_dtype != PBPQLP_F32) return PBPQLP_EINVAL;
    int rc = check_ws(P, workspace, ws_bytes);
    if (rc) return rc;
    if ((rc = check_device_addressable(A))) return rc;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    const int l = P->l;
    const int64_t m = P->m, n = P->n, ldp = P->ldp;
    const int f32 = a_dtype == PBPQLP_F32;
    double host[2] = {0.0, 0.0};
    if (method == PBPQLP_ERR_IDENTITY) {
        PBQ_TRY(launch_sumsq(m, n, A, f32, lda, nullptr, 0, w.red, w.scal + 0, s));
        PBQ_TRY(launch_sumsq(r, r, L, 0, l, nullptr, 0, w.red + 1024, w.scal + 1, s));
        PBQ_TRY(cudaMemcpyAsync(host, w.scal, sizeof(host), cudaMemcpyDeviceToHost, s));
        PBQ_TRY(cudaStreamSynchronize(s));
        const double d = host[0] - host[1];
        *rel_err = host[0] > 0.0 ? std::sqrt(d > 0.0 ? d : 0.0) / std::sqrt(host[0]) : 0.0;
    } else if (method == PBPQLP_ERR_RESIDUAL) {
        PBQ_TRY(launch_sumsq(m, n, A, f32, lda, nullptr, 0, w.red, w.scal + 0, s));
        PBQ_TRY(qa_times_l(m, r, Qa, L, l, w.Ym, ldp, s));
        int nb = 0;
        PBQ_TRY(launch_dgemm_nt(m, n, r, w.Ym, ldp, Qb, l, nullptr, 0, A, f32, lda, w.part, &nb, s));
        PBQ_TRY(launch_sum(nb, w.part, w.scal + 1, s));
        PBQ_TRY(cudaMemcpyAsync(host, w.scal, sizeof(host), cudaMemcpyDeviceToHost, s));
        PBQ_TRY(cudaStreamSynchronize(s));
        *rel_err = host[0] > 0.0 ? std::sqrt(host[1]) / std::sqrt(host[0]) : 0.0;
    } else if (method == PBPQLP_ERR_PROBES) {
        if (nprobes < 1 || nprobes > ldp || nprobes > kMaxEll) return PBPQLP_EINVAL;
        if (f32) return PBPQLP_EUNSUPPORTED;
        const int ns = nprobes;
        // W (n x s) Gaussian; AW = A W (m x s); T = Qa_r (L_r (Qb_r^T W))
        PBQ_TRY(launch_gaussian(probe_seed, n, ns, w.Yn, ldp, s));
        if ((rc = gemm_pass(P, w, false, m, n, (const double*)A, lda, w.Yn, ldp, w.Ym, ldp, ns, P->S_nn, P->kc_nn)))
            return rc;
        PBQ_TRY(launch_dgemm_skinny(true, r, ns, n, Qb, l, w.Yn, ldp, w.R, ldp, 1, n, 0, nullptr, s));
        PBQ_TRY(launch_dgemm_skinny(false, r, ns, r, L, l, w.R, ldp, w.Pt, ldp, 1, r, 0, nullptr, s));
        PBQ_TRY(launch_dgemm_skinny(false, m, ns, r, Qa, l, w.Pt, ldp, w.Xm, ldp, 1, r, 0, nullptr, s));
        PBQ_TRY(launch_sumsq(m, ns, w.Ym, 0, ldp, nullptr, 0, w.red, w.scal + 0, s));
        PBQ_TRY(launch_sumsq(m, ns, w.Ym, 0, ldp, w.Xm, ldp, w.red + 1024, w.scal + 1, s));
        PBQ_TRY(cudaMemcpyAsync(host, w.scal, sizeof(host), cudaMemcpyDeviceToHost, s));
        PBQ_TRY(cudaStreamSynchronize(s));
        *rel_err = host[0] > 0.0 ? std::sqrt(host[1] / host[0]) : 0.0;
    } else {
        return PBPQLP_EINVAL;
    }
    if (!std::isfinite(*rel_err)) return PBPQLP_ENONFINITE;
    return PBPQLP_OK;
}

int pbpqlp_rank_revealing(pbpqlp_plan_t P, const double* L, double tol, double* lvalues, void* workspace,
                          size_t ws_bytes, double* norm2_est, int* rank_est) {
    if (!P || !L || !lvalues || !norm2_est || !rank_est || !(tol >= 0.0)) return PBPQLP_EINVAL;
    int rc = check_ws(P, workspace, ws_bytes);
    if (rc) return rc;
    const Ws w = carve(P, workspace);
    cudaStream_t s = P->stream;
    PBQ_TRY(launch_lvalues(P->l, L, tol, lvalues, w.scal, s));
    double host[2] = {0.0, 0.0};
    PBQ_TRY(cudaMemcpyAsync(host, w.scal, sizeof(host), cudaMemcpyDeviceToHost, s));
    PBQ_TRY(cudaStreamSynchronize(s));
    *norm2_est = host[0];
    *rank_est = (int)host[1];
    return PBPQLP_OK;
}

int pbpqlp_set_timing(pbpqlp_plan_t P, int enable) {
    if (!P) return PBPQLP_EINVAL;
    P->timing_mask = enable ? (P->timing_mask | 1u) : (P->timing_mask & ~1u);
    return PBPQLP_OK;
}

int pbpqlp_read_timing_class(pbpqlp_plan_t P, int cls, double* ms_total, int64_t* launches) {
    if (!P || !ms_total || !launches || cls < 0 || cls >= kTimeClasses) return PBPQLP_EINVAL;
    if (cudaStreamSynchronize(P->stream) != cudaSuccess) return PBPQLP_ECUDA;
    double tot = 0.0;
    for (size_t i = 0; i < P->ev_used[cls]; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, P->ev[cls][i].first, P->ev[cls][i].second) != cudaSuccess) return PBPQLP_ECUDA;
        tot += ms;
    }
    *ms_total = tot;
    *launches = (int64_t)P->ev_used[cls];
    P->ev_used[cls] = 0;
    return PBPQLP_OK;
}

int pbpqlp_read_timing(pbpqlp_plan_t P, double* ms_total, int64_t* launches) {
    return pbpqlp_read_timing_class(P, PBPQLP_TIME_PASS, ms_total, launches);
}

int pbpqlp_set_timing_classes(pbpqlp_plan_t P, unsigned mask) {
    if (!P || (mask >> kTimeClasses) != 0) return PBPQLP_EINVAL;
    P->timing_mask = mask;
    return PBPQLP_OK;
}

int64_t pbpqlp_kernel_launch_count(void) { return launch_count(); }

}  // extern "C"
