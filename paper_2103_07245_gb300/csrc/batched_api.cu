// Batched PbP-QLP: many independent factorizations (uneven shapes) advanced
// together, one step of Algorithm 3 per launch over host-built work lists.
// The launch sequence is captured once into a CUDA graph and replayed while
// the buffers stay the same.  Matrix i draws its Gaussian test matrix from
// the Philox stream with key seed + i.
#include <cuda.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/pbpqlp.h"
#include "batched.h"
#include "internal.h"
#include "oz_internal.h"
#include "tc_internal.h"

using namespace pbq;

namespace {

struct MatWs {
    size_t Xm, Ym, Dm, Xn, Yn, part, G, Rp, R, Pt, work;
    int S_m, S_n;          // Gram split counts (rows chunks) of the m- and n-side panels
    // TF32 modes: split copies of A and A^T, transposed panels
    size_t Ahi, Alo, Athi, Atlo, Bnhi, Bnlo, Bmhi, Bmlo;
    int64_t ldn, ldm;      // their leading dimensions (n, m rounded up to 32)
    // digit Grams: panel digits of the m side, the n side and of D (kept for R = Q^T D)
    size_t Z[3];
    // Qb = Pbar Ptil as a digit product: row digits of Pbar (exponents Eq, n of
    // them) and column digits of Ptil
    size_t Zq, Zt, Eq;
};

// Digit sets of one matrix: 0 = m-side panels, 1 = n-side panels, 2 = D;
// exponent row 3 holds the column exponents of Ptil.
constexpr int kZm = 0, kZn = 1, kZd = 2, kEt = 3;
constexpr int kOzMaps = 8;          // per matrix: 2 per digit set, then Pbar (X box) and Ptil (Y box)

enum LaunchKind {
    L_GAUSS, L_GEMM, L_REDUCE, L_CHOL, L_TRSM, L_SQR, L_MEMSET_CTL, L_SPLIT, L_PSPLIT, L_TC,
    L_MEMSET,      // workspace bytes [off, off + n) to zero
    L_OZEXP, L_OZSLICE, L_OZ, L_OZROWS,
    L_FORK,        // the side stream waits for the main stream here
    L_JOIN         // the main stream waits for the side stream here
};

struct Launch {
    int kind;
    int TN;                // GEMM: column groups of 16; TRSM: the bucket's largest l
    bool transA;
    size_t off;            // byte offset of the unit list inside the list region
    int n;
    bool side = false;     // runs on the side stream (between L_FORK and L_JOIN)
};

constexpr int64_t kGaussPairsPerUnit = 8192;
constexpr int64_t kPanelRowsPerUnit = 256;

}  // namespace

struct pbpqlp_batch_s {
    int count = 0, p = 0, q = 0, mode = 0;
    uint64_t seed = 0;
    cudaStream_t stream = nullptr;
    int num_sms = 152;
    std::vector<int64_t> m, n;
    std::vector<int> k, l;
    int lmax = 0;
    int64_t ldp = 0;
    int gram_chunk = 512;           // rows per Gram partial (tuned by pbpqlp_batch_autotune)
    int trsm_rows = 64;             // rows per triangular-solve unit (tuned)
    int tc_sorted = 1;              // grouped products: longest contraction first (tuned)
    bool oz = false;                // Grams and R = Q^T D as digit products (PBPQLP_NO_OZ_GRAM=1: FP64 FMA)
    bool fault_producer = false;    // PBPQLP_FAULT=batch_producer at plan creation (failure-detection test)
    bool timing = false;            // event pairs around each grouped product kernel
    std::vector<cudaEvent_t> ev;    // 2 per timed launch
    int ev_used = 0;
    int nprod = 0;                  // TF32 modes: 1 (TF32) or 3 (split TF32); 0 in FP64 mode
    int a_f32 = 0;                  // element type of the A pointers the lists were built for
    std::vector<MatWs> mw;
    size_t off_status = 0, off_ctl = 0, off_lists = 0, lists_cap = 0, total = 0;
    size_t maps_off = 0;            // tensor-map table inside the list region
    size_t oz_maps_off = 0;         // digit tensor maps: kOzMaps per matrix (3 sets x {X, Y} boxes, Pbar, Ptil)
    size_t off_oze = 0;             // column exponents of the digit sets and of Ptil: [4][count][ldp] ints
    // host copy of the work lists and the launch sequence built for the last buffers
    std::vector<unsigned char> host_lists;
    std::vector<Launch> seq;
    std::vector<const void*> key;   // pointers the lists were built for
    cudaGraphExec_t exec = nullptr;
    cudaStream_t capture_stream = nullptr;   // private stream the graph is recorded on
    cudaStream_t side_stream = nullptr;      // second branch: the Gaussian draw beside the split of A
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    bool use_graph = true;
    void* last_ws = nullptr;
    ~pbpqlp_batch_s() {
        if (exec) cudaGraphExecDestroy(exec);
        if (capture_stream) cudaStreamDestroy(capture_stream);
        if (side_stream) cudaStreamDestroy(side_stream);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (cudaEvent_t e : ev) cudaEventDestroy(e);
    }
};

namespace {

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Upper bound of the list bytes for the current sizes (used to size the workspace).
size_t lists_bound(const pbpqlp_batch_s* B, int gram_chunk_min) {
    size_t units = 0;
    for (int i = 0; i < B->count; ++i) {
        const int64_t mt = (B->m[i] + kGemmBM - 1) / kGemmBM, nt = (B->n[i] + kGemmBM - 1) / kGemmBM;
        const int64_t lt = (B->l[i] + kGemmBM - 1) / kGemmBM;
        const int64_t gm = (B->m[i] + gram_chunk_min - 1) / gram_chunk_min;
        const int64_t gn = (B->n[i] + gram_chunk_min - 1) / gram_chunk_min;
        const int64_t passes = 2 * B->q + 2;
        // A passes, Grams (6 passes per orth), R = Q^T D, Qb
        units += (size_t)(passes * (mt + nt)) * sizeof(GemmUnit);
        units += (size_t)((passes * 6) * lt * std::max(gm, gn) + lt * gm) * sizeof(GemmUnit);
        units += (size_t)(mt + nt) * sizeof(GemmUnit);
        // reductions, Cholesky / small QR / Gaussian units, TRSM row blocks
        units += (size_t)(passes * 6 + 2) * sizeof(ReduceUnit);
        units += (size_t)(passes * 6 + 2) * sizeof(MatUnit);
        units += (size_t)((B->m[i] * B->l[i] / 2 + kGaussPairsPerUnit) / kGaussPairsPerUnit + 1) * sizeof(MatUnit);
        units += (size_t)(passes * 6) * ((std::max(B->m[i], B->n[i]) + 63) / 64) * sizeof(TrsmUnit);
        if (B->nprod) {
            units += 8 * 128;                                                   // tensor maps
            units += (size_t)(passes * ((B->m[i] + 127) / 128 + (B->n[i] + 127) / 128)) * sizeof(TcUnit);
            units += (size_t)((B->m[i] + 63) / 64) * sizeof(SplitUnit);
            units += (size_t)passes * ((std::max(B->m[i], B->n[i]) + kPanelRowsPerUnit - 1) / kPanelRowsPerUnit) *
                     sizeof(PanelUnit);
        }
        if (B->oz) {
            // digit maps; per Gram (and R): panel units twice (exponents, digits) and <= 2 x 5 tiles
            const int64_t pr = (std::max(B->m[i], B->n[i]) + kOzPanelRows - 1) / kOzPanelRows + 1;
            units += kOzMaps * 128;
            units += (size_t)(passes * 6 + 1) * (2 * pr * sizeof(OzPanelUnit) + 10 * sizeof(OzListUnit));
            // Qb: Pbar row units, Ptil panel units, tiles; Qa copy blocks
            units += (size_t)((B->n[i] + kOzRowsPerUnit - 1) / kOzRowsPerUnit + 4) * sizeof(OzPanelUnit);
            units += (size_t)((B->n[i] + kOzBM - 1) / kOzBM * 5) * sizeof(OzListUnit);
        }
        {
            units += (size_t)((B->m[i] + 255) / 256) * sizeof(ReduceUnit);
        }
    }
    // one list per width bucket: up to 14 GEMM and 14 TRSM buckets per step, 256-byte aligned
    return units + 64 * 1024 + 256 * 64 + (size_t)(2 * B->q + 2) * 6 * 36 * 256 + 64 * 256;
}

class ListBuilder {
  public:
    explicit ListBuilder(pbpqlp_batch_s* B) : B_(B) { B_->host_lists.clear(); B_->seq.clear(); }
    template <typename T>
    void add(int kind, const std::vector<T>& units, int TN = 0, bool transA = false, bool side = false) {
        if (units.empty()) return;
        size_t off = align_up(B_->host_lists.size(), 256);
        B_->host_lists.resize(off + units.size() * sizeof(T));
        std::memcpy(B_->host_lists.data() + off, units.data(), units.size() * sizeof(T));
        B_->seq.push_back(Launch{kind, TN, transA, off, (int)units.size(), side});
    }
    void fork() { B_->seq.push_back(Launch{L_FORK, 0, false, 0, 0}); }
    void join() { B_->seq.push_back(Launch{L_JOIN, 0, false, 0, 0}); }
    void memset_ctl() { B_->seq.push_back(Launch{L_MEMSET_CTL, 0, false, 0, 0}); }
    void memset_ws(size_t off, size_t bytes) { B_->seq.push_back(Launch{L_MEMSET, 0, false, off, (int)bytes}); }
    // GEMM units bucketed by their own width (16-column groups), one launch per bucket
    void add_gemm(const std::vector<GemmUnit>& units, bool transA) {
        std::vector<GemmUnit> bucket[kMaxEll / 16 + 1];
        for (const GemmUnit& g : units) bucket[(g.N + 15) / 16].push_back(g);
        for (int tn = 1; tn <= kMaxEll / 16; ++tn) add(L_GEMM, bucket[tn], tn, transA);
    }
    // triangular-solve units bucketed by `width`-column groups of their l
    // (32: warp-per-row FP64 solves; 16: the unrolled FP32 row solves)
    void add_trsm(const std::vector<TrsmUnit>& units, int width) {
        std::vector<TrsmUnit> bucket[kMaxEll / 16 + 2];
        int lm[kMaxEll / 16 + 2] = {};
        for (const TrsmUnit& t : units) {
            const int u = (t.l + width - 1) / width;
            bucket[u].push_back(t);
            lm[u] = std::max(lm[u], t.l);
        }
        for (int u = 1; u <= kMaxEll / width + 1; ++u) add(L_TRSM, bucket[u], lm[u]);
    }
    // raw table at the start of the list region (the tensor maps)
    size_t raw(const void* data, size_t bytes) {
        size_t off = align_up(B_->host_lists.size(), 256);
        B_->host_lists.resize(off + bytes);
        std::memcpy(B_->host_lists.data() + off, data, bytes);
        return off;
    }

  private:
    pbpqlp_batch_s* B_;
};

struct Ptrs {
    char* ws;
    const void* const* A;
    const int64_t* lda;
    double* const* Qa;
    double* const* L;
    double* const* Qb;
};

double* P64(const Ptrs& p, size_t off) { return (double*)(p.ws + off); }
float* P32(const Ptrs& p, size_t off) { return (float*)(p.ws + off); }

// Build the whole launch sequence of one batched factorization (FP64 mode).
int build_lists(pbpqlp_batch_s* B, const Ptrs& pt) {
    ListBuilder lb(B);
    const int cnt = B->count;
    const int64_t ldp = B->ldp;
    uint32_t* status = (uint32_t*)(pt.ws + B->off_status);
    int* ctl = (int*)(pt.ws + B->off_ctl);

    // Gaussian test matrices Phi_i (m_i x l_i) into Xm_i, on the side stream:
    // FP64-pipe bound, it runs beside the split of A (HBM bound)
    {
        std::vector<MatUnit> u;
        for (int i = 0; i < cnt; ++i) {
            const int64_t npairs = (B->m[i] * (int64_t)B->l[i] + 1) / 2;
            for (int64_t b0 = 0; b0 < npairs; b0 += kGaussPairsPerUnit) {
                MatUnit x{};
                x.l = B->l[i]; x.rows = B->m[i]; x.out = P64(pt, B->mw[i].Xm); x.ld = ldp;
                x.seed = B->seed + (uint64_t)i; x.b0 = b0; x.b1 = b0 + kGaussPairsPerUnit;
                u.push_back(x);
            }
        }
        lb.fork();
        lb.add(L_GAUSS, u, 0, false, true);
    }
    // TF32 modes: the tensor-map table (8 maps per matrix) and the split of every A_i
    if (B->nprod) {
        std::vector<CUtensorMap> maps((size_t)8 * cnt);
        for (int i = 0; i < cnt; ++i) {
            const MatWs& w = B->mw[i];
            const int npad = (int)round_up(B->l[i], 16);
            const void* bases[8] = {P32(pt, w.Ahi), P32(pt, w.Alo ? w.Alo : w.Ahi), P32(pt, w.Athi),
                                    P32(pt, w.Atlo ? w.Atlo : w.Athi), P32(pt, w.Bnhi), P32(pt, w.Bnlo ? w.Bnlo : w.Bnhi),
                                    P32(pt, w.Bmhi), P32(pt, w.Bmlo ? w.Bmlo : w.Bmhi)};
            const int64_t rows[8] = {B->m[i], B->m[i], B->n[i], B->n[i], B->l[i], B->l[i], B->l[i], B->l[i]};
            const int64_t cols[8] = {B->n[i], B->n[i], B->m[i], B->m[i], B->n[i], B->n[i], B->m[i], B->m[i]};
            const int64_t lds[8] = {w.ldn, w.ldn, w.ldm, w.ldm, w.ldn, w.ldn, w.ldm, w.ldm};
            for (int t = 0; t < 8; ++t)
                if (!make_map_f32(&maps[(size_t)8 * i + t], bases[t], rows[t], cols[t], lds[t], t < 4 ? 128 : npad))
                    return PBPQLP_EINVAL;
        }
        B->maps_off = lb.raw(maps.data(), maps.size() * sizeof(CUtensorMap));
        std::vector<SplitUnit> su;
        for (int i = 0; i < cnt; ++i) {
            const MatWs& w = B->mw[i];
            for (int64_t r0 = 0; r0 < B->m[i]; r0 += 64) {
                SplitUnit x{};
                x.A = pt.A[i]; x.lda = pt.lda[i]; x.a_f32 = B->a_f32; x.m = B->m[i]; x.n = B->n[i]; x.r0 = r0;
                x.hi = P32(pt, w.Ahi); x.lo = w.Alo ? P32(pt, w.Alo) : nullptr; x.ldh = w.ldn;
                x.thi = P32(pt, w.Athi); x.tlo = w.Atlo ? P32(pt, w.Atlo) : nullptr; x.ldt = w.ldm;
                // hi / lo and their transposes sit 256-aligned with ld a multiple of 32 floats
                x.vec_ok = ((uintptr_t)x.A & 15u) == 0 && (x.lda * (B->a_f32 ? 4 : 8)) % 16 == 0;
                su.push_back(x);
            }
        }
        int64_t nmax = 1;
        for (int i = 0; i < cnt; ++i) nmax = std::max(nmax, B->n[i]);
        lb.add(L_SPLIT, su, (int)((nmax + 63) / 64));
    }
    // digit Grams: maps of the three digit sets of every matrix (X box 128 rows, Y box 48)
    if (B->oz) {
        std::vector<CUtensorMap> zm((size_t)kOzMaps * cnt);
        for (int i = 0; i < cnt; ++i) {
            CUtensorMap* mp = &zm[(size_t)kOzMaps * i];
            for (int st = 0; st < 3; ++st) {
                const void* S = pt.ws + B->mw[i].Z[st];
                const int64_t K = st == kZn ? B->n[i] : B->m[i];
                if (!make_oz_map(&mp[2 * st], S, B->l[i], K, kOzBM) ||
                    !make_oz_map(&mp[2 * st + 1], S, B->l[i], K, kOzBN))
                    return PBPQLP_EINVAL;
            }
            if (!make_oz_map(&mp[6], pt.ws + B->mw[i].Zq, B->n[i], B->l[i], kOzBM) ||
                !make_oz_map(&mp[7], pt.ws + B->mw[i].Zt, B->l[i], B->l[i], kOzBN))
                return PBPQLP_EINVAL;
        }
        B->oz_maps_off = lb.raw(zm.data(), zm.size() * sizeof(CUtensorMap));
    }
    auto oz_exps = [&](int st, int i) {
        return (int*)(pt.ws + B->off_oze) + ((size_t)st * cnt + (size_t)i) * (size_t)ldp;
    };
    // panel P_i of digit set st (rows m_i or n_i) -> its column exponents and digits
    auto oz_panel_units = [&](int st, int i, const double* P, const int* cond, std::vector<OzPanelUnit>& pu) {
        const int64_t rows = st == kZn ? B->n[i] : B->m[i];
        for (int64_t r0 = 0; r0 < oz_kpad(rows); r0 += kOzPanelRows) {
            OzPanelUnit x{};
            x.P = P; x.ldp = ldp; x.rows = rows; x.r0 = r0; x.N = B->l[i];
            x.eraw = oz_exps(st, i); x.S = pt.ws + B->mw[i].Z[st]; x.cond = cond;
            pu.push_back(x);
        }
    };
    auto oz_add_panels = [&](int st, const std::vector<OzPanelUnit>& pu) {
        lb.memset_ws(B->off_oze + sizeof(int) * (size_t)st * cnt * ldp, sizeof(int) * (size_t)cnt * ldp);
        lb.add(L_OZEXP, pu);
        lb.add(L_OZSLICE, pu);
    };
    // C_i (l_i x l_i, ld l_i) = X^T Y for the panels of digit sets sx and sy
    auto oz_tiles = [&](int i, int sx, int sy, double* C, const int* cond, std::vector<OzListUnit>& ou) {
        const int64_t rows = sx == kZn ? B->n[i] : B->m[i];
        for (int m0 = 0; m0 < B->l[i]; m0 += kOzBM)
            for (int n0 = 0; n0 < B->l[i]; n0 += kOzBN) {
                OzListUnit u{};
                u.mapx = kOzMaps * i + 2 * sx; u.mapy = kOzMaps * i + 2 * sy + 1;
                u.m0 = m0; u.n0 = n0; u.KI = (int)((rows + kOzBK - 1) / kOzBK);
                u.Rx = B->l[i]; u.Ry = B->l[i]; u.ex = oz_exps(sx, i); u.ey = oz_exps(sy, i);
                u.C = C; u.ldc = B->l[i]; u.cond = cond;
                ou.push_back(u);
            }
    };
    auto oz_add_tiles = [&](std::vector<OzListUnit>& ou) {
        if (B->tc_sorted)
            std::stable_sort(ou.begin(), ou.end(), [](const OzListUnit& a, const OzListUnit& b) { return a.KI > b.KI; });
        lb.add(L_OZ, ou);
    };
    // one product with A_i for every matrix: out_i = op(A_i) Y_i
    auto product = [&](bool transA, auto ysel, auto csel) {
        if (B->nprod) {
            std::vector<PanelUnit> pu;
            std::vector<TcUnit> tu;
            for (int i = 0; i < cnt; ++i) {
                const MatWs& w = B->mw[i];
                const int64_t prow = transA ? B->m[i] : B->n[i];
                for (int64_t r0 = 0; r0 < prow; r0 += kPanelRowsPerUnit) {
                    PanelUnit x{};
                    x.Y = ysel(i); x.ldy = ldp; x.N = B->l[i];
                    x.r0 = r0;
                    x.rows = std::min<int64_t>(kPanelRowsPerUnit, prow - r0);
                    x.thi = P32(pt, transA ? w.Bmhi : w.Bnhi);
                    const size_t lo = transA ? w.Bmlo : w.Bnlo;
                    x.tlo = lo ? P32(pt, lo) : nullptr;
                    x.ldt = transA ? w.ldm : w.ldn;
                    pu.push_back(x);
                }
                const int64_t M = transA ? B->n[i] : B->m[i], K = transA ? B->m[i] : B->n[i];
                for (int64_t m0 = 0; m0 < M; m0 += 128) {
                    TcUnit t{};
                    t.amap_hi = 8 * i + (transA ? 2 : 0); t.amap_lo = t.amap_hi + 1;
                    t.bmap_hi = 8 * i + (transA ? 6 : 4); t.bmap_lo = t.bmap_hi + 1;
                    t.m0 = (int)m0; t.N = B->l[i]; t.npad = (int)round_up(B->l[i], 16); t.KI = (int)((K + 31) / 32);
                    t.C = csel(i); t.ldc = ldp; t.rows = M;
                    tu.push_back(t);
                }
            }
            // longest contraction first, then dealt round-robin to the persistent CTAs
            if (B->tc_sorted)
                std::stable_sort(tu.begin(), tu.end(), [](const TcUnit& a, const TcUnit& b) { return a.KI > b.KI; });
            lb.add(L_PSPLIT, pu);
            lb.add(L_TC, tu);
            return;
        }
        std::vector<GemmUnit> u;
        for (int i = 0; i < cnt; ++i) {
            const int64_t M = transA ? B->n[i] : B->m[i], K = transA ? B->m[i] : B->n[i];
            for (int64_t m0 = 0; m0 < M; m0 += kGemmBM) {
                GemmUnit g{};
                g.A = (const double*)pt.A[i]; g.lda = pt.lda[i];
                g.B = ysel(i); g.ldb = ldp;
                g.C = csel(i); g.ldc = ldp;   // tile rows are absolute (m0 + r)
                g.M = M; g.m0 = m0; g.kbeg = 0; g.kend = K; g.N = B->l[i]; g.transA = transA; g.cond = nullptr;
                u.push_back(g);
            }
        }
        lb.add_gemm(u, transA);
    };
    // CholeskyQR passes for every matrix's panel (side 0: m x l panels, side 1: n x l)
    // (digit Grams: pass 1 of the last orth of D takes digit set D, which R = Q^T D reuses)
    auto orth = [&](int side, auto srcsel, auto xsel, auto ysel, bool d_digits = false) {
        lb.memset_ctl();
        for (int pass = 1; pass <= 6; ++pass) {
            std::vector<GemmUnit> gu;
            std::vector<ReduceUnit> ru;
            std::vector<MatUnit> cu;
            std::vector<TrsmUnit> tu;
            std::vector<OzPanelUnit> pu;
            std::vector<OzListUnit> ou;
            const int st = (pass == 1 && d_digits) ? kZd : (side == 0 ? kZm : kZn);
            for (int i = 0; i < cnt; ++i) {
                const int64_t rows = side == 0 ? B->m[i] : B->n[i];
                const int l = B->l[i];
                const int S = side == 0 ? B->mw[i].S_m : B->mw[i].S_n;
                const double* src = pass == 1 ? srcsel(i) : ((pass & 1) ? xsel(i) : ysel(i));
                double* dst = (pass & 1) ? ysel(i) : xsel(i);
                int* c = ctl + 16 * i;
                const int* cond = pass <= 2 ? nullptr : c + 8 + (pass + 1) / 2;
                double* part = P64(pt, B->mw[i].part);
                const int64_t ps = (int64_t)l * ldp;
                if (B->oz) {
                    oz_panel_units(st, i, src, cond, pu);
                    oz_tiles(i, st, st, P64(pt, B->mw[i].G), cond, ou);
                } else {
                    for (int s = 0; s < S; ++s)
                        for (int64_t m0 = 0; m0 < l; m0 += kGemmBM) {
                            GemmUnit g{};
                            g.A = src; g.lda = ldp; g.B = src; g.ldb = ldp; g.C = part + s * ps; g.ldc = ldp;
                            g.M = l; g.m0 = m0; g.kbeg = (int64_t)s * B->gram_chunk;
                            g.kend = std::min<int64_t>(rows, (int64_t)(s + 1) * B->gram_chunk);
                            g.N = l; g.transA = 1; g.cond = cond;
                            gu.push_back(g);
                        }
                    ReduceUnit r{};
                    r.part = part; r.C = P64(pt, B->mw[i].G); r.ps = ps; r.ldp = ldp; r.ldc = l; r.M = l; r.N = l;
                    r.S = S; r.cond = cond;
                    ru.push_back(r);
                }
                MatUnit m{};
                m.l = l; m.pass = pass; m.rows = rows; m.G = P64(pt, B->mw[i].G); m.Rp = P64(pt, B->mw[i].Rp);
                m.ctl = c; m.status = status + i;
                cu.push_back(m);
                for (int64_t r0 = 0; r0 < rows; r0 += B->trsm_rows) {
                    TrsmUnit t{};
                    t.X = src; t.Y = dst; t.Rp = P64(pt, B->mw[i].Rp); t.ldx = ldp; t.ldy = ldp; t.r0 = r0;
                    t.r1 = std::min<int64_t>(rows, r0 + B->trsm_rows); t.l = l; t.cond = cond;
                    tu.push_back(t);
                }
            }
            if (B->oz) {
                oz_add_panels(st, pu);
                oz_add_tiles(ou);
            } else {
                lb.add_gemm(gu, true);
                lb.add(L_REDUCE, ru);
            }
            lb.add(L_CHOL, cu);
            lb.add_trsm(tu, B->nprod ? 16 : 32);
        }
    };
    auto Xm = [&](int i) { return P64(pt, B->mw[i].Xm); };
    auto Ym = [&](int i) { return P64(pt, B->mw[i].Ym); };
    auto Dm = [&](int i) { return P64(pt, B->mw[i].Dm); };
    auto Xn = [&](int i) { return P64(pt, B->mw[i].Xn); };
    auto Yn = [&](int i) { return P64(pt, B->mw[i].Yn); };

    lb.join();
    // failure-detection hook: the host producer gives up half-way through the
    // launch sequence, as a failing host call would; nothing has been launched
    if (B->fault_producer) return PBPQLP_ECUDA;
    product(true, Xm, Xn);                  // C = A^T Phi (Eq. 3)
    orth(1, Xn, Xn, Yn);                    // Pbar = orth(C) (Eq. 4)
    for (int it = 0; it < B->q; ++it) {     // power iterations (Section III-B)
        product(false, Xn, Xm);
        orth(0, Xm, Xm, Ym);
        product(true, Xm, Xn);
        orth(1, Xn, Xn, Yn);
    }
    product(false, Xn, Dm);                 // D = A Pbar (Eq. 5)
    orth(0, Dm, Xm, Ym, B->oz);             // Q = orth(D) (Eq. 6), result in Xm
    if (B->oz) {                            // R = Q^T D from the digits of Q and of D
        std::vector<OzPanelUnit> pu;
        std::vector<OzListUnit> ou;
        for (int i = 0; i < cnt; ++i) {
            oz_panel_units(kZm, i, Xm(i), nullptr, pu);
            oz_tiles(i, kZm, kZd, P64(pt, B->mw[i].R), nullptr, ou);
        }
        oz_add_panels(kZm, pu);
        oz_add_tiles(ou);
    } else {                                // R = Q^T D
        std::vector<GemmUnit> gu;
        std::vector<ReduceUnit> ru;
        for (int i = 0; i < cnt; ++i) {
            const int l = B->l[i];
            const int S = B->mw[i].S_m;
            double* part = P64(pt, B->mw[i].part);
            const int64_t ps = (int64_t)l * ldp;
            for (int s = 0; s < S; ++s)
                for (int64_t m0 = 0; m0 < l; m0 += kGemmBM) {
                    GemmUnit g{};
                    g.A = Xm(i); g.lda = ldp; g.B = Dm(i); g.ldb = ldp; g.C = part + s * ps; g.ldc = ldp;
                    g.M = l; g.m0 = m0; g.kbeg = (int64_t)s * B->gram_chunk;
                    g.kend = std::min<int64_t>(B->m[i], (int64_t)(s + 1) * B->gram_chunk);
                    g.N = l; g.transA = 1; g.cond = nullptr;
                    gu.push_back(g);
                }
            ReduceUnit r{};
            r.part = part; r.C = P64(pt, B->mw[i].R); r.ps = ps; r.ldp = ldp; r.ldc = l; r.M = l; r.N = l; r.S = S;
            r.cond = nullptr;
            ru.push_back(r);
        }
        lb.add_gemm(gu, true);
        lb.add(L_REDUCE, ru);
    }
    {                                       // [Ptil, Rtil] = qr(R^T), L = Rtil^T (Eq. 7)
        std::vector<MatUnit> u;
        for (int i = 0; i < cnt; ++i) {
            MatUnit x{};
            x.l = B->l[i]; x.G = P64(pt, B->mw[i].R); x.L = pt.L[i]; x.Pt = P64(pt, B->mw[i].Pt);
            x.work = P64(pt, B->mw[i].work);
            u.push_back(x);
        }
        lb.add(L_SQR, u);
    }
    if (B->oz) {                            // Qb = Pbar Ptil (Eq. 8) from the digits of Pbar and Ptil
        std::vector<OzPanelUnit> ru, pu;
        std::vector<OzListUnit> ou;
        for (int i = 0; i < cnt; ++i) {
            const MatWs& w = B->mw[i];
            const int l = B->l[i];
            for (int64_t r0 = 0; r0 < B->n[i]; r0 += kOzRowsPerUnit) {
                OzPanelUnit x{};
                x.P = Xn(i); x.ldp = ldp; x.rows = B->n[i]; x.r0 = r0; x.N = l;
                x.eraw = (int*)(pt.ws + w.Eq); x.S = pt.ws + w.Zq;
                ru.push_back(x);
            }
            for (int64_t r0 = 0; r0 < oz_kpad(l); r0 += kOzPanelRows) {
                OzPanelUnit y{};
                y.P = P64(pt, w.Pt); y.ldp = l; y.rows = l; y.r0 = r0; y.N = l; y.eraw = oz_exps(kEt, i);
                y.S = pt.ws + w.Zt;
                pu.push_back(y);
            }
            for (int m0 = 0; m0 < B->n[i]; m0 += kOzBM)
                for (int n0 = 0; n0 < l; n0 += kOzBN) {
                    OzListUnit u{};
                    u.mapx = kOzMaps * i + 6; u.mapy = kOzMaps * i + 7;
                    u.m0 = m0; u.n0 = n0; u.KI = (l + kOzBK - 1) / kOzBK;
                    u.Rx = (int)B->n[i]; u.Ry = l; u.ex = (const int*)(pt.ws + w.Eq); u.ey = oz_exps(kEt, i);
                    u.C = pt.Qb[i]; u.ldc = l;
                    ou.push_back(u);
                }
        }
        lb.add(L_OZROWS, ru);
        oz_add_panels(kEt, pu);
        oz_add_tiles(ou);
    } else {                                // Qb = Pbar Ptil (Eq. 8)
        std::vector<GemmUnit> gu;
        for (int i = 0; i < cnt; ++i) {
            const int l = B->l[i];
            for (int64_t m0 = 0; m0 < B->n[i]; m0 += kGemmBM) {
                GemmUnit g{};
                g.A = Xn(i); g.lda = ldp; g.B = P64(pt, B->mw[i].Pt); g.ldb = l; g.C = pt.Qb[i]; g.ldc = l;
                g.M = B->n[i]; g.m0 = m0; g.kbeg = 0; g.kend = l; g.N = l; g.transA = 0; g.cond = nullptr;
                gu.push_back(g);
            }
        }
        lb.add_gemm(gu, false);
    }
    {                                       // Qa = Q (copy to ld l; a one-term "reduction"), 256-row blocks
        std::vector<ReduceUnit> cu;
        for (int i = 0; i < cnt; ++i)
            for (int64_t r0 = 0; r0 < B->m[i]; r0 += 256) {
                ReduceUnit r{};
                r.part = Xm(i) + r0 * ldp; r.C = pt.Qa[i] + r0 * B->l[i]; r.ps = 0; r.ldp = ldp; r.ldc = B->l[i];
                r.M = std::min<int64_t>(256, B->m[i] - r0); r.N = B->l[i]; r.S = 1; r.cond = nullptr;
                cu.push_back(r);
            }
        lb.add(L_REDUCE, cu);
    }
    if (B->host_lists.size() > B->lists_cap) return PBPQLP_EWORKSPACE;
    return PBPQLP_OK;
}

#define PBQ_TRY(expr) do { cudaError_t e_ = PBQ_DBG(expr); if (e_ != cudaSuccess) return PBPQLP_ECUDA; } while (0)

int enqueue(pbpqlp_batch_s* B, char* ws, cudaStream_t s) {
    char* lists = ws + B->off_lists;
    int evi = 0;
    int* ctl = (int*)(ws + B->off_ctl);
    PBQ_TRY(cudaMemsetAsync(ws + B->off_status, 0, sizeof(uint32_t) * (size_t)B->count, s));
    if (B->timing) {   // the FP64 mode times its product launches (L_GEMM with the A operand) instead
        int need = 0;
        for (const Launch& L : B->seq) need += 2 * (L.kind == L_TC);
        while ((int)B->ev.size() < need) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return PBPQLP_ECUDA;
            B->ev.push_back(e);
        }
    }
    if (!B->side_stream && cudaStreamCreateWithFlags(&B->side_stream, cudaStreamNonBlocking) != cudaSuccess)
        return PBPQLP_ECUDA;
    if (!B->ev_fork && cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming) != cudaSuccess) return PBPQLP_ECUDA;
    if (!B->ev_join && cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming) != cudaSuccess) return PBPQLP_ECUDA;
    for (const Launch& L : B->seq) {
        const void* u = lists + L.off;
        const cudaStream_t ls = L.side ? B->side_stream : s;
        switch (L.kind) {
            case L_FORK:
                PBQ_TRY(cudaEventRecord(B->ev_fork, s));
                PBQ_TRY(cudaStreamWaitEvent(B->side_stream, B->ev_fork, 0));
                break;
            case L_JOIN:
                PBQ_TRY(cudaEventRecord(B->ev_join, B->side_stream));
                PBQ_TRY(cudaStreamWaitEvent(s, B->ev_join, 0));
                break;
            case L_MEMSET_CTL: PBQ_TRY(cudaMemsetAsync(ctl, 0, sizeof(int) * 16 * (size_t)B->count, s)); break;
            case L_MEMSET: PBQ_TRY(cudaMemsetAsync(ws + L.off, 0, (size_t)L.n, s)); break;
            case L_OZEXP: PBQ_TRY(launch_oz_panel_exp_list((const OzPanelUnit*)u, L.n, s)); break;
            case L_OZSLICE: PBQ_TRY(launch_oz_panel_slice_list((const OzPanelUnit*)u, L.n, s)); break;
            case L_OZROWS: PBQ_TRY(launch_oz_rows_list((const OzPanelUnit*)u, L.n, s)); break;
            case L_OZ:
                PBQ_TRY(launch_oz_list(lists + B->oz_maps_off, (const OzListUnit*)u, L.n, B->num_sms,
                                       (uint32_t*)(ws + B->off_status), s));
                break;
            case L_GAUSS: PBQ_TRY(launch_gaussian_list((const MatUnit*)u, L.n, ls)); break;
            case L_GEMM: PBQ_TRY(launch_dgemm_list(L.TN, L.transA, (const GemmUnit*)u, L.n, s)); break;
            case L_REDUCE: PBQ_TRY(launch_reduce_list((const ReduceUnit*)u, L.n, s)); break;
            case L_CHOL: PBQ_TRY(launch_cholesky_list((const MatUnit*)u, L.n, B->lmax, s)); break;
            case L_TRSM: PBQ_TRY(launch_trsm_list((const TrsmUnit*)u, L.n, L.TN, s, B->nprod > 0)); break;
            case L_SQR: PBQ_TRY(launch_small_qr_list((const MatUnit*)u, L.n, B->lmax, s)); break;
            case L_SPLIT: PBQ_TRY(launch_split_tf32_list((const SplitUnit*)u, L.n, L.TN, B->a_f32, s)); break;
            case L_PSPLIT: PBQ_TRY(launch_split_panel_tf32_list((const PanelUnit*)u, L.n, s)); break;
            case L_TC: {
                const bool t = B->timing && evi + 1 < (int)B->ev.size();
                // under capture an event record must be an external node to be recorded at replay
                cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
                PBQ_TRY(cudaStreamIsCapturing(s, &cs));
                const unsigned flags = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
                if (t) PBQ_TRY(cudaEventRecordWithFlags(B->ev[evi], s, flags));
                PBQ_TRY(launch_tc_list(B->nprod, lists + B->maps_off, (const TcUnit*)u, L.n, B->num_sms,
                                       (uint32_t*)(ws + B->off_status), s));
                if (t) { PBQ_TRY(cudaEventRecordWithFlags(B->ev[evi + 1], s, flags)); evi += 2; }
                break;
            }
            default: return PBPQLP_EINVAL;
        }
    }
    return PBPQLP_OK;
}

void layout(pbpqlp_batch_s* B) {
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes, 256); return o; };
    B->off_status = take(sizeof(uint32_t) * (size_t)B->count);
    B->off_ctl = take(sizeof(int) * 16 * (size_t)B->count);
    const int64_t ldp = B->ldp;
    B->mw.assign(B->count, MatWs{});
    for (int i = 0; i < B->count; ++i) {
        MatWs& w = B->mw[i];
        const int64_t m = B->m[i], n = B->n[i], l = B->l[i];
        w.S_m = (int)((m + B->gram_chunk - 1) / B->gram_chunk);
        w.S_n = (int)((n + B->gram_chunk - 1) / B->gram_chunk);
        const int smax = (int)((std::max(m, n) + 255) / 256);   // sized for the smallest tuned chunk
        w.Xm = take(8 * (size_t)(m * ldp));
        w.Ym = take(8 * (size_t)(m * ldp));
        w.Dm = take(8 * (size_t)(m * ldp));
        w.Xn = take(8 * (size_t)(n * ldp));
        w.Yn = take(8 * (size_t)(n * ldp));
        w.part = take(8 * (size_t)(smax * l * ldp));
        w.G = take(8 * (size_t)(l * l));
        w.Rp = take(8 * (size_t)(packed_tri((int)l) + l));
        w.R = take(8 * (size_t)(l * l));
        w.Pt = take(8 * (size_t)(l * l));
        w.work = take(8 * (size_t)(3 * l * l + 2 * l));
        if (B->nprod) {
            const bool split = B->nprod == 3;
            const int64_t npad = round_up(l, 16);
            w.ldn = round_up(n, 32);
            w.ldm = round_up(m, 32);
            w.Ahi = take(4 * (size_t)(m * w.ldn));
            w.Alo = split ? take(4 * (size_t)(m * w.ldn)) : 0;
            w.Athi = take(4 * (size_t)(n * w.ldm));
            w.Atlo = split ? take(4 * (size_t)(n * w.ldm)) : 0;
            w.Bnhi = take(4 * (size_t)(npad * w.ldn));
            w.Bnlo = split ? take(4 * (size_t)(npad * w.ldn)) : 0;
            w.Bmhi = take(4 * (size_t)(npad * w.ldm));
            w.Bmlo = split ? take(4 * (size_t)(npad * w.ldm)) : 0;
        }
        if (B->oz) {
            w.Z[kZm] = take(oz_digit_bytes(l, m));
            w.Z[kZn] = take(oz_digit_bytes(l, n));
            w.Z[kZd] = take(oz_digit_bytes(l, m));
            w.Zq = take(oz_digit_bytes(n, l));
            w.Zt = take(oz_digit_bytes(l, l));
            w.Eq = take(sizeof(int) * (size_t)n);
        }
    }
    if (B->oz) B->off_oze = take(sizeof(int) * 4 * (size_t)B->count * (size_t)ldp);
    B->lists_cap = lists_bound(B, 256);
    B->off_lists = take(B->lists_cap);
    B->total = off;
}

int run(pbpqlp_batch_s* B, const Ptrs& pt, size_t ws_bytes) {
    std::vector<const void*> key;
    key.push_back(pt.ws);
    for (int i = 0; i < B->count; ++i) {
        key.push_back(pt.A[i]); key.push_back((const void*)(intptr_t)pt.lda[i]);
        key.push_back(pt.Qa[i]); key.push_back(pt.L[i]); key.push_back(pt.Qb[i]);
    }
    (void)ws_bytes;
    const bool rebuilt = key != B->key || B->seq.empty();
    if (rebuilt) {
        if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
        int rc = build_lists(B, pt);
        if (rc) return rc;
        B->key = key;
    }
    // from here on this workspace holds the batch's status words
    B->last_ws = pt.ws;
    // the lists live in the caller's workspace: refresh them on every call
    // (a pageable-memory copy is staged before the call returns)
    PBQ_TRY(cudaMemcpyAsync(pt.ws + B->off_lists, B->host_lists.data(), B->host_lists.size(),
                            cudaMemcpyHostToDevice, B->stream));
    if (rebuilt) {
        if (B->use_graph && !B->capture_stream &&
            cudaStreamCreateWithFlags(&B->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
            B->capture_stream = nullptr;
            B->use_graph = false;
            cudaGetLastError();
        }
        if (B->use_graph) {
            // record on the private stream (nothing runs); the graph is launched on the caller's stream
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(B->capture_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const int64_t before = launch_count();
                const int rc2 = enqueue(B, pt.ws, B->capture_stream);
                count_launches(before - launch_count());   // captured, not run
                const cudaError_t ec = cudaStreamEndCapture(B->capture_stream, &g);
                if (rc2 == PBPQLP_OK && ec == cudaSuccess && g &&
                    cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess) {
                    cudaGraphDestroy(g);
                } else {
                    if (g) cudaGraphDestroy(g);
                    B->exec = nullptr;
                    B->use_graph = false;
                    cudaGetLastError();
                }
            } else {
                B->use_graph = false;
                cudaGetLastError();
            }
        }
    }
    if (B->timing) {
        B->ev_used = 0;
        for (const Launch& L : B->seq) B->ev_used += 2 * (L.kind == L_TC);
    }
    if (B->exec) {
        PBQ_TRY(cudaGraphLaunch(B->exec, B->stream));
        int64_t kernels = 0;
        for (const Launch& L : B->seq)
            kernels += (L.kind != L_MEMSET_CTL && L.kind != L_MEMSET && L.kind != L_FORK && L.kind != L_JOIN);
        count_launches(kernels);
        return PBPQLP_OK;
    }
    return enqueue(B, pt.ws, B->stream);
}

}  // namespace

extern "C" {

int pbpqlp_plan_batched(pbpqlp_batch_t* out, int count, const int64_t* m, const int64_t* n, const int* k, int p, int q,
                        uint64_t seed, int mode, void* stream) {
    if (!out) return PBPQLP_EINVAL;
    *out = nullptr;
    if (count < 1 || !m || !n || !k || p < 0 || q < 0 || q > 64) return PBPQLP_EINVAL;
    if (mode != PBPQLP_MODE_FP64 && mode != PBPQLP_MODE_TF32 && mode != PBPQLP_MODE_TF32X3) return PBPQLP_EUNSUPPORTED;
    pbpqlp_batch_s* B = new (std::nothrow) pbpqlp_batch_s();
    if (!B) return PBPQLP_ENOMEM;
    B->count = count; B->p = p; B->q = q; B->seed = seed; B->mode = mode; B->stream = (cudaStream_t)stream;
    B->m.assign(m, m + count);
    B->n.assign(n, n + count);
    B->k.assign(k, k + count);
    B->l.resize(count);
    for (int i = 0; i < count; ++i) {
        const int64_t l = (int64_t)k[i] + p;
        if (m[i] < 1 || n[i] < 1 || k[i] < 1 || l > m[i] || l > n[i] || l > kMaxEll) { delete B; return PBPQLP_EINVAL; }
        B->l[i] = (int)l;
        B->lmax = std::max(B->lmax, (int)l);
    }
    B->nprod = mode == PBPQLP_MODE_TF32X3 ? 3 : mode == PBPQLP_MODE_TF32 ? 1 : 0;
    if (B->nprod) B->trsm_rows = 128;   // the FP32 row solves run 128 rows per CTA
    if (B->nprod && B->lmax > kTcListBNMax) { delete B; return PBPQLP_EUNSUPPORTED; }
    {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            B->num_sms = sms;
        cudaGetLastError();
    }
    B->ldp = round_up(B->lmax, 8);
    const char* env = std::getenv("PBPQLP_BATCH_NO_GRAPH");
    if (env && env[0] == '1') B->use_graph = false;
    const char* no = std::getenv("PBPQLP_NO_OZ_GRAM");
    B->oz = !(no && no[0] == '1');
    const char* fault = std::getenv("PBPQLP_FAULT");
    B->fault_producer = fault && std::strcmp(fault, "batch_producer") == 0;
    layout(B);
    *out = B;
    return PBPQLP_OK;
}

int pbpqlp_batch_destroy(pbpqlp_batch_t B) {
    delete B;
    return PBPQLP_OK;
}

size_t pbpqlp_batch_workspace_bytes(pbpqlp_batch_t B) { return B ? B->total : 0; }

int pbpqlp_factor_batched(pbpqlp_batch_t B, const void* const* A, const int64_t* lda, int a_dtype, void* workspace,
                          size_t ws_bytes, double* const* Qa, double* const* L, double* const* Qb) {
    if (!B || !A || !lda || !Qa || !L || !Qb) return PBPQLP_EINVAL;
    if (B->nprod ? (a_dtype != PBPQLP_F64 && a_dtype != PBPQLP_F32) : a_dtype != PBPQLP_F64) return PBPQLP_EUNSUPPORTED;
    if (!workspace || ws_bytes < B->total || ((uintptr_t)workspace & 255u)) return PBPQLP_EWORKSPACE;
    for (int i = 0; i < B->count; ++i) {
        if (!A[i] || !Qa[i] || !L[i] || !Qb[i] || lda[i] < B->n[i]) return PBPQLP_EINVAL;
        // device, managed, or pinned host memory mapped at the same address
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, A[i]) != cudaSuccess) { cudaGetLastError(); return PBPQLP_EINVAL; }
        if (at.type == cudaMemoryTypeUnregistered || (at.type == cudaMemoryTypeHost && at.devicePointer != A[i]))
            return PBPQLP_EINVAL;
    }
    if (B->a_f32 != (a_dtype == PBPQLP_F32)) { B->a_f32 = a_dtype == PBPQLP_F32; B->key.clear(); }
    Ptrs pt{(char*)workspace, A, lda, Qa, L, Qb};
    return run(B, pt, ws_bytes);
}

int pbpqlp_batch_set_timing(pbpqlp_batch_t B, int enable) {
    if (!B) return PBPQLP_EINVAL;
    if (B->timing != (enable != 0)) {
        B->timing = enable != 0;
        B->key.clear();   // re-record the graph with or without the event nodes
    }
    return PBPQLP_OK;
}

int pbpqlp_batch_read_timing(pbpqlp_batch_t B, double* ms_total, int64_t* launches) {
    if (!B || !ms_total || !launches) return PBPQLP_EINVAL;
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PBPQLP_ECUDA;
    double t = 0.0;
    for (int i = 0; i + 1 < B->ev_used && i + 1 < (int)B->ev.size(); i += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, B->ev[i], B->ev[i + 1]) != cudaSuccess) return PBPQLP_ECUDA;
        t += ms;
    }
    *ms_total = t;
    *launches = B->ev_used / 2;
    return PBPQLP_OK;
}

int pbpqlp_batch_autotune(pbpqlp_batch_t B, const void* const* A, const int64_t* lda, int a_dtype, void* workspace,
                          size_t ws_bytes, double* const* Qa, double* const* L, double* const* Qb, const char* table_path,
                          double* best_ms) {
    if (!B) return PBPQLP_EINVAL;
    const int chunks[] = {256, 512, 1024, 2048};
    const int trows[] = {64, 128, 256};
    const int sorts[] = {1, 0};
    double best = 1e300;
    int bc = B->gram_chunk, bt = B->trsm_rows, bs = B->tc_sorted;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PBPQLP_ECUDA;
    int rc = PBPQLP_OK;
    for (int gc : chunks)
        for (int tr : trows)
            for (int so : sorts) {
                if (!B->nprod && so == 0) continue;   // unit order only matters for the grouped products
                if (B->oz && gc != 512) continue;     // digit Grams take whole contractions: no row chunks
                B->gram_chunk = gc; B->trsm_rows = tr; B->tc_sorted = so;
                for (int i = 0; i < B->count; ++i) {
                    B->mw[i].S_m = (int)((B->m[i] + gc - 1) / gc);
                    B->mw[i].S_n = (int)((B->n[i] + gc - 1) / gc);
                }
                B->key.clear();
                // first call records the graph, the second is timed
                if ((rc = pbpqlp_factor_batched(B, A, lda, a_dtype, workspace, ws_bytes, Qa, L, Qb))) goto done;
                if (cudaEventRecord(e0, B->stream) != cudaSuccess) { rc = PBPQLP_ECUDA; goto done; }
                if ((rc = pbpqlp_factor_batched(B, A, lda, a_dtype, workspace, ws_bytes, Qa, L, Qb))) goto done;
                if (cudaEventRecord(e1, B->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
                    rc = PBPQLP_ECUDA;
                    goto done;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (ms < best) { best = ms; bc = gc; bt = tr; bs = so; }
            }
done:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    B->gram_chunk = bc; B->trsm_rows = bt; B->tc_sorted = bs;
    for (int i = 0; i < B->count; ++i) {
        B->mw[i].S_m = (int)((B->m[i] + bc - 1) / bc);
        B->mw[i].S_n = (int)((B->n[i] + bc - 1) / bc);
    }
    B->key.clear();
    if (rc) return rc;
    if (best_ms) *best_ms = best;
    if (table_path && table_path[0]) {
        // one JSON line per tuning: the batch signature and the chosen tiles
        uint64_t h = 1469598103934665603ull;
        auto mix = [&](uint64_t v) { h = (h ^ v) * 1099511628211ull; };
        mix((uint64_t)B->count); mix((uint64_t)B->p); mix((uint64_t)B->q); mix((uint64_t)B->mode);
        for (int i = 0; i < B->count; ++i) { mix((uint64_t)B->m[i]); mix((uint64_t)B->n[i]); mix((uint64_t)B->k[i]); }
        FILE* f = std::fopen(table_path, "a");
        if (f) {
            std::fprintf(f,
                         "{\"signature\": \"%016llx\", \"count\": %d, \"mode\": %d, \"gram_chunk\": %d, "
                         "\"trsm_rows\": %d, \"tc_sorted\": %d, \"ms\": %.4f}\n",
                         (unsigned long long)h, B->count, B->mode, bc, bt, bs, best);
            std::fclose(f);
        }
    }
    return PBPQLP_OK;
}

int pbpqlp_batch_sync_status(pbpqlp_batch_t B, uint32_t* flags_host) {
    if (!B) return PBPQLP_EINVAL;
    if (cudaStreamSynchronize(B->stream) != cudaSuccess) return PBPQLP_ECUDA;
    std::vector<uint32_t> st(B->count, 0);
    if (B->last_ws && cudaMemcpy(st.data(), (char*)B->last_ws + B->off_status, sizeof(uint32_t) * st.size(),
                                 cudaMemcpyDeviceToHost) != cudaSuccess)
        return PBPQLP_ECUDA;
    uint32_t all = 0;
    for (int i = 0; i < B->count; ++i) {
        all |= st[i];
        if (flags_host) flags_host[i] = st[i];
    }
    if (all & kStNonFinite) return PBPQLP_ENONFINITE;
    if (all & kStTimeout) return PBPQLP_ETIMEOUT;
    if (all & kStBreakdown) return PBPQLP_EBREAKDOWN;
    return PBPQLP_OK;
}

}  // extern "C"
