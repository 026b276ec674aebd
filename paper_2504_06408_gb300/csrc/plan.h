// Host-side plan of one SpGEMM call: tuning, workspace layout, kernel
// launchers.  Shared by the kernel translation units and the C ABI.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace spg {

constexpr int kMaxProb = 128;    // products in one batched call
constexpr int kTiers = 5;        // 0 dense, 1 block, 2 warp, 3 empty, 4 light dense (numeric)
constexpr int kSymTiers = 4;     // the symbolic phase uses tiers 0..3
constexpr int kSubBins = 40;     // per tier: by floor(log2(work)), heaviest first
constexpr int kNumBins = kTiers * kSubBins;
constexpr int kTierDense = 0, kTierBlock = 1, kTierWarp = 2, kTierEmpty = 3, kTierDenseLight = 4;

struct Tuning {
    int64_t sym_warp_max_ub;
    int64_t sym_block_max_ub;
    int64_t num_warp_max_nnz;
    int64_t num_block_max_nnz;
    int64_t dense_slab_cols;
    int64_t sym_slab_cols;
    int64_t bitmap_cache_bytes;   // < 0: no bitmap cache
    int64_t rank_light_ub;        // light rows of the rank kernel: ub_i below this (<= 0: none)
};

// Per-semiring defaults chosen so that every tier's shared memory fits.
Tuning default_tuning(int sr);
// Clamp user values into what the kernels can hold for this semiring.
Tuning clamp_tuning(Tuning t, int sr);

struct ProbTable {
    Prob p[kMaxProb];
};

// Work counters and bin tables at the head of the workspace.
struct Counters {
    int32_t sym_bin_count[kNumBins];
    int32_t sym_bin_off[kNumBins + 1];
    int32_t sym_bin_cursor[kNumBins];
    int32_t num_bin_count[kNumBins];
    int32_t num_bin_off[kNumBins + 1];
    int32_t num_bin_cursor[kNumBins];
    int32_t claim[16];                  // per-kernel dynamic row counters
    int32_t bm_next;                    // next free bitmap cache slot
    unsigned long long products;        // sum of ub over all rows
    unsigned long long dense_products;  // sum of ub over the symbolic dense tier's rows
    int32_t words_ready;                // the word-packed copies of B were built
    int32_t ovl_wide;                   // overlap semiring: a position is outside [0, 2^16)
    int64_t num_block_max;              // numeric: block-tier limit in effect (0: the tuning's)
    int64_t light_n;                    // numeric: largest nnz(C_i) of a light dense row (0: none)
    unsigned long long learned_nnz;     // learned path: entries of the rows it finished
    int64_t nnz[kMaxProb];              // per-product nnz(C)
};

struct WsLayout {
    size_t status, counters, probs, ub, cnt, rows_sym, rows_num, scan_part, cursor, slab_ptr,
        slab_ptr_bytes, row_slot, bm_cache, bm_cache_bytes, words, words_bytes, total;
    int64_t bm_cache_words, bm_cache_slots;
    int64_t R;          // flat rows
    int64_t E;          // flat entries of A (cursor array length)
};

// R flat rows, E flat entries of A; slab_bytes: the slab-start tables of the
// distinct B matrices; ncols_b: columns of the widest B (bitmap cache rows);
// words_bytes: room for the word-packed copies of B (word_pack_bytes of each
// distinct B)
WsLayout ws_layout(int64_t R, int64_t E, size_t slab_bytes, int64_t ncols_b,
                   int64_t cache_bytes, size_t words_bytes);

struct WsPtrs {
    DevStatus* status;
    Counters* ctr;
    Prob* probs;
    int64_t* ub;
    int64_t* cnt;
    int32_t* rows_sym;
    int32_t* rows_num;
    int64_t* scan_part;
    int32_t* cursor;
    int32_t* slab_ptr;       // slab starts of B's rows (numeric dense tier)
    size_t slab_ptr_bytes;
    const uint8_t* skip = nullptr;   // rows to leave out of binning (learned path), or null
    uint32_t* bm_cache;      // row bitmaps kept by the symbolic dense tier, or null
    int64_t bm_cache_words;  // words per cached bitmap
    int64_t bm_cache_slots;  // cached bitmaps that fit
    int32_t* row_slot;       // per flat row: cache slot or -1
};
WsPtrs ws_ptrs(void* ws, const WsLayout& L);

// Optional per-stage CUDA-event timing: an event is recorded on the launch
// stream after each stage; stage time = its event minus the previous one.
enum StageTag : int {
    kStBegin = 0, kStAnalyze, kStSymDense, kStSymBlock, kStSymWarp, kStScan,
    kStNumBin, kStSlabPtr, kStNumDense, kStNumBlock, kStNumWarp, kStMerge, kStLearned, kStCount
};
struct StageTimer {
    static constexpr int kMax = 32;
    cudaEvent_t ev[kMax];
    int tag[kMax];
    int n = 0;
    bool on = false;
};

struct DevInfo {
    int sms;
    int max_smem_optin;
    int max_smem_sm = 0;           // shared memory per SM (0: unknown)
    int64_t* launches = nullptr;   // kernels launched (incremented by the launchers)
    StageTimer* timer = nullptr;
};

inline void count_launch(const DevInfo& d, int k = 1) {
    if (d.launches) *d.launches += k;
}
inline void mark_stage(const DevInfo& d, int tag, cudaStream_t st) {
    if (d.timer && d.timer->on && d.timer->n < StageTimer::kMax) {
        cudaEventRecord(d.timer->ev[d.timer->n], st);
        d.timer->tag[d.timer->n++] = tag;
    }
}

// ---- word-packed B for the symbolic dense tier (symbolic.cu) ----
//
// Row k of Bw holds one entry per distinct 32-column word of B_k: col = the
// word index (column >> 5), val = the uint32 mask of B_k's columns in that
// word.  The symbolic dense tier ORs whole masks into the row bitmap: one
// product per word instead of one per column.
// Bytes of one packed copy (worst case: every entry in its own word).
size_t word_pack_bytes(int64_t nrows, int64_t nnz);
// Use the packed walk at all: B large enough that packing pays for its launches.
constexpr int64_t kWordPackMinNnz = 65536;
struct WordPack {
    int n = 0;                  // distinct B matrices to pack
    DCsr src[kMaxProb];
    int64_t nnz[kMaxProb];      // entries of each src (its row pointers may be a view's)
    DCsr dst[kMaxProb];         // dst.rp / col / val point into the workspace
    int64_t* part[kMaxProb];    // scan scratch of each
};
// carves the copies out of [base, base + word_pack_bytes...) and fills dst
void word_pack_plan(WordPack& wp, void* base);
// packs every src into dst when the symbolic dense tier's products are at
// least 4 x the entries of all src (packing costs about one pass over B):
// decided on the device from launch_analyze's counters, which then carry
// words_ready for the symbolic dense tier
cudaError_t launch_word_pack(const WordPack& wp, Counters* ctr, const DevInfo& dev,
                             cudaStream_t st);

// ---- launchers (asynchronous on `st`; return the launch error) ----
cudaError_t launch_write_probs(const ProbTable& tab, int nprob, const WsPtrs& w,
                               const DevInfo& dev, cudaStream_t st);
cudaError_t launch_analyze(const WsPtrs& w, int nprob, int64_t R, const Tuning& t,
                           const DevInfo& dev, cudaStream_t st);
// words: every product's Prob.Bw is built (launch_word_pack): the dense tier
// walks the packed copies
cudaError_t launch_symbolic(const WsPtrs& w, int nprob, int64_t R, const Tuning& t,
                            int64_t max_ncols, const DevInfo& dev, cudaStream_t st,
                            bool words = false);
cudaError_t launch_scan_rowptr(const WsPtrs& w, int nprob, int64_t R, const DevInfo& dev,
                               cudaStream_t st);
// in-place exclusive scan of cnt[0, R) (int64), cnt[R] = total; part holds
// scan_parts_needed(R) int64
cudaError_t launch_scan_inplace(int64_t* cnt, int64_t R, int64_t* part, cudaStream_t st);
int64_t scan_parts_needed(int64_t R);
cudaError_t launch_transpose(const DCsr& A, int64_t nnz, int value_bytes, int64_t* t_rp,
                             int32_t* t_col, void* t_val, void* ws, const DevInfo& dev,
                             cudaStream_t st);
size_t transpose_ws_bytes(int64_t ncols, int64_t nnz);
// Slab-start tables of the numeric dense tier, one per distinct B of a call
// (Prob::sp points into them): built by launch_numeric before its kernels.
struct SlabTables {
    int n = 0;
    int64_t slab = 0;           // slab width (columns)
    int nslabs = 0;             // slabs of the widest B; every table's stride is nslabs + 1
    DCsr B[kMaxProb];
    int32_t* sp[kMaxProb];
};
// effective slab width and count of a launch over B's of at most max_ncols columns
void dense_slabs(const Tuning& t, int64_t max_ncols, int64_t* slab, int* nslabs);
cudaError_t launch_numeric(int sr, const WsPtrs& w, const DCsr& B0, int nprob, int64_t R,
                           const Tuning& t, int64_t max_ncols, const DevInfo& dev,
                           cudaStream_t st, const SlabTables* tables = nullptr,
                           const ProbTable* probs_host = nullptr);
// overlap semiring: rows of up to this many outputs take the CTA hash tier
// with 12-byte slots when every position of A and B is below 2^16
constexpr int64_t kOvlCompactMax = 2048;
cudaError_t launch_validate(const DCsr& M, int64_t nnz, DevStatus* status, cudaStream_t st);
// C's row pointers of every product against the nnz its symbolic call counted
// (status->invalid on a mismatch); used by the checked build
cudaError_t launch_check_rowptr(const WsPtrs& w, int nprob, DevStatus* status, cudaStream_t st);
// masked product (masked.cu): accumulators per mask entry; cnt = C's row
// pointers (R + 1), counted then scanned in place
size_t masked_slot_bytes(int sr);
cudaError_t launch_masked_count(int sr, const DCsr& A, const DCsr& B, const DCsr& M,
                                int64_t nnz_m, void* slots, uint8_t* touched, int64_t* cnt,
                                int64_t* part, const DevInfo& dev, cudaStream_t st);
cudaError_t launch_masked_write(int sr, const DCsr& M, const void* slots, const uint8_t* touched,
                                const int64_t* c_rp, int32_t* c_col, void* c_val,
                                DevStatus* status, const DevInfo& dev, cudaStream_t st);
// plus-times FP64/FP32: values of the written C rows recomputed in A's entry
// order (deterministic mode); no-op for other semirings
cudaError_t launch_det_values(int sr, const WsPtrs& w, int nprob, int64_t R, const DevInfo& dev,
                              cudaStream_t st);

// shared-memory bytes of each tier (for tuning clamps and launches)
size_t sym_warp_smem_per_warp(const Tuning& t);
size_t num_warp_smem_per_warp(int sr, const Tuning& t);
size_t num_block_smem(int sr, const Tuning& t);
size_t num_dense_smem(int sr, int64_t slab_cols);

constexpr int kWarpTierWarps = 8;     // warps per CTA in the warp tiers
constexpr int kBlockThreads = 512;    // CTA size of the block and dense tiers

// ---- merge of stage partials (batched) and column split ----

constexpr int kMaxStages = 16;     // partials per merge
constexpr int kMaxMerge = 32;      // merges per batched call

struct MergeProb {
    int64_t nrows, ncols;
    int nparts;
    const int64_t* rp[kMaxStages];
    const int32_t* col[kMaxStages];
    const void* val[kMaxStages];
    int64_t* c_rp;
    int32_t* c_col;
    void* c_val;
    int64_t row_base;   // first flat row
};
struct MergeProbTable {
    MergeProb p[kMaxMerge];
};

SPG_DEV int find_merge_prob(const MergeProb* mp, int nprob, int64_t g) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (mp[mid].row_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// merges of at most this many columns run row by row (bitmap per heavy row)
constexpr int64_t kMergeBitmapCols = (int64_t)1 << 18;

struct MergeWs {
    bool row_path;   // row kernels (else: sort every entry into the merged sequence)
    int32_t* heavy;  // [R] rows with more than 32 entries (row path)
    DevStatus* status;
    Counters* ctr;
    MergeProb* probs;
    int64_t* trp;    // [R + 1] merged-row starts (with duplicates)
    int64_t* cnt;    // [R + 1] distinct counts -> flat C row starts
    int32_t* tcol;   // [T] merged columns
    void* tval;      // [T] merged values
    int64_t* part;   // scan partials
    size_t total;
};
MergeWs merge_ws_layout(void* base, int64_t R, int64_t T, int out_bytes, int64_t max_ncols);

cudaError_t launch_merge_count(int sr, const MergeProbTable& tab, int nprob, int64_t R,
                               int64_t max_part_nnz, int max_parts, int64_t max_ncols,
                               const MergeWs& w, const DevInfo& dev, cudaStream_t st);
cudaError_t launch_merge_rowptr(const MergeWs& w, int nprob, const DevInfo& dev, cudaStream_t st);
cudaError_t launch_merge_write(int sr, const MergeProbTable& tab, int nprob, int64_t R,
                               int64_t max_ncols, const MergeWs& w, const DevInfo& dev,
                               cudaStream_t st);
cudaError_t launch_split_columns(const DCsr& M, int nparts, const int32_t* cuts_dev,
                                 int64_t* prp, int64_t* part_base_dev, int32_t* pcol, void* pval,
                                 int vbytes, int64_t* part, const DevInfo& dev, cudaStream_t st);

// ---- learned sizing (mlp.cu, learned.cu) ----

constexpr size_t kLearnedSmemBudget = 200 * 1024;

struct LearnedWs {
    float* feat;       // [R][4] row features
    float* z;          // [R] network output (logit of nnz / ub)
    int64_t* soff;     // [R + 1] staging offsets (scan of the capacities)
    uint8_t* route;    // [R] 0 learned, 1 exact
    uint8_t* skip;     // [R] skip mask handed to the exact path
    int32_t* scol;     // staging columns
    void* sval;        // staging values
    int64_t entries;   // staging capacity (entries) fixed by the plan
};

int mlp_param_count();
size_t mlp_train_ws_bytes(int64_t B);
// long_rows: R int32 scratch; ctr: its length counter (claim slot 13)
cudaError_t launch_row_features(const Prob* probs, int nprob, int64_t R, float* feat,
                                int64_t* ub, int32_t* long_rows, Counters* ctr,
                                const DevInfo& dev, cudaStream_t st);
// rows with ub[r] <= min_ub are skipped when ub is given
cudaError_t launch_mlp_forward(const float* feat, int64_t R, const void* params, float* z,
                               const int64_t* ub, int64_t min_ub, const DevInfo& dev,
                               cudaStream_t st);
cudaError_t launch_mlp_grad(const float* feat, const float* logt, int64_t B, float tau,
                            const void* params, float* grad, float* loss, void* ws,
                            const DevInfo& dev, cudaStream_t st);
cudaError_t launch_mlp_adam(float* master, float* m, float* v, const float* grad, void* params,
                            float lr, int step, const DevInfo& dev, cudaStream_t st);
cudaError_t launch_mlp_to_bf16(const float* master, void* params, cudaStream_t st);

// largest capacity <= want whose hash table fits the warp (or CTA) tier
int64_t learned_capacity_limit(int sr, int64_t want, bool warp);
cudaError_t launch_learned_caps(const WsPtrs& w, const LearnedWs& lw, int nprob, int64_t R,
                                const float* z, float margin, int64_t exact_max,
                                int64_t learned_max, const DevInfo& dev, cudaStream_t st);
cudaError_t launch_learned_direct(int sr, const WsPtrs& w, const LearnedWs& lw, int nprob,
                                  int64_t R, int64_t warp_max, int64_t block_max,
                                  const DevInfo& dev, cudaStream_t st);
cudaError_t launch_learned_compact(int sr, const WsPtrs& w, const LearnedWs& lw, int nprob,
                                   int64_t R, const DevInfo& dev, cudaStream_t st);

}  // namespace spg
