// C ABI of the SpGEMM library: argument checks, workspace layout, the order
// of the phases, and the host side of errors.  Every arithmetic step runs in
// the kernels of symbolic.cu / numeric.cu.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/spgemm.h"
#include "plan.h"
#include "semiring.cuh"

using namespace spg;

static constexpr size_t kPinnedBytes = 16384;

// Device buffers owned by the handle for the host-memory API.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct spg_handle {
    spg_tuning user;               // user overrides (0 = default)
    DevInfo dev;
    int device;
    std::string err;
    spg_stats stats;
    void* pinned;                  // small pinned staging buffer for device counters
    int64_t launches = 0;          // kernels launched by the last symbolic/numeric call
    StageTimer timer;
    bool timer_events = false;
    // host-memory API state
    cudaStream_t hstream = nullptr;
    DevBuf a_rp, a_col, a_val, b_rp, b_col, b_val, ws, c_rp, c_col, c_val;
    spg_csr hA{}, hB{};            // device descriptors of the last host-API inputs
    int host_sr = -1;
    int64_t host_nnz = -1;
    std::vector<int64_t> host_arp, host_crp;   // host copies of A's and C's row pointers
    cudaStream_t cstream = nullptr;            // download stream of the panel pipeline
    cudaEvent_t ev_done[2] = {}, ev_copied[2] = {};
    bool pipe_events = false;
    DevBuf p_rp[2], p_col[2], p_val[2];        // double-buffered panel outputs
    // checked build: device status of the input validation (256 bytes)
    void* chk_status = nullptr;
    // learned path: values fixed by the last spgemm_learned_plan
    int lrn_sr = -1;
    int64_t lrn_entries = -1, lrn_warp_max = 0, lrn_block_max = 0, lrn_rows = -1;
};

namespace spg {

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

WsLayout ws_layout(int64_t R, int64_t E, size_t slab_bytes, int64_t ncols_b,
                   int64_t cache_bytes, size_t words_bytes) {
    WsLayout L{};
    L.R = R;
    L.E = E;
    size_t o = 0;
    L.status = o;    o = align256(o + sizeof(DevStatus));
    L.counters = o;  o = align256(o + sizeof(Counters));
    L.probs = o;     o = align256(o + sizeof(Prob) * kMaxProb);
    L.ub = o;        o = align256(o + sizeof(int64_t) * (size_t)R);
    L.cnt = o;       o = align256(o + sizeof(int64_t) * (size_t)(R + 1));
    L.rows_sym = o;  o = align256(o + sizeof(int32_t) * (size_t)R);
    L.rows_num = o;  o = align256(o + sizeof(int32_t) * (size_t)R);
    const int64_t nparts = (R + 2047) / 2048;
    L.scan_part = o; o = align256(o + sizeof(int64_t) * (size_t)(nparts + 1));
    L.cursor = o;    o = align256(o + sizeof(int32_t) * (size_t)E);
    L.slab_ptr_bytes = slab_bytes;
    L.slab_ptr = o;  o = align256(o + L.slab_ptr_bytes);
    // bitmap cache: one bitmap of ncols_b bits per cached row (rank kernel rows only)
    L.bm_cache_words = (ncols_b + 1023) / 1024 * 32;
    L.bm_cache_slots = 0;
    if (cache_bytes > 0 && L.bm_cache_words > 0 && L.bm_cache_words * 8 + 16 < 180 * 1024) {
        L.bm_cache_slots = cache_bytes / (L.bm_cache_words * 4);
        if (L.bm_cache_slots > R) L.bm_cache_slots = R;
    }
    L.row_slot = o;  o = align256(o + (L.bm_cache_slots ? sizeof(int32_t) * (size_t)R : 0));
    L.bm_cache_bytes = (size_t)L.bm_cache_slots * (size_t)L.bm_cache_words * 4;
    L.bm_cache = o;  o = align256(o + L.bm_cache_bytes);
    L.words_bytes = words_bytes;
    L.words = o;     o = align256(o + words_bytes);
    L.total = o;
    return L;
}

WsPtrs ws_ptrs(void* ws, const WsLayout& L) {
    char* b = (char*)ws;
    WsPtrs w;
    w.status = (DevStatus*)(b + L.status);
    w.ctr = (Counters*)(b + L.counters);
    w.probs = (Prob*)(b + L.probs);
    w.ub = (int64_t*)(b + L.ub);
    w.cnt = (int64_t*)(b + L.cnt);
    w.rows_sym = (int32_t*)(b + L.rows_sym);
    w.rows_num = (int32_t*)(b + L.rows_num);
    w.scan_part = (int64_t*)(b + L.scan_part);
    w.cursor = (int32_t*)(b + L.cursor);
    w.slab_ptr = L.slab_ptr_bytes ? (int32_t*)(b + L.slab_ptr) : nullptr;
    w.slab_ptr_bytes = L.slab_ptr_bytes;
    w.bm_cache = L.bm_cache_slots ? (uint32_t*)(b + L.bm_cache) : nullptr;
    w.bm_cache_words = L.bm_cache_words;
    w.bm_cache_slots = L.bm_cache_slots;
    w.row_slot = L.bm_cache_slots ? (int32_t*)(b + L.row_slot) : nullptr;
    return w;
}

// Shared-memory budget for one CTA's dynamic allocation (leaves room for the
// kernels' static shared variables).
constexpr size_t kSmemBudget = 200 * 1024;

Tuning default_tuning(int sr) {
    Tuning t;
    t.sym_warp_max_ub = 512;
    t.sym_block_max_ub = 8192;
    t.sym_slab_cols = 1 << 20;
    t.num_warp_max_nnz = 128;
    t.num_block_max_nnz = 2048;
    t.bitmap_cache_bytes = (int64_t)4 << 30;
    t.rank_light_ub = 8192;
    switch (sr) {
        case SR_BOOL: t.dense_slab_cols = 1 << 18; break;
        case SR_MP_F32: case SR_PT_F32: t.dense_slab_cols = 16384; break;
        case SR_OVERLAP: t.dense_slab_cols = 4096; break;
        default: t.dense_slab_cols = 8192; break;
    }
    return t;
}

static int64_t round_down_pow2(int64_t x) {
    int64_t p = 1;
    while (p * 2 <= x) p *= 2;
    return p;
}

Tuning clamp_tuning(Tuning t, int sr) {
    if (t.sym_warp_max_ub < 1) t.sym_warp_max_ub = 1;
    if (t.sym_block_max_ub < t.sym_warp_max_ub) t.sym_block_max_ub = t.sym_warp_max_ub;
    while (sym_warp_smem_per_warp(t) * kWarpTierWarps > kSmemBudget)
        t.sym_warp_max_ub = round_down_pow2(t.sym_warp_max_ub) / 2;
    while ((size_t)next_pow2(2 * t.sym_block_max_ub) * 4 > kSmemBudget)
        t.sym_block_max_ub = round_down_pow2(t.sym_block_max_ub) / 2;
    if (t.sym_block_max_ub < t.sym_warp_max_ub) t.sym_warp_max_ub = t.sym_block_max_ub;
    t.sym_slab_cols = (t.sym_slab_cols + 1023) / 1024 * 1024;
    if (t.sym_slab_cols < 1024) t.sym_slab_cols = 1024;
    while ((size_t)t.sym_slab_cols / 8 > kSmemBudget) t.sym_slab_cols -= 1024;
    if (t.num_warp_max_nnz < 1) t.num_warp_max_nnz = 1;
    if (t.num_block_max_nnz < t.num_warp_max_nnz) t.num_block_max_nnz = t.num_warp_max_nnz;
    while (num_warp_smem_per_warp(sr, t) * kWarpTierWarps > kSmemBudget)
        t.num_warp_max_nnz = round_down_pow2(t.num_warp_max_nnz) / 2;
    while (num_block_smem(sr, t) > kSmemBudget)
        t.num_block_max_nnz = round_down_pow2(t.num_block_max_nnz) / 2;
    if (t.num_block_max_nnz < t.num_warp_max_nnz) t.num_warp_max_nnz = t.num_block_max_nnz;
    t.dense_slab_cols = (t.dense_slab_cols + 1023) / 1024 * 1024;
    if (t.dense_slab_cols < 1024) t.dense_slab_cols = 1024;
    if (t.dense_slab_cols > 65536 * 16) t.dense_slab_cols = 65536 * 16;
    while (num_dense_smem(sr, t.dense_slab_cols) > kSmemBudget && t.dense_slab_cols > 1024)
        t.dense_slab_cols -= 1024;
    if (t.rank_light_ub < 0) t.rank_light_ub = 0;
    if (t.rank_light_ub > ((int64_t)1 << 30)) t.rank_light_ub = (int64_t)1 << 30;
    if (t.rank_light_ub > 0) t.rank_light_ub = next_pow2(t.rank_light_ub);
    return t;
}

}  // namespace spg

// ---------------------------------------------------------------------------------

static spg_status fail(spg_handle* h, spg_status s, const char* fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->err = buf;
    }
    return s;
}

static spg_status cuda_fail(spg_handle* h, cudaError_t e, const char* where) {
    return fail(h, SPG_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static bool sr_valid(int sr) { return sr >= 0 && sr <= 5; }

static Tuning effective_tuning(const spg_handle* h, int sr) {
    Tuning t = default_tuning(sr);
    const spg_tuning& u = h->user;
    if (u.sym_warp_max_ub > 0) t.sym_warp_max_ub = u.sym_warp_max_ub;
    if (u.sym_block_max_ub > 0) t.sym_block_max_ub = u.sym_block_max_ub;
    if (u.num_warp_max_nnz > 0) t.num_warp_max_nnz = u.num_warp_max_nnz;
    if (u.num_block_max_nnz > 0) t.num_block_max_nnz = u.num_block_max_nnz;
    if (u.dense_slab_cols > 0) t.dense_slab_cols = u.dense_slab_cols;
    if (u.sym_slab_cols > 0) t.sym_slab_cols = u.sym_slab_cols;
    if (u.bitmap_cache_bytes != 0) t.bitmap_cache_bytes = u.bitmap_cache_bytes;
    if (u.rank_light_ub != 0) t.rank_light_ub = u.rank_light_ub;
    return clamp_tuning(t, sr);
}

static DCsr to_dcsr(const spg_csr* M) {
    return DCsr{M->nrows, M->ncols, M->row_ptr, M->col, M->val};
}

// Distinct B matrices of a call (the same arrays passed for several products
// count once): idx[p] = the index of product p's B among them; returns their
// number.
static int distinct_b(int nprob, const spg_csr* B, int* idx, int* first) {
    int n = 0;
    for (int p = 0; p < nprob; ++p) {
        int j = 0;
        for (; j < n; ++j) {
            const spg_csr& o = B[first[j]];
            if (o.row_ptr == B[p].row_ptr && o.col == B[p].col && o.nrows == B[p].nrows &&
                o.nnz == B[p].nnz && o.ncols == B[p].ncols)
                break;
        }
        if (j == n) first[n++] = p;
        idx[p] = j;
    }
    return n;
}

// Room for the word-packed copies of the distinct B matrices (0: the call
// walks B's columns; the packing pays only for large enough B).
static size_t words_bytes_for(int nprob, const spg_csr* B) {
    int idx[kMaxProb], first[kMaxProb];
    const int n = distinct_b(nprob, B, idx, first);
    int64_t nnz = 0;
    size_t bytes = 0;
    for (int j = 0; j < n; ++j) {
        nnz += B[first[j]].nnz;
        bytes += word_pack_bytes(B[first[j]].nrows, B[first[j]].nnz);
    }
    return nnz >= kWordPackMinNnz ? bytes : 0;
}

// Slab-start tables of the numeric dense tier: one per distinct B, all with
// the launch's slab count (from the widest B); a B whose table would be
// larger than twice its column array (plus 64 MB) gets none (its rows use
// per-entry cursors).  Returns the bytes; with `out`, also carves the tables
// out of `base` and points the products at them.
static size_t slab_tables(int nprob, const spg_csr* B, const Tuning& t, void* base,
                          ProbTable* tab, SlabTables* out) {
    int64_t maxc = 0;
    for (int p = 0; p < nprob; ++p) maxc = B[p].ncols > maxc ? B[p].ncols : maxc;
    int64_t slab;
    int nslabs;
    dense_slabs(t, maxc, &slab, &nslabs);
    if (out) {
        out->n = 0;
        out->slab = slab;
        out->nslabs = nslabs;
    }
    if (nslabs <= 1) return 0;
    int idx[kMaxProb], first[kMaxProb];
    const int n = distinct_b(nprob, B, idx, first);
    size_t total = 0;
    int32_t* table[kMaxProb];
    for (int j = 0; j < n; ++j) {
        const spg_csr& b = B[first[j]];
        const size_t need = (size_t)(b.nrows + 1) * (size_t)(nslabs + 1) * 4;
        const size_t cap = (size_t)b.nnz * 8 + ((size_t)64 << 20);
        table[j] = nullptr;
        if (need > cap || b.nnz == 0) continue;
        if (out) {
            table[j] = (int32_t*)((char*)base + total);
            out->B[out->n] = to_dcsr(&b);
            out->sp[out->n] = table[j];
            ++out->n;
        }
        total += align256(need);
    }
    if (tab)
        for (int p = 0; p < nprob; ++p) tab->p[p].sp = table[idx[p]];
    return total;
}

static size_t slab_bytes_for(int nprob, const spg_csr* B, const Tuning& t) {
    return slab_tables(nprob, B, t, nullptr, nullptr, nullptr);
}

// workspace of one product: the bitmap cache is kept only when the symbolic
// dense tier sees whole rows in one slab and SR is not pattern-free of use
static WsLayout layout_for(const spg_csr* A, const spg_csr* B, const Tuning& t) {
    const int64_t cache = (t.bitmap_cache_bytes > 0 && B->ncols <= t.sym_slab_cols)
                              ? t.bitmap_cache_bytes : 0;
    return ws_layout(A->nrows, A->nnz, slab_bytes_for(1, B, t), B->ncols, cache,
                     words_bytes_for(1, B));
}



// Points every product's Prob::Bw at its B's word-packed copy in the
// workspace (when the layout has room for them) and lists the copies to
// build; returns whether the symbolic dense tier walks them.
static bool plan_words(int nprob, const spg_csr* B, void* workspace, const WsLayout& L,
                       ProbTable* tab, WordPack* wp) {
    wp->n = 0;
    if (L.words_bytes == 0) return false;
    int idx[kMaxProb], first[kMaxProb];
    wp->n = distinct_b(nprob, B, idx, first);
    for (int j = 0; j < wp->n; ++j) {
        wp->src[j] = to_dcsr(B + first[j]);
        wp->nnz[j] = B[first[j]].nnz;
    }
    word_pack_plan(*wp, (char*)workspace + L.words);
    for (int p = 0; p < nprob; ++p) tab->p[p].Bw = wp->dst[idx[p]];
    return true;
}

static spg_status check_csr_arg(spg_handle* h, const spg_csr* M, const char* name, int sr,
                                bool need_val) {
    if (!M) return fail(h, SPG_ERR_INVALID_ARG, "%s is NULL", name);
    if (M->nrows < 0 || M->ncols < 0 || M->nnz < 0)
        return fail(h, SPG_ERR_INVALID_ARG, "%s has a negative size", name);
    if (M->nrows >= INT32_MAX || M->ncols >= INT32_MAX)
        return fail(h, SPG_ERR_UNSUPPORTED, "%s: rows and columns must be < 2^31 - 1", name);
    if (!M->row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "%s.row_ptr is NULL", name);
    if (M->nnz > 0 && !M->col) return fail(h, SPG_ERR_INVALID_ARG, "%s.col is NULL", name);
    if (need_val && sr != SR_BOOL && M->nnz > 0 && !M->val)
        return fail(h, SPG_ERR_INVALID_ARG, "%s.val is NULL", name);
    return SPG_OK;
}

static spg_status check_pair(spg_handle* h, int sr, const spg_csr* A, const spg_csr* B,
                             bool need_val) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (!sr_valid(sr)) return fail(h, SPG_ERR_INVALID_ARG, "unknown semiring id %d", sr);
    spg_status s = check_csr_arg(h, A, "A", sr, need_val);
    if (s != SPG_OK) return s;
    s = check_csr_arg(h, B, "B", sr, need_val);
    if (s != SPG_OK) return s;
    if (A->ncols != B->nrows)
        return fail(h, SPG_ERR_INVALID_ARG, "A.ncols (%lld) != B.nrows (%lld)",
                    (long long)A->ncols, (long long)B->nrows);
    return SPG_OK;
}

extern "C" {

spg_status spgemm_create(spg_handle** handle) {
    if (!handle) return SPG_ERR_INVALID_ARG;
    *handle = nullptr;
    spg_handle* h = new spg_handle();
    std::memset(&h->user, 0, sizeof h->user);
    std::memset(&h->stats, 0, sizeof h->stats);
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->dev.sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->dev.max_smem_optin,
                                   cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&h->dev.max_smem_sm,
                                   cudaDevAttrMaxSharedMemoryPerMultiprocessor, h->device);
    if (e == cudaSuccess) e = cudaMallocHost(&h->pinned, kPinnedBytes);
    if (e != cudaSuccess) {
        delete h;
        return SPG_ERR_CUDA;
    }
    h->dev.launches = &h->launches;
    h->dev.timer = &h->timer;
    *handle = h;
    return SPG_OK;
}

spg_status spgemm_destroy(spg_handle* h) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (h->pinned) cudaFreeHost(h->pinned);
    if (h->chk_status) cudaFree(h->chk_status);
    if (h->timer_events)
        for (int i = 0; i < StageTimer::kMax; ++i) cudaEventDestroy(h->timer.ev[i]);
    for (DevBuf* b : {&h->a_rp, &h->a_col, &h->a_val, &h->b_rp, &h->b_col, &h->b_val, &h->ws,
                      &h->c_rp, &h->c_col, &h->c_val, &h->p_rp[0], &h->p_rp[1], &h->p_col[0],
                      &h->p_col[1], &h->p_val[0], &h->p_val[1]})
        if (b->p) cudaFree(b->p);
    if (h->pipe_events)
        for (int i = 0; i < 2; ++i) {
            cudaEventDestroy(h->ev_done[i]);
            cudaEventDestroy(h->ev_copied[i]);
        }
    if (h->cstream) cudaStreamDestroy(h->cstream);
    if (h->hstream) cudaStreamDestroy(h->hstream);
    delete h;
    return SPG_OK;
}

spg_status spgemm_set_timing(spg_handle* h, int enable) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (enable && !h->timer_events) {
        for (int i = 0; i < StageTimer::kMax; ++i) {
            cudaError_t e = cudaEventCreate(&h->timer.ev[i]);
            if (e != cudaSuccess) return cuda_fail(h, e, "event create");
        }
        h->timer_events = true;
    }
    h->timer.on = enable != 0;
    h->timer.n = 0;
    return SPG_OK;
}

spg_status spgemm_get_stage_times(spg_handle* h, float* ms, int n) {
    if (!h || !ms || n < kStCount) return SPG_ERR_INVALID_ARG;
    for (int i = 0; i < kStCount; ++i) ms[i] = 0.f;
    StageTimer& t = h->timer;
    if (!h->timer_events || t.n == 0) return SPG_OK;
    cudaError_t e = cudaEventSynchronize(t.ev[t.n - 1]);
    if (e != cudaSuccess) return cuda_fail(h, e, "event sync");
    for (int i = 1; i < t.n; ++i) {
        float d = 0.f;
        e = cudaEventElapsedTime(&d, t.ev[i - 1], t.ev[i]);
        if (e != cudaSuccess) return cuda_fail(h, e, "event time");
        ms[t.tag[i]] += d;
    }
    return SPG_OK;
}

const char* spgemm_last_error(const spg_handle* h) { return h ? h->err.c_str() : "no handle"; }

spg_status spgemm_set_tuning(spg_handle* h, const spg_tuning* t) {
    if (!h || !t) return SPG_ERR_INVALID_ARG;
    h->user = *t;
    return SPG_OK;
}

spg_status spgemm_get_tuning(const spg_handle* h, spg_tuning* t) {
    if (!h || !t) return SPG_ERR_INVALID_ARG;
    // report the effective values for plus-times FP64 where the user left 0
    *t = h->user;
    return SPG_OK;
}

spg_status spgemm_get_stats(const spg_handle* h, spg_stats* s) {
    if (!h || !s) return SPG_ERR_INVALID_ARG;
    *s = h->stats;
    s->launches = h->launches;
    return SPG_OK;
}

spg_status spgemm_workspace_size(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                 const spg_csr* B, size_t* bytes) {
    spg_status s = check_pair(h, sr, A, B, false);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    const Tuning t = effective_tuning(h, sr);
    *bytes = layout_for(A, B, t).total;
    return SPG_OK;
}

static spg_status read_status(spg_handle* h, const WsPtrs& w, cudaStream_t st) {
    DevStatus* hs = (DevStatus*)h->pinned;
    cudaError_t e = cudaMemcpyAsync(hs, w.status, sizeof(DevStatus), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "status read");
    if (hs->overflow)
        return fail(h, SPG_ERR_OVERFLOW, "hash table overflow or inconsistent counts (flat row %lld)",
                    (long long)hs->info[0]);
    if (hs->invalid)
        return fail(h, SPG_ERR_INVALID_CSR, "invalid CSR (row %lld)", (long long)hs->info[1]);
    return SPG_OK;
}

#ifdef SPG_CHECKS
// Checked build: the input matrices are validated on the device (bounds-safe,
// spgemm_validate_csr's kernel) and the call returns SPG_ERR_INVALID_CSR
// before any product kernel is queued on a malformed matrix.  Synchronises.
static spg_status checked_inputs(spg_handle* h, int n, const spg_csr* const* mats,
                                 cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    if (!h->chk_status) e = cudaMalloc(&h->chk_status, 256);
    if (e != cudaSuccess) return cuda_fail(h, e, "checked build status");
    DevStatus* ds = (DevStatus*)h->chk_status;
    e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        const spg_csr* M = mats[i];
        bool seen = false;   // the same matrix passed twice (A = B) is checked once
        for (int j = 0; j < i; ++j)
            seen |= mats[j]->row_ptr == M->row_ptr && mats[j]->col == M->col &&
                    mats[j]->nrows == M->nrows && mats[j]->ncols == M->ncols;
        if (!seen) e = launch_validate(to_dcsr(M), M->nnz, ds, st);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "validate");
    WsPtrs w{};
    w.status = ds;
    spg_status s = read_status(h, w, st);
    if (s == SPG_ERR_INVALID_CSR) h->err = "checked build: an input matrix is not valid CSR (" + h->err + ")";
    return s;
}

static spg_status checked_pairs(spg_handle* h, int nprob, const spg_csr* A, const spg_csr* B,
                                cudaStream_t st) {
    std::vector<const spg_csr*> mats;
    for (int p = 0; p < nprob; ++p) {
        mats.push_back(A + p);
        mats.push_back(B + p);
    }
    return checked_inputs(h, (int)mats.size(), mats.data(), st);
}
#endif

// ---- symbolic / numeric, single and batched ---------------------------------------

static spg_status check_batch(spg_handle* h, int sr, int nprob, const spg_csr* A,
                              const spg_csr* B, bool need_val) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (nprob < 1 || nprob > kMaxProb)
        return fail(h, SPG_ERR_INVALID_ARG, "batch of %d products (1..%d)", nprob, kMaxProb);
    if (!A || !B) return fail(h, SPG_ERR_INVALID_ARG, "A / B is NULL");
    int64_t R = 0;
    for (int p = 0; p < nprob; ++p) {
        spg_status s = check_pair(h, sr, A + p, B + p, need_val);
        if (s != SPG_OK) return s;
        R += A[p].nrows;
    }
    if (R >= INT32_MAX) return fail(h, SPG_ERR_UNSUPPORTED, "batch has >= 2^31 rows");
    return SPG_OK;
}

static WsLayout layout_batch(int nprob, const spg_csr* A, const spg_csr* B, const Tuning& t) {
    if (nprob == 1) return layout_for(A, B, t);
    int64_t R = 0, E = 0, maxc = 0;
    for (int p = 0; p < nprob; ++p) {
        R += A[p].nrows;
        E += A[p].nnz;
        if (B[p].ncols > maxc) maxc = B[p].ncols;
    }
    // no slab table for batches (segments come from per-entry cursors)
    const int64_t cache = (t.bitmap_cache_bytes > 0 && maxc <= t.sym_slab_cols) ? t.bitmap_cache_bytes : 0;
    return ws_layout(R, E, slab_bytes_for(nprob, B, t), maxc, cache, words_bytes_for(nprob, B));
}

static void fill_probs(ProbTable* tab, int nprob, const spg_csr* A, const spg_csr* B,
                       int64_t* const* c_rp, int32_t* const* c_col, void* const* c_val) {
    std::memset(tab, 0, sizeof *tab);
    int64_t rb = 0, eb = 0;
    for (int p = 0; p < nprob; ++p) {
        tab->p[p] = Prob{to_dcsr(A + p), to_dcsr(B + p), DCsr{},   // Bw: set by plan_words
                         nullptr,                                    // sp: set by plan_slab_tables
                         c_rp[p], c_col ? c_col[p] : nullptr, c_val ? c_val[p] : nullptr, rb, eb};
        rb += A[p].nrows;
        eb += A[p].nnz;
    }
}

static int64_t max_ncols(int nprob, const spg_csr* B) {
    int64_t m = 0;
    for (int p = 0; p < nprob; ++p) m = B[p].ncols > m ? B[p].ncols : m;
    return m;
}

// Launches of the symbolic phase, no host synchronisation.  reset_status =
// false keeps the error flags of earlier calls in the same workspace.
static spg_status symbolic_launch(spg_handle* h, int sr, int nprob, const spg_csr* A,
                                  const spg_csr* B, int64_t* const* c_row_ptr, void* workspace,
                                  size_t workspace_bytes, cudaStream_t st, bool reset_status,
                                  WsLayout* Lout, WsPtrs* wout) {
    const Tuning t = effective_tuning(h, sr);
    const WsLayout L = layout_batch(nprob, A, B, t);
    if (!workspace || workspace_bytes < L.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", L.total);
    const WsPtrs w = ws_ptrs(workspace, L);
#ifdef SPG_CHECKS
    {
        const spg_status cs = checked_pairs(h, nprob, A, B, st);
        if (cs != SPG_OK) return cs;
    }
#endif
    h->launches = 0;
    h->timer.n = 0;
    cudaError_t e = reset_status ? cudaMemsetAsync(workspace, 0, L.probs, st)   // status + counters
                                 : cudaMemsetAsync(w.ctr, 0, sizeof(Counters), st);
    if (e == cudaSuccess && w.row_slot)
        e = cudaMemsetAsync(w.row_slot, 0xff, sizeof(int32_t) * (size_t)L.R, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    ProbTable* tab = new ProbTable;
    WordPack* wp = new WordPack;
    fill_probs(tab, nprob, A, B, c_row_ptr, nullptr, nullptr);
    const bool words = plan_words(nprob, B, workspace, L, tab, wp);
    e = launch_write_probs(*tab, nprob, w, h->dev, st);
    delete tab;
    if (e == cudaSuccess) e = launch_analyze(w, nprob, L.R, t, h->dev, st);
    if (e == cudaSuccess && words) e = launch_word_pack(*wp, w.ctr, h->dev, st);
    delete wp;
    if (e == cudaSuccess)
        e = launch_symbolic(w, nprob, L.R, t, max_ncols(nprob, B), h->dev, st, words);
    if (e == cudaSuccess) e = launch_scan_rowptr(w, nprob, L.R, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "symbolic launch");
    if (Lout) *Lout = L;
    if (wout) *wout = w;
    return SPG_OK;
}

static spg_status symbolic_impl(spg_handle* h, int sr, int nprob, const spg_csr* A,
                                const spg_csr* B, int64_t* const* c_row_ptr, int64_t* c_nnz,
                                void* workspace, size_t workspace_bytes, cudaStream_t st) {
    WsLayout L;
    WsPtrs w;
    spg_status s = symbolic_launch(h, sr, nprob, A, B, c_row_ptr, workspace, workspace_bytes, st,
                                   true, &L, &w);
    if (s != SPG_OK) return s;
    if (!c_nnz) return SPG_OK;   // no host copy, no synchronisation (see the header)
    // bring back nnz, products, bin counts and the status in one copy
    Counters* hc = (Counters*)((char*)h->pinned);
    static_assert(sizeof(Counters) <= kPinnedBytes, "staging buffer too small");
    cudaError_t e = cudaMemcpyAsync(hc, w.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "symbolic");
    int64_t tot = 0;
    for (int p = 0; p < nprob; ++p) {
        c_nnz[p] = hc->nnz[p];
        tot += hc->nnz[p];
    }
    h->stats.products = (int64_t)hc->products;
    h->stats.nnz_c = tot;
    for (int tier = 0; tier < kSymTiers; ++tier) {
        int64_t n = 0;
        for (int b = 0; b < kSubBins; ++b) n += hc->sym_bin_count[tier * kSubBins + b];
        h->stats.rows_per_tier[tier] = n;
    }
    return read_status(h, w, st);
}

static spg_status numeric_impl(spg_handle* h, int sr, int nprob, const spg_csr* A,
                               const spg_csr* B, const int64_t* const* c_row_ptr,
                               int32_t* const* c_col, void* const* c_val, void* workspace,
                               size_t workspace_bytes, cudaStream_t st) {
    const Tuning t = effective_tuning(h, sr);
    const WsLayout L = layout_batch(nprob, A, B, t);
    if (!workspace || workspace_bytes < L.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", L.total);
    const WsPtrs w = ws_ptrs(workspace, L);
#ifdef SPG_CHECKS
    {
        const spg_status cs = checked_pairs(h, nprob, A, B, st);
        if (cs != SPG_OK) return cs;
    }
#endif
    h->launches = 0;
    h->timer.n = 0;
    std::unique_ptr<ProbTable> tab(new ProbTable);
    std::unique_ptr<SlabTables> spt(new SlabTables);
    fill_probs(tab.get(), nprob, A, B, const_cast<int64_t* const*>(c_row_ptr), c_col, c_val);
    if (w.slab_ptr) slab_tables(nprob, B, t, w.slab_ptr, tab.get(), spt.get());
    cudaError_t e = launch_write_probs(*tab, nprob, w, h->dev, st);
#ifdef SPG_CHECKS
    // C's row pointers must be those of the symbolic call that left this
    // workspace (their last entry its nnz(C)): no kernel writes C otherwise.
    // The result goes to the handle's own status, so a refused call leaves
    // the workspace's error flags as they were.
    if (e == cudaSuccess) e = cudaMemsetAsync(h->chk_status, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = launch_check_rowptr(w, nprob, (DevStatus*)h->chk_status, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "row pointer check");
    {
        WsPtrs cw{};
        cw.status = (DevStatus*)h->chk_status;
        const spg_status cs = read_status(h, cw, st);
        if (cs == SPG_ERR_INVALID_CSR) {
            h->err = "checked build: C's row pointers are not those of the symbolic call (" + h->err + ")";
            return cs;
        }
        if (cs != SPG_OK) return cs;
    }
#endif
    if (e == cudaSuccess)
        e = launch_numeric(sr, w, to_dcsr(B), nprob, L.R, t, max_ncols(nprob, B), h->dev, st,
                           spt.get(), tab.get());
    if (e == cudaSuccess && h->user.deterministic)
        e = launch_det_values(sr, w, nprob, L.R, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "numeric launch");
    return SPG_OK;
}

spg_status spgemm_symbolic(spg_handle* h, spg_semiring sr, const spg_csr* A, const spg_csr* B,
                           int64_t* c_row_ptr, int64_t* c_nnz, void* workspace,
                           size_t workspace_bytes, void* stream) {
    spg_status s = check_pair(h, sr, A, B, false);
    if (s != SPG_OK) return s;
    if (!c_row_ptr || !c_nnz) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr / c_nnz is NULL");
    return symbolic_impl(h, sr, 1, A, B, &c_row_ptr, c_nnz, workspace, workspace_bytes,
                         (cudaStream_t)stream);
}

spg_status spgemm_numeric(spg_handle* h, spg_semiring sr, const spg_csr* A, const spg_csr* B,
                          const int64_t* c_row_ptr, int32_t* c_col, void* c_val,
                          void* workspace, size_t workspace_bytes, void* stream) {
    spg_status s = check_pair(h, sr, A, B, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr is NULL");
    return numeric_impl(h, sr, 1, A, B, &c_row_ptr, &c_col, &c_val, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}

spg_status spgemm_workspace_size_batched(spg_handle* h, spg_semiring sr, int nprob,
                                         const spg_csr* A, const spg_csr* B, size_t* bytes) {
    spg_status s = check_batch(h, sr, nprob, A, B, false);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = layout_batch(nprob, A, B, effective_tuning(h, sr)).total;
    return SPG_OK;
}

spg_status spgemm_symbolic_batched(spg_handle* h, spg_semiring sr, int nprob, const spg_csr* A,
                                   const spg_csr* B, int64_t* const* c_row_ptr, int64_t* c_nnz,
                                   void* workspace, size_t workspace_bytes, void* stream) {
    spg_status s = check_batch(h, sr, nprob, A, B, false);
    if (s != SPG_OK) return s;
    if (!c_row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr is NULL");
    for (int p = 0; p < nprob; ++p)
        if (!c_row_ptr[p]) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr[%d] is NULL", p);
    return symbolic_impl(h, sr, nprob, A, B, c_row_ptr, c_nnz, workspace, workspace_bytes,
                         (cudaStream_t)stream);
}

spg_status spgemm_numeric_batched(spg_handle* h, spg_semiring sr, int nprob, const spg_csr* A,
                                  const spg_csr* B, const int64_t* const* c_row_ptr,
                                  int32_t* const* c_col, void* const* c_val, void* workspace,
                                  size_t workspace_bytes, void* stream) {
    spg_status s = check_batch(h, sr, nprob, A, B, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr || !c_col) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr / c_col is NULL");
    return numeric_impl(h, sr, nprob, A, B, c_row_ptr, c_col, c_val, workspace, workspace_bytes,
                        (cudaStream_t)stream);
}

// ---- merge of stage partials ---------------------------------------------------------

static spg_status merge_check(spg_handle* h, int sr, int nmerge, const int* nparts,
                              const spg_csr* parts, int64_t* R, int64_t* T, int64_t* maxp,
                              int* maxs, int64_t* maxc) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (!sr_valid(sr)) return fail(h, SPG_ERR_INVALID_ARG, "unknown semiring id %d", sr);
    if (nmerge < 1 || nmerge > kMaxMerge || !nparts || !parts)
        return fail(h, SPG_ERR_INVALID_ARG, "merges: 1..%d, nparts and parts non-NULL", kMaxMerge);
    *R = *T = *maxp = 0;
    *maxs = 0;
    *maxc = 0;
    int off = 0;
    for (int m = 0; m < nmerge; ++m) {
        if (nparts[m] < 1 || nparts[m] > kMaxStages)
            return fail(h, SPG_ERR_INVALID_ARG, "merge %d: 1..%d partials", m, kMaxStages);
        for (int s = 0; s < nparts[m]; ++s) {
            const spg_csr* P = parts + off + s;
            spg_status st = check_csr_arg(h, P, "partial", sr, true);
            if (st != SPG_OK) return st;
            if (P->nrows != parts[off].nrows || P->ncols != parts[off].ncols)
                return fail(h, SPG_ERR_INVALID_ARG, "merge %d: partials differ in shape", m);
            *T += P->nnz;
            if (P->nnz > *maxp) *maxp = P->nnz;
        }
        *R += parts[off].nrows;
        if (parts[off].ncols > *maxc) *maxc = parts[off].ncols;
        if (nparts[m] > *maxs) *maxs = nparts[m];
        off += nparts[m];
    }
    if (*R >= INT32_MAX) return fail(h, SPG_ERR_UNSUPPORTED, "too many rows");
    return SPG_OK;
}

static void fill_merge_probs(MergeProbTable* tab, int nmerge, const int* nparts,
                             const spg_csr* parts, int64_t* const* c_rp, int32_t* const* c_col,
                             void* const* c_val) {
    std::memset(tab, 0, sizeof *tab);
    int off = 0;
    int64_t rb = 0;
    for (int m = 0; m < nmerge; ++m) {
        MergeProb& M = tab->p[m];
        M.nrows = parts[off].nrows;
        M.ncols = parts[off].ncols;
        M.nparts = nparts[m];
        for (int s = 0; s < nparts[m]; ++s) {
            M.rp[s] = parts[off + s].row_ptr;
            M.col[s] = parts[off + s].col;
            M.val[s] = parts[off + s].val;
        }
        M.c_rp = c_rp[m];
        M.c_col = c_col ? c_col[m] : nullptr;
        M.c_val = c_val ? c_val[m] : nullptr;
        M.row_base = rb;
        rb += M.nrows;
        off += nparts[m];
    }
}

spg_status spgemm_merge_workspace_size(spg_handle* h, spg_semiring sr, int nmerge,
                                       const int* nparts, const spg_csr* parts, size_t* bytes) {
    int64_t R, T, mp, mc;
    int ms;
    spg_status s = merge_check(h, sr, nmerge, nparts, parts, &R, &T, &mp, &ms, &mc);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = merge_ws_layout(nullptr, R, T, out_bytes(sr), mc).total;
    return SPG_OK;
}

spg_status spgemm_merge_stages_batched(spg_handle* h, spg_semiring sr, int nmerge,
                                       const int* nparts, const spg_csr* parts,
                                       int64_t* const* c_row_ptr, int64_t* c_nnz,
                                       int32_t* const* c_col, void* const* c_val,
                                       void* workspace, size_t workspace_bytes, void* stream) {
    int64_t R, T, maxp, maxc;
    int maxs;
    spg_status s = merge_check(h, sr, nmerge, nparts, parts, &R, &T, &maxp, &maxs, &maxc);
    if (s != SPG_OK) return s;
    if (!c_row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr is NULL");
    for (int m = 0; m < nmerge; ++m)
        if (!c_row_ptr[m]) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr[%d] is NULL", m);
    const MergeWs w = merge_ws_layout(workspace, R, T, out_bytes(sr), maxc);
    if (!workspace || workspace_bytes < w.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", w.total);
    cudaStream_t st = (cudaStream_t)stream;
    h->launches = 0;
    h->timer.n = 0;
    MergeProbTable* tab = new MergeProbTable;
    fill_merge_probs(tab, nmerge, nparts, parts, c_row_ptr, c_col, c_val);
    cudaError_t e;
    if (!c_col) {   // count: C row pointers and nnz
        e = cudaMemsetAsync(workspace, 0, (char*)w.probs - (char*)workspace, st);
        if (e == cudaSuccess)
            e = launch_merge_count(sr, *tab, nmerge, R, maxp, maxs, maxc, w, h->dev, st);
        if (e == cudaSuccess) e = launch_merge_rowptr(w, nmerge, h->dev, st);
        delete tab;
        if (e != cudaSuccess) return cuda_fail(h, e, "merge count");
        if (!c_nnz) return SPG_OK;   // no host copy, no synchronisation (see the header)
        Counters* hc = (Counters*)h->pinned;
        e = cudaMemcpyAsync(hc, w.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(h, e, "merge count");
        for (int m = 0; m < nmerge; ++m) c_nnz[m] = hc->nnz[m];
        return SPG_OK;
    }
    for (int m = 0; m < nmerge; ++m)
        if (!c_col[m] || (out_bytes(sr) && (!c_val || !c_val[m]))) {
            delete tab;
            return fail(h, SPG_ERR_INVALID_ARG, "c_col / c_val of merge %d is NULL", m);
        }
    e = launch_merge_write(sr, *tab, nmerge, R, maxc, w, h->dev, st);
    delete tab;
    if (e != cudaSuccess) return cuda_fail(h, e, "merge write");
    return SPG_OK;
}

spg_status spgemm_merge_stages(spg_handle* h, spg_semiring sr, int nstages, const spg_csr* parts,
                               int64_t* c_row_ptr, int64_t* c_nnz, int32_t* c_col, void* c_val,
                               void* workspace, size_t workspace_bytes, void* stream) {
    return spgemm_merge_stages_batched(h, sr, 1, &nstages, parts, &c_row_ptr, c_nnz,
                                       c_col ? &c_col : nullptr, c_col ? &c_val : nullptr,
                                       workspace, workspace_bytes, stream);
}

// ---- column split -----------------------------------------------------------------

static size_t split_ws_bytes(int64_t nrows, int nparts) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(sizeof(int32_t) * (size_t)(nparts + 1)) + al(sizeof(int64_t) * (size_t)(nparts + 1)) +
           al(sizeof(int64_t) * (size_t)scan_parts_needed(nrows));
}

spg_status spgemm_split_workspace_size(spg_handle* h, const spg_csr* M, int nparts, size_t* bytes) {
    if (!h) return SPG_ERR_INVALID_ARG;
    spg_status s = check_csr_arg(h, M, "M", SR_BOOL, false);
    if (s != SPG_OK) return s;
    if (nparts < 1 || !bytes) return fail(h, SPG_ERR_INVALID_ARG, "nparts >= 1 and bytes");
    *bytes = split_ws_bytes(M->nrows, nparts);
    return SPG_OK;
}

spg_status spgemm_split_columns(spg_handle* h, const spg_csr* M, int nparts, const int32_t* cuts,
                                int value_bytes, int64_t* part_row_ptr, int32_t* part_col,
                                void* part_val, int64_t* part_nnz, void* workspace,
                                size_t workspace_bytes, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    spg_status s = check_csr_arg(h, M, "M", SR_BOOL, false);
    if (s != SPG_OK) return s;
    if (nparts < 1 || !cuts || !part_row_ptr || !part_nnz || (M->nnz > 0 && !part_col))
        return fail(h, SPG_ERR_INVALID_ARG, "split: NULL argument or nparts < 1");
    if (value_bytes < 0 || value_bytes > 64 || (value_bytes && M->nnz > 0 && (!M->val || !part_val)))
        return fail(h, SPG_ERR_INVALID_ARG, "split: bad value_bytes or NULL values");
    if (cuts[0] != 0 || cuts[nparts] != M->ncols)
        return fail(h, SPG_ERR_INVALID_ARG, "split: cuts must run from 0 to ncols");
    for (int p = 0; p < nparts; ++p)
        if (cuts[p + 1] < cuts[p]) return fail(h, SPG_ERR_INVALID_ARG, "split: cuts must not decrease");
    if (!workspace || workspace_bytes < split_ws_bytes(M->nrows, nparts))
        return fail(h, SPG_ERR_WORKSPACE, "split workspace too small");
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* b = (char*)workspace;
    int32_t* cuts_dev = (int32_t*)b;
    int64_t* base_dev = (int64_t*)(b + al(sizeof(int32_t) * (size_t)(nparts + 1)));
    int64_t* part = (int64_t*)((char*)base_dev + al(sizeof(int64_t) * (size_t)(nparts + 1)));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(cuts_dev, cuts, sizeof(int32_t) * (size_t)(nparts + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_split_columns(to_dcsr(M), nparts, cuts_dev, part_row_ptr, base_dev, part_col,
                                 part_val, value_bytes, part, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "split");
    int64_t* hb = (int64_t*)h->pinned;
    if ((size_t)(nparts + 1) * 8 > kPinnedBytes) return fail(h, SPG_ERR_UNSUPPORTED, "too many parts");
    e = cudaMemcpyAsync(hb, base_dev, sizeof(int64_t) * (size_t)(nparts + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "split");
    for (int p = 0; p < nparts; ++p) part_nnz[p] = hb[p + 1] - hb[p];
    return SPG_OK;
}

spg_status spgemm_check(spg_handle* h, void* workspace, void* stream) {
    if (!h || !workspace) return SPG_ERR_INVALID_ARG;
    const WsLayout L = ws_layout(0, 0, 0, 0, 0, 0);
    return read_status(h, ws_ptrs(workspace, L), (cudaStream_t)stream);
}

spg_status spgemm_transpose_workspace_size(spg_handle* h, const spg_csr* A, size_t* bytes) {
    if (!h) return SPG_ERR_INVALID_ARG;
    spg_status s = check_csr_arg(h, A, "A", SR_BOOL, false);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = transpose_ws_bytes(A->ncols, A->nnz);
    return SPG_OK;
}

spg_status spgemm_transpose(spg_handle* h, const spg_csr* A, int value_bytes,
                            int64_t* t_row_ptr, int32_t* t_col, void* t_val, void* workspace,
                            size_t workspace_bytes, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    spg_status s = check_csr_arg(h, A, "A", SR_BOOL, false);
    if (s != SPG_OK) return s;
    if (A->nnz >= INT32_MAX) return fail(h, SPG_ERR_UNSUPPORTED, "transpose needs nnz < 2^31 - 1");
    if (value_bytes < 0 || value_bytes > 64)
        return fail(h, SPG_ERR_INVALID_ARG, "value_bytes must be in [0, 64]");
    if (value_bytes > 0 && A->nnz > 0 && (!A->val || !t_val))
        return fail(h, SPG_ERR_INVALID_ARG, "values requested but A.val or t_val is NULL");
    if (!t_row_ptr || (A->nnz > 0 && !t_col))
        return fail(h, SPG_ERR_INVALID_ARG, "t_row_ptr / t_col is NULL");
    const size_t need = transpose_ws_bytes(A->ncols, A->nnz);
    if (!workspace || workspace_bytes < need)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaError_t e = launch_transpose(to_dcsr(A), A->nnz, value_bytes, t_row_ptr, t_col, t_val,
                                     workspace, h->dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "transpose");
    return SPG_OK;
}

// ---- host-memory API ------------------------------------------------------------

// device bytes held by the handle's host-API buffers
static size_t held_bytes(const spg_handle* h) {
    const DevBuf* all[] = {&h->a_rp, &h->a_col, &h->a_val, &h->b_rp, &h->b_col, &h->b_val,
                           &h->ws, &h->c_rp, &h->c_col, &h->c_val, &h->p_rp[0], &h->p_rp[1],
                           &h->p_col[0], &h->p_col[1], &h->p_val[0], &h->p_val[1]};
    size_t n = 0;
    for (const DevBuf* b : all) n += b->bytes;
    return n;
}

// b holds at least `bytes` afterwards.  SPG_ERR_OOM when the handle's buffers
// would exceed spg_tuning.host_alloc_limit (checked before anything is freed
// or allocated) or when cudaMalloc runs out of memory.
static spg_status ensure(spg_handle* h, DevBuf& b, size_t bytes, const char* what) {
    if (bytes <= b.bytes && b.p) return SPG_OK;
    const size_t n = bytes ? bytes : 16;
    const int64_t lim = h->user.host_alloc_limit;
    if (lim > 0 && held_bytes(h) - b.bytes + n > (size_t)lim)
        return fail(h, SPG_ERR_OOM, "%s: %zu more bytes would exceed host_alloc_limit (%lld)",
                    what, n, (long long)lim);
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    const cudaError_t e = cudaMalloc(&b.p, n);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(h, SPG_ERR_OOM, "%s: cudaMalloc of %zu bytes: out of device memory", what, n);
    }
    if (e != cudaSuccess) return cuda_fail(h, e, what);
    b.bytes = n;
    return SPG_OK;
}

static spg_status upload(spg_handle* h, DevBuf& b, const void* src, size_t bytes,
                         cudaStream_t st, const char* what) {
    spg_status s = ensure(h, b, bytes, what);
    if (s != SPG_OK) return s;
    if (bytes) {
        const cudaError_t e = cudaMemcpyAsync(b.p, src, bytes, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "upload");
    }
    return SPG_OK;
}

spg_status spgemm_host_symbolic(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                const spg_csr* B, int64_t* c_row_ptr, int64_t* c_nnz) {
    spg_status s = check_pair(h, sr, A, B, false);
    if (s != SPG_OK) return s;
    if (!c_row_ptr || !c_nnz) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr / c_nnz is NULL");
    cudaError_t e = cudaSuccess;
    if (!h->hstream) e = cudaStreamCreateWithFlags(&h->hstream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(h, e, "stream");
    cudaStream_t st = h->hstream;
    const int vb = in_bytes(sr);
    const bool same = A->row_ptr == B->row_ptr && A->col == B->col && A->val == B->val &&
                      A->nrows == B->nrows && A->nnz == B->nnz;
    s = upload(h, h->a_rp, A->row_ptr, sizeof(int64_t) * (size_t)(A->nrows + 1), st, "A.row_ptr");
    if (s == SPG_OK) s = upload(h, h->a_col, A->col, sizeof(int32_t) * (size_t)A->nnz, st, "A.col");
    if (s == SPG_OK && vb) s = upload(h, h->a_val, A->val, (size_t)vb * (size_t)A->nnz, st, "A.val");
    if (!same) {
        if (s == SPG_OK)
            s = upload(h, h->b_rp, B->row_ptr, sizeof(int64_t) * (size_t)(B->nrows + 1), st, "B.row_ptr");
        if (s == SPG_OK) s = upload(h, h->b_col, B->col, sizeof(int32_t) * (size_t)B->nnz, st, "B.col");
        if (s == SPG_OK && vb) s = upload(h, h->b_val, B->val, (size_t)vb * (size_t)B->nnz, st, "B.val");
    }
    if (s != SPG_OK) return s;
    h->hA = spg_csr{A->nrows, A->ncols, A->nnz, (const int64_t*)h->a_rp.p,
                    (const int32_t*)h->a_col.p, vb ? h->a_val.p : nullptr};
    h->hB = same ? h->hA
                 : spg_csr{B->nrows, B->ncols, B->nnz, (const int64_t*)h->b_rp.p,
                           (const int32_t*)h->b_col.p, vb ? h->b_val.p : nullptr};
    size_t wsb = 0;
    s = spgemm_workspace_size(h, sr, &h->hA, &h->hB, &wsb);
    if (s != SPG_OK) return s;
    s = ensure(h, h->ws, wsb, "workspace");
    if (s == SPG_OK) s = ensure(h, h->c_rp, sizeof(int64_t) * (size_t)(A->nrows + 1), "C.row_ptr");
    if (s != SPG_OK) return s;
    s = spgemm_symbolic(h, sr, &h->hA, &h->hB, (int64_t*)h->c_rp.p, c_nnz, h->ws.p, h->ws.bytes, st);
    if (s != SPG_OK) return s;
    e = cudaMemcpyAsync(c_row_ptr, h->c_rp.p, sizeof(int64_t) * (size_t)(A->nrows + 1),
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "row_ptr download");
    h->host_sr = sr;
    h->host_nnz = *c_nnz;
    h->host_arp.assign(A->row_ptr, A->row_ptr + A->nrows + 1);
    h->host_crp.assign(c_row_ptr, c_row_ptr + A->nrows + 1);
    return SPG_OK;
}

// Default panel size of the host API's pipelined download (spg_tuning.host_panel_bytes).
static constexpr size_t kPipePanelBytes = (size_t)1 << 30;

static size_t host_panel_bytes(const spg_handle* h) {
    return h->user.host_panel_bytes > 0 ? (size_t)h->user.host_panel_bytes : kPipePanelBytes;
}

// Row panels [cuts[k], cuts[k+1]) of about equal output size.
static std::vector<int64_t> panel_cuts(const std::vector<int64_t>& crp, int npanels) {
    const int64_t R = (int64_t)crp.size() - 1, nnz = crp[R];
    std::vector<int64_t> cuts{0};
    for (int k = 1; k < npanels; ++k) {
        const int64_t target = nnz * k / npanels;
        int64_t r = std::lower_bound(crp.begin(), crp.end(), target) - crp.begin();
        if (r <= cuts.back()) r = cuts.back() + 1;
        if (r >= R) break;
        cuts.push_back(r);
    }
    cuts.push_back(R);
    return cuts;
}

// spgemm_host_numeric for large outputs: for each row panel of A, symbolic +
// numeric into one of two device buffers on the compute stream, then the
// panel's download on the copy stream while the next panel computes.
static spg_status host_numeric_pipelined(spg_handle* h, int sr, int32_t* c_col, void* c_val) {
    const int ob = out_bytes(sr);
    const int64_t nnz = h->host_nnz, R = h->hA.nrows;
    const size_t out_bytes_total = (size_t)nnz * (size_t)(4 + ob);
    const size_t panel = host_panel_bytes(h);
    int64_t npl = (int64_t)((out_bytes_total + panel - 1) / panel);
    int np = (int)std::max<int64_t>(2, std::min<int64_t>(npl, 64));
    const std::vector<int64_t> cuts = panel_cuts(h->host_crp, np);
    np = (int)cuts.size() - 1;
    int64_t max_rows = 0, max_nnz = 0;
    for (int k = 0; k < np; ++k) {
        max_rows = std::max(max_rows, cuts[k + 1] - cuts[k]);
        max_nnz = std::max(max_nnz, h->host_crp[cuts[k + 1]] - h->host_crp[cuts[k]]);
    }
    cudaError_t e = cudaSuccess;
    if (!h->cstream) e = cudaStreamCreateWithFlags(&h->cstream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !h->pipe_events) {
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) {
            e = cudaEventCreateWithFlags(&h->ev_done[i], cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_copied[i], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) h->pipe_events = true;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "panel streams");
    for (int b = 0; b < 2; ++b) {
        spg_status s = ensure(h, h->p_rp[b], sizeof(int64_t) * (size_t)(max_rows + 1), "panel row_ptr");
        if (s == SPG_OK) s = ensure(h, h->p_col[b], sizeof(int32_t) * (size_t)max_nnz, "panel col");
        if (s == SPG_OK && ob) s = ensure(h, h->p_val[b], (size_t)ob * (size_t)max_nnz, "panel val");
        if (s != SPG_OK) return s;
    }
    cudaStream_t st = h->hstream, cs = h->cstream;
    // no host synchronisation inside the loop: the panels' sizes are known from
    // the symbolic call on the whole of A, and a device-to-host copy on the
    // compute stream would queue behind the panel downloads; error flags
    // accumulate in the workspace and are read once at the end
    WsPtrs w{};
    for (int k = 0; k < np; ++k) {
        const int b = k & 1;
        const int64_t r0 = cuts[k], r1 = cuts[k + 1];
        if (k >= 2) {
            e = cudaStreamWaitEvent(st, h->ev_copied[b], 0);
            if (e != cudaSuccess) return cuda_fail(h, e, "panel wait");
        }
        spg_csr Ap = h->hA;
        Ap.nrows = r1 - r0;
        Ap.row_ptr = h->hA.row_ptr + r0;
        Ap.nnz = h->host_arp[r1] - h->host_arp[r0];
        int64_t* prp = (int64_t*)h->p_rp[b].p;
        spg_status s = symbolic_launch(h, sr, 1, &Ap, &h->hB, &prp, h->ws.p, h->ws.bytes, st,
                                       k == 0, nullptr, &w);
        if (s != SPG_OK) return s;
        int32_t* pcol = (int32_t*)h->p_col[b].p;
        void* pval = ob ? h->p_val[b].p : nullptr;
        const int64_t* cprp = prp;
        s = numeric_impl(h, sr, 1, &Ap, &h->hB, &cprp, &pcol, &pval, h->ws.p, h->ws.bytes, st);
        if (s != SPG_OK) return s;
        e = cudaEventRecord(h->ev_done[b], st);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->ev_done[b], 0);
        const int64_t at = h->host_crp[r0], pn = h->host_crp[r1] - at;
        if (e == cudaSuccess && pn > 0)
            e = cudaMemcpyAsync(c_col + at, pcol, sizeof(int32_t) * (size_t)pn,
                                cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess && ob && pn > 0)
            e = cudaMemcpyAsync((char*)c_val + (size_t)at * ob, pval, (size_t)ob * (size_t)pn,
                                cudaMemcpyDeviceToHost, cs);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_copied[b], cs);
        if (e != cudaSuccess) return cuda_fail(h, e, "panel download");
    }
    e = cudaStreamSynchronize(cs);
    if (e != cudaSuccess) return cuda_fail(h, e, "panel download");
    (void)R;
    return read_status(h, w, st);   // every panel's kernel-detected errors
}

spg_status spgemm_host_numeric(spg_handle* h, spg_semiring sr, int32_t* c_col, void* c_val) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (h->host_sr != (int)sr || h->host_nnz < 0)
        return fail(h, SPG_ERR_INVALID_ARG, "call spgemm_host_symbolic with this semiring first");
    const int64_t nnz = h->host_nnz;
    const int ob = out_bytes(sr);
    if (nnz > 0 && (!c_col || (ob && !c_val)))
        return fail(h, SPG_ERR_INVALID_ARG, "c_col / c_val is NULL");
    if ((size_t)nnz * (size_t)(4 + ob) > host_panel_bytes(h) &&
        (int64_t)h->host_crp.size() == h->hA.nrows + 1 && h->hA.nrows >= 2)
        return host_numeric_pipelined(h, sr, c_col, c_val);
    cudaStream_t st = h->hstream;
    spg_status s = ensure(h, h->c_col, sizeof(int32_t) * (size_t)nnz, "C.col");
    if (s == SPG_OK && ob) s = ensure(h, h->c_val, (size_t)ob * (size_t)nnz, "C.val");
    if (s != SPG_OK) return s;
    cudaError_t e = cudaSuccess;
    s = spgemm_numeric(h, sr, &h->hA, &h->hB, (const int64_t*)h->c_rp.p,
                                  (int32_t*)h->c_col.p, ob ? h->c_val.p : nullptr, h->ws.p,
                                  h->ws.bytes, st);
    if (s != SPG_OK) return s;
    if (nnz > 0) {
        e = cudaMemcpyAsync(c_col, h->c_col.p, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && ob)
            e = cudaMemcpyAsync(c_val, h->c_val.p, (size_t)ob * (size_t)nnz, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(h, e, "download");
    }
    return spgemm_check(h, h->ws.p, st);
}

spg_status spgemm_validate_csr(spg_handle* h, const spg_csr* M, void* workspace,
                               size_t workspace_bytes, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    spg_status s = check_csr_arg(h, M, "M", SR_BOOL, false);
    if (s != SPG_OK) return s;
    if (!workspace || workspace_bytes < 64) return fail(h, SPG_ERR_WORKSPACE, "needs 64 bytes");
    cudaStream_t st = (cudaStream_t)stream;
    DevStatus* ds = (DevStatus*)workspace;
    cudaError_t e = cudaMemsetAsync(ds, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess) e = launch_validate(to_dcsr(M), M->nnz, ds, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "validate");
    WsPtrs w{};
    w.status = ds;
    return read_status(h, w, st);
}

}  // extern "C"

// ---- learned output sizing --------------------------------------------------------

struct LearnedLayout {
    size_t feat, z, soff, route, skip, total;
};

static LearnedLayout learned_layout(const WsLayout& L) {
    LearnedLayout M;
    const size_t R = (size_t)L.R;
    size_t o = L.total;
    M.feat = o;  o = align256(o + 16 * R);
    M.z = o;     o = align256(o + 4 * R);
    M.soff = o;  o = align256(o + 8 * (R + 1));
    M.route = o; o = align256(o + R);
    M.skip = o;  o = align256(o + R);
    M.total = o;
    return M;
}

static size_t staging_bytes_for(int sr, int64_t S) {
    if (S <= 0) return 0;
    return align256((size_t)S * 4) + (size_t)S * (size_t)out_bytes(sr);
}

static LearnedWs learned_ptrs(void* ws, const LearnedLayout& M, void* staging, int64_t S) {
    char* b = (char*)ws;
    LearnedWs lw;
    lw.feat = (float*)(b + M.feat);
    lw.z = (float*)(b + M.z);
    lw.soff = (int64_t*)(b + M.soff);
    lw.route = (uint8_t*)(b + M.route);
    lw.skip = (uint8_t*)(b + M.skip);
    lw.scol = (int32_t*)staging;
    lw.sval = staging ? (void*)((char*)staging + align256((size_t)S * 4)) : nullptr;
    lw.entries = S;
    return lw;
}

extern "C" {

spg_status spgemm_learned_workspace_size(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                         const spg_csr* B, size_t* bytes) {
    spg_status s = check_pair(h, sr, A, B, false);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = learned_layout(layout_for(A, B, effective_tuning(h, sr))).total;
    return SPG_OK;
}

spg_status spgemm_learned_plan(spg_handle* h, spg_semiring sr, const spg_csr* A,
                               const spg_csr* B, const spg_learned_opts* opts, void* workspace,
                               size_t workspace_bytes, size_t* staging_bytes, void* stream) {
    spg_status s = check_pair(h, sr, A, B, false);
    if (s != SPG_OK) return s;
    if (!staging_bytes) return fail(h, SPG_ERR_INVALID_ARG, "staging_bytes is NULL");
    const Tuning t = effective_tuning(h, sr);
    const WsLayout L = layout_for(A, B, t);
    const LearnedLayout M = learned_layout(L);
    if (!workspace || workspace_bytes < M.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", M.total);
    const float margin = opts && opts->margin > 0.f ? opts->margin : 1.f;
    const int64_t exact_max = opts && opts->exact_max_ub > 0 ? opts->exact_max_ub : 32;
    const int64_t want = opts && opts->learned_max > 0 ? opts->learned_max : 2048;
    const int64_t block_max = learned_capacity_limit(sr, want, false);
    int64_t warp_max = t.num_warp_max_nnz < block_max ? t.num_warp_max_nnz : block_max;
    warp_max = learned_capacity_limit(sr, warp_max, true);
    const void* model = opts ? opts->model : nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    const WsPtrs w = ws_ptrs(workspace, L);
    const LearnedWs lw = learned_ptrs(workspace, M, nullptr, 0);
#ifdef SPG_CHECKS
    {
        const spg_status cs = checked_pairs(h, 1, A, B, st);
        if (cs != SPG_OK) return cs;
    }
#endif
    h->launches = 0;
    h->timer.n = 0;
    h->lrn_sr = -1;
    cudaError_t e = cudaMemsetAsync(workspace, 0, L.probs, st);   // status + counters
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    ProbTable* tab = new ProbTable;
    int64_t* no_rp = nullptr;
    fill_probs(tab, 1, A, B, &no_rp, nullptr, nullptr);
    e = launch_write_probs(*tab, 1, w, h->dev, st);
    delete tab;
    if (e == cudaSuccess)
        e = launch_row_features(w.probs, 1, L.R, lw.feat, w.ub, w.rows_num, w.ctr, h->dev, st);
    if (e == cudaSuccess && model)   // only the rows whose capacity the prediction sets
        e = launch_mlp_forward(lw.feat, L.R, model, lw.z, w.ub, exact_max, h->dev, st);
    if (e == cudaSuccess)
        e = launch_learned_caps(w, lw, 1, L.R, model ? lw.z : nullptr, margin, exact_max,
                                block_max, h->dev, st);
    int64_t* hs = (int64_t*)h->pinned;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs, lw.soff + L.R, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned plan");
    const int64_t S = hs[0];
    h->lrn_sr = sr;
    h->lrn_entries = S;
    h->lrn_warp_max = warp_max;
    h->lrn_block_max = block_max;
    h->lrn_rows = L.R;
    h->stats.staging_entries = S;
    *staging_bytes = staging_bytes_for(sr, S);
    return SPG_OK;
}

static spg_status learned_check(spg_handle* h, int sr, const spg_csr* A, const void* staging,
                                size_t staging_bytes) {
    if (h->lrn_sr != sr || h->lrn_rows != A->nrows)
        return fail(h, SPG_ERR_INVALID_ARG, "call spgemm_learned_plan first (same semiring and A)");
    const size_t need = staging_bytes_for(sr, h->lrn_entries);
    if (need > 0 && (!staging || staging_bytes < need))
        return fail(h, SPG_ERR_WORKSPACE, "staging needs %zu bytes", need);
    return SPG_OK;
}

spg_status spgemm_learned_symbolic(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                   const spg_csr* B, int64_t* c_row_ptr, int64_t* c_nnz,
                                   void* workspace, size_t workspace_bytes, void* staging,
                                   size_t staging_bytes, void* stream) {
    spg_status s = check_pair(h, sr, A, B, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr || !c_nnz) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr / c_nnz is NULL");
    s = learned_check(h, sr, A, staging, staging_bytes);
    if (s != SPG_OK) return s;
    const Tuning t = effective_tuning(h, sr);
    const WsLayout L = layout_for(A, B, t);
    const LearnedLayout M = learned_layout(L);
    if (!workspace || workspace_bytes < M.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", M.total);
    cudaStream_t st = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(workspace, L);
    const LearnedWs lw = learned_ptrs(workspace, M, staging, h->lrn_entries);
    h->launches = 0;
    h->timer.n = 0;
    cudaError_t e = cudaMemsetAsync(workspace, 0, L.probs, st);
    if (e == cudaSuccess && w.row_slot)
        e = cudaMemsetAsync(w.row_slot, 0xff, sizeof(int32_t) * (size_t)L.R, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "memset");
    ProbTable* tab = new ProbTable;
    WordPack* wp = new WordPack;
    fill_probs(tab, 1, A, B, &c_row_ptr, nullptr, nullptr);
    const bool words = plan_words(1, B, workspace, L, tab, wp);
    e = launch_write_probs(*tab, 1, w, h->dev, st);
    delete tab;
    if (e == cudaSuccess)
        e = launch_learned_direct(sr, w, lw, 1, L.R, h->lrn_warp_max, h->lrn_block_max, h->dev, st);
    w.skip = lw.skip;
    if (e == cudaSuccess) e = launch_analyze(w, 1, L.R, t, h->dev, st);
    if (e == cudaSuccess && words) e = launch_word_pack(*wp, w.ctr, h->dev, st);
    delete wp;
    if (e == cudaSuccess) e = launch_symbolic(w, 1, L.R, t, B->ncols, h->dev, st, words);
    if (e == cudaSuccess) e = launch_scan_rowptr(w, 1, L.R, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned symbolic launch");
    Counters* hc = (Counters*)h->pinned;
    e = cudaMemcpyAsync(hc, w.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned symbolic");
    *c_nnz = hc->nnz[0];
    h->stats.products = (int64_t)hc->products;
    h->stats.nnz_c = hc->nnz[0];
    for (int tier = 0; tier < kSymTiers; ++tier) {
        int64_t n = 0;
        for (int b = 0; b < kSubBins; ++b) n += hc->sym_bin_count[tier * kSubBins + b];
        h->stats.rows_per_tier[tier] = n;
    }
    h->stats.overflow_rows = hc->claim[11];
    h->stats.learned_rows = (int64_t)hc->claim[8] + hc->claim[9] + hc->claim[12] - hc->claim[11];
    h->stats.staging_entries = h->lrn_entries;
    h->stats.learned_nnz = (int64_t)hc->learned_nnz;
    return read_status(h, w, st);
}

spg_status spgemm_learned_numeric(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                  const spg_csr* B, const int64_t* c_row_ptr, int32_t* c_col,
                                  void* c_val, void* workspace, size_t workspace_bytes,
                                  const void* staging, size_t staging_bytes, void* stream) {
    spg_status s = check_pair(h, sr, A, B, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr is NULL");
    s = learned_check(h, sr, A, staging, staging_bytes);
    if (s != SPG_OK) return s;
    const Tuning t = effective_tuning(h, sr);
    const WsLayout L = layout_for(A, B, t);
    const LearnedLayout M = learned_layout(L);
    if (!workspace || workspace_bytes < M.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", M.total);
    cudaStream_t st = (cudaStream_t)stream;
    WsPtrs w = ws_ptrs(workspace, L);
    const LearnedWs lw = learned_ptrs(workspace, M, const_cast<void*>(staging), h->lrn_entries);
    h->launches = 0;
    h->timer.n = 0;
    ProbTable* tab = new ProbTable;
    SlabTables* spt = new SlabTables;
    int64_t* rp = const_cast<int64_t*>(c_row_ptr);
    fill_probs(tab, 1, A, B, &rp, &c_col, &c_val);
    if (w.slab_ptr) slab_tables(1, B, t, w.slab_ptr, tab, spt);
    cudaError_t e = launch_write_probs(*tab, 1, w, h->dev, st);
    if (e == cudaSuccess) e = launch_learned_compact(sr, w, lw, 1, L.R, h->dev, st);
    w.skip = lw.skip;
    if (e == cudaSuccess)
        e = launch_numeric(sr, w, to_dcsr(B), 1, L.R, t, B->ncols, h->dev, st, spt, tab);
    delete spt;
    delete tab;
    w.skip = nullptr;
    if (e == cudaSuccess && h->user.deterministic)
        e = launch_det_values(sr, w, 1, L.R, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "learned numeric launch");
    return SPG_OK;
}

spg_status spgemm_row_features(spg_handle* h, const spg_csr* A, const spg_csr* B, float* feat,
                               int64_t* ub, void* workspace, size_t workspace_bytes,
                               void* stream) {
    spg_status s = check_pair(h, SPG_SR_BOOL_OR_AND, A, B, false);
    if (s != SPG_OK) return s;
    if (!feat && A->nrows > 0) return fail(h, SPG_ERR_INVALID_ARG, "feat is NULL");
    if ((uintptr_t)feat % 16 != 0)
        return fail(h, SPG_ERR_INVALID_ARG, "feat must be 16-byte aligned");
    const WsLayout L = layout_for(A, B, effective_tuning(h, SPG_SR_BOOL_OR_AND));
    if (!workspace || workspace_bytes < L.rows_num + sizeof(int32_t) * (size_t)L.R)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes",
                    L.rows_num + sizeof(int32_t) * (size_t)L.R);
    cudaStream_t st = (cudaStream_t)stream;
    const WsPtrs w = ws_ptrs(workspace, L);
    ProbTable* tab = new ProbTable;
    int64_t* no_rp = nullptr;
    fill_probs(tab, 1, A, B, &no_rp, nullptr, nullptr);
    cudaError_t e = launch_write_probs(*tab, 1, w, h->dev, st);
    delete tab;
    if (e == cudaSuccess)
        e = launch_row_features(w.probs, 1, A->nrows, feat, ub, w.rows_num, w.ctr, h->dev, st);
    if (e != cudaSuccess) return cuda_fail(h, e, "row features");
    return SPG_OK;
}

spg_status spgemm_mlp_forward(spg_handle* h, const float* feat, int64_t n,
                              const void* params_bf16, float* z, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!feat || !params_bf16 || !z)))
        return fail(h, SPG_ERR_INVALID_ARG, "feat / params / z NULL or n < 0");
    cudaError_t e = launch_mlp_forward(feat, n, params_bf16, z, nullptr, 0, h->dev,
                                       (cudaStream_t)stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(h, e, "mlp forward");
}

size_t spgemm_mlp_train_workspace_size(int64_t n) { return mlp_train_ws_bytes(n < 0 ? 0 : n); }

spg_status spgemm_mlp_grad(spg_handle* h, const float* feat, const float* log_target, int64_t n,
                           float tau, const void* params_bf16, float* grad, float* loss,
                           void* workspace, size_t workspace_bytes, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (n < 1 || !feat || !log_target || !params_bf16 || !grad || !loss)
        return fail(h, SPG_ERR_INVALID_ARG, "NULL argument or n < 1");
    if (!(tau > 0.f && tau < 1.f)) return fail(h, SPG_ERR_INVALID_ARG, "tau must be in (0, 1)");
    const size_t need = mlp_train_ws_bytes(n);
    if (!workspace || workspace_bytes < need)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", need);
    cudaError_t e = launch_mlp_grad(feat, log_target, n, tau, params_bf16, grad, loss, workspace,
                                    h->dev, (cudaStream_t)stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(h, e, "mlp grad");
}

spg_status spgemm_mlp_adam(spg_handle* h, float* master, float* m, float* v, const float* grad,
                           void* params_bf16, float lr, int step, void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (!master || !m || !v || !grad || !params_bf16 || step < 1)
        return fail(h, SPG_ERR_INVALID_ARG, "NULL argument or step < 1");
    cudaError_t e = launch_mlp_adam(master, m, v, grad, params_bf16, lr, step, h->dev,
                                    (cudaStream_t)stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(h, e, "mlp adam");
}

spg_status spgemm_mlp_to_bf16(spg_handle* h, const float* master, void* params_bf16,
                              void* stream) {
    if (!h) return SPG_ERR_INVALID_ARG;
    if (!master || !params_bf16) return fail(h, SPG_ERR_INVALID_ARG, "NULL argument");
    cudaError_t e = launch_mlp_to_bf16(master, params_bf16, (cudaStream_t)stream);
    return e == cudaSuccess ? SPG_OK : cuda_fail(h, e, "mlp to bf16");
}

}  // extern "C"

// ---- masked product -------------------------------------------------------------

struct MaskedLayout {
    size_t status, slots, touched, part, total;
};

static MaskedLayout masked_layout(int sr, int64_t nnz_m, int64_t R) {
    MaskedLayout L;
    size_t o = 0;
    L.status = o;  o = align256(o + sizeof(DevStatus));
    L.slots = o;   o = align256(o + masked_slot_bytes(sr) * (size_t)nnz_m);
    L.touched = o; o = align256(o + (size_t)nnz_m);
    L.part = o;    o = align256(o + sizeof(int64_t) * (size_t)(scan_parts_needed(R) + 1));
    L.total = o;
    return L;
}

static spg_status masked_check(spg_handle* h, int sr, const spg_csr* A, const spg_csr* B,
                               const spg_csr* M, bool need_val) {
    spg_status s = check_pair(h, sr, A, B, need_val);
    if (s != SPG_OK) return s;
    s = check_csr_arg(h, M, "M", SPG_SR_BOOL_OR_AND, false);
    if (s != SPG_OK) return s;
    if (M->nrows != A->nrows || M->ncols != B->ncols)
        return fail(h, SPG_ERR_INVALID_ARG, "mask shape %lld x %lld, product %lld x %lld",
                    (long long)M->nrows, (long long)M->ncols, (long long)A->nrows,
                    (long long)B->ncols);
    return SPG_OK;
}

extern "C" {

spg_status spgemm_masked_workspace_size(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                        const spg_csr* B, const spg_csr* M, size_t* bytes) {
    spg_status s = masked_check(h, sr, A, B, M, false);
    if (s != SPG_OK) return s;
    if (!bytes) return fail(h, SPG_ERR_INVALID_ARG, "bytes is NULL");
    *bytes = masked_layout(sr, M->nnz, A->nrows).total;
    return SPG_OK;
}

spg_status spgemm_masked_symbolic(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                  const spg_csr* B, const spg_csr* M, int64_t* c_row_ptr,
                                  int64_t* c_nnz, void* workspace, size_t workspace_bytes,
                                  void* stream) {
    spg_status s = masked_check(h, sr, A, B, M, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr || !c_nnz) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr / c_nnz is NULL");
    const MaskedLayout L = masked_layout(sr, M->nnz, A->nrows);
    if (!workspace || workspace_bytes < L.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", L.total);
    cudaStream_t st = (cudaStream_t)stream;
    char* b = (char*)workspace;
#ifdef SPG_CHECKS
    {
        const spg_csr* mats[3] = {A, B, M};
        const spg_status cs = checked_inputs(h, 3, mats, st);
        if (cs != SPG_OK) return cs;
    }
#endif
    h->launches = 0;
    cudaError_t e = cudaMemsetAsync(b + L.status, 0, sizeof(DevStatus), st);
    if (e == cudaSuccess)
        e = launch_masked_count(sr, to_dcsr(A), to_dcsr(B), to_dcsr(M), M->nnz, b + L.slots,
                                (uint8_t*)(b + L.touched), c_row_ptr, (int64_t*)(b + L.part),
                                h->dev, st);
    int64_t* hs = (int64_t*)h->pinned;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs, c_row_ptr + A->nrows, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(h, e, "masked symbolic");
    *c_nnz = hs[0];
    h->stats.nnz_c = hs[0];
    return SPG_OK;
}

spg_status spgemm_masked_numeric(spg_handle* h, spg_semiring sr, const spg_csr* A,
                                 const spg_csr* B, const spg_csr* M, const int64_t* c_row_ptr,
                                 int32_t* c_col, void* c_val, void* workspace,
                                 size_t workspace_bytes, void* stream) {
    spg_status s = masked_check(h, sr, A, B, M, true);
    if (s != SPG_OK) return s;
    if (!c_row_ptr) return fail(h, SPG_ERR_INVALID_ARG, "c_row_ptr is NULL");
    const MaskedLayout L = masked_layout(sr, M->nnz, A->nrows);
    if (!workspace || workspace_bytes < L.total)
        return fail(h, SPG_ERR_WORKSPACE, "workspace needs %zu bytes", L.total);
    char* b = (char*)workspace;
    h->launches = 0;
    cudaError_t e = launch_masked_write(sr, to_dcsr(M), b + L.slots, (const uint8_t*)(b + L.touched),
                                        c_row_ptr, c_col, c_val, (DevStatus*)(b + L.status),
                                        h->dev, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "masked numeric");
    return SPG_OK;
}

}  // extern "C"
