// Row analysis and binning, symbolic phase, scan into C's row pointers, and
// the CSR validity check.
//
// Symbolic phase: nnz(C_i) = |union over k in cols(A_i) of cols(B_k)| (the
// pattern of the Section 2.1 product), computed per row in one of three
// tiers chosen from ub_i = sum_{k in A_i} nnz(B_k):
//   warp  : one warp per row, key-only hash table in the warp's shared memory
//   block : one CTA per row, key-only hash table in the CTA's shared memory
//   dense : one CTA per row, a bitmap over a slab of columns in shared
//           memory, slab after slab; nnz = popcount.
#include <type_traits>

#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

SPG_DEV int sym_tier(int64_t ub, const Tuning& t) {
    if (ub == 0) return kTierEmpty;
    if (ub <= t.sym_warp_max_ub) return kTierWarp;
    if (ub <= t.sym_block_max_ub) return kTierBlock;
    return kTierDense;
}

// tier-major key; inside a tier rows with more work come first.  Tiny rows
// (ub <= 32) of the warp tier share its last sub-bin, where the warp kernel
// takes them several at a time.
SPG_DEV int bin_key(int tier, int64_t work) {
    if (tier == kTierWarp && work <= kTinyMax) return tier * kSubBins + kSubBins - 1;
    int lg = work > 0 ? 63 - __clzll(work) : 0;
    if (lg > kSubBins - 1) lg = kSubBins - 1;
    return tier * kSubBins + (kSubBins - 1 - lg);
}

SPG_DEV int64_t dev_next_pow2(int64_t x) {
    return x <= 1 ? 1 : (int64_t)1 << (64 - __clzll(x - 1));
}

__global__ void k_write_probs(ProbTable tab, int nprob, Prob* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nprob) dst[i] = tab.p[i];
}

// ub_i, the empty rows' counts, the symbolic bin histogram and P = sum ub:
// pass 1, 32 consecutive rows per warp; rows with more than kRowShort entries
// go to the long list (skipped rows keep the ub they have).
SPG_DEV void analyze_add(int* s_hist, unsigned long long& prod, unsigned long long& dprod,
                         int64_t g, int64_t s, bool skipped, const Tuning& t, int64_t* ub,
                         int64_t* cnt) {
    if (skipped) {
        s = ub[g];
    } else {
        ub[g] = s;
        if (s == 0) cnt[g] = 0;
    }
    const int tier = skipped ? kTierEmpty : sym_tier(s, t);
    atomicAdd(&s_hist[bin_key(tier, s)], 1);
    prod += (unsigned long long)s;
    if (tier == kTierDense) dprod += (unsigned long long)s;
}

SPG_DEV void analyze_flush(int* s_hist, unsigned long long prod, unsigned long long dprod,
                           Counters* ctr) {
    prod = warp_sum(prod);
    dprod = warp_sum(dprod);
    if (lane_id() == 0 && prod) atomicAdd(&ctr->products, prod);
    if (lane_id() == 0 && dprod) atomicAdd(&ctr->dense_products, dprod);
    __syncthreads();
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&ctr->sym_bin_count[b], s_hist[b]);
}

__global__ void __launch_bounds__(256) k_analyze(const Prob* __restrict__ probs, int nprob,
                                                 int64_t R, Tuning t, int64_t* __restrict__ ub,
                                                 int64_t* __restrict__ cnt, Counters* ctr,
                                                 const uint8_t* __restrict__ skip,
                                                 int32_t* long_rows) {
    __shared__ int s_hist[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    const int lane = lane_id();
    unsigned long long prod = 0, dprod = 0;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id()) * 32; g0 < R;
         g0 += nw * 32) {
        const int64_t g = g0 + lane;
        const bool in = g < R;
        const bool skipped = in && skip && skip[g];
        bool is_long = false;
        if (in && !skipped) {
            const RowRange rr = row_range(probs, nprob, g);
            const int64_t na = rr.a1 - rr.a0;
            if (na > kRowShort) {
                is_long = true;
            } else {
                int64_t s, mx;
                lane_row_counts(probs[rr.pi], rr.a0, na, s, mx);
                analyze_add(s_hist, prod, dprod, g, s, false, t, ub, cnt);
            }
        } else if (skipped) {
            analyze_add(s_hist, prod, dprod, g, 0, true, t, ub, cnt);
        }
        append_rows(is_long, g, long_rows, ctr);
    }
    analyze_flush(s_hist, prod, dprod, ctr);
}

// pass 2: a warp per long row
__global__ void __launch_bounds__(256) k_analyze_long(const Prob* __restrict__ probs, int nprob,
                                                      Tuning t, int64_t* __restrict__ ub,
                                                      int64_t* __restrict__ cnt, Counters* ctr,
                                                      const int32_t* __restrict__ long_rows) {
    __shared__ int s_hist[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    unsigned long long prod = 0, dprod = 0;
    const int n = ctr->claim[kClLongRows];
    const int nw = gridDim.x * (blockDim.x >> 5);
    for (int r = blockIdx.x * (blockDim.x >> 5) + warp_id(); r < n; r += nw) {
        const int64_t g = long_rows[r];
        const RowRange rr = row_range(probs, nprob, g);
        int64_t s, mx;
        warp_row_long(probs[rr.pi], rr.a0, rr.a1, s, mx);
        if (lane_id() == 0) analyze_add(s_hist, prod, dprod, g, s, false, t, ub, cnt);
    }
    analyze_flush(s_hist, prod, dprod, ctr);
}

// exclusive scan of the kNumBins bin counts (tiny: one thread)
__global__ void k_bin_offsets(const int32_t* count, int32_t* off, int32_t* cursor) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t s = 0;
        for (int b = 0; b < kNumBins; ++b) {
            off[b] = s;
            cursor[b] = s;
            s += count[b];
        }
        off[kNumBins] = s;
    }
}

// rows[...] = flat rows ordered by bin key; per-block aggregation of the
// global cursor atomics.
template <class KeyFn>
SPG_DEV void scatter_by_key(int64_t R, int32_t* cursor, int32_t* rows, KeyFn key_of) {
    __shared__ int s_cnt[kNumBins];
    __shared__ int s_base[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int key = -1, rank = 0;
    if (g < R) {
        key = key_of(g);
        rank = atomicAdd(&s_cnt[key], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x)
        if (s_cnt[b]) s_base[b] = atomicAdd(&cursor[b], s_cnt[b]);
    __syncthreads();
    if (g < R) rows[s_base[key] + rank] = (int32_t)g;
}

__global__ void __launch_bounds__(1024) k_scatter_sym(int64_t R, Tuning t,
                                                      const int64_t* __restrict__ ub,
                                                      Counters* ctr, int32_t* rows,
                                                      const uint8_t* __restrict__ skip) {
    scatter_by_key(R, ctr->sym_bin_cursor, rows, [&](int64_t g) {
        const int64_t u = ub[g];
        return bin_key((skip && skip[g]) ? kTierEmpty : sym_tier(u, t), u);
    });
}

// ---- symbolic tiers ---------------------------------------------------------------

struct KeyInsertOp {
    int32_t* tab;
    int shift;
    uint32_t mask;
    DevStatus* st;
    int64_t g;
    int mine;
    SPG_DEV void any(int32_t col, char, char, bool valid) {
        if (!valid) return;
        const int r = hash_insert(tab, shift, mask, col);
        if (r > 0) ++mine;
        else if (r < 0) flag_overflow(st, g);
    }
    SPG_DEV void sorted(int32_t col, char a, char b, bool valid) { any(col, a, b, valid); }
};

constexpr int kTinyRows = 4;   // tiny rows in flight per warp

__global__ void __launch_bounds__(kWarpTierWarps * 32)
    k_sym_warp(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
               const Counters* __restrict__ ctr, const int64_t* __restrict__ ub,
               int64_t* __restrict__ cnt, DevStatus* st, int per_warp_slots) {
    extern __shared__ int32_t smem_i32[];
    int32_t* tab = smem_i32 + (size_t)warp_id() * per_warp_slots;
    const int lane = lane_id();
    const int beg = ctr->sym_bin_off[kTierWarp * kSubBins];
    const int tiny = ctr->sym_bin_off[(kTierWarp + 1) * kSubBins - 1];
    const int end = ctr->sym_bin_off[(kTierWarp + 1) * kSubBins];
    const int nwarps = gridDim.x * kWarpTierWarps;
    const int wg = blockIdx.x * kWarpTierWarps + warp_id();
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    for (int r = beg + wg; r < tiny; r += nwarps) {
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t u = ub[g];
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        const int64_t distinct = u < P.B.ncols ? u : P.B.ncols;
        int64_t T = dev_next_pow2(2 * distinct);
        if (T < 32) T = 32;
        if (T > per_warp_slots) {   // cannot happen with consistent tuning
            if (lane == 0) flag_overflow(st, g);
            continue;
        }
        for (int s = lane; s < T; s += 32) tab[s] = kEmptyKey;
        __syncwarp();
        KeyInsertOp op{tab, 32 - log2_exact(T), (uint32_t)(T - 1), st, g, 0};
        for (int64_t p0 = a0; p0 < a1; p0 += 32)
            chunk_products<char, false>(P.A, P.B, p0, a1, 0, single, op);
        const int tot = warp_sum(op.mine);
        if (lane == 0) cnt[g] = tot;
        __syncwarp();
    }
    // tiny rows: products sorted in registers, kTinyRows rows per warp at a time
    for (int r = tiny + wg * kTinyRows; r < end; r += nwarps * kTinyRows) {
        tiny_batch<SrBool, kTinyRows, false, false>(
            probs, nprob, rows, r, end,
            [&](int64_t g, const Prob&, int32_t, char, int, int m, bool ok) {
                if (lane == 0) {
                    if (ok) cnt[g] = m;
                    else flag_overflow(st, g);
                }
            });
    }
}

constexpr int kSymBlockSmallThreads = 256;   // CTA size for rows with ub < 4096

// One launch per class of rows (sub-bins [sub_lo, sub_hi) of the tier, by
// floor(log2 ub_i)), each with the shared memory its largest table needs, so
// that classes of small rows keep many CTAs per SM.
template <int NT>
__global__ void __launch_bounds__(NT)
    k_sym_block(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                Counters* ctr, const int64_t* __restrict__ ub, int64_t* __restrict__ cnt,
                DevStatus* st, int table_slots, int64_t dense_min, uint32_t* bm_cache,
                int32_t* row_slot, int64_t cache_words, int64_t cache_slots, int sub_lo,
                int sub_hi, int claim) {
    extern __shared__ int32_t smem_i32[];
    int32_t* tab = smem_i32;
    __shared__ BatchSmem<char, NT> bs;
    __shared__ int s_row, s_cnt, s_slot;
    const int lane = lane_id();
    const int beg = ctr->sym_bin_off[kTierBlock * kSubBins + sub_lo];
    const int end = ctr->sym_bin_off[kTierBlock * kSubBins + sub_hi];
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = beg + atomicAdd(&ctr->claim[claim], 1);
            s_cnt = 0;
        }
        __syncthreads();
        const int r = s_row;
        if (r >= end) break;
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t u = ub[g];
        const int64_t distinct = u < P.B.ncols ? u : P.B.ncols;
        int64_t T = dev_next_pow2(2 * distinct);
        if (T < 32) T = 32;
        if (T > table_slots) {
            if (threadIdx.x == 0) flag_overflow(st, g);
            __syncthreads();
            continue;
        }
        for (int s = threadIdx.x; s < T; s += blockDim.x) tab[s] = kEmptyKey;
        __syncthreads();
        KeyInsertOp op{tab, 32 - log2_exact(T), (uint32_t)(T - 1), st, g, 0};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        cta_row_products<char, false>(P.A, P.B, a0, a1, 0, single, bs, op);
        const int tot = warp_sum(op.mine);
        if (lane == 0 && tot) atomicAdd(&s_cnt, tot);
        __syncthreads();
        if (threadIdx.x == 0) cnt[g] = s_cnt;
        // a row the numeric phase will take in its dense tier: keep the row's
        // bitmap (from the table's keys) so that the numeric phase does not
        // rebuild it from the products
        const int64_t words = (P.B.ncols + 31) >> 5;
        if (bm_cache && s_cnt > dense_min && words <= cache_words) {
            if (threadIdx.x == 0) {
                const int sl = atomicAdd(&ctr->bm_next, 1);
                s_slot = sl < cache_slots ? sl : -1;
                row_slot[g] = s_slot;
            }
            __syncthreads();
            if (s_slot >= 0) {
                uint32_t* dst = bm_cache + (int64_t)s_slot * cache_words;
                uint4* d4 = reinterpret_cast<uint4*>(dst);
                for (int64_t w = threadIdx.x; w < (words + 3) / 4; w += blockDim.x)
                    d4[w] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
                for (int s = threadIdx.x; s < T; s += blockDim.x) {
                    const int32_t k = tab[s];
                    if (k != kEmptyKey) atomicOr(dst + (k >> 5), 1u << (k & 31));
                }
            }
        }
        __syncthreads();
    }
}

struct BitOrOp {
    uint32_t* bm;
    int32_t lo;
    // a plain atomicOr, whose result nothing waits for: reading the word
    // first to skip bits already set puts a dependent shared-memory round trip
    // on every product, which costs more than the atomics it saves (R-MAT 18
    // symbolic dense tier 8.4 -> 7.5 ms)
    SPG_DEV void any(int32_t col, char, char, bool valid) {
        if (!valid) return;
        const int32_t c = col - lo;
        atomicOr(bm + (c >> 5), 1u << (c & 31));
    }
    SPG_DEV void sorted(int32_t col, char a, char b, bool valid) { any(col, a, b, valid); }
};

// The same on the word-packed B: one entry = the mask of B_k's columns in one
// 32-column word (w relative to the slab's first word lo); the word is ORed
// in whole.
struct BitOrMaskOp {
    uint32_t* bm;
    int32_t lo;
    SPG_DEV void any(int32_t w, uint32_t, uint32_t mask, bool valid) {
        if (!valid) return;
        atomicOr(bm + (w - lo), mask);   // as BitOrOp: no read first
    }
    SPG_DEV void sorted(int32_t w, uint32_t a, uint32_t mask, bool valid) { any(w, a, mask, valid); }
};

// ---- word-packed B ----------------------------------------------------------------

__device__ __forceinline__ bool no_dense_rows(const Counters* ctr) {
    return ctr->sym_bin_off[(kTierDense + 1) * kSubBins] == ctr->sym_bin_off[kTierDense * kSubBins];
}

// pack only when the dense tier's walk visits B's entries many times over
__device__ __forceinline__ bool pack_pays(const Counters* ctr, int64_t min_products) {
    return !no_dense_rows(ctr) && ctr->dense_products >= (unsigned long long)min_products;
}

// distinct words of each row of B (a warp per row, 32 entries at a time):
// wrp[k] = count (scanned into row pointers afterwards)
__global__ void k_bw_count(DCsr B, int64_t* wrp, Counters* ctr, int64_t min_products) {
    if (!pack_pays(ctr, min_products)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->words_ready = 1;
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); k < B.nrows; k += nw) {
        const int64_t rs = ld_i64(B.rp + k), re = ld_i64(B.rp + k + 1);
        int32_t carry = -1;   // word of the previous chunk's last entry
        int64_t n = 0;
        for (int64_t q0 = rs; q0 < re; q0 += 32) {
            const int64_t q = q0 + lane;
            const bool v = q < re;
            const int32_t w = v ? (ld_i32(B.col + q) >> 5) : -1;
            int32_t prev = __shfl_up_sync(kFull, w, 1);
            if (lane == 0) prev = carry;
            n += __popc(__ballot_sync(kFull, v && w != prev));
            const int last = (int)min((int64_t)31, re - 1 - q0);
            carry = __shfl_sync(kFull, w, last);
        }
        if (lane == 0) wrp[k] = n;
    }
}

// the packed rows: word ids and the OR of their columns' bits; a run of equal
// words (columns ascending) gets one entry, continued across 32-entry chunks
__global__ void k_bw_fill(DCsr B, DCsr Bw, const Counters* ctr, int64_t min_products) {
    if (!pack_pays(ctr, min_products)) return;
    const int lane = lane_id();
    int32_t* wcol = const_cast<int32_t*>(Bw.col);
    uint32_t* wmask = reinterpret_cast<uint32_t*>(const_cast<void*>(Bw.val));
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); k < B.nrows; k += nw) {
        const int64_t rs = ld_i64(B.rp + k), re = ld_i64(B.rp + k + 1);
        const int64_t base = ld_i64(Bw.rp + k);
        int32_t cw = -1;       // last word of the previous chunk and its mask so far
        uint32_t cm = 0u;
        int64_t heads = 0;     // entries written for this row so far
        for (int64_t q0 = rs; q0 < re; q0 += 32) {
            const int64_t q = q0 + lane;
            const bool v = q < re;
            const int32_t c = v ? ld_i32(B.col + q) : 0;
            const int32_t w = v ? (c >> 5) : -1 - lane;   // invalid lanes: distinct words
            int32_t prev = __shfl_up_sync(kFull, w, 1);
            if (lane == 0) prev = cw;
            const bool head = v && w != prev;
            const unsigned hm = __ballot_sync(kFull, head);
            // entry of this lane's run: heads so far, counting its own (the
            // first run may continue the previous chunk's last entry)
            const int64_t idx = base + heads + __popc(hm & (0xffffffffu >> (31 - lane))) - 1;
            uint32_t m = v ? (1u << (c & 31)) : 0u;
            if (lane == 0 && v && !head) m |= cm;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t om = __shfl_up_sync(kFull, m, d);
                const int32_t ow = __shfl_up_sync(kFull, w, d);
                if (lane >= d && ow == w) m |= om;
            }
            const int32_t nxt = __shfl_down_sync(kFull, w, 1);
            const bool tail = v && (lane == 31 || nxt != w);
            if (tail) {
                wcol[idx] = w;
                wmask[idx] = m;
            }
            heads += __popc(hm);
            const int last = (int)min((int64_t)31, re - 1 - q0);
            cw = __shfl_sync(kFull, w, last);
            cm = __shfl_sync(kFull, m, last);
            __syncwarp();   // a run continued by the next chunk rewrites its entry after this
        }
    }
}

size_t word_pack_bytes(int64_t nrows, int64_t nnz) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(sizeof(int64_t) * (size_t)(nrows + 1)) + 2 * al(sizeof(int32_t) * (size_t)nnz) +
           al(sizeof(int64_t) * (size_t)scan_parts_needed(nrows + 1));
}

void word_pack_plan(WordPack& wp, void* base) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* b = (char*)base;
    for (int i = 0; i < wp.n; ++i) {
        const DCsr& B = wp.src[i];
        DCsr& D = wp.dst[i];
        D.nrows = B.nrows;
        D.ncols = (B.ncols + 31) / 32;
        D.rp = (const int64_t*)b;
        b += al(sizeof(int64_t) * (size_t)(B.nrows + 1));
        D.col = (const int32_t*)b;
        b += al(sizeof(int32_t) * (size_t)wp.nnz[i]);
        D.val = (const void*)b;
        b += al(sizeof(int32_t) * (size_t)wp.nnz[i]);
        wp.part[i] = (int64_t*)b;
        b += al(sizeof(int64_t) * (size_t)scan_parts_needed(B.nrows + 1));
    }
}

cudaError_t launch_word_pack(const WordPack& wp, Counters* ctr, const DevInfo& dev,
                             cudaStream_t st) {
    int64_t nnz = 0;
    for (int i = 0; i < wp.n; ++i) nnz += wp.nnz[i];
    const int64_t min_products = 4 * nnz;
    for (int i = 0; i < wp.n; ++i) {
        const DCsr& B = wp.src[i];
        if (B.nrows == 0) continue;
        int64_t blocks = (B.nrows + 7) / 8;
        if (blocks > (int64_t)dev.sms * 16) blocks = (int64_t)dev.sms * 16;
        int64_t* wrp = const_cast<int64_t*>(wp.dst[i].rp);
        k_bw_count<<<(unsigned)blocks, 256, 0, st>>>(B, wrp, ctr, min_products);
        cudaError_t e = launch_scan_inplace(wrp, B.nrows, wp.part[i], st);
        if (e != cudaSuccess) return e;
        k_bw_fill<<<(unsigned)blocks, 256, 0, st>>>(B, wp.dst[i], ctr, min_products);
        count_launch(dev, 5);
    }
    return cudaGetLastError();
}

// 3 CTAs of 512 threads per SM (registers capped at 42): the walk is latency-bound,
// more resident warps measured ~12% faster than 2 CTAs at 64 registers, and 6
// windows of 32 products in flight per warp ~5% faster than 4.
// kWords: the walk goes over the word-packed B (Prob::Bw): one entry per
// distinct 32-column word of each B row, its mask ORed into the bitmap; the
// slab bounds, cursors and segment lengths are then in words and packed
// entries.  The walk loads one value per A entry and per B entry; in the
// packed walk B's value is the mask and A's is a placeholder (A's column
// array, which has one element per entry of A and is never empty when a row
// has entries).
constexpr int kSymDenseWin = 6;
template <bool kWords>
__global__ void __launch_bounds__(kBlockThreads, 3)
    k_sym_dense(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                Counters* ctr, int64_t* __restrict__ cnt, int32_t* cursor, int slab_cols,
                uint32_t* bm_cache, int32_t* row_slot, int64_t cache_words, int64_t cache_slots) {
    using In = typename std::conditional<kWords, uint32_t, char>::type;
    using Op = typename std::conditional<kWords, BitOrMaskOp, BitOrOp>::type;
    extern __shared__ uint32_t smem_u32[];
    uint32_t* bm = smem_u32;
    __shared__ BatchSmem<In> bs;
    __shared__ int s_row, s_slot;
    __shared__ unsigned long long s_tot;
    // both walks are launched when the copies may have been built; the one
    // that does not match words_ready leaves every row to the other
    if ((ctr->words_ready != 0) != kWords) return;
    const int lane = lane_id();
    const int beg = ctr->sym_bin_off[kTierDense * kSubBins];
    const int end = ctr->sym_bin_off[(kTierDense + 1) * kSubBins];
    // slab width in the walked matrix's columns (words when packed)
    const int slab_x = kWords ? slab_cols / 32 : slab_cols;
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = beg + atomicAdd(&ctr->claim[1], 1);
            s_tot = 0;
        }
        __syncthreads();
        const int r = s_row;
        if (r >= end) break;
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        DCsr Ax = P.A;
        if constexpr (kWords) Ax.val = P.A.col;
        const DCsr& Bx = kWords ? P.Bw : P.B;
        const int64_t ncols_x = kWords ? (P.B.ncols + 31) / 32 : P.B.ncols;
        const int nslabs = (int)((ncols_x + slab_x - 1) / slab_x);
        for (int s = 0; s < nslabs; ++s) {
            const int32_t lo = (int32_t)((int64_t)s * slab_x);
            const int64_t hi64 = (int64_t)lo + slab_x < ncols_x ? (int64_t)lo + slab_x : ncols_x;
            const int32_t hi = (int32_t)hi64;
            const int words = kWords ? hi - lo : (hi - lo + 31) >> 5;
            for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
            __syncthreads();
            Op op{bm, lo};
            if (nslabs == 1 && a1 - a0 <= 32) {
                // <= 32 entries: every warp holds the entry table and takes an
                // equal share of the products (no batch compaction)
                LaneEntry<In, kWords> le;
                le.load(Ax, Bx, a0 + lane, a0 + lane < a1);
                int64_t b, e;
                le.range(nullptr, 0, 1, 0, 1, b, e);
                warp_table_walk<In, kWords, Op, kSymDenseWin>(Bx, b, e, le.a, op);
                __syncthreads();
            } else {
                const Slab slab{lo, hi, s == 0, s == nslabs - 1, nslabs == 1, cursor, nullptr, 0, s};
                cta_row_products<In, kWords, Op, kBatch, kSymDenseWin>(
                    Ax, Bx, a0, a1, P.nnz_base + (a0 - ld_i64(P.A.rp)), slab, bs, op);
            }
            int mine = 0;
            bool counted = false;   // (CTA-uniform)
            if (nslabs == 1 && cache_slots > 0 && words <= cache_words) {
                // keep the row's bitmap for the numeric phase while cache slots
                // last; the copy counts the row's columns on the way (words past
                // `words` in the last group of four are not the row's)
                if (threadIdx.x == 0) {
                    const int sl = atomicAdd(&ctr->bm_next, 1);
                    s_slot = sl < cache_slots ? sl : -1;
                    row_slot[g] = s_slot;
                }
                __syncthreads();
                if (s_slot >= 0) {
                    uint4* dst = reinterpret_cast<uint4*>(bm_cache + (int64_t)s_slot * cache_words);
                    const uint4* src = reinterpret_cast<const uint4*>(bm);
                    for (int w = threadIdx.x; w < (words + 3) / 4; w += blockDim.x) {
                        const uint4 v = src[w];
                        __stcs(dst + w, v);
                        const int rest = words - 4 * w;   // >= 1
                        mine += __popc(v.x) + (rest > 1 ? __popc(v.y) : 0) +
                                (rest > 2 ? __popc(v.z) : 0) + (rest > 3 ? __popc(v.w) : 0);
                    }
                    counted = true;
                }
            }
            if (!counted)
                for (int w = threadIdx.x; w < words; w += blockDim.x) mine += __popc(bm[w]);
            mine = warp_sum(mine);
            if (lane == 0 && mine) atomicAdd(&s_tot, (unsigned long long)mine);
            __syncthreads();
        }
        if (threadIdx.x == 0) cnt[g] = (int64_t)s_tot;
        __syncthreads();
    }
}

// ---- scan of the flat counts into row pointers ------------------------------------

constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

SPG_DEV int64_t block_excl_scan(int64_t v, int64_t* total) {
    __shared__ int64_t s_w[kScanThreads / 32];
    const int lane = lane_id(), w = warp_id();
    int64_t incl = warp_incl_scan(v);
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
        int64_t x = lane < kScanThreads / 32 ? s_w[lane] : 0;
        int64_t xi = warp_incl_scan(x);
        if (lane < kScanThreads / 32) s_w[lane] = xi - x;
        if (lane == kScanThreads / 32 - 1) *total = xi;
    }
    __syncthreads();
    const int64_t r = s_w[w] + incl - v;
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const int64_t* cnt, int64_t R,
                                                              int64_t* part) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int64_t s = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t g = base + (int64_t)t * kScanThreads + threadIdx.x;
        if (g < R) s += cnt[g];
    }
    __shared__ int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_parts(int64_t* part, int64_t nparts) {
    __shared__ int64_t tot;
    int64_t carry = 0;
    for (int64_t base = 0; base < nparts; base += kScanThreads) {
        const int64_t idx = base + threadIdx.x;
        const int64_t v = idx < nparts ? part[idx] : 0;
        const int64_t ex = block_excl_scan(v, &tot);
        if (idx < nparts) part[idx] = carry + ex;
        carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) part[nparts] = carry;
}

// in-place exclusive scan of cnt[0, R) using per-tile offsets; cnt[R] = total
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(int64_t* cnt, int64_t R,
                                                             const int64_t* part, int64_t nparts) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems];
    int64_t s = 0;
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t g = base + t;
        v[t] = g < R ? cnt[g] : 0;
        s += v[t];
    }
    __shared__ int64_t tot;
    int64_t run = block_excl_scan(s, &tot) + part[blockIdx.x];
    for (int t = 0; t < kScanItems; ++t) {
        const int64_t g = base + t;
        if (g < R) cnt[g] = run;
        run += v[t];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) cnt[R] = part[nparts];
}

__global__ void k_write_rowptr(const Prob* __restrict__ probs, const int64_t* __restrict__ cnt,
                               Counters* ctr) {
    const Prob& P = probs[blockIdx.y];
    const int64_t n = P.A.nrows;
    const int64_t b = cnt[P.row_base];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x)
        P.c_rp[i] = cnt[P.row_base + i] - b;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->nnz[blockIdx.y] = cnt[P.row_base + n] - b;
}

// ---- CSR validity check -----------------------------------------------------------

// Reads only M.rp[0 .. nrows] and the entries a row's bounds allow: a row
// whose bounds are decreasing or outside [rp[0], rp[0] + nnz) is reported
// without reading its columns, so a malformed matrix is never read out of
// bounds.  (M may be a row view: its entries start at rp[0].)
__global__ void k_validate(DCsr M, int64_t nnz, DevStatus* st) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t e0 = M.rp[0];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (e0 < 0 || M.rp[M.nrows] != e0 + nnz) atomicExch(&st->invalid, 1);
    }
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < M.nrows; i += nw) {
        const int64_t a = M.rp[i], b = M.rp[i + 1];
        bool bad = b < a || a < e0 || b > e0 + nnz || e0 < 0;
        if (!bad) {
            for (int64_t q = a + lane; q < b; q += 32) {
                const int32_t c = M.col[q];
                if (c < 0 || c >= M.ncols) bad = true;
                if (q > a && M.col[q - 1] >= c) bad = true;
            }
        }
        bad = __any_sync(kFull, bad);
        if (bad && lane == 0 && atomicExch(&st->invalid, 1) == 0) st->info[1] = i;
    }
}

// C's row pointers handed to a numeric call against the counts of the
// symbolic call that left its workspace: c_rp[0] = 0, non-decreasing,
// c_rp[nrows] = that call's nnz(C) for the product (blockIdx.y).
__global__ void k_check_rowptr(const Prob* __restrict__ probs, const Counters* ctr,
                               DevStatus* st) {
    const Prob& P = probs[blockIdx.y];
    const int64_t n = P.A.nrows;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        if (P.c_rp[0] != 0 || P.c_rp[n] != ctr->nnz[blockIdx.y]) {
            if (atomicExch(&st->invalid, 1) == 0) st->info[1] = P.row_base + n;
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (P.c_rp[i + 1] < P.c_rp[i] && atomicExch(&st->invalid, 1) == 0)
            st->info[1] = P.row_base + i;
    }
}

// ---- launchers -------------------------------------------------------------------

cudaError_t launch_check_rowptr(const WsPtrs& w, int nprob, DevStatus* status, cudaStream_t st) {
    k_check_rowptr<<<dim3(64, nprob), 256, 0, st>>>(w.probs, w.ctr, status);
    return cudaGetLastError();
}

cudaError_t launch_write_probs(const ProbTable& tab, int nprob, const WsPtrs& w,
                               const DevInfo& dev, cudaStream_t st) {
    mark_stage(dev, kStBegin, st);
    k_write_probs<<<1, kMaxProb, 0, st>>>(tab, nprob, w.probs);
    count_launch(dev);
    return cudaGetLastError();
}

cudaError_t launch_analyze(const WsPtrs& w, int nprob, int64_t R, const Tuning& t,
                           const DevInfo& dev, cudaStream_t st) {
    if (R > 0) {
        int64_t blocks = (R + 255) / 256;    // 8 warps x 32 rows
        if (blocks > (int64_t)dev.sms * 16) blocks = (int64_t)dev.sms * 16;
        cudaMemsetAsync(&w.ctr->claim[kClLongRows], 0, sizeof(int32_t), st);
        k_analyze<<<(unsigned)blocks, 256, 0, st>>>(w.probs, nprob, R, t, w.ub, w.cnt, w.ctr,
                                                    w.skip, w.rows_num);
        k_analyze_long<<<(unsigned)(dev.sms * 8), 256, 0, st>>>(w.probs, nprob, t, w.ub, w.cnt,
                                                                 w.ctr, w.rows_num);
        count_launch(dev, 2);
    }
    k_bin_offsets<<<1, 32, 0, st>>>(w.ctr->sym_bin_count, w.ctr->sym_bin_off,
                                    w.ctr->sym_bin_cursor);
    count_launch(dev);
    if (R > 0) {
        k_scatter_sym<<<(unsigned)((R + 1023) / 1024), 1024, 0, st>>>(R, t, w.ub, w.ctr,
                                                                       w.rows_sym, w.skip);
        count_launch(dev);
    }
    mark_stage(dev, kStAnalyze, st);
    return cudaGetLastError();
}

size_t sym_warp_smem_per_warp(const Tuning& t) {
    int64_t T = next_pow2(2 * t.sym_warp_max_ub);
    if (T < 32) T = 32;
    return (size_t)T * sizeof(int32_t);
}

static int occupancy(const void* fn, int threads, size_t smem, const DevInfo& dev) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * dev.sms;
}

template <bool kWords>
static cudaError_t launch_sym_dense(const WsPtrs& w, int nprob, int64_t slab, size_t smem,
                                   const DevInfo& dev, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(k_sym_dense<kWords>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = occupancy((const void*)k_sym_dense<kWords>, kBlockThreads, smem, dev);
    k_sym_dense<kWords><<<grid, kBlockThreads, smem, st>>>(
        w.probs, nprob, w.rows_sym, w.ctr, w.cnt, w.cursor, (int)slab, w.bm_cache, w.row_slot,
        w.bm_cache_words, w.bm_cache_slots);
    count_launch(dev);
    return cudaGetLastError();
}

cudaError_t launch_symbolic(const WsPtrs& w, int nprob, int64_t R, const Tuning& t,
                            int64_t max_ncols, const DevInfo& dev, cudaStream_t st, bool words) {
    if (R == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    // dense tier first: it holds the heaviest rows
    {
        int64_t slab = t.sym_slab_cols;
        if (slab > max_ncols) slab = (max_ncols + 1023) / 1024 * 1024;
        if (slab < 1024) slab = 1024;
        const size_t smem = (size_t)slab / 8;
        if (words) e = launch_sym_dense<true>(w, nprob, slab, smem, dev, st);
        if (e == cudaSuccess) e = launch_sym_dense<false>(w, nprob, slab, smem, dev, st);
        if (e != cudaSuccess) return e;
        mark_stage(dev, kStSymDense, st);
    }
    {
        // classes by floor(log2 ub_i), heaviest first: sub-bins [0, 28) ub >= 4096
        // (tables up to the tier's limit, 512 threads), 28: ub in [2048, 4096)
        // (8192 slots), [29, 40): ub < 2048 (4096 slots); 256 threads for both
        int64_t Tmax = next_pow2(2 * t.sym_block_max_ub);
        if (Tmax < 32) Tmax = 32;
        struct Class { int64_t min_ub, T; int lo, hi, claim; bool wide; };
        const Class classes[3] = {{4096, Tmax, 0, kSubBins - 12, 0, true},
                                  {2048, 8192, kSubBins - 12, kSubBins - 11, 7, false},
                                  {0, 4096, kSubBins - 11, kSubBins, 15, false}};
        e = cudaFuncSetAttribute(k_sym_block<kBlockThreads>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(Tmax * 4));
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_sym_block<kSymBlockSmallThreads>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 4);
        if (e != cudaSuccess) return e;
        for (const Class& c : classes) {
            if (t.sym_block_max_ub < c.min_ub) continue;   // no row of this class
            const int64_t T = c.T < Tmax ? c.T : Tmax;
            const size_t smem = (size_t)T * sizeof(int32_t);
            if (c.wide) {
                const int grid = occupancy((const void*)k_sym_block<kBlockThreads>, kBlockThreads,
                                           smem, dev);
                k_sym_block<kBlockThreads><<<grid, kBlockThreads, smem, st>>>(
                    w.probs, nprob, w.rows_sym, w.ctr, w.ub, w.cnt, w.status, (int)T,
                    t.num_block_max_nnz, w.bm_cache, w.row_slot, w.bm_cache_words,
                    w.bm_cache_slots, c.lo, c.hi, c.claim);
            } else {
                const int grid = occupancy((const void*)k_sym_block<kSymBlockSmallThreads>,
                                           kSymBlockSmallThreads, smem, dev);
                k_sym_block<kSymBlockSmallThreads><<<grid, kSymBlockSmallThreads, smem, st>>>(
                    w.probs, nprob, w.rows_sym, w.ctr, w.ub, w.cnt, w.status, (int)T,
                    t.num_block_max_nnz, w.bm_cache, w.row_slot, w.bm_cache_words,
                    w.bm_cache_slots, c.lo, c.hi, c.claim);
            }
            count_launch(dev);
        }
        mark_stage(dev, kStSymBlock, st);
    }
    {
        const size_t per_warp = sym_warp_smem_per_warp(t);
        const size_t smem = per_warp * kWarpTierWarps;
        e = cudaFuncSetAttribute(k_sym_warp, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        const int grid = occupancy((const void*)k_sym_warp, kWarpTierWarps * 32, smem, dev);
        k_sym_warp<<<grid, kWarpTierWarps * 32, smem, st>>>(
            w.probs, nprob, w.rows_sym, w.ctr, w.ub, w.cnt, w.status,
            (int)(per_warp / sizeof(int32_t)));
        count_launch(dev);
        mark_stage(dev, kStSymWarp, st);
    }
    return cudaGetLastError();
}

int64_t scan_parts_needed(int64_t R) { return (R + kScanTile - 1) / kScanTile + 1; }

cudaError_t launch_scan_inplace(int64_t* cnt, int64_t R, int64_t* part, cudaStream_t st) {
    const int64_t nparts = (R + kScanTile - 1) / kScanTile;
    if (R > 0) {
        k_scan_reduce<<<(unsigned)nparts, kScanThreads, 0, st>>>(cnt, R, part);
        k_scan_parts<<<1, kScanThreads, 0, st>>>(part, nparts);
        k_scan_apply<<<(unsigned)nparts, kScanThreads, 0, st>>>(cnt, R, part, nparts);
    } else {
        cudaMemsetAsync(cnt, 0, sizeof(int64_t), st);
    }
    return cudaGetLastError();
}

cudaError_t launch_scan_rowptr(const WsPtrs& w, int nprob, int64_t R, const DevInfo& dev,
                               cudaStream_t st) {
    cudaError_t e = launch_scan_inplace(w.cnt, R, w.scan_part, st);
    if (e != cudaSuccess) return e;
    count_launch(dev, R > 0 ? 3 : 0);
    k_write_rowptr<<<dim3(64, nprob), 256, 0, st>>>(w.probs, w.cnt, w.ctr);
    count_launch(dev);
    mark_stage(dev, kStScan, st);
    return cudaGetLastError();
}

cudaError_t launch_validate(const DCsr& M, int64_t nnz, DevStatus* status, cudaStream_t st) {
    int64_t blocks = (M.nrows + 7) / 8;
    if (blocks < 1) blocks = 1;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_validate<<<(unsigned)blocks, 256, 0, st>>>(M, nnz, status);
    return cudaGetLastError();
}

}  // namespace spg
