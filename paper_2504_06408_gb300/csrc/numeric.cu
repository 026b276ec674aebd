// Numeric phase: accumulation of every product with the semiring, and the
// sorted, compacted write of each output row (Section 2.1 definition, Section
// 2.2 semirings).  Rows are binned by their exact nnz(C_i) (from the
// symbolic phase) into three tiers:
//   warp  : one warp per row; hash table of (column, accumulator) in the
//           warp's shared memory; occupied keys compacted and sorted by a
//           register (<= 32 keys) or shared-memory bitonic sort; each sorted
//           key looks its accumulator up again and the warp writes the row.
//   block : the same with one CTA per row.
//   dense : one CTA per row; a dense accumulator array over a slab of
//           columns in shared memory, slab after slab.  Output comes out of
//           a bitmap scan, already sorted: no sort.
#include <type_traits>

#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

SPG_DEV int64_t dev_next_pow2_n(int64_t x) {
    return x <= 1 ? 1 : (int64_t)1 << (64 - __clzll(x - 1));
}

// block_max: the block tier's limit in effect (the tuning's, or the compact
// overlap tier's when the positions allow it, set on the device)
// Dense rows with fewer than t.rank_light_ub products whose outputs fit one
// value pass of a half-SM CTA (nnz <= light_n, set on the device) are light:
// their own tier, taken by the 512-thread rank kernel.
SPG_DEV int num_tier(int64_t nnz, int64_t ub, const Tuning& t, int64_t block_max,
                     int64_t light_n) {
    if (nnz == 0) return kTierEmpty;
    if (nnz <= t.num_warp_max_nnz) return kTierWarp;
    if (nnz <= block_max) return kTierBlock;
    if (nnz <= light_n && ub < t.rank_light_ub) return kTierDenseLight;
    return kTierDense;
}

SPG_DEV int64_t block_limit(const Tuning& t, const Counters* ctr) {
    return ctr->num_block_max > 0 ? ctr->num_block_max : t.num_block_max_nnz;
}

// Overlap semiring: positions of A and B all in [0, 2^16)?  Clears
// ctr->num_block_max (block 0) and raises ctr->ovl_wide on a position outside.
__global__ void k_ovl_check(DCsr M, Counters* ctr) {
    const int64_t e0 = M.rp[0], e1 = M.rp[M.nrows];
    const int32_t* v = reinterpret_cast<const int32_t*>(M.val);
    bool wide = false;
    for (int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e1;
         e += (int64_t)gridDim.x * blockDim.x)
        wide |= (uint32_t)ld_i32(v + e) > 0xffffu;
    if (__any_sync(kFull, wide) && lane_id() == 0) atomicExch(&ctr->ovl_wide, 1);
}

// block-tier limit of the compact overlap tier when every position fits 16 bits
__global__ void k_ovl_limit(Counters* ctr, int64_t compact_max) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ctr->num_block_max = ctr->ovl_wide ? 0 : compact_max;
}

// as the symbolic bins: tiny rows (ub <= 32) of the warp tier in its last sub-bin
SPG_DEV int num_bin_key(int tier, int64_t work) {
    if (tier == kTierWarp && work <= kTinyMax) return tier * kSubBins + kSubBins - 1;
    int lg = work > 0 ? 63 - __clzll(work) : 0;
    if (lg > kSubBins - 1) lg = kSubBins - 1;
    return tier * kSubBins + (kSubBins - 1 - lg);
}

SPG_DEV int64_t row_nnz(const Prob* probs, int nprob, int64_t g, const Prob** pp) {
    const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
    *pp = &P;
    const int64_t i = g - P.row_base;
    return P.c_rp[i + 1] - P.c_rp[i];
}

__global__ void __launch_bounds__(256) k_num_hist(const Prob* __restrict__ probs, int nprob,
                                                  int64_t R, Tuning t,
                                                  const int64_t* __restrict__ ub, Counters* ctr,
                                                  const uint8_t* __restrict__ skip) {
    __shared__ int s_hist[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x) {
        const Prob* P;
        const int64_t n = row_nnz(probs, nprob, g, &P);
        const int64_t u = ub[g];
        const int tier = (skip && skip[g]) ? kTierEmpty
                                           : num_tier(n, u, t, block_limit(t, ctr), ctr->light_n);
        atomicAdd(&s_hist[num_bin_key(tier, u)], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x)
        if (s_hist[b]) atomicAdd(&ctr->num_bin_count[b], s_hist[b]);
}

__global__ void k_num_bin_offsets(Counters* ctr) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int32_t s = 0;
        for (int b = 0; b < kNumBins; ++b) {
            ctr->num_bin_off[b] = s;
            ctr->num_bin_cursor[b] = s;
            s += ctr->num_bin_count[b];
        }
        ctr->num_bin_off[kNumBins] = s;
    }
}

__global__ void __launch_bounds__(1024) k_num_scatter(const Prob* __restrict__ probs, int nprob,
                                                      int64_t R, Tuning t,
                                                      const int64_t* __restrict__ ub,
                                                      Counters* ctr, int32_t* rows,
                                                      const uint8_t* __restrict__ skip) {
    __shared__ int s_cnt[kNumBins];
    __shared__ int s_base[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int key = -1, rank = 0;
    if (g < R) {
        const Prob* P;
        const int64_t n = row_nnz(probs, nprob, g, &P);
        const int64_t u = ub[g];
        key = num_bin_key((skip && skip[g]) ? kTierEmpty
                                            : num_tier(n, u, t, block_limit(t, ctr), ctr->light_n),
                          u);
        rank = atomicAdd(&s_cnt[key], 1);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x)
        if (s_cnt[b]) s_base[b] = atomicAdd(&ctr->num_bin_cursor[b], s_cnt[b]);
    __syncthreads();
    if (g < R) rows[s_base[key] + rank] = (int32_t)g;
}

// ---- accumulation ops ----------------------------------------------------------

template <class S>
struct HashAccOp {
    int32_t* keys;
    typename S::Slot* vals;
    int shift;
    uint32_t mask;
    DevStatus* st;
    int64_t g;
    SPG_DEV void any(int32_t col, typename S::In a, typename S::In b, bool valid) {
        if (!valid) return;
        const int s = hash_slot_of(keys, shift, mask, col);
        if (s < 0) {
            flag_overflow(st, g);
            return;
        }
        if constexpr (S::kVal) S::acc(vals + s, a, b);
    }
    SPG_DEV void sorted(int32_t col, typename S::In a, typename S::In b, bool valid) {
        any(col, a, b, valid);
    }
};

// Dense slab accumulator.  The presence bitmap is kept for every semiring:
// semirings whose Slot cannot mark presence set the bit on every product
// (a plain atomicOr: no read of the word first); the others set it only on a
// column's first product, which their Slot reveals.
template <class S>
struct DenseAccOp {
    typename S::Slot* vals;
    uint32_t* bm;
    int32_t lo;
    SPG_DEV void any(int32_t col, typename S::In a, typename S::In b, bool valid) {
        if (!valid) return;
        const int32_t c = col - lo;
        const uint32_t bit = 1u << (c & 31);
        if constexpr (S::kBitmap) {
            atomicOr(bm + (c >> 5), bit);
            if constexpr (S::kVal) S::acc(vals + c, a, b);
        } else {
            if (S::acc_first(vals + c, a, b)) atomicOr(bm + (c >> 5), bit);
        }
    }
    SPG_DEV void sorted(int32_t col, typename S::In a, typename S::In b, bool valid) {
        any(col, a, b, valid);
    }
};

template <class S>
SPG_DEV void write_entry(const Prob& P, int64_t pos, int32_t col, const typename S::Slot& v) {
    st_stream(P.c_col + pos, col);
    if constexpr (S::kVal) st_stream(reinterpret_cast<typename S::Out*>(P.c_val) + pos, S::out(v));
}

template <class S>
SPG_DEV size_t hash_region_bytes(int T) {
    // vals[T] | keys[T] | sort buffer[T/2], 16-byte aligned
    size_t b = (size_t)T * sizeof(typename S::Slot) + (size_t)T * 4 + (size_t)(T / 2) * 4;
    return (b + 15) & ~(size_t)15;
}

// ---- warp tier ------------------------------------------------------------------

constexpr int kTinyRows = 1;   // tiny rows per warp at a time (more costs registers)

template <class S>
__global__ void __launch_bounds__(kWarpTierWarps * 32)
    k_num_warp(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
               const Counters* __restrict__ ctr, const int64_t* __restrict__ ub, DevStatus* st,
               int Tw) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + hash_region_bytes<S>(Tw) * warp_id();
    Slot* vals = reinterpret_cast<Slot*>(base);
    int32_t* keys = reinterpret_cast<int32_t*>(base + (size_t)Tw * sizeof(Slot));
    int32_t* sbuf = keys + Tw;
    const int lane = lane_id();
    const int beg = ctr->num_bin_off[kTierWarp * kSubBins];
    const int tiny = ctr->num_bin_off[(kTierWarp + 1) * kSubBins - 1];
    const int end = ctr->num_bin_off[(kTierWarp + 1) * kSubBins];
    const int stride = gridDim.x * kWarpTierWarps;
    const int wg = blockIdx.x * kWarpTierWarps + warp_id();
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    // tiny rows: products sorted and folded in registers, kTinyRows at a time
    for (int r = tiny + wg * kTinyRows; r < end; r += stride * kTinyRows) {
        tiny_batch<S, kTinyRows, S::kVal, true>(
            probs, nprob, rows, r, end,
            [&](int64_t g, const Prob& P, int32_t col, const typename S::Out& val, int rank, int m,
                bool ok) {
                const int64_t i = g - P.row_base;
                const int64_t off = P.c_rp[i];
                if (!ok || m != P.c_rp[i + 1] - off) {   // inconsistent with the symbolic phase
                    if (lane == 0) flag_overflow(st, g);
                    return;
                }
                if (rank >= 0) {
                    P.c_col[off + rank] = col;
                    if constexpr (S::kVal)
                        reinterpret_cast<typename S::Out*>(P.c_val)[off + rank] = val;
                }
            });
    }
    for (int r = beg + wg; r < tiny; r += stride) {
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t off = P.c_rp[i];
        const int n = (int)(P.c_rp[i + 1] - off);
        int T = (int)dev_next_pow2_n(2 * (int64_t)n);
        if (T < 32) T = 32;
        if (T > Tw) {
            if (lane == 0) flag_overflow(st, g);
            continue;
        }
        for (int s = lane; s < T; s += 32) {
            keys[s] = kEmptyKey;
            vals[s] = S::empty();
        }
        __syncwarp();
        const int shift = 32 - log2_exact(T);
        HashAccOp<S> op{keys, vals, shift, (uint32_t)(T - 1), st, g};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        for (int64_t p0 = a0; p0 < a1; p0 += 32)
            chunk_products<In, S::kVal>(P.A, P.B, p0, a1, 0, single, op);
        __syncwarp();
        // compact occupied keys
        int m = 0;
        for (int s0 = 0; s0 < T; s0 += 32) {
            const int32_t k = keys[s0 + lane];
            const unsigned occ = __ballot_sync(kFull, k != kEmptyKey);
            const int pos = m + __popc(occ & ((1u << lane) - 1));
            if (k != kEmptyKey && pos < T / 2) sbuf[pos] = k;
            m += __popc(occ);
        }
        if (m != n) {   // symbolic and numeric disagree: inconsistent inputs
            if (lane == 0) flag_overflow(st, g);
            continue;
        }
        __syncwarp();
        if (n <= 32) {
            int32_t v = lane < n ? sbuf[lane] : INT32_MAX;
            v = warp_bitonic_sort32(v);
            if (lane < n) {
                const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
                write_entry<S>(P, off + lane, v, vals[s < 0 ? 0 : s]);
            }
        } else {
            const int N = (int)dev_next_pow2_n(n);
            for (int t = n + lane; t < N; t += 32) sbuf[t] = INT32_MAX;
            __syncwarp();
            smem_bitonic_sort(sbuf, N, lane, 32, [] { __syncwarp(); });
            for (int t = lane; t < n; t += 32) {
                const int32_t v = sbuf[t];
                const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
                write_entry<S>(P, off + t, v, vals[s < 0 ? 0 : s]);
            }
        }
        __syncwarp();
    }
}

// ---- block tier -----------------------------------------------------------------

template <class S>
__global__ void __launch_bounds__(kBlockThreads)
    k_num_block(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                Counters* ctr, DevStatus* st, int Tb, int only_wide) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    // compact overlap slots: tables up to 3/4 full and a sort buffer of a
    // whole table (the rows are twice as long for the same memory)
    constexpr bool kC = std::is_same<S, SrOverlapC>::value;
    // the compact kernel runs when every position fits 16 bits, the 24-byte
    // one launched beside it (only_wide) when one does not
    if (kC && ctr->ovl_wide) return;
    if (only_wide && !ctr->ovl_wide) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw + (size_t)Tb * sizeof(Slot));
    int32_t* sbuf = keys + Tb;   // [Tb / 2], or [Tb] with compact slots
    __shared__ BatchSmem<In> bs;
    __shared__ int s_row, s_m;
    const int lane = lane_id();
    const int beg = ctr->num_bin_off[kTierBlock * kSubBins];
    const int end = ctr->num_bin_off[(kTierBlock + 1) * kSubBins];
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = beg + atomicAdd(&ctr->claim[2], 1);
            s_m = 0;
        }
        __syncthreads();
        const int r = s_row;
        if (r >= end) break;
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t off = P.c_rp[i];
        const int n = (int)(P.c_rp[i + 1] - off);
        int T = (int)dev_next_pow2_n(kC ? (4 * (int64_t)n + 2) / 3 : 2 * (int64_t)n);
        if (T < 32) T = 32;
        if (T > Tb) {
            if (threadIdx.x == 0) flag_overflow(st, g);
            __syncthreads();
            continue;
        }
        for (int s = threadIdx.x; s < T; s += blockDim.x) {
            keys[s] = kEmptyKey;
            vals[s] = S::empty();
        }
        __syncthreads();
        const int shift = 32 - log2_exact(T);
        HashAccOp<S> op{keys, vals, shift, (uint32_t)(T - 1), st, g};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        cta_row_products<In, S::kVal>(P.A, P.B, a0, a1, 0, single, bs, op);
        // compact occupied keys (order irrelevant: sorted next)
        for (int s0 = warp_id() * 32; s0 < T; s0 += blockDim.x) {
            const int32_t k = keys[s0 + lane];
            const unsigned occ = __ballot_sync(kFull, k != kEmptyKey);
            int b = 0;
            if (lane == 0 && occ) b = atomicAdd(&s_m, __popc(occ));
            b = __shfl_sync(kFull, b, 0);
            const int pos = b + __popc(occ & ((1u << lane) - 1));
            if (k != kEmptyKey && pos < (kC ? T : T / 2)) sbuf[pos] = k;
        }
        __syncthreads();
        const int m = s_m;
        if (m != n) {
            if (threadIdx.x == 0) flag_overflow(st, g);
            __syncthreads();
            continue;
        }
        const int N = (int)dev_next_pow2_n(n);
        for (int t = n + threadIdx.x; t < N; t += blockDim.x) sbuf[t] = INT32_MAX;
        __syncthreads();
        smem_bitonic_sort(sbuf, N, threadIdx.x, blockDim.x, [] { __syncthreads(); });
        for (int t = threadIdx.x; t < n; t += blockDim.x) {
            const int32_t v = sbuf[t];
            const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
            write_entry<S>(P, off + t, v, vals[s < 0 ? 0 : s]);
        }
        __syncthreads();
    }
}

// ---- dense tier -----------------------------------------------------------------

// vals[0, width) = S::empty(), 16-byte stores where the slot size allows
template <class S>
SPG_DEV void fill_slots(typename S::Slot* vals, int width) {
    using Slot = typename S::Slot;
    if constexpr (sizeof(Slot) == 4 || sizeof(Slot) == 8) {
        constexpr int per = 16 / (int)sizeof(Slot);
        alignas(16) Slot e[per];
#pragma unroll
        for (int u = 0; u < per; ++u) e[u] = S::empty();
        uint4 v;
        memcpy(&v, e, sizeof v);
        uint4* v4 = reinterpret_cast<uint4*>(vals);
        const int n4 = width / per;
        for (int c = threadIdx.x; c < n4; c += blockDim.x) v4[c] = v;
        for (int c = n4 * per + threadIdx.x; c < width; c += blockDim.x) vals[c] = S::empty();
    } else {
        for (int c = threadIdx.x; c < width; c += blockDim.x) vals[c] = S::empty();
    }
}

template <class S>
__host__ __device__ inline size_t dense_val_bytes(int64_t slab_cols) {
    return S::kVal ? (size_t)slab_cols * sizeof(typename S::Slot) : 0;
}

// Segment tables of one group of up to 16 slabs for a row with at most 32 A
// entries: warp w fills slab (group * 16 + w); lane e = entry e.
template <class In>
struct SmallRowSmem {
    int64_t beg[16][32];   // segment start of entry e in the slab
    int32_t end[16][32];   // inclusive prefix of segment lengths (products of entries <= e)
    In a[32];
};

// Products of one slab of a row with <= 32 entries, split evenly over the
// warps.  Lane e keeps entry e's segment start and prefix end; a 32-product
// window inside one segment is addressed directly, a window that crosses
// segment ends finds each lane's entry by a 5-step search over the prefixes.
template <class S, class Op>
SPG_DEV void small_row_slab_products(const DCsr& B, const SmallRowSmem<typename S::In>& sr,
                                     int sl, Op& op) {
    using In = typename S::In;
    const int lane = lane_id(), wid = warp_id();
    const int nwarps = blockDim.x >> 5;
    const int64_t my_beg = sr.beg[sl][lane];
    const int my_end = sr.end[sl][lane];
    In my_a = In();
    if constexpr (S::kVal) my_a = sr.a[lane];
    const int total = __shfl_sync(kFull, my_end, 31);
    const int lo_w = (int)((int64_t)total * wid / nwarps);
    const int hi_w = (int)((int64_t)total * (wid + 1) / nwarps);
    const int up = __shfl_up_sync(kFull, my_end, 1);
    const int excl = lane ? up : 0;   // products of entries < lane
    for (int t0 = lo_w; t0 < hi_w; t0 += 128) {   // warp-uniform
        int64_t qv[4];
        In av[4];
        bool vv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int t = t0 + 32 * u + lane;
            vv[u] = t < hi_w;
            int k = 0;   // entry of product t: number of prefix ends <= t
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int bv = __shfl_sync(kFull, my_end, k + step - 1);
                if (bv <= t) k += step;
            }
            const int64_t b = __shfl_sync(kFull, my_beg, k);
            const int ex = __shfl_sync(kFull, excl, k);
            qv[u] = b + (t - ex);
            if constexpr (S::kVal) av[u] = __shfl_sync(kFull, my_a, k);
            else av[u] = In();
        }
        int32_t col[4];
        In bval[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            col[u] = vv[u] ? ld_i32(B.col + qv[u]) : 0;
            bval[u] = vv[u] ? load_val<In, S::kVal>(B.val, qv[u]) : In();
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) op.any(col[u], av[u], bval[u], vv[u]);
    }
}

template <class S>
__global__ void __launch_bounds__(kBlockThreads, 2)
    k_num_dense(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                Counters* ctr, DevStatus* st, int32_t* cursor, int slab_cols, int sp_stride) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw + dense_val_bytes<S>(slab_cols));
    int32_t* word_off = reinterpret_cast<int32_t*>(bm + slab_cols / 32);   // [words + 1]
    __shared__ BatchSmem<In> bs;
    __shared__ SmallRowSmem<In> srs;
    __shared__ int s_row;
    __shared__ int s_wsum[kBlockThreads / 32];
    __shared__ int64_t s_written;
    const int lane = lane_id(), wid = warp_id(), nwarps = blockDim.x >> 5;
    const int tid = threadIdx.x;
    const int beg = ctr->num_bin_off[kTierDense * kSubBins];
    const int end = ctr->num_bin_off[(kTierDense + 1) * kSubBins];
    for (;;) {
        if (tid == 0) {
            s_row = beg + atomicAdd(&ctr->claim[3], 1);
            s_written = 0;
        }
        __syncthreads();
        const int r = s_row;
        if (r >= end) break;
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t off = P.c_rp[i];
        const int64_t n = P.c_rp[i + 1] - off;
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        const int64_t ncols = P.B.ncols;
        const int nslabs = (int)((ncols + slab_cols - 1) / slab_cols);
        const int32_t* __restrict__ sp = P.sp;
        // small rows: <= 32 entries, slab table available (or one slab)
        const bool small = a1 - a0 <= 32 && (sp != nullptr || nslabs == 1);
        const bool one_batch = !small && a1 - a0 <= kBatch;
        const Slab first{0, 0, true, nslabs == 1, nslabs == 1, cursor, sp, sp_stride, 0};
        RowEntry<In, S::kVal> ent;
        if (one_batch) ent.load(P.A, P.B, a0 + tid, a0 + tid < a1, first);
        // small-row entry, the same in every warp (lane e = entry e)
        int32_t sk = 0;
        int64_t srs0 = 0, sre0 = 0;
        if (small) {
            const int64_t p = a0 + lane;
            if (p < a1) {
                sk = ld_i32(P.A.col + p);
                srs0 = ld_i64(P.B.rp + sk);
                sre0 = ld_i64(P.B.rp + sk + 1);
                if (wid == 0) {
                    if constexpr (S::kVal) srs.a[lane] = load_val<In, S::kVal>(P.A.val, p);
                }
            } else if (wid == 0) {
                if constexpr (S::kVal) srs.a[lane] = In();
            }
        }
        for (int s = 0; s < nslabs; ++s) {
            if (small && (s & 15) == 0) {
                // warp w tabulates slab s + w of this group
                const int ss = s + wid;
                if (ss < nslabs) {
                    int64_t b = srs0, e = sre0;
                    if (nslabs > 1 && a0 + lane < a1) {
                        const int32_t* spk = sp + (int64_t)sk * sp_stride;
                        b = srs0 + __ldg(spk + ss);
                        e = srs0 + __ldg(spk + ss + 1);
                    }
                    const int len = (int)(e - b);
                    srs.beg[wid][lane] = b;
                    srs.end[wid][lane] = warp_incl_scan(len);
                }
            }
            const int32_t lo = (int32_t)((int64_t)s * slab_cols);
            const int64_t hi64 = (int64_t)lo + slab_cols < ncols ? (int64_t)lo + slab_cols : ncols;
            const int32_t hi = (int32_t)hi64;
            const int width = hi - lo;
            const int words = (width + 31) >> 5;
            if constexpr (S::kVal) fill_slots<S>(vals, width);
            for (int w = tid; w < words; w += blockDim.x) bm[w] = 0u;
            __syncthreads();
            const Slab slab{lo, hi, s == 0, s == nslabs - 1, nslabs == 1, cursor, sp, sp_stride, s};
            DenseAccOp<S> op{vals, bm, lo};
            if (small) {
                small_row_slab_products<S>(P.B, srs, s & 15, op);
                __syncthreads();
            } else if (one_batch) {
                int64_t sb, se;
                ent.segment(P.B, slab, nslabs, sb, se);
                cta_walk_segments<In, S::kVal>(P.B, sb, se - sb, ent.a, bs, op);
            } else {
                cta_row_products<In, S::kVal>(P.A, P.B, a0, a1, P.nnz_base + (a0 - ld_i64(P.A.rp)), slab, bs, op);
            }
            // exclusive scan of the words' popcounts (contiguous words per thread)
            const int wpt = (words + (int)blockDim.x - 1) / (int)blockDim.x;
            const int w0 = tid * wpt;
            int mine = 0;
            for (int j = 0; j < wpt; ++j)
                if (w0 + j < words) mine += __popc(bm[w0 + j]);
            const int incl = warp_incl_scan(mine);
            if (lane == 31) s_wsum[wid] = incl;
            __syncthreads();
            if (wid == 0) {
                const int x = lane < nwarps ? s_wsum[lane] : 0;
                const int xi = warp_incl_scan(x);
                if (lane < nwarps) s_wsum[lane] = xi - x;
                if (lane == 31) word_off[words] = xi;
            }
            __syncthreads();
            {
                int run = s_wsum[wid] + incl - mine;
                for (int j = 0; j < wpt; ++j)
                    if (w0 + j < words) {
                        word_off[w0 + j] = run;
                        run += __popc(bm[w0 + j]);
                    }
            }
            __syncthreads();
            // Warp w writes the outputs [T w / nwarps, T (w+1) / nwarps) of the
            // slab: it visits the words holding them 32 at a time (lane j =
            // word wc + j, bits outside the range masked off); output o of a
            // group is the (o - excl)-th set bit of the lane whose prefix holds o.
            const int T = word_off[words];
            const int64_t slab_base = off + s_written;
            const int o_lo = (int)((int64_t)T * wid / nwarps), o_hi = (int)((int64_t)T * (wid + 1) / nwarps);
            if (o_lo < o_hi) {
                int wlo = 0, whi = words - 1;   // word holding output o_lo
                while (wlo < whi) {
                    const int mid = (wlo + whi + 1) >> 1;
                    if (word_off[mid] <= o_lo) wlo = mid; else whi = mid - 1;
                }
                for (int wc = wlo; wc < words; wc += 32) {   // warp-uniform
                    const int wj = wc + lane;
                    uint32_t bits = 0u;
                    int first_out = 0;   // slab output index of the lane's first kept bit
                    if (wj < words) {
                        const uint32_t all = bm[wj];
                        const int base = word_off[wj];
                        const int nb = __popc(all);
                        const int lo_k = min(max(o_lo - base, 0), nb);
                        const int hi_k = min(max(o_hi - base, 0), nb);
                        bits = all;
                        for (int x = 0; x < lo_k; ++x) bits &= bits - 1u;   // drop lowest
                        for (int x = hi_k; x < nb; ++x) bits &= ~(0x80000000u >> __clz(bits));
                        first_out = base + lo_k;
                    }
                    const int cnt = __popc(bits);
                    const int incl2 = warp_incl_scan(cnt);
                    const int ex2 = incl2 - cnt;
                    const int TT = __shfl_sync(kFull, incl2, 31);
                    for (int o0 = 0; o0 < TT; o0 += 32) {   // warp-uniform
                        const int o = o0 + lane;
                        int owner = 0;
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1) {
                            const int c = owner + step;
                            if (__shfl_sync(kFull, ex2, c) <= o) owner = c;
                        }
                        const uint32_t ob = __shfl_sync(kFull, bits, owner);
                        const int k = o - __shfl_sync(kFull, ex2, owner);
                        const int fo = __shfl_sync(kFull, first_out, owner);
                        if (o < TT) {
                            const unsigned bit = (unsigned)select_bit(ob, k);
                            const int64_t at = slab_base + fo + k;
                            if (bit < 32u && at < off + n) {
                                const int c = (wc + owner) * 32 + (int)bit;
                                write_entry<S>(P, at, lo + c, vals[c]);
                            } else {
                                flag_overflow(st, g);   // counts disagree: never write past the row
                            }
                        }
                    }
                    if (word_off[min(wc + 32, words)] >= o_hi) break;
                }
            }
            __syncthreads();
            if (tid == 0) s_written += T;
            __syncthreads();
        }
        if (tid == 0 && s_written != n) flag_overflow(st, g);
        __syncthreads();
    }
}

// ---- dense tier, rank-indexed (rows whose bitmap fits in shared memory) ----------
//
// Per row: (1) a presence bitmap over all ncols columns is built from the
// products (read before atomicOr); (2) a block-wide prefix of the words'
// popcounts gives every present column its rank = its position in the
// output row; (3) C.col is written from the bitmap, coalesced; (4) values are
// accumulated into a shared array indexed by rank, in passes over groups of
// consecutive column slabs whose outputs fit the array, and each pass writes
// its stretch of C.val in order.  Ranks of ascending columns are consecutive,
// so the accumulation atomics are free of bank conflicts, and a row is walked
// 1 + (number of value passes) times instead of once per column slab.

// How a row's entries reach the product walk: one per lane, the same in
// every warp (<= 32 entries); one per thread, loaded once per row (<= the
// CTA's threads); or loaded batch by batch in every pass.
enum RowEntries { kEntriesPerLane, kEntriesPerThread, kEntriesBatched };

// Products of row entries [a0, a1) restricted to slabs [s0, s1), spread over the CTA.
template <class In, bool kVal, class Op, int NT>
SPG_DEV void cta_range_products(const DCsr& A, const DCsr& B, int64_t a0, int64_t a1,
                                const LaneEntry<In, kVal>& le, RowEntries mode, const int32_t* sp,
                                int sp_stride, int nslabs, int s0, int s1,
                                BatchSmem<In, NT>& bs, Op& op) {
    if (mode == kEntriesPerLane) {
        int64_t b, e;
        le.range(sp, sp_stride, nslabs, s0, s1, b, e);
        warp_table_walk<In, kVal>(B, b, e, le.a, op);
        __syncthreads();
        return;
    }
    if (mode == kEntriesPerThread) {
        int64_t b, e;
        le.range(sp, sp_stride, nslabs, s0, s1, b, e);
        cta_walk_segments<In, kVal>(B, b, e - b, le.a, bs, op);
        return;
    }
    for (int64_t b0 = a0; b0 < a1; b0 += NT) {
        const int64_t p = b0 + threadIdx.x;
        LaneEntry<In, kVal> ent;
        ent.load(A, B, p, p < a1);
        int64_t b, e;
        ent.range(sp, sp_stride, nslabs, s0, s1, b, e);
        cta_walk_segments<In, kVal>(B, b, e - b, ent.a, bs, op);
    }
}

// The rank kernel keeps word w of the row bitmap (x) and the number of set
// bits before it (y) side by side, so one 8-byte load gives a product's rank.
struct BitSetOp {
    uint2* bw;
    template <class In> SPG_DEV void any(int32_t col, In, In, bool valid) {
        if (!valid) return;
        atomicOr(&bw[col >> 5].x, 1u << (col & 31));   // plain atomic: no read of the word first
    }
};

// kFilter: the walk may reach products outside the pass's columns (no slab
// table), which are skipped
template <class S, bool kFilter>
struct RankAccOp {
    typename S::Slot* vals;
    int32_t* cols;      // column of each rank (every product of a column stores the same value)
    const uint2* bw;
    int32_t r1;         // rank of the pass's first output, plus one
    int32_t clo;        // columns of this pass: [clo, clo + width)
    uint32_t width;
    int32_t cnt;        // outputs of the pass (checked build: ranks must fall below it)
    DevStatus* st;
    SPG_DEV void any(int32_t col, typename S::In a, typename S::In b, bool valid) {
        if (!valid) return;
        if constexpr (kFilter) {
            if ((uint32_t)(col - clo) >= width) return;
        }
        const uint2 e = bw[col >> 5];
        // bits of the word at or below col's bit (col's own bit is set): its rank + 1
        const int r = (int)e.y + __popc(e.x << (~col & 31)) - r1;
#ifdef SPG_CHECKS
        // a column missing from the row's bitmap (B's pattern changed since the
        // symbolic call) or a rank outside the pass: skip the write
        if (!((e.x >> (col & 31)) & 1u) || (uint32_t)r >= (uint32_t)cnt) {
            flag_invalid(st, col);
            return;
        }
#endif
        S::acc(vals + r, a, b);
        cols[r] = col;
    }
};

constexpr int kRankThreads = 1024;
// rank scan: chunks of 32 words scanned together (one for the overlap slots,
// whose walk needs the registers)
template <class S>
constexpr int rank_scan_chunks() { return sizeof(typename S::Slot) > 8 ? 1 : 4; }

// bytes of the rank kernel's value array, rounded up to 16
template <class S>
__host__ __device__ inline size_t rank_slot_bytes(int64_t cap) {
    return S::kVal ? (((size_t)cap * sizeof(typename S::Slot) + 15) & ~(size_t)15) : 0;
}
// the value array followed by the column of each rank
template <class S>
__host__ __device__ inline size_t rank_val_bytes(int64_t cap) {
    return S::kVal ? rank_slot_bytes<S>(cap) + (((size_t)cap * 4 + 15) & ~(size_t)15) : 0;
}
// shared-memory bytes per output of a value pass
template <class S>
constexpr size_t rank_entry_bytes() {
    return S::kVal ? sizeof(typename S::Slot) + 4 : 0;
}
// the value array's region; without values it serves as the warps' C.col
// staging instead: at least 3 KB per warp of an NT-thread CTA
template <class S, int NT>
__host__ __device__ inline size_t rank_region_bytes(int64_t cap) {
    const size_t v = rank_val_bytes<S>(cap);
    constexpr size_t kStageMin = S::kVal ? 0 : (size_t)(NT / 32) * 3072;
    return v > kStageMin ? v : kStageMin;
}

// NT = 1024: one CTA per SM, the whole shared memory for the bitmap and the
// value array (value passes over slab groups).  NT = 512: two CTAs per SM,
// each with half of it, for rows whose outputs fit one pass: two rows in
// flight per SM hide the per-row phases' latency.  The 512-thread kernel
// takes the light dense rows (their own tier: ub_i below the tuning's
// rank_light_ub, a few thousand products whose time is per-row latency, not
// product work, and outputs within one pass), the 1024-thread one the dense
// tier's; each kernel has its own claim counter.
template <class S, int NT>
__global__ void __launch_bounds__(NT, kRankThreads / NT)
    k_num_rank(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
               Counters* ctr, DevStatus* st, int sp_stride,
               int slab_cols, int bm_words, int cap, const uint32_t* __restrict__ bm_cache,
               const int32_t* __restrict__ row_slot, int cache_words, int64_t cache_slots,
               int stage_words, int ovl_mode, int tier, int claim) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);                          // [cap]
    int32_t* cols = reinterpret_cast<int32_t*>(smem_raw + rank_slot_bytes<S>(cap));   // [cap]
    // filled with 16-byte stores: its offset must be 16-aligned
    uint2* bw = reinterpret_cast<uint2*>(smem_raw + rank_region_bytes<S, NT>(cap));   // [words + 1]
    __shared__ BatchSmem<In, NT> bs;
    __shared__ int s_row;
    __shared__ int s_wsum[NT / 32];
    const int lane = lane_id(), wid = warp_id(), nwarps = blockDim.x >> 5;
    const int tid = threadIdx.x;
    const int tbeg = ctr->num_bin_off[tier * kSubBins];
    const int tend = ctr->num_bin_off[(tier + 1) * kSubBins];
    // the value array holds `empty` between passes: filled once here, and each
    // pass's write-out empties the slots it reads
    // overlap: the compact-slot kernel (ovl_mode 1) takes the rows when every
    // position fits 16 bits, the 24-byte one (ovl_mode 2) when one does not
    if ((ovl_mode == 1 && ctr->ovl_wide) || (ovl_mode == 2 && !ctr->ovl_wide)) return;
    if constexpr (S::kVal) fill_slots<S>(vals, cap);
    // Rows are claimed one ahead: thread 0 claims the next row while this one
    // starts, and loads its id, then its cache slot, each a phase later, and
    // prefetches its cached bitmap into L2 after the first value pass's walk,
    // so the next row's bitmap copy does not wait on DRAM (nothing waits on
    // these loads until a phase boundary has passed).
    if (tid == 0) s_row = tbeg + atomicAdd(&ctr->claim[claim], 1);
    __syncthreads();
    for (;;) {
        const int r = s_row;   // written one row ahead, read after a barrier
        if (r >= tend) break;
        int nr = tend;
        int64_t g2 = -1;
        int slot2 = -1;
        if (tid == 0) nr = tbeg + atomicAdd(&ctr->claim[claim], 1);
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t off = P.c_rp[i];
        const int64_t n = P.c_rp[i + 1] - off;
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        const int ncols = (int)P.B.ncols;
        const int words = (ncols + 31) >> 5;
        const int nslabs = (ncols + slab_cols - 1) / slab_cols;
        const int32_t* __restrict__ sp = P.sp;   // this product's slab-start table, or null
        const RowEntries mode = a1 - a0 <= 32 ? kEntriesPerLane
                                : a1 - a0 <= NT ? kEntriesPerThread : kEntriesBatched;
        // (a slot outside the cache means the workspace did not come from this
        // product's symbolic call: the row is rebuilt and checked against c_rp)
        const int slot = row_slot ? row_slot[g] : -1;
        const bool cached = slot >= 0 && slot < cache_slots && words <= cache_words;
        // the row's entries, held in registers for every walk of the row (none
        // without values when the bitmap comes from the cache)
        LaneEntry<In, S::kVal> le;
        if (S::kVal || !cached) {
            if (mode == kEntriesPerLane) le.load(P.A, P.B, a0 + lane, a0 + lane < a1);
            else if (mode == kEntriesPerThread) le.load(P.A, P.B, a0 + tid, a0 + tid < a1);
        }
        // (1) presence bitmap of the whole row: the symbolic phase's copy if it
        //     kept one, else rebuilt from the products
        if (cached) {
            const uint4* src = reinterpret_cast<const uint4*>(bm_cache + (int64_t)slot * cache_words);
            uint4* dst = reinterpret_cast<uint4*>(bw);   // two (word, offset) pairs per store
            for (int w = tid; w < (words + 3) / 4; w += blockDim.x) {
                const uint4 v = __ldcs(src + w);
                dst[2 * w] = make_uint4(v.x, 0u, v.y, 0u);
                dst[2 * w + 1] = make_uint4(v.z, 0u, v.w, 0u);
            }
            __syncthreads();
        } else {
            for (int w = tid; w < words; w += blockDim.x) bw[w] = make_uint2(0u, 0u);
            __syncthreads();
            BitSetOp op{bw};
            cta_range_products<In, S::kVal>(P.A, P.B, a0, a1, le, mode, sp, sp_stride, nslabs, 0,
                                            nslabs, bs, op);
        }
        if (tid == 0) {   // every thread has read r: publish the next row
            s_row = nr;
            if (nr < tend && row_slot) g2 = rows[nr];
        }
        // (2) ranks: exclusive prefix of the words' popcounts.  Warp w scans a
        //     contiguous block of words, lane l reading word base + l + 32 j
        //     (no bank conflicts), into block-local offsets; the warps' block
        //     offsets come from a scan of the block totals and are added in
        //     step 3.
        const int per_warp = ((words + nwarps - 1) / nwarps + 31) & ~31;
        const int wb = wid * per_warp;
        {
            constexpr int kSU = rank_scan_chunks<S>();
            int run = 0;
            // kSU chunks of 32 words at a time: their scans are independent
            // (only the running total links them), so their shuffles overlap
            for (int j0 = 0; j0 < per_warp; j0 += 32 * kSU) {
                int c[kSU], inc[kSU];
#pragma unroll
                for (int u = 0; u < kSU; ++u) {
                    const int w = wb + j0 + 32 * u + lane;
                    c[u] = (j0 + 32 * u < per_warp && w < words) ? __popc(bw[w].x) : 0;
                }
#pragma unroll
                for (int u = 0; u < kSU; ++u) inc[u] = warp_incl_scan(c[u]);
#pragma unroll
                for (int u = 0; u < kSU; ++u) {
                    const int w = wb + j0 + 32 * u + lane;
                    if (j0 + 32 * u < per_warp && w < words) bw[w].y = (uint32_t)(run + inc[u] - c[u]);
                    run += __shfl_sync(kFull, inc[u], 31);
                }
            }
            if (lane == 0) s_wsum[wid] = run;
            __syncthreads();
            if (wid == 0) {
                const int x = lane < nwarps ? s_wsum[lane] : 0;
                const int xi = warp_incl_scan(x);
                if (lane < nwarps) s_wsum[lane] = xi - x;
                if (lane == 31) bw[words].y = (uint32_t)xi;
            }
            __syncthreads();
        }
        if (g2 >= 0) slot2 = row_slot[g2];
        const int T = (int)bw[words].y;
        if (T != n) {   // symbolic and numeric disagree: leave the row
            if (tid == 0) flag_overflow(st, g);
            __syncthreads();
            continue;
        }
        // (3) The block-local offsets made global, and (semirings without
        //     values only) C.col from the bitmap; with values, step 4 writes
        //     C.col from the columns its products store by rank.
        //     Warp w walks its block 32 words at a time (lane = word).  When
        //     the chunk's set bits are spread evenly over its words, each lane
        //     expands its own word into the warp's staging area (the value
        //     array is free until step 4) at its offset, and the chunk is
        //     copied to C.col 32 consecutive entries per store (a chunk too
        //     dense for the staging area writes each lane's columns directly).
        //     When a few words hold most of the bits (a skewed column
        //     distribution such as R-MAT's), that loop would run as long as
        //     the densest word: the chunk is expanded output by output
        //     instead.  Lane l takes outputs t = l, l + 32, ..., finds the
        //     word holding t by a binary search over the words' prefix
        //     counts, the bit by select_bit, and stores C.col[t] (coalesced).
        if constexpr (S::kVal) {
            const int add = s_wsum[wid];
            const int wend = min(wb + per_warp, words);
#pragma unroll 4
            for (int w = wb + lane; w < wend; w += 32) bw[w].y += (uint32_t)add;
        } else {
            int32_t* stage = reinterpret_cast<int32_t*>(smem_raw) + (size_t)wid * stage_words;
            const int add = s_wsum[wid];
            const int wtot = (wid + 1 < nwarps ? s_wsum[wid + 1] : T) - add;
            for (int j = 0; j < per_warp && wb + j < words; j += 32) {
                const int w0 = wb + j;
                const int w = w0 + lane;
                const int lbase = (int)bw[w0].y;
                const int lnext = (j + 32 < per_warp && w0 + 32 < words) ? (int)bw[w0 + 32].y : wtot;
                const int lw = w < words ? (int)bw[w].y : 0;
                __syncwarp();
                if (w < words) bw[w].y = (uint32_t)(lw + add);
                const int Tc = lnext - lbase;
                if (Tc == 0) continue;
                uint32_t bits = w < words ? bw[w].x : 0u;
                int pos = w < words ? lw - lbase : Tc;   // chunk-local exclusive prefix
                const int cbase = w * 32;
                int32_t* dst = P.c_col + off + add + lbase;
                const int maxc = (int)__reduce_max_sync(kFull, (unsigned)__popc(bits));
                if (maxc > 4 * ((Tc + 31) >> 5)) {
                    const int inc = pos + __popc(bits);
                    for (int t0 = 0; t0 < Tc; t0 += 32) {   // warp-uniform
                        const int t = t0 + lane;
                        int k = 0;   // number of words whose outputs all precede t
#pragma unroll
                        for (int step = 16; step > 0; step >>= 1)
                            if (__shfl_sync(kFull, inc, k + step - 1) <= t) k += step;
                        const uint32_t bk = __shfl_sync(kFull, bits, k);
                        const int ek = __shfl_sync(kFull, pos, k);
                        if (t < Tc) st_stream(dst + t, (int32_t)((w0 + k) * 32 + select_bit(bk, t - ek)));
                    }
                } else if (Tc <= stage_words) {
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        stage[pos++] = cbase + b;
                    }
                    __syncwarp();
                    for (int t = lane; t < Tc; t += 32) st_stream(dst + t, stage[t]);
                    __syncwarp();
                } else {
                    while (bits) {
                        const int b = __ffs(bits) - 1;
                        bits &= bits - 1u;
                        st_stream(dst + pos++, (int32_t)(cbase + b));
                    }
                }
            }
        }
        __syncthreads();
        // (the next row's bitmap: with values, prefetched after the first
        // pass's walk, by when thread 0's load of its cache slot has landed)
        if (!S::kVal && slot2 >= 0 && slot2 < cache_slots)
            prefetch_l2(bm_cache + (int64_t)slot2 * cache_words, (uint32_t)cache_words * 4u);
        // (4) values, in passes over groups of column slabs that fit `cap` outputs;
        //     each pass writes its stretch of C.col and C.val
        if constexpr (S::kVal) {
            int s0 = 0;
            while (s0 < nslabs) {
                const int r0 = (int)bw[(s0 * slab_cols) >> 5].y;
                // s1 = s0 + 1, then every later slab while the group's outputs
                // fit cap.  The output count before a slab end grows with the
                // end, so the lanes test 32 ends at once and the ones that
                // pass are a prefix of the lanes.
                int s1 = s0 + 1;
                for (;;) {
                    const int t = s1 + 1 + lane;   // group [s0, t)
                    const bool fits =
                        t <= nslabs &&
                        (int)bw[min((int64_t)t * slab_cols, (int64_t)ncols + 31) >> 5].y - r0 <= cap;
                    const int k = __popc(__ballot_sync(kFull, fits));
                    s1 += k;
                    if (k < 32) break;
                }
                const int r1 = (int)bw[min((int64_t)s1 * slab_cols, (int64_t)ncols + 31) >> 5].y;
                const int cnt = r1 - r0;
                if (cnt > 0) {
                    const int clo = s0 * slab_cols;
                    const int chi = s1 >= nslabs ? ncols : s1 * slab_cols;
                    // with the slab table the walk covers only the pass's slabs;
                    // without it every product is visited and filtered
                    if (sp != nullptr || (s0 == 0 && s1 >= nslabs)) {
                        RankAccOp<S, false> op{vals, cols, bw, r0 + 1, clo, (uint32_t)(chi - clo),
                                               cnt, st};
                        cta_range_products<In, S::kVal>(P.A, P.B, a0, a1, le, mode, sp, sp_stride,
                                                        nslabs, s0, s1, bs, op);
                    } else {
                        RankAccOp<S, true> op{vals, cols, bw, r0 + 1, clo, (uint32_t)(chi - clo),
                                              cnt, st};
                        cta_range_products<In, S::kVal>(P.A, P.B, a0, a1, le, mode, sp, sp_stride,
                                                        nslabs, 0, nslabs, bs, op);
                    }
                    if (slot2 >= 0 && slot2 < cache_slots)
                        prefetch_l2(bm_cache + (int64_t)slot2 * cache_words, (uint32_t)cache_words * 4u);
                    slot2 = -1;   // once per row
                    typename S::Out* cv = reinterpret_cast<typename S::Out*>(P.c_val) + off + r0;
                    int32_t* cc = P.c_col + off + r0;
                    for (int t = tid; t < cnt; t += blockDim.x) {
                        st_stream(cv + t, S::out(vals[t]));
                        st_stream(cc + t, cols[t]);
                        vals[t] = S::empty();
                    }
                    __syncthreads();
                }
                s0 = s1;
            }
        }
        __syncthreads();
    }
}

// ---- deterministic plus-times values ---------------------------------------------
//
// Recomputes the values of C rows already written (sorted columns known): a
// warp per row takes A_i's entries in order; for entry k the lanes cover
// B_k's entries (distinct columns), find each column's position in the row by
// binary search and add the product there.  Every position is updated in k
// order, starting from -0 (the identity that keeps the first product exactly,
// signed zeros included), with separately rounded products and sums: the
// result is the sequential left fold of the definition (Section 2.1),
// whatever the schedule.
template <class S>
SPG_DEV typename S::Out det_zero() {
    if constexpr (std::is_floating_point<typename S::Out>::value) return -typename S::Out(0);
    else return typename S::Out(0);
}

template <class S>
__global__ void k_det_values(const Prob* __restrict__ probs, int nprob, int64_t R) {
    using In = typename S::In;
    using Out = typename S::Out;
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); g < R; g += nw) {
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t cs = P.c_rp[i], ce = P.c_rp[i + 1];
        Out* cv = reinterpret_cast<Out*>(P.c_val);
        const int32_t* cc = P.c_col;
        for (int64_t t = cs + lane; t < ce; t += 32) cv[t] = det_zero<S>();
        __syncwarp();
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        for (int64_t p = a0; p < a1; ++p) {
            const int32_t k = ld_i32(P.A.col + p);
            const In a = load_val<In, true>(P.A.val, p);
            const int64_t b0 = ld_i64(P.B.rp + k), b1 = ld_i64(P.B.rp + k + 1);
            for (int64_t q = b0 + lane; q < b1; q += 32) {
                const int32_t j = ld_i32(P.B.col + q);
                int64_t lo = cs, hi = ce;   // first position with column >= j
                while (lo < hi) {
                    const int64_t m = (lo + hi) >> 1;
                    if (cc[m] < j) lo = m + 1; else hi = m;
                }
                if (lo < ce && cc[lo] == j)
                    cv[lo] = S::add(cv[lo], S::prod(a, load_val<In, true>(P.B.val, q)));
            }
            __syncwarp();   // entry k's updates land before entry k+1's
        }
    }
}

struct DetLaunch {
    const WsPtrs* w;
    int nprob;
    int64_t R;
    const DevInfo* dev;
    cudaStream_t st;
    template <class S> void operator()() {
        if constexpr (std::is_same<S, SrPtF64>::value || std::is_same<S, SrPtF32>::value) {
            int64_t blocks = (R + 7) / 8;
            if (blocks > (int64_t)dev->sms * 32) blocks = (int64_t)dev->sms * 32;
            if (blocks < 1) blocks = 1;
            k_det_values<S><<<(unsigned)blocks, 256, 0, st>>>(w->probs, nprob, R);
            count_launch(*dev);
        }
    }
};

cudaError_t launch_det_values(int sr, const WsPtrs& w, int nprob, int64_t R, const DevInfo& dev,
                              cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    DetLaunch f{&w, nprob, R, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

// ---- slab starts of B's rows ------------------------------------------------------

// sp[k * (nslabs + 1) + t] = offset in row k of B of its first column >= t * W
// (t = nslabs gives the row length).  Skipped when no row is in the dense tier.
__global__ void k_slab_ptr(DCsr B, int W, int nslabs, int32_t* sp, const Counters* ctr) {
    if (ctr->num_bin_off[(kTierDense + 1) * kSubBins] == ctr->num_bin_off[kTierDense * kSubBins])
        return;
    const int lane = lane_id();
    const int stride = nslabs + 1;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t k = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); k < B.nrows; k += nw) {
        const int64_t rs = ld_i64(B.rp + k), re = ld_i64(B.rp + k + 1);
        for (int t = lane; t <= nslabs; t += 32) {
            const int64_t lim = (int64_t)t * W;
            int64_t a = rs, b = re;
            while (a < b) {
                const int64_t m = (a + b) >> 1;
                if ((int64_t)ld_i32(B.col + m) < lim) a = m + 1; else b = m;
            }
            sp[k * stride + t] = (int32_t)(a - rs);
        }
    }
}

// ---- launchers -------------------------------------------------------------------

template <class S>
size_t num_warp_bytes(const Tuning& t) {
    int64_t T = next_pow2(2 * t.num_warp_max_nnz);
    if (T < 32) T = 32;
    size_t b = (size_t)T * sizeof(typename S::Slot) + (size_t)T * 4 + (size_t)(T / 2) * 4;
    return (b + 15) & ~(size_t)15;
}

template <class S>
size_t num_block_bytes(const Tuning& t) {
    int64_t T = next_pow2(2 * t.num_block_max_nnz);
    if (T < 32) T = 32;
    return (size_t)T * sizeof(typename S::Slot) + (size_t)T * 4 + (size_t)(T / 2) * 4;
}

template <class S>
size_t num_dense_bytes(int64_t slab_cols) {
    return dense_val_bytes<S>(slab_cols) + (size_t)slab_cols / 8 +
           ((size_t)slab_cols / 32 + 1) * 4;
}

struct SizeFn {
    int which;
    const Tuning* t;
    int64_t slab;
    size_t out = 0;
    template <class S> void operator()() {
        if (which == 0) out = num_warp_bytes<S>(*t);
        else if (which == 1) out = num_block_bytes<S>(*t);
        else out = num_dense_bytes<S>(slab);
    }
};

size_t num_warp_smem_per_warp(int sr, const Tuning& t) {
    SizeFn f{0, &t, 0};
    dispatch_semiring(sr, f);
    return f.out;
}
size_t num_block_smem(int sr, const Tuning& t) {
    SizeFn f{1, &t, 0};
    dispatch_semiring(sr, f);
    return f.out;
}
size_t num_dense_smem(int sr, int64_t slab_cols) {
    SizeFn f{2, nullptr, slab_cols};
    dispatch_semiring(sr, f);
    return f.out;
}

static int occupancy_grid(const void* fn, int threads, size_t smem, const DevInfo& dev) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem);
    if (per_sm < 1) per_sm = 1;
    return per_sm * dev.sms;
}

// Launch parameters of the rank-indexed kernel for semiring S on NT-thread
// CTAs: the row bitmap ((word, prefix) pairs) and the value array of `cap`
// outputs share the CTA's dynamic shared memory.  NT = 1024 takes the whole
// per-block limit and needs room for at least one slab's outputs (rows of any
// size, in value passes); NT = 512 takes half an SM (two CTAs per SM) and is
// given only rows whose outputs all fit one pass.  ok = false when it does
// not fit.
struct RankCfg {
    bool ok;
    int64_t bm_words, cap;
    size_t smem;
    int stage_words;
};
template <class S, int NT>
RankCfg rank_cfg(int64_t max_ncols, int64_t slab, const DevInfo& dev) {
    RankCfg c{};
    c.bm_words = (max_ncols + 1023) / 1024 * 32;
    const size_t fixed = (size_t)c.bm_words * 8 + 16;
    // dynamic shared memory: the per-block limit (half an SM's for NT = 512)
    // less the kernel's static variables (the batch arrays and a little more)
    size_t lim = dev.max_smem_optin > 0 ? (size_t)dev.max_smem_optin : 212 * 1024;
    if (NT < kRankThreads) {
        const size_t per_sm = dev.max_smem_sm > 0 ? (size_t)dev.max_smem_sm : 228 * 1024;
        const size_t half = per_sm / (kRankThreads / NT) - 1024;   // 1 KB reserved per CTA
        if (half < lim) lim = half;
    }
    const size_t stat = sizeof(BatchSmem<typename S::In, NT>) + 1024;
    if (lim <= stat + fixed + 32) return c;
    const size_t budget = lim - stat;
    int64_t cap = S::kVal ? (int64_t)((budget - fixed - 32) / rank_entry_bytes<S>()) : 0;
    if (cap > (int64_t)1 << 30) cap = (int64_t)1 << 30;
    c.cap = cap;
    const bool room = NT == kRankThreads ? (!S::kVal || cap >= slab) : (!S::kVal || cap >= 1);
    c.ok = room && rank_region_bytes<S, NT>(cap) + fixed <= budget && max_ncols < INT32_MAX;
    const size_t region = rank_region_bytes<S, NT>(cap);
    c.smem = region + fixed;
    c.stage_words = (int)(region / (NT / 32) / 4);
    return c;
}

// The largest nnz(C_i) of a light dense row for semiring S (0: none): the
// 1024-thread rank kernel must serve the dense tier, the 512-thread one must
// fit two CTAs per SM; a light row's outputs fit one pass of the latter.
template <class S>
int64_t light_limit(const Tuning& t, int64_t max_ncols, const DevInfo& dev) {
    if (t.rank_light_ub <= 0) return 0;
    int64_t slab;
    int nslabs;
    dense_slabs(t, max_ncols, &slab, &nslabs);
    if (!rank_cfg<S, kRankThreads>(max_ncols, slab, dev).ok) return 0;
    const RankCfg small = rank_cfg<S, kRankThreads / 2>(max_ncols, slab, dev);
    if (!small.ok) return 0;
    if (cudaFuncSetAttribute(k_num_rank<S, kRankThreads / 2>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)small.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, (const void*)k_num_rank<S, kRankThreads / 2>, kRankThreads / 2,
            small.smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (per_sm < 2) return 0;
    return S::kVal ? small.cap : INT64_MAX;
}

// light limits of the semiring: with compact overlap slots (narrow) and
// without (wide); the same for the other semirings
struct LightFn {
    const Tuning* t;
    int64_t max_ncols;
    const DevInfo* dev;
    int64_t narrow = 0, wide = 0;
    template <class S> void operator()() {
        if constexpr (std::is_same<S, SrOverlap>::value) {
            narrow = light_limit<SrOverlapC>(*t, max_ncols, *dev);
            wide = light_limit<S>(*t, max_ncols, *dev);
        } else {
            narrow = wide = light_limit<S>(*t, max_ncols, *dev);
        }
    }
};

__global__ void k_set_light(Counters* ctr, int64_t narrow, int64_t wide) {
    if (threadIdx.x == 0 && blockIdx.x == 0) ctr->light_n = ctr->ovl_wide ? wide : narrow;
}

struct NumericLaunch {
    const WsPtrs* w;
    DCsr B0;              // B of the first product (slab pointers: single product only)
    int nprob;
    const Tuning* t;
    int64_t max_ncols;
    const DevInfo* dev;
    cudaStream_t st;
    const SlabTables* tables;
    int64_t light_narrow, light_wide;   // light-row limits (LightFn)
    cudaError_t err = cudaSuccess;
    template <class S, int NT>
    cudaError_t launch_rank(const RankCfg& c, int64_t slab, int nslabs, int ovl_mode,
                            int tier, int claim) {
        cudaError_t e = cudaFuncSetAttribute(
            k_num_rank<S, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c.smem);
        if (e != cudaSuccess) return e;
        const int grid = occupancy_grid((const void*)k_num_rank<S, NT>, NT, c.smem, *dev);
        const bool cached = w->bm_cache && w->bm_cache_words >= c.bm_words;
        k_num_rank<S, NT><<<grid, NT, c.smem, st>>>(
            w->probs, nprob, w->rows_num, w->ctr, w->status, nslabs + 1, (int)slab,
            (int)c.bm_words, (int)c.cap, cached ? w->bm_cache : nullptr,
            cached ? w->row_slot : nullptr, (int)w->bm_cache_words, w->bm_cache_slots,
            c.stage_words, ovl_mode, tier, claim);
        count_launch(*dev);
        return cudaGetLastError();
    }
    // the dense tier on the 1024-thread kernel (claim slot 3) and, when light
    // rows can exist, the light tier on the 512-thread one (claim slot 4)
    template <class S>
    cudaError_t launch_rank_pair(int64_t slab, int nslabs, int ovl_mode, int64_t light_n) {
        const RankCfg big = rank_cfg<S, kRankThreads>(max_ncols, slab, *dev);
        cudaError_t e = launch_rank<S, kRankThreads>(big, slab, nslabs, ovl_mode, kTierDense, 3);
        if (e == cudaSuccess && light_n > 0) {
            const RankCfg small = rank_cfg<S, kRankThreads / 2>(max_ncols, slab, *dev);
            e = launch_rank<S, kRankThreads / 2>(small, slab, nslabs, ovl_mode, kTierDenseLight, 4);
        }
        return e;
    }
    template <class S> void operator()() {
        cudaError_t e;
        {   // dense tier
            int64_t slab;
            int nslabs;
            dense_slabs(*t, max_ncols, &slab, &nslabs);
            const size_t smem = num_dense_bytes<S>(slab);
            e = cudaFuncSetAttribute(k_num_dense<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            // the slab-start table of every distinct B (skipped on the device
            // when no row is in the dense tier)
            const bool sp = tables && tables->n > 0;
            for (int j = 0; sp && j < tables->n; ++j) {
                k_slab_ptr<<<dev->sms * 8, 256, 0, st>>>(tables->B[j], (int)slab, nslabs,
                                                         tables->sp[j], w->ctr);
                count_launch(*dev);
            }
            mark_stage(*dev, kStSlabPtr, st);
            // rank-indexed kernel when the row bitmap, its prefix and a value
            // array of at least one slab fit in shared memory
            const RankCfg rc = rank_cfg<S, kRankThreads>(max_ncols, slab, *dev);
            if (rc.ok) {
                if constexpr (std::is_same<S, SrOverlap>::value) {
                    // compact 12-byte slots when every position fits 16 bits
                    // (twice the outputs per value pass, 32-bit atomics)
                    e = launch_rank_pair<SrOverlapC>(slab, nslabs, 1, light_narrow);
                    if (e == cudaSuccess) e = launch_rank_pair<S>(slab, nslabs, 2, light_wide);
                } else {
                    e = launch_rank_pair<S>(slab, nslabs, 0, light_narrow);
                }
                if (e != cudaSuccess) { err = e; return; }
            } else {
                const int grid = occupancy_grid((const void*)k_num_dense<S>, kBlockThreads, smem, *dev);
                k_num_dense<S><<<grid, kBlockThreads, smem, st>>>(w->probs, nprob, w->rows_num, w->ctr,
                                                                  w->status, w->cursor, (int)slab,
                                                                  nslabs + 1);
                count_launch(*dev);
            }
            mark_stage(*dev, kStNumDense, st);
        }
        {   // block tier
            int only_wide = 0;
            if constexpr (std::is_same<S, SrOverlap>::value) {
                // compact slots first (they leave every row to the 24-byte
                // kernel when a position needs more than 16 bits)
                const int64_t Tc = next_pow2((4 * kOvlCompactMax + 2) / 3);
                const size_t smc = (size_t)Tc * (sizeof(OvSlotC) + 8);
                e = cudaFuncSetAttribute(k_num_block<SrOverlapC>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smc);
                if (e != cudaSuccess) { err = e; return; }
                const int gc = occupancy_grid((const void*)k_num_block<SrOverlapC>, kBlockThreads,
                                              smc, *dev);
                k_num_block<SrOverlapC><<<gc, kBlockThreads, smc, st>>>(
                    w->probs, nprob, w->rows_num, w->ctr, w->status, (int)Tc, 0);
                count_launch(*dev);
                only_wide = 1;
            }
            int64_t T = next_pow2(2 * t->num_block_max_nnz);
            if (T < 32) T = 32;
            const size_t smem = num_block_bytes<S>(*t);
            e = cudaFuncSetAttribute(k_num_block<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            const int grid = occupancy_grid((const void*)k_num_block<S>, kBlockThreads, smem, *dev);
            k_num_block<S><<<grid, kBlockThreads, smem, st>>>(w->probs, nprob, w->rows_num, w->ctr,
                                                              w->status, (int)T, only_wide);
            count_launch(*dev);
            mark_stage(*dev, kStNumBlock, st);
        }
        {   // warp tier
            int64_t T = next_pow2(2 * t->num_warp_max_nnz);
            if (T < 32) T = 32;
            const size_t smem = num_warp_bytes<S>(*t) * kWarpTierWarps;
            e = cudaFuncSetAttribute(k_num_warp<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            const int grid =
                occupancy_grid((const void*)k_num_warp<S>, kWarpTierWarps * 32, smem, *dev);
            k_num_warp<S><<<grid, kWarpTierWarps * 32, smem, st>>>(w->probs, nprob, w->rows_num,
                                                                   w->ctr, w->ub, w->status,
                                                                   (int)T);
            count_launch(*dev);
            mark_stage(*dev, kStNumWarp, st);
        }
        err = cudaGetLastError();
    }
};

void dense_slabs(const Tuning& t, int64_t max_ncols, int64_t* slab, int* nslabs) {
    int64_t s = t.dense_slab_cols;
    if (s > max_ncols) s = (max_ncols + 1023) / 1024 * 1024;
    if (s < 1024) s = 1024;
    *slab = s;
    *nslabs = (int)((max_ncols + s - 1) / s);
}

cudaError_t launch_numeric(int sr, const WsPtrs& w, const DCsr& B0, int nprob, int64_t R,
                           const Tuning& t, int64_t max_ncols, const DevInfo& dev,
                           cudaStream_t st, const SlabTables* tables, const ProbTable* probs_host) {
    if (R == 0) return cudaSuccess;
    // reset numeric bins and claims
    cudaMemsetAsync(w.ctr->num_bin_count, 0, sizeof(w.ctr->num_bin_count), st);
    cudaMemsetAsync(&w.ctr->claim[2], 0, 3 * sizeof(int32_t), st);   // slots 2..4
    cudaMemsetAsync(&w.ctr->ovl_wide, 0, sizeof(int32_t), st);
    cudaMemsetAsync(&w.ctr->num_block_max, 0, sizeof(int64_t), st);
    if (sr == SR_OVERLAP && !probs_host) {
        // positions unchecked: no compact overlap slots
        cudaMemsetAsync(&w.ctr->ovl_wide, 1, 1, st);
    } else if (sr == SR_OVERLAP) {
        // compact overlap slots (block and rank tiers) when every position of
        // every A and B fits 16 bits
        for (int p = 0; p < nprob; ++p) {
            const DCsr* mats[2] = {&probs_host->p[p].A, &probs_host->p[p].B};
            for (const DCsr* M : mats) {
                int64_t blocks = (M->nrows + 255) / 256;
                if (blocks > (int64_t)dev.sms * 8) blocks = (int64_t)dev.sms * 8;
                if (blocks < 1) blocks = 1;
                if (M->val) k_ovl_check<<<(unsigned)blocks, 256, 0, st>>>(*M, w.ctr);
            }
        }
        k_ovl_limit<<<1, 32, 0, st>>>(
            w.ctr, t.num_block_max_nnz <= kOvlCompactMax ? kOvlCompactMax : 0);
        count_launch(dev, 2 * nprob + 1);
    }
    LightFn lf{&t, max_ncols, &dev};
    if (!dispatch_semiring(sr, lf)) return cudaErrorInvalidValue;
    k_set_light<<<1, 32, 0, st>>>(w.ctr, lf.narrow, lf.wide);
    count_launch(dev);
    int64_t blocks = (R + 255) / 256;
    if (blocks > (int64_t)dev.sms * 8) blocks = (int64_t)dev.sms * 8;
    k_num_hist<<<(unsigned)blocks, 256, 0, st>>>(w.probs, nprob, R, t, w.ub, w.ctr, w.skip);
    k_num_bin_offsets<<<1, 32, 0, st>>>(w.ctr);
    k_num_scatter<<<(unsigned)((R + 1023) / 1024), 1024, 0, st>>>(w.probs, nprob, R, t, w.ub,
                                                                   w.ctr, w.rows_num, w.skip);
    count_launch(dev, 3);
    mark_stage(dev, kStNumBin, st);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    NumericLaunch f{&w, B0, nprob, &t, max_ncols, &dev, st, tables, lf.narrow, lf.wide};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    return f.err;
}

}  // namespace spg
