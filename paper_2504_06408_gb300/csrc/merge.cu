// Merge of per-stage partial products and column splits of a matrix.
//
// Merge (Sections 2.1 and 3.4: the partial products of the Sparse-SUMMA
// stages are combined into C; the paper does this on the CPU through COO
// tuples and names a GPU merge as future work):
//     C[i,j] = P_0[i,j] (+) P_1[i,j] (+) ... (+) P_{S-1}[i,j]
// folded in stage order, over the entries present in each partial.
//   1. every entry of every partial gets its position in row i of the merged
//      sequence (duplicates kept, equal columns ordered by stage): its index
//      in its own list plus, per other stage t, the number of entries of row
//      i of P_t with a smaller column (t > s) or a smaller-or-equal column
//      (t < s), by binary search; entries are scattered there;
//   2. a row's distinct columns are the first entries of runs of equal
//      columns; their count gives C's row pointers (scan);
//   3. each run is folded in stage order by the thread at its head and
//      written at its rank among the distinct columns.
// Deterministic: the same partials give the same bits whatever the schedule.
//
// Column split (the block layout of Sparse SUMMA, Section 2.1): part p of M
// keeps columns [cut_p, cut_{p+1}) of every row, with column ids made local.
// Rows of a CSR are views (row pointer offsets), so blocks (I, J) are a row
// view of column part J.
#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

// ---- merge ---------------------------------------------------------------------

// row of entry e of a CSR with n rows: last i with rp[i] <= e
SPG_DEV int64_t row_of(const int64_t* rp, int64_t n, int64_t e) {
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (ld_i64(rp + mid) <= e) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// first position q in [lo, hi) with col[q] >= v (or > v when `upper`)
SPG_DEV int64_t lower_pos(const int32_t* col, int64_t lo, int64_t hi, int32_t v, bool upper) {
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        const int32_t c = ld_i32(col + m);
        if (c < v || (upper && c == v)) lo = m + 1; else hi = m;
    }
    return lo;
}

// trp[g] (g = flat row) = total entries of row g over all stages
__global__ void k_merge_rowlen(const MergeProb* __restrict__ mp, int nprob, int64_t R,
                               int64_t* trp) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x) {
        const MergeProb& M = mp[nprob == 1 ? 0 : find_merge_prob(mp, nprob, g)];
        const int64_t i = g - M.row_base;
        int64_t s = 0;
        for (int t = 0; t < M.nparts; ++t) s += ld_i64(M.rp[t] + i + 1) - ld_i64(M.rp[t] + i);
        trp[g] = s;
    }
}

// one thread per entry of one stage of one product (blockIdx.y = stage,
// blockIdx.z = product); scatter (col, value) to its merged position
template <class S>
__global__ void k_merge_scatter(const MergeProb* __restrict__ mp, const int64_t* __restrict__ trp,
                                int32_t* __restrict__ tcol, typename S::Out* __restrict__ tval) {
    const MergeProb& M = mp[blockIdx.z];
    const int s = blockIdx.y;
    if (s >= M.nparts) return;
    const int64_t* rps = M.rp[s];
    const int64_t e_end = ld_i64(rps + M.nrows);   // partials may be row views:
    for (int64_t e = ld_i64(rps) + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e_end;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = row_of(rps, M.nrows, e);
        const int32_t c = ld_i32(M.col[s] + e);
        int64_t pos = e - ld_i64(rps + i);
        for (int t = 0; t < M.nparts; ++t) {
            if (t == s) continue;
            const int64_t a = ld_i64(M.rp[t] + i), b = ld_i64(M.rp[t] + i + 1);
            pos += lower_pos(M.col[t], a, b, c, t < s) - a;
        }
        const int64_t at = trp[M.row_base + i] + pos;
        tcol[at] = c;
        if constexpr (S::kVal) tval[at] = reinterpret_cast<const typename S::Out*>(M.val[s])[e];
    }
}

// warp per flat row: number of distinct columns (heads of runs)
__global__ void k_merge_count(const MergeProb* __restrict__ mp, int nprob, int64_t R,
                              const int64_t* __restrict__ trp, const int32_t* __restrict__ tcol,
                              int64_t* cnt) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); g < R; g += nw) {
        const int64_t a = trp[g], b = trp[g] + (trp[g + 1] - trp[g]);
        int64_t c = 0;
        for (int64_t q = a + lane; q < b; q += 32) c += (q == a || tcol[q] != tcol[q - 1]) ? 1 : 0;
        c = warp_sum(c);
        if (lane == 0) cnt[g] = c;
    }
    (void)mp;
    (void)nprob;
}

// warp per flat row: heads fold their run in stage order and write at their rank
template <class S>
__global__ void k_merge_write(const MergeProb* __restrict__ mp, int nprob, int64_t R,
                              const int64_t* __restrict__ trp, const int32_t* __restrict__ tcol,
                              const typename S::Out* __restrict__ tval, DevStatus* st) {
    using Out = typename S::Out;
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); g < R; g += nw) {
        const MergeProb& M = mp[nprob == 1 ? 0 : find_merge_prob(mp, nprob, g)];
        const int64_t i = g - M.row_base;
        const int64_t a = trp[g], b = trp[g + 1];
        const int64_t off = M.c_rp[i], n = M.c_rp[i + 1] - M.c_rp[i];
        int64_t rank = 0;
        for (int64_t q0 = a; q0 < b; q0 += 32) {   // warp-uniform
            const int64_t q = q0 + lane;
            const bool head = q < b && (q == a || tcol[q] != tcol[q - 1]);
            const unsigned hm = __ballot_sync(kFull, head);
            if (head) {
                const int64_t r = rank + __popc(hm & ((1u << lane) - 1));
                if (r < n) {
                    const int32_t c = tcol[q];
                    M.c_col[off + r] = c;
                    if constexpr (S::kVal) {
                        Out v = tval[q];
                        for (int64_t u = q + 1; u < b && tcol[u] == c; ++u) v = S::add(v, tval[u]);
                        reinterpret_cast<Out*>(M.c_val)[off + r] = v;
                    }
                } else {
                    flag_overflow(st, g);
                }
            }
            rank += __popc(hm);
        }
    }
}


// ---- merge by rows (merges of at most kMergeBitmapCols columns) ------------------
//
// Light rows (at most 32 entries over all partials): a warp loads them, one
// per lane, sorts (column, stage) in registers and folds each run of equal
// columns in stage order.  Heavy rows: a CTA ORs the row's columns into a
// shared-memory bitmap; the prefix count of the bitmap words gives every
// column its rank in the merged row (the count is the last prefix); the
// stages are then taken in order (a barrier between stages): an entry whose
// column has not been written yet writes C at its rank, a later one folds its
// value into it with (+).  Both are deterministic: every column's value is the
// stage-order fold of the definition, as in the sequence-sort path above.

constexpr int kMergeThreads = 256;
constexpr int kClMergeHeavy = 14;   // Counters::claim slot: length of the heavy-row list

// stage of entry q of a row from the stages' inclusive prefix ends (held by
// lanes 0..nparts-1): the number of stages whose end is <= q (all lanes call)
SPG_DEV int merge_stage_of(int64_t incl, int nparts, int64_t q) {
    int s = 0;
    for (int t = 0; t < nparts; ++t) s += (__shfl_sync(kFull, incl, t) <= q) ? 1 : 0;
    return s;
}

template <class S, bool kWrite>
__global__ void __launch_bounds__(256)
    k_merge_light(const MergeProb* __restrict__ mp, int nprob, int64_t R, int64_t* cnt,
                  int32_t* heavy, Counters* ctr, DevStatus* st) {
    using Out = typename S::Out;
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); g < R; g += nw) {
        const MergeProb& M = mp[nprob == 1 ? 0 : find_merge_prob(mp, nprob, g)];
        const int64_t i = g - M.row_base;
        int64_t a = 0, len = 0;
        if (lane < M.nparts) {
            a = ld_i64(M.rp[lane] + i);
            len = ld_i64(M.rp[lane] + i + 1) - a;
        }
        const int64_t incl = warp_incl_scan(len);
        const int64_t total = __shfl_sync(kFull, incl, 31);
        if (total > 32) {   // heavy row: listed by the count call, merged by k_merge_heavy
            if (!kWrite && lane == 0) heavy[atomicAdd(&ctr->claim[kClMergeHeavy], 1)] = (int32_t)g;
            continue;
        }
        if (total == 0) {
            if (!kWrite && lane == 0) cnt[g] = 0;
            continue;
        }
        // lane q < total takes entry q of the row (stages in order, columns in order)
        const int s = merge_stage_of(incl, M.nparts, lane);
        const int64_t ex = __shfl_sync(kFull, incl - len, s & 31);
        const int64_t as = __shfl_sync(kFull, a, s & 31);
        uint64_t key = ~0ull;
        Out v{};
        if (lane < total) {
            const int64_t q = as + (lane - ex);
            const int32_t c = ld_i32(M.col[s] + q);
            key = ((uint64_t)(uint32_t)c << 9) | ((uint64_t)s << 5) | (uint64_t)lane;
            if constexpr (kWrite && S::kVal) v = reinterpret_cast<const Out*>(M.val[s])[q];
        }
        // ascending bitonic sort of the keys (column, stage, source lane)
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                const uint64_t o = __shfl_xor_sync(kFull, key, j);
                const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
                key = keep_min ? (o < key ? o : key) : (o > key ? o : key);
            }
        }
        const bool valid = key != ~0ull;
        const uint32_t col = (uint32_t)(key >> 9);
        const uint32_t prev = __shfl_up_sync(kFull, col, 1);
        const bool head = valid && (lane == 0 || prev != col);
        const unsigned hm = __ballot_sync(kFull, head);
        if constexpr (!kWrite) {
            if (lane == 0) cnt[g] = __popc(hm);
        } else {
            // the values in sorted order, then each run folded left to right
            const Out sv = shfl_words<0>(v, (int)(key & 31u));
            Out acc = sv;
            bool run = head;
            for (int d = 1; d < kMaxStages; ++d) {   // a run holds at most one entry per stage
                const Out nv = shfl_words<2>(sv, d);
                const uint32_t nc = __shfl_down_sync(kFull, col, d);
                const uint64_t nk = __shfl_down_sync(kFull, key, d);
                run = run && lane + d < 32 && nk != ~0ull && nc == col;
                if constexpr (S::kVal) {
                    if (run) acc = S::add(acc, nv);
                }
                if (!__any_sync(kFull, run)) break;
            }
            const int64_t off = M.c_rp[i], n = M.c_rp[i + 1] - off;
            if (head) {
                const int r = __popc(hm & ((1u << lane) - 1u));
                if (r < n) {
                    M.c_col[off + r] = (int32_t)col;
                    if constexpr (S::kVal) reinterpret_cast<Out*>(M.c_val)[off + r] = acc;
                } else {
                    flag_overflow(st, g);
                }
            }
        }
    }
}

// shared-memory bytes of k_merge_heavy for rows of `ncols` columns
__host__ __device__ inline size_t merge_heavy_smem(int64_t ncols) {
    const size_t words = (size_t)((ncols + 31) >> 5);
    return (words + 1) * 8 + words * 4;
}

template <class S, bool kWrite>
__global__ void __launch_bounds__(kMergeThreads)
    k_merge_heavy(const MergeProb* __restrict__ mp, int nprob, const int32_t* __restrict__ heavy,
                  const Counters* __restrict__ ctr, int64_t* cnt, DevStatus* st) {
    using Out = typename S::Out;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_wsum[kMergeThreads / 32];
    // the row's entries in every stage: start in the stage's partial, and
    // offset in the stages' concatenation (s_off[nparts] = all entries)
    __shared__ int64_t s_a[kMaxStages], s_off[kMaxStages + 1];
    const int tid = threadIdx.x, lane = lane_id(), wid = warp_id();
    constexpr int nwarps = kMergeThreads / 32;
    constexpr int kU = 4;   // entry loads in flight per thread
    const int nheavy = ctr->claim[kClMergeHeavy];
    for (int r = blockIdx.x; r < nheavy; r += gridDim.x) {
        const int64_t g = heavy[r];
        const MergeProb& M = mp[nprob == 1 ? 0 : find_merge_prob(mp, nprob, g)];
        const int64_t i = g - M.row_base;
        const int words = (int)((M.ncols + 31) >> 5);
        // (word, prefix) pairs of the row's bitmap, then the written bits
        uint2* pw = reinterpret_cast<uint2*>(smem_raw);
        uint32_t* done = reinterpret_cast<uint32_t*>(smem_raw + ((size_t)words + 1) * 8);
        const int np = M.nparts;
        if (wid == 0) {   // every stage's row bounds at once (np <= 32)
            int64_t a = 0, len = 0;
            if (lane < np) {
                a = ld_i64(M.rp[lane] + i);
                len = ld_i64(M.rp[lane] + i + 1) - a;
                s_a[lane] = a;
            }
            const int64_t incl = warp_incl_scan(len);
            if (lane < np) s_off[lane + 1] = incl;
            if (lane == 0) s_off[0] = 0;
        }
        for (int w = tid; w < words; w += kMergeThreads) {
            pw[w] = make_uint2(0u, 0u);
            if (kWrite) done[w] = 0u;
        }
        __syncthreads();
        // bitmap of the row's columns (no barrier between stages: the OR does
        // not depend on their order), kU loads in flight per thread
        for (int s = 0; s < np; ++s) {
            const int64_t a = s_a[s], len = s_off[s + 1] - s_off[s];
            for (int64_t j0 = tid; j0 < len; j0 += kU * kMergeThreads) {
                int32_t c[kU];
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    const int64_t j = j0 + (int64_t)u * kMergeThreads;
                    c[u] = j < len ? ld_i32(M.col[s] + a + j) : -1;
                }
#pragma unroll
                for (int u = 0; u < kU; ++u) {
                    if (c[u] < 0) continue;
                    atomicOr(&pw[c[u] >> 5].x, 1u << (c[u] & 31));   // no read of the word first
                }
            }
        }
        __syncthreads();
        // prefix count of the words (contiguous words per thread)
        const int wpt = (words + kMergeThreads - 1) / kMergeThreads;
        const int w0 = tid * wpt;
        int mine = 0;
        for (int j = 0; j < wpt; ++j)
            if (w0 + j < words) mine += __popc(pw[w0 + j].x);
        const int incl = warp_incl_scan(mine);
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const int x = lane < nwarps ? s_wsum[lane] : 0;
            const int xi = warp_incl_scan(x);
            if (lane < nwarps) s_wsum[lane] = xi - x;
            if (!kWrite && lane == 31) cnt[g] = xi;   // lanes >= nwarps add nothing
        }
        __syncthreads();
        if constexpr (kWrite) {
            int run = s_wsum[wid] + incl - mine;
            for (int j = 0; j < wpt; ++j)
                if (w0 + j < words) {
                    pw[w0 + j].y = (uint32_t)run;
                    run += __popc(pw[w0 + j].x);
                }
            __syncthreads();
            const int64_t off = M.c_rp[i], n = M.c_rp[i + 1] - off;
            Out* cv = reinterpret_cast<Out*>(M.c_val);
            for (int s = 0; s < np; ++s) {   // stage order: (+) folds left to right
                const int64_t a = s_a[s], len = s_off[s + 1] - s_off[s];
                const Out* sv = reinterpret_cast<const Out*>(M.val[s]);
                for (int64_t j0 = tid; j0 < len; j0 += kU * kMergeThreads) {
                    int32_t c[kU];
                    Out x[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {   // the loads first, kU in flight
                        const int64_t j = j0 + (int64_t)u * kMergeThreads;
                        c[u] = -1;
                        if (j < len) {
                            c[u] = ld_i32(M.col[s] + a + j);
                            if constexpr (S::kVal) x[u] = sv[a + j];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        if (c[u] < 0) continue;
                        const uint2 e = pw[c[u] >> 5];
                        const uint32_t bit = 1u << (c[u] & 31);
                        const int64_t rk = (int64_t)e.y + __popc(e.x & (bit - 1u));
                        if (rk >= n) {
                            flag_overflow(st, g);
                            continue;
                        }
                        if (!(done[c[u] >> 5] & bit)) {   // the first stage that holds this column
                            M.c_col[off + rk] = c[u];
                            if constexpr (S::kVal) cv[off + rk] = x[u];
                            atomicOr(done + (c[u] >> 5), bit);
                        } else {
                            if constexpr (S::kVal) cv[off + rk] = S::add(cv[off + rk], x[u]);
                        }
                    }
                }
                __syncthreads();   // this stage's values land before the next stage folds into them
            }
        }
        __syncthreads();
    }
}

// ---- column split --------------------------------------------------------------

// warp per row: counts of each part's columns in the row -> prp[p][i + 1]
__global__ void k_split_count(DCsr M, int nparts, const int32_t* __restrict__ cuts,
                              int64_t* prp, int64_t stride) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < M.nrows; i += nw) {
        const int64_t a = ld_i64(M.rp + i), b = ld_i64(M.rp + i + 1);
        for (int p = lane; p < nparts; p += 32) {
            const int64_t lo = lower_pos(M.col, a, b, cuts[p], false);
            const int64_t hi = lower_pos(M.col, a, b, cuts[p + 1], false);
            prp[p * stride + i] = hi - lo;
        }
    }
}

// warp per row: copy each part's segment with local column ids
__global__ void k_split_copy(DCsr M, int nparts, const int32_t* __restrict__ cuts,
                             const int64_t* __restrict__ prp, int64_t stride,
                             const int64_t* __restrict__ part_base, int32_t* pcol, char* pval,
                             int vbytes) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < M.nrows; i += nw) {
        const int64_t a = ld_i64(M.rp + i), b = ld_i64(M.rp + i + 1);
        for (int p = 0; p < nparts; ++p) {
            const int64_t lo = lower_pos(M.col, a, b, cuts[p], false);
            const int64_t hi = lower_pos(M.col, a, b, cuts[p + 1], false);
            const int64_t dst = part_base[p] + prp[p * stride + i];
            for (int64_t q = lo + lane; q < hi; q += 32) {
                pcol[dst + (q - lo)] = ld_i32(M.col + q) - cuts[p];
                for (int k = 0; k < vbytes; ++k)
                    pval[(dst + (q - lo)) * vbytes + k] = reinterpret_cast<const char*>(M.val)[q * vbytes + k];
            }
        }
    }
}

// part_base[p] = sum of the earlier parts' nnz
__global__ void k_split_bases(const int64_t* prp, int64_t stride, int64_t nrows, int nparts,
                              int64_t* base) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t s = 0;
        for (int p = 0; p < nparts; ++p) {
            base[p] = s;
            s += prp[p * stride + nrows];
        }
        base[nparts] = s;
    }
}

// C row pointers of each merge from the flat scanned counts, and its nnz
__global__ void k_merge_rowptr(const MergeProb* __restrict__ mp, const int64_t* __restrict__ cnt,
                               Counters* ctr) {
    const MergeProb& M = mp[blockIdx.y];
    const int64_t b = cnt[M.row_base];
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= M.nrows;
         i += (int64_t)gridDim.x * blockDim.x)
        M.c_rp[i] = cnt[M.row_base + i] - b;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctr->nnz[blockIdx.y] = cnt[M.row_base + M.nrows] - b;
}

__global__ void k_write_merge_probs(MergeProbTable tab, int nprob, MergeProb* dst) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nprob) dst[i] = tab.p[i];
}

// ---- launchers -------------------------------------------------------------------

struct MergeLaunch {
    const MergeWs* w;
    int nprob;
    int64_t R;
    int64_t max_part_nnz;
    int max_parts;
    bool count_only;
    const DevInfo* dev;
    cudaStream_t st;
    int64_t max_ncols = 0;
    cudaError_t err = cudaSuccess;
    template <class S> void row_path() {
        int64_t blocks = (R + 7) / 8;
        if (blocks > (int64_t)dev->sms * 16) blocks = (int64_t)dev->sms * 16;
        if (blocks < 1) blocks = 1;
        const size_t smem = merge_heavy_smem(max_ncols);
        // as many CTAs as fit the SMs (one heavy row each at a time)
        auto grid_of = [&](const void* fn) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kMergeThreads, smem);
            return (per_sm < 1 ? 1 : per_sm) * dev->sms;
        };
        if (count_only) {
            k_merge_light<S, false><<<(unsigned)blocks, 256, 0, st>>>(w->probs, nprob, R, w->cnt,
                                                                       w->heavy, w->ctr, w->status);
            err = cudaFuncSetAttribute(k_merge_heavy<S, false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return;
            k_merge_heavy<S, false><<<grid_of((const void*)k_merge_heavy<S, false>), kMergeThreads,
                                      smem, st>>>(w->probs, nprob, w->heavy, w->ctr, w->cnt,
                                                  w->status);
        } else {
            k_merge_light<S, true><<<(unsigned)blocks, 256, 0, st>>>(w->probs, nprob, R, w->cnt,
                                                                      w->heavy, w->ctr, w->status);
            err = cudaFuncSetAttribute(k_merge_heavy<S, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (err != cudaSuccess) return;
            k_merge_heavy<S, true><<<grid_of((const void*)k_merge_heavy<S, true>), kMergeThreads,
                                     smem, st>>>(w->probs, nprob, w->heavy, w->ctr, w->cnt,
                                                 w->status);
        }
        count_launch(*dev, 2);
        err = cudaGetLastError();
    }
    template <class S> void operator()() {
        using Out = typename S::Out;
        if (w->row_path) {
            row_path<S>();
            return;
        }
        Out* tval = reinterpret_cast<Out*>(w->tval);
        if (count_only) {
            int64_t gx = (max_part_nnz + 255) / 256;
            if (gx < 1) gx = 1;
            if (gx > (int64_t)dev->sms * 8) gx = (int64_t)dev->sms * 8;
            k_merge_scatter<S><<<dim3((unsigned)gx, max_parts, nprob), 256, 0, st>>>(
                w->probs, w->trp, w->tcol, tval);
            count_launch(*dev);
            int64_t blocks = (R + 7) / 8;
            if (blocks > (int64_t)dev->sms * 16) blocks = (int64_t)dev->sms * 16;
            if (blocks < 1) blocks = 1;
            k_merge_count<<<(unsigned)blocks, 256, 0, st>>>(w->probs, nprob, R, w->trp, w->tcol,
                                                           w->cnt);
            count_launch(*dev);
        } else {
            int64_t blocks = (R + 7) / 8;
            if (blocks > (int64_t)dev->sms * 16) blocks = (int64_t)dev->sms * 16;
            if (blocks < 1) blocks = 1;
            k_merge_write<S><<<(unsigned)blocks, 256, 0, st>>>(w->probs, nprob, R, w->trp, w->tcol,
                                                              tval, w->status);
            count_launch(*dev);
        }
        err = cudaGetLastError();
    }
};

cudaError_t launch_merge_count(int sr, const MergeProbTable& tab, int nprob, int64_t R,
                               int64_t max_part_nnz, int max_parts, int64_t max_ncols,
                               const MergeWs& w, const DevInfo& dev, cudaStream_t st) {
    mark_stage(dev, kStBegin, st);
    k_write_merge_probs<<<1, kMaxProb, 0, st>>>(tab, nprob, w.probs);
    count_launch(dev);
    cudaError_t e = cudaSuccess;
    if (!w.row_path) {
        if (R > 0) {
            int64_t blocks = (R + 255) / 256;
            if (blocks > (int64_t)dev.sms * 8) blocks = (int64_t)dev.sms * 8;
            k_merge_rowlen<<<(unsigned)blocks, 256, 0, st>>>(w.probs, nprob, R, w.trp);
            count_launch(dev);
        }
        e = launch_scan_inplace(w.trp, R, w.part, st);   // trp -> row starts
        if (e != cudaSuccess) return e;
        count_launch(dev, R > 0 ? 3 : 0);
    }
    MergeLaunch f{&w, nprob, R, max_part_nnz, max_parts, true, &dev, st, max_ncols};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    if (f.err != cudaSuccess) return f.err;
    e = launch_scan_inplace(w.cnt, R, w.part, st);                // cnt -> C row starts (flat)
    count_launch(dev, R > 0 ? 3 : 0);
    mark_stage(dev, kStMerge, st);
    return e;
}

cudaError_t launch_merge_rowptr(const MergeWs& w, int nprob, const DevInfo& dev, cudaStream_t st) {
    k_merge_rowptr<<<dim3(64, nprob), 256, 0, st>>>(w.probs, w.cnt, w.ctr);
    count_launch(dev);
    return cudaGetLastError();
}

MergeWs merge_ws_layout(void* base, int64_t R, int64_t T, int out_bytes, int64_t max_ncols) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    char* b = (char*)base;
    MergeWs w{};
    // merges of at most kMergeBitmapCols columns take the row kernels, which
    // need no copy of the partials' entries
    w.row_path = max_ncols <= kMergeBitmapCols;
    const int64_t Tt = w.row_path ? 0 : T;
    size_t o = 0;
    w.status = (DevStatus*)(b + o);  o = al(o + sizeof(DevStatus));
    w.ctr = (Counters*)(b + o);      o = al(o + sizeof(Counters));
    w.probs = (MergeProb*)(b + o);   o = al(o + sizeof(MergeProb) * kMaxMerge);
    w.trp = (int64_t*)(b + o);       o = al(o + (w.row_path ? 0 : sizeof(int64_t) * (size_t)(R + 1)));
    w.cnt = (int64_t*)(b + o);       o = al(o + sizeof(int64_t) * (size_t)(R + 1));
    w.heavy = (int32_t*)(b + o);     o = al(o + (w.row_path ? sizeof(int32_t) * (size_t)R : 0));
    w.tcol = (int32_t*)(b + o);      o = al(o + sizeof(int32_t) * (size_t)Tt);
    w.tval = (void*)(b + o);         o = al(o + (size_t)out_bytes * (size_t)Tt);
    w.part = (int64_t*)(b + o);      o = al(o + sizeof(int64_t) * (size_t)scan_parts_needed(R));
    w.total = o;
    return w;
}

cudaError_t launch_merge_write(int sr, const MergeProbTable& tab, int nprob, int64_t R,
                               int64_t max_ncols, const MergeWs& w, const DevInfo& dev,
                               cudaStream_t st) {
    mark_stage(dev, kStBegin, st);
    k_write_merge_probs<<<1, kMaxProb, 0, st>>>(tab, nprob, w.probs);
    count_launch(dev);
    MergeLaunch f{&w, nprob, R, 0, 0, false, &dev, st, max_ncols};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    mark_stage(dev, kStMerge, st);
    return f.err;
}

cudaError_t launch_split_columns(const DCsr& M, int nparts, const int32_t* cuts_dev,
                                 int64_t* prp, int64_t* part_base_dev, int32_t* pcol, void* pval,
                                 int vbytes, int64_t* part, const DevInfo& dev, cudaStream_t st) {
    const int64_t stride = M.nrows + 1;
    int64_t blocks = (M.nrows + 7) / 8;
    if (blocks > (int64_t)dev.sms * 16) blocks = (int64_t)dev.sms * 16;
    if (blocks < 1) blocks = 1;
    if (M.nrows > 0) k_split_count<<<(unsigned)blocks, 256, 0, st>>>(M, nparts, cuts_dev, prp, stride);
    for (int p = 0; p < nparts; ++p) {
        cudaError_t e = launch_scan_inplace(prp + p * stride, M.nrows, part, st);
        if (e != cudaSuccess) return e;
    }
    // part_base[p] = sum of earlier parts' nnz (small: one thread)
    k_split_bases<<<1, 1, 0, st>>>(prp, stride, M.nrows, nparts, part_base_dev);
    if (M.nrows > 0)
        k_split_copy<<<(unsigned)blocks, 256, 0, st>>>(M, nparts, cuts_dev, prp, stride,
                                                        part_base_dev, pcol, (char*)pval, vbytes);
    return cudaGetLastError();
}

}  // namespace spg
