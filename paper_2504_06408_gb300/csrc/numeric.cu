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
#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

SPG_DEV int64_t dev_next_pow2_n(int64_t x) {
    return x <= 1 ? 1 : (int64_t)1 << (64 - __clzll(x - 1));
}

SPG_DEV int num_tier(int64_t nnz, const Tuning& t) {
    if (nnz == 0) return kTierEmpty;
    if (nnz <= t.num_warp_max_nnz) return kTierWarp;
    if (nnz <= t.num_block_max_nnz) return kTierBlock;
    return kTierDense;
}

SPG_DEV int num_bin_key(int tier, int64_t work) {
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
                                                  const int64_t* __restrict__ ub, Counters* ctr) {
    __shared__ int s_hist[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_hist[b] = 0;
    __syncthreads();
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x) {
        const Prob* P;
        const int64_t n = row_nnz(probs, nprob, g, &P);
        atomicAdd(&s_hist[num_bin_key(num_tier(n, t), ub[g])], 1);
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
                                                      Counters* ctr, int32_t* rows) {
    __shared__ int s_cnt[kNumBins];
    __shared__ int s_base[kNumBins];
    for (int b = threadIdx.x; b < kNumBins; b += blockDim.x) s_cnt[b] = 0;
    __syncthreads();
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int key = -1, rank = 0;
    if (g < R) {
        const Prob* P;
        const int64_t n = row_nnz(probs, nprob, g, &P);
        key = num_bin_key(num_tier(n, t), ub[g]);
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
    const int32_t* bcol;
    const typename S::In* bval;
    DevStatus* st;
    int64_t g;
    SPG_DEV void operator()(int64_t q, typename S::In a, bool valid) {
        if (!valid) return;
        const int s = hash_slot_of(keys, shift, mask, ld_i32(bcol + q));
        if (s < 0) {
            flag_overflow(st, g);
            return;
        }
        if constexpr (S::kVal) S::acc(vals + s, a, __ldg(bval + q));
    }
};

template <class S>
struct DenseAccOp {
    typename S::Slot* vals;
    uint32_t* bm;
    int32_t lo;
    const int32_t* bcol;
    const typename S::In* bval;
    SPG_DEV void operator()(int64_t q, typename S::In a, bool valid) {
        if (!valid) return;
        const int32_t c = ld_i32(bcol + q) - lo;
        if constexpr (S::kBitmap) atomicOr(bm + (c >> 5), 1u << (c & 31));
        if constexpr (S::kVal) S::acc(vals + c, a, __ldg(bval + q));
    }
};

template <class S>
SPG_DEV void write_entry(const Prob& P, int64_t pos, int32_t col, const typename S::Slot& v) {
    P.c_col[pos] = col;
    if constexpr (S::kVal) reinterpret_cast<typename S::Out*>(P.c_val)[pos] = S::out(v);
}

template <class S>
SPG_DEV size_t hash_region_bytes(int T) {
    // vals[T] | keys[T] | sort buffer[T/2], 16-byte aligned
    size_t b = (size_t)T * sizeof(typename S::Slot) + (size_t)T * 4 + (size_t)(T / 2) * 4;
    return (b + 15) & ~(size_t)15;
}

// ---- warp tier ------------------------------------------------------------------

template <class S>
__global__ void __launch_bounds__(kWarpTierWarps * 32)
    k_num_warp(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
               const Counters* __restrict__ ctr, DevStatus* st, int Tw) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char* base = smem_raw + hash_region_bytes<S>(Tw) * warp_id();
    Slot* vals = reinterpret_cast<Slot*>(base);
    int32_t* keys = reinterpret_cast<int32_t*>(base + (size_t)Tw * sizeof(Slot));
    int32_t* sbuf = keys + Tw;
    const int lane = lane_id();
    const int beg = ctr->num_bin_off[kTierWarp * kSubBins];
    const int end = ctr->num_bin_off[(kTierWarp + 1) * kSubBins];
    const int stride = gridDim.x * kWarpTierWarps;
    const Slab single{0, 0, true, true, true, nullptr};
    for (int r = beg + blockIdx.x * kWarpTierWarps + warp_id(); r < end; r += stride) {
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
        HashAccOp<S> op{keys, vals, shift, (uint32_t)(T - 1), P.B.col,
                        reinterpret_cast<const In*>(P.B.val), st, g};
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
                Counters* ctr, DevStatus* st, int Tb) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw + (size_t)Tb * sizeof(Slot));
    int32_t* sbuf = keys + Tb;
    __shared__ int s_row, s_next, s_m;
    const int lane = lane_id();
    const int beg = ctr->num_bin_off[kTierBlock * kSubBins];
    const int end = ctr->num_bin_off[(kTierBlock + 1) * kSubBins];
    const Slab single{0, 0, true, true, true, nullptr};
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = beg + atomicAdd(&ctr->claim[2], 1);
            s_next = 0;
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
        int T = (int)dev_next_pow2_n(2 * (int64_t)n);
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
        HashAccOp<S> op{keys, vals, shift, (uint32_t)(T - 1), P.B.col,
                        reinterpret_cast<const In*>(P.B.val), st, g};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        for (;;) {
            int c = 0;
            if (lane == 0) c = atomicAdd(&s_next, 1);
            c = __shfl_sync(kFull, c, 0);
            const int64_t p0 = a0 + (int64_t)c * 32;
            if (p0 >= a1) break;
            chunk_products<In, S::kVal>(P.A, P.B, p0, a1, 0, single, op);
        }
        __syncthreads();
        // compact occupied keys (order irrelevant: sorted next)
        for (int s0 = warp_id() * 32; s0 < T; s0 += blockDim.x) {
            const int32_t k = keys[s0 + lane];
            const unsigned occ = __ballot_sync(kFull, k != kEmptyKey);
            int b = 0;
            if (lane == 0 && occ) b = atomicAdd(&s_m, __popc(occ));
            b = __shfl_sync(kFull, b, 0);
            const int pos = b + __popc(occ & ((1u << lane) - 1));
            if (k != kEmptyKey && pos < T / 2) sbuf[pos] = k;
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

template <class S>
__host__ __device__ inline size_t dense_val_bytes(int64_t slab_cols) {
    return S::kVal ? (size_t)slab_cols * sizeof(typename S::Slot) : 0;
}

template <class S>
__global__ void __launch_bounds__(kBlockThreads)
    k_num_dense(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                Counters* ctr, DevStatus* st, int32_t* cursor, int slab_cols) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);
    uint32_t* bm = reinterpret_cast<uint32_t*>(smem_raw + dense_val_bytes<S>(slab_cols));
    int32_t* chunk_off = reinterpret_cast<int32_t*>(bm + slab_cols / 32);
    __shared__ int s_row, s_next;
    __shared__ int64_t s_written;
    __shared__ int s_slab_total;
    const int lane = lane_id(), wid = warp_id(), nwarps = blockDim.x >> 5;
    const int beg = ctr->num_bin_off[kTierDense * kSubBins];
    const int end = ctr->num_bin_off[(kTierDense + 1) * kSubBins];
    for (;;) {
        if (threadIdx.x == 0) {
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
        for (int s = 0; s < nslabs; ++s) {
            const int32_t lo = (int32_t)((int64_t)s * slab_cols);
            const int64_t hi64 = (int64_t)lo + slab_cols < ncols ? (int64_t)lo + slab_cols : ncols;
            const int32_t hi = (int32_t)hi64;
            const int width = hi - lo;
            const int words = (width + 31) >> 5;
            if constexpr (S::kVal)
                for (int c = threadIdx.x; c < width; c += blockDim.x) vals[c] = S::empty();
            if constexpr (S::kBitmap)
                for (int w = threadIdx.x; w < words; w += blockDim.x) bm[w] = 0u;
            if (threadIdx.x == 0) s_next = 0;
            __syncthreads();
            const Slab slab{lo, hi, s == 0, s == nslabs - 1, nslabs == 1, cursor};
            DenseAccOp<S> op{vals, bm, lo, P.B.col, reinterpret_cast<const In*>(P.B.val)};
            for (;;) {
                int c = 0;
                if (lane == 0) c = atomicAdd(&s_next, 1);
                c = __shfl_sync(kFull, c, 0);
                const int64_t p0 = a0 + (int64_t)c * 32;
                if (p0 >= a1) break;
                chunk_products<In, S::kVal>(P.A, P.B, p0, a1, P.nnz_base + p0, slab, op);
            }
            __syncthreads();
            // count per 1024-column chunk (and build the bitmap if values mark presence)
            const int nchunks = (width + 1023) >> 10;
            for (int ch = wid; ch < nchunks; ch += nwarps) {
                uint32_t bits = 0;
                if constexpr (S::kBitmap) {
                    const int w = ch * 32 + lane;
                    bits = w < words ? bm[w] : 0u;
                } else {
                    for (int t = 0; t < 32; ++t) {
                        const int c = (ch * 32 + t) * 32 + lane;
                        const unsigned m = __ballot_sync(kFull, c < width && S::touched(vals[c]));
                        if (lane == t) bits = m;
                    }
                    const int w = ch * 32 + lane;
                    if (w < words) bm[w] = bits;
                }
                const int cc = warp_sum(__popc(bits));
                if (lane == 0) chunk_off[ch] = cc;
            }
            __syncthreads();
            if (wid == 0) {   // exclusive scan of chunk counts (nchunks <= 64)
                const int v0 = 2 * lane < nchunks ? chunk_off[2 * lane] : 0;
                const int v1 = 2 * lane + 1 < nchunks ? chunk_off[2 * lane + 1] : 0;
                const int incl = warp_incl_scan(v0 + v1);
                const int ex = incl - v0 - v1;
                if (2 * lane < nchunks) chunk_off[2 * lane] = ex;
                if (2 * lane + 1 < nchunks) chunk_off[2 * lane + 1] = ex + v0;
                if (lane == 31) s_slab_total = incl;
            }
            __syncthreads();
            const int64_t slab_base = off + s_written;
            for (int ch = wid; ch < nchunks; ch += nwarps) {
                int64_t pos = slab_base + chunk_off[ch];
                for (int t = 0; t < 32; ++t) {
                    const int w = ch * 32 + t;
                    const uint32_t bits = w < words ? bm[w] : 0u;
                    if ((bits >> lane) & 1u) {
                        const int c = w * 32 + lane;
                        const int64_t at = pos + __popc(bits & ((1u << lane) - 1));
                        if (at < off + n) write_entry<S>(P, at, lo + c, vals[c]);
                        else flag_overflow(st, g);   // counts disagree: never write past the row
                    }
                    pos += __popc(bits);
                }
            }
            __syncthreads();
            if (threadIdx.x == 0) s_written += s_slab_total;
            __syncthreads();
        }
        if (threadIdx.x == 0 && s_written != n) flag_overflow(st, g);
        __syncthreads();
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
           ((size_t)slab_cols / 1024 + 1) * 4;
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

struct NumericLaunch {
    const WsPtrs* w;
    int nprob;
    const Tuning* t;
    int64_t max_ncols;
    const DevInfo* dev;
    cudaStream_t st;
    cudaError_t err = cudaSuccess;
    template <class S> void operator()() {
        cudaError_t e;
        {   // dense tier
            int64_t slab = t->dense_slab_cols;
            if (slab > max_ncols) slab = (max_ncols + 1023) / 1024 * 1024;
            if (slab < 1024) slab = 1024;
            const size_t smem = num_dense_bytes<S>(slab);
            e = cudaFuncSetAttribute(k_num_dense<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            const int grid = occupancy_grid((const void*)k_num_dense<S>, kBlockThreads, smem, *dev);
            k_num_dense<S><<<grid, kBlockThreads, smem, st>>>(w->probs, nprob, w->rows_num, w->ctr,
                                                              w->status, w->cursor, (int)slab);
        }
        {   // block tier
            int64_t T = next_pow2(2 * t->num_block_max_nnz);
            if (T < 32) T = 32;
            const size_t smem = num_block_bytes<S>(*t);
            e = cudaFuncSetAttribute(k_num_block<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            const int grid = occupancy_grid((const void*)k_num_block<S>, kBlockThreads, smem, *dev);
            k_num_block<S><<<grid, kBlockThreads, smem, st>>>(w->probs, nprob, w->rows_num, w->ctr,
                                                              w->status, (int)T);
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
                                                                   w->ctr, w->status, (int)T);
        }
        err = cudaGetLastError();
    }
};

cudaError_t launch_numeric(int sr, const WsPtrs& w, int nprob, int64_t R, const Tuning& t,
                           int64_t max_ncols, const DevInfo& dev, cudaStream_t st) {
    if (R == 0) return cudaSuccess;
    // reset numeric bins and claims
    cudaMemsetAsync(w.ctr->num_bin_count, 0, sizeof(w.ctr->num_bin_count), st);
    cudaMemsetAsync(&w.ctr->claim[2], 0, 2 * sizeof(int32_t), st);
    int64_t blocks = (R + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_num_hist<<<(unsigned)blocks, 256, 0, st>>>(w.probs, nprob, R, t, w.ub, w.ctr);
    k_num_bin_offsets<<<1, 32, 0, st>>>(w.ctr);
    k_num_scatter<<<(unsigned)((R + 1023) / 1024), 1024, 0, st>>>(w.probs, nprob, R, t, w.ub,
                                                                   w.ctr, w.rows_num);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    NumericLaunch f{&w, nprob, &t, max_ncols, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    return f.err;
}

}  // namespace spg
