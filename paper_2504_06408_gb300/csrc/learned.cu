// Learned-sizing path: rows whose output size is predicted small skip the
// symbolic phase (the paper sizes every row by a symbolic pass, Section 2.1
// Gustavson; this path keeps that pass only for the rows that need it).
//
// plan      per row a capacity cap_i: the exact bound min(ub_i, ncols) when
//           ub_i is small or no model is given, else
//           min(bound, ceil(ub_i * r_i * margin)) with r_i = sigmoid(z_i) from
//           the MLP.  Rows whose capacity exceeds the hash tiers' limit take
//           the exact path.  Staging offsets = exclusive scan of the caps.
// direct    each learned row accumulates into a shared-memory hash table of
//           2 cap_i (rounded up to a power of two) slots; a row whose distinct
//           columns exceed cap_i aborts at the first extra insert and is
//           re-routed to the exact path.  A finished row is sorted and written
//           to its staging slice.
// exact     the plain symbolic kernels on the exact rows only (skip mask);
//           then the counts of all rows are scanned into C's row pointers.
// numeric   learned rows are copied from staging into C, exact rows run the
//           plain numeric kernels (skip mask).  C is the plain path's C.
#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

constexpr uint8_t kRouteLearned = 0, kRouteExact = 1;

// claim[] slots used here (the plain kernels use 0..4, 7 and 15)
constexpr int kClWarpRows = 8, kClBlockRows = 9, kClBlockNext = 10, kClOverflow = 11,
              kClTinyRows = 12;
constexpr int kTinyRows = 1;   // tiny rows per warp at a time (more costs registers)

__global__ void k_learned_caps(const Prob* __restrict__ probs, int nprob, int64_t R,
                               const float* __restrict__ z, float margin, int64_t exact_max,
                               int64_t learned_max, const int64_t* __restrict__ ub,
                               int64_t* __restrict__ soff, uint8_t* __restrict__ route,
                               int64_t* __restrict__ cnt) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x) {
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t u = ub[g];
        const int64_t lim = u < P.B.ncols ? u : P.B.ncols;
        int64_t c = lim;
        if (z && u > exact_max) {
            const float r = 1.f / (1.f + expf(-z[g]));
            const double want = ceil((double)u * (double)r * (double)margin);
            c = want < (double)lim ? (int64_t)want : lim;
            if (c < 1) c = 1;
        }
        uint8_t rt = kRouteLearned;
        if (c > learned_max) {
            rt = kRouteExact;
            c = 0;
        }
        if (u == 0) {
            rt = kRouteLearned;
            c = 0;
            cnt[g] = 0;
        }
        route[g] = rt;
        soff[g] = c;
    }
}

// Start of a learned symbolic call: the routes fixed by the plan (a row is
// learned iff it has a capacity or no products) and zero counts of empty
// rows, so that the call can be repeated after one plan.
__global__ void k_learned_reset(int64_t R, const int64_t* __restrict__ soff,
                                const int64_t* __restrict__ ub, uint8_t* __restrict__ route,
                                int64_t* __restrict__ cnt) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x) {
        const bool empty = ub[g] == 0;
        route[g] = (empty || soff[g + 1] > soff[g]) ? kRouteLearned : kRouteExact;
        if (empty) cnt[g] = 0;
    }
}

// Lists of learned rows with products: tiny rows (ub <= 32, at most 32
// entries) in tiny_rows; of the others, cap <= warp_max grows up from rows[0],
// the rest grows down from rows[R - 1].
__global__ void __launch_bounds__(1024) k_learned_bin(const Prob* __restrict__ probs, int nprob,
                                                      int64_t R, const int64_t* __restrict__ soff,
                                                      const uint8_t* __restrict__ route,
                                                      const int64_t* __restrict__ ub,
                                                      int64_t warp_max, int32_t* rows,
                                                      int32_t* tiny_rows, Counters* ctr) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int which = -1;
    if (g < R && route[g] == kRouteLearned && ub[g] > 0) {
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t na = ld_i64(P.A.rp + i + 1) - ld_i64(P.A.rp + i);
        if (ub[g] <= kTinyMax && na <= 32) which = 2;
        else which = (soff[g + 1] - soff[g]) <= warp_max ? 0 : 1;
    }
    for (int l = 0; l < 3; ++l) {
        const unsigned m = __ballot_sync(kFull, which == l);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        int base = 0;
        const int slot = l == 2 ? kClTinyRows : kClWarpRows + l;
        if (lane_id() == leader) base = atomicAdd(&ctr->claim[slot], __popc(m));
        base = __shfl_sync(kFull, base, leader);
        if (which == l) {
            const int pos = base + __popc(m & ((1u << lane_id()) - 1));
            if (l == 2) tiny_rows[pos] = (int32_t)g;
            else rows[l == 0 ? (int64_t)pos : R - 1 - pos] = (int32_t)g;
        }
    }
}

template <class S>
SPG_DEV void stage_write(void* sval, int32_t* scol, int64_t pos, int32_t col,
                         const typename S::Slot& v) {
    scol[pos] = col;
    if constexpr (S::kVal) reinterpret_cast<typename S::Out*>(sval)[pos] = S::out(v);
}

// Hash accumulation bounded by the row's capacity: the insert that would make
// the distinct count exceed cap sets *abort and the row goes to the exact
// path.  The table holds 2 cap slots or more, so probing stays short; a full
// table also aborts.
template <class S>
struct CapHashOp {
    int32_t* keys;
    typename S::Slot* vals;
    int shift;
    uint32_t mask;
    int* count;            // distinct keys inserted (shared)
    volatile int* abort;   // shared
    int cap;
    SPG_DEV void any(int32_t col, typename S::In a, typename S::In b, bool valid) {
        // (the abort flag is read only before inserting a new key)
        if (!valid) return;
        uint32_t s = hash_slot(col, shift);
        for (uint32_t n = 0;; ++n) {
            if (n > mask) {
                *abort = 1;
                return;
            }
            const int32_t cur = *(volatile int32_t*)(keys + s);
            if (cur == col) break;
            if (cur == kEmptyKey) {
                if (*abort) return;   // abandoned table: no more keys, probes stay short
                const int32_t old = atomicCAS(keys + s, kEmptyKey, col);
                if (old == kEmptyKey) {
                    if (atomicAdd(count, 1) >= cap) {
                        *abort = 1;
                        return;
                    }
                    break;
                }
                if (old == col) break;
            }
            s = (s + 1) & mask;
        }
        if constexpr (S::kVal) S::acc(vals + s, a, b);
    }
    SPG_DEV void sorted(int32_t col, typename S::In a, typename S::In b, bool valid) {
        any(col, a, b, valid);
    }
};

// vals[T] | keys[T] | sort buffer[T/2], 16-byte aligned
template <class S>
__host__ __device__ inline size_t learned_table_bytes(int T) {
    size_t b = (size_t)T * sizeof(typename S::Slot) + (size_t)T * 4 + (size_t)(T / 2) * 4;
    return (b + 15) & ~(size_t)15;
}

SPG_DEV int table_size_for(int64_t cap, int Tmax) {
    int64_t T = next_pow2(2 * cap);
    if (T < 32) T = 32;
    return T > Tmax ? Tmax : (int)T;
}

// warp per learned row of the warp list
template <class S>
__global__ void __launch_bounds__(kWarpTierWarps * 32)
    k_learned_warp(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                   const int32_t* __restrict__ tiny_rows, Counters* ctr,
                   const int64_t* __restrict__ soff, uint8_t* __restrict__ route,
                   int64_t* __restrict__ cnt, int32_t* scol, void* sval, int64_t S_entries,
                   DevStatus* st, int Tw) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_count[kWarpTierWarps], s_abort[kWarpTierWarps];
    const int lane = lane_id(), wid = warp_id();
    unsigned char* base = smem_raw + learned_table_bytes<S>(Tw) * wid;
    Slot* vals = reinterpret_cast<Slot*>(base);
    int32_t* keys = reinterpret_cast<int32_t*>(base + (size_t)Tw * sizeof(Slot));
    int32_t* sbuf = keys + Tw;
    const int end = ctr->claim[kClWarpRows];
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    for (int r = blockIdx.x * kWarpTierWarps + wid; r < end; r += gridDim.x * kWarpTierWarps) {
        const int64_t g = rows[r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t cap = soff[g + 1] - soff[g];
        if (soff[g] < 0 || cap < 0 || soff[g + 1] > S_entries) {   // not this plan's workspace
            if (lane == 0) flag_overflow(st, g);
            continue;
        }
        const int T = table_size_for(cap, Tw);
        for (int s = lane; s < T; s += 32) {
            keys[s] = kEmptyKey;
            vals[s] = S::empty();
        }
        if (lane == 0) {
            s_count[wid] = 0;
            s_abort[wid] = 0;
        }
        __syncwarp();
        const int shift = 32 - log2_exact(T);
        CapHashOp<S> op{keys, vals, shift, (uint32_t)(T - 1), &s_count[wid], &s_abort[wid],
                        (int)cap};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        for (int64_t p0 = a0; p0 < a1; p0 += 32) {
            chunk_products<In, S::kVal>(P.A, P.B, p0, a1, 0, single, op);
            if (__any_sync(kFull, *(volatile int*)&s_abort[wid] != 0)) break;
        }
        __syncwarp();
        if (*(volatile int*)&s_abort[wid]) {   // more distinct columns than cap: exact path
            if (lane == 0) {
                route[g] = kRouteExact;
                atomicAdd(&ctr->claim[kClOverflow], 1);
            }
            __syncwarp();
            continue;
        }
        const int m = *(volatile int*)&s_count[wid];
        int pos0 = 0;
        for (int s0 = 0; s0 < T; s0 += 32) {
            const int32_t k = keys[s0 + lane];
            const unsigned occ = __ballot_sync(kFull, k != kEmptyKey);
            if (k != kEmptyKey) sbuf[pos0 + __popc(occ & ((1u << lane) - 1))] = k;
            pos0 += __popc(occ);
        }
        __syncwarp();
        const int64_t off = soff[g];
        if (m <= 32) {
            int32_t v = lane < m ? sbuf[lane] : INT32_MAX;
            v = warp_bitonic_sort32(v);
            if (lane < m) {
                const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
                stage_write<S>(sval, scol, off + lane, v, vals[s < 0 ? 0 : s]);
            }
        } else {
            const int N = (int)next_pow2(m);
            for (int t = m + lane; t < N; t += 32) sbuf[t] = INT32_MAX;
            __syncwarp();
            smem_bitonic_sort(sbuf, N, lane, 32, [] { __syncwarp(); });
            for (int t = lane; t < m; t += 32) {
                const int32_t v = sbuf[t];
                const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
                stage_write<S>(sval, scol, off + t, v, vals[s < 0 ? 0 : s]);
            }
        }
        if (lane == 0) {
            cnt[g] = m;
            atomicAdd(&ctr->learned_nnz, (unsigned long long)m);
        }
        __syncwarp();
    }
    // tiny rows: products sorted and folded in registers, kTinyRows at a time
    const int tend = ctr->claim[kClTinyRows];
    const int nwarps = gridDim.x * kWarpTierWarps;
    const int wg = blockIdx.x * kWarpTierWarps + wid;
    for (int r = wg * kTinyRows; r < tend; r += nwarps * kTinyRows) {
        tiny_batch<S, kTinyRows, S::kVal, true>(
            probs, nprob, tiny_rows, r, tend,
            [&](int64_t g, const Prob&, int32_t col, const typename S::Out& val, int rank, int m,
                bool ok) {
                const int64_t off = soff[g], cap = soff[g + 1] - off;
                if (off < 0 || cap < 0 || soff[g + 1] > S_entries) {   // another plan's workspace
                    if (lane == 0) flag_overflow(st, g);
                    return;
                }
                if (!ok || m > cap) {   // the exact path takes the row
                    if (lane == 0) {
                        route[g] = kRouteExact;
                        atomicAdd(&ctr->claim[kClOverflow], 1);
                    }
                    return;
                }
                if (rank >= 0) {
                    scol[off + rank] = col;
                    if constexpr (S::kVal) reinterpret_cast<typename S::Out*>(sval)[off + rank] = val;
                }
                if (lane == 0) {
                    cnt[g] = m;
                    atomicAdd(&ctr->learned_nnz, (unsigned long long)m);
                }
            });
    }
}

// CTA per learned row of the CTA list
template <class S>
__global__ void __launch_bounds__(kBlockThreads)
    k_learned_block(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                    int64_t R, Counters* ctr, const int64_t* __restrict__ soff,
                    uint8_t* __restrict__ route, int64_t* __restrict__ cnt, int32_t* scol,
                    void* sval, int64_t S_entries, DevStatus* st, int Tb) {
    using Slot = typename S::Slot;
    using In = typename S::In;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Slot* vals = reinterpret_cast<Slot*>(smem_raw);
    int32_t* keys = reinterpret_cast<int32_t*>(smem_raw + (size_t)Tb * sizeof(Slot));
    int32_t* sbuf = keys + Tb;
    __shared__ BatchSmem<In> bs;
    __shared__ int s_row, s_count, s_abort, s_pos;
    const int lane = lane_id();
    const int end = ctr->claim[kClBlockRows];
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    for (;;) {
        if (threadIdx.x == 0) {
            s_row = atomicAdd(&ctr->claim[kClBlockNext], 1);
            s_count = 0;
            s_abort = 0;
            s_pos = 0;
        }
        __syncthreads();
        const int r = s_row;
        if (r >= end) break;
        const int64_t g = rows[R - 1 - r];
        const Prob& P = probs[nprob == 1 ? 0 : find_prob(probs, nprob, g)];
        const int64_t i = g - P.row_base;
        const int64_t cap = soff[g + 1] - soff[g];
        if (soff[g] < 0 || cap < 0 || soff[g + 1] > S_entries) {
            if (threadIdx.x == 0) flag_overflow(st, g);
            __syncthreads();
            continue;
        }
        const int T = table_size_for(cap, Tb);
        for (int s = threadIdx.x; s < T; s += blockDim.x) {
            keys[s] = kEmptyKey;
            vals[s] = S::empty();
        }
        __syncthreads();
        const int shift = 32 - log2_exact(T);
        CapHashOp<S> op{keys, vals, shift, (uint32_t)(T - 1), &s_count, &s_abort, (int)cap};
        const int64_t a0 = ld_i64(P.A.rp + i), a1 = ld_i64(P.A.rp + i + 1);
        cta_row_products<In, S::kVal>(P.A, P.B, a0, a1, 0, single, bs, op);   // ends synced
        if (s_abort) {
            if (threadIdx.x == 0) {
                route[g] = kRouteExact;
                atomicAdd(&ctr->claim[kClOverflow], 1);
            }
            __syncthreads();
            continue;
        }
        const int m = s_count;
        for (int s0 = warp_id() * 32; s0 < T; s0 += blockDim.x) {
            const int32_t k = keys[s0 + lane];
            const unsigned occ = __ballot_sync(kFull, k != kEmptyKey);
            int b = 0;
            if (lane == 0 && occ) b = atomicAdd(&s_pos, __popc(occ));
            b = __shfl_sync(kFull, b, 0);
            if (k != kEmptyKey) sbuf[b + __popc(occ & ((1u << lane) - 1))] = k;
        }
        __syncthreads();
        const int N = (int)next_pow2(m);
        for (int t = m + threadIdx.x; t < N; t += blockDim.x) sbuf[t] = INT32_MAX;
        __syncthreads();
        smem_bitonic_sort(sbuf, N, threadIdx.x, blockDim.x, [] { __syncthreads(); });
        const int64_t off = soff[g];
        for (int t = threadIdx.x; t < m; t += blockDim.x) {
            const int32_t v = sbuf[t];
            const int s = hash_find(keys, shift, (uint32_t)(T - 1), v);
            stage_write<S>(sval, scol, off + t, v, vals[s < 0 ? 0 : s]);
        }
        if (threadIdx.x == 0) {
            cnt[g] = m;
            atomicAdd(&ctr->learned_nnz, (unsigned long long)m);
        }
        __syncthreads();
    }
}

// skip mask of the exact path: rows finished by the learned path
__global__ void k_learned_skip(int64_t R, const uint8_t* __restrict__ route, uint8_t* skip) {
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < R;
         g += (int64_t)gridDim.x * blockDim.x)
        skip[g] = route[g] == kRouteLearned ? 1 : 0;
}

// staging slices -> C rows, 32 rows per warp: rows of at most 8 entries are
// copied by their lane, longer ones by the whole warp one after another
template <class S>
__global__ void k_learned_compact(const Prob* __restrict__ probs, int nprob, int64_t R,
                                  const uint8_t* __restrict__ route,
                                  const int64_t* __restrict__ soff, const int32_t* __restrict__ scol,
                                  const void* __restrict__ sval, int64_t S_entries,
                                  DevStatus* st) {
    using Out = typename S::Out;
    constexpr int kShort = 8;
    const int lane = lane_id();
    const Out* sv = reinterpret_cast<const Out*>(sval);
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t g0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id()) * 32; g0 < R;
         g0 += nw * 32) {
        const int64_t g = g0 + lane;
        int pi = 0;
        int64_t dst = 0, n = 0, src = 0;
        if (g < R && route[g] == kRouteLearned) {
            pi = nprob == 1 ? 0 : find_prob(probs, nprob, g);
            const Prob& P = probs[pi];
            const int64_t i = g - P.row_base;
            dst = P.c_rp[i];
            n = P.c_rp[i + 1] - dst;
            src = soff[g];
            if (src < 0 || n < 0 || src + n > soff[g + 1] || soff[g + 1] > S_entries) {
                flag_overflow(st, g);   // workspace of another plan or product
                n = 0;
            }
        }
        if (n <= kShort) {
            const Prob& P = probs[pi];
#pragma unroll
            for (int t = 0; t < kShort; ++t) {
                if (t < n) {
                    P.c_col[dst + t] = scol[src + t];
                    if constexpr (S::kVal) reinterpret_cast<Out*>(P.c_val)[dst + t] = sv[src + t];
                }
            }
        }
        unsigned longm = __ballot_sync(kFull, n > kShort);
        while (longm) {
            const int l = __ffs(longm) - 1;
            longm &= longm - 1;
            const Prob& P = probs[__shfl_sync(kFull, pi, l)];
            const int64_t d = __shfl_sync(kFull, dst, l), m = __shfl_sync(kFull, n, l),
                          q = __shfl_sync(kFull, src, l);
            for (int64_t t = lane; t < m; t += 32) {
                P.c_col[d + t] = scol[q + t];
                if constexpr (S::kVal) reinterpret_cast<Out*>(P.c_val)[d + t] = sv[q + t];
            }
        }
    }
}

// ---- launchers -------------------------------------------------------------------

static unsigned grid_for(int64_t R, int per_block, int cap) {
    int64_t b = (R + per_block - 1) / per_block;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_learned_caps(const WsPtrs& w, const LearnedWs& lw, int nprob, int64_t R,
                                const float* z, float margin, int64_t exact_max,
                                int64_t learned_max, const DevInfo& dev, cudaStream_t st) {
    if (R > 0) {
        k_learned_caps<<<grid_for(R, 256, dev.sms * 8), 256, 0, st>>>(
            w.probs, nprob, R, z, margin, exact_max, learned_max, w.ub, lw.soff, lw.route, w.cnt);
        count_launch(dev);
    }
    cudaError_t e = launch_scan_inplace(lw.soff, R, w.scan_part, st);
    count_launch(dev, R > 0 ? 3 : 0);
    return e != cudaSuccess ? e : cudaGetLastError();
}

struct CapacityLimit {
    int64_t want;
    bool warp;
    int64_t out = 0;
    template <class S> void operator()() {
        int64_t c = want < 1 ? 1 : want;
        for (;;) {
            int64_t T = next_pow2(2 * c);
            if (T < 32) T = 32;
            const size_t b = learned_table_bytes<S>((int)T) * (warp ? kWarpTierWarps : 1);
            if (b <= kLearnedSmemBudget || c <= 16) break;
            c /= 2;
        }
        out = c;
    }
};

// largest capacity (halving from want) whose table fits the tier's budget
int64_t learned_capacity_limit(int sr, int64_t want, bool warp) {
    CapacityLimit f{want, warp};
    if (!dispatch_semiring(sr, f)) return 0;
    return f.out;
}

struct LearnedDirectLaunch {
    const WsPtrs* w;
    const LearnedWs* lw;
    int nprob;
    int64_t R, warp_max, block_max;
    const DevInfo* dev;
    cudaStream_t st;
    cudaError_t err = cudaSuccess;
    template <class S> void operator()() {
        cudaError_t e = cudaMemsetAsync(&w->ctr->claim[kClWarpRows], 0, 5 * sizeof(int32_t), st);
        if (e != cudaSuccess) { err = e; return; }
        if (R <= 0) return;
        k_learned_reset<<<grid_for(R, 256, dev->sms * 8), 256, 0, st>>>(R, lw->soff, w->ub,
                                                                        lw->route, w->cnt);
        count_launch(*dev);
        k_learned_bin<<<(unsigned)((R + 1023) / 1024), 1024, 0, st>>>(
            w->probs, nprob, R, lw->soff, lw->route, w->ub, warp_max, w->rows_num, w->rows_sym,
            w->ctr);
        count_launch(*dev);
        {
            int64_t T = next_pow2(2 * warp_max);
            if (T < 32) T = 32;
            const size_t smem = learned_table_bytes<S>((int)T) * kWarpTierWarps;
            e = cudaFuncSetAttribute(k_learned_warp<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_learned_warp<S>,
                                                          kWarpTierWarps * 32, smem);
            k_learned_warp<S><<<(per > 0 ? per : 1) * dev->sms, kWarpTierWarps * 32, smem, st>>>(
                w->probs, nprob, w->rows_num, w->rows_sym, w->ctr, lw->soff, lw->route, w->cnt,
                lw->scol, lw->sval, lw->entries, w->status, (int)T);
            count_launch(*dev);
        }
        {
            int64_t T = next_pow2(2 * block_max);
            if (T < 32) T = 32;
            const size_t smem = learned_table_bytes<S>((int)T);
            e = cudaFuncSetAttribute(k_learned_block<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) { err = e; return; }
            int per = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_learned_block<S>, kBlockThreads,
                                                          smem);
            k_learned_block<S><<<(per > 0 ? per : 1) * dev->sms, kBlockThreads, smem, st>>>(
                w->probs, nprob, w->rows_num, R, w->ctr, lw->soff, lw->route, w->cnt, lw->scol,
                lw->sval, lw->entries, w->status, (int)T);
            count_launch(*dev);
        }
        k_learned_skip<<<grid_for(R, 256, dev->sms * 8), 256, 0, st>>>(R, lw->route, lw->skip);
        count_launch(*dev);
        err = cudaGetLastError();
    }
};

cudaError_t launch_learned_direct(int sr, const WsPtrs& w, const LearnedWs& lw, int nprob,
                                  int64_t R, int64_t warp_max, int64_t block_max,
                                  const DevInfo& dev, cudaStream_t st) {
    LearnedDirectLaunch f{&w, &lw, nprob, R, warp_max, block_max, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    mark_stage(dev, kStLearned, st);
    return f.err;
}

struct CompactLaunch {
    const WsPtrs* w;
    const LearnedWs* lw;
    int nprob;
    int64_t R;
    const DevInfo* dev;
    cudaStream_t st;
    template <class S> void operator()() {
        k_learned_compact<S><<<grid_for(R, 256, dev->sms * 16), 256, 0, st>>>(
            w->probs, nprob, R, lw->route, lw->soff, lw->scol, lw->sval, lw->entries, w->status);
        count_launch(*dev);
    }
};

cudaError_t launch_learned_compact(int sr, const WsPtrs& w, const LearnedWs& lw, int nprob,
                                   int64_t R, const DevInfo& dev, cudaStream_t st) {
    if (R <= 0) return cudaSuccess;
    CompactLaunch f{&w, &lw, nprob, R, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    mark_stage(dev, kStLearned, st);
    return cudaGetLastError();
}

}  // namespace spg
