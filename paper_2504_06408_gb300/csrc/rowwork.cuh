// Row-wise Gustavson building blocks: enumeration of the intermediate
// products of one output row, shared-memory hash tables, and sorts.
//
// Products of row i (Section 2.1 definition of SpGEMM): for every entry
// (i, k) of A and every entry (k, j) of B, the product A[i,k] (x) B[k,j]
// belongs to output column j.  A warp takes 32 consecutive entries of A_i at
// a time, one per lane.  Segments of B (the entries of B_k inside the current
// column slab) of length >= 32 are walked by the whole warp, one segment
// after another (coalesced, no shuffles); shorter segments are flattened: the
// warp walks their concatenation 32 products at a time and each lane finds
// the segment its product belongs to by a 5-step binary search over the
// lanes' exclusive prefix sums.
#pragma once

#include "common.cuh"

namespace spg {

// First position q in [lo, hi) with col[q] >= lim (col ascending), searched by
// galloping from lo: cost ~ 2 log2(distance).
SPG_DEV int64_t gallop_lower_bound(const int32_t* __restrict__ col, int64_t lo, int64_t hi,
                                   int32_t lim) {
    if (lo >= hi || ld_i32(col + lo) >= lim) return lo;
    int64_t prev = lo, step = 1;
    while (prev + step < hi && ld_i32(col + prev + step) < lim) {
        prev += step;
        step <<= 1;
    }
    int64_t a = prev + 1, b = (prev + step < hi) ? prev + step : hi;  // answer in [a, b]
    while (a < b) {
        int64_t m = (a + b) >> 1;
        if (ld_i32(col + m) < lim) a = m + 1; else b = m;
    }
    return a;
}

// Column slab [lo, hi) of B's columns, plus the per-entry cursors that let a
// row be processed slab after slab without searching B_k from its start.
struct Slab {
    int32_t lo, hi;       // column range
    bool first, last;     // first / last slab of the row
    bool single;          // the only slab: no cursors used
    int32_t* cursor;      // per entry of A (flat entry numbering), or null
};

template <class In, bool kVal>
SPG_DEV In shfl_val(In a, int src) {
    if constexpr (kVal) return __shfl_sync(kFull, a, src);
    else return In();
}

// Enumerates the products of A entries [p0, min(p0 + 32, p_end)) restricted to
// the slab; calls op(q, a, lane_valid) for each product with q the position in
// B (all 32 lanes call op together; lane_valid false for padding lanes).
template <class In, bool kVal, class Op>
SPG_DEV void chunk_products(const DCsr& A, const DCsr& B, int64_t p0, int64_t p_end,
                            int64_t flat_p0, const Slab& slab, Op& op) {
    const int lane = lane_id();
    const int64_t p = p0 + lane;
    const bool valid = p < p_end;
    int64_t beg = 0, end = 0;
    In a = In();
    if (valid) {
        const int32_t k = ld_i32(A.col + p);
        if constexpr (kVal) a = __ldg(reinterpret_cast<const In*>(A.val) + p);
        if (slab.single) {
            beg = ld_i64(B.rp + k);
            end = ld_i64(B.rp + k + 1);
        } else {
            const int64_t rowend = ld_i64(B.rp + k + 1);
            beg = slab.first ? ld_i64(B.rp + k) : (ld_i64(B.rp + k) + slab.cursor[flat_p0 + lane]);
            end = slab.last ? rowend : gallop_lower_bound(B.col, beg, rowend, slab.hi);
            if (!slab.last) slab.cursor[flat_p0 + lane] = (int32_t)(end - ld_i64(B.rp + k));
        }
    }
    const int len = (int)(end - beg);
    // long segments: whole warp per segment
    unsigned longm = __ballot_sync(kFull, len >= 32);
    while (longm) {
        const int src = __ffs(longm) - 1;
        longm &= longm - 1;
        const int64_t b0 = __shfl_sync(kFull, beg, src);
        const int64_t e0 = __shfl_sync(kFull, end, src);
        const In av = shfl_val<In, kVal>(a, src);
        for (int64_t q0 = b0; q0 < e0; q0 += 32) {   // warp-uniform trip count
            const int64_t q = q0 + lane;
            op(q, av, q < e0);
        }
    }
    // short segments: flattened
    const int sl = (len < 32) ? len : 0;
    const int incl = warp_incl_scan(sl);
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - sl;
    for (int base = 0; base < total; base += 32) {
        const int t = base + lane;
        int owner = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int c = owner + step;
            const int ex = __shfl_sync(kFull, excl, c);
            if (ex <= t) owner = c;
        }
        const int64_t ob = __shfl_sync(kFull, beg, owner);
        const int oex = __shfl_sync(kFull, excl, owner);
        const In oa = shfl_val<In, kVal>(a, owner);
        op(ob + (t - oex), oa, t < total);
    }
}

// ---- shared-memory hash tables (linear probing, power-of-two size) ----------

// Inserts key; returns 1 if it was new, 0 if present, -1 if the table is full.
SPG_DEV int hash_insert(int32_t* keys, int shift, uint32_t mask, int32_t key) {
    uint32_t s = hash_slot(key, shift);
    for (uint32_t n = 0; n <= mask; ++n) {
        const int32_t cur = *(volatile int32_t*)(keys + s);
        if (cur == key) return 0;
        if (cur == kEmptyKey) {
            const int32_t old = atomicCAS(keys + s, kEmptyKey, key);
            if (old == kEmptyKey) return 1;
            if (old == key) return 0;
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// Inserts key if absent; returns its slot, or -1 if the table is full.
SPG_DEV int hash_slot_of(int32_t* keys, int shift, uint32_t mask, int32_t key) {
    uint32_t s = hash_slot(key, shift);
    for (uint32_t n = 0; n <= mask; ++n) {
        const int32_t cur = *(volatile int32_t*)(keys + s);
        if (cur == key) return (int)s;
        if (cur == kEmptyKey) {
            const int32_t old = atomicCAS(keys + s, kEmptyKey, key);
            if (old == kEmptyKey || old == key) return (int)s;
        }
        s = (s + 1) & mask;
    }
    return -1;
}

// Slot of a key known to be present (after accumulation, no concurrent writes).
SPG_DEV int hash_find(const int32_t* keys, int shift, uint32_t mask, int32_t key) {
    uint32_t s = hash_slot(key, shift);
    for (uint32_t n = 0; n <= mask; ++n) {
        const int32_t cur = keys[s];
        if (cur == key) return (int)s;
        if (cur == kEmptyKey) return -1;
        s = (s + 1) & mask;
    }
    return -1;
}

// ---- sorts --------------------------------------------------------------------

// Ascending bitonic sort of 32 keys held one per lane.
SPG_DEV int32_t warp_bitonic_sort32(int32_t v) {
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t o = __shfl_xor_sync(kFull, v, j);
            const bool lower = (lane & j) == 0;
            const bool up = (lane & k) == 0;
            const int32_t lo = v < o ? v : o, hi = v < o ? o : v;
            v = (lower == up) ? lo : hi;
        }
    }
    return v;
}

// Ascending bitonic sort of buf[0, n) in shared memory (n a power of two) by
// nthreads threads with ids tid; `sync` is the group barrier.
template <class Sync>
SPG_DEV void smem_bitonic_sort(int32_t* buf, int n, int tid, int nthreads, Sync sync) {
    for (int k = 2; k <= n; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = tid; q < (n >> 1); q += nthreads) {
                const int i = ((q & ~(j - 1)) << 1) | (q & (j - 1));
                const int l = i + j;
                const bool up = (i & k) == 0;
                const int32_t a = buf[i], b = buf[l];
                if ((a > b) == up) {
                    buf[i] = b;
                    buf[l] = a;
                }
            }
            sync();
        }
    }
}

}  // namespace spg
