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

#include <cstring>

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
    // precomputed slab starts of B's rows: sp[k * sp_stride + s] = offset in
    // row k of its first column >= s * slab width (null: cursor mode)
    const int32_t* sp;
    int sp_stride;
    int s;
};

template <class In, bool kVal>
SPG_DEV In shfl_val(In a, int src) {
    if constexpr (kVal) return __shfl_sync(kFull, a, src);
    else return In();
}

template <class In, bool kVal>
SPG_DEV In load_val(const void* v, int64_t q) {
    if constexpr (kVal) return __ldg(reinterpret_cast<const In*>(v) + q);
    else return In();
}

// Segment of B_k (its entries inside the current slab) for one A entry p,
// held by the calling lane.  Advances the entry's slab cursor.
template <class In, bool kVal>
SPG_DEV void entry_segment(const DCsr& A, const DCsr& B, int64_t p, int64_t flat_p,
                           const Slab& slab, int64_t& beg, int64_t& end, In& a) {
    const int32_t k = ld_i32(A.col + p);
    a = load_val<In, kVal>(A.val, p);
    const int64_t rs = ld_i64(B.rp + k);
    if (slab.single) {
        beg = rs;
        end = ld_i64(B.rp + k + 1);
    } else if (slab.sp) {
        const int32_t* spk = slab.sp + (int64_t)k * slab.sp_stride + slab.s;
        beg = rs + __ldg(spk);
        end = rs + __ldg(spk + 1);
    } else {
        const int64_t re = ld_i64(B.rp + k + 1);
        beg = slab.first ? rs : rs + slab.cursor[flat_p];
        end = slab.last ? re : gallop_lower_bound(B.col, beg, re, slab.hi);
        if (!slab.last) slab.cursor[flat_p] = (int32_t)(end - rs);
    }
}

// Flattened walk over the short segments held by the 32 lanes (len < 32 each,
// 0 for lanes without one): the warp takes 32 consecutive products of their
// concatenation at a time; each lane finds its segment by a 5-step binary
// search over the lanes' exclusive prefix sums.  op.any(col, a, b, valid).
template <class In, bool kVal, class Op>
SPG_DEV void warp_short_segments(const DCsr& B, int64_t beg, int len, In a, Op& op) {
    const int lane = lane_id();
    const int incl = warp_incl_scan(len);
    const int total = __shfl_sync(kFull, incl, 31);
    const int excl = incl - len;
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
        const bool v = t < total;
        const int64_t q = ob + (t - oex);
        const int32_t col = v ? ld_i32(B.col + q) : 0;
        const In bv = v ? load_val<In, kVal>(B.val, q) : In();
        op.any(col, oa, bv, v);
    }
}

// One whole segment [b0, e0) walked by the warp, 4 x 32 products in flight
// while at least 128 remain; within one pass the lanes hold ascending columns.
// op.sorted(col, a, b, valid).
template <class In, bool kVal, class Op>
SPG_DEV void warp_long_segment(const DCsr& B, int64_t b0, int64_t e0, In av, Op& op) {
    const int lane = lane_id();
    int64_t q0 = b0;
    for (; q0 + 128 <= e0; q0 += 128) {
        int32_t col[4];
        In bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t q = q0 + 32 * u + lane;
            col[u] = ld_i32(B.col + q);
            bv[u] = load_val<In, kVal>(B.val, q);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) op.sorted(col[u], av, bv[u], true);
    }
    for (; q0 < e0; q0 += 32) {   // warp-uniform trip count
        const int64_t q = q0 + lane;
        const bool v = q < e0;
        const int32_t col = v ? ld_i32(B.col + q) : 0;
        const In bv = v ? load_val<In, kVal>(B.val, q) : In();
        op.sorted(col, av, bv, v);
    }
}

// Enumerates the products of A entries [p0, min(p0 + 32, p_end)) (one warp,
// one entry per lane) restricted to the slab.
template <class In, bool kVal, class Op>
SPG_DEV void chunk_products(const DCsr& A, const DCsr& B, int64_t p0, int64_t p_end,
                            int64_t flat_p0, const Slab& slab, Op& op) {
    const int lane = lane_id();
    const int64_t p = p0 + lane;
    int64_t beg = 0, end = 0;
    In a = In();
    if (p < p_end) entry_segment<In, kVal>(A, B, p, flat_p0 + lane, slab, beg, end, a);
    const int len = (int)(end - beg);
    unsigned longm = __ballot_sync(kFull, len >= 32);
    while (longm) {
        const int src = __ffs(longm) - 1;
        longm &= longm - 1;
        const int64_t b0 = __shfl_sync(kFull, beg, src);
        const int64_t e0 = __shfl_sync(kFull, end, src);
        warp_long_segment<In, kVal>(B, b0, e0, shfl_val<In, kVal>(a, src), op);
    }
    warp_short_segments<In, kVal>(B, beg, len < 32 ? len : 0, a, op);
}

// ---- CTA-wide, load-balanced enumeration (block and dense tiers) -------------
//
// Each thread brings the segment of one A entry (a batch of up to kBatch =
// blockDim.x entries).  The non-empty segments are compacted and the products
// of all of them form one flattened range (exclusive scan of the lengths);
// warp w takes the w-th of nwarps equal contiguous parts and walks it 128
// products (4 windows of 32 loads in flight) at a time.  A pass that lies in
// one segment is addressed from registers; a window that crosses segment
// boundaries loads the next 32 boundaries (one per lane) and each lane finds
// its segment by a 5-step binary search (segments are non-empty, so 32
// boundaries cover a window).  Every warp holds its share of the products to
// within one pass, whatever the mix of long hub segments and short ones.
constexpr int kBatch = 512;
constexpr int kWalkWin = 4;     // windows of 32 products in flight per warp
constexpr int kCountShift = 50;   // scan packs (entry count << 50) + product count

template <class In, int NT = kBatch>
struct BatchSmem {
    static constexpr int kN = NT;  // entries per batch = threads of the CTA
    int64_t base[NT];              // compacted non-empty segments: start - flat offset
    int64_t off[NT + 1];           // exclusive scan of their lengths
    In a[NT];
    int64_t wsum[NT / 32];
    int nseg;
};

// All threads of the CTA call this with their own segment [beg, beg + len)
// and A value (len 0 for none).  Ends with __syncthreads.
template <class In, bool kVal, class Op, int NT, int kWin = kWalkWin>
SPG_DEV void cta_walk_segments(const DCsr& B, int64_t beg, int64_t len, In a,
                               BatchSmem<In, NT>& bs, Op& op) {
    constexpr int kBatch = NT;
    const int lane = lane_id(), wid = warp_id();
    const int tid = threadIdx.x;
    const int nwarps = kBatch / 32;
    const int64_t kLenMask = ((int64_t)1 << kCountShift) - 1;
    const int64_t packed = len > 0 ? (((int64_t)1 << kCountShift) | len) : 0;
    const int64_t incl = warp_incl_scan(packed);
    if (lane == 31) bs.wsum[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        const int64_t x = lane < nwarps ? bs.wsum[lane] : 0;
        const int64_t xi = warp_incl_scan(x);
        if (lane < nwarps) bs.wsum[lane] = xi - x;
        if (lane == 31) {
            bs.off[kBatch] = xi & kLenMask;            // total products
            bs.nseg = (int)(xi >> kCountShift);        // non-empty segments
        }
    }
    __syncthreads();
    const int64_t ex = bs.wsum[wid] + incl - packed;   // exclusive (count, length)
    if (len > 0) {
        const int c = (int)(ex >> kCountShift);
        bs.base[c] = beg - (ex & kLenMask);
        bs.off[c] = ex & kLenMask;
        if constexpr (kVal) bs.a[c] = a;
    }
    __syncthreads();
    const int nseg = bs.nseg;
    const int64_t W = bs.off[kBatch];
    if (nseg < kBatch && tid == 0) bs.off[nseg] = W;   // end of the last segment
    __syncthreads();
    const int64_t lo_w = W * wid / nwarps, hi_w = W * (wid + 1) / nwarps;
    if (lo_w < hi_w) {
        int e;
        {   // largest segment e with off[e] <= lo_w
            int lo = 0, hi = nseg - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (bs.off[mid] <= lo_w) lo = mid; else hi = mid - 1;
            }
            e = lo;
        }
        int64_t ebase = bs.base[e];   // q = ebase + t inside segment e
        int64_t eend = bs.off[e + 1];
        In ea = In();
        if constexpr (kVal) ea = bs.a[e];
        for (int64_t t0 = lo_w; t0 < hi_w; t0 += 32 * kWin) {   // warp-uniform
            int32_t col[kWin];
            In bval[kWin];
            In av[kWin];
            bool vv[kWin];
            if (eend >= t0 + 32 * kWin || eend >= hi_w) {       // the pass lies in segment e
                // one base pointer per lane; the windows are fixed offsets from it
                const int64_t q0 = ebase + t0 + lane;
                const int64_t left = hi_w - t0 - lane;   // products of the pass from this lane on
                const int rem = left < 32 * kWin ? (int)left : 32 * kWin;
                const int32_t* cp = B.col + q0;
#pragma unroll
                for (int u = 0; u < kWin; ++u) {
                    vv[u] = 32 * u < rem;
                    col[u] = vv[u] ? __ldg(cp + 32 * u) : 0;
                    if constexpr (kVal)
                        bval[u] = vv[u] ? __ldg(reinterpret_cast<const In*>(B.val) + q0 + 32 * u) : In();
                    else
                        bval[u] = In();
                    av[u] = ea;
                }
            } else if (bs.off[e + 2] >= t0 + 32 * kWin || bs.off[e + 2] >= hi_w) {
                // one segment end inside the pass (eend < hi_w <= total, so
                // segment e + 1 exists): products before it are segment e's,
                // the rest segment e + 1's
                const int64_t nbase = bs.base[e + 1];
                In na = In();
                if constexpr (kVal) na = bs.a[e + 1];
                const int64_t left = hi_w - t0 - lane;
                const int rem = left < 32 * kWin ? (int)left : 32 * kWin;
                const int64_t cut = eend - t0 - lane;    // windows u with 32u >= cut are past the end
#pragma unroll
                for (int u = 0; u < kWin; ++u) {
                    vv[u] = 32 * u < rem;
                    const bool second = 32 * u >= cut;
                    const int64_t q = (second ? nbase : ebase) + t0 + 32 * u + lane;
                    col[u] = vv[u] ? ld_i32(B.col + q) : 0;
                    bval[u] = vv[u] ? load_val<In, kVal>(B.val, q) : In();
                    av[u] = second ? na : ea;
                }
                ++e;
                ebase = nbase;
                eend = bs.off[e + 1];
                ea = na;
            } else {
                int64_t qv[kWin];
#pragma unroll
                for (int u = 0; u < kWin; ++u) {
                    const int64_t tu = t0 + 32 * u;
                    const int64_t t = tu + lane;
                    vv[u] = t < hi_w;
                    int me = e;
                    if (tu < hi_w) {                         // warp-uniform
                        while (bs.off[e + 1] <= tu) ++e;     // segments are non-empty
                        me = e;
                        if (bs.off[e + 1] < tu + 32 && bs.off[e + 1] < hi_w) {
                            const int ej = e + lane;       // lane j: end of segment e + j
                            // ends relative to the window start fit 32 bits
                            const int64_t bnd = ej < nseg ? bs.off[ej + 1] - tu : INT32_MAX;
                            const int32_t rb = bnd < INT32_MAX ? (int32_t)bnd : INT32_MAX;
                            int k = 0;                     // number of ends <= t
#pragma unroll
                            for (int step = 16; step > 0; step >>= 1) {
                                const int32_t bv = __shfl_sync(kFull, rb, k + step - 1);
                                if (bv <= lane) k += step;
                            }
                            me = e + k;
                            // the next window starts in lane 31's segment or
                            // later: no walk over this window's segments again
                            const int e31 = __shfl_sync(kFull, me, 31);
                            e = e31 < nseg - 1 ? e31 : nseg - 1;
                        }
                    }
                    qv[u] = bs.base[me] + t;
                    if constexpr (kVal) av[u] = bs.a[me];
                    else av[u] = In();
                }
                const int64_t tn = t0 + 32 * kWin;              // segment of the next pass
                if (tn < hi_w) {
                    while (bs.off[e + 1] <= tn) ++e;
                }
                ebase = bs.base[e];
                eend = bs.off[e + 1];
                if constexpr (kVal) ea = bs.a[e];
#pragma unroll
                for (int u = 0; u < kWin; ++u) {
                    col[u] = vv[u] ? ld_i32(B.col + qv[u]) : 0;
                    bval[u] = vv[u] ? load_val<In, kVal>(B.val, qv[u]) : In();
                }
            }
#pragma unroll
            for (int u = 0; u < kWin; ++u) op.any(col[u], av[u], bval[u], vv[u]);
        }
    }
    __syncthreads();
}

// One A entry per thread, kept in registers while a row is processed slab
// after slab (rows with at most kBatch entries): its segment in each slab
// comes from the slab-start table (next bound prefetched one slab ahead) or,
// without a table, from a cursor advanced by galloping.
template <class In, bool kVal>
struct RowEntry {
    bool v;
    int32_t k;
    In a;
    int64_t rs, re, cur;
    int32_t sp_lo, sp_hi, sp_nx;

    SPG_DEV void load(const DCsr& A, const DCsr& B, int64_t p, bool valid, const Slab& first) {
        v = valid;
        k = 0;
        a = In();
        rs = re = cur = 0;
        sp_lo = sp_hi = sp_nx = 0;
        if (!v) return;
        k = ld_i32(A.col + p);
        a = load_val<In, kVal>(A.val, p);
        rs = ld_i64(B.rp + k);
        re = ld_i64(B.rp + k + 1);
        cur = rs;
        if (first.sp) {
            const int32_t* spk = first.sp + (int64_t)k * first.sp_stride;
            sp_lo = __ldg(spk);
            sp_hi = __ldg(spk + 1);
        }
    }
    // slabs must be visited in order s = 0, 1, ...
    SPG_DEV void segment(const DCsr& B, const Slab& sl, int nslabs, int64_t& beg, int64_t& end) {
        beg = end = 0;
        if (!v) return;
        if (sl.single) {
            beg = rs;
            end = re;
        } else if (sl.sp) {
            beg = rs + sp_lo;
            end = rs + sp_hi;
            sp_nx = (sl.s + 2 <= nslabs) ? __ldg(sl.sp + (int64_t)k * sl.sp_stride + sl.s + 2) : 0;
            sp_lo = sp_hi;
            sp_hi = sp_nx;
        } else {
            beg = cur;
            end = sl.last ? re : gallop_lower_bound(B.col, cur, re, sl.hi);
            cur = end;
        }
    }
};

// Products of row entries [a0, a1) restricted to the slab, spread over the CTA.
template <class In, bool kVal, class Op, int NT, int kWin = kWalkWin>
SPG_DEV void cta_row_products(const DCsr& A, const DCsr& B, int64_t a0, int64_t a1,
                              int64_t flat_base, const Slab& slab, BatchSmem<In, NT>& bs, Op& op) {
    for (int64_t b0 = a0; b0 < a1; b0 += NT) {
        const int64_t p = b0 + threadIdx.x;
        int64_t beg = 0, end = 0;
        In a = In();
        if (p < a1) entry_segment<In, kVal>(A, B, p, flat_base + (p - a0), slab, beg, end, a);
        cta_walk_segments<In, kVal, Op, NT, kWin>(B, beg, end - beg, a, bs, op);
    }
}

// one A entry per lane, the same in every warp (rows with <= 32 entries)
template <class In, bool kVal>
struct LaneEntry {
    bool v;
    int32_t k;
    In a;
    int64_t rs, re;
    SPG_DEV void load(const DCsr& A, const DCsr& B, int64_t p, bool valid) {
        v = valid;
        k = 0;
        a = In();
        rs = re = 0;
        if (!v) return;
        k = ld_i32(A.col + p);
        a = load_val<In, kVal>(A.val, p);
        rs = ld_i64(B.rp + k);
        re = ld_i64(B.rp + k + 1);
    }
    // segment of slabs [s0, s1) (nslabs slabs in the row; sp may be null only
    // when the range is the whole row)
    SPG_DEV void range(const int32_t* sp, int sp_stride, int nslabs, int s0, int s1,
                       int64_t& b, int64_t& e) const {
        b = e = 0;
        if (!v) return;
        b = (s0 == 0) ? rs : rs + __ldg(sp + (int64_t)k * sp_stride + s0);
        e = (s1 >= nslabs) ? re : rs + __ldg(sp + (int64_t)k * sp_stride + s1);
    }
};

// Products of the <= 32 lane entries' segments [b, e) split evenly over the
// warps: each warp holds the whole 32-entry table in registers.
template <class In, bool kVal, class Op, int kWin = kWalkWin>
SPG_DEV void warp_table_walk(const DCsr& B, int64_t b, int64_t e, In a, Op& op) {
    const int lane = lane_id(), wid = warp_id();
    const int nwarps = blockDim.x >> 5;
    const int64_t len = e - b;
    const int64_t my_end = warp_incl_scan(len);
    const int64_t excl = my_end - len;
    const int64_t qbase = b - excl;   // q = qbase + t for the lane's products
    const int64_t total = __shfl_sync(kFull, my_end, 31);
    const int64_t lo_w = total * wid / nwarps, hi_w = total * (wid + 1) / nwarps;
    int kc = 0;   // entry holding product t0 (warp-uniform, advances with t0)
    for (int64_t t0 = lo_w; t0 < hi_w; t0 += 32 * kWin) {   // warp-uniform
        int64_t qv[kWin];
        In av[kWin];
        bool vv[kWin];
        // entries whose products all precede t0 (ends are non-decreasing)
        kc = __popc(__ballot_sync(kFull, my_end <= t0));
        if (kc > 31) kc = 31;
        const int64_t endk = __shfl_sync(kFull, my_end, kc);
        // first entry with products after endk (empty entries are skipped)
        const unsigned later = __ballot_sync(kFull, my_end > endk);
        const int kn = later ? __ffs(later) - 1 : 31;
        const int64_t endn = __shfl_sync(kFull, my_end, kn);
        if (t0 + 32 * kWin <= endk && t0 + 32 * kWin <= hi_w) {
            // the window lies in one segment (the common case for hub rows of
            // B): addresses without a per-lane search
            const int64_t base = __shfl_sync(kFull, qbase, kc);
            const In ak = shfl_val<In, kVal>(a, kc);
#pragma unroll
            for (int u = 0; u < kWin; ++u) {
                qv[u] = base + t0 + 32 * u + lane;
                av[u] = ak;
                vv[u] = true;
            }
        } else if (later && (endn >= t0 + 32 * kWin || endn >= hi_w)) {
            // one segment end inside the pass: entry kc before it, entry kn after
            const int64_t base = __shfl_sync(kFull, qbase, kc);
            const int64_t nbase = __shfl_sync(kFull, qbase, kn);
            const In ak = shfl_val<In, kVal>(a, kc);
            const In an = shfl_val<In, kVal>(a, kn);
#pragma unroll
            for (int u = 0; u < kWin; ++u) {
                const int64_t t = t0 + 32 * u + lane;
                vv[u] = t < hi_w;
                const bool second = t >= endk;
                qv[u] = (second ? nbase : base) + t;
                av[u] = second ? an : ak;
            }
        } else {
#pragma unroll
            for (int u = 0; u < kWin; ++u) {
                const int64_t tu = t0 + 32 * u, t = tu + lane;
                vv[u] = t < hi_w;
                // prefix ends relative to the pass start (clamped to 32 bits:
                // only their order against 0..31 matters)
                const int64_t rel = my_end - tu;
                const int32_t re = rel > INT32_MAX ? INT32_MAX : (rel < INT32_MIN ? INT32_MIN : (int32_t)rel);
                int k = 0;   // entry of product t: number of prefix ends <= t
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const int32_t bv = __shfl_sync(kFull, re, k + step - 1);
                    if (bv <= lane) k += step;
                }
                qv[u] = __shfl_sync(kFull, qbase, k) + t;
                av[u] = shfl_val<In, kVal>(a, k);
            }
        }
        int32_t col[kWin];
        In bval[kWin];
#pragma unroll
        for (int u = 0; u < kWin; ++u) {
            col[u] = vv[u] ? ld_i32(B.col + qv[u]) : 0;
            bval[u] = vv[u] ? load_val<In, kVal>(B.val, qv[u]) : In();
        }
#pragma unroll
        for (int u = 0; u < kWin; ++u) op.any(col[u], av[u], bval[u], vv[u]);
    }
}

// OR of one bit per lane into a shared bitmap, for lanes holding ascending
// columns (c relative to the slab): lanes of one 32-bit word form a run; a
// segmented OR-scan gives the run's last lane the word's bits, and only that
// lane issues the atomic (one atomic per word instead of one per column).
SPG_DEV void bitmap_or_sorted(uint32_t* bm, int32_t c, bool valid) {
    const int lane = lane_id();
    const int w = valid ? (c >> 5) : -1 - lane;
    uint32_t bit = valid ? (1u << (c & 31)) : 0u;
    const int wprev = __shfl_up_sync(kFull, w, 1);
    const unsigned heads = __ballot_sync(kFull, lane == 0 || wprev != w);
    const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t o = __shfl_up_sync(kFull, bit, d);
        if (lane - d >= start) bit |= o;
    }
    const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
    if (valid && tail) atomicOr(bm + w, bit);
}

// ---- tiny rows: at most 32 products, one per lane, sorted in registers -------
//
// A row whose products fit the warp (ub_i <= 32) needs no table: lane t takes
// product t (owner search over the lanes' prefix sums, as in
// warp_short_segments), the warp sorts the (column, value) pairs by column
// with a bitonic network of shuffles, a segmented suffix reduction gives the
// first lane of each run of equal columns the (+) of the run, and the run
// heads are the row's sorted output.

constexpr int kTinyMax = 32;

// shuffles of any trivially copyable value, word by word (kMode 0: from lane
// src, 1: xor src, 2: down by src)
template <int kMode, class T>
SPG_DEV T shfl_words(const T& v, int src) {
    constexpr int W = (int)((sizeof(T) + 3) / 4);
    uint32_t w[W] = {};
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < W; ++i) {
        if constexpr (kMode == 0) w[i] = __shfl_sync(kFull, w[i], src);
        else if constexpr (kMode == 1) w[i] = __shfl_xor_sync(kFull, w[i], src);
        else w[i] = __shfl_down_sync(kFull, w[i], src);
    }
    T out;
    memcpy(&out, w, sizeof(T));
    return out;
}

// Sorts the lanes' (col, val) by column (INT32_MAX last) and folds equal
// columns with (+) into the first lane of their run.  Returns the number of
// distinct columns; `rank` = position of a head lane among them (-1 else).
// Branch-free: every compare-exchange is a select.
template <class S, bool kWithVal>
SPG_DEV int tiny_sort_reduce(int32_t& col, typename S::Out& val, int& rank) {
    using Out = typename S::Out;
    const int lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int32_t oc = __shfl_xor_sync(kFull, col, j);
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            const bool take = keep_min ? (oc < col) : (oc > col);
            col = take ? oc : col;
            if constexpr (kWithVal) {
                const Out ov = shfl_words<1>(val, j);
                val = take ? ov : val;
            }
        }
    }
    if constexpr (kWithVal) {
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int32_t oc = __shfl_down_sync(kFull, col, d);
            const Out ov = shfl_words<2>(val, d);
            const Out sum = S::add(val, ov);
            val = (lane + d < 32 && oc == col) ? sum : val;
        }
    }
    const int32_t prev = __shfl_up_sync(kFull, col, 1);
    const bool head = col != INT32_MAX && (lane == 0 || prev != col);
    const unsigned hm = __ballot_sync(kFull, head);
    rank = head ? __popc(hm & ((1u << lane) - 1)) : -1;
    return __popc(hm);
}

// Number of distinct columns held by the lanes (INT32_MAX = none): the lowest
// lane of each group of equal columns counts it.
SPG_DEV int tiny_count_distinct(int32_t col) {
    const unsigned same = __match_any_sync(kFull, col);
    const bool head = col != INT32_MAX && (__ffs(same) - 1) == lane_id();
    return __popc(__ballot_sync(kFull, head));
}

// G tiny rows at once (rows[r0 .. r0 + G) below rend): every load phase is
// issued for the G rows before the next phase starts, so one warp keeps G
// rows' dependent loads (row range -> A entries -> B row ranges -> B entries)
// in flight together.  For each row, emit(g, P, col, val, rank, m, ok) is
// called by all lanes (ok = false if the row is not tiny after all).  With
// kSorted = false only m (the distinct count) is computed: no sort, rank -1.
template <class S, int G, bool kWithVal, bool kSorted, class Emit>
SPG_DEV void tiny_batch(const Prob* __restrict__ probs, int nprob, const int32_t* __restrict__ rows,
                        int r0, int rend, Emit&& emit) {
    using In = typename S::In;
    using Out = typename S::Out;
    const int lane = lane_id();
    int64_t gl = -1, a0l = 0, a1l = 0;
    int pil = 0;
    if (lane < G && r0 + lane < rend) {
        gl = rows[r0 + lane];
        pil = nprob == 1 ? 0 : find_prob(probs, nprob, gl);
        const Prob& P = probs[pil];
        const int64_t i = gl - P.row_base;
        a0l = ld_i64(P.A.rp + i);
        a1l = ld_i64(P.A.rp + i + 1);
    }
    int64_t g[G], a0[G], na[G];
    int pi[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        g[j] = __shfl_sync(kFull, gl, j);
        a0[j] = __shfl_sync(kFull, a0l, j);
        na[j] = __shfl_sync(kFull, a1l, j) - a0[j];
        pi[j] = __shfl_sync(kFull, pil, j);
    }
    int32_t k[G];
    In a[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        k[j] = 0;
        a[j] = In();
        if (g[j] >= 0 && lane < na[j]) {
            const Prob& P = probs[pi[j]];
            k[j] = ld_i32(P.A.col + a0[j] + lane);
            a[j] = load_val<In, S::kVal>(P.A.val, a0[j] + lane);
        }
    }
    int64_t b0[G], len[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        b0[j] = 0;
        len[j] = 0;
        if (g[j] >= 0 && lane < na[j]) {
            const Prob& P = probs[pi[j]];
            b0[j] = ld_i64(P.B.rp + k[j]);
            len[j] = ld_i64(P.B.rp + k[j] + 1) - b0[j];
        }
    }
    int64_t q[G];
    In oa[G];
    int total[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const int64_t incl = warp_incl_scan(len[j]);
        const int64_t tot = __shfl_sync(kFull, incl, 31);
        total[j] = (tot > kTinyMax || na[j] > 32) ? -1 : (int)tot;
        q[j] = 0;
        oa[j] = In();
        if (total[j] > 0) {
            const int excl = (int)(incl - len[j]);
            int owner = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const int c = owner + step;
                if (__shfl_sync(kFull, excl, c) <= lane) owner = c;
            }
            q[j] = __shfl_sync(kFull, b0[j], owner) + (lane - __shfl_sync(kFull, excl, owner));
            oa[j] = shfl_val<In, S::kVal>(a[j], owner);
        }
    }
    int32_t col[G];
    Out val[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        col[j] = INT32_MAX;
        In bv = In();
        if (lane < total[j]) {
            const Prob& P = probs[pi[j]];
            col[j] = ld_i32(P.B.col + q[j]);
            if constexpr (kWithVal) bv = load_val<In, true>(P.B.val, q[j]);
        }
        if constexpr (kWithVal) val[j] = S::prod(oa[j], bv);
    }
#pragma unroll
    for (int j = 0; j < G; ++j) {
        if (g[j] < 0) continue;
        const Prob& P = probs[pi[j]];
        if (total[j] < 0) {
            emit(g[j], P, col[j], val[j], -1, 0, false);
            continue;
        }
        int rank = -1;
        int m;
        if constexpr (kSorted) m = tiny_sort_reduce<S, kWithVal>(col[j], val[j], rank);
        else m = tiny_count_distinct(col[j]);
        emit(g[j], P, col[j], val[j], rank, m, true);
    }
}

// ---- per-row product counts: short rows by their lane, long rows by a warp -----
//
// Pass 1 gives a warp 32 consecutive rows, one per lane (coalesced row
// pointers): rows with at most kRowShort entries are summed by their lane with
// independent, unrolled gathers; longer rows are appended to a list.  Pass 2
// gives every listed row a whole warp (4 gathers in flight per lane), so the
// hub rows of a graph spread over all warps.  Both give ub = sum nnz(B_k),
// the largest nnz(B_k) and nnz(A_i).
constexpr int kRowShort = 8;
constexpr int kClLongRows = 13;   // Counters::claim slot of the long-row list length

struct RowRange {
    int pi;
    int64_t a0, a1;
};

SPG_DEV RowRange row_range(const Prob* __restrict__ probs, int nprob, int64_t g) {
    RowRange r;
    r.pi = nprob > 1 ? find_prob(probs, nprob, g) : 0;
    const Prob& P = probs[r.pi];
    const int64_t i = g - P.row_base;
    r.a0 = ld_i64(P.A.rp + i);
    r.a1 = ld_i64(P.A.rp + i + 1);
    return r;
}

// sum and max of nnz(B_k) over the <= kRowShort entries of a row (one lane)
SPG_DEV void lane_row_counts(const Prob& P, int64_t a0, int64_t na, int64_t& ub, int64_t& mx) {
    ub = 0;
    mx = 0;
#pragma unroll
    for (int t = 0; t < kRowShort; ++t) {
        if (t < na) {
            const int32_t k = ld_i32(P.A.col + a0 + t);
            const int64_t l = ld_i64(P.B.rp + k + 1) - ld_i64(P.B.rp + k);
            ub += l;
            mx = l > mx ? l : mx;
        }
    }
}

// appends the calling lanes' rows (flag set) to list[ctr->claim[kClLongRows]...]
SPG_DEV void append_rows(bool flag, int64_t g, int32_t* list, Counters* ctr) {
    const unsigned m = __ballot_sync(kFull, flag);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    int base = 0;
    if (lane_id() == leader) base = atomicAdd(&ctr->claim[kClLongRows], __popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (flag) list[base + __popc(m & ((1u << lane_id()) - 1))] = (int32_t)g;
}

// sum and max of nnz(B_k) over the entries [a0, a1) of one row, whole warp
SPG_DEV void warp_row_long(const Prob& P, int64_t a0, int64_t a1, int64_t& ub, int64_t& mx) {
    const int lane = lane_id();
    int64_t s = 0, m = 0;
    int64_t q = a0 + lane;
    for (; q + 96 < a1; q += 128) {   // 4 independent gathers in flight per lane
        int32_t k[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) k[u] = ld_i32(P.A.col + q + 32 * u);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t l = ld_i64(P.B.rp + k[u] + 1) - ld_i64(P.B.rp + k[u]);
            s += l;
            m = l > m ? l : m;
        }
    }
    for (; q < a1; q += 32) {
        const int32_t k = ld_i32(P.A.col + q);
        const int64_t l = ld_i64(P.B.rp + k + 1) - ld_i64(P.B.rp + k);
        s += l;
        m = l > m ? l : m;
    }
    ub = warp_sum(s);
    mx = warp_max(m);
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
