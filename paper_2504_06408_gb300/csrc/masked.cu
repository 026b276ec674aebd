// Masked product: C = (A (x).(+) B) restricted to the pattern of a mask M,
// C[i,j] present iff (i,j) is in M and at least one product reaches it (the
// Section 2.1 product, kept where the mask allows; e.g. triangle counting
// multiplies L L under the mask L).
//
// Every mask entry owns one accumulator: the mask's own positions index the
// accumulators, so no table is needed.
// 1. slots <- empty, touched <- 0 (one per mask entry).
// 2. a warp per row walks the products of A_i (the product walk of the plain
//    tiers); each product's column is looked up in M_i by binary search and,
//    when present, folded into that entry's accumulator (global atomics,
//    the same semiring functors as the shared-memory tiers).
// 3. counts of touched entries per row, scanned into C's row pointers.
// 4. a warp per row compacts the touched entries in column order.
#include "plan.h"
#include "rowwork.cuh"
#include "semiring.cuh"

namespace spg {

template <class S>
__global__ void k_mask_init(int64_t nnz_m, typename S::Slot* slots, uint8_t* touched) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nnz_m;
         t += (int64_t)gridDim.x * blockDim.x) {
        if constexpr (S::kVal) slots[t] = S::empty();
        touched[t] = 0;
    }
}

// first position q in [lo, hi) with col[q] >= v (col ascending)
SPG_DEV int64_t mask_lower(const int32_t* __restrict__ col, int64_t lo, int64_t hi, int32_t v) {
    while (lo < hi) {
        const int64_t m = (lo + hi) >> 1;
        if (ld_i32(col + m) < v) lo = m + 1; else hi = m;
    }
    return lo;
}

template <class S>
struct MaskAccOp {
    const int32_t* mcol;
    int64_t ms, me, m0;   // the row's mask entries; accumulators start at M's first entry m0
    typename S::Slot* slots;
    uint8_t* touched;
    SPG_DEV void any(int32_t col, typename S::In a, typename S::In b, bool valid) {
        if (!valid) return;
        const int64_t q = mask_lower(mcol, ms, me, col);
        if (q >= me || ld_i32(mcol + q) != col) return;
        if constexpr (S::kVal) S::acc(slots + (q - m0), a, b);
        if (!touched[q - m0]) touched[q - m0] = 1;
    }
    SPG_DEV void sorted(int32_t col, typename S::In a, typename S::In b, bool valid) {
        any(col, a, b, valid);
    }
};

template <class S>
__global__ void k_mask_acc(DCsr A, DCsr B, DCsr M, typename S::Slot* slots, uint8_t* touched) {
    using In = typename S::In;
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const Slab single{0, 0, true, true, true, nullptr, nullptr, 0, 0};
    const int64_t m0 = ld_i64(M.rp);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < A.nrows; i += nw) {
        const int64_t ms = ld_i64(M.rp + i), me = ld_i64(M.rp + i + 1);
        if (ms == me) continue;
        MaskAccOp<S> op{M.col, ms, me, m0, slots, touched};
        const int64_t a0 = ld_i64(A.rp + i), a1 = ld_i64(A.rp + i + 1);
        for (int64_t p0 = a0; p0 < a1; p0 += 32)
            chunk_products<In, S::kVal>(A, B, p0, a1, 0, single, op);
    }
}

// cnt[i] = touched entries of row i
__global__ void k_mask_count(DCsr M, const uint8_t* __restrict__ touched, int64_t* cnt) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t m0 = ld_i64(M.rp);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < M.nrows; i += nw) {
        const int64_t ms = ld_i64(M.rp + i), me = ld_i64(M.rp + i + 1);
        int64_t c = 0;
        for (int64_t q = ms + lane; q < me; q += 32) c += touched[q - m0];
        c = warp_sum(c);
        if (lane == 0) cnt[i] = c;
    }
}

template <class S>
__global__ void k_mask_write(DCsr M, const typename S::Slot* __restrict__ slots,
                             const uint8_t* __restrict__ touched, const int64_t* __restrict__ c_rp,
                             int32_t* c_col, void* c_val, DevStatus* st) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t m0 = ld_i64(M.rp);
    for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id(); i < M.nrows; i += nw) {
        const int64_t ms = ld_i64(M.rp + i), me = ld_i64(M.rp + i + 1);
        const int64_t off = c_rp[i], n = c_rp[i + 1] - off;
        int64_t rank = 0;
        for (int64_t q0 = ms; q0 < me; q0 += 32) {   // warp-uniform
            const int64_t q = q0 + lane;
            const bool t = q < me && touched[q - m0];
            const unsigned tm = __ballot_sync(kFull, t);
            if (t) {
                const int64_t r = rank + __popc(tm & ((1u << lane) - 1));
                if (r < n) {
                    st_stream(c_col + off + r, ld_i32(M.col + q));
                    if constexpr (S::kVal)
                        st_stream(reinterpret_cast<typename S::Out*>(c_val) + off + r,
                                  S::out(slots[q - m0]));
                } else {
                    flag_overflow(st, i);
                }
            }
            rank += __popc(tm);
        }
    }
}

// ---- launchers --------------------------------------------------------------------

struct MaskedAccLaunch {
    DCsr A, B, M;
    int64_t nnz_m;
    void* slots;
    uint8_t* touched;
    int64_t* cnt;   // C's row pointers: counts, then scanned in place
    int64_t* part;
    const DevInfo* dev;
    cudaStream_t st;
    cudaError_t err = cudaSuccess;
    template <class S> void operator()() {
        using Slot = typename S::Slot;
        const int grid = dev->sms * 8;
        if (nnz_m > 0)
            k_mask_init<S><<<grid, 256, 0, st>>>(nnz_m, (Slot*)slots, touched);
        if (A.nrows > 0 && nnz_m > 0)
            k_mask_acc<S><<<grid, 256, 0, st>>>(A, B, M, (Slot*)slots, touched);
        if (M.nrows > 0) k_mask_count<<<grid, 256, 0, st>>>(M, touched, cnt);
        count_launch(*dev, 3);
        err = cudaGetLastError();
        if (err == cudaSuccess) err = launch_scan_inplace(cnt, M.nrows, part, st);
    }
};

cudaError_t launch_masked_count(int sr, const DCsr& A, const DCsr& B, const DCsr& M,
                                int64_t nnz_m, void* slots, uint8_t* touched, int64_t* cnt,
                                int64_t* part, const DevInfo& dev, cudaStream_t st) {
    MaskedAccLaunch f{A, B, M, nnz_m, slots, touched, cnt, part, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    return f.err;
}

struct MaskedWriteLaunch {
    DCsr M;
    const void* slots;
    const uint8_t* touched;
    const int64_t* c_rp;
    int32_t* c_col;
    void* c_val;
    DevStatus* status;
    const DevInfo* dev;
    cudaStream_t st;
    template <class S> void operator()() {
        if (M.nrows <= 0) return;
        k_mask_write<S><<<dev->sms * 8, 256, 0, st>>>(M, (const typename S::Slot*)slots, touched,
                                                       c_rp, c_col, c_val, status);
        count_launch(*dev);
    }
};

cudaError_t launch_masked_write(int sr, const DCsr& M, const void* slots, const uint8_t* touched,
                                const int64_t* c_rp, int32_t* c_col, void* c_val,
                                DevStatus* status, const DevInfo& dev, cudaStream_t st) {
    MaskedWriteLaunch f{M, slots, touched, c_rp, c_col, c_val, status, &dev, st};
    if (!dispatch_semiring(sr, f)) return cudaErrorInvalidValue;
    return cudaGetLastError();
}

struct SlotBytes {
    size_t out = 0;
    template <class S> void operator()() { out = sizeof(typename S::Slot); }
};

size_t masked_slot_bytes(int sr) {
    SlotBytes f;
    dispatch_semiring(sr, f);
    return f.out;
}

}  // namespace spg
