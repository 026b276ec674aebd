// Shared device helpers of the SpGEMM kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#define SPG_DEV __device__ __forceinline__

namespace spg {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int32_t kEmptyKey = -1;          // free hash slot
constexpr int kWarp = 32;

// One CSR matrix as the kernels see it.
struct DCsr {
    int64_t nrows, ncols;
    const int64_t* rp;
    const int32_t* col;
    const void* val;
};

// One product C = A (x).(+) B of a batch.  Rows of all products of a batch
// are numbered consecutively ("flat rows"): flat row g of product p is row
// g - row_base of A.
struct Prob {
    DCsr A, B;
    // B packed by 32-column words for the symbolic dense tier: row k lists the
    // distinct words w of B_k's columns (ascending, col = w) with the mask of
    // B_k's columns in w (val, uint32); rp == nullptr when not built
    DCsr Bw;
    // slab starts of B's rows for the numeric dense tier: sp[k * stride + s] =
    // offset in row k of its first column >= s * slab width (stride = the
    // launch's slab count + 1); nullptr: none (per-entry cursors instead)
    const int32_t* sp;
    int64_t* c_rp;       // output row pointers [A.nrows + 1]
    int32_t* c_col;      // output columns [nnz(C)]
    void* c_val;         // output values  [nnz(C)]
    int64_t row_base;    // first flat row
    int64_t nnz_base;    // first entry of A in the flat entry numbering (cursors); entry p
                         // of row-view A is flat entry nnz_base + (p - A.rp[0])
};

// Kernel-detected errors, kept in the workspace.
struct DevStatus {
    int32_t overflow;    // a hash table ran out of slots
    int32_t unused;
    int32_t invalid;     // validation failure
    int32_t pad;
    int64_t info[5];     // first offending flat row etc.
};

SPG_DEV int lane_id() { return threadIdx.x & 31; }
SPG_DEV int warp_id() { return threadIdx.x >> 5; }

template <class T>
SPG_DEV T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <class T>
SPG_DEV T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// inclusive prefix sum across the warp
template <class T>
SPG_DEV T warp_incl_scan(T v) {
    const int l = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T w = __shfl_up_sync(kFull, v, o);
        if (l >= o) v += w;
    }
    return v;
}

// Store that streams past L2 (evict-first): output written once and not read
// back by the kernel, so it does not push the input matrices out of L2.
template <class T>
SPG_DEV void st_stream(T* p, const T& v) {
    if constexpr (sizeof(T) == 4 && alignof(T) >= 4) {
        __stcs(reinterpret_cast<unsigned int*>(p), *reinterpret_cast<const unsigned int*>(&v));
    } else if constexpr (sizeof(T) == 8 && alignof(T) >= 8) {
        __stcs(reinterpret_cast<unsigned long long*>(p),
               *reinterpret_cast<const unsigned long long*>(&v));
    } else {
        *p = v;
    }
}

SPG_DEV int64_t ld_i64(const int64_t* p) { return __ldg(p); }

// Bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16); a hint, nothing waits for it.
SPG_DEV void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;"
                 :: "l"(__cvta_generic_to_global(p)), "r"(bytes) : "memory");
}
SPG_DEV int32_t ld_i32(const int32_t* p) { return __ldg(p); }

// Fibonacci hashing of a column id into a table of 2^(32 - shift) slots
// (shift in [1, 31]): the high bits of key * 2^32 / golden ratio.
SPG_DEV uint32_t hash_slot(int32_t key, int shift) {
    return ((uint32_t)key * 2654435769u) >> shift;
}

SPG_DEV int log2_exact(int64_t pow2) { return 63 - __clzll(pow2); }

// Position of the k-th (0-based) set bit of x, by halving on popcounts;
// requires k < popc(x).
SPG_DEV int select_bit(uint32_t x, int k) {
    int pos = 0;
    int c = __popc(x & 0xffffu);
    if (k >= c) { k -= c; x >>= 16; pos += 16; }
    c = __popc(x & 0xffu);
    if (k >= c) { k -= c; x >>= 8; pos += 8; }
    c = __popc(x & 0xfu);
    if (k >= c) { k -= c; x >>= 4; pos += 4; }
    c = __popc(x & 0x3u);
    if (k >= c) { k -= c; x >>= 2; pos += 2; }
    if (k >= (int)(x & 1u)) pos += 1;
    return pos;
}

__host__ __device__ inline int64_t next_pow2(int64_t x) {
    int64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Flat row -> product index (batches are small; linear/binary search).
SPG_DEV int find_prob(const Prob* probs, int nprob, int64_t g) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (probs[mid].row_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

SPG_DEV void flag_overflow(DevStatus* st, int64_t g) {
    if (atomicExch(&st->overflow, 1) == 0) st->info[0] = g;
}

// A data-dependent index found out of range (checked build): recorded, and the
// access it would have made is skipped.
SPG_DEV void flag_invalid(DevStatus* st, int64_t info) {
    if (atomicExch(&st->invalid, 1) == 0) st->info[1] = info;
}

}  // namespace spg
