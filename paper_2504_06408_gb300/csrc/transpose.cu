// CSR transpose A -> A^T (values carried), the data movement behind the
// identity AB = (B^T A^T)^T (Section 3.1) and behind C = A A^T for the k-mer
// overlap workload.
//
// 1. t_rp[j] = number of entries in column j (atomics), exclusive scan.
// 2. Every entry e of A is scattered to a free position of its column's
//    segment (atomic cursor); what is scattered is e - A.rp[0], its number
//    inside A (A may be a row view whose first entry is far into the
//    arrays), which fits int32 because nnz < 2^31 - 1.  Entry numbers grow
//    with the row index, so sorting a segment by them orders it by row.
// 3. Each segment is sorted (warp registers <= 32, CTA shared memory <= 16384,
//    otherwise a CTA bitonic sort in a global scratch area of next_pow2(len)
//    <= 2 len slots at 2 * t_rp[j]).
// 4. Gather: e = A.rp[0] + the stored number; t_col = row of e (binary search
//    in A's row pointers), t_val = A.val[e].
#include "plan.h"
#include "rowwork.cuh"

namespace spg {

constexpr int kTSmemKeys = 16384;

// entries of A are A.col[A.rp[0] .. A.rp[0] + nnz) (A may be a row view)
__global__ void k_t_count(DCsr A, int64_t nnz, int64_t* t_rp) {
    const int64_t e0 = A.rp[0];
    for (int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e0 + nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd((unsigned long long*)(t_rp + A.col[e]), 1ull);
}

__global__ void k_t_scatter(DCsr A, int64_t nnz, const int64_t* t_rp, int32_t* cursor,
                            int32_t* t_col) {
    const int64_t e0 = A.rp[0];
    for (int64_t e = e0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < e0 + nnz;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t j = A.col[e];
        const int32_t r = atomicAdd(cursor + j, 1);
        t_col[t_rp[j] + r] = (int32_t)(e - e0);
    }
}

// 32 columns per warp (coalesced lengths): segments of 2..32 entries are sorted
// by the warp in registers, one after another; longer ones are listed for the
// CTA sort (most of a wide A^T's columns are empty or single).
__global__ void k_t_sort_warp(int64_t ncols, const int64_t* t_rp, int32_t* t_col,
                              int32_t* long_list, int32_t* n_long) {
    const int lane = lane_id();
    const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t j0 = ((int64_t)blockIdx.x * (blockDim.x >> 5) + warp_id()) * 32; j0 < ncols;
         j0 += nw * 32) {
        const int64_t j = j0 + lane;
        int64_t a = 0, len = 0;
        if (j < ncols) {
            a = t_rp[j];
            len = t_rp[j + 1] - a;
        }
        const unsigned lg = __ballot_sync(kFull, len > 32);
        if (lg) {
            const int leader = __ffs(lg) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(n_long, __popc(lg));
            base = __shfl_sync(kFull, base, leader);
            if (len > 32) long_list[base + __popc(lg & ((1u << lane) - 1))] = (int32_t)j;
        }
        unsigned sm = __ballot_sync(kFull, len > 1 && len <= 32);
        while (sm) {
            const int src = __ffs(sm) - 1;
            sm &= sm - 1;
            const int64_t sa = __shfl_sync(kFull, a, src);
            const int sl = (int)__shfl_sync(kFull, len, src);
            int32_t v = lane < sl ? t_col[sa + lane] : INT32_MAX;
            v = warp_bitonic_sort32(v);
            if (lane < sl) t_col[sa + lane] = v;
        }
    }
}

// CTA per listed segment (longer than 32); those longer than kTSmemKeys sort in
// a global scratch area
__global__ void __launch_bounds__(512) k_t_sort_block(const int64_t* t_rp, int32_t* t_col,
                                                      int32_t* scratch,
                                                      const int32_t* __restrict__ long_list,
                                                      const int32_t* __restrict__ n_long) {
    extern __shared__ int32_t buf[];   // kTSmemKeys
    const int n = *n_long;
    for (int r = blockIdx.x; r < n; r += gridDim.x) {
        const int64_t j = long_list[r];
        const int64_t a = t_rp[j], len = t_rp[j + 1] - a;
        int64_t N = 1;
        while (N < len) N <<= 1;
        int32_t* b = N <= kTSmemKeys ? buf : scratch + 2 * a;
        for (int64_t t = threadIdx.x; t < N; t += blockDim.x)
            b[t] = t < len ? t_col[a + t] : INT32_MAX;
        __syncthreads();
        smem_bitonic_sort(b, (int)N, threadIdx.x, blockDim.x, [] { __syncthreads(); });
        for (int64_t t = threadIdx.x; t < len; t += blockDim.x) t_col[a + t] = b[t];
        __syncthreads();
    }
}

__global__ void k_t_gather(DCsr A, int64_t nnz, int value_bytes, int32_t* t_col, void* t_val) {
    const int64_t e0 = A.rp[0];
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = e0 + t_col[p];
        // row of entry e: last i with rp[i] <= e
        int64_t lo = 0, hi = A.nrows - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (A.rp[mid] <= e) lo = mid; else hi = mid - 1;
        }
        if (value_bytes == 8)
            reinterpret_cast<uint64_t*>(t_val)[p] = reinterpret_cast<const uint64_t*>(A.val)[e];
        else if (value_bytes == 4)
            reinterpret_cast<uint32_t*>(t_val)[p] = reinterpret_cast<const uint32_t*>(A.val)[e];
        else if (value_bytes > 0)
            for (int b = 0; b < value_bytes; ++b)
                reinterpret_cast<char*>(t_val)[p * value_bytes + b] =
                    reinterpret_cast<const char*>(A.val)[e * value_bytes + b];
        t_col[p] = (int32_t)lo;
    }
}

size_t transpose_ws_bytes(int64_t ncols, int64_t nnz) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(sizeof(int32_t) * (size_t)ncols) + al(sizeof(int64_t) * (size_t)scan_parts_needed(ncols)) +
           al(sizeof(int32_t) * 2 * (size_t)nnz) + al(sizeof(int32_t) * (size_t)(ncols + 1));
}

cudaError_t launch_transpose(const DCsr& A, int64_t nnz, int value_bytes, int64_t* t_rp,
                             int32_t* t_col, void* t_val, void* ws, const DevInfo& dev,
                             cudaStream_t st) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const int64_t n = A.ncols;
    char* b = (char*)ws;
    int32_t* cursor = (int32_t*)b;
    int64_t* part = (int64_t*)(b + al(sizeof(int32_t) * (size_t)n));
    int32_t* scratch = (int32_t*)((char*)part + al(sizeof(int64_t) * (size_t)scan_parts_needed(n)));
    int32_t* long_list = (int32_t*)((char*)scratch + al(sizeof(int32_t) * 2 * (size_t)nnz));
    int32_t* n_long = long_list + n;
    cudaError_t e = cudaMemsetAsync(t_rp, 0, sizeof(int64_t) * (size_t)(n + 1), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(cursor, 0, sizeof(int32_t) * (size_t)n, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(n_long, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return e;
    const int grid = dev.sms * 8;
    if (nnz > 0) k_t_count<<<grid, 256, 0, st>>>(A, nnz, t_rp);
    e = launch_scan_inplace(t_rp, n, part, st);
    if (e != cudaSuccess) return e;
    if (nnz > 0) {
        k_t_scatter<<<grid, 256, 0, st>>>(A, nnz, t_rp, cursor, t_col);
        int64_t wblocks = (n + 255) / 256;   // 8 warps x 32 columns
        if (wblocks > (int64_t)dev.sms * 16) wblocks = (int64_t)dev.sms * 16;
        k_t_sort_warp<<<(unsigned)wblocks, 256, 0, st>>>(n, t_rp, t_col, long_list, n_long);
        e = cudaFuncSetAttribute(k_t_sort_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTSmemKeys * 4);
        if (e != cudaSuccess) return e;
        k_t_sort_block<<<dev.sms * 2, 512, kTSmemKeys * 4, st>>>(t_rp, t_col, scratch, long_list,
                                                                  n_long);
        k_t_gather<<<grid, 256, 0, st>>>(A, nnz, value_bytes, t_col, t_val);
    }
    return cudaGetLastError();
}

}  // namespace spg
