// A CSR transpose that allocates no memory, for callers that cannot call
// cudaMalloc at the point where they need the transpose: code running
// inside a CUDA-graph-building framework that forbids allocation, a custom
// allocator's own callbacks, or a process whose device memory is already
// reserved by a pool it does not own.  The same kernels as spgemm_transpose
// run; their scratch (per-column cursors, scan partials, sort buffer) lives in
// one file-scope device array of kNoAllocScratchBytes, which every GPU that
// loads this library holds until the process exits.  The caller still
// provides the input and the outputs.
#include <mutex>

#include "../../include/spgemm.h"
#include "plan.h"

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Per device: the array's device address, looked up by the first call that
// succeeds (a lookup that failed, e.g. during a stream capture, is retried by
// the next call rather than remembered).
struct DeviceSetup {
    std::mutex mu;
    bool done = false;
    void* scratch = nullptr;   // device address of g_noalloc_scratch on this device
    int sms = 0;
};
DeviceSetup g_setup[kMaxDevices];

}  // namespace

extern "C" spg_status spgemm_transpose_noalloc(const spg_csr* A, int value_bytes,
                                                int64_t* t_row_ptr, int32_t* t_col,
                                                void* t_val, void* stream) {
    if (!A || A->nrows < 0 || A->ncols < 0 || A->nnz < 0 || !A->row_ptr) return SPG_ERR_INVALID_ARG;
    if (A->nnz > 0 && !A->col) return SPG_ERR_INVALID_ARG;
    if (value_bytes < 0 || value_bytes > 64) return SPG_ERR_INVALID_ARG;
    if (value_bytes > 0 && A->nnz > 0 && (!A->val || !t_val)) return SPG_ERR_INVALID_ARG;
    if (!t_row_ptr || (A->nnz > 0 && !t_col)) return SPG_ERR_INVALID_ARG;
    if (A->nrows >= INT32_MAX || A->ncols >= INT32_MAX || A->nnz >= INT32_MAX)
        return SPG_ERR_UNSUPPORTED;
    if (spg::transpose_ws_bytes(A->ncols, A->nnz) > kNoAllocScratchBytes) return SPG_ERR_UNSUPPORTED;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPG_ERR_CUDA;
    // once per device, with that device current: the array's device address
    DeviceSetup& s = g_setup[dev];
    void* scratch = nullptr;
    int sms = 0;
    {
        std::lock_guard<std::mutex> lock(s.mu);
        if (!s.done) {
            void* p = nullptr;
            int n = 0;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p ||
                cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                cudaGetLastError();   // clear the error so the next call can retry
                return SPG_ERR_CUDA;
            }
            s.scratch = p;
            s.sms = n;
            s.done = true;
        }
        scratch = s.scratch;
        sms = s.sms;
    }
    spg::DevInfo di{sms, 0};
    const spg::DCsr a{A->nrows, A->ncols, A->row_ptr, A->col, A->val};
    const cudaError_t e = spg::launch_transpose(a, A->nnz, value_bytes, t_row_ptr, t_col, t_val,
                                                scratch, di, (cudaStream_t)stream);
    return e == cudaSuccess ? SPG_OK : SPG_ERR_CUDA;
}
