// spmm_csr_noalloc: the merge-based SpMM (and the rest of spmm_csr_ex) for
// callers that cannot allocate device memory at call time.
//
// Who needs it: code that runs inside a host that owns all device memory and
// forbids its plugins from calling the CUDA allocator (inference-server and
// solver plugins, for instance), and real-time loops that must not risk
// allocator latency or an out-of-memory failure in the middle of a run.  Such
// callers cannot use spmm_csr (which obtains the merge workspace with
// cudaMallocAsync) and may have no buffer of their own to lend to spmm_csr_ex.
//
// The merge-based path needs scratch memory (tile boundaries, and the partial
// sums of rows that cross tiles).  Here that scratch is a fixed array in
// device global memory, reserved when the library's device code is loaded on
// a device (with CUDA's default lazy loading, at the first merge-path call on
// that device) and held until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/spmm.h"

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;  // 16 MiB per device

// The scratch.  In host code this name is only a stand-in for the device
// array: its device address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_spmm_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this look-up).
int scratch_address(void** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPMM_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_spmm_static_scratch) != cudaSuccess || p == nullptr) return SPMM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SPMM_OK;
}

}  // namespace

extern "C" {

size_t spmm_csr_static_scratch_bytes(void) { return kStaticScratchBytes; }

int spmm_csr_noalloc(int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind, const void* vals,
                     int vals_type, const void* B, int b_type, long long ldb, void* C, int c_type, long long ldc,
                     int alg, const spmm_tuning_t* tuning, int* d_status, void* stream) {
    if (m < 0 || k < 0 || n < 0 || nnz < -1) return SPMM_ERR_INVALID_VALUE;
    if (alg < SPMM_ALG_AUTO || alg > SPMM_ALG_MERGE) return SPMM_ERR_INVALID_VALUE;
    if (m == 0 || n == 0) return SPMM_OK;
    if (!row_ptr) return SPMM_ERR_INVALID_VALUE;
    if (nnz < 0) {  // 4-byte read into a host variable: synchronises the stream, allocates nothing
        int v = 0;
        if (cudaMemcpyAsync(&v, row_ptr + m, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
                cudaSuccess ||
            cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
            return SPMM_ERR_CUDA;
        if (v < 0) return SPMM_ERR_BAD_CSR;
        nnz = v;
    }
    const double threshold = tuning ? tuning->merge_threshold : 0.0;
    const int a = alg == SPMM_ALG_AUTO ? spmm_select_alg(m, nnz, threshold) : alg;
    if (a != SPMM_ALG_MERGE)  // row split needs no scratch
        return spmm_csr_ex(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, a,
                           tuning, nullptr, 0, d_status, stream);
    // spmm_csr_ex checks the exact scratch of the launch shape it picks against the array's size and
    // returns SPMM_ERR_WORKSPACE, before any device work, when the problem does not fit
    void* ws = nullptr;
    const int st = scratch_address(&ws);
    if (st != SPMM_OK) return st;
    return spmm_csr_ex(m, k, n, nnz, row_ptr, col_ind, vals, vals_type, B, b_type, ldb, C, c_type, ldc, a, tuning,
                       ws, kStaticScratchBytes, d_status, stream);
}

}  // extern "C"
