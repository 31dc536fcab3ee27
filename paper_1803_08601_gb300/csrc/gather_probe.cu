// Gather-rate probe: the memory-system ceiling under every SpMM kernel here.
//
// Each nonzero of A makes the SpMM kernels read one whole row of B at a
// random row index (Section 4.1: "each thread loads a column of B", so a
// lane group reads one row of B with coalesced 16-byte accesses).  This
// kernel does only that: lane groups of row_bytes / 16 lanes read rows of B
// at the indices idx[0 .. count), eight rows in flight per lane, and fold the
// words they read into one word so that no load can be dropped.  Its rate over
// B sizes and row widths gives the gather ceilings (L2-resident and HBM) and
// the effective L2 capacity that bound the SpMM kernels' rooflines.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/spmm.h"

namespace spmm {
extern std::atomic<long long> g_launches;
}

namespace {

constexpr int kProbeThreads = 256;
constexpr int kProbeInFlight = 8;

template <int W>
__global__ void __launch_bounds__(kProbeThreads) gather_probe_kernel(const uint4* __restrict__ B, long long rows,
                                                                     const int* __restrict__ idx, long long count,
                                                                     unsigned* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int sl = lane & (W - 1);
    const long long group = ((long long)blockIdx.x * kProbeThreads + threadIdx.x) / W;
    const long long groups = (long long)gridDim.x * kProbeThreads / W;
    unsigned acc = 0;
    for (long long i = group * kProbeInFlight; i < count; i += groups * kProbeInFlight) {
        int r[kProbeInFlight];
#pragma unroll
        for (int u = 0; u < kProbeInFlight; ++u) r[u] = i + u < count ? __ldg(idx + i + u) : -1;
        uint4 v[kProbeInFlight];
#pragma unroll
        for (int u = 0; u < kProbeInFlight; ++u)
            v[u] = (r[u] >= 0 && r[u] < rows) ? __ldg(B + (long long)r[u] * W + sl) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int u = 0; u < kProbeInFlight; ++u) acc ^= v[u].x ^ v[u].y ^ v[u].z ^ v[u].w;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc ^= __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) atomicXor(out, acc);
}

template <int W>
cudaError_t launch(const void* B, long long rows, const int* idx, long long count, unsigned* out, cudaStream_t st) {
    int dev = 0, sms = 0, blocks = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, gather_probe_kernel<W>, kProbeThreads, 0);
    if (e != cudaSuccess) return e;
    const long long grid = (long long)(blocks < 1 ? 1 : blocks) * sms;
    gather_probe_kernel<W><<<(unsigned)grid, kProbeThreads, 0, st>>>(static_cast<const uint4*>(B), rows, idx, count,
                                                                      out);
    e = cudaGetLastError();
    if (e == cudaSuccess) spmm::g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

}  // namespace

extern "C" int spmm_gather_probe(const void* B, long long rows, int row_bytes, const int* idx, long long count,
                                 unsigned* out, void* stream) {
    if (rows < 0 || count < 0 || !out || (count > 0 && (!B || !idx))) return SPMM_ERR_INVALID_VALUE;
    if (((uintptr_t)B % 16) != 0) return SPMM_ERR_INVALID_VALUE;
    if (count == 0) return SPMM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    switch (row_bytes) {
        case 16: e = launch<1>(B, rows, idx, count, out, st); break;
        case 32: e = launch<2>(B, rows, idx, count, out, st); break;
        case 64: e = launch<4>(B, rows, idx, count, out, st); break;
        case 128: e = launch<8>(B, rows, idx, count, out, st); break;
        case 256: e = launch<16>(B, rows, idx, count, out, st); break;
        case 512: e = launch<32>(B, rows, idx, count, out, st); break;
        default: return SPMM_ERR_INVALID_VALUE;
    }
    return e == cudaSuccess ? SPMM_OK : SPMM_ERR_LAUNCH;
}
