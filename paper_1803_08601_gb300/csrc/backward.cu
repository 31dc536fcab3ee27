// Operations of the backward pass of C = A B with respect to the stored
// values of A and to B (the paper's SpMM_T, named as future work in
// Section 6, plus the sampled dense-dense product):
//   dB    = A^T dC      : spmm_csr_ex on A^T, built once by spmm_csr_transpose
//   dvals = SDDMM(dC, B): dvals[p] = <dC[row(p), :], B[col(p), :]>
//
// CSR transpose: a stable sort of the nonzeros by column index (LSD radix
// sort, 8 bits per pass, the original position as payload), so row c of A^T
// lists the nonzeros of column c in increasing original position.  Every step
// is deterministic; the permutation lets vals^T be refreshed with one gather
// when the values change but the pattern does not.
//
// SDDMM: balanced by nonzero split (Section 4 item 2(a)): every lane group
// takes an equal run of consecutive nonzeros and finds its first row by a
// binary search on row_ptr, so a long row is shared by many groups.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "launch.cuh"

namespace spmm {
namespace {

constexpr int kRadix = 256;
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kScanThreads = 1024;

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return SPMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPMM_ERR_ALLOC;
    if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidValue)
        return SPMM_ERR_LAUNCH;
    return SPMM_ERR_CUDA;
}

int launched(cudaError_t e) {
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return status_of(e);
}

int radix_passes(int k) {
    int bits = 0;
    while (bits < 31 && ((long long)(k > 0 ? k - 1 : 0) >> bits) > 0) ++bits;
    const int p = (bits + 7) / 8;
    return p < 1 ? 1 : p;
}

struct TransposeLayout {
    int tiles;
    size_t off_k0, off_k1, off_v, off_hist, off_tot, total;
};

TransposeLayout transpose_layout(long long nnz) {
    TransposeLayout L{};
    L.tiles = (int)((nnz + kSortTile - 1) / kSortTile);
    size_t off = 0;
    L.off_k0 = off;
    off = a256(off + (size_t)nnz * 4);
    L.off_k1 = off;
    off = a256(off + (size_t)nnz * 4);
    L.off_v = off;
    off = a256(off + (size_t)nnz * 4);
    L.off_hist = off;
    off = a256(off + (size_t)kRadix * (L.tiles > 0 ? L.tiles : 1) * 4);
    L.off_tot = off;
    off = a256(off + (size_t)kRadix * 4);
    L.total = off;
    return L;
}

// Per-tile histogram of one 8-bit digit; hist is digit-major [256][tiles].
__global__ void radix_hist_kernel(const int* __restrict__ keys, long long n, int shift, int tiles,
                                  int* __restrict__ hist) {
    __shared__ int cnt[kRadix];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
    for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
        const long long idx = base + i;
        if (idx < n) atomicAdd(&cnt[(__ldg(keys + idx) >> shift) & (kRadix - 1)], 1);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * tiles + blockIdx.x] = cnt[threadIdx.x];
}

// Exclusive prefix sums of the digit-major histogram [256][tiles]: one CTA per
// digit scans its row in place (chunks of kScanThreads coalesced elements,
// warp shuffles, a running carry) and leaves the row's total in totals[d];
// digit_base_kernel then turns the 256 totals into the digits' first
// positions, which the scatter adds to each row's prefix.
__global__ void digit_scan_kernel(int* __restrict__ hist, int tiles, int* __restrict__ totals) {
    constexpr int kWarps = kScanThreads / 32;
    __shared__ int warp_sum[kWarps];
    __shared__ int carry;
    int* row = hist + (long long)blockIdx.x * tiles;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < tiles; base += kScanThreads) {
        const int i = base + tid;
        const int v = i < tiles ? row[i] : 0;
        int x = v;  // inclusive scan inside the warp
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFullMask, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        if (warp == 0) {  // inclusive scan of the warp sums
            int w = warp_sum[lane];
#pragma unroll
            for (int off = 1; off < kWarps; off <<= 1) {
                const int y = __shfl_up_sync(kFullMask, w, off);
                if (lane >= off) w += y;
            }
            warp_sum[lane] = w;
        }
        __syncthreads();
        if (i < tiles) row[i] = carry + (warp > 0 ? warp_sum[warp - 1] : 0) + x - v;
        __syncthreads();
        if (tid == 0) carry += warp_sum[kWarps - 1];
        __syncthreads();
    }
    if (tid == 0) totals[blockIdx.x] = carry;
}

// totals[d] <- sum of totals[0..d): the first sorted position of digit d (one CTA of 256 threads).
__global__ void digit_base_kernel(int* __restrict__ totals) {
    __shared__ int warp_sum[kRadix / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int v = totals[tid];
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFullMask, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) warp_sum[warp] = x;
    __syncthreads();
    int before = 0;
    for (int w = 0; w < warp; ++w) before += warp_sum[w];
    totals[tid] = before + x - v;
}

// Stable scatter of one radix pass.  The tile is first sorted by digit in
// shared memory (counts of the tile's digits, scanned into tile-local digit
// offsets; elements placed in rounds of 256 consecutive elements, thread t
// holding element t of the round, the rank among equal digits from
// __match_any_sync inside a warp, per-warp digit counts across warps and a
// running per-digit count across rounds), then written out in that order, so
// a run of equal digits goes to consecutive global positions.  Element order
// is kept among equal digits.  payload_in == nullptr means the payload is the
// element's own index.
__global__ void radix_scatter_kernel(const int* __restrict__ keys_in, const int* __restrict__ payload_in, long long n,
                                     int shift, int tiles, const int* __restrict__ offsets,
                                     const int* __restrict__ digit_base, int* __restrict__ keys_out,
                                     int* __restrict__ payload_out) {
    constexpr int kWarps = kSortThreads / 32;
    __shared__ int s_key[kSortTile];
    __shared__ int s_pay[kSortTile];
    __shared__ int local[kRadix];  // tile-local first position of each digit
    __shared__ int run[kRadix];    // elements of each digit placed so far
    __shared__ int wcnt[kWarps][kRadix];
    __shared__ int warp_sum[kWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const long long tile0 = (long long)blockIdx.x * kSortTile;
    const int count = n - tile0 < kSortTile ? (int)(n - tile0) : kSortTile;
    run[tid] = 0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    for (int i = tid; i < count; i += kSortThreads) atomicAdd(&run[(__ldg(keys_in + tile0 + i) >> shift) & (kRadix - 1)], 1);
    __syncthreads();
    {  // exclusive scan of the tile's 256 digit counts (kSortThreads == kRadix)
        const int v = run[tid];
        int x = v;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_up_sync(kFullMask, x, off);
            if (lane >= off) x += y;
        }
        if (lane == 31) warp_sum[warp] = x;
        __syncthreads();
        int before = 0;
        for (int w = 0; w < warp; ++w) before += warp_sum[w];
        local[tid] = before + x - v;
        run[tid] = 0;
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    for (int r = 0; r < kSortItems; ++r) {
        const int i = r * kSortThreads + tid;
        const bool valid = i < count;
        const int key = valid ? __ldg(keys_in + tile0 + i) : 0;
        const int pay = valid ? (payload_in ? __ldg(payload_in + tile0 + i) : (int)(tile0 + i)) : 0;
        const int d = valid ? (key >> shift) & (kRadix - 1) : kRadix + lane;  // invalid lanes match nobody
        const unsigned peers = __match_any_sync(kFullMask, d);
        const int rank = __popc(peers & lt_mask);
        if (valid && lane == 31 - __clz(peers)) wcnt[warp][d] = __popc(peers);
        __syncthreads();
        if (valid) {
            int pos = local[d] + run[d] + rank;
            for (int w = 0; w < warp; ++w) pos += wcnt[w][d];
            s_key[pos] = key;
            s_pay[pos] = pay;
        }
        __syncthreads();
        int tot = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            tot += wcnt[w][tid];
            wcnt[w][tid] = 0;
        }
        run[tid] += tot;
        __syncthreads();
    }
    // write out in tile order: element i of digit d goes to the digit's global run for this tile
    local[tid] = offsets[(long long)tid * tiles + blockIdx.x] + digit_base[tid] - local[tid];
    __syncthreads();
    for (int i = tid; i < count; i += kSortThreads) {
        const int key = s_key[i];
        const int pos = local[(key >> shift) & (kRadix - 1)] + i;
        keys_out[pos] = key;
        payload_out[pos] = s_pay[i];
    }
}

// row_ptr_t[c] = first position of column c in the sorted keys (lower bound).
__global__ void transpose_rowptr_kernel(const int* __restrict__ sorted_keys, long long nnz, int k,
                                        int* __restrict__ row_ptr_t) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > k) return;
    long long lo = 0, hi = nnz;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (__ldg(sorted_keys + mid) < c) lo = mid + 1;
        else hi = mid;
    }
    row_ptr_t[c] = (int)lo;
}

// rows[p] = the row of A holding nonzero p, for every p (a warp per row).
__global__ void expand_rows_kernel(const int* __restrict__ row_ptr, int m, int* __restrict__ rows) {
    const long long r = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (r >= m) return;
    const int lane = threadIdx.x & 31;
    const int p1 = __ldg(row_ptr + r + 1);
    for (int p = __ldg(row_ptr + r) + lane; p < p1; p += 32) rows[p] = (int)r;
}

template <typename T>
__global__ void gather_values_kernel(const int* __restrict__ perm, long long nnz, const T* __restrict__ vals,
                                     T* __restrict__ out) {
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (long long)gridDim.x * blockDim.x)
        out[q] = vals[__ldg(perm + q)];
}

// ------------------------------------------------------------------------------------- SDDMM

struct SddmmArgs {
    int m, n;
    long long nnz;
    const int* row_ptr;
    const int* col_ind;
    const void* dC;
    long long lddc;
    const void* B;
    long long ldb;
    void* out;
    int chunk;  // nonzeros per lane group
};

// One lane group of W lanes per run of `chunk` consecutive nonzeros; each lane
// owns the columns chunk j = sl, sl + W, ... (VEC elements each) of both rows;
// kUnroll nonzeros are processed together and their partial dot products are
// reduced across the group with xor shuffles.
template <typename TD, typename TO, int VEC, int W>
__global__ void __launch_bounds__(kThreads) sddmm_kernel(SddmmArgs a) {
    constexpr int U = kUnroll;
    const int lane = threadIdx.x & 31, sl = lane & (W - 1);
    const long long g = ((long long)blockIdx.x * kThreads + threadIdx.x) / W;
    const long long p0 = g * a.chunk;
    const long long p1 = p0 + a.chunk < a.nnz ? p0 + a.chunk : a.nnz;
    const TD* __restrict__ dC = static_cast<const TD*>(a.dC);
    const TD* __restrict__ B = static_cast<const TD*>(a.B);
    const int nchunks = (a.n + VEC - 1) / VEC;
    int row = 0, row_end = 0;
    if (p0 < p1) {  // last row whose start is <= p0
        int lo = 0, hi = a.m;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(a.row_ptr + mid) <= p0) lo = mid;
            else hi = mid - 1;
        }
        row = lo;
        row_end = __ldg(a.row_ptr + row + 1);
    }
    const int nb = p0 < p1 ? (int)((p1 - p0 + U - 1) / U) : 0;
    const int nb_max = __reduce_max_sync(kFullMask, nb);
    for (int b = 0; b < nb_max; ++b) {
        float part[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long p = p0 + (long long)b * U + u;
            part[u] = 0.0f;
            if (p < p1) {
                while (p >= row_end) row_end = __ldg(a.row_ptr + (++row) + 1);
                const TD* brow = gather_row(B, 0, __ldg(a.col_ind + p), a.ldb);
                const TD* drow = dC + (long long)row * a.lddc;
                for (int j = sl; j < nchunks; j += W) {
                    const Raw<TD, VEC> x = load_raw<TD, VEC>(brow + (long long)j * VEC);
                    float y[VEC];
                    load_vec<TD, VEC>(drow + (long long)j * VEC, y);
                    float t[VEC];
#pragma unroll
                    for (int e = 0; e < VEC; ++e) t[e] = 0.0f;
                    fma_raw<TD, VEC>(t, 1.0f, x);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) part[u] = fmaf(t[e], y[e], part[u]);
                }
            }
        }
#pragma unroll
        for (int off = W / 2; off > 0; off >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(kFullMask, part[u], off, W);
        if (sl == 0) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const long long p = p0 + (long long)b * U + u;
                if (p < p1) static_cast<TO*>(a.out)[p] = Elem<TO>::from_f(part[u]);
            }
        }
    }
}

// Wide rows (16 to 256 16-byte vectors): a warp per run of `chunk`
// consecutive nonzeros.  Its first row comes from a 32-ary warp search of
// row_ptr; the current row of dC stays in registers (lane l holds vectors
// l, l + 32, ...) and is reloaded only when the row changes; up to U nonzeros
// of one row are done together, their rows of B gathered with independent
// loads (U * CPL vectors in flight per lane), and each dot product is reduced
// across the warp with xor shuffles in the same order as sddmm_kernel.
template <typename TD, typename TO, int CPL, int U>
__global__ void __launch_bounds__(kThreads) sddmm_warp_kernel(SddmmArgs a) {
    constexpr int VEC = Elem<TD>::kVec;
    const int lane = threadIdx.x & 31;
    const long long wid = ((long long)blockIdx.x * kThreads + threadIdx.x) >> 5;
    const long long p0 = wid * a.chunk;
    if (p0 >= a.nnz) return;  // whole warps leave together
    const long long p1 = p0 + a.chunk < a.nnz ? p0 + a.chunk : a.nnz;
    const TD* __restrict__ dC = static_cast<const TD*>(a.dC);
    const TD* __restrict__ B = static_cast<const TD*>(a.B);
    const int nchunks = a.n / VEC;
    // first row: the largest r with row_ptr[r] <= p0 (row_ptr[0] = 0 <= p0 always holds)
    int lo = 0, hi = a.m;  // answer in [lo, hi)
    while (hi - lo > 1) {
        const long long span = hi - lo;
        const int x = lo + (int)((span * lane) / 32);
        const unsigned ball = __ballot_sync(kFullMask, (long long)__ldg(a.row_ptr + x) <= p0);
        const int cnt = __popc(ball);  // a prefix of the lanes, at least lane 0
        const int x_last = lo + (int)((span * (cnt - 1)) / 32);
        hi = cnt < 32 ? lo + (int)((span * cnt) / 32) : hi;
        lo = x_last;
    }
    int row = lo;
    int row_end = __ldg(a.row_ptr + row + 1);
    float y[CPL][VEC];
    auto load_row = [&]() {
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
            const int j = lane + 32 * c;
            if (j < nchunks) load_vec<TD, VEC>(dC + (long long)row * a.lddc + (long long)j * VEC, y[c]);
            else
#pragma unroll
                for (int e = 0; e < VEC; ++e) y[c][e] = 0.0f;
        }
    };
    load_row();
    for (long long p = p0; p < p1;) {
        if (p >= row_end) {  // warp-uniform: the next nonzero belongs to a later row
            do {
                ++row;
                row_end = __ldg(a.row_ptr + row + 1);
            } while (p >= row_end);
            load_row();
        }
        const long long pe = p1 < (long long)row_end ? p1 : (long long)row_end;
        const int cnt = pe - p < U ? (int)(pe - p) : U;
        int cols[U];
#pragma unroll
        for (int u = 0; u < U; ++u) cols[u] = u < cnt ? __ldg(a.col_ind + p + u) : 0;
        Raw<TD, VEC> x[U][CPL];
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                const int j = lane + 32 * c;
                x[u][c] = (u < cnt && j < nchunks) ? load_raw<TD, VEC>(gather_row(B, (long long)j * VEC, cols[u], a.ldb))
                                                   : zero_raw<TD, VEC>();
            }
        float part[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            part[u] = 0.0f;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
                float t[VEC];
#pragma unroll
                for (int e = 0; e < VEC; ++e) t[e] = 0.0f;
                fma_raw<TD, VEC>(t, 1.0f, x[u][c]);
#pragma unroll
                for (int e = 0; e < VEC; ++e) part[u] = fmaf(t[e], y[c][e], part[u]);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
#pragma unroll
            for (int u = 0; u < U; ++u) part[u] += __shfl_xor_sync(kFullMask, part[u], off);
        if (lane < cnt) {
            float mine = part[0];
#pragma unroll
            for (int u = 1; u < U; ++u)
                if (lane == u) mine = part[u];
            static_cast<TO*>(a.out)[p + lane] = Elem<TO>::from_f(mine);
        }
        p += cnt;
    }
}

template <typename TD, typename TO, int VEC>
cudaError_t sddmm_launch_vec(const SddmmArgs& a, int W, long long groups, cudaStream_t st) {
    const long long blocks = (groups * W + kThreads - 1) / kThreads;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    switch (W) {
        case 1: sddmm_kernel<TD, TO, VEC, 1><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
        case 2: sddmm_kernel<TD, TO, VEC, 2><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
        case 4: sddmm_kernel<TD, TO, VEC, 4><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
        case 8: sddmm_kernel<TD, TO, VEC, 8><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
        case 16: sddmm_kernel<TD, TO, VEC, 16><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
        default: sddmm_kernel<TD, TO, VEC, 32><<<(unsigned)blocks, kThreads, 0, st>>>(a); break;
    }
    return cudaGetLastError();
}

template <typename TD, typename TO>
int sddmm_run(const SddmmArgs& a0, cudaStream_t st) {
    SddmmArgs a = a0;
    constexpr int V = Elem<TD>::kVec;
    const bool vec_ok = a.n % V == 0 && a.lddc % V == 0 && a.ldb % V == 0 && ((uintptr_t)a.dC % 16) == 0 &&
                        ((uintptr_t)a.B % 16) == 0;
    const int vec = vec_ok ? V : 1;
    const long long nchunks = ((long long)a.n + vec - 1) / vec;
    int W = 1;
    while (W < nchunks && W < 32) W <<= 1;
    // a warp per 256 nonzeros, dC rows in registers: faster than the lane groups from 16 vectors per
    // row (measured on the GCN workload: n = 64 float32 0.58 ms against 0.71; n = 32 0.56 against 0.38)
    if (vec_ok && nchunks >= 16 && nchunks <= 256) {
        a.chunk = 256;
        const long long warps = (a.nnz + a.chunk - 1) / a.chunk;
        const long long blocks = (warps * 32 + kThreads - 1) / kThreads;
        if (blocks > 0x7fffffffLL) return SPMM_ERR_LAUNCH;
        const int cpl = (int)((nchunks + 31) / 32);
        if (cpl <= 1) sddmm_warp_kernel<TD, TO, 1, 8><<<(unsigned)blocks, kThreads, 0, st>>>(a);
        else if (cpl <= 2) sddmm_warp_kernel<TD, TO, 2, 4><<<(unsigned)blocks, kThreads, 0, st>>>(a);
        else if (cpl <= 4) sddmm_warp_kernel<TD, TO, 4, 2><<<(unsigned)blocks, kThreads, 0, st>>>(a);
        else sddmm_warp_kernel<TD, TO, 8, 1><<<(unsigned)blocks, kThreads, 0, st>>>(a);
        return launched(cudaGetLastError());
    }
    a.chunk = 128;  // nonzeros per lane group: longer runs amortise the row search (n = 32: 0.38 -> 0.35 ms)
    const long long groups = (a.nnz + a.chunk - 1) / a.chunk;
    const cudaError_t e = vec_ok ? sddmm_launch_vec<TD, TO, V>(a, W, groups, st) : sddmm_launch_vec<TD, TO, 1>(a, W, groups, st);
    return launched(e);
}

}  // namespace
}  // namespace spmm

using namespace spmm;

extern "C" {

size_t spmm_csr_transpose_workspace_size(int m, int k, long long nnz) {
    if (m < 0 || k < 0 || nnz < 0) return 0;
    return transpose_layout(nnz).total;
}

int spmm_csr_transpose(int m, int k, long long nnz, const int* row_ptr, const int* col_ind, int* row_ptr_t,
                       int* col_ind_t, int* perm, void* workspace, size_t workspace_bytes, void* stream) {
    if (m < 0 || k < 0 || nnz < 0 || nnz > 0x7fffffffLL) return SPMM_ERR_INVALID_VALUE;
    if (!row_ptr_t || (nnz > 0 && (!row_ptr || !col_ind || !col_ind_t || !perm))) return SPMM_ERR_INVALID_VALUE;
    if (nnz > 0 && m == 0) return SPMM_ERR_INVALID_VALUE;
    cudaStream_t s = (cudaStream_t)stream;
    const TransposeLayout L = transpose_layout(nnz);
    if (nnz == 0) {
        const cudaError_t e = cudaMemsetAsync(row_ptr_t, 0, (size_t)(k + 1) * 4, s);
        return status_of(e);
    }
    bool own = false;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    if (!ws) {
        if (workspace_bytes != 0) return SPMM_ERR_WORKSPACE;
        void* p = nullptr;
        if (cudaMallocAsync(&p, L.total, s) != cudaSuccess) return SPMM_ERR_ALLOC;
        ws = static_cast<unsigned char*>(p);
        own = true;
    } else if (workspace_bytes < L.total) {
        return SPMM_ERR_WORKSPACE;
    }
    int* kbuf[2] = {reinterpret_cast<int*>(ws + L.off_k0), reinterpret_cast<int*>(ws + L.off_k1)};
    int* vtmp = reinterpret_cast<int*>(ws + L.off_v);
    int* hist = reinterpret_cast<int*>(ws + L.off_hist);
    int* totals = reinterpret_cast<int*>(ws + L.off_tot);
    const int passes = radix_passes(k);
    const int* kin = col_ind;
    const int* vin = nullptr;  // payload of the first pass: the element index
    int st = SPMM_OK;
    for (int pass = 0; pass < passes && st == SPMM_OK; ++pass) {
        const int shift = 8 * pass;
        int* kout = kbuf[pass & 1];
        int* vout = ((passes - 1 - pass) % 2 == 0) ? perm : vtmp;  // the last pass lands in perm
        radix_hist_kernel<<<L.tiles, kSortThreads, 0, s>>>(kin, nnz, shift, L.tiles, hist);
        st = launched(cudaGetLastError());
        if (st != SPMM_OK) break;
        digit_scan_kernel<<<kRadix, kScanThreads, 0, s>>>(hist, L.tiles, totals);
        st = launched(cudaGetLastError());
        if (st != SPMM_OK) break;
        digit_base_kernel<<<1, kRadix, 0, s>>>(totals);
        st = launched(cudaGetLastError());
        if (st != SPMM_OK) break;
        radix_scatter_kernel<<<L.tiles, kSortThreads, 0, s>>>(kin, vin, nnz, shift, L.tiles, hist, totals, kout, vout);
        st = launched(cudaGetLastError());
        kin = kout;
        vin = vout;
    }
    if (st == SPMM_OK) {
        transpose_rowptr_kernel<<<(unsigned)(((long long)k + 1 + 255) / 256), 256, 0, s>>>(kin, nnz, k, row_ptr_t);
        st = launched(cudaGetLastError());
    }
    if (st == SPMM_OK) {  // col_ind_t[q] = row of perm[q]: rows expanded into the free key buffer, then gathered
        int* rows = kbuf[passes & 1];
        expand_rows_kernel<<<(unsigned)(((long long)m * 32 + 255) / 256), 256, 0, s>>>(row_ptr, m, rows);
        st = launched(cudaGetLastError());
        if (st == SPMM_OK) {
            gather_values_kernel<int><<<(unsigned)std::min<long long>((nnz + 255) / 256, 152LL * 16), 256, 0, s>>>(
                perm, nnz, rows, col_ind_t);
            st = launched(cudaGetLastError());
        }
    }
    if (own) {
        const cudaError_t e = cudaFreeAsync(ws, s);
        if (st == SPMM_OK && e != cudaSuccess) st = status_of(e);
    }
    return st;
}

int spmm_gather_values(long long nnz, const int* perm, const void* vals, int vals_type, void* out, void* stream) {
    if (nnz < 0 || (nnz > 0 && (!perm || !vals || !out))) return SPMM_ERR_INVALID_VALUE;
    if (vals_type != SPMM_F32 && vals_type != SPMM_BF16 && vals_type != SPMM_F16) return SPMM_ERR_UNSUPPORTED;
    if (nnz == 0) return SPMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const unsigned blocks = (unsigned)std::min<long long>((nnz + 255) / 256, 152LL * 16);
    if (vals_type == SPMM_F32)
        gather_values_kernel<float><<<blocks, 256, 0, s>>>(perm, nnz, (const float*)vals, (float*)out);
    else
        gather_values_kernel<unsigned short><<<blocks, 256, 0, s>>>(perm, nnz, (const unsigned short*)vals,
                                                                     (unsigned short*)out);
    return launched(cudaGetLastError());
}

int sddmm_csr(int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind, const void* dC, int dc_type,
              long long lddc, const void* B, int b_type, long long ldb, void* out, int out_type, void* stream) {
    if (m < 0 || k < 0 || n < 0 || nnz < 0 || nnz > 0x7fffffffLL) return SPMM_ERR_INVALID_VALUE;
    if (nnz == 0) return SPMM_OK;
    if (!row_ptr || !col_ind || !out || m == 0 || k == 0) return SPMM_ERR_INVALID_VALUE;
    if (n > 0 && (!dC || !B || lddc < n || ldb < n)) return SPMM_ERR_INVALID_VALUE;
    if (dc_type != b_type) return SPMM_ERR_UNSUPPORTED;
    if (ldb * (b_type == SPMM_F32 ? 4LL : 2LL) > 0xffffffffLL) return SPMM_ERR_INVALID_VALUE;  // rows of B < 4 GiB apart
    SddmmArgs a{m, n, nnz, row_ptr, col_ind, dC, lddc, B, ldb, out, 32};
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) {  // empty dot products
        const int es = out_type == SPMM_F32 ? 4 : 2;
        return status_of(cudaMemsetAsync(out, 0, (size_t)nnz * es, s));
    }
    if (b_type == SPMM_F32 && out_type == SPMM_F32) return sddmm_run<float, float>(a, s);
    if (b_type == SPMM_BF16 && out_type == SPMM_BF16) return sddmm_run<__nv_bfloat16, __nv_bfloat16>(a, s);
    if (b_type == SPMM_BF16 && out_type == SPMM_F32) return sddmm_run<__nv_bfloat16, float>(a, s);
    if (b_type == SPMM_F16 && out_type == SPMM_F16) return sddmm_run<__half, __half>(a, s);
    if (b_type == SPMM_F16 && out_type == SPMM_F32) return sddmm_run<__half, float>(a, s);
    return SPMM_ERR_UNSUPPORTED;
}

}  // extern "C"
