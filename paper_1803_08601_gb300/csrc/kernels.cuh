// CSR x dense SpMM kernels for sm_103a: row split (Section 4.1), merge-path
// partition / compute / carry-out fix-up (Section 4.2, Algorithm 1).
//
// Both families share the memory access pattern the paper identifies as the
// key to SpMM performance (Section 4.1, "Memory access pattern"; Fig. 3(c)):
// a group of W lanes owns one row of A at a time, and each lane owns VEC
// consecutive columns of B and C, so that every gathered row of B and every
// stored row of C is read or written with W coalesced 16-byte accesses.  The
// column index and value of a nonzero are loaded by one lane and broadcast to
// the other lanes of its group with warp shuffles (Section 4.1, "Shared
// memory": shuffle broadcast instead of shared memory).  A batch of kUnroll
// gathers is issued before any of them is accumulated (instruction-level
// parallelism, Section 3.1).
//
// Column slabs: gridDim.y (row split) or the slab part of the work index
// (merge) selects which W * VEC columns a CTA covers, so n of any size is
// handled, and a narrower slab keeps the slab of B that is being gathered
// resident in L2.
#pragma once

#include <climits>

#include "common.cuh"

namespace spmm {

struct RowSplitArgs {
    int m, n;
    const int* row_ptr;
    const int* col_ind;
    const void* vals;
    const void* B;
    long long ldb;
    void* C;
    long long ldc;
};

// ============================================================================ row split
//
// Algorithm I (Section 4.1, Fig. 3).  Sub-warp of W lanes per row; the warp's
// 32 / W rows are processed together.  Loop trip counts are made uniform over
// the warp (the longest row of the warp sets them) so that the shuffles always
// run with the full mask; lanes past the end of their row load nothing
// (Section 4.1 passes a dummy column index there; predication does the same
// without the load).
// One row per lane group: the lane group owning `row` (row >= a.m: nothing to
// do, but the lanes still join the warp's shuffles) computes the `slab`-th
// W * VEC columns of C[row, :].  Every lane of the warp must call this the
// same number of times.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__device__ __forceinline__ void rowsplit_row(const RowSplitArgs& a, long long row, int slab) {
    constexpr int U = gathers_per_batch<TB, VEC>();
    constexpr int CV = (U > W) ? U / W : 1;  // (column, value) pairs per lane per batch
    constexpr int BS = W * CV;               // nonzeros per batch
    constexpr int G = BS / U;                // groups of U gathers per batch
    const int lane = threadIdx.x & 31;
    const int sl = lane & (W - 1);
    const long long col0 = (long long)slab * (W * VEC) + (long long)sl * VEC;
    const bool col_ok = col0 < a.n;
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const TB* __restrict__ B = static_cast<const TB*>(a.B);

    int rs = 0, re = 0;
    if (row < a.m) {
        rs = __ldg(a.row_ptr + row);
        re = __ldg(a.row_ptr + row + 1);
    }
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();

    const int nb = (re - rs + BS - 1) / BS;
    const int nb_max = __reduce_max_sync(kFullMask, nb);
    for (int b = 0; b < nb_max; ++b) {
        const int base = rs + b * BS;
        const int cnt = re - base;  // nonzeros left in this row (may be <= 0)
        int mc[CV];
        float mv[CV];
#pragma unroll
        for (int c = 0; c < CV; ++c) {
            const int p = base + c * W + sl;
            const bool ok = p < re;
            mc[c] = ok ? __ldg(a.col_ind + p) : 0;
            mv[c] = ok ? load_f(vals + p) : 0.0f;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g > 0 && __all_sync(kFullMask, g * U >= cnt)) break;
            Raw<TB, VEC> bv[U];
            float vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = g * U + u;  // nonzero j of the batch sits in lane j % W, slot j / W
                const int c = __shfl_sync(kFullMask, mc[j / W], j % W, W);
                vv[u] = __shfl_sync(kFullMask, mv[j / W], j % W, W);
                bv[u] = (j < cnt && col_ok) ? load_raw<TB, VEC>(gather_row(B, col0, c, a.ldb)) : zero_raw<TB, VEC>();
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if constexpr (SR::kZeroPadOk) fma_raw<TB, VEC>(acc, vv[u], bv[u]);
                else if (g * U + u < cnt) accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
            }
        }
    }
    if (row < a.m && col_ok) store_vec<TC, VEC>(static_cast<TC*>(a.C) + row * a.ldc + col0, acc);
}

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads) rowsplit_kernel(RowSplitArgs a) {
    constexpr int RPW = 32 / W;  // rows per warp
    const long long row =
        (long long)blockIdx.x * (kThreads / W) + (threadIdx.x >> 5) * RPW + (threadIdx.x & 31) / W;
    rowsplit_row<TV, TB, TC, VEC, W, SR>(a, row, blockIdx.y);
}

// ============================================================================ merge path
//
// Algorithm II (Section 4.2, Algorithm 1).  The path that merges the row end
// offsets row_ptr[1..m] with the nonzero indices 0..nnz-1 (Section 4 item
// 2(b), Fig. 2(c)) is cut into tiles of equal length (rows + nonzeros): every
// CTA-sized tile carries the same amount of work whatever the row lengths.
//
struct MergeArgs {
    int m, n;
    long long nnz;
    const int* row_ptr;
    const int* col_ind;
    const void* vals;
    const void* B;
    long long ldb;
    void* C;
    long long ldc;
    const int2* limits;  // [num_tiles + 1] tile boundary coordinates
    int num_tiles;
    int slabs;            // column slabs; work item = slab * num_tiles + tile
    int ips;              // merge-path items per lane group
    float* carry;         // [num_tiles][n] partial sum of the row a tile leaves unfinished
    float* head;          // [num_tiles][n] partial sum of the row a tile finishes but did not start
    int* carry_row;       // [num_tiles] that row, or -1
    int* head_row;        // [num_tiles] that row, or -1
    int* status;          // optional device status word
    int use_tma;          // 1: 1-D bulk copies into shared memory, 0: cooperative loads
    unsigned long long wait_ns;  // limit of every mbarrier wait
};

// Shared-memory plan of the merge kernel: two staging buffers (row_ptr window,
// col_ind window, vals window), then the per-lane-group first-row and carry
// partial sums used to combine rows that cross lane groups inside a tile.
template <typename TV, int VEC, int W, int NT = kThreads>
struct MergeSmem {
    static constexpr int S = NT / W;  // lane groups per CTA of NT threads
    static constexpr int SW = W * VEC;      // columns per slab
    static __host__ __device__ int ipt(int ips) { return S * ips; }
    static __host__ __device__ int rp_cap(int ips) { return ipt(ips) + 8; }
    static __host__ __device__ int col_cap(int ips) { return ipt(ips) + 8; }
    static __host__ __device__ int val_cap(int ips) { return ipt(ips) + 16; }
    static __host__ __device__ size_t r16(size_t b) { return (b + 15) & ~size_t(15); }
    static __host__ __device__ size_t buf_bytes(int ips) {
        return r16(rp_cap(ips) * 4) + r16(col_cap(ips) * 4) + r16(val_cap(ips) * sizeof(TV));
    }
    static constexpr size_t kHeader = 128;  // 2 mbarriers + 2 x (int4 coords + int4 offsets)
    static __host__ __device__ size_t groups_offset(int ips) { return kHeader + 2 * buf_bytes(ips); }
    static __host__ __device__ size_t total(int ips) {
        return groups_offset(ips) + 2 * (size_t)S * SW * 4 + 2 * (size_t)S * 4;
    }
};

struct Window {
    long long a, e;  // bulk-copied element range [a, e), 16-byte aligned ends
};

// Elements [lo, hi) of an array of `len` elements: the bulk copy covers the
// 16-byte-aligned span [a, e) around them that stays inside the array; only
// the array's last partial 16 bytes (when the window reaches them) are loaded
// with plain loads.
template <typename T>
__device__ __forceinline__ Window make_window(long long lo, long long hi, long long len) {
    Window w;
    w.a = align_down16<T>(lo);
    long long e = align_up16<T>(hi);
    const long long lim = align_down16<T>(len);
    if (e > lim) e = lim;
    w.e = e > w.a ? e : w.a;
    return w;
}

template <typename TV, int VEC, int W, int NT = kThreads>
struct MergeView {
    using L = MergeSmem<TV, VEC, W, NT>;
    unsigned char* base;
    int ips;
    __device__ uint64_t* bar(int b) const { return reinterpret_cast<uint64_t*>(base) + b; }
    __device__ int4* coords(int b) const { return reinterpret_cast<int4*>(base + 16) + 2 * b; }
    __device__ int4* offs(int b) const { return reinterpret_cast<int4*>(base + 16) + 2 * b + 1; }
    __device__ unsigned char* buf(int b) const { return base + L::kHeader + b * L::buf_bytes(ips); }
    __device__ int* rp(int b) const { return reinterpret_cast<int*>(buf(b)); }
    __device__ int* col(int b) const { return reinterpret_cast<int*>(buf(b) + L::r16(L::rp_cap(ips) * 4)); }
    __device__ TV* val(int b) const {
        return reinterpret_cast<TV*>(buf(b) + L::r16(L::rp_cap(ips) * 4) + L::r16(L::col_cap(ips) * 4));
    }
    __device__ float* first(int s) const {
        return reinterpret_cast<float*>(base + L::groups_offset(ips)) + (size_t)s * L::SW;
    }
    __device__ float* carry(int s) const {
        return reinterpret_cast<float*>(base + L::groups_offset(ips)) + (size_t)(L::S + s) * L::SW;
    }
    __device__ int* first_row() const {
        return reinterpret_cast<int*>(base + L::groups_offset(ips) + 2 * (size_t)L::S * L::SW * 4);
    }
    __device__ int* carry_row() const { return first_row() + L::S; }
};

// GLOBALTOSHARED of Algorithm 1: bring a tile's row_ptr window [r0, r1] and its
// col_ind / vals window [z0, z1) into staging buffer b.  Run by warp 0 only.
// With TMA, lane 0 announces the byte count on the buffer's mbarrier and
// issues up to three 1-D bulk copies; the array tails (at most 15 bytes each)
// are loaded by the other lanes.  Without TMA the caller loads cooperatively.
template <typename TV, int VEC, int W, int NT>
__device__ __forceinline__ void merge_stage(const MergeArgs& a, const MergeView<TV, VEC, W, NT>& v, int item, int b) {
    const int lane = threadIdx.x & 31;
    const int tile = item % a.num_tiles;
    int2 l0 = make_int2(0, 0), l1 = make_int2(0, 0);
    if (lane == 0) {
        l0 = a.limits[tile];
        l1 = a.limits[tile + 1];
    }
    l0.x = __shfl_sync(kFullMask, l0.x, 0);
    l0.y = __shfl_sync(kFullMask, l0.y, 0);
    l1.x = __shfl_sync(kFullMask, l1.x, 0);
    l1.y = __shfl_sync(kFullMask, l1.y, 0);
    const int r0 = l0.x, z0 = l0.y, r1 = l1.x, z1 = l1.y;
    const Window wr = make_window<int>(r0, (long long)r1 + 1, (long long)a.m + 1);
    const Window wc = make_window<int>(z0, z1, a.nnz);
    const Window wv = make_window<TV>(z0, z1, a.nnz);
    int* srp = v.rp(b);
    int* scol = v.col(b);
    TV* sval = v.val(b);
    if (lane == 0) {
        *v.coords(b) = make_int4(r0, z0, r1, z1);
        *v.offs(b) = make_int4((int)wr.a, (int)wc.a, (int)wv.a, 0);
        const uint32_t bytes = (uint32_t)((wr.e - wr.a) * 4 + (wc.e - wc.a) * 4 + (wv.e - wv.a) * (long long)sizeof(TV));
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(v.bar(b), bytes);
        if (wr.e > wr.a) bulk_copy_g2s(srp, a.row_ptr + wr.a, (uint32_t)((wr.e - wr.a) * 4), v.bar(b));
        if (wc.e > wc.a) bulk_copy_g2s(scol, a.col_ind + wc.a, (uint32_t)((wc.e - wc.a) * 4), v.bar(b));
        if (wv.e > wv.a)
            bulk_copy_g2s(sval, static_cast<const TV*>(a.vals) + wv.a, (uint32_t)((wv.e - wv.a) * sizeof(TV)), v.bar(b));
    }
    // array tails not covered by the aligned bulk copies
    {
        const long long i = (wr.e > r0 ? wr.e : r0) + lane;
        if (i < (long long)r1 + 1) srp[i - wr.a] = a.row_ptr[i];
    }
    {
        const long long i = (wc.e > z0 ? wc.e : z0) + lane;
        if (i < z1) scol[i - wc.a] = a.col_ind[i];
    }
    {
        const long long i = (wv.e > z0 ? wv.e : z0) + lane;
        if (i < z1) sval[i - wv.a] = static_cast<const TV*>(a.vals)[i];
    }
}

// Cooperative (all threads) load of a tile's windows, used when an array
// base is not 16-byte aligned.  Uses the same smem indexing as merge_stage.
template <typename TV, int VEC, int W, int NT>
__device__ __forceinline__ void merge_load_plain(const MergeArgs& a, const MergeView<TV, VEC, W, NT>& v, int item,
                                                 int b) {
    const int tile = item % a.num_tiles;
    const int2 l0 = a.limits[tile], l1 = a.limits[tile + 1];
    const int r0 = l0.x, z0 = l0.y, r1 = l1.x, z1 = l1.y;
    if (threadIdx.x == 0) {
        *v.coords(b) = make_int4(r0, z0, r1, z1);
        *v.offs(b) = make_int4(r0, z0, z0, 0);
    }
    int* srp = v.rp(b);
    int* scol = v.col(b);
    TV* sval = v.val(b);
    for (int i = r0 + threadIdx.x; i <= r1; i += blockDim.x) srp[i - r0] = a.row_ptr[i];
    for (int i = z0 + threadIdx.x; i < z1; i += blockDim.x) {
        scol[i - z0] = a.col_ind[i];
        sval[i - z0] = static_cast<const TV*>(a.vals)[i];
    }
}

// Phase 2 of Algorithm 1 for one tile held in staging buffer b.
//
// Inside the tile every lane group takes an equal share of the tile's path
// items (a second merge-path search, in shared memory) and walks it: a
// nonzero adds val * B[col, slab] to the running sum; a row end emits the sum
// (PREPARESPMM / REDUCETOGLOBALSPMM).  The first row a group emits may have
// begun in an earlier group, so it is held back in shared memory together with
// every group's trailing partial sum (its carry-out) and combined after a
// barrier.  Of the tile as a whole, the partial sum of a row that began in an
// earlier tile (head) and of the row left unfinished at its end (carry) go to
// global memory for the fix-up pass.
template <typename TV, typename TB, typename TC, int VEC, int W, int NT, typename SR = PlusTimes>
__device__ __forceinline__ void merge_tile(const MergeArgs& a, const MergeView<TV, VEC, W, NT>& v, int item, int b) {
    using L = MergeSmem<TV, VEC, W, NT>;
    constexpr int U = gathers_per_batch<TB, VEC>();
    constexpr int CV = (U > W) ? U / W : 1;
    constexpr int BS = W * CV;
    constexpr int G = BS / U;
    const int tile = item % a.num_tiles;
    const int slab = item / a.num_tiles;
    const int lane = threadIdx.x & 31;
    const int sl = lane & (W - 1);
    const int s = threadIdx.x / W;  // lane group
    const long long col0 = (long long)slab * L::SW + (long long)sl * VEC;
    const bool col_ok = col0 < a.n;
    const int4 cz = *v.coords(b);
    const int4 of = *v.offs(b);
    const int r0 = cz.x, z0 = cz.y, r1 = cz.z, z1 = cz.w;
    const int* srp = v.rp(b) - of.x;    // srp[i] = row_ptr[i] for i in [r0, r1]
    const int* scol = v.col(b) - of.y;  // scol[p] = col_ind[p] for p in [z0, z1)
    const TV* sval = v.val(b) - of.z;
    const TB* __restrict__ B = static_cast<const TB*>(a.B);
    TC* __restrict__ C = static_cast<TC*>(a.C);
    const int rows_t = r1 - r0, nz_t = z1 - z0, items = rows_t + nz_t;

    // this group's share of the tile's path
    auto search = [&](int d) {
        int lo = d - nz_t > 0 ? d - nz_t : 0, hi = d < rows_t ? d : rows_t;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (srp[r0 + mid + 1] <= z0 + d - mid - 1) lo = mid + 1;
            else hi = mid;
        }
        return lo;
    };
    const int ds = min(s * a.ips, items), de = min((s + 1) * a.ips, items);
    const int xs = search(ds), xe = search(de);
    int row = r0 + xs;
    const int z_s = z0 + ds - xs;
    const int row_e = r0 + xe, z_e = z0 + de - xe;
    int rend = row < r1 ? srp[row + 1] : INT_MAX;
    int first_row = -1;
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();

    auto emit = [&]() {
        if (first_row < 0) {
            first_row = row;
            if (col_ok) {
                float* f = v.first(s) + sl * VEC;
#pragma unroll
                for (int e = 0; e < VEC; ++e) f[e] = acc[e];
            }
        } else if (col_ok) {
            store_vec<TC, VEC>(C + (long long)row * a.ldc + col0, acc);
        }
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();
        ++row;
        rend = row < r1 ? srp[row + 1] : INT_MAX;
    };

    const int nb = (z_e - z_s + BS - 1) / BS;
    const int nb_max = __reduce_max_sync(kFullMask, nb);
    for (int bt = 0; bt < nb_max; ++bt) {
        const int base = z_s + bt * BS;
        const int cnt = z_e - base;
        int mc[CV];
        float mv[CV];
#pragma unroll
        for (int c = 0; c < CV; ++c) {
            const int p = base + c * W + sl;
            const bool ok = p < z_e;
            mc[c] = ok ? scol[p] : 0;
            mv[c] = ok ? Elem<TV>::to_f(sval[p]) : 0.0f;
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (g > 0 && __all_sync(kFullMask, g * U >= cnt)) break;
            Raw<TB, VEC> bv[U];
            float vv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = g * U + u;
                const int c = __shfl_sync(kFullMask, mc[j / W], j % W, W);
                vv[u] = __shfl_sync(kFullMask, mv[j / W], j % W, W);
                bv[u] = (j < cnt && col_ok) ? load_raw<TB, VEC>(gather_row(B, col0, c, a.ldb)) : zero_raw<TB, VEC>();
            }
            // no row of any lane group ends among these U nonzeros (the common case inside the long
            // rows of a skewed matrix): accumulate without the per-nonzero row-end checks
            if (__all_sync(kFullMask, base + min(cnt, (g + 1) * U) <= rend)) {
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (g * U + u < cnt) accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = g * U + u;
                    if (j < cnt) {
                        const int p = base + j;
                        while (p >= rend) emit();  // rows (possibly empty) that end before nonzero p
                        accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
                    }
                }
            }
        }
    }
    while (row < row_e) emit();  // row ends after the group's last nonzero
    if (col_ok) {
        float* cpart = v.carry(s) + sl * VEC;
#pragma unroll
        for (int e = 0; e < VEC; ++e) cpart[e] = acc[e];
    }
    if (sl == 0) {
        v.first_row()[s] = first_row;
        v.carry_row()[s] = row;
    }
    __syncthreads();

    // combine: a group's first emitted row adds the carries of the groups before it
    const bool head_exists = r0 < r1 && srp[r0] < z0;  // row r0 began in an earlier tile and ends here
    const int fr = v.first_row()[s];
    if (fr >= 0 && col_ok) {
        int t = s - 1;
        while (t >= 0 && v.carry_row()[t] == fr) --t;
        float sum[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) sum[e] = SR::identity();
        for (int u = t + 1; u < s; ++u) {
            const float* c = v.carry(u) + sl * VEC;
#pragma unroll
            for (int e = 0; e < VEC; ++e) sum[e] = SR::add(sum[e], c[e]);
        }
        const float* f = v.first(s) + sl * VEC;
#pragma unroll
        for (int e = 0; e < VEC; ++e) sum[e] = SR::add(sum[e], f[e]);
        if (fr == r0 && head_exists) {
            float* h = a.head + (size_t)tile * a.n + col0;
#pragma unroll
            for (int e = 0; e < VEC; ++e) h[e] = sum[e];
        } else {
            store_vec<TC, VEC>(C + (long long)fr * a.ldc + col0, sum);
        }
    }
    // the tile's carry-out: the row left unfinished at the tile's end
    const bool carry_exists = r1 < a.m && z1 > srp[r1];
    if (s == L::S - 1 && carry_exists && col_ok) {
        int t = s;
        while (t > 0 && v.carry_row()[t - 1] == r1) --t;
        float sum[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) sum[e] = SR::identity();
        for (int u = t; u <= s; ++u) {
            const float* c = v.carry(u) + sl * VEC;
#pragma unroll
            for (int e = 0; e < VEC; ++e) sum[e] = SR::add(sum[e], c[e]);
        }
        float* cg = a.carry + (size_t)tile * a.n + col0;
#pragma unroll
        for (int e = 0; e < VEC; ++e) cg[e] = sum[e];
    }
    if (slab == 0 && threadIdx.x == 0) {
        a.head_row[tile] = head_exists ? r0 : -1;
        a.carry_row[tile] = carry_exists ? r1 : -1;
    }
}

// Phase 2 driver: persistent CTAs walk the work items (slab-major, so the
// CTAs running together gather from the same slab of B), with the next item's
// windows brought into the other staging buffer by TMA while the current one
// is computed.  Every mbarrier wait is bounded: when one runs out the kernel
// records SPMM_ERR_TIMEOUT, waits (bounded) for its copies still in flight
// and returns.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__device__ __forceinline__ void merge_kernel_body(const MergeArgs& a) {
    constexpr int NT = merge_cta_threads(W);
    extern __shared__ __align__(128) unsigned char smem[];
    MergeView<TV, VEC, W, NT> v{smem, a.ips};
    pdl_wait();               // the partition (launched just before) has finished writing limits
    pdl_launch_dependents();  // the fix-up may be scheduled; it waits for this grid to finish
    const int total = a.num_tiles * a.slabs;
    int item = blockIdx.x;
    if (item >= total) return;
    const int warp = threadIdx.x >> 5;
    if (!a.use_tma) {
        for (; item < total; item += gridDim.x) {
            merge_load_plain<TV, VEC, W, NT>(a, v, item, 0);
            __syncthreads();
            merge_tile<TV, TB, TC, VEC, W, NT, SR>(a, v, item, 0);
            __syncthreads();
        }
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(v.bar(0), 1);
        mbar_init(v.bar(1), 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0u;   // bit b: parity of the next phase of buffer b's mbarrier
    uint32_t pending = 0u; // bit b: a copy into buffer b is in flight
    if (warp == 0) merge_stage<TV, VEC, W, NT>(a, v, item, 0);
    pending |= 1u;
    for (int it = 0; item < total; ++it, item += gridDim.x) {
        const int b = it & 1;
        const int nxt = item + gridDim.x;
        if (nxt < total) {
            if (warp == 0) merge_stage<TV, VEC, W, NT>(a, v, nxt, b ^ 1);
            pending |= 2u >> b;  // bit (b ^ 1)
        }
        const uint32_t par = (phase >> b) & 1u;
        const bool ok = mbar_wait_bounded(v.bar(b), par, a.wait_ns);
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) report(a.status, SPMM_ERR_TIMEOUT);
            // let the copies still in flight land before shared memory is released
            if (!ok) mbar_wait_bounded(v.bar(b), par, a.wait_ns);
            if (pending & (2u >> b)) mbar_wait_bounded(v.bar(b ^ 1), (phase >> (b ^ 1)) & 1u, a.wait_ns);
            return;
        }
        phase ^= 1u << b;
        pending &= ~(1u << b);
        merge_tile<TV, TB, TC, VEC, W, NT, SR>(a, v, item, b);
        __syncthreads();
    }
}

// Narrow rows (W <= 8): 128-thread CTAs, six per SM.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(128, 6) merge_kernel_narrow(MergeArgs a) {
    merge_kernel_body<TV, TB, TC, VEC, W, SR>(a);
}

// Wide rows (W >= 16): 256-thread CTAs.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(256) merge_kernel_wide(MergeArgs a) {
    merge_kernel_body<TV, TB, TC, VEC, W, SR>(a);
}

// FIXCARRYOUT of Algorithm 1.  For every run of consecutive tiles whose
// carry-out belongs to the same row R (a row spanning several tiles), the row
// is finished by the tile right after the run, which left R's remaining
// partial sum in head[]; C[R] = carries (in tile order) + head, rounded once.
// One warp per tile (grid-stride); only run heads do work.  Lanes stride n in
// 16-byte vectors of four columns when n allows (so one pass covers up to 128
// columns), with up to 16 of a run's tiles loaded at once: the long runs of
// rows that span many tiles are the kernel's critical path.  Each column is
// still summed in tile order.
template <typename TC, typename SR = PlusTimes>
__global__ void merge_fixup_kernel(const int* __restrict__ carry_row, const int* __restrict__ head_row,
                                   const float* __restrict__ carry, const float* __restrict__ head, int num_tiles,
                                   int n, TC* __restrict__ C, long long ldc, int* status) {
    pdl_wait();  // launched early behind the merge kernel: its writes are visible after this
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (blockDim.x >> 5);
    for (int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < num_tiles; i += warps) {
        const int R = carry_row[i];
        if (R < 0 || (i > 0 && carry_row[i - 1] == R)) continue;
        // the run's last tile j: the tiles carrying R are consecutive, so the
        // first tile after i that does not carry R ends it (32 tiles per probe)
        int j = i;
        for (int base = i + 1;; base += 32) {
            const int t = base + lane;
            const unsigned same = __ballot_sync(kFullMask, t < num_tiles && carry_row[t] == R);
            if (same != kFullMask) {
                j = base + __ffs(~same) - 2;
                break;
            }
        }
        if (j + 1 >= num_tiles || head_row[j + 1] != R) {
            if (lane == 0) report(status, SPMM_ERR_BAD_CSR);
            continue;
        }
        if ((n & 3) == 0) {  // rows of carry / head are 16-byte aligned
            auto add4 = [](float4 s, float4 x) {
                return make_float4(SR::add(s.x, x.x), SR::add(s.y, x.y), SR::add(s.z, x.z), SR::add(s.w, x.w));
            };
            for (int c = lane * 4; c < n; c += 128) {
                float4 sum = make_float4(SR::identity(), SR::identity(), SR::identity(), SR::identity());
                int t = i;
                for (; t + 15 <= j; t += 16) {  // 16 loads in flight, then the adds in tile order
                    float4 x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) x[u] = *reinterpret_cast<const float4*>(carry + (size_t)(t + u) * n + c);
#pragma unroll
                    for (int u = 0; u < 16; ++u) sum = add4(sum, x[u]);
                }
                for (; t <= j; ++t) sum = add4(sum, *reinterpret_cast<const float4*>(carry + (size_t)t * n + c));
                const float4 h = *reinterpret_cast<const float4*>(head + (size_t)(j + 1) * n + c);
                TC* out = C + (long long)R * ldc + c;
                out[0] = Elem<TC>::from_f(SR::add(sum.x, h.x));
                out[1] = Elem<TC>::from_f(SR::add(sum.y, h.y));
                out[2] = Elem<TC>::from_f(SR::add(sum.z, h.z));
                out[3] = Elem<TC>::from_f(SR::add(sum.w, h.w));
            }
        } else {
            for (int c = lane; c < n; c += 32) {
                float sum = SR::identity();
                int t = i;
                for (; t + 15 <= j; t += 16) {
                    float x[16];
#pragma unroll
                    for (int u = 0; u < 16; ++u) x[u] = carry[(size_t)(t + u) * n + c];
#pragma unroll
                    for (int u = 0; u < 16; ++u) sum = SR::add(sum, x[u]);
                }
                for (; t <= j; ++t) sum = SR::add(sum, carry[(size_t)t * n + c]);
                sum = SR::add(sum, head[(size_t)(j + 1) * n + c]);
                C[(long long)R * ldc + c] = Elem<TC>::from_f(sum);
            }
        }
    }
}

// ============================================================================ SpMV (n = 1)
//
// Both families specialised for one dense column, y = A x (the SpMV case the
// paper contrasts with SpMM in Section 3 and Table 1).  With n = 1 the lane
// groups above shrink to one lane per row reading its row's nonzeros alone,
// and every merge item costs a whole walk step for one 4-byte gather; here
// the nonzeros are spread over the lanes instead.

// Row split: G lanes per row stride over the row's nonzeros, so a warp reads
// col_ind / vals in runs of G consecutive entries; four independent gathers
// of x are in flight per lane; a shuffle reduction over the G lanes finishes
// the row.  G = 1 is the thread-per-row form.
template <typename TV, typename TB, typename TC, int G, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads) spmv_rowsplit_kernel(RowSplitArgs a) {
    static_assert(G >= 1 && G <= 32 && (G & (G - 1)) == 0, "lanes per row");
    const long long row = (long long)blockIdx.x * (kThreads / G) + threadIdx.x / G;
    const int lane = threadIdx.x & (G - 1);
    const int* __restrict__ col = a.col_ind;
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const TB* __restrict__ x = static_cast<const TB*>(a.B);
    float acc = SR::identity();
    if (row < a.m) {
        const int re = __ldg(a.row_ptr + row + 1);
        int p = __ldg(a.row_ptr + row) + lane;
        for (; p + 3 * G < re; p += 4 * G) {
            int c[4];
            float v[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                c[u] = __ldg(col + p + u * G);
                v[u] = load_f(vals + p + u * G);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = load_f(gather_row(x, 0, c[u], a.ldb));
#pragma unroll
            for (int u = 0; u < 4; ++u) acc = SR::mul_add(acc, v[u], b[u]);
        }
        for (; p < re; p += G) acc = SR::mul_add(acc, load_f(vals + p), load_f(gather_row(x, 0, __ldg(col + p), a.ldb)));
    }
    if constexpr (G > 1) {
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) acc = SR::add(acc, __shfl_xor_sync(kFullMask, acc, off, G));
    }
    if (lane == 0 && row < a.m) static_cast<TC*>(a.C)[row * a.ldc] = Elem<TC>::from_f(acc);
}

// Merge based: one CTA per merge-path tile of kThreads * T items (the
// partition kernel's limits).  Every product val[p] (x) x[col[p]] of the tile
// is gathered first, all loads independent and coalesced over the CTA, into
// shared memory together with the row end offsets of the tile's rows; then
// each thread walks its T items of the path over shared memory only.  A
// thread's first finished row adds the carries of the threads before it that
// worked on the same row; the tile's head and carry go to the fix-up as in
// the SpMM kernel (same layout with n = 1).
constexpr int kSpmvItems = 8;  // default merge items per thread

template <typename TV, typename TB, typename TC, int T, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads) spmv_merge_kernel(MergeArgs a) {
    constexpr int kTile = kThreads * T;
    __shared__ float s_prod[kTile];
    __shared__ int s_end[kTile];
    __shared__ float s_carry[kThreads];
    __shared__ int s_carry_row[kThreads];
    __shared__ float s_warp_run[kThreads / 32];
    __shared__ int s_warp_key[kThreads / 32], s_warp_first_key[kThreads / 32];
    pdl_wait();               // the partition (launched just before) has finished writing limits
    pdl_launch_dependents();  // the fix-up may be scheduled; it waits for this grid to finish
    const int tile = blockIdx.x;
    const int tid = threadIdx.x;
    const int2 lo = a.limits[tile], hi = a.limits[tile + 1];
    const int r0 = lo.x, z0 = lo.y, r1 = hi.x, z1 = hi.y;
    const int nr = r1 - r0, nz = z1 - z0, items = nr + nz;
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const TB* __restrict__ x = static_cast<const TB*>(a.B);
    TC* __restrict__ y = static_cast<TC*>(a.C);

    {
        int c[T];
        float v[T], b[T];
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const int i = tid + u * kThreads;
            c[u] = i < nz ? __ldg(a.col_ind + z0 + i) : 0;
            v[u] = i < nz ? load_f(vals + z0 + i) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < T; ++u)
            b[u] = tid + u * kThreads < nz ? load_f(gather_row(x, 0, c[u], a.ldb)) : 0.0f;
#pragma unroll
        for (int u = 0; u < T; ++u) {
            const int i = tid + u * kThreads;
            if (i < nz) s_prod[i] = SR::mul_add(SR::identity(), v[u], b[u]);
        }
        for (int i = tid; i < nr; i += kThreads) s_end[i] = __ldg(a.row_ptr + r0 + 1 + i);
    }
    __syncthreads();

    // this thread's share of the tile's path: the first row end not taken
    // before diagonal d (row ends go first on ties, as in the partition)
    auto search = [&](int d) {
        int l = d - nz > 0 ? d - nz : 0, h = d < nr ? d : nr;
        while (l < h) {
            const int mid = (l + h) >> 1;
            if (s_end[mid] <= z0 + d - mid - 1) l = mid + 1;
            else h = mid;
        }
        return l;
    };
    const int ds = min(tid * T, items), de = min(ds + T, items);
    int ri = search(ds);
    int zi = ds - ri;
    int rend = ri < nr ? s_end[ri] - z0 : INT_MAX;  // tile-local end of the current row
    float acc = SR::identity();
    int first = -1;
    float first_val = SR::identity();
    for (int d = ds; d < de; ++d) {
        if (zi >= rend) {  // row r0 + ri ends here
            if (first < 0) {
                first = ri;
                first_val = acc;
            } else {
                y[(long long)(r0 + ri) * a.ldc] = Elem<TC>::from_f(acc);
            }
            acc = SR::identity();
            ++ri;
            rend = ri < nr ? s_end[ri] - z0 : INT_MAX;
        } else {
            acc = SR::add(acc, s_prod[zi]);
            ++zi;
        }
    }
    // Carry rows do not decrease with the thread index, so the threads that
    // carry one row are consecutive.  A keyed inclusive scan over the threads
    // (in-warp by shuffles, across warps from the warps' last values) gives
    // each thread the carries of its own run up to itself.
    const int key = r0 + ri;
    const int lane = tid & 31, warp = tid >> 5;
    float run = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float v = __shfl_up_sync(kFullMask, run, off);
        const int k = __shfl_up_sync(kFullMask, key, off);
        if (lane >= off && k == key) run = SR::add(v, run);
    }
    if (lane == 31) {
        s_warp_run[warp] = run;
        s_warp_key[warp] = key;
    }
    if (lane == 0) s_warp_first_key[warp] = key;
    __syncthreads();
    // carries of earlier warps in the same run
    auto from_earlier_warps = [&](int k, int w) {
        float sum = SR::identity();
        for (int u = w - 1; u >= 0 && s_warp_key[u] == k; --u) {
            sum = SR::add(s_warp_run[u], sum);
            if (s_warp_first_key[u] != k) break;  // the run starts inside warp u
        }
        return sum;
    };
    // inclusive run of this thread's carry: earlier warps, then this warp
    const bool lane0_in_run = __shfl_sync(kFullMask, key, 0) == key;
    float inclusive = run;
    if (lane0_in_run) inclusive = SR::add(from_earlier_warps(key, warp), run);
    s_carry[tid] = inclusive;
    s_carry_row[tid] = key;
    __syncthreads();

    const bool head_exists = nr > 0 && __ldg(a.row_ptr + r0) < z0;  // row r0 began in an earlier tile, ends here
    if (first >= 0) {
        const int fr = r0 + first;
        float sum = first_val;
        if (tid > 0 && s_carry_row[tid - 1] == fr) sum = SR::add(s_carry[tid - 1], sum);
        if (fr == r0 && head_exists) a.head[tile] = sum;
        else y[(long long)fr * a.ldc] = Elem<TC>::from_f(sum);
    }
    if (tid == kThreads - 1) {
        const bool carry_exists = r1 < a.m && z1 > __ldg(a.row_ptr + r1);  // row r1 began here, ends later
        if (carry_exists) a.carry[tile] = s_carry[tid];  // the last thread's key is r1
        a.carry_row[tile] = carry_exists ? r1 : -1;
        a.head_row[tile] = head_exists ? r0 : -1;
    }
}

// ============================================================================ A/B tiling
//
// Tiling of both A and B for denser matrices, the direction Section 6 names
// for rows with many nonzeros (after Greiner and Jacob): a CTA owns a block of
// rows and walks B in panels of KT rows held in shared memory (two buffers,
// filled by 16-byte asynchronous copies while the other is used).  Every
// nonzero of the block whose column falls in the current panel reads its B row
// from shared memory, so one staged row serves all of the block's nonzeros in
// that column instead of costing each of them an L2 gather.
//
// Each row keeps a cursor that moves once through its columns, so rows must
// list their columns in increasing order; an entry whose column lies below the
// current panel is reported as SPMM_ERR_BAD_CSR and skipped (never read out of
// range).  Lane groups of W lanes own kTiledRows rows each (the rows g, g + S,
// ...); within a group the in-panel entries of a row are loaded one per lane
// and broadcast by shuffles, as in the row split.
struct TiledArgs {
    int m, n, k;
    const int* row_ptr;
    const int* col_ind;
    const void* vals;
    const void* B;
    long long ldb;
    void* C;
    long long ldc;
    int* status;
};

constexpr int kTiledRows = 8;           // rows per lane group
constexpr int kTiledPanel = 32 * 1024;  // bytes of one B panel in shared memory

template <typename TV, typename TB, int VEC, int W>
struct TiledShape {
    static constexpr int S = kThreads / W;                       // lane groups per CTA
    static constexpr int RB = S * kTiledRows;                    // rows per CTA
    static constexpr int SW = W * VEC;                           // columns per slab
    static constexpr int KT = kTiledPanel / (SW * (int)sizeof(TB));  // B rows per panel
    static constexpr int CPR = SW * (int)sizeof(TB) / 16;        // 16-byte copies per B row
};

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads) tiled_kernel(TiledArgs a) {
    using TS = TiledShape<TV, TB, VEC, W>;
    constexpr int R = kTiledRows;
    static_assert(VEC * sizeof(TB) == 16, "tiling stages 16-byte vectors");
    extern __shared__ __align__(128) unsigned char smem[];
    TB* const panel0 = reinterpret_cast<TB*>(smem);
    TB* const panel1 = reinterpret_cast<TB*>(smem + kTiledPanel);
    const int lane = threadIdx.x & 31;
    const int sl = lane & (W - 1);
    const int g = threadIdx.x / W;
    const int gshift = lane & ~(W - 1);
    const unsigned gmask = W == 32 ? 0xffffffffu : ((1u << W) - 1u);
    const long long slab_col = (long long)blockIdx.y * TS::SW;
    const long long col0 = slab_col + (long long)sl * VEC;
    const bool col_ok = col0 < a.n;
    const TB* __restrict__ B = static_cast<const TB*>(a.B);
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const int* __restrict__ col = a.col_ind;

    int p[R], re[R], nc[R];
    float nv[R];
    float acc[R][VEC];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        const long long row = (long long)blockIdx.x * TS::RB + g + i * TS::S;
        p[i] = row < a.m ? __ldg(a.row_ptr + row) : 0;
        re[i] = row < a.m ? __ldg(a.row_ptr + row + 1) : 0;
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[i][e] = SR::identity();
    }
    // the next entry of each row for this lane: (column, value), column INT_MAX past the row's end
    auto fetch = [&](int i) {
        const int q = p[i] + sl;
        nc[i] = q < re[i] ? __ldg(col + q) : INT_MAX;
        nv[i] = q < re[i] ? load_f(vals + q) : 0.0f;
    };
#pragma unroll
    for (int i = 0; i < R; ++i) fetch(i);

    const int panels = (a.k + TS::KT - 1) / TS::KT;
    // this thread's 16-byte pieces of a panel: rows r0, r0 + RS, ..., column piece `part`
    constexpr int RS = kThreads / TS::CPR;  // panel rows covered by one pass of the CTA
    const int part = threadIdx.x % TS::CPR, r0 = threadIdx.x / TS::CPR;
    const long long bc = slab_col + (long long)part * VEC;
    auto stage = [&](int t, TB* dst) {
        if (bc < a.n) {
            const long long base = (long long)t * TS::KT;
#pragma unroll 4
            for (int r = r0; r < TS::KT; r += RS)
                if (base + r < a.k) cp_async16(dst + r * TS::SW + part * VEC, B + (base + r) * a.ldb + bc);
        }
        cp_async_commit();
    };
    stage(0, panel0);
    for (int t = 0; t < panels; ++t) {
        TB* const cur = (t & 1) ? panel1 : panel0;
        if (t + 1 < panels) stage(t + 1, (t & 1) ? panel0 : panel1);
        else cp_async_commit();  // an empty group keeps the wait count uniform
        cp_async_wait<1>();      // this thread's copies of panel t have landed ...
        __syncthreads();         // ... and every thread's
        const int k0 = t * TS::KT, kend = min(a.k, k0 + TS::KT);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            for (;;) {
                // the row's in-panel entries are a prefix of the group's lanes (columns increase)
                const bool in = nc[i] < kend;
                const unsigned ball = (__ballot_sync(kFullMask, in) >> gshift) & gmask;
                const int cnt = ball == gmask ? W : __ffs(~ball) - 1;
                const int cmax = __reduce_max_sync(kFullMask, cnt);
                // four entries per step: their shuffles and shared-memory reads are independent
                for (int j = 0; j < cmax; j += 4) {
                    int cj[4];
                    float vj[4];
                    Raw<TB, VEC> bj[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        cj[u] = __shfl_sync(kFullMask, nc[i], j + u, W);
                        vj[u] = __shfl_sync(kFullMask, nv[i], j + u, W);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const bool use = j + u < cnt && cj[u] >= k0 && col_ok;
                        bj[u] = use ? lds_raw<TB, VEC>(cur + (cj[u] - k0) * TS::SW + sl * VEC) : zero_raw<TB, VEC>();
                        if (j + u < cnt && cj[u] < k0 && sl == 0)
                            report(a.status, SPMM_ERR_BAD_CSR);  // columns not increasing: entry skipped
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        if (j + u < cnt && cj[u] >= k0) accum_raw<SR, TB, VEC>(acc[i], vj[u], bj[u]);
                }
                p[i] += cnt;
                if (cnt > 0) fetch(i);
                if (!__any_sync(kFullMask, cnt == W)) break;
            }
        }
        __syncthreads();  // panel t's buffer is refilled in the next iteration
    }
    cp_async_wait<0>();
    if (col_ok) {
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const long long row = (long long)blockIdx.x * TS::RB + g + i * TS::S;
            if (row < a.m) store_vec<TC, VEC>(static_cast<TC*>(a.C) + row * a.ldc + col0, acc[i]);
        }
    }
}

}  // namespace spmm
