// Batched SpMM: many independent float32 products C_b = A_b B_b of uneven
// sizes in ONE persistent kernel launch (plus one fix-up launch), replayable
// as a CUDA graph.  Not in the paper; it applies the paper's two algorithm
// families per matrix:
//   - a row-split matrix contributes work items of consecutive rows (one row
//     per lane group at a time, Section 4.1);
//   - a merge-based matrix contributes one item per merge-path tile (Section
//     4.2); its partition is computed once, when the plan is made, because
//     the sparsity pattern of a plan never changes; rows that cross tiles are
//     finished by one batched fix-up pass over every merge matrix.
// The per-matrix choice (algorithm, items per lane group) comes from the GB300
// selector or from an autotuner that times candidate schedules on a sample of
// the plan's own matrices, bucketed by shape, and caches the winners.
#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "launch.cuh"

namespace spmm {
namespace {

struct MatDesc {
    int m, k, n, alg, W, vec, slabs, ips, num_tiles, tile_base;  // vec: B / C columns per lane access (4 or 8)
    long long nnz, ldb, ldc;
    const int* row_ptr;
    const int* col_ind;
    const float* vals;
    const float* B;
    float* C;
    const int2* limits;
    float* carry;
    float* head;
};

struct Item {
    int mat;
    int kind_slab;  // bit 0: 1 = merge tile, 0 = row chunk; slab = kind_slab >> 1
    int a, b;       // row chunk [a, b) or merge tile a
};

constexpr int kRowsPerGroupPerItem = 8;

template <int W, int VEC>
__device__ __forceinline__ void batched_rows(const MatDesc& d, int r0, int r1, int slab) {
    RowSplitArgs ra{d.m, d.n, d.row_ptr, d.col_ind, d.vals, d.B, d.ldb, d.C, d.ldc};
    constexpr int G = kThreads / W;
    const int g = threadIdx.x / W;
    for (int base = r0; base < r1; base += G) {  // same trip count for the whole CTA
        const int row = base + g;
        rowsplit_row<float, float, float, VEC, W>(ra, row < r1 ? row : d.m, slab);
    }
}

template <int VEC>
__device__ __forceinline__ void batched_rows_any(const MatDesc& d, int r0, int r1, int slab) {
    switch (d.W) {
        case 1: batched_rows<1, VEC>(d, r0, r1, slab); break;
        case 2: batched_rows<2, VEC>(d, r0, r1, slab); break;
        case 4: batched_rows<4, VEC>(d, r0, r1, slab); break;
        case 8: batched_rows<8, VEC>(d, r0, r1, slab); break;
        case 16: batched_rows<16, VEC>(d, r0, r1, slab); break;
        default: batched_rows<32, VEC>(d, r0, r1, slab); break;
    }
}

template <int W>
__device__ __forceinline__ void batched_tile(const MatDesc& d, int* carry_row_all, int* head_row_all, int tile, int slab,
                                             unsigned char* smem, int* status) {
    MergeArgs ma{};
    ma.m = d.m;
    ma.n = d.n;
    ma.nnz = d.nnz;
    ma.row_ptr = d.row_ptr;
    ma.col_ind = d.col_ind;
    ma.vals = d.vals;
    ma.B = d.B;
    ma.ldb = d.ldb;
    ma.C = d.C;
    ma.ldc = d.ldc;
    ma.limits = d.limits;
    ma.num_tiles = d.num_tiles;
    ma.slabs = d.slabs;
    ma.ips = d.ips;
    ma.carry = d.carry;
    ma.head = d.head;
    ma.carry_row = carry_row_all + d.tile_base;
    ma.head_row = head_row_all + d.tile_base;
    ma.status = status;
    ma.use_tma = 0;
    MergeView<float, 4, W> v{smem, d.ips};
    const int item = slab * d.num_tiles + tile;
    merge_load_plain<float, 4, W>(ma, v, item, 0);
    __syncthreads();
    merge_tile<float, float, float, 4, W>(ma, v, item, 0);
    __syncthreads();
}

// Next work item of a persistent CTA: taken from a counter (zeroed before the
// launch), so that the items in flight at any moment are a contiguous window
// of the plan's item list (largest matrices first) rather than spreading as
// fast and slow CTAs drift apart: fewer matrices' B rows then share the L2.
__device__ __forceinline__ long long next_item(unsigned long long* counter) {
    __shared__ long long s_item;
    if (threadIdx.x == 0) s_item = (long long)atomicAdd(counter, 1ull);
    __syncthreads();
    const long long it = s_item;
    __syncthreads();
    return it;
}

// Row-split items: a lean kernel of its own (no shared memory, the row
// split's registers), so that it runs at the occupancy of the row split; one
// instantiation per access width VEC (the plan keeps the matrices of each
// width in a range of items of its own).
template <int VEC>
__global__ void __launch_bounds__(kThreads)
    batched_rows_kernel(const MatDesc* __restrict__ mats, const Item* __restrict__ items, long long n_items,
                        unsigned long long* counter) {
    for (long long it = next_item(counter); it < n_items; it = next_item(counter)) {
        const Item item = items[it];
        const MatDesc d = mats[item.mat];
        batched_rows_any<VEC>(d, item.a, item.b, item.kind_slab >> 1);
    }
}

// Merge-tile items.  Three CTAs per SM: caps the registers of the (inlined)
// worst-case tile variant at 80.
__global__ void __launch_bounds__(kThreads, 3)
    batched_tiles_kernel(const MatDesc* __restrict__ mats, const Item* __restrict__ items, long long n_items,
                         int* carry_row_all, int* head_row_all, int* status, unsigned long long* counter) {
    extern __shared__ __align__(128) unsigned char smem[];
    for (long long it = next_item(counter); it < n_items; it = next_item(counter)) {
        const Item item = items[it];
        const MatDesc d = mats[item.mat];
        const int slab = item.kind_slab >> 1;
        switch (d.W) {
            case 1: batched_tile<1>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
            case 2: batched_tile<2>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
            case 4: batched_tile<4>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
            case 8: batched_tile<8>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
            case 16: batched_tile<16>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
            default: batched_tile<32>(d, carry_row_all, head_row_all, item.a, slab, smem, status); break;
        }
    }
}

// FIXCARRYOUT over every merge matrix of the plan (global tile numbering;
// runs never cross matrices because a matrix's last tile has no carry).
__global__ void batched_fixup_kernel(const MatDesc* __restrict__ mats, const int* __restrict__ tile_mat, int total_tiles,
                                     const int* __restrict__ carry_row_all, const int* __restrict__ head_row_all,
                                     int* status) {
    const int i = blockIdx.x;
    const int R = carry_row_all[i];
    if (R < 0) return;
    const int b = tile_mat[i];
    if (i > 0 && tile_mat[i - 1] == b && carry_row_all[i - 1] == R) return;
    // the run's last tile j, 32 tiles per probe (each warp of the block finds the same j)
    const int lane = threadIdx.x & 31;
    int j = i;
    for (int base = i + 1;; base += 32) {
        const int t = base + lane;
        const unsigned same =
            __ballot_sync(kFullMask, t < total_tiles && tile_mat[t] == b && carry_row_all[t] == R);
        if (same != kFullMask) {
            j = base + __ffs(~same) - 2;
            break;
        }
    }
    if (j + 1 >= total_tiles || tile_mat[j + 1] != b || head_row_all[j + 1] != R) {
        if (threadIdx.x == 0) report(status, SPMM_ERR_BAD_CSR);
        return;
    }
    const MatDesc& d = mats[b];
    for (int c = threadIdx.x; c < d.n; c += blockDim.x) {
        float sum = 0.0f;
        for (int t = i; t <= j; ++t) sum += d.carry[(size_t)(t - d.tile_base) * d.n + c];
        sum += d.head[(size_t)(j + 1 - d.tile_base) * d.n + c];
        d.C[(long long)R * d.ldc + c] = sum;
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int status_of(cudaError_t e) {
    if (e == cudaSuccess) return SPMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPMM_ERR_ALLOC;
    if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidValue)
        return SPMM_ERR_LAUNCH;
    return SPMM_ERR_CUDA;
}

int lanes_for(int n) {
    const int chunks = (n + 3) / 4;
    int W = 1;
    while (W < chunks && W < 32) W <<= 1;
    return W;
}

int default_ips(int W) {
    const int ips = 2048 / (kThreads / W);
    return ips < 4 ? 4 : ips;
}

size_t merge_smem_bytes(int W, int ips) {
    switch (W) {
        case 1: return MergeSmem<float, 4, 1>::total(ips);
        case 2: return MergeSmem<float, 4, 2>::total(ips);
        case 4: return MergeSmem<float, 4, 4>::total(ips);
        case 8: return MergeSmem<float, 4, 8>::total(ips);
        case 16: return MergeSmem<float, 4, 16>::total(ips);
        default: return MergeSmem<float, 4, 32>::total(ips);
    }
}

// ------------------------------------------------------------------ autotuner cache

struct Choice {
    int alg;
    int ips_scale;  // merge: ips = default * 2^ips_scale (ips_scale in {-1, 0, 1})
    int lanes_div;  // row split: lanes per row = the full lane group / lanes_div (1, 2 or 4; more column slabs)
    int vec;        // row split: columns per lane access, 4 (one 16-byte vector) or 8 (two)
};

// Lanes per row of the row split for width n and vec columns per lane: the power of two covering
// the row's vectors (at most 32), divided by lanes_div.
int lanes_of(int n, int lanes_div, int vec = 4) {
    const int chunks = (std::max(n, 1) + vec - 1) / vec;
    int W = 1;
    while (W < chunks && W < 32) W <<= 1;
    return std::max(1, W / std::max(1, lanes_div));
}

// Two 16-byte vectors per lane need n, ldb and ldc to be multiples of 8.
bool two_vectors_ok(const spmm_batch_matrix_t& mt) { return mt.n % 8 == 0 && mt.ldb % 8 == 0 && mt.ldc % 8 == 0; }

using BucketKey = std::tuple<int, int, int, int>;  // (device SMs, n, floor(log2 m), mean-row-length bucket)
std::mutex g_tune_mu;
std::map<BucketKey, Choice> g_tune_cache;

BucketKey bucket_of(int sms, const spmm_batch_matrix_t& mt) {
    const int lm = mt.m > 0 ? (int)std::floor(std::log2((double)mt.m)) : 0;
    const double d = mt.m > 0 ? (double)mt.nnz / mt.m : 0.0;
    const int db = d < 4 ? 0 : d < 8 ? 1 : d < 16 ? 2 : d < 32 ? 3 : 4;
    return BucketKey{sms, mt.n, lm, db};
}

}  // namespace
}  // namespace spmm

using namespace spmm;

struct spmm_batched_plan {
    int device = 0;
    int count = 0;
    std::vector<int> algs;
    std::vector<int> ips;
    std::vector<int> lanes;  // lanes per row of each matrix
    std::vector<int> vecs;   // columns per lane access of each matrix
    unsigned char* mem = nullptr;
    MatDesc* d_mats = nullptr;
    Item* d_items = nullptr;       // row-split items, then merge-tile items
    long long n_items = 0;
    long long n_row_items = 0;   // row-split items (one-vector matrices first, then two-vector ones)
    long long n_row_items8 = 0;  // of which the last ones, of matrices read with two vectors per lane
    int grid_rows8 = 0;
    int grid_rows = 0;
    int total_tiles = 0;
    int* d_tile_mat = nullptr;
    int* d_carry_row = nullptr;
    int* d_head_row = nullptr;
    int* d_status = nullptr;
    unsigned long long* d_counters = nullptr;  // work-item counters of the persistent kernels (tiles, rows, rows x2)
    cudaStream_t side = nullptr;                // the row-split kernel runs here, beside the merge tiles
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    size_t smem = 0;
    int grid = 0;
    cudaGraphExec_t exec = nullptr;
    std::vector<spmm_batch_matrix_t> mats;
    std::vector<long long> max_row;
};

namespace spmm {
namespace {

void destroy_plan(spmm_batched_plan* p) {
    if (!p) return;
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->ev_fork) cudaEventDestroy(p->ev_fork);
    if (p->ev_join) cudaEventDestroy(p->ev_join);
    if (p->side) cudaStreamDestroy(p->side);
    if (p->mem) cudaFree(p->mem);
    delete p;
}

// Build a plan for matrices `mats` with per-matrix (alg, ips) already chosen.
int build_plan(const std::vector<spmm_batch_matrix_t>& mats, const std::vector<int>& algs, const std::vector<int>& ips,
               const std::vector<int>& lanes, const std::vector<int>& vecs, cudaStream_t s, spmm_batched_plan** out) {
    auto* p = new spmm_batched_plan();
    p->count = (int)mats.size();
    p->algs = algs;
    p->ips = ips;
    p->lanes = lanes;
    p->vecs = vecs;
    p->mats = mats;
    cudaGetDevice(&p->device);
    std::vector<MatDesc> descs(mats.size());
    std::vector<Item> items, tile_items;
    std::vector<int> row_mats;  // matrices computed by row split
    std::vector<int> tile_mat;
    size_t carry_floats = 0, limit_entries = 0;
    size_t smem = 0;
    for (size_t b = 0; b < mats.size(); ++b) {
        const auto& mt = mats[b];
        MatDesc& d = descs[b];
        d.m = mt.m;
        d.k = mt.k;
        d.n = mt.n;
        d.nnz = mt.nnz;
        d.ldb = mt.ldb;
        d.ldc = mt.ldc;
        d.row_ptr = mt.row_ptr;
        d.col_ind = mt.col_ind;
        d.vals = mt.vals;
        d.B = mt.B;
        d.C = mt.C;
        d.alg = algs[b];
        d.W = lanes[b];
        d.vec = d.alg == SPMM_ALG_MERGE ? 4 : vecs[b];
        d.slabs = ((mt.n + d.vec - 1) / d.vec + d.W - 1) / d.W;
        d.ips = ips[b];
        d.tile_base = (int)tile_mat.size();
        if (mt.m == 0 || mt.n == 0) {
            d.num_tiles = 0;
            continue;
        }
        if (d.alg == SPMM_ALG_MERGE) {
            const long long ipt = (long long)(kThreads / d.W) * d.ips;
            d.num_tiles = (int)((mt.m + mt.nnz + ipt - 1) / ipt);
            for (int sl = 0; sl < d.slabs; ++sl)
                for (int t = 0; t < d.num_tiles; ++t) tile_items.push_back(Item{(int)b, 1 | (sl << 1), t, 0});
            for (int t = 0; t < d.num_tiles; ++t) tile_mat.push_back((int)b);
            carry_floats += (size_t)d.num_tiles * mt.n;
            limit_entries += d.num_tiles + 1;
            smem = std::max(smem, merge_smem_bytes(d.W, d.ips));
        } else {
            d.num_tiles = 0;
            row_mats.push_back((int)b);
        }
    }
    // row-split chunks, largest matrices first: the big matrices' rows of B are then gathered
    // while few other matrices compete for L2, and the small ones fill the tail of the launch
    std::stable_sort(row_mats.begin(), row_mats.end(), [&](int x, int y) {
        if (descs[x].vec != descs[y].vec) return descs[x].vec < descs[y].vec;  // one-vector matrices first
        return mats[x].nnz > mats[y].nnz;
    });
    long long first8 = -1;
    for (const int b : row_mats) {
        if (descs[b].vec == 8 && first8 < 0) first8 = (long long)items.size();
        const auto& mt = mats[b];
        const MatDesc& d = descs[b];
        const int chunk = kRowsPerGroupPerItem * (kThreads / d.W);
        for (int sl = 0; sl < d.slabs; ++sl)
            for (int r = 0; r < mt.m; r += chunk) items.push_back(Item{b, sl << 1, r, std::min(mt.m, r + chunk)});
    }
    p->n_row_items = (long long)items.size();
    p->n_row_items8 = first8 < 0 ? 0 : p->n_row_items - first8;
    items.insert(items.end(), tile_items.begin(), tile_items.end());
    p->n_items = (long long)items.size();
    p->total_tiles = (int)tile_mat.size();
    // one device allocation: descriptors, items, tile map, row marks, limits, carries, heads, status
    const size_t sz_desc = a256(descs.size() * sizeof(MatDesc)), sz_items = a256(items.size() * sizeof(Item)),
                 sz_tm = a256(tile_mat.size() * 4), sz_lim = a256(limit_entries * sizeof(int2)),
                 sz_carry = a256(carry_floats * 4);
    const size_t total = sz_desc + sz_items + 3 * sz_tm + sz_lim + 2 * sz_carry + 256;
    if (cudaMalloc(&p->mem, total) != cudaSuccess) {
        delete p;
        return SPMM_ERR_ALLOC;
    }
    unsigned char* q = p->mem;
    p->d_mats = reinterpret_cast<MatDesc*>(q);
    q += sz_desc;
    p->d_items = reinterpret_cast<Item*>(q);
    q += sz_items;
    p->d_tile_mat = reinterpret_cast<int*>(q);
    q += sz_tm;
    p->d_carry_row = reinterpret_cast<int*>(q);
    q += sz_tm;
    p->d_head_row = reinterpret_cast<int*>(q);
    q += sz_tm;
    int2* lim = reinterpret_cast<int2*>(q);
    q += sz_lim;
    float* carry = reinterpret_cast<float*>(q);
    q += sz_carry;
    float* head = reinterpret_cast<float*>(q);
    q += sz_carry;
    p->d_status = reinterpret_cast<int*>(q);
    p->d_counters = reinterpret_cast<unsigned long long*>(q + 16);
    size_t lim_off = 0, carry_off = 0;
    int st = SPMM_OK;
    for (size_t b = 0; b < descs.size() && st == SPMM_OK; ++b) {
        MatDesc& d = descs[b];
        if (d.alg != SPMM_ALG_MERGE || d.num_tiles == 0) continue;
        d.limits = lim + lim_off;
        d.carry = carry + carry_off;
        d.head = head + carry_off;
        st = spmm_merge_partition(d.m, d.nnz, d.row_ptr, (kThreads / d.W) * d.ips, d.num_tiles,
                                  reinterpret_cast<int*>(lim + lim_off), s);
        lim_off += d.num_tiles + 1;
        carry_off += (size_t)d.num_tiles * d.n;
    }
    cudaError_t e = cudaSuccess;
    if (st == SPMM_OK) e = cudaMemcpyAsync(p->d_mats, descs.data(), descs.size() * sizeof(MatDesc), cudaMemcpyHostToDevice, s);
    if (st == SPMM_OK && e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(p->d_items, items.data(), items.size() * sizeof(Item), cudaMemcpyHostToDevice, s);
    if (st == SPMM_OK && e == cudaSuccess && !tile_mat.empty())
        e = cudaMemcpyAsync(p->d_tile_mat, tile_mat.data(), tile_mat.size() * 4, cudaMemcpyHostToDevice, s);
    if (st == SPMM_OK && e == cudaSuccess) e = cudaMemsetAsync(p->d_status, 0, 4, s);
    if (st == SPMM_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);  // host vectors die with this call
    if (st == SPMM_OK && e != cudaSuccess) st = status_of(e);
    p->smem = smem;
    if (st == SPMM_OK && smem > 48 * 1024)
        st = status_of(cudaFuncSetAttribute(batched_tiles_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int blocks = 0, blocks_rows = 0, blocks_rows8 = 0, sms = 0;
    if (st == SPMM_OK)
        st = status_of(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, batched_tiles_kernel, kThreads, smem));
    if (st == SPMM_OK)
        st = status_of(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_rows, batched_rows_kernel<4>, kThreads, 0));
    if (st == SPMM_OK)
        st = status_of(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_rows8, batched_rows_kernel<8>, kThreads, 0));
    if (st == SPMM_OK) st = status_of(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device));
    if (st == SPMM_OK && p->n_row_items > 0 && p->n_items > p->n_row_items) {
        st = status_of(cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking));
        if (st == SPMM_OK) st = status_of(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
        if (st == SPMM_OK) st = status_of(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
    }
    if (st != SPMM_OK) {
        destroy_plan(p);
        return st;
    }
    const long long n_tile_items = p->n_items - p->n_row_items;
    p->grid = (int)std::max<long long>(1, std::min<long long>((long long)std::max(blocks, 1) * sms, n_tile_items));
    const long long n_row4 = p->n_row_items - p->n_row_items8;
    p->grid_rows = (int)std::max<long long>(1, std::min<long long>((long long)std::max(blocks_rows, 1) * sms, n_row4));
    p->grid_rows8 =
        (int)std::max<long long>(1, std::min<long long>((long long)std::max(blocks_rows8, 1) * sms, p->n_row_items8));
    *out = p;
    return SPMM_OK;
}

// One run: zero the work counters, then the row-split kernel (on the plan's side stream when the
// plan also has merge tiles, so that the two persistent kernels share the GPU) and the merge-tile
// kernel followed by the fix-up on `s`; `s` then waits for the side stream.
int run_plan(const spmm_batched_plan* p, cudaStream_t s) {
    const long long n_tile_items = p->n_items - p->n_row_items;
    if (p->n_items > 0) {
        const cudaError_t e = cudaMemsetAsync(p->d_counters, 0, 3 * sizeof(unsigned long long), s);
        if (e != cudaSuccess) return status_of(e);
    }
    const bool fork = p->side && n_tile_items > 0 && p->n_row_items > 0;
    cudaStream_t rs = s;
    if (fork) {
        cudaError_t e = cudaEventRecord(p->ev_fork, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->side, p->ev_fork, 0);
        if (e != cudaSuccess) return status_of(e);
        rs = p->side;
    }
    int st = SPMM_OK;
    const long long n_row4 = p->n_row_items - p->n_row_items8;
    if (n_row4 > 0) {
        batched_rows_kernel<4><<<p->grid_rows, kThreads, 0, rs>>>(p->d_mats, p->d_items, n_row4, p->d_counters + 1);
        st = status_of(cudaGetLastError());
        if (st == SPMM_OK) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    if (st == SPMM_OK && p->n_row_items8 > 0) {
        batched_rows_kernel<8><<<p->grid_rows8, kThreads, 0, rs>>>(p->d_mats, p->d_items + n_row4, p->n_row_items8,
                                                                   p->d_counters + 2);
        st = status_of(cudaGetLastError());
        if (st == SPMM_OK) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    if (st == SPMM_OK && n_tile_items > 0) {
        batched_tiles_kernel<<<p->grid, kThreads, p->smem, s>>>(p->d_mats, p->d_items + p->n_row_items, n_tile_items,
                                                               p->d_carry_row, p->d_head_row, p->d_status,
                                                               p->d_counters);
        st = status_of(cudaGetLastError());
        if (st == SPMM_OK) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    if (st == SPMM_OK && p->total_tiles > 1) {
        batched_fixup_kernel<<<p->total_tiles, 128, 0, s>>>(p->d_mats, p->d_tile_mat, p->total_tiles, p->d_carry_row,
                                                           p->d_head_row, p->d_status);
        st = status_of(cudaGetLastError());
        if (st == SPMM_OK) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    if (fork) {  // joined whatever happened above, so that a capture ends with every stream joined
        cudaError_t e = cudaEventRecord(p->ev_join, p->side);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->ev_join, 0);
        if (st == SPMM_OK && e != cudaSuccess) st = status_of(e);
    }
    return st;
}

// Time one candidate schedule for a sample of matrices (median of 3 runs, ms).
float time_candidate(const std::vector<spmm_batch_matrix_t>& sample, const Choice& c, cudaStream_t s) {
    std::vector<int> algs(sample.size(), c.alg), ips(sample.size()), lanes(sample.size()), vecs(sample.size(), 4);
    for (size_t i = 0; i < sample.size(); ++i) {
        if (c.alg != SPMM_ALG_MERGE && c.vec == 8 && two_vectors_ok(sample[i])) vecs[i] = 8;
        lanes[i] = c.alg == SPMM_ALG_MERGE ? lanes_for(std::max(sample[i].n, 1)) : lanes_of(sample[i].n, c.lanes_div, vecs[i]);
        const int d = default_ips(lanes[i]);
        ips[i] = c.ips_scale > 0 ? d * 2 : c.ips_scale < 0 ? std::max(4, d / 2) : d;
    }
    spmm_batched_plan* p = nullptr;
    if (build_plan(sample, algs, ips, lanes, vecs, s, &p) != SPMM_OK) return INFINITY;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    run_plan(p, s);  // warm-up
    std::vector<float> ts;
    for (int r = 0; r < 3; ++r) {
        cudaEventRecord(e0, s);
        run_plan(p, s);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = INFINITY;
        cudaEventElapsedTime(&ms, e0, e1);
        ts.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    destroy_plan(p);
    std::sort(ts.begin(), ts.end());
    return ts[1];
}

}  // namespace
}  // namespace spmm

extern "C" {

int spmm_batched_plan_create(int count, const spmm_batch_matrix_t* mats, int policy, void* stream,
                             spmm_batched_plan_t** plan) {
    if (!plan || count < 0 || (count > 0 && !mats)) return SPMM_ERR_INVALID_VALUE;
    if (policy != SPMM_BATCHED_MODEL && policy != SPMM_BATCHED_AUTOTUNE && policy != SPMM_BATCHED_ROW_SPLIT &&
        policy != SPMM_BATCHED_MERGE && policy != SPMM_BATCHED_ROW_SPLIT_X2)
        return SPMM_ERR_INVALID_VALUE;
    *plan = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<spmm_batch_matrix_t> v(mats, mats + count);
    for (const auto& mt : v) {
        if (mt.m < 0 || mt.k < 0 || mt.n < 0 || mt.nnz < 0 || mt.nnz > INT_MAX) return SPMM_ERR_INVALID_VALUE;
        if (mt.m > 0 && mt.n > 0) {
            if (!mt.row_ptr || !mt.C || mt.ldc < mt.n || (mt.nnz > 0 && (!mt.col_ind || !mt.vals || !mt.B || mt.ldb < mt.n)))
                return SPMM_ERR_INVALID_VALUE;
            if (mt.ldb > 0xffffffffLL / 4) return SPMM_ERR_INVALID_VALUE;  // rows of B < 4 GiB apart
            // the batched kernel uses 16-byte accesses only
            if (mt.n % 4 || mt.ldb % 4 || mt.ldc % 4 || ((uintptr_t)mt.B % 16) || ((uintptr_t)mt.C % 16))
                return SPMM_ERR_UNSUPPORTED;
        }
    }
    // longest rows (for the selector): host copies of every row_ptr
    std::vector<long long> lmax(v.size(), 0);
    if (policy == SPMM_BATCHED_MODEL) {
        std::vector<std::vector<int>> rps(v.size());
        for (size_t b = 0; b < v.size(); ++b) {
            if (v[b].m <= 0) continue;
            rps[b].resize((size_t)v[b].m + 1);
            if (cudaMemcpyAsync(rps[b].data(), v[b].row_ptr, rps[b].size() * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
                return SPMM_ERR_CUDA;
        }
        if (cudaStreamSynchronize(s) != cudaSuccess) return SPMM_ERR_CUDA;
        for (size_t b = 0; b < v.size(); ++b)
            for (int i = 0; i < v[b].m; ++i) lmax[b] = std::max<long long>(lmax[b], rps[b][i + 1] - rps[b][i]);
    }
    std::vector<int> algs(v.size()), ips(v.size());
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (policy == SPMM_BATCHED_AUTOTUNE) {
        // group the matrices by bucket; time candidates on up to 8 matrices of every bucket not yet cached
        std::map<BucketKey, std::vector<size_t>> groups;
        for (size_t b = 0; b < v.size(); ++b) groups[bucket_of(sms, v[b])].push_back(b);
        for (auto& kv : groups) {
            {
                std::lock_guard<std::mutex> lock(g_tune_mu);
                if (g_tune_cache.count(kv.first)) continue;
            }
            // a sample big enough that the timed kernel runs well above launch latency:
            // matrices of the bucket until 4M rows + nonzeros (at most 64 matrices)
            std::vector<spmm_batch_matrix_t> sample;
            long long work = 0;
            for (size_t i = 0; i < kv.second.size() && sample.size() < 64 && work < (4LL << 20); ++i) {
                sample.push_back(v[kv.second[i]]);
                work += v[kv.second[i]].m + v[kv.second[i]].nnz;
            }
            // In the full batch a bucket's matrices run on a GPU kept busy by the rest of the batch; a
            // small sample alone would be timed on its tail.  Repeat the sample (same matrices, same
            // outputs, identical values written) until it holds 32M rows + nonzeros, at most 32 times.
            const size_t base = sample.size();
            for (int rep = 1; rep < 32 && work > 0 && work < (32LL << 20); ++rep) {
                long long w = 0;
                for (size_t i = 0; i < base; ++i) {
                    sample.push_back(sample[i]);
                    w += sample[i].m + sample[i].nnz;
                }
                work += w;
            }
            // candidates: row split with one and with two 16-byte vectors per lane, each with the
            // full lane group and with 1/2 and 1/4 of it (column slabs); merge based with three
            // tile sizes
            std::vector<Choice> cands = {{SPMM_ALG_ROW_SPLIT, 0, 1, 4}, {SPMM_ALG_ROW_SPLIT, 0, 2, 4},
                                         {SPMM_ALG_ROW_SPLIT, 0, 4, 4}, {SPMM_ALG_ROW_SPLIT, 0, 1, 8},
                                         {SPMM_ALG_ROW_SPLIT, 0, 2, 8}, {SPMM_ALG_ROW_SPLIT, 0, 4, 8},
                                         {SPMM_ALG_MERGE, 0, 1, 4},     {SPMM_ALG_MERGE, -1, 1, 4},
                                         {SPMM_ALG_MERGE, 1, 1, 4}};
            Choice best = cands[0];
            float best_ms = INFINITY;
            const int n0 = v[kv.second[0]].n;  // every matrix of a bucket has the same n
            const bool two_ok = two_vectors_ok(v[kv.second[0]]);
            for (const Choice& c : cands) {
                if (c.vec == 8 && !two_ok) continue;
                if (c.lanes_div > 1 && lanes_of(n0, c.lanes_div, c.vec) == lanes_of(n0, c.lanes_div / 2, c.vec))
                    continue;  // no narrower lane group for this width
                const float ms = time_candidate(sample, c, s);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
            std::lock_guard<std::mutex> lock(g_tune_mu);
            g_tune_cache[kv.first] = best;
        }
    }
    std::vector<int> lanes(v.size()), vecs(v.size(), 4);
    for (size_t b = 0; b < v.size(); ++b) {
        int alg = SPMM_ALG_ROW_SPLIT, sc = 0, div = 1, vec = 4;
        if (policy == SPMM_BATCHED_MERGE) {
            alg = SPMM_ALG_MERGE;
        } else if (policy == SPMM_BATCHED_ROW_SPLIT_X2) {
            vec = two_vectors_ok(v[b]) ? 8 : 4;
        } else if (policy == SPMM_BATCHED_MODEL) {
            // Inside the batch the merge tiles run about 2x slower than the row chunks (no bulk-copy
            // staging, 24 warps per SM; measured on the 2048-matrix batch: every matrix merge 23.9 ms,
            // every matrix row split 10.7 ms), so merge only where the longest row would make the
            // matrix's row chunks the critical path (the Type 1 guard of the GB300 selector)
            const bool type1 = lmax[b] > 1024 && lmax[b] * 8192 > v[b].nnz;
            alg = type1 ? SPMM_ALG_MERGE : SPMM_ALG_ROW_SPLIT;
            // one 16-byte vector per lane: two made the 2048-matrix batch slower (10.1 -> 12.8 ms)
        } else if (policy == SPMM_BATCHED_AUTOTUNE) {
            std::lock_guard<std::mutex> lock(g_tune_mu);
            const Choice c = g_tune_cache[bucket_of(sms, v[b])];
            alg = c.alg;
            sc = c.ips_scale;
            div = c.lanes_div;
            vec = c.vec == 8 && two_vectors_ok(v[b]) ? 8 : 4;
        }
        if (alg == SPMM_ALG_MERGE) vec = 4;
        vecs[b] = vec;
        lanes[b] = alg == SPMM_ALG_MERGE ? lanes_for(std::max(v[b].n, 1)) : lanes_of(v[b].n, div, vec);
        const int d = default_ips(lanes[b]);
        algs[b] = alg;
        ips[b] = sc > 0 ? d * 2 : sc < 0 ? std::max(4, d / 2) : d;
    }
    spmm_batched_plan* p = nullptr;
    const int st = build_plan(v, algs, ips, lanes, vecs, s, &p);
    if (st != SPMM_OK) return st;
    p->max_row = lmax;
    *plan = p;
    return SPMM_OK;
}

int spmm_batched_run(const spmm_batched_plan_t* plan, void* stream) {
    if (!plan) return SPMM_ERR_INVALID_VALUE;
    return run_plan(plan, (cudaStream_t)stream);
}

int spmm_batched_capture_graph(spmm_batched_plan_t* plan, void* stream) {
    (void)stream;  // capture runs on a private stream: the legacy default stream cannot be captured
    if (!plan) return SPMM_ERR_INVALID_VALUE;
    if (plan->exec) {
        cudaGraphExecDestroy(plan->exec);
        plan->exec = nullptr;
    }
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return status_of(e);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        cudaStreamDestroy(s);
        return status_of(e);
    }
    const long long before = g_launches.load();
    const int st = run_plan(plan, s);
    e = cudaStreamEndCapture(s, &g);
    g_launches.store(before);  // captured launches run only when the graph is launched
    cudaStreamDestroy(s);
    if (st != SPMM_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return status_of(e);
    e = cudaGraphInstantiate(&plan->exec, g, 0);
    cudaGraphDestroy(g);
    return status_of(e);
}

int spmm_batched_launch_graph(const spmm_batched_plan_t* plan, void* stream) {
    if (!plan || !plan->exec) return SPMM_ERR_INVALID_VALUE;
    const cudaError_t e = cudaGraphLaunch(plan->exec, (cudaStream_t)stream);
    if (e == cudaSuccess)
        g_launches.fetch_add((plan->n_row_items > plan->n_row_items8) + (plan->n_row_items8 > 0) +
                                 (plan->n_items > plan->n_row_items) + (plan->total_tiles > 1),
                             std::memory_order_relaxed);
    return status_of(e);
}

int spmm_batched_run_unfused(const spmm_batched_plan_t* plan, void* stream) {
    if (!plan) return SPMM_ERR_INVALID_VALUE;
    for (int b = 0; b < plan->count; ++b) {
        const auto& mt = plan->mats[b];
        spmm_tuning_t t{};
        t.items_per_subwarp = plan->ips[b];
        t.lanes_per_row = std::min(32, plan->lanes[b] * plan->vecs[b] / 4);  // the same columns per lane group
        const int st = spmm_csr_ex(mt.m, mt.k, mt.n, mt.nnz, mt.row_ptr, mt.col_ind, mt.vals, SPMM_F32, mt.B, SPMM_F32,
                                   mt.ldb, mt.C, SPMM_F32, mt.ldc, plan->algs[b], &t, nullptr, 0, nullptr, stream);
        if (st != SPMM_OK) return st;
    }
    return SPMM_OK;
}

int spmm_batched_plan_query(const spmm_batched_plan_t* plan, int* algs, long long* num_items, int* num_tiles) {
    if (!plan) return SPMM_ERR_INVALID_VALUE;
    if (algs)
        for (int b = 0; b < plan->count; ++b) algs[b] = plan->algs[b];
    if (num_items) *num_items = plan->n_items;
    if (num_tiles) *num_tiles = plan->total_tiles;
    return SPMM_OK;
}

int spmm_batched_plan_destroy(spmm_batched_plan_t* plan) {
    destroy_plan(plan);
    return SPMM_OK;
}

long long spmm_autotune_cache_entries(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    return (long long)g_tune_cache.size();
}

int spmm_autotune_cache_clear(void) {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache.clear();
    return SPMM_OK;
}

}  // extern "C"
