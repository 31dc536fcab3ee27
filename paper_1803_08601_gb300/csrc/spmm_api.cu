// C ABI of the SpMM library (include/spmm.h): argument checks, the Section 5.4
// heuristic, launch-shape selection, merge workspace layout, and dispatch to
// the per-dtype launchers.
#include <cstdint>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "launch.cuh"

namespace spmm {

std::atomic<long long> g_launches{0};


// Merge-path tiles (Section 4.2): the path that merges the row end offsets
// row_ptr[1..m] with the nonzero indices 0..nnz-1 is cut into tiles of equal
// length (rows + nonzeros).
//
// Phase 1 (PARTITIONSPMM): one thread per tile boundary finds the boundary's
// (rows, nonzeros) coordinate by binary search on its diagonal.
// One warp per tile boundary: a 32-ary search on the boundary's diagonal.  The
// predicate "row x ends no later than nonzero d-x-1" (row_ptr[x+1] <= d-x-1)
// holds exactly for x below the number of row ends among the first d merged
// items; every round the 32 lanes test 32 evenly spaced candidates and the
// ballot narrows the interval about 32-fold, so a diagonal of 10^7 items
// needs about 6 rounds of dependent loads instead of 24.
__global__ void merge_partition_kernel(const int* __restrict__ row_ptr, int m, long long nnz, int items_per_tile,
                                       int num_tiles, int2* __restrict__ limits) {
    pdl_launch_dependents();  // the merge kernel may be scheduled now; it waits for this grid to finish
    const int lane = threadIdx.x & 31;
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t > num_tiles) return;  // whole warps exit together
    const long long total = (long long)m + nnz;
    long long d = t * items_per_tile;
    if (d > total) d = total;
    long long lo = d - nnz > 0 ? d - nnz : 0;  // answer in [lo, hi]
    long long hi = d < m ? d : m;
    while (hi > lo) {
        const long long span = hi - lo;
        const long long x = lo + (span * lane) / 32;  // candidates lo .. hi-1, increasing with the lane
        const bool p = (long long)__ldg(row_ptr + x + 1) <= d - x - 1;
        const unsigned ball = __ballot_sync(kFullMask, p);
        const int cnt = __popc(ball);  // the predicate holds on a prefix of the lanes
        if (cnt == 0) {
            hi = lo;
        } else {
            const long long x_last = lo + (span * (cnt - 1)) / 32;
            if (cnt < 32) hi = lo + (span * cnt) / 32;
            lo = x_last + 1;
        }
    }
    if (lane == 0) limits[t] = make_int2((int)lo, (int)(d - lo));
}

// Bounded-wait self test: waits on a phase that nothing completes.
__global__ void bounded_wait_probe_kernel(int* status, unsigned long long limit_ns) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit_ns);
    if (__syncthreads_or(!ok) && threadIdx.x == 0) report(status, SPMM_ERR_TIMEOUT);
}


namespace {

constexpr double kPaperThreshold = 9.35;  // Section 5.4
constexpr unsigned long long kWaitLimitNs = 1000000000ull;  // 1 s per bounded wait
constexpr size_t kMaxSmem = 200 * 1024;  // dynamic shared memory the merge kernel may request

struct TypeCombo {
    int tv, tb, tc;
    Launchers (*make)();
};

const TypeCombo kCombos[] = {
    {SPMM_F32, SPMM_F32, SPMM_F32, &launchers_f32_f32_f32},
    {SPMM_BF16, SPMM_BF16, SPMM_BF16, &launchers_bf16_bf16_bf16},
    {SPMM_BF16, SPMM_BF16, SPMM_F32, &launchers_bf16_bf16_f32},
    {SPMM_BF16, SPMM_F16, SPMM_F16, &launchers_bf16_f16_f16},
    {SPMM_BF16, SPMM_F16, SPMM_F32, &launchers_bf16_f16_f32},
    {SPMM_F16, SPMM_F16, SPMM_F16, &launchers_f16_f16_f16},
    {SPMM_F16, SPMM_F16, SPMM_F32, &launchers_f16_f16_f32},
};

const Launchers* find_launchers(int tv, int tb, int tc) {
    static Launchers table[sizeof(kCombos) / sizeof(kCombos[0])];
    static std::once_flag once;
    std::call_once(once, [] {
        for (size_t i = 0; i < sizeof(kCombos) / sizeof(kCombos[0]); ++i) table[i] = kCombos[i].make();
    });
    for (size_t i = 0; i < sizeof(kCombos) / sizeof(kCombos[0]); ++i)
        if (kCombos[i].tv == tv && kCombos[i].tb == tb && kCombos[i].tc == tc) return &table[i];
    return nullptr;
}

int dtype_size(int t) { return t == SPMM_F32 ? 4 : (t == SPMM_BF16 || t == SPMM_F16) ? 2 : 0; }

int pow2_ceil(long long x) {
    int p = 1;
    while (p < x && p < 32) p <<= 1;
    return p;
}

double threshold_of(const spmm_tuning_t* t) {
    return (t && t->merge_threshold > 0.0) ? t->merge_threshold : kPaperThreshold;
}

int resolve_alg(int alg, int m, long long nnz, const spmm_tuning_t* t) {
    if (alg != SPMM_ALG_AUTO) return alg;
    return spmm_select_alg(m, nnz, threshold_of(t));
}

// row_ptr[i] -= base for i < count: a row chunk's offsets made to start at 0.
__global__ void rebase_kernel(int* __restrict__ row_ptr, int count, int base) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) row_ptr[i] -= base;
}

// Longest row by a grid-stride max reduction over row_ptr differences into
// out[0] (zeroed before the launch); the first thread also copies
// row_ptr[m] (= nnz) to out[1].
__global__ void row_length_max_kernel(const int* __restrict__ row_ptr, int m, int* __restrict__ out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) out[1] = __ldg(row_ptr + m);
    int best = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
        best = max(best, __ldg(row_ptr + i + 1) - __ldg(row_ptr + i));
    best = __reduce_max_sync(0xffffffffu, best);
    if ((threadIdx.x & 31) == 0 && best > 0) atomicMax(out, best);
}

// Launch shape for a given access width.  The lane group of a row covers
// W * vec columns; W is the smallest power of two whose group spans the
// columns of one slab.
bool shape_for(int n, int vec, const spmm_tuning_t* t, Shape* s) {
    s->vec = vec;
    const long long chunks = ((long long)n + vec - 1) / vec;
    int W;
    if (t && t->lanes_per_row > 0) {
        W = t->lanes_per_row;
        if (W > 32 || (W & (W - 1))) return false;
    } else if (t && t->column_slabs > 0) {
        W = pow2_ceil((chunks + t->column_slabs - 1) / t->column_slabs);
    } else {
        W = pow2_ceil(chunks);
    }
    s->W = W;
    s->slabs = (int)((chunks + W - 1) / W);
    if (s->slabs > 65535) return false;
    const int groups = merge_cta_threads(W) / W;  // lane groups per merge CTA
    int ips = (t && t->items_per_subwarp > 0) ? t->items_per_subwarp : merge_tile_items(W) / groups;
    if (ips < 4) ips = 4;
    if (ips > 4096) ips = 4096;
    s->ips = ips;
    return true;
}

// 16-byte accesses when n, both leading dimensions and both base pointers allow them.
bool choose_shape(int n, int tb, int tc, const void* B, long long ldb, const void* C, long long ldc,
                  const spmm_tuning_t* t, Shape* s) {
    const int V = 16 / dtype_size(tb);
    const bool vec_ok = n % V == 0 && ldb % V == 0 && ldc % V == 0 && ((uintptr_t)B % 16) == 0 &&
                        ((uintptr_t)C % (uintptr_t)(V * dtype_size(tc))) == 0;
    return shape_for(n, vec_ok ? V : 1, t, s);
}

// The hybrid row split reads float32 rows of B as two 16-byte vectors per
// lane (8 columns, half as many gathers in flight) once rows hold 32 columns
// or more: on a 1M x 1M power-law matrix, n = 32 / 64 / 128, 0.354 / 0.644 /
// 1.217 -> 0.319 / 0.584 / 1.129 ms; at n = 8 one vector per lane stays faster.
bool hybrid_two_vectors(int n, int b_type, long long ldb, long long ldc, const Shape& s) {
    return b_type == SPMM_F32 && s.vec == 4 && n >= 32 && n % 8 == 0 && ldb % 8 == 0 && ldc % 8 == 0;
}

// Column slabs when B is much larger than L2 and its rows are wide: each pass
// then gathers half of every row, over a B slab twice as likely to be found in
// L2 (measured on GB300: merge with 512-byte rows and row split with >= 256-byte
// rows of a B beyond L2 gain 6-14 %; narrower rows lose).
int default_slabs(int alg, int k, int n, int b_type) {
    static std::atomic<int> l2_cache[64];  // 0 until first queried; every thread stores the same value
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    int l2 = l2_cache[dev].load(std::memory_order_relaxed);
    if (l2 == 0) {
        if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) return 1;
        l2_cache[dev].store(l2, std::memory_order_relaxed);
    }
    const long long row_bytes = (long long)n * dtype_size(b_type);
    if ((long long)k * row_bytes <= 2LL * l2) return 1;
    const long long min_row = alg == SPMM_ALG_MERGE ? 512 : 256;
    return row_bytes >= min_row ? 2 : 1;
}

struct MergeLayout {
    int num_tiles;
    size_t off_limits, off_carry_row, off_head_row, off_carry, off_head, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

MergeLayout merge_layout_items(int m, long long nnz, int n, long long ipt) {
    MergeLayout L{};
    const long long total = (long long)m + nnz;
    L.num_tiles = (int)((total + ipt - 1) / ipt);
    size_t off = 0;
    L.off_limits = off;
    off = align256(off + (size_t)(L.num_tiles + 1) * sizeof(int2));
    L.off_carry_row = off;
    off = align256(off + (size_t)L.num_tiles * 4);
    L.off_head_row = off;
    off = align256(off + (size_t)L.num_tiles * 4);
    L.off_carry = off;
    off = align256(off + (size_t)L.num_tiles * n * 4);
    L.off_head = off;
    off = align256(off + (size_t)L.num_tiles * n * 4);
    L.total = off;
    return L;
}

MergeLayout merge_layout(int m, long long nnz, int n, const Shape& s) {
    return merge_layout_items(m, nnz, n, (long long)(merge_cta_threads(s.W) / s.W) * s.ips);
}

// Hybrid row split (SPMM_ALG_ROW_SPLIT_HYBRID).  A lane group of W lanes
// takes BS = max(W, kUnroll) nonzeros per batch.  Rows of at most long_len
// nonzeros stay in the row-block pass (long_len = max(32, BS) unless the
// caller sets it), whose warps own 128 consecutive rows (64 for W >= 16);
// queued rows of at most mid_len = 4 long_len go to one lane group each; with
// W >= 4 those of more than mid_split = 2 long_len are taken first, so a warp's
// work item holds rows of similar length and the longest items do not come
// last (measured on the 1M x 1M power-law matrix, same box, alternating runs:
// n = 16 0.199 -> 0.193 ms, n = 32 0.303 -> 0.298 ms; with W = 2, n = 8, it
// lost 3 %, so there every mid row is one queue); a warp segment holds 16 warp
// batches (32 / W lane groups x BS nonzeros each).
// The defaults are the fastest of a sweep of long_len in {16, ..., 256} and
// block_rows in {64, 128, 256} on a 1M x 1M power-law matrix, n = 8 to 128.
struct HybridLayout {
    int long_len, mid_len, mid_split, seg_len, block_rows, max_mid, max_singles, max_parts;
    size_t off_counts, off_mid, off_single, off_multi, off_arrive, off_partial, total;
};

HybridLayout hybrid_layout(int m, long long nnz, int n, const Shape& s, const spmm_tuning_t& t) {
    HybridLayout H{};
    const int bs = std::max(s.W, kUnroll);
    const long long def_long = std::max(32, bs);
    const long long long_len = t.long_row_len > 0 ? t.long_row_len : def_long;
    H.long_len = (int)std::min<long long>(long_len, 0x3fffffffLL);
    H.mid_len = (int)std::min<long long>(4 * long_len, 0x7fffffffLL);
    H.mid_split = s.W >= 4 ? (int)std::min<long long>(2 * long_len, H.mid_len) : H.mid_len;  // split_mid_rows
    H.seg_len = 16 * (32 / s.W) * bs;
    H.block_rows = t.block_rows > 0 ? std::min(t.block_rows, kMaxBlockRows) : (s.W >= 16 ? 64 : 128);
    // mid rows: at most nnz / (long_len + 1) rows are longer than long_len; single rows: at most
    // nnz / (mid_len + 1); partial slots: a row of L > seg_len nonzeros takes at most
    // ceil(L / seg_len) <= L / seg_len + 1 of them, and there are at most nnz / (seg_len + 1) such rows
    const long long mids = std::min<long long>(m, nnz / ((long long)H.long_len + 1) + 1);
    const long long singles = std::min<long long>(m, nnz / ((long long)H.mid_len + 1) + 1);
    const long long parts = 2 * (nnz / H.seg_len) + 2;
    H.max_mid = (int)std::min<long long>(mids, 0x7fffffffLL);
    H.max_singles = (int)std::min<long long>(singles, 0x7fffffffLL);
    H.max_parts = (int)std::min<long long>(parts, 0x7fffffffLL);
    size_t off = 0;
    H.off_counts = off;
    off = align256(off + 5 * sizeof(int));
    H.off_mid = off;
    off = align256(off + (size_t)H.max_mid * sizeof(int));
    H.off_single = off;
    off = align256(off + (size_t)H.max_singles * sizeof(int));
    H.off_multi = off;
    off = align256(off + (size_t)H.max_parts * sizeof(int2));
    H.off_arrive = off;
    off = align256(off + (size_t)H.max_parts * sizeof(int));
    H.off_partial = off;
    off = align256(off + (size_t)H.max_parts * (size_t)n * sizeof(float));
    H.total = off;
    return H;
}

// Lanes per row of the SpMV row split: the power of two at or below a sixth
// of the mean row length, at most 8 (measured on GB300 over mean lengths 2 to
// 1000: fewer lanes per row, so more rows per warp, keep more independent
// gathers in flight than one lane per nonzero does).
int spmv_lanes(int m, long long nnz) {
    const double d = m > 0 ? (double)nnz / m : 0.0;
    int g = 1;
    while (g < 8 && 12.0 * g <= d) g <<= 1;
    return g;
}

// Items per thread of the SpMV merge kernel: 4, 8 (default) or 16, the
// largest not above the requested items_per_subwarp.
int spmv_items(const spmm_tuning_t* t) {
    const int r = (t && t->items_per_subwarp > 0) ? t->items_per_subwarp : kSpmvItems;
    return r >= 16 ? 16 : r >= 8 ? 8 : 4;
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}

// Shrink the merge tile until the double-buffered staging fits one CTA's
// shared memory (sv = bytes per value; the float32 bound covers 16-bit vals).
void clamp_tile(Shape* s, int sv) {
    auto bytes = [&](const Shape& t) -> size_t {
        if (sv == 4) return t.vec == 1 ? merge_smem_vec<float, 1>(t) : t.vec == 4 ? merge_smem_vec<float, 4>(t) : merge_smem_vec<float, 8>(t);
        return t.vec == 1 ? merge_smem_vec<__half, 1>(t) : t.vec == 4 ? merge_smem_vec<__half, 4>(t) : merge_smem_vec<__half, 8>(t);
    };
    while (s->ips > 4 && bytes(*s) > kMaxSmem) s->ips = s->ips * 3 / 4;
}

// Stream-ordered allocations of this library come from the device's default
// memory pool.  Its default release threshold (0) hands freed memory back to
// the CUDA driver at every synchronisation, which makes each call pay the full
// mapping cost again; keep it cached instead (once per device, for this
// process only).
void keep_pool_memory() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        unsigned long long thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    done[dev] = true;
}

// Staging memory of the host-buffer entries: a pool of their own per device,
// created once.  A call's buffer is allocated on the upload stream and freed
// on the download stream; the pool may reuse it for a later call once the
// free has completed, but never by making the later call's uploads wait on
// the earlier call's downloads (the default pool may insert such a wait),
// which would serialise back-to-back asynchronous calls.  Freed memory stays
// cached until exit.
cudaMemPool_t host_staging_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) return nullptr;
        unsigned long long thr = ~0ull;
        int no = 0;
        if (cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &thr) != cudaSuccess ||
            cudaMemPoolSetAttribute(p, cudaMemPoolReuseAllowInternalDependencies, &no) != cudaSuccess) {
            cudaMemPoolDestroy(p);
            return nullptr;
        }
        pools[dev] = p;
    }
    return pools[dev];
}

// Two copy streams per device (host-to-device, device-to-host), created once.
bool copy_streams(cudaStream_t* up, cudaStream_t* down) {
    static std::mutex mu;
    static cudaStream_t streams[64][2] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return false;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < 2; ++i)
        if (!streams[dev][i] && cudaStreamCreateWithFlags(&streams[dev][i], cudaStreamNonBlocking) != cudaSuccess)
            return false;
    *up = streams[dev][0];
    *down = streams[dev][1];
    return true;
}

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return SPMM_OK;
    if (e == cudaErrorMemoryAllocation) return SPMM_ERR_ALLOC;
    if (e == cudaErrorInvalidConfiguration || e == cudaErrorLaunchOutOfResources || e == cudaErrorInvalidValue)
        return SPMM_ERR_LAUNCH;
    return SPMM_ERR_CUDA;
}

// Checks of everything a host can see.  Returns SPMM_OK or an error status.
int check_args(int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind, const void* vals,
               const void* B, long long ldb, const void* C, long long ldc, int alg) {
    if (m < 0 || k < 0 || n < 0 || nnz < -1 || nnz > 0x7fffffffLL) return SPMM_ERR_INVALID_VALUE;
    if (alg < SPMM_ALG_AUTO || alg > SPMM_ALG_ROW_SPLIT_HYBRID) return SPMM_ERR_INVALID_VALUE;
    if (m > 0 && n > 0) {
        if (!row_ptr || !C) return SPMM_ERR_INVALID_VALUE;
        if (ldc < n) return SPMM_ERR_INVALID_VALUE;
        if (nnz != 0 && (!col_ind || !vals)) return SPMM_ERR_INVALID_VALUE;
        if (nnz != 0 && k > 0 && (!B || ldb < n)) return SPMM_ERR_INVALID_VALUE;
        if (nnz > 0 && k == 0) return SPMM_ERR_INVALID_VALUE;  // a nonzero needs a column
    }
    return SPMM_OK;
}

// Longest row of A and, when nnz is not NULL, nnz = row_ptr[m], in one launch
// and one synchronisation of st.  The two result words live in a device
// buffer per host thread and device, allocated on first use and kept until
// exit; the call synchronises st before it returns, so no two calls have the
// same words in flight.
int probe_rows(const int* row_ptr, int m, cudaStream_t st, long long* lmax, long long* nnz) {
    static thread_local int* words[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SPMM_ERR_CUDA;
    if (!words[dev] && cudaMalloc(&words[dev], 2 * sizeof(int)) != cudaSuccess) {
        words[dev] = nullptr;
        return SPMM_ERR_ALLOC;
    }
    int* d = words[dev];
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(int), st);
    const int threads = 256;
    const int blocks = (int)std::max<long long>(1, std::min<long long>(((long long)m + threads - 1) / threads, 4 * 152));
    if (e == cudaSuccess) {
        row_length_max_kernel<<<blocks, threads, 0, st>>>(row_ptr, m, d);
        e = cudaGetLastError();
        if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    }
    int h[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (h[1] < 0) return SPMM_ERR_BAD_CSR;
    *lmax = h[0];
    if (nnz) *nnz = h[1];
    return SPMM_OK;
}

int read_nnz(const int* row_ptr, int m, cudaStream_t st, long long* nnz) {
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, row_ptr + m, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (v < 0) return SPMM_ERR_BAD_CSR;
    *nnz = v;
    return SPMM_OK;
}

}  // namespace

// The body of every C = A (x) B entry point (spmm_csr_ex, spmm_csr_semiring):
// argument checks, algorithm choice, launch shape, then row split, SpMV, A/B
// tiling or partition + merge + fix-up with the given launcher table.
int run_spmm(const Launchers* L, int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind,
             const void* vals, int vals_type, const void* B, int b_type, long long ldb, void* C, int c_type,
             long long ldc, int alg, const spmm_tuning_t* tuning, void* workspace, size_t workspace_bytes,
             int* d_status, void* stream) {
    int st = check_args(m, k, n, nnz, row_ptr, col_ind, vals, B, ldb, C, ldc, alg);
    if (st != SPMM_OK) return st;
    if (ldb * (long long)dtype_size(b_type) > 0xffffffffLL) return SPMM_ERR_INVALID_VALUE;  // rows of B < 4 GiB apart
    if (!L) return SPMM_ERR_UNSUPPORTED;
    if (m == 0 || n == 0) return SPMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    long long lmax = tuning ? tuning->max_row_len : 0;
    if (alg == SPMM_ALG_AUTO_GB300 && lmax <= 0) {  // longest row (and nnz if unknown): one synchronisation
        st = probe_rows(row_ptr, m, s, &lmax, nnz < 0 ? &nnz : nullptr);
        if (st != SPMM_OK) return st;
    } else if (nnz < 0) {
        st = read_nnz(row_ptr, m, s, &nnz);
        if (st != SPMM_OK) return st;
    }
    Shape shape;
    if (alg == SPMM_ALG_AUTO_GB300) alg = spmm_select_alg_gb300(m, nnz, lmax, n, b_type);
    const int a = resolve_alg(alg, m, nnz, tuning);
    spmm_tuning_t t_eff = tuning ? *tuning : spmm_tuning_t{};
    if (t_eff.column_slabs <= 0 && t_eff.lanes_per_row <= 0) t_eff.column_slabs = default_slabs(a, k, n, b_type);
    if (!choose_shape(n, b_type, c_type, B, ldb, C, ldc, &t_eff, &shape)) return SPMM_ERR_INVALID_VALUE;
    if (a == SPMM_ALG_ROW_SPLIT_HYBRID && hybrid_two_vectors(n, b_type, ldb, ldc, shape) && !shape_for(n, 8, &t_eff, &shape))
        return SPMM_ERR_INVALID_VALUE;
    const bool spmv = n == 1;  // y = A x: the SpMV forms of both families
    if (a == SPMM_ALG_TILED && shape.vec > 1 && !spmv) {
        TiledArgs ta{m, n, k, row_ptr, col_ind, vals, B, ldb, C, ldc, d_status};
        return cuda_status(L->tiled(ta, shape, s));
    }
    if (a == SPMM_ALG_ROW_SPLIT_HYBRID) {
        const HybridLayout H = hybrid_layout(m, nnz, n, shape, t_eff);
        bool own = false;
        unsigned char* ws = static_cast<unsigned char*>(workspace);
        if (!ws) {
            if (workspace_bytes != 0) return SPMM_ERR_WORKSPACE;
            void* p = nullptr;
            keep_pool_memory();
            if (cudaMallocAsync(&p, H.total, s) != cudaSuccess) return SPMM_ERR_ALLOC;
            ws = static_cast<unsigned char*>(p);
            own = true;
        } else if (workspace_bytes < H.total || ((uintptr_t)ws % 256) != 0) {
            return SPMM_ERR_WORKSPACE;
        }
        RowSplitArgs ra{m, n, row_ptr, col_ind, vals, B, ldb, C, ldc};
        LongRowArgs la{};
        la.long_len = H.long_len;
        la.mid_len = H.mid_len;
        la.mid_split = H.mid_split;
        la.seg_len = H.seg_len;
        la.block_rows = H.block_rows;
        la.max_mid = H.max_mid;
        la.max_singles = H.max_singles;
        la.max_parts = H.max_parts;
        la.counts = reinterpret_cast<int*>(ws + H.off_counts);
        la.mid = reinterpret_cast<int*>(ws + H.off_mid);
        la.single = reinterpret_cast<int*>(ws + H.off_single);
        la.multi = reinterpret_cast<int2*>(ws + H.off_multi);
        la.arrive = reinterpret_cast<int*>(ws + H.off_arrive);
        la.partial = reinterpret_cast<float*>(ws + H.off_partial);
        la.status = d_status;
        st = cuda_status(L->rowsplit_hybrid(ra, la, shape, sm_count(), s));
        if (own) {
            const cudaError_t e = cudaFreeAsync(ws, s);
            if (st == SPMM_OK && e != cudaSuccess) st = cuda_status(e);
        }
        return st;
    }
    if (a == SPMM_ALG_ROW_SPLIT || a == SPMM_ALG_TILED) {  // tiling without 16-byte access: row split
        RowSplitArgs ra{m, n, row_ptr, col_ind, vals, B, ldb, C, ldc};
        if (spmv)
            return cuda_status(
                L->spmv_rowsplit(ra, t_eff.lanes_per_row > 0 ? t_eff.lanes_per_row : spmv_lanes(m, nnz), s));
        return cuda_status(L->rowsplit(ra, shape, s));
    }

    // merge based: partition, compute, fix-up.  SpMM tiles are capped so that
    // the double-buffered staging fits the shared memory of one CTA.
    const int spmv_t = spmv_items(&t_eff);
    long long ipt = (long long)kThreads * spmv_t;
    if (!spmv) {
        clamp_tile(&shape, dtype_size(vals_type));
        if (L->merge_smem(shape) > kMaxSmem) return SPMM_ERR_INVALID_VALUE;
        ipt = (long long)(merge_cta_threads(shape.W) / shape.W) * shape.ips;
    }
    const MergeLayout lay = merge_layout_items(m, nnz, n, ipt);
    bool own = false;
    unsigned char* ws = static_cast<unsigned char*>(workspace);
    if (!ws) {
        if (workspace_bytes != 0) return SPMM_ERR_WORKSPACE;
        void* p = nullptr;
        keep_pool_memory();
        const cudaError_t e = cudaMallocAsync(&p, lay.total, s);
        if (e != cudaSuccess) return SPMM_ERR_ALLOC;
        ws = static_cast<unsigned char*>(p);
        own = true;
    } else if (workspace_bytes < lay.total || ((uintptr_t)ws % 256) != 0) {
        return SPMM_ERR_WORKSPACE;
    }
    MergeArgs ma{};
    ma.m = m;
    ma.n = n;
    ma.nnz = nnz;
    ma.row_ptr = row_ptr;
    ma.col_ind = col_ind;
    ma.vals = vals;
    ma.B = B;
    ma.ldb = ldb;
    ma.C = C;
    ma.ldc = ldc;
    ma.limits = reinterpret_cast<const int2*>(ws + lay.off_limits);
    ma.num_tiles = lay.num_tiles;
    ma.slabs = shape.slabs;
    ma.ips = shape.ips;
    ma.carry = reinterpret_cast<float*>(ws + lay.off_carry);
    ma.head = reinterpret_cast<float*>(ws + lay.off_head);
    ma.carry_row = reinterpret_cast<int*>(ws + lay.off_carry_row);
    ma.head_row = reinterpret_cast<int*>(ws + lay.off_head_row);
    ma.status = d_status;
    ma.use_tma = ((uintptr_t)row_ptr % 16 == 0) && ((uintptr_t)col_ind % 16 == 0) && ((uintptr_t)vals % 16 == 0);
    ma.wait_ns = kWaitLimitNs;

    st = spmm_merge_partition(m, nnz, row_ptr, (int)ipt, lay.num_tiles, reinterpret_cast<int*>(ws + lay.off_limits),
                              stream);
    if (st == SPMM_OK) st = cuda_status(spmv ? L->spmv_merge(ma, spmv_t, s) : L->merge(ma, shape, sm_count(), s));
    if (st == SPMM_OK && lay.num_tiles > 1) st = cuda_status(L->fixup(ma, s));
    if (own) {
        const cudaError_t e = cudaFreeAsync(ws, s);
        if (st == SPMM_OK && e != cudaSuccess) st = cuda_status(e);
    }
    return st;
}

}  // namespace spmm

using namespace spmm;

extern "C" {

const char* spmm_status_string(int status) {
    switch (status) {
        case SPMM_OK: return "SPMM_OK";
        case SPMM_ERR_INVALID_VALUE: return "SPMM_ERR_INVALID_VALUE: invalid size, pointer, stride or enum";
        case SPMM_ERR_ALLOC: return "SPMM_ERR_ALLOC: device memory allocation failed";
        case SPMM_ERR_LAUNCH: return "SPMM_ERR_LAUNCH: kernel launch rejected";
        case SPMM_ERR_BAD_CSR: return "SPMM_ERR_BAD_CSR: inconsistent CSR structure";
        case SPMM_ERR_TIMEOUT: return "SPMM_ERR_TIMEOUT: a bounded device-side wait ran out";
        case SPMM_ERR_UNSUPPORTED: return "SPMM_ERR_UNSUPPORTED: dtype combination not provided";
        case SPMM_ERR_CUDA: return "SPMM_ERR_CUDA: CUDA runtime error";
        case SPMM_ERR_WORKSPACE: return "SPMM_ERR_WORKSPACE: workspace missing or too small";
        default: return "unknown status";
    }
}

int spmm_version(void) { return 101; }

long long spmm_launch_count(void) { return g_launches.load(); }

int spmm_select_alg(int m, long long nnz, double threshold) {
    if (m <= 0) return SPMM_ALG_ROW_SPLIT;
    if (threshold <= 0.0) threshold = kPaperThreshold;
    const double d = (double)nnz / (double)m;  // mean row length (Section 5.4)
    return d < threshold ? SPMM_ALG_MERGE : SPMM_ALG_ROW_SPLIT;
}

int spmm_select_alg_gb300(int m, long long nnz, long long max_row_len, int n, int b_type) {
    if (m <= 0) return SPMM_ALG_ROW_SPLIT;
    const long long row_bytes = (long long)n * (dtype_size(b_type) ? dtype_size(b_type) : 4);
    const double d = (double)nnz / (double)m;
    const bool uneven = (double)max_row_len >= 2.0 * d;
    // Type 1 guard: the hybrid when most rows are short beside the long ones (the longest at least
    // 16 times the mean) and rows of B are at most 128 bytes, else merge (rows all long: merge's
    // equal tiles beat the hybrid's warp segments)
    if (max_row_len > 1024 && max_row_len * 8192 >= nnz)
        return (row_bytes <= 128 && (double)max_row_len >= 16.0 * d) ? SPMM_ALG_ROW_SPLIT_HYBRID : SPMM_ALG_MERGE;
    // rows of 768 or more nonzeros with rows of B under 256 bytes: a lane group of the row split
    // waits on its row, merge spreads it over tiles
    if (row_bytes < 256 && d >= 768.0) return SPMM_ALG_MERGE;
    if (row_bytes < 64) return SPMM_ALG_ROW_SPLIT;
    // mean-length rules measured on GB300 (uniform and Poisson rows, 1M x 1M, float32): below 3
    // nonzeros per row the hybrid's packed runs of short rows win (merge for uneven rows of 512-byte
    // rows of B); from 3 on the row split wins for rows of B under 256 bytes, and for wider rows
    // merge wins below 3 (256 bytes) or 5 (512 bytes and more), or below 8 when the longest row is at
    // least twice the mean (uneven rows cost the row split more than the merge path)
    if (d < 3.0) return (row_bytes >= 512 && uneven) ? SPMM_ALG_MERGE : SPMM_ALG_ROW_SPLIT_HYBRID;
    if (row_bytes < 256) return SPMM_ALG_ROW_SPLIT;
    const double threshold = uneven ? 8.0 : (row_bytes >= 512 ? 5.0 : 3.0);
    return d < threshold ? SPMM_ALG_MERGE : SPMM_ALG_ROW_SPLIT;
}

double spmm_tiled_reuse(int m, int k, long long nnz, int n, int b_type) {
    if (m <= 0 || k <= 0 || n <= 0 || nnz <= 0 || dtype_size(b_type) == 0) return 0.0;
    const long long chunks = ((long long)n + 16 / dtype_size(b_type) - 1) / (16 / dtype_size(b_type));
    const int W = pow2_ceil(chunks);  // at most 32: wider B takes column slabs
    const double rows_per_block = (double)(kThreads / W) * kTiledRows;
    return rows_per_block * (double)nnz / ((double)m * (double)k);
}

int spmm_default_column_slabs(int alg, int k, int n, int b_type) {
    if (k < 0 || n < 0 || dtype_size(b_type) == 0) return 1;
    return spmm::default_slabs(alg, k, n, b_type);
}

int spmm_csr_max_row_length(int m, const int* row_ptr, long long* max_row_len, void* stream) {
    if (m < 0 || !max_row_len || (m > 0 && !row_ptr)) return SPMM_ERR_INVALID_VALUE;
    *max_row_len = 0;
    if (m == 0) return SPMM_OK;
    return probe_rows(row_ptr, m, (cudaStream_t)stream, max_row_len, nullptr);
}

size_t spmm_csr_workspace_size(int m, int k, int n, long long nnz, int alg, int b_type, const spmm_tuning_t* tuning) {
    if (m < 0 || k < 0 || n < 0 || nnz < 0 || dtype_size(b_type) == 0) return 0;
    if (alg == SPMM_ALG_AUTO_GB300)  // the choice may need the longest row: size for merge and the hybrid
        return std::max(spmm_csr_workspace_size(m, k, n, nnz, SPMM_ALG_MERGE, b_type, tuning),
                        spmm_csr_workspace_size(m, k, n, nnz, SPMM_ALG_ROW_SPLIT_HYBRID, b_type, tuning));
    if (alg == SPMM_ALG_TILED) return 0;
    if (alg == SPMM_ALG_ROW_SPLIT_HYBRID) {
        if (m == 0 || n == 0) return 0;
        size_t best = 0;
        for (int vec : {1, 16 / dtype_size(b_type), 8}) {
            for (int slabs : {0, 2}) {
                spmm_tuning_t t = tuning ? *tuning : spmm_tuning_t{};
                if (slabs && (t.column_slabs > 0 || t.lanes_per_row > 0)) continue;
                if (slabs) t.column_slabs = slabs;
                Shape s;
                if (!shape_for(n, vec, &t, &s)) return 0;
                best = std::max(best, hybrid_layout(m, nnz, n, s, t).total);
            }
        }
        return best;
    }
    if (resolve_alg(alg, m, nnz, tuning) != SPMM_ALG_MERGE || m == 0 || n == 0) return 0;
    // the access width depends on pointer alignment and the default slab count on the device's L2,
    // neither known here: size for every combination
    size_t best = 0;
    for (int vec : {1, 16 / dtype_size(b_type)}) {
        for (int slabs : {0, 2}) {
            spmm_tuning_t t = tuning ? *tuning : spmm_tuning_t{};
            if (slabs && (t.column_slabs > 0 || t.lanes_per_row > 0)) continue;
            if (slabs) t.column_slabs = slabs;
            Shape s;
            if (!shape_for(n, vec, &t, &s)) return 0;
            clamp_tile(&s, 4);
            const size_t need = merge_layout(m, nnz, n, s).total;
            if (need > best) best = need;
        }
    }
    if (n == 1) {  // the SpMV form's tiles
        const size_t need = merge_layout_items(m, nnz, n, (long long)kThreads * spmv_items(tuning)).total;
        if (need > best) best = need;
    }
    return best;
}

int spmm_merge_partition(int m, long long nnz, const int* row_ptr, int items_per_tile, int num_tiles, int* limits,
                         void* stream) {
    if (m < 0 || nnz < 0 || items_per_tile <= 0 || num_tiles < 0 || !limits || (m > 0 && !row_ptr))
        return SPMM_ERR_INVALID_VALUE;
    if ((long long)num_tiles * items_per_tile < (long long)m + nnz) return SPMM_ERR_INVALID_VALUE;
    const int threads = 256;  // 8 boundaries per block, one warp each
    const long long blocks = ((long long)num_tiles + 1 + 7) / 8;
    merge_partition_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        row_ptr, m, nnz, items_per_tile, num_tiles, reinterpret_cast<int2*>(limits));
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_status(e);
}

int spmm_csr_ex(int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind, const void* vals,
                int vals_type, const void* B, int b_type, long long ldb, void* C, int c_type, long long ldc, int alg,
                const spmm_tuning_t* tuning, void* workspace, size_t workspace_bytes, int* d_status, void* stream) {
    return spmm::run_spmm(find_launchers(vals_type, b_type, c_type), m, k, n, nnz, row_ptr, col_ind, vals, vals_type,
                          B, b_type, ldb, C, c_type, ldc, alg, tuning, workspace, workspace_bytes, d_status, stream);
}

int spmm_csr_semiring(int m, int k, int n, long long nnz, const int* row_ptr, const int* col_ind, const float* vals,
                      const float* B, long long ldb, float* C, long long ldc, int semiring, int alg,
                      const spmm_tuning_t* tuning, void* workspace, size_t workspace_bytes, int* d_status,
                      void* stream) {
    if (semiring < SPMM_SEMIRING_PLUS_TIMES || semiring > SPMM_SEMIRING_MAX_TIMES) return SPMM_ERR_INVALID_VALUE;
    const Launchers* L = semiring == SPMM_SEMIRING_PLUS_TIMES ? find_launchers(SPMM_F32, SPMM_F32, SPMM_F32)
                                                              : spmm::find_semiring_launchers(semiring);
    return spmm::run_spmm(L, m, k, n, nnz, row_ptr, col_ind, vals, SPMM_F32, B, SPMM_F32, ldb, C, SPMM_F32, ldc, alg,
                          tuning, workspace, workspace_bytes, d_status, stream);
}


int spmm_csr(int m, int k, int n, const int* row_ptr, const int* col_ind, const float* vals, const float* B,
             long long ldb, float* C, long long ldc, int alg, void* stream) {
    return spmm_csr_ex(m, k, n, -1, row_ptr, col_ind, vals, SPMM_F32, B, SPMM_F32, ldb, C, SPMM_F32, ldc, alg,
                       nullptr, nullptr, 0, nullptr, stream);
}

// The host-buffer products C_i = A B_i (i < count), enqueued on `stream` and the two copy streams:
// A goes up once for all of them.  With `wait` the call returns only when every C_i is in host
// memory.
static int host_products(int m, int k, const int* row_ptr, const int* col_ind, const void* vals, int vals_type,
                         int count, const int* n_of, const void* const* B_of, int b_type, const long long* ldb_of,
                         void* const* C_of, int c_type, const long long* ldc_of, int alg_req,
                         const spmm_tuning_t* tuning, void* stream, bool wait) {
    if (m < 0 || k < 0 || count < 0) return SPMM_ERR_INVALID_VALUE;
    if (count > 0 && (!n_of || !B_of || !ldb_of || !C_of || !ldc_of)) return SPMM_ERR_INVALID_VALUE;
    if (m > 0 && !row_ptr) return SPMM_ERR_INVALID_VALUE;
    if (count == 0) return SPMM_OK;  // no products: the types name nothing
    const long long nnz = m > 0 ? row_ptr[m] : 0;
    for (int i = 0; i < count; ++i) {
        const int st = check_args(m, k, n_of[i], nnz, row_ptr, col_ind, vals, B_of[i], ldb_of[i], C_of[i], ldc_of[i],
                                  alg_req);
        if (st != SPMM_OK) return st;
    }
    const int sv = dtype_size(vals_type), sb = dtype_size(b_type), sc = dtype_size(c_type);
    if (!find_launchers(vals_type, b_type, c_type)) return SPMM_ERR_UNSUPPORTED;
    std::vector<int> prods;  // the products with work to do
    for (int i = 0; i < count; ++i)
        if (n_of[i] > 0) prods.push_back(i);
    if (m == 0 || prods.empty()) return SPMM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    keep_pool_memory();
    cudaStream_t up = nullptr, down = nullptr;
    if (!copy_streams(&up, &down)) return SPMM_ERR_CUDA;

    // The algorithm is chosen once per product, for the whole matrix (the longest row once for all).
    spmm_tuning_t t = tuning ? *tuning : spmm_tuning_t{};
    if (alg_req == SPMM_ALG_AUTO_GB300 && t.max_row_len <= 0)
        for (int i = 0; i < m; ++i) t.max_row_len = std::max<long long>(t.max_row_len, row_ptr[i + 1] - row_ptr[i]);

    // Pipeline over the full-duplex host link.  Column slabs of each B_i and C_i (at least 128
    // bytes of a row each) let slab j be computed while slab j+1 of B goes up and slab j-1 of C
    // comes down; row chunks of A (equal shares of rows + nonzeros) let the first slab start as
    // soon as the first chunk of A is on the device instead of all of A.  Order on the upload
    // stream, products in the caller's order: B_0 slab 0, A chunk 0 .. R-1, the other slabs of
    // B_0, then B_1, B_2, ... in turn (putting the widest product first, measured on the power-law
    // step of n = 8, 32, 64, 128, delays the first compute behind a large B slab: 7.39 -> 7.58 ms).
    const long long vb = 16 / sb, vc = 16 / sc;
    struct Prod {
        int n, alg, slabs;
        long long w, ldb_d, ldc_d;
        size_t off_B, off_C;
    };
    std::vector<Prod> P(prods.size());
    for (size_t q = 0; q < prods.size(); ++q) {
        Prod& p = P[q];
        p.n = n_of[prods[q]];
        p.alg = alg_req == SPMM_ALG_AUTO_GB300 ? spmm_select_alg_gb300(m, nnz, t.max_row_len, p.n, b_type) : alg_req;
        p.alg = resolve_alg(p.alg, m, nnz, &t);
        p.ldb_d = (p.n + vb - 1) / vb * vb;
        p.ldc_d = (p.n + vc - 1) / vc * vc;
        int slabs = (int)std::min<long long>(4, std::max<long long>(1, (long long)p.n * sb / 128));
        long long w = (p.n + slabs - 1) / slabs;
        p.w = (w + 15) / 16 * 16;  // whole 16-byte vectors for every element size
        p.slabs = (int)((p.n + p.w - 1) / p.w);
    }
    const long long a_bytes = (long long)(m + 1) * 4 + nnz * (4 + sv);
    const int chunks = (int)std::max<long long>(1, std::min<long long>({4, m, a_bytes / (8LL << 20)}));
    std::vector<int> r(chunks + 1);  // chunk c holds rows [r[c], r[c+1])
    r[0] = 0;
    r[chunks] = m;
    for (int c = 1; c < chunks; ++c) {  // equal shares of the merge path (rows + nonzeros)
        const long long target = ((long long)m + nnz) * c / chunks;
        int lo = r[c - 1], hi = m;
        while (lo < hi) {
            const int mid = lo + (hi - lo) / 2;
            if ((long long)mid + row_ptr[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        r[c] = lo;
    }
    // Each chunk's row_ptr (rebased to 0), col_ind and vals start on a 256-byte boundary, so the
    // merge kernel keeps its bulk-copy staging.
    std::vector<size_t> off_rp(chunks), off_col(chunks), off_val(chunks);
    size_t total = 0;
    for (int c = 0; c < chunks; ++c) {
        const long long cnnz = row_ptr[r[c + 1]] - row_ptr[r[c]];
        off_rp[c] = total;
        total += align256((size_t)(r[c + 1] - r[c] + 1) * 4);
        off_col[c] = total;
        total += align256((size_t)cnnz * 4);
        off_val[c] = total;
        total += align256((size_t)cnnz * sv);
    }
    // one workspace, lent to every block's call in turn (they run in order on `stream`)
    size_t ws_need = 0;
    for (Prod& p : P) {
        if (p.alg == SPMM_ALG_MERGE || p.alg == SPMM_ALG_ROW_SPLIT_HYBRID)
            for (int c = 0; c < chunks; ++c)
                for (int j = 0; j < p.slabs; ++j) {
                    const long long cw = std::min<long long>(p.w, p.n - j * p.w);
                    ws_need = std::max(ws_need, spmm_csr_workspace_size(r[c + 1] - r[c], k, (int)cw,
                                                                        row_ptr[r[c + 1]] - row_ptr[r[c]], p.alg,
                                                                        b_type, &t));
                }
        p.off_B = total;
        total += align256((size_t)k * p.ldb_d * sb);
        p.off_C = total;
        total += align256((size_t)m * p.ldc_d * sc);
    }
    const size_t off_ws = total;
    total = off_ws + align256(ws_need);
    cudaMemPool_t pool = host_staging_pool();
    if (!pool) return SPMM_ERR_CUDA;
    // events: [0] uploads done, [1] compute done, [2] downloads + free done, [3] inputs ready,
    // then A chunk c uploaded, then per product: slab j of B uploaded, block (j, c) of C computed
    std::vector<size_t> ev_b(P.size()), ev_c(P.size());
    size_t nev = 4 + chunks;
    for (size_t q = 0; q < P.size(); ++q) {
        ev_b[q] = nev;
        nev += P[q].slabs;
        ev_c[q] = nev;
        nev += (size_t)P[q].slabs * chunks;
    }
    std::vector<cudaEvent_t> ev(nev, nullptr);
    cudaError_t e = cudaSuccess;
    for (auto& x : ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&x, cudaEventDisableTiming);
    auto destroy_events = [&] {
        for (auto& x : ev)  // an event still pending is released once it completes
            if (x) cudaEventDestroy(x);
    };
    if (e != cudaSuccess) {
        destroy_events();
        return cuda_status(e);
    }
    // The synchronous entry orders its uploads after the work already queued on `stream` (which may
    // write the host inputs); the asynchronous entries read them from call time on, so that their
    // uploads can overlap the previous call's downloads.
    if (wait) {
        e = cudaEventRecord(ev[3], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(up, ev[3], 0);
        if (e != cudaSuccess) {
            destroy_events();
            return cuda_status(e);
        }
    }
    // The buffer is allocated in the upload stream's order, so the uploads need no other wait;
    // compute and downloads reach it only through events recorded after those uploads.
    void* mem = nullptr;
    e = cudaMallocFromPoolAsync(&mem, total, pool, up);
    if (e != cudaSuccess) {
        destroy_events();
        return SPMM_ERR_ALLOC;
    }
    unsigned char* base = static_cast<unsigned char*>(mem);
    cudaEvent_t e_up = ev[0], e_s = ev[1], e_end = ev[2];
    cudaEvent_t* e_a = ev.data() + 4;
    auto upload_b = [&](size_t q, int j) {
        const Prod& p = P[q];
        const void* Bh = B_of[prods[q]];
        const long long ldb = ldb_of[prods[q]];
        const long long c0 = j * p.w, cw = std::min<long long>(p.w, p.n - c0);
        unsigned char* d_B = base + p.off_B;
        cudaError_t x = cudaSuccess;
        if (k > 0 && nnz > 0)
            x = (p.slabs == 1 && ldb == p.ldb_d)
                    ? cudaMemcpyAsync(d_B, Bh, (size_t)k * p.ldb_d * sb, cudaMemcpyHostToDevice, up)
                    : cudaMemcpy2DAsync(d_B + c0 * sb, (size_t)p.ldb_d * sb,
                                        static_cast<const unsigned char*>(Bh) + c0 * sb, (size_t)ldb * sb,
                                        (size_t)cw * sb, (size_t)k, cudaMemcpyHostToDevice, up);
        if (x == cudaSuccess) x = cudaEventRecord(ev[ev_b[q] + j], up);
        return x;
    };
    e = upload_b(0, 0);
    for (int c = 0; c < chunks && e == cudaSuccess; ++c) {
        const long long p0 = row_ptr[r[c]], p1 = row_ptr[r[c + 1]];
        e = cudaMemcpyAsync(base + off_rp[c], row_ptr + r[c], (size_t)(r[c + 1] - r[c] + 1) * 4, cudaMemcpyHostToDevice,
                            up);
        if (e == cudaSuccess && p1 > p0)
            e = cudaMemcpyAsync(base + off_col[c], col_ind + p0, (size_t)(p1 - p0) * 4, cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess && p1 > p0)
            e = cudaMemcpyAsync(base + off_val[c], static_cast<const unsigned char*>(vals) + p0 * sv,
                                (size_t)(p1 - p0) * sv, cudaMemcpyHostToDevice, up);
        if (e == cudaSuccess) e = cudaEventRecord(e_a[c], up);
    }
    for (size_t q = 0; q < P.size() && e == cudaSuccess; ++q)
        for (int j = q == 0 ? 1 : 0; j < P[q].slabs && e == cudaSuccess; ++j) e = upload_b(q, j);
    int st = e == cudaSuccess ? SPMM_OK : cuda_status(e);

    for (size_t q = 0; q < P.size() && st == SPMM_OK; ++q) {
        const Prod& p = P[q];
        unsigned char* d_B = base + p.off_B;
        unsigned char* d_C = base + p.off_C;
        const long long ldc = ldc_of[prods[q]];
        for (int j = 0; j < p.slabs && st == SPMM_OK; ++j) {
            const long long c0 = j * p.w, cw = std::min<long long>(p.w, p.n - c0);
            st = cuda_status(cudaStreamWaitEvent(s, ev[ev_b[q] + j], 0));
            for (int c = 0; c < chunks && st == SPMM_OK; ++c) {
                const int rows = r[c + 1] - r[c];
                const long long p0 = row_ptr[r[c]], cnnz = row_ptr[r[c + 1]] - p0;
                int* rp_c = reinterpret_cast<int*>(base + off_rp[c]);
                if (q == 0 && j == 0) {  // chunk c arrives once: rebase its row offsets to start at 0
                    st = cuda_status(cudaStreamWaitEvent(s, e_a[c], 0));
                    if (st == SPMM_OK && p0 != 0) {
                        rebase_kernel<<<(unsigned)((rows + 1 + 255) / 256), 256, 0, s>>>(rp_c, rows + 1, (int)p0);
                        const cudaError_t x = cudaGetLastError();
                        if (x == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
                        st = cuda_status(x);
                    }
                }
                if (st == SPMM_OK && rows > 0)
                    st = spmm_csr_ex(rows, k, (int)cw, cnnz, rp_c, reinterpret_cast<const int*>(base + off_col[c]),
                                     base + off_val[c], vals_type, d_B + c0 * sb, b_type, p.ldb_d,
                                     d_C + ((size_t)r[c] * p.ldc_d + c0) * sc, c_type, p.ldc_d, p.alg, &t,
                                     ws_need ? base + off_ws : nullptr, ws_need, nullptr, stream);
                cudaEvent_t done = ev[ev_c[q] + (size_t)j * chunks + c];
                if (st == SPMM_OK) st = cuda_status(cudaEventRecord(done, s));
                if (st == SPMM_OK) st = cuda_status(cudaStreamWaitEvent(down, done, 0));
                if (st == SPMM_OK && rows > 0) {
                    unsigned char* hc = static_cast<unsigned char*>(C_of[prods[q]]) + ((size_t)r[c] * ldc + c0) * sc;
                    const unsigned char* dc = d_C + ((size_t)r[c] * p.ldc_d + c0) * sc;
                    st = cuda_status((p.slabs == 1 && ldc == p.ldc_d)
                                         ? cudaMemcpyAsync(hc, dc, (size_t)rows * p.ldc_d * sc, cudaMemcpyDeviceToHost,
                                                           down)
                                         : cudaMemcpy2DAsync(hc, (size_t)ldc * sc, dc, (size_t)p.ldc_d * sc,
                                                             (size_t)cw * sc, (size_t)rows, cudaMemcpyDeviceToHost,
                                                             down));
                }
            }
        }
    }
    // Free the buffer in the download stream's order once every stream that touched it is done
    // with it, then make `stream` wait for that point: work queued on `stream` after this call,
    // and a synchronisation of it, see C in host memory.  Nothing here blocks the host, so the
    // next call's uploads can overlap this call's last downloads.
    bool freed = false;
    cudaError_t f = cudaEventRecord(e_up, up);
    if (f == cudaSuccess) f = cudaEventRecord(e_s, s);
    if (f == cudaSuccess) f = cudaStreamWaitEvent(down, e_up, 0);
    if (f == cudaSuccess) f = cudaStreamWaitEvent(down, e_s, 0);
    if (f == cudaSuccess) freed = (f = cudaFreeAsync(mem, down)) == cudaSuccess;
    if (f == cudaSuccess) f = cudaEventRecord(e_end, down);
    if (f == cudaSuccess) f = cudaStreamWaitEvent(s, e_end, 0);
    if (f != cudaSuccess) {  // the stream order is broken: drain all three streams instead
        cudaStreamSynchronize(up);
        cudaStreamSynchronize(down);
        if (!freed) cudaFreeAsync(mem, s);
        cudaStreamSynchronize(s);
        if (st == SPMM_OK) st = cuda_status(f);
    }
    destroy_events();
    if (wait) {
        e = cudaStreamSynchronize(s);
        if (st == SPMM_OK && e != cudaSuccess) st = cuda_status(e);
    }
    return st;
}

int spmm_csr_host(int m, int k, int n, const int* row_ptr, const int* col_ind, const void* vals, int vals_type,
                  const void* B, int b_type, long long ldb, void* C, int c_type, long long ldc, int alg,
                  const spmm_tuning_t* tuning, void* stream) {
    if (n < 0) return SPMM_ERR_INVALID_VALUE;
    void* Cs[1] = {C};
    return host_products(m, k, row_ptr, col_ind, vals, vals_type, 1, &n, &B, b_type, &ldb, Cs, c_type, &ldc, alg,
                         tuning, stream, true);
}

int spmm_csr_host_async(int m, int k, int n, const int* row_ptr, const int* col_ind, const void* vals, int vals_type,
                        const void* B, int b_type, long long ldb, void* C, int c_type, long long ldc, int alg,
                        const spmm_tuning_t* tuning, void* stream) {
    if (n < 0) return SPMM_ERR_INVALID_VALUE;
    void* Cs[1] = {C};
    return host_products(m, k, row_ptr, col_ind, vals, vals_type, 1, &n, &B, b_type, &ldb, Cs, c_type, &ldc, alg,
                         tuning, stream, false);
}

int spmm_csr_host_multi(int m, int k, const int* row_ptr, const int* col_ind, const void* vals, int vals_type,
                        int count, const int* n, const void* const* B, int b_type, const long long* ldb, void* const* C,
                        int c_type, const long long* ldc, int alg, const spmm_tuning_t* tuning, void* stream) {
    return host_products(m, k, row_ptr, col_ind, vals, vals_type, count, n, B, b_type, ldb, C, c_type, ldc, alg,
                         tuning, stream, false);
}

int spmm_debug_bounded_wait(int* d_status, long long limit_ns, void* stream) {
    if (!d_status) return SPMM_ERR_INVALID_VALUE;
    if (limit_ns < 1000) limit_ns = 1000;
    if (limit_ns > 2000000000LL) limit_ns = 2000000000LL;
    bounded_wait_probe_kernel<<<1, 32, 0, (cudaStream_t)stream>>>(d_status, (unsigned long long)limit_ns);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return cuda_status(e);
}

}  // extern "C"
