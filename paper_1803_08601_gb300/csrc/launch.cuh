// Host-side launchers of the SpMM kernels, one set per (vals, B, C) element
// type combination.  Each combination is instantiated in its own translation
// unit (inst_*.cu) so the library builds in parallel.
#pragma once

#include <algorithm>
#include <atomic>

#include "hybrid.cuh"
#include "kernels.cuh"

namespace spmm {

// Launch shape chosen by the host: vec = elements per lane access (1 or the
// 16-byte width of B's type), W = lanes per row, slabs = column slabs,
// ips = merge-path items per lane group.
struct Shape {
    int vec;
    int W;
    int slabs;
    int ips;
};

extern std::atomic<long long> g_launches;

using RowSplitFn = cudaError_t (*)(const RowSplitArgs&, const Shape&, cudaStream_t);
using MergeFn = cudaError_t (*)(const MergeArgs&, const Shape&, int grid_cap, cudaStream_t);
using MergeSmemFn = size_t (*)(const Shape&);
using FixupFn = cudaError_t (*)(const MergeArgs&, cudaStream_t);
using SpmvRowSplitFn = cudaError_t (*)(const RowSplitArgs&, int lanes, cudaStream_t);
using SpmvMergeFn = cudaError_t (*)(const MergeArgs&, int items_per_thread, cudaStream_t);
using TiledFn = cudaError_t (*)(const TiledArgs&, const Shape&, cudaStream_t);
using RowSplitHybridFn = cudaError_t (*)(const RowSplitArgs&, const LongRowArgs&, const Shape&, int sms, cudaStream_t);

struct Launchers {
    RowSplitFn rowsplit;
    MergeFn merge;
    MergeSmemFn merge_smem;
    FixupFn fixup;
    SpmvRowSplitFn spmv_rowsplit;  // n = 1
    SpmvMergeFn spmv_merge;        // n = 1, tiles of kThreads * items_per_thread items (4, 8 or 16)
    TiledFn tiled;                 // A/B tiling; 16-byte vectors only (shape.vec > 1)
    RowSplitHybridFn rowsplit_hybrid;  // row pass + segment pass of the hybrid row split
};

// defined in inst_*.cu
Launchers launchers_f32_f32_f32();
Launchers launchers_bf16_bf16_bf16();
Launchers launchers_bf16_bf16_f32();
Launchers launchers_bf16_f16_f16();
Launchers launchers_bf16_f16_f32();
Launchers launchers_f16_f16_f16();
Launchers launchers_f16_f16_f32();
// float32 launchers of SPMM_SEMIRING_MIN_PLUS / MAX_PLUS / MAX_TIMES (inst_semiring.cu)
const Launchers* find_semiring_launchers(int semiring);

// ---------------------------------------------------------------------------- templates

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR>
cudaError_t rowsplit_launch_one(const RowSplitArgs& a, const Shape& s, cudaStream_t st) {
    const long long rows_per_cta = kThreads / W;
    const long long gx = (a.m + rows_per_cta - 1) / rows_per_cta;
    if (gx > 0x7fffffffLL || s.slabs > 65535) return cudaErrorInvalidConfiguration;
    rowsplit_kernel<TV, TB, TC, VEC, W, SR><<<dim3((unsigned)gx, (unsigned)s.slabs), kThreads, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, int VEC, typename SR>
cudaError_t rowsplit_launch_vec(const RowSplitArgs& a, const Shape& s, cudaStream_t st) {
    switch (s.W) {
        case 1: return rowsplit_launch_one<TV, TB, TC, VEC, 1, SR>(a, s, st);
        case 2: return rowsplit_launch_one<TV, TB, TC, VEC, 2, SR>(a, s, st);
        case 4: return rowsplit_launch_one<TV, TB, TC, VEC, 4, SR>(a, s, st);
        case 8: return rowsplit_launch_one<TV, TB, TC, VEC, 8, SR>(a, s, st);
        case 16: return rowsplit_launch_one<TV, TB, TC, VEC, 16, SR>(a, s, st);
        case 32: return rowsplit_launch_one<TV, TB, TC, VEC, 32, SR>(a, s, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TV, typename TB, typename TC, typename SR>
cudaError_t rowsplit_launch(const RowSplitArgs& a, const Shape& s, cudaStream_t st) {
    constexpr int V = Elem<TB>::kVec;
    return s.vec == 1 ? rowsplit_launch_vec<TV, TB, TC, 1, SR>(a, s, st) : rowsplit_launch_vec<TV, TB, TC, V, SR>(a, s, st);
}

// Hybrid row split: zero the queue counters, then the row-block pass (a warp
// per block of l.block_rows rows) and the segment pass, a persistent grid of
// one wave chained behind it with programmatic dependent launch.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR>
cudaError_t hybrid_launch_one(const RowSplitArgs& a, const LongRowArgs& l, const Shape& s, int sms, cudaStream_t st) {
    constexpr long long warps_per_cta = kThreads / 32;
    if (l.block_rows < 1 || l.block_rows > kMaxBlockRows) return cudaErrorInvalidValue;
    const long long blocks = ((long long)a.m + l.block_rows - 1) / l.block_rows;
    const long long gx = (blocks + warps_per_cta - 1) / warps_per_cta;
    if (gx > 0x7fffffffLL || s.slabs > 65535 || s.slabs < 1) return cudaErrorInvalidConfiguration;
    auto seg_kern = rowsplit_segment_kernel<TV, TB, TC, VEC, W, SR>;
    static thread_local int cached_dev = -1;
    static thread_local int cached_blocks = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != cached_dev) {
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, seg_kern, kThreads, 0);
        if (e != cudaSuccess) return e;
        cached_dev = dev;
        cached_blocks = nb < 1 ? 1 : nb;
    }
    e = cudaMemsetAsync(l.counts, 0, 5 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    rowsplit_block_kernel<TV, TB, TC, VEC, W, SR><<<dim3((unsigned)gx, (unsigned)s.slabs), kThreads, 0, st>>>(a, l);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    g_launches.fetch_add(1, std::memory_order_relaxed);
    const long long max_items = (long long)l.max_singles + l.max_parts + (l.max_mid + 32 / W - 1) / (32 / W) + 1;
    long long sx = (long long)cached_blocks * std::max(sms, 1);
    sx = std::min<long long>(sx, (max_items * s.slabs + warps_per_cta - 1) / warps_per_cta);
    if (sx < 1) sx = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)sx);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, seg_kern, a, l, s.slabs);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, int VEC, typename SR>
cudaError_t hybrid_launch_vec(const RowSplitArgs& a, const LongRowArgs& l, const Shape& s, int sms, cudaStream_t st) {
    switch (s.W) {
        case 1: return hybrid_launch_one<TV, TB, TC, VEC, 1, SR>(a, l, s, sms, st);
        case 2: return hybrid_launch_one<TV, TB, TC, VEC, 2, SR>(a, l, s, sms, st);
        case 4: return hybrid_launch_one<TV, TB, TC, VEC, 4, SR>(a, l, s, sms, st);
        case 8: return hybrid_launch_one<TV, TB, TC, VEC, 8, SR>(a, l, s, sms, st);
        case 16: return hybrid_launch_one<TV, TB, TC, VEC, 16, SR>(a, l, s, sms, st);
        case 32: return hybrid_launch_one<TV, TB, TC, VEC, 32, SR>(a, l, s, sms, st);
        default: return cudaErrorInvalidValue;
    }
}

// vec: 1, the 16-byte width of TB, or for float32 B also 8 (two 16-byte
// vectors per lane).
template <typename TV, typename TB, typename TC, typename SR>
cudaError_t hybrid_launch(const RowSplitArgs& a, const LongRowArgs& l, const Shape& s, int sms, cudaStream_t st) {
    constexpr int V = Elem<TB>::kVec;
    if (s.vec == 1) return hybrid_launch_vec<TV, TB, TC, 1, SR>(a, l, s, sms, st);
    if constexpr (sizeof(TB) == 4) {
        if (s.vec == 8) return hybrid_launch_vec<TV, TB, TC, 8, SR>(a, l, s, sms, st);
    }
    return hybrid_launch_vec<TV, TB, TC, V, SR>(a, l, s, sms, st);
}

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR>
cudaError_t merge_launch_one(const MergeArgs& a, const Shape& s, int grid_cap, cudaStream_t st) {
    constexpr int NT = merge_cta_threads(W);
    using L = MergeSmem<TV, VEC, W, NT>;
    auto kern = [] {
        if constexpr (NT == 256) return merge_kernel_wide<TV, TB, TC, VEC, W, SR>;
        else return merge_kernel_narrow<TV, TB, TC, VEC, W, SR>;
    }();
    static_assert(NT == 128 || NT == 256, "merge CTA shapes");
    const size_t smem = L::total(s.ips);
    // per-instantiation cache of the opt-in shared-memory size and occupancy
    static thread_local int cached_dev = -1;
    static thread_local size_t cached_smem = 0;
    static thread_local int cached_blocks = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != cached_dev || smem != cached_smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int blocks = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, NT, smem);
        if (e != cudaSuccess) return e;
        cached_dev = dev;
        cached_smem = smem;
        cached_blocks = blocks < 1 ? 1 : blocks;
    }
    const long long items = (long long)a.num_tiles * a.slabs;
    long long grid = (long long)cached_blocks * grid_cap;
    if (grid > items) grid = items;
    if (grid < 1) return cudaSuccess;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;  // overlap the partition's tail
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, int VEC, typename SR>
cudaError_t merge_launch_vec(const MergeArgs& a, const Shape& s, int grid_cap, cudaStream_t st) {
    switch (s.W) {
        case 1: return merge_launch_one<TV, TB, TC, VEC, 1, SR>(a, s, grid_cap, st);
        case 2: return merge_launch_one<TV, TB, TC, VEC, 2, SR>(a, s, grid_cap, st);
        case 4: return merge_launch_one<TV, TB, TC, VEC, 4, SR>(a, s, grid_cap, st);
        case 8: return merge_launch_one<TV, TB, TC, VEC, 8, SR>(a, s, grid_cap, st);
        case 16: return merge_launch_one<TV, TB, TC, VEC, 16, SR>(a, s, grid_cap, st);
        case 32: return merge_launch_one<TV, TB, TC, VEC, 32, SR>(a, s, grid_cap, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TV, typename TB, typename TC, typename SR>
cudaError_t merge_launch(const MergeArgs& a, const Shape& s, int grid_cap, cudaStream_t st) {
    constexpr int V = Elem<TB>::kVec;
    return s.vec == 1 ? merge_launch_vec<TV, TB, TC, 1, SR>(a, s, grid_cap, st)
                      : merge_launch_vec<TV, TB, TC, V, SR>(a, s, grid_cap, st);
}

// FIXCARRYOUT launch: a warp per tile (grid-stride), chained behind the merge
// kernel with programmatic dependent launch.
template <typename TC, typename SR>
cudaError_t fixup_launch(const MergeArgs& ma, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)std::min<long long>(((long long)ma.num_tiles + 7) / 8, 152LL * 8));
    cfg.blockDim = dim3(256);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, merge_fixup_kernel<TC, SR>, (const int*)ma.carry_row,
                                       (const int*)ma.head_row, (const float*)ma.carry, (const float*)ma.head,
                                       ma.num_tiles, ma.n, static_cast<TC*>(ma.C), ma.ldc, ma.status);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, int G, typename SR>
cudaError_t spmv_rowsplit_one(const RowSplitArgs& a, cudaStream_t st) {
    const long long rows_per_cta = kThreads / G;
    const long long gx = (a.m + rows_per_cta - 1) / rows_per_cta;
    if (gx > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    spmv_rowsplit_kernel<TV, TB, TC, G, SR><<<(unsigned)gx, kThreads, 0, st>>>(a);
    const cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, typename SR>
cudaError_t spmv_rowsplit_launch(const RowSplitArgs& a, int lanes, cudaStream_t st) {
    switch (lanes) {
        case 1: return spmv_rowsplit_one<TV, TB, TC, 1, SR>(a, st);
        case 2: return spmv_rowsplit_one<TV, TB, TC, 2, SR>(a, st);
        case 4: return spmv_rowsplit_one<TV, TB, TC, 4, SR>(a, st);
        case 8: return spmv_rowsplit_one<TV, TB, TC, 8, SR>(a, st);
        case 16: return spmv_rowsplit_one<TV, TB, TC, 16, SR>(a, st);
        case 32: return spmv_rowsplit_one<TV, TB, TC, 32, SR>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

// One CTA per tile, chained behind the partition with programmatic dependent launch.
template <typename TV, typename TB, typename TC, typename SR>
cudaError_t spmv_merge_launch(const MergeArgs& a, int items_per_thread, cudaStream_t st) {
    if (a.num_tiles < 1) return cudaSuccess;
    void (*kern)(MergeArgs) = nullptr;
    switch (items_per_thread) {
        case 4: kern = spmv_merge_kernel<TV, TB, TC, 4, SR>; break;
        case 8: kern = spmv_merge_kernel<TV, TB, TC, 8, SR>; break;
        case 16: kern = spmv_merge_kernel<TV, TB, TC, 16, SR>; break;
        default: return cudaErrorInvalidValue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)a.num_tiles);
    cfg.blockDim = dim3(kThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, a);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR>
cudaError_t tiled_launch_one(const TiledArgs& a, const Shape& s, cudaStream_t st) {
    using TS = TiledShape<TV, TB, VEC, W>;
    auto kern = tiled_kernel<TV, TB, TC, VEC, W, SR>;
    constexpr int smem = 2 * kTiledPanel;
    static thread_local int configured_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev != configured_dev) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured_dev = dev;
    }
    const long long gx = (a.m + TS::RB - 1) / TS::RB;
    if (gx > 0x7fffffffLL || s.slabs > 65535) return cudaErrorInvalidConfiguration;
    kern<<<dim3((unsigned)gx, (unsigned)s.slabs), kThreads, smem, st>>>(a);
    e = cudaGetLastError();
    if (e == cudaSuccess) g_launches.fetch_add(1, std::memory_order_relaxed);
    return e;
}

template <typename TV, typename TB, typename TC, typename SR>
cudaError_t tiled_launch(const TiledArgs& a, const Shape& s, cudaStream_t st) {
    constexpr int V = Elem<TB>::kVec;
    if (s.vec != V) return cudaErrorInvalidValue;
    switch (s.W) {
        case 1: return tiled_launch_one<TV, TB, TC, V, 1, SR>(a, s, st);
        case 2: return tiled_launch_one<TV, TB, TC, V, 2, SR>(a, s, st);
        case 4: return tiled_launch_one<TV, TB, TC, V, 4, SR>(a, s, st);
        case 8: return tiled_launch_one<TV, TB, TC, V, 8, SR>(a, s, st);
        case 16: return tiled_launch_one<TV, TB, TC, V, 16, SR>(a, s, st);
        case 32: return tiled_launch_one<TV, TB, TC, V, 32, SR>(a, s, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename TV, int VEC>
size_t merge_smem_vec(const Shape& s) {
    switch (s.W) {
        case 1: return MergeSmem<TV, VEC, 1, merge_cta_threads(1)>::total(s.ips);
        case 2: return MergeSmem<TV, VEC, 2, merge_cta_threads(2)>::total(s.ips);
        case 4: return MergeSmem<TV, VEC, 4, merge_cta_threads(4)>::total(s.ips);
        case 8: return MergeSmem<TV, VEC, 8, merge_cta_threads(8)>::total(s.ips);
        case 16: return MergeSmem<TV, VEC, 16, merge_cta_threads(16)>::total(s.ips);
        default: return MergeSmem<TV, VEC, 32, merge_cta_threads(32)>::total(s.ips);
    }
}

template <typename TV, typename TB, typename TC>
size_t merge_smem(const Shape& s) {
    constexpr int V = Elem<TB>::kVec;
    return s.vec == 1 ? merge_smem_vec<TV, 1>(s) : merge_smem_vec<TV, V>(s);
}

template <typename TV, typename TB, typename TC, typename SR = PlusTimes>
Launchers make_launchers() {
    return Launchers{&rowsplit_launch<TV, TB, TC, SR>, &merge_launch<TV, TB, TC, SR>, &merge_smem<TV, TB, TC>,
                     &fixup_launch<TC, SR>, &spmv_rowsplit_launch<TV, TB, TC, SR>, &spmv_merge_launch<TV, TB, TC, SR>,
                     &tiled_launch<TV, TB, TC, SR>, &hybrid_launch<TV, TB, TC, SR>};
}

}  // namespace spmm

#define SPMM_DEFINE_LAUNCHERS(NAME, TV, TB, TC) \
    namespace spmm {                            \
    Launchers NAME() { return make_launchers<TV, TB, TC>(); } \
    }
