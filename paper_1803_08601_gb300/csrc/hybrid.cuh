// Hybrid row split for sm_103a: the row split of Section 4.1 with the
// granularity chosen per row (rows of a warp's block split among its lane
// groups by nonzero count; long rows queued and taken by a lane group or by
// warp segments), the paper's Type 1 / Type 2 imbalance (Section 3.2)
// answered inside the row-split family.
#pragma once

#include <climits>

#include "kernels.cuh"

namespace spmm {

// Queues of the hybrid row split (rowsplit_block_kernel, rowsplit_segment_kernel).
// A row of more than long_len nonzeros leaves the row-block pass.  A row of at
// most mid_len is queued in mid[] and later taken by one lane group: rows of at
// most mid_split nonzeros from the front of mid[], longer ones from its back, so
// that the segment pass can take the longer ones first and put rows of similar
// length in one warp's work item.  A longer row is cut into
// nseg = min(ceil(len / seg_len), kMaxRowSegs) segments of equal length, each
// taken by a whole warp: a row of one segment is queued in single[]; a row of
// several reserves nseg consecutive partial slots, and slot p holds its segment
// p - first in multi[p].
constexpr int kMaxRowSegs = 64;
constexpr int kMaxBlockRows = 256;  // rows per warp of the row-block pass, at most

// Lane groups of 4 or more lanes queue their mid rows in two length classes
// (mid_split); narrower ones keep one class, and their kernels carry no code
// for the second.
template <int W>
__host__ __device__ constexpr bool split_mid_rows() { return W >= 4; }

__host__ __device__ __forceinline__ int long_row_segments(long long len, int seg_len) {
    const long long s = (len + seg_len - 1) / seg_len;
    return (int)(s < kMaxRowSegs ? s : kMaxRowSegs);
}

struct LongRowArgs {
    int long_len;     // rows with more nonzeros than this leave the row-block pass
    int mid_len;      // queued rows of at most this many nonzeros are taken by one lane group
    int seg_len;      // nonzeros per warp segment of a longer row (before the kMaxRowSegs cap)
    int block_rows;   // rows per warp in the row-block pass (1 .. kMaxBlockRows)
    int max_mid;      // capacity of mid[]
    int max_singles;  // capacity of single[]
    int max_parts;    // capacity of multi[], arrive[] and the rows of partial[]
    int* counts;      // [5]: single rows queued, partial slots reserved, segment-pass work items taken,
                      // mid rows queued at the front, at the back (zeroed before the row-block pass)
    int* mid;         // [max_mid]: rows of long_len < len <= mid_split from index 0 up, rows of
                      // mid_split < len <= mid_len from index max_mid - 1 down
    int* single;      // [max_singles]: rows of one warp segment
    int2* multi;      // [max_parts]: (row, first partial slot of the row) of the segment in this slot
    int* arrive;      // [max_parts]: segments of a row finished so far, at the row's first partial slot
    float* partial;   // [max_parts][n]: one partial sum per segment of a row with several segments
    int* status;      // optional device status word
    int mid_split;    // mid rows of at most this many nonzeros fill mid[] from the front, longer from the back
};

// ============================================================================ hybrid row split
//
// Type 1 imbalance (Section 3.2): under the row split a row of L nonzeros
// holds its lane group for L / BS batches, so with power-law row lengths a few
// rows of 10^5 nonzeros set the time of the whole launch; and with a lane
// group per row, the many rows of one to three nonzeros use a small part of a
// batch's gathers and pay a whole chain of dependent loads each.  The hybrid
// chooses the granularity of Section 4.1 by row length, in two passes:
//
// * row-block pass (rowsplit_block_kernel): a warp owns block_rows
//   consecutive rows.  The rows of at most long_len nonzeros are split among
//   the warp's lane groups into runs of consecutive rows with equal numbers of
//   nonzeros (a prefix sum over the block in shared memory and one search per
//   group).  Each group walks its run's nonzeros in full batches, so one batch
//   of gathers serves several short rows, and stores every row as it ends.  No
//   row is split, so no partial sums arise.  Longer rows are queued.
// * segment pass (rowsplit_segment_kernel): a queued row of at most mid_len
//   nonzeros is taken by one lane group; a longer row by one warp per segment
//   of about seg_len nonzeros.  Within a warp batch lane group g owns the
//   nonzeros at positions c * 32 + g * W + (0 .. W-1) of the batch, so the
//   warp reads col_ind / vals in whole 128-byte lines; the lane groups' sums
//   are added by xor shuffles.  A row of one segment is stored by its warp.
//   The segments of a longer row leave their partial sums in global memory;
//   the warp that finishes the row's last segment (counted on the row's
//   arrival counter, after a device-scope fence) adds them in segment order
//   and stores the row, so the result does not depend on which warp finishes
//   last.

// Row-block pass.  The segment pass may be scheduled as soon as every CTA has
// started; it waits for this grid to finish.  Lane groups of up to 8 lanes run
// 4 CTAs per SM at 64 registers, with a few bytes of spills for two-vector
// rows: at 3 CTAs and no spills (72 registers) the pass was 7-15 % slower on
// GB300, since its warps wait on the gathers and more of them keep more in flight.
template <int VEC, int W>
__host__ __device__ constexpr int block_pass_min_blocks() { return W >= 16 ? 3 : 4; }

template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads, block_pass_min_blocks<VEC, W>()) rowsplit_block_kernel(RowSplitArgs a,
                                                                                                   LongRowArgs l) {
    pdl_launch_dependents();
    constexpr int U = gathers_per_batch<TB, VEC>();
    constexpr int CV = (U > W) ? U / W : 1;  // (column, value) pairs per lane per batch
    constexpr int BS = W * CV;               // nonzeros per batch
    constexpr int G = BS / U;                // groups of U gathers per batch
    constexpr int NG = 32 / W;               // lane groups per warp
    constexpr int WPC = kThreads / 32;       // warps per CTA
    __shared__ int s_rp_all[WPC][kMaxBlockRows + 1];  // row_ptr of the warp's block
    __shared__ int s_w_all[WPC][kMaxBlockRows + 1];   // exclusive prefix of the short rows' lengths
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sl = lane & (W - 1), grp = lane / W;
    const long long r0 = ((long long)blockIdx.x * WPC + warp) * l.block_rows;
    if (r0 >= a.m) return;  // whole warp
    const int nr = (int)min((long long)l.block_rows, (long long)a.m - r0);
    int* s_rp = s_rp_all[warp];
    int* s_w = s_w_all[warp];
    for (int i = lane; i <= nr; i += 32) s_rp[i] = __ldg(a.row_ptr + r0 + i);
    __syncwarp();

    // each lane takes a run of the block's rows: weights (length of a short row, else 0) and queue counts
    constexpr bool kSplit = split_mid_rows<W>();
    const int rpl = (nr + 31) / 32;
    const int i0 = min(lane * rpl, nr), i1 = min(i0 + rpl, nr);
    int wsum = 0, nmid = 0, nmid2 = 0, nsingle = 0, nparts = 0;
    for (int i = i0; i < i1; ++i) {
        const int len = s_rp[i + 1] - s_rp[i];
        if (len <= l.long_len) {
            wsum += len;
        } else if (len <= l.mid_len) {
            if constexpr (kSplit) {
                if (len <= l.mid_split) ++nmid;
                else ++nmid2;
            } else {
                ++nmid;
            }
        } else {
            const int ns = long_row_segments(len, l.seg_len);
            if (ns == 1) ++nsingle;
            else nparts += ns;
        }
    }
    int incl = wsum;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(kFullMask, incl, off);
        if (lane >= off) incl += y;
    }
    {
        int run = incl - wsum;
        for (int i = i0; i < i1; ++i) {
            s_w[i] = run;
            const int len = s_rp[i + 1] - s_rp[i];
            if (len <= l.long_len) run += len;
        }
        if (lane == 31) s_w[nr] = incl;
    }
    // queue the longer rows (the slab-0 CTA only): one reservation per queue per warp.  The one-class
    // form is kept verbatim for narrow lane groups: their kernels ran up to 15 % slower on long rows
    // when compiled from the two-class source, even with the second class folded away.
    if constexpr (kSplit) {
        if (blockIdx.y == 0 && __any_sync(kFullMask, nmid + nmid2 + nsingle + nparts > 0)) {
            int xm = nmid, xm2 = nmid2, xs = nsingle, xp = nparts;  // inclusive prefixes over the lanes
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int ym = __shfl_up_sync(kFullMask, xm, off);
                const int ys = __shfl_up_sync(kFullMask, xs, off);
                const int yp = __shfl_up_sync(kFullMask, xp, off);
                const int ym2 = __shfl_up_sync(kFullMask, xm2, off);
                if (lane >= off) {
                    xm += ym;
                    xm2 += ym2;
                    xs += ys;
                    xp += yp;
                }
            }
            int bm = 0, bm2 = 0, bs = 0, bp = 0;
            if (lane == 31) {
                if (xm) bm = atomicAdd(l.counts + 3, xm);
                if (xm2) bm2 = atomicAdd(l.counts + 4, xm2);
                if (xs) bs = atomicAdd(l.counts + 0, xs);
                if (xp) bp = atomicAdd(l.counts + 1, xp);
            }
            bm = __shfl_sync(kFullMask, bm, 31) + xm - nmid;
            bm2 = __shfl_sync(kFullMask, bm2, 31) + xm2 - nmid2;
            bs = __shfl_sync(kFullMask, bs, 31) + xs - nsingle;
            bp = __shfl_sync(kFullMask, bp, 31) + xp - nparts;
            for (int i = i0; i < i1; ++i) {
                const int len = s_rp[i + 1] - s_rp[i];
                if (len <= l.long_len) continue;
                const int row = (int)(r0 + i);
                if (len <= l.mid_len) {
                    // the front and the back of mid[] together hold at most max_mid rows for a valid matrix;
                    // the segment pass checks that they did not meet
                    const int slot = len <= l.mid_split ? bm++ : l.max_mid - 1 - bm2++;
                    if (slot >= 0 && slot < l.max_mid) l.mid[slot] = row;
                    else report(l.status, SPMM_ERR_BAD_CSR);  // more nonzeros than the workspace was sized for
                    continue;
                }
                const int ns = long_row_segments(len, l.seg_len);
                if (ns == 1) {
                    if (bs < l.max_singles) l.single[bs] = row;
                    else report(l.status, SPMM_ERR_BAD_CSR);
                    ++bs;
                } else if ((long long)bp + ns <= l.max_parts) {
                    for (int t = 0; t < ns; ++t) l.multi[bp + t] = make_int2(row, bp);
                    l.arrive[bp] = 0;
                    bp += ns;
                } else {
                    // the row is left out; its reserved slots that exist are marked empty for the segment pass
                    for (long long t = bp; t < (long long)bp + ns && t < l.max_parts; ++t) l.multi[t] = make_int2(-1, 0);
                    report(l.status, SPMM_ERR_BAD_CSR);
                    bp += ns;
                }
            }
        }
    } else {
        if (blockIdx.y == 0 && __any_sync(kFullMask, nmid + nsingle + nparts > 0)) {
            int xm = nmid, xs = nsingle, xp = nparts;  // inclusive prefixes over the lanes
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
                const int ym = __shfl_up_sync(kFullMask, xm, off);
                const int ys = __shfl_up_sync(kFullMask, xs, off);
                const int yp = __shfl_up_sync(kFullMask, xp, off);
                if (lane >= off) {
                    xm += ym;
                    xs += ys;
                    xp += yp;
                }
            }
            int bm = 0, bs = 0, bp = 0;
            if (lane == 31) {
                if (xm) bm = atomicAdd(l.counts + 3, xm);
                if (xs) bs = atomicAdd(l.counts + 0, xs);
                if (xp) bp = atomicAdd(l.counts + 1, xp);
            }
            bm = __shfl_sync(kFullMask, bm, 31) + xm - nmid;
            bs = __shfl_sync(kFullMask, bs, 31) + xs - nsingle;
            bp = __shfl_sync(kFullMask, bp, 31) + xp - nparts;
            for (int i = i0; i < i1; ++i) {
                const int len = s_rp[i + 1] - s_rp[i];
                if (len <= l.long_len) continue;
                const int row = (int)(r0 + i);
                if (len <= l.mid_len) {
                    if (bm < l.max_mid) l.mid[bm] = row;
                    else report(l.status, SPMM_ERR_BAD_CSR);  // more nonzeros than the workspace was sized for
                    ++bm;
                    continue;
                }
                const int ns = long_row_segments(len, l.seg_len);
                if (ns == 1) {
                    if (bs < l.max_singles) l.single[bs] = row;
                    else report(l.status, SPMM_ERR_BAD_CSR);
                    ++bs;
                } else if ((long long)bp + ns <= l.max_parts) {
                    for (int t = 0; t < ns; ++t) l.multi[bp + t] = make_int2(row, bp);
                    l.arrive[bp] = 0;
                    bp += ns;
                } else {
                    // the row is left out; its reserved slots that exist are marked empty for the segment pass
                    for (long long t = bp; t < (long long)bp + ns && t < l.max_parts; ++t) l.multi[t] = make_int2(-1, 0);
                    report(l.status, SPMM_ERR_BAD_CSR);
                    bp += ns;
                }
            }
        }
    }
    __syncwarp();

    // this lane group's run: rows [ia, ib) of the block, about 1 / NG of its short nonzeros
    const int total = s_w[nr];
    auto lower = [&](long long t) {  // first row i with s_w[i] >= t
        int lo = 0, hi = nr;
        while (lo < hi) {
            const int md = (lo + hi) >> 1;
            if ((long long)s_w[md] < t) lo = md + 1;
            else hi = md;
        }
        return lo;
    };
    const int ia = grp == 0 ? 0 : lower(((long long)grp * total + NG - 1) / NG);
    const int ib = grp == NG - 1 ? nr : lower(((long long)(grp + 1) * total + NG - 1) / NG);

    // walk the run's nonzeros in batches of BS (a batch may span several rows); a row is stored when
    // the walk passes its end, and the nonzeros of a queued row are skipped
    const long long col0 = (long long)blockIdx.y * (W * VEC) + (long long)sl * VEC;
    const bool col_ok = col0 < a.n;
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const TB* __restrict__ B = static_cast<const TB*>(a.B);
    TC* __restrict__ C = static_cast<TC*>(a.C);
    int row = ia;
    int rend = s_rp[ia < nr ? ia + 1 : nr];
    bool skip = ia < ib && rend - s_rp[ia] > l.long_len;  // the current row is queued
    int p = s_rp[ia];
    const int pe = s_rp[ib];
    float acc[VEC];
#pragma unroll
    for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();
    auto next_row = [&]() {  // the current row ends: store it (unless queued), move to the next
        if (!skip && col_ok) store_vec<TC, VEC>(C + (r0 + row) * a.ldc + col0, acc);
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();
        ++row;
        if (row < ib) {
            const int rs = rend;
            rend = s_rp[row + 1];
            skip = rend - rs > l.long_len;
        }
    };
    for (;;) {
        if (skip && p < rend) p = rend;  // a queued row's nonzeros are not gathered here
        const int cnt = pe - p;          // nonzeros left in the run (may be <= 0)
        if (!__any_sync(kFullMask, cnt > 0)) break;
        int mc[CV];
        float mv[CV];
#pragma unroll
        for (int c = 0; c < CV; ++c) {
            const int q = p + c * W + sl;
            const bool ok = q < pe;
            mc[c] = ok ? __ldg(a.col_ind + q) : 0;
            mv[c] = ok ? load_f(vals + q) : 0.0f;
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
            if (__all_sync(kFullMask, !skip && p + min(cnt, (g + 1) * U) <= rend)) {  // no row ends here
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (g * U + u < cnt) accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = g * U + u;
                    if (j < cnt) {
                        while (p + j >= rend && row < ib) next_row();  // rows (empty or queued too) ending before it
                        if (!skip) accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
                    }
                }
            }
        }
        p += BS;
    }
    while (row < ib) next_row();  // the last row and the empty or queued rows after it
}

// C[row, :] = partial sums of the row's nseg segments added in segment order
// (all n columns, by one warp), rounded once to TC.
template <typename TC, typename SR>
__device__ __forceinline__ void finish_long_row(const float* __restrict__ part, int nseg, int n, TC* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    if ((n & 3) == 0) {  // rows of partial[] are 16-byte aligned
        for (int c = lane * 4; c < n; c += 128) {
            float4 sum = make_float4(SR::identity(), SR::identity(), SR::identity(), SR::identity());
            int t = 0;
            for (; t + 8 <= nseg; t += 8) {  // 8 loads in flight, then the adds in segment order
                float4 x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = __ldcg(reinterpret_cast<const float4*>(part + (size_t)(t + u) * n + c));
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    sum = make_float4(SR::add(sum.x, x[u].x), SR::add(sum.y, x[u].y), SR::add(sum.z, x[u].z),
                                      SR::add(sum.w, x[u].w));
            }
            for (; t < nseg; ++t) {
                const float4 x = __ldcg(reinterpret_cast<const float4*>(part + (size_t)t * n + c));
                sum = make_float4(SR::add(sum.x, x.x), SR::add(sum.y, x.y), SR::add(sum.z, x.z), SR::add(sum.w, x.w));
            }
            out[c] = Elem<TC>::from_f(sum.x);
            out[c + 1] = Elem<TC>::from_f(sum.y);
            out[c + 2] = Elem<TC>::from_f(sum.z);
            out[c + 3] = Elem<TC>::from_f(sum.w);
        }
    } else {
        for (int c = lane; c < n; c += 32) {
            float sum = SR::identity();
            int t = 0;
            for (; t + 8 <= nseg; t += 8) {
                float x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) x[u] = __ldcg(part + (size_t)(t + u) * n + c);
#pragma unroll
                for (int u = 0; u < 8; ++u) sum = SR::add(sum, x[u]);
            }
            for (; t < nseg; ++t) sum = SR::add(sum, __ldcg(part + (size_t)t * n + c));
            out[c] = Elem<TC>::from_f(sum);
        }
    }
}

// Segment pass of the hybrid: persistent warps take (slab, segment) work items
// from a counter, slab-major, so the warps running together gather from one
// column slab of B.  The (column, value) pairs of the next warp batch are
// loaded while the current batch's gathers are in flight.
template <typename TV, typename TB, typename TC, int VEC, int W, typename SR = PlusTimes>
__global__ void __launch_bounds__(kThreads, 3) rowsplit_segment_kernel(RowSplitArgs a, LongRowArgs l, int slabs) {
    constexpr int U = gathers_per_batch<TB, VEC>();
    constexpr int CV = (U > W) ? U / W : 1;  // (column, value) pairs per lane per warp batch
    constexpr int BS = W * CV;               // nonzeros per lane group per warp batch
    constexpr int G = BS / U;                // groups of U gathers per batch
    constexpr int WB = 32 * CV;              // nonzeros per warp batch
    pdl_wait();  // the row-block pass has queued every long row
    const int lane = threadIdx.x & 31;
    const int sl = lane & (W - 1);
    const int grp = lane / W;
    const TV* __restrict__ vals = static_cast<const TV*>(a.vals);
    const TB* __restrict__ B = static_cast<const TB*>(a.B);
    TC* __restrict__ C = static_cast<TC*>(a.C);
    constexpr int NG = 32 / W;               // lane groups per warp
    // segments of rows with several first (the longest rows start earliest), then the single rows, then
    // the mid rows, NG to a work item: the longer ones (from the back of mid[]) before the shorter ones
    const int n_multi = min(__ldcg(l.counts + 1), l.max_parts);
    const int n_single = min(__ldcg(l.counts), l.max_singles);
    constexpr bool kSplit = split_mid_rows<W>();
    const int n_mid = min(__ldcg(l.counts + 3), l.max_mid);
    int n_mid2 = 0;  // stays 0 for narrow lane groups (one class)
    if constexpr (kSplit) {
        n_mid2 = min(__ldcg(l.counts + 4), l.max_mid);
        if (n_mid + n_mid2 > l.max_mid) {  // the two ends met: not a valid matrix for this workspace
            if (threadIdx.x == 0 && blockIdx.x == 0) report(l.status, SPMM_ERR_BAD_CSR);
            n_mid2 = l.max_mid - n_mid;
        }
    }
    const int items2 = (n_mid2 + NG - 1) / NG;  // work items of the longer mid rows
    const int count = n_multi + n_single + items2 + (n_mid + NG - 1) / NG;
    const long long items = (long long)count * slabs;
    for (;;) {
        long long item = 0;
        if (lane == 0) item = (long long)atomicAdd(reinterpret_cast<unsigned int*>(l.counts + 2), 1u);
        item = __shfl_sync(kFullMask, item, 0);
        if (item >= items) break;
        const int slab = (int)(item / count);
        const int i = (int)(item - (long long)slab * count);
        if (i >= n_multi + n_single) {  // one lane group per mid row
            if constexpr (kSplit) {
                const int t = i - n_multi - n_single;
                int r = -1;
                if (t < items2) {
                    const int q = t * NG + grp;
                    if (q < n_mid2) r = __ldcg(l.mid + (l.max_mid - 1 - q));
                } else {
                    const int q = (t - items2) * NG + grp;
                    if (q < n_mid) r = __ldcg(l.mid + q);
                }
                rowsplit_row<TV, TB, TC, VEC, W, SR>(a, (r < 0 || r >= a.m) ? (long long)a.m : (long long)r, slab);
            } else {
                const int q = (i - n_multi - n_single) * NG + grp;
                const int r = q < n_mid ? __ldcg(l.mid + q) : -1;
                rowsplit_row<TV, TB, TC, VEC, W, SR>(a, (r < 0 || r >= a.m) ? (long long)a.m : (long long)r, slab);
            }
            continue;
        }
        const long long col0 = (long long)slab * (W * VEC) + (long long)sl * VEC;
        const bool col_ok = col0 < a.n;
        int row, pfirst = -1;
        if (i < n_multi) {
            const int2 d = __ldcg(l.multi + i);
            row = d.x;
            pfirst = d.y;
        } else {
            row = __ldcg(l.single + (i - n_multi));
        }
        if (row < 0 || row >= a.m) continue;  // a slot of a reservation that did not fit
        const int rs = __ldg(a.row_ptr + row), re = __ldg(a.row_ptr + row + 1);
        const int nseg = pfirst < 0 ? 1 : long_row_segments(re - rs, l.seg_len);
        const int len_s = (re - rs + nseg - 1) / nseg;  // nonzeros per segment of this row
        const int p0 = pfirst < 0 ? rs : rs + (i - pfirst) * len_s;
        const int p1 = (int)min((long long)p0 + len_s, (long long)re);
        float acc[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = SR::identity();
        int mc[CV];
        float mv[CV];
#pragma unroll
        for (int c = 0; c < CV; ++c) {
            const int p = p0 + c * 32 + lane;
            const bool ok = p < p1;
            mc[c] = ok ? __ldg(a.col_ind + p) : 0;
            mv[c] = ok ? load_f(vals + p) : 0.0f;
        }
        for (int base = p0; base < p1; base += WB) {
            int nc[CV];
            float nv[CV];
#pragma unroll
            for (int c = 0; c < CV; ++c) {
                const int p = base + WB + c * 32 + lane;
                const bool ok = p < p1;
                nc[c] = ok ? __ldg(a.col_ind + p) : 0;
                nv[c] = ok ? load_f(vals + p) : 0.0f;
            }
            // this lane group's nonzero j of the batch sits at base + grp * W + (j / W) * 32 + j % W,
            // so it exists iff (j / W) * 32 + j % W < lim
            const int lim = p1 - base - grp * W;
            auto in = [&](int j) { return (j / W) * 32 + (j % W) < lim; };
#pragma unroll
            for (int g = 0; g < G; ++g) {
                if (g > 0 && __all_sync(kFullMask, !in(g * U))) break;
                Raw<TB, VEC> bv[U];
                float vv[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = g * U + u;
                    const int c = __shfl_sync(kFullMask, mc[j / W], j % W, W);
                    vv[u] = __shfl_sync(kFullMask, mv[j / W], j % W, W);
                    bv[u] = (in(j) && col_ok) ? load_raw<TB, VEC>(gather_row(B, col0, c, a.ldb))
                                              : zero_raw<TB, VEC>();
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if constexpr (SR::kZeroPadOk) fma_raw<TB, VEC>(acc, vv[u], bv[u]);
                    else if (in(g * U + u)) accum_raw<SR, TB, VEC>(acc, vv[u], bv[u]);
                }
            }
#pragma unroll
            for (int c = 0; c < CV; ++c) {
                mc[c] = nc[c];
                mv[c] = nv[c];
            }
        }
#pragma unroll
        for (int off = W; off < 32; off <<= 1)
#pragma unroll
            for (int e = 0; e < VEC; ++e) acc[e] = SR::add(acc[e], __shfl_xor_sync(kFullMask, acc[e], off));
        if (nseg == 1) {
            if (grp == 0 && col_ok) store_vec<TC, VEC>(C + (long long)row * a.ldc + col0, acc);
            continue;
        }
        const int slot = i;
        if (grp == 0 && col_ok) {
            float* pp = l.partial + (size_t)slot * a.n + col0;
#pragma unroll
            for (int e = 0; e < VEC; ++e) pp[e] = acc[e];
        }
        __threadfence();  // this lane's partial is visible device-wide before the arrival below
        __syncwarp();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(l.arrive + pfirst, 1);
        prev = __shfl_sync(kFullMask, prev, 0);
        if ((long long)prev == (long long)nseg * slabs - 1) {  // every segment of every slab is in
            __threadfence();
            finish_long_row<TC, SR>(l.partial + (size_t)pfirst * a.n, nseg, a.n, C + (long long)row * a.ldc);
        }
    }
}

}  // namespace spmm
