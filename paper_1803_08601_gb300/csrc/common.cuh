// Device-side building blocks shared by the SpMM kernels: element types and
// 128-bit vector loads/stores, float32 accumulation helpers, and the bulk-copy
// (TMA) / mbarrier primitives with bounded waits.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spmm.h"

namespace spmm {

constexpr unsigned kFullMask = 0xffffffffu;
constexpr int kThreads = 256;       // threads per CTA of the row-split, SDDMM and batched kernels
// CTA shape of the merge-based kernel for W lanes per row: narrow rows (W <= 8)
// use 128-thread CTAs with 1024-item tiles (small barrier domains, six CTAs per
// SM); wide rows use 256-thread CTAs with 2048-item tiles (fewer tiles).
__host__ __device__ constexpr int merge_cta_threads(int W) { return W >= 16 ? 256 : 128; }
__host__ __device__ constexpr int merge_tile_items(int W) { return W >= 16 ? 2048 : 1024; }
constexpr int kUnroll = 8;     // gathers of B in flight per lane
// Gathers in flight per lane for accesses of VEC elements of T: kUnroll for one
// 16-byte vector, half as many for the two 16-byte vectors of the float32
// access of 8 columns (so a lane keeps 128 bytes in flight either way).
template <typename T, int VEC>
__host__ __device__ constexpr int gathers_per_batch() { return VEC * (int)sizeof(T) > 16 ? kUnroll / 2 : kUnroll; }

// ------------------------------------------------------------------ element types

template <typename T> struct Elem;
template <> struct Elem<float> {
    static constexpr int kVec = 4;  // elements per 16-byte vector
    __device__ __forceinline__ static float to_f(float x) { return x; }
    __device__ __forceinline__ static float from_f(float x) { return x; }
};
template <> struct Elem<__nv_bfloat16> {
    static constexpr int kVec = 8;
    __device__ __forceinline__ static float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
    __device__ __forceinline__ static __nv_bfloat16 from_f(float x) { return __float2bfloat16_rn(x); }
    __device__ __forceinline__ static __nv_bfloat16 from_bits(uint16_t b) { return __ushort_as_bfloat16(b); }
    __device__ __forceinline__ static uint16_t to_bits(__nv_bfloat16 x) { return __bfloat16_as_ushort(x); }
};
template <> struct Elem<__half> {
    static constexpr int kVec = 8;
    __device__ __forceinline__ static float to_f(__half x) { return __half2float(x); }
    __device__ __forceinline__ static __half from_f(float x) { return __float2half_rn(x); }
    __device__ __forceinline__ static __half from_bits(uint16_t b) { return __ushort_as_half(b); }
    __device__ __forceinline__ static uint16_t to_bits(__half x) { return __half_as_ushort(x); }
};

// Read-only load of one value as float.
template <typename T>
__device__ __forceinline__ float load_f(const T* p) {
    return Elem<T>::to_f(__ldg(p));
}

// Load VEC consecutive elements starting at p (VEC == 1 or the 16-byte width
// of T, in which case p is 16-byte aligned) and widen them to float.
template <typename T, int VEC>
__device__ __forceinline__ void load_vec(const T* p, float (&out)[VEC]) {
    if constexpr (VEC == 1) {
        out[0] = load_f(p);
    } else if constexpr (sizeof(T) == 4) {
        static_assert(VEC == 4 || VEC == 8, "float accesses are one or two 16-byte vectors");
#pragma unroll
        for (int i = 0; i < VEC; i += 4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(p + i));
            out[i] = v.x; out[i + 1] = v.y; out[i + 2] = v.z; out[i + 3] = v.w;
        }
    } else {
        static_assert(VEC == 8, "16-bit vectors are 8 wide");
        const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            out[2 * i] = Elem<T>::to_f(Elem<T>::from_bits((uint16_t)(w[i] & 0xffffu)));
            out[2 * i + 1] = Elem<T>::to_f(Elem<T>::from_bits((uint16_t)(w[i] >> 16)));
        }
    }
}

// Raw (not yet widened) storage of VEC elements of T as one load brings them
// in: the gathers of a batch are issued into these, and widened only when they
// are accumulated, so a batch of 16-bit rows costs 4 registers per gather.
template <typename T, int VEC> struct Raw;
template <typename T> struct Raw<T, 1> { T v; };
template <> struct Raw<float, 4> { float4 v; };
template <> struct Raw<float, 8> { float4 v, w; };  // two 16-byte vectors of one lane
template <> struct Raw<__nv_bfloat16, 8> { uint4 v; };
template <> struct Raw<__half, 8> { uint4 v; };

template <typename T, int VEC>
__device__ __forceinline__ Raw<T, VEC> load_raw(const T* p) {
    Raw<T, VEC> r;
    if constexpr (VEC == 1) {
        r.v = __ldg(p);
    } else if constexpr (sizeof(T) == 4 && VEC == 8) {
        r.v = __ldg(reinterpret_cast<const float4*>(p));
        r.w = __ldg(reinterpret_cast<const float4*>(p) + 1);
    } else if constexpr (sizeof(T) == 4) {
        r.v = __ldg(reinterpret_cast<const float4*>(p));
    }
    else r.v = __ldg(reinterpret_cast<const uint4*>(p));
    return r;
}

template <typename T, int VEC>
__device__ __forceinline__ Raw<T, VEC> zero_raw() {
    Raw<T, VEC> r;
    if constexpr (VEC == 1) {
        r.v = Elem<T>::from_f(0.0f);
    } else if constexpr (sizeof(T) == 4 && VEC == 8) {
        r.v = make_float4(0.f, 0.f, 0.f, 0.f);
        r.w = r.v;
    } else if constexpr (sizeof(T) == 4) {
        r.v = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    else r.v = make_uint4(0u, 0u, 0u, 0u);
    return r;
}

// Row r of a row-major matrix whose rows are stride_bytes apart, from the
// address of row 0 (offset to the caller's columns).  A 32-bit row index times
// a 32-bit byte stride is one wide multiply-add per gather, where a 64-bit
// index product costs several instructions on the path every nonzero takes;
// the host entry points reject leading dimensions of 2^32 bytes or more.
template <typename T>
__device__ __forceinline__ const T* row_at(const T* base, int r, unsigned stride_bytes) {
    return reinterpret_cast<const T*>(reinterpret_cast<const char*>(base) + (unsigned long long)(unsigned)r * stride_bytes);
}

// The gathered row r of B at column offset col0 with leading dimension ld.
// float32 rows take the byte-stride form above.  For 16-bit rows the compiler
// then keeps fewer of a batch's gathers in flight (the row split of bf16 rows
// of 256 bytes: 2.06 -> 2.51 ms on a 2M x 2M, 32 per row matrix), so they keep
// the 64-bit index product.
template <typename T>
__device__ __forceinline__ const T* gather_row(const T* B, long long col0, int r, long long ld) {
    if constexpr (sizeof(T) == 4) return row_at(B + col0, r, (unsigned)(ld * (long long)sizeof(T)));
    else return B + (long long)r * ld + col0;
}

// acc[e] += a * element e of r, in float32 (fused multiply-add).
template <typename T, int VEC>
__device__ __forceinline__ void fma_raw(float (&acc)[VEC], float a, const Raw<T, VEC>& r) {
    if constexpr (VEC == 1) {
        acc[0] = fmaf(a, Elem<T>::to_f(r.v), acc[0]);
    } else if constexpr (sizeof(T) == 4 && VEC == 8) {
        acc[0] = fmaf(a, r.v.x, acc[0]);
        acc[1] = fmaf(a, r.v.y, acc[1]);
        acc[2] = fmaf(a, r.v.z, acc[2]);
        acc[3] = fmaf(a, r.v.w, acc[3]);
        acc[4] = fmaf(a, r.w.x, acc[4]);
        acc[5] = fmaf(a, r.w.y, acc[5]);
        acc[6] = fmaf(a, r.w.z, acc[6]);
        acc[7] = fmaf(a, r.w.w, acc[7]);
    } else if constexpr (sizeof(T) == 4) {
        acc[0] = fmaf(a, r.v.x, acc[0]);
        acc[1] = fmaf(a, r.v.y, acc[1]);
        acc[2] = fmaf(a, r.v.z, acc[2]);
        acc[3] = fmaf(a, r.v.w, acc[3]);
    } else {
        const uint32_t w[4] = {r.v.x, r.v.y, r.v.z, r.v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[2 * i] = fmaf(a, Elem<T>::to_f(Elem<T>::from_bits((uint16_t)(w[i] & 0xffffu))), acc[2 * i]);
            acc[2 * i + 1] = fmaf(a, Elem<T>::to_f(Elem<T>::from_bits((uint16_t)(w[i] >> 16))), acc[2 * i + 1]);
        }
    }
}

// ------------------------------------------------------------------ semirings
//
// C = A (+).(x) B (the GraphBLAS matrix product named in Section 1).  Each tag
// gives the identity of (+), (+) itself, and acc (+) (a (x) b).  PlusTimes is
// the ordinary product; its padding lanes may add 0 * 0, the others must skip
// padded terms (kZeroPadOk = false).
struct PlusTimes {
    static constexpr bool kZeroPadOk = true;
    __device__ __forceinline__ static float identity() { return 0.0f; }
    __device__ __forceinline__ static float add(float x, float y) { return x + y; }
    __device__ __forceinline__ static float mul_add(float acc, float a, float b) { return fmaf(a, b, acc); }
};
struct MinPlus {
    static constexpr bool kZeroPadOk = false;
    __device__ __forceinline__ static float identity() { return __int_as_float(0x7f800000); }  // +inf
    __device__ __forceinline__ static float add(float x, float y) { return fminf(x, y); }
    __device__ __forceinline__ static float mul_add(float acc, float a, float b) { return fminf(acc, a + b); }
};
struct MaxPlus {
    static constexpr bool kZeroPadOk = false;
    __device__ __forceinline__ static float identity() { return __int_as_float(0xff800000); }  // -inf
    __device__ __forceinline__ static float add(float x, float y) { return fmaxf(x, y); }
    __device__ __forceinline__ static float mul_add(float acc, float a, float b) { return fmaxf(acc, a + b); }
};
struct MaxTimes {
    static constexpr bool kZeroPadOk = false;
    __device__ __forceinline__ static float identity() { return __int_as_float(0xff800000); }  // -inf
    __device__ __forceinline__ static float add(float x, float y) { return fmaxf(x, y); }
    __device__ __forceinline__ static float mul_add(float acc, float a, float b) { return fmaxf(acc, a * b); }
};

// acc[e] = acc[e] (+) (a (x) element e of r).
template <typename SR, typename T, int VEC>
__device__ __forceinline__ void accum_raw(float (&acc)[VEC], float a, const Raw<T, VEC>& r) {
    if constexpr (SR::kZeroPadOk) {
        fma_raw<T, VEC>(acc, a, r);
    } else {
        float b[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) b[e] = 0.0f;
        fma_raw<T, VEC>(b, 1.0f, r);  // widen
#pragma unroll
        for (int e = 0; e < VEC; ++e) acc[e] = SR::mul_add(acc[e], a, b[e]);
    }
}

// Store VEC floats as TC at p (p aligned to VEC * sizeof(TC) when VEC > 1).
template <typename TC, int VEC>
__device__ __forceinline__ void store_vec(TC* p, const float (&v)[VEC]) {
    if constexpr (VEC == 1) {
        p[0] = Elem<TC>::from_f(v[0]);
    } else if constexpr (sizeof(TC) == 4) {
#pragma unroll
        for (int i = 0; i < VEC; i += 4)
            *reinterpret_cast<float4*>(p + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
    } else {
        // 16-bit output: pack pairs, write 8 or 16 bytes at a time
        uint32_t w[VEC / 2];
#pragma unroll
        for (int i = 0; i < VEC / 2; ++i) {
            const uint32_t l = Elem<TC>::to_bits(Elem<TC>::from_f(v[2 * i]));
            const uint32_t h = Elem<TC>::to_bits(Elem<TC>::from_f(v[2 * i + 1]));
            w[i] = l | (h << 16);
        }
        if constexpr (VEC == 8) {
            *reinterpret_cast<uint4*>(p) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            static_assert(VEC == 4, "unexpected vector width");
            *reinterpret_cast<uint2*>(p) = make_uint2(w[0], w[1]);
        }
    }
}

// ------------------------------------------------------------------ timing / status

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start while its predecessor drains; pdl_wait() returns once
// the predecessor grid has completed and its memory is visible (a no-op when
// the kernel was launched without the attribute).  pdl_launch_dependents()
// lets the next kernel in the stream be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ void report(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ mbarrier + bulk copy

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned),
// completed by cp_async_wait<N>() once at most N newer groups are pending.
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// VEC elements of T from shared memory (16-byte aligned when VEC > 1).
template <typename T, int VEC>
__device__ __forceinline__ Raw<T, VEC> lds_raw(const T* p) {
    Raw<T, VEC> r;
    if constexpr (VEC == 1) {
        r.v = *p;
    } else if constexpr (sizeof(T) == 4 && VEC == 8) {
        r.v = *reinterpret_cast<const float4*>(p);
        r.w = *(reinterpret_cast<const float4*>(p) + 1);
    } else if constexpr (sizeof(T) == 4) {
        r.v = *reinterpret_cast<const float4*>(p);
    }
    else r.v = *reinterpret_cast<const uint4*>(p);
    return r;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// One arrival that also announces `bytes` of asynchronous transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait until phase `parity` of the barrier completes, for at most limit_ns of
// device time.  Returns false if the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned long long limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > limit_ns) return false;
    }
}

// 1-D bulk copy global -> shared (TMA engine, no multicast), completing
// `bytes` transactions on `bar`.  dst and src 16-byte aligned, bytes % 16 == 0.
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Round an element index down / up to a 16-byte boundary of T.
template <typename T>
__host__ __device__ __forceinline__ long long align_down16(long long i) {
    constexpr long long g = 16 / (long long)sizeof(T);
    return i - (i % g + g) % g;
}
template <typename T>
__host__ __device__ __forceinline__ long long align_up16(long long i) {
    constexpr long long g = 16 / (long long)sizeof(T);
    return align_down16<T>(i + g - 1);
}

}  // namespace spmm
