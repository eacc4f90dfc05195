// Device helpers shared by the translation units of libmace.so: constants,
// inline-PTX wrappers (mbarrier, TMA bulk copy, cp.async), the stored column
// format and the super-voxel band bookkeeping.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "../../include/mace.h"

static constexpr int kMaxViews = 4096;     // per geometry
// Column ring stages per warp (a power of two).  Four cover the copy latency
// at the sweep's pixel rate and leave shared memory for more warps per SM.
#ifndef MACE_RING
#define MACE_RING 4
#endif
static constexpr int kRing = MACE_RING;
static constexpr uint32_t kSpinLimit = 1u << 26;  // bounded device waits
static constexpr int kStatusTimeout = 1;
static constexpr int kStatusBounds = 2;      // a MACE_DEBUG bounds check failed

// MACE_DEBUG builds check the indices the kernels read from stored data
// (run headers, three-channel list codes, band descriptors, column sizes)
// against the buffers they address; a failed check sets the device status
// word to kStatusBounds (the host returns an error) and the access is
// redirected to a safe location instead of being made.
#ifdef MACE_DEBUG
static constexpr bool kDebug = true;
#else
static constexpr bool kDebug = false;
#endif
__device__ __forceinline__ bool debug_ok(bool cond, int *status)
{
    if (kDebug && !cond) atomicExch(status, kStatusBounds);
    return !kDebug || cond;
}

// --- stored column format ----------------------------------------------------
// Column of one pixel for one agent with Vg views: the per-view runs (first
// channel, run length <= 3, values) of the paper's stored matrix, laid out so
// that lane l of a warp can take view l:
//   u16 n3                        views whose run has three channels
//   u8  hdr[Vg]                   per view: r | L << 6, with L the run length
//                                 (0..3) and r = c0 - lo the first channel
//                                 relative to the super-voxel's band of that
//                                 view (0 when L = 0)
//   (pad to 8 bytes)  T v01[Vg][2] the run's first two values (zero past L)
//   u16 ovc[n3]                   the views with L = 3, each coded as
//                                 (r + 2) * vpad + v: the band position
//                                 (row r + 2, view v) of the third value
//   (pad to 4 bytes)  T ov[n3]    their third values
//   (zero padding to 16 bytes)
// The value the run stores for channel lo_v + r + k is v01[v][k] (k < 2) or
// the matching ov entry (k = 2).  vpad (the view stride of a band row) is a
// property of the matrix: the number of views of its largest agent rounded
// up to a multiple of 16.
__host__ __device__ inline int col_v01(int Vg) { return (2 + Vg + 7) & ~7; }
__host__ __device__ inline int col_ovc(int Vg, int vb) { return col_v01(Vg) + 2 * vb * Vg; }
__host__ __device__ inline int col_ovv(int Vg, int vb, int n3) { return (col_ovc(Vg, vb) + 2 * n3 + 3) & ~3; }
__host__ __device__ inline uint32_t col_bytes(int Vg, int vb, int n3)
{
    return (uint32_t)((col_ovv(Vg, vb, n3) + n3 * vb + 15) & ~15);
}
static constexpr int kMaxRunOff = 63;   // r is stored in 6 bits

template <typename T> __device__ __forceinline__ float ld_val(const uint8_t *p, int idx);
template <> __device__ __forceinline__ float ld_val<float>(const uint8_t *p, int idx) { return ((const float *)p)[idx]; }
template <> __device__ __forceinline__ float ld_val<__nv_bfloat16>(const uint8_t *p, int idx)
{
    return __bfloat162float(((const __nv_bfloat16 *)p)[idx]);
}
template <> __device__ __forceinline__ float ld_val<__half>(const uint8_t *p, int idx)
{
    return __half2float(((const __half *)p)[idx]);
}

// values 2k and 2k+1 of a value array, widened to float
template <typename T> __device__ __forceinline__ float2 ld_pair(const uint8_t *p, int k);
template <> __device__ __forceinline__ float2 ld_pair<float>(const uint8_t *p, int k) { return ((const float2 *)p)[k]; }
template <> __device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const uint8_t *p, int k)
{
    return __bfloat1622float2(((const __nv_bfloat162 *)p)[k]);
}
template <> __device__ __forceinline__ float2 ld_pair<__half>(const uint8_t *p, int k)
{
    return __half22float2(((const __half2 *)p)[k]);
}

__device__ __forceinline__ float ld_any(const uint8_t *p, int idx, int dtype)
{
    if (dtype == MACE_F32) return ld_val<float>(p, idx);
    if (dtype == MACE_BF16) return ld_val<__nv_bfloat16>(p, idx);
    return ld_val<__half>(p, idx);
}

// --- order-independent accumulation of e --------------------------------------
// Changes of e that several warps add to one entry go into a 64-bit integer
// accumulator in units of 2^-40 (integer addition is associative, so the sum
// does not depend on the order of the additions) and are folded into e once
// all are in.  |changes| < 2^23.
static constexpr float kEScale = 1099511627776.0f;        // 2^40
static constexpr float kEUnit = 9.094947017729282e-13f;   // 2^-40
__device__ __forceinline__ void efix_add(unsigned long long *p, float d)
{
    const long long q = __float2ll_rn(d * kEScale);
    if (q != 0) atomicAdd(p, (unsigned long long)q);
}
__device__ __forceinline__ float efix_value(unsigned long long v) { return __ll2float_rn((long long)v) * kEUnit; }

// --- PTX helpers -------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1D TMA bulk copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// L2 policy for data read once per pass (the stored matrix): evicted first,
// so the small state every super-voxel re-reads (e, Lambda, X, w, theta2)
// stays in L2 while the matrix streams through
__device__ __forceinline__ uint64_t l2_evict_first_policy()
{
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// The same, armed and issued by lane 0 of the warp only (predicated, so the
// warp does not diverge around it), with an L2 cache policy
__device__ __forceinline__ void tma_load_1d_lane0(void *dst, const void *src, uint32_t bytes, uint64_t *bar, int lane,
                                                  uint64_t policy)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.eq.u32 p, %4, 0;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%3], %2;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %5;\n\t}"
        ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "r"((uint32_t)lane), "l"(policy)
        : "memory");
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
// the same with 32-bit shared-window destination addresses
__device__ __forceinline__ void cp_async4_s(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8_s(uint32_t dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ float lds_f32(uint32_t a)
{
    float v;
    asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds_u32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_f2(uint32_t a, float2 v)
{
    asm volatile("st.shared.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a)
{
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a) : "memory");
    return v;
}
// stored values at a shared address, widened to float: one, or two adjacent
template <typename T> __device__ __forceinline__ float lds_val(uint32_t a);
template <> __device__ __forceinline__ float lds_val<float>(uint32_t a) { return lds_f32(a); }
template <> __device__ __forceinline__ float lds_val<__nv_bfloat16>(uint32_t a)
{
    return __uint_as_float(lds_u16(a) << 16);
}
template <> __device__ __forceinline__ float lds_val<__half>(uint32_t a)
{
    return __half2float(__ushort_as_half((unsigned short)lds_u16(a)));
}
template <typename T> __device__ __forceinline__ float2 lds_pair(uint32_t a);
template <> __device__ __forceinline__ float2 lds_pair<float>(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
template <> __device__ __forceinline__ float2 lds_pair<__nv_bfloat16>(uint32_t a)
{
    const uint32_t w = lds_u32(a);
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
template <> __device__ __forceinline__ float2 lds_pair<__half>(uint32_t a)
{
    const uint32_t w = lds_u32(a);
    return __half22float2(*reinterpret_cast<const __half2 *>(&w));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// --- super-voxel band in shared memory ----------------------------------------
// The kernels that walk a super-voxel's columns keep its band of the agent's
// sinogram as rows t = 0 .. wmax-1 of vpad views: entry (t, v) is channel
// lo_v + t of view v, for t < len_v (band descriptor lo_v | len_v << 16), and
// otherwise a spare that no channel maps to.  A run (r, L) of view v touches
// rows r .. r + L - 1; wmax is the widest band plus one, so row r + 1 always
// exists.
__host__ __device__ inline size_t aux_warp_bytes(int vpad, int wmax)
{
    return ((size_t)vpad * 4 + 15) / 16 * 16 + ((size_t)wmax * vpad * 4 + 15) / 16 * 16;
}
