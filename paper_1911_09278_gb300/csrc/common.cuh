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

// --- stored column format ----------------------------------------------------
// Column of one pixel for one agent (the per-view runs, flattened):
//   u32 nnz; u16 bidx[nnz]   (position of each value in the super-voxel's band:
//                             runs of the agent's views in view order)
//   zero padding to 16 bytes; T vals[nnz]; zero padding to 16 bytes.
// The 4-byte header puts entries (2k, 2k+1) of bidx in one aligned u32 and of
// vals in one aligned 8-byte (FP32) or 4-byte (BF16/FP16) word, so one lane
// loads a pair with two instructions.  For odd nnz the pair's second half is
// padding: index 0, value 0.
// View v's band covers channels [lo_v, lo_v + len_v) and starts at
// boff_v = sum_{u < v} len_u, so the value of channel c sits at
// boff_v + c - lo_v: the run (first channel, length, values) of every view is
// recoverable from bidx and the band descriptors.
__host__ __device__ inline uint32_t col_idx_bytes(int nnz)
{
    return (4u + 2u * (uint32_t)nnz + 15u) & ~15u;
}
__host__ __device__ inline uint32_t col_bytes_of(int nnz, int vbytes)
{
    return col_idx_bytes(nnz) + (((uint32_t)nnz * vbytes + 15u) & ~15u);
}

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

// values 2k and 2k+1 of a column's value array, widened to float
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

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// --- super-voxel band bookkeeping ---------------------------------------------
// Shared by the kernels that walk a super-voxel's columns: per view the band
// descriptor, its offset in the flattened band and, per band entry, its view.
// Returns the band size.  Warp-cooperative.  bd may point to global or shared
// memory; bdesc may alias bd.
__device__ __forceinline__ int load_band_layout(const uint32_t *bd, int Vg, uint32_t *bdesc,
                                                uint16_t *boff, uint16_t *bview, int lane)
{
    const unsigned FULL = 0xffffffffu;
    int run = 0;
    for (int r = 0; r * 32 < Vg; ++r) {
        const int v = r * 32 + lane;
        const uint32_t d = v < Vg ? bd[v] : 0u;
        const int len = (int)(d >> 16);
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (v < Vg) {
            const int b0 = run + incl - len;
            boff[v] = (uint16_t)b0;
            bdesc[v] = d;
            for (int k = 0; k < len; ++k) bview[b0 + k] = (uint16_t)v;
        }
        run += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    return run;
}

// The same bookkeeping with, per band entry, its index in the agent block
// ([Vg][D]) instead of its view, so loading and flushing the band need one
// shared-memory read per entry.  Returns the band size.  Warp-cooperative.
__device__ __forceinline__ int load_band_index(const uint32_t *bd, int Vg, int D, uint32_t *bdesc,
                                               uint32_t *bglob, int lane)
{
    const unsigned FULL = 0xffffffffu;
    int run = 0;
    for (int r = 0; r * 32 < Vg; ++r) {
        const int v = r * 32 + lane;
        const uint32_t d = v < Vg ? bd[v] : 0u;
        const int len = (int)(d >> 16);
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += y;
        }
        if (v < Vg) {
            const int b0 = run + incl - len;
            bdesc[v] = d;
            const uint32_t g0 = (uint32_t)v * (uint32_t)D + (d & 0xFFFFu);
            for (int k = 0; k < len; ++k) bglob[b0 + k] = g0 + (uint32_t)k;
        }
        run += __shfl_sync(FULL, incl, 31);
    }
    __syncwarp();
    return run;
}

// global index (row of the agent block, [Vg][D]) of band entry f
__device__ __forceinline__ int64_t band_global(int f, const uint32_t *bdesc, const uint16_t *boff,
                                               const uint16_t *bview, int D)
{
    const int v = bview[f];
    return (int64_t)v * D + (int)(bdesc[v] & 0xFFFFu) + (f - boff[v]);
}

// Per-warp shared memory of the kernels that walk columns outside the sweep:
// band descriptors, offsets, entry views and one float per band entry.
__host__ __device__ inline size_t aux_warp_bytes(int max_band, int max_views)
{
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    return r16((size_t)max_views * 4) + r16((size_t)max_views * 2) + r16((size_t)max_band * 2) +
           r16((size_t)max_band * 4);
}
