// The ICD sweep of partial-update MACE: one pass of Algorithm 2 (iterative
// coordinate descent for the proximal map F_i(v_i; sigma), Eq. "ICDUpdate1")
// for every agent of every reconstruction of a batch, over the stored system
// matrix.  Instantiated per stored value type in sweep_<type>.cu.
#pragma once

#include "common.cuh"

struct SweepArgs {
    const uint8_t *cols;
    const int64_t *sv_base;
    const uint32_t *col_off;
    const uint32_t *band;
    const int *view_off;
    const int32_t *sv_order;
    float2 *eL;
    float *X;
    const float *w;
    const double *wbar;
    const float *vexp;
    const float *theta2;        // [B][N][n]: sum over the agent's views of A_js^2 Lambda_j
    int *status;
    int B, N, nsv, nsvx, nx, ny, D;
    int64_t ne;
    int nwarps;                 // warps with work (the last block may have idle ones)
    int backward;
    int max_band, col_stride, max_views;   // per-warp shared-memory layout (S is a template parameter)
    float inv_s2, pscale;
    int prior;                  // 0 quadratic, 1 Q-GGMRF
    float inv_sx2, inv_Tsx, qexp, half_q_inv_sx2;   // prior constants
    float b_edge, b_diag;       // 8-neighbourhood weights (face, diagonal)
    int nb26;                   // 1: the batch is the z-stack of one volume, 26-neighbourhood prior
    float b26[3];               // 26-neighbourhood weights by squared distance 1, 2, 3
};

typedef void (*sweep_fn)(SweepArgs);

// Per-warp shared-memory layout (bytes, each part 16-aligned).  Shared by
// the warp's K chains (reconstructions of one batch group that run the same
// agent over the same super-voxels, so every column is loaded once for all):
//   ring:   kRing * col_stride            column staging (TMA destination)
//   bars:   kRing * 8                     mbarriers
//   bdesc:  2 * max_views * 4             band descriptors (lo | len << 16), current and next super-voxel
//   bglob:  max_band * 4                  index of each band entry in the agent block [Vg][D]
//   coff:   (S^2 + 1) * 4                 column byte offsets of the next super-voxel (staging)
//   pl:     2 * S^2 * 4                   per visited pixel: tile index | neighbour mask << 9
//   cl:     2 * S^2 * 8                   per visited pixel: (column offset from the matrix start
//                                         in 16-byte units, bytes)
//   halo:   2 * (S+2)^2 * 4               X tiles of the slices below and above (volumes only)
// and per chain:
//   beL:    (max_band + 1) * 8            (e, Lambda) of the band, e kept current; the last
//                                         entry takes the stores of lanes past a column's end
//   bsnap:  max_band * 4                  e of the band when the super-voxel began
//   xt:     (S+2)^2 * 4                   X tile with one-pixel halo
//   vt2:    S^2 * 8                       per visited pixel (v / sigma^2, theta2 + 1 / sigma^2)
struct WarpSmem {
    size_t ring, bars, bdesc, bglob, coff, pl, cl, halo, chain0, chain_size;
    size_t beL, bsnap, xt, vt2;
    size_t total;
};

__host__ __device__ inline WarpSmem warp_smem_layout(int max_band, int col_stride, int S, int max_views, int K,
                                                     int halo)
{
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t S2 = (size_t)S * S, TA = (size_t)(S + 2) * (S + 2);
    if (max_band < 1) max_band = 1;   // the gathers may read band entry 0
    WarpSmem L;
    size_t o = 0;
    L.ring = o;  o += r16((size_t)kRing * col_stride);
    L.bars = o;  o += r16(kRing * 8);
    L.bdesc = o; o += r16((size_t)2 * max_views * 4);
    L.bglob = o; o += r16((size_t)max_band * 4);
    L.coff = o;  o += r16((S2 + 1) * 4);
    L.pl = o;    o += r16(2 * S2 * 4);
    L.cl = o;    o += r16(2 * S2 * 8);
    L.halo = o;  o += halo ? r16(2 * TA * 4) : 0;
    L.chain0 = o;
    size_t c = 0;
    L.beL = c;   c += r16((size_t)(max_band + 1) * 8);   // + a sink entry for masked-off stores
    L.bsnap = c; c += r16((size_t)max_band * 4);
    L.xt = c;    c += r16(TA * 4);
    L.vt2 = c;   c += r16(S2 * 8);
    L.chain_size = c;
    L.total = o + (size_t)K * c;
    return L;
}

// Approximate reciprocal, base-2 logarithm and exponential (single PTX
// instructions, flush-to-zero).  They only enter step sizes and the prior's
// surrogate weight; their relative error (a few ulp) moves the fixed point by
// an amount of the order of FP32 rounding.
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float lg2_approx(float x)
{
    float r;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float ex2_approx(float x)
{
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Surrogate weight rho'(D)/D of the prior potential (quadratic: 1/sigma_x^2;
// Q-GGMRF with p = 2: (2 + q a) / (2 sigma_x^2 (1 + a)^2), a = |D/(T sigma_x)|^(p-q),
// the power taken as 2^((p-q) log2 |D/(T sigma_x)|); a = 0 at D = 0).
__device__ __forceinline__ float prior_weight(const SweepArgs &A, float d)
{
    if (A.prior == 0) return A.inv_sx2;
    const float a = ex2_approx(A.qexp * lg2_approx(fabsf(d * A.inv_Tsx)));
    const float r = rcp_approx(1.f + a);
    return fmaf(A.half_q_inv_sx2, a, A.inv_sx2) * r * r;
}

// Register cap of the one-chain sweep kernel: residency is limited by
// registers and shared memory together, and at 96 registers (21 warps per SM)
// the one-chain kernels do not spill; two-chain kernels are capped at 128
// (16 warps per SM), four-chain kernels keep their registers.
#ifndef MACE_SWEEP_MAXNREG
#define MACE_SWEEP_MAXNREG 96
#endif

// One warp runs K chains (reconstructions b0 .. b0+K-1 of one batch group,
// all on agent g) over a fixed sequence of super-voxels: slots c, c+C, c+2C,
// ... of the visiting order, where C warps serve the same (group, agent) -- so
// about C super-voxels of one agent of one reconstruction are in flight at a
// time.  Inside a super-voxel the pixels are visited in order; each pixel's
// column (a flat list of (band position, value) pairs) is streamed once by
// TMA for all K chains.  With one or four chains lane k takes the pairs k,
// k+32, ... for every chain (PR rounds: at most 64*PR entries; PR == 0: any
// count, one chain); with two chains the warp works as two 16-lane halves,
// half h updating chain h and taking the pairs hl, hl+16, ... (PR rounds of
// 16 lanes: at most 32*PR entries).  Pairs stay in registers between the
// reduction and the update, and the ring slot is refilled once they have been
// consumed.  The next super-voxel's metadata, visiting list and first columns
// are prepared while the current one is processed.
// NB26: the batch is the z-stack of one volume, 26-neighbourhood prior (K = 1).
template <typename T, int PR, int S, int K, bool NB26>
__global__ void __maxnreg__(K == 1 ? MACE_SWEEP_MAXNREG : K == 2 ? 128 : 224) icd_sweep_kernel(SweepArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int S2 = S * S, TS = S + 2, TA = TS * TS;
    static_assert(PR > 0 || K == 1, "uncached columns support one chain");
    static_assert(!NB26 || K == 1, "volumes run one chain per warp");
    static_assert((kRing & (kRing - 1)) == 0, "ring size is a power of two");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const WarpSmem Ly = warp_smem_layout(A.max_band, A.col_stride, S, A.max_views, K, NB26);
    uint8_t *base = smem + wib * Ly.total;
    uint8_t *ring = base + Ly.ring;
    uint64_t *bars = (uint64_t *)(base + Ly.bars);
    uint32_t *bdesc2 = (uint32_t *)(base + Ly.bdesc);
    uint32_t *bglob = (uint32_t *)(base + Ly.bglob);
    uint32_t *scoff = (uint32_t *)(base + Ly.coff);
    uint32_t *pl2 = (uint32_t *)(base + Ly.pl);
    uint2 *cl2 = (uint2 *)(base + Ly.cl);
    uint8_t *chains = base + Ly.chain0;
    float *halo_lo = (float *)(base + Ly.halo);
    float *halo_hi = halo_lo + TA;

    if (lane == 0)
        for (int k = 0; k < kRing; ++k) mbar_init(&bars[k], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();

    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = (int64_t)A.nx * A.ny;
    const int gw = blockIdx.x * (blockDim.x >> 5) + wib;
    if (gw >= A.nwarps) return;
    const int G = A.B / K;                      // batch groups
    const int pair = gw % (G * A.N);            // (group, agent)
    const int cidx = gw / (G * A.N);            // this warp's place among the C serving the pair
    const int grp = pair / A.N, g = pair - grp * A.N;
    const int v0 = A.view_off[g], Vg = A.view_off[g + 1] - v0;
    const int Cw = A.nwarps / (G * A.N);
    auto chain = [&](int k) { return chains + (size_t)k * Ly.chain_size; };

    // this lane's prior neighbour: lanes 0..7 the in-plane 8-neighbourhood,
    // or (volumes) lanes 0..25 the 26-neighbourhood; other lanes read the
    // pixel itself with weight 0.  mbit: the neighbour's bit in a pixel's
    // 3x3 in-image mask.  With two chains the warp works as two 16-lane
    // halves (half h: chain h), each with its own lanes 0..7.
    const int plane_lane = K == 2 ? (lane & 15) : lane;
    int pdz = 0, pdi = 0, pdj = 0;
    float pb = 0.f;
    if (NB26) {
        if (lane < 26) {
            const int kk = lane < 13 ? lane : lane + 1;   // skip the centre of the 3x3x3
            pdz = kk / 9 - 1;
            pdi = (kk / 3) % 3 - 1;
            pdj = kk % 3 - 1;
            const int d2 = pdz * pdz + pdi * pdi + pdj * pdj;
            const int zz = grp + pdz;
            pb = (zz >= 0 && zz < A.B) ? A.pscale * A.b26[d2 - 1] : 0.f;
        }
    } else if (plane_lane < 8) {
        const int kk = plane_lane < 4 ? plane_lane : plane_lane + 1;
        pdi = kk / 3 - 1;
        pdj = kk % 3 - 1;
        pb = A.pscale * ((pdi != 0 && pdj != 0) ? A.b_diag : A.b_edge);
    }
    const int mbit = (pdi + 1) * 3 + (pdj + 1);
    const int noff = pdi * TS + pdj;
    const float *nbase[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const float *xt = (const float *)(chain(k) + Ly.xt);
        nbase[k] = (pdz == 0 ? xt : (pdz < 0 ? halo_lo : halo_hi)) + noff;
    }
    // two chains: this lane's half's neighbour pointer
    const float *nb_half = (const float *)(chain(K == 2 ? (lane >> 4) : 0) + Ly.xt) + noff;

    // chain k: reconstruction grp*K + k
    auto eLk = [&](int k) { return A.eL + (int64_t)(grp * K + k) * A.ne + (int64_t)v0 * A.D; };
    auto Xk = [&](int k) { return A.X + ((int64_t)(grp * K + k) * A.N + g) * n; };

    // pixel t = ti * S + tj of a visiting-list word (tile index (ti+1)*TS + tj+1)
    auto tile_pixel = [&](uint32_t word) {
        const int tc = (int)(word & 0x1FFu);
        return (tc / TS - 1) * S + (tc % TS - 1);
    };

    // --- super-voxel metadata -------------------------------------------
    auto sv_of = [&](int m) {           // m-th super-voxel of this warp, -1 past the end
        const int slot = cidx + m * Cw;
        if (slot >= A.nsv) return -1;
        return A.sv_order[A.backward ? A.nsv - 1 - slot : slot];
    };
    // visiting list of super-voxel sv from its column offsets sc: per
    // non-empty pixel in visiting order its pixel/tile indices and in-image
    // neighbour mask, and its column's offset and size; returns the count
    auto build_list = [&](int svb, const uint32_t *sc, uint32_t *pl, uint2 *cl) {
        const int bi = (svb / A.nsvx) * S, bj = (svb % A.nsvx) * S;
        const int64_t svoff = A.sv_base[(int64_t)g * A.nsv + svb];
        int count = 0;
        for (int k0 = 0; k0 < S2; k0 += 32) {
            const int k = k0 + lane;
            const int t = A.backward ? S2 - 1 - k : k;
            const bool ne = k < S2 && sc[t + 1] != sc[t];
            const unsigned m = __ballot_sync(FULL, ne);
            if (ne) {
                const int ti = t / S, tj = t % S, i = bi + ti, j = bj + tj;
                uint32_t mask = 0;
#pragma unroll
                for (int di = -1; di <= 1; ++di)
#pragma unroll
                    for (int dj = -1; dj <= 1; ++dj)
                        if (i + di >= 0 && i + di < A.ny && j + dj >= 0 && j + dj < A.nx)
                            mask |= 1u << ((di + 1) * 3 + dj + 1);
                const int pos = count + __popc(m & lt_mask);
                pl[pos] = (uint32_t)((ti + 1) * TS + tj + 1) | mask << 9;
                cl[pos] = make_uint2((uint32_t)((svoff + sc[t]) >> 4), sc[t + 1] - sc[t]);
            }
            count += __popc(m);
        }
        __syncwarp();
        return count;
    };
    // TMA of one column into ring stage idx % kRing (one lane)
    auto issue = [&](uint32_t idx, const uint8_t *src, uint32_t bytes) {
        const uint32_t stg = idx & (kRing - 1);
        mbar_expect_tx(&bars[stg], bytes);
        tma_load_1d(ring + (size_t)stg * A.col_stride, src, bytes, &bars[stg]);
    };

    int sv = sv_of(0);
    if (sv < 0) return;
    // first super-voxel: metadata with plain loads
    {
        const uint32_t *coff = A.col_off + ((int64_t)g * A.nsv + sv) * (S2 + 1);
        for (int k = lane; k <= S2; k += 32) scoff[k] = coff[k];
        const uint32_t *bd = A.band + (int64_t)A.nsv * v0 + (int64_t)sv * Vg;
        for (int v = lane; v < Vg; v += 32) bdesc2[v] = bd[v];
        __syncwarp();
    }
    int count = build_list(sv, scoff, pl2, cl2);
    // The warp's columns form one sequence (its super-voxels' visiting lists
    // one after the other).  seq: columns consumed; issued: columns whose
    // copy has been started; seq0: sequence number of the current
    // super-voxel's first column.  Columns of the current and of the next
    // super-voxel (once its list is built) may be in flight, at most kRing.
    uint32_t issued = 0, seq = 0, seq0 = 0;
    int count_n = 0;
    int cur = 0;
    auto list_entry = [&](uint32_t x, const uint2 *cl, const uint2 *cl_n) {
        return x < (uint32_t)count ? cl[x] : cl_n[x - count];
    };
    auto col_src = [&](uint2 c) { return A.cols + ((uint64_t)c.x << 4); };
    auto fill_ring = [&](const uint2 *cl, const uint2 *cl_n) {
        while (issued - seq < (uint32_t)kRing && issued - seq0 < (uint32_t)(count + count_n)) {
            const uint2 c = list_entry(issued - seq0, cl, cl_n);
            if (lane == 0) issue(issued, col_src(c), c.y);
            ++issued;
        }
    };
    fill_ring(cl2, cl2 + S2);
    int status_seen = 0;
    // wait for column seq; false when the bounded wait gave up (the host is
    // flagged and this warp's copies in flight are drained first)
    auto wait_column = [&]() {
        const uint32_t stg = seq & (kRing - 1);
        const uint32_t parity = (seq / kRing) & 1u;
        uint32_t spins = 0;
        while (!__all_sync(FULL, mbar_try_wait(&bars[stg], parity))) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicExch(A.status, kStatusTimeout);
                for (uint32_t q2 = seq + 1; q2 < issued; ++q2) {
                    uint32_t sp2 = 0;
                    while (!mbar_try_wait(&bars[q2 & (kRing - 1)], (q2 / kRing) & 1u) && ++sp2 < kSpinLimit) {}
                }
                return false;
            }
        }
        return true;
    };

    for (int m = 0; sv >= 0; ++m) {
        uint32_t *bdesc = bdesc2 + cur * A.max_views;
        const uint32_t *pl = pl2 + cur * S2;
        const uint2 *cl = cl2 + cur * S2;
        uint32_t *bdesc_n = bdesc2 + (cur ^ 1) * A.max_views;
        uint32_t *pl_n = pl2 + (cur ^ 1) * S2;
        uint2 *cl_n = cl2 + (cur ^ 1) * S2;
        const int si = sv / A.nsvx, sj = sv - si * A.nsvx;

        // --- band layout; band, X and theta2 tiles of every chain -----------
        const int band_tot = load_band_index(bdesc, Vg, A.D, bdesc, bglob, lane);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint8_t *ch = chain(k);
            float2 *beL = (float2 *)(ch + Ly.beL);
            float *xt = (float *)(ch + Ly.xt);
            float2 *vt2 = (float2 *)(ch + Ly.vt2);
            const float2 *eL = eLk(k);
            for (int f = lane; f < band_tot; f += 32) cp_async8(&beL[f], &eL[bglob[f]]);
            // lanes past a column's end gather entry 0 with weight 0: keep it finite
            if (band_tot == 0 && lane == 0) beL[0] = make_float2(0.f, 0.f);
            const float *Xg = Xk(k);
            for (int q = lane; q < TA; q += 32) {
                const int i = si * S + q / TS - 1, j = sj * S + q % TS - 1;
                if (i >= 0 && i < A.ny && j >= 0 && j < A.nx) cp_async4(&xt[q], &Xg[(int64_t)i * A.nx + j]);
                else xt[q] = 0.f;
            }
            const float *t2g = A.theta2 + ((int64_t)(grp * K + k) * A.N + g) * n;
            for (int q = lane; q < count; q += 32) {
                const int t = tile_pixel(pl[q]);
                cp_async4(&vt2[q].y, &t2g[(int64_t)(si * S + t / S) * A.nx + sj * S + t % S]);
            }
        }
        if (NB26) {
            // X tiles of the neighbouring slices
            for (int h = 0; h < 2; ++h) {
                const int zz = grp + (h ? 1 : -1);
                float *ht = h ? halo_hi : halo_lo;
                const float *Xz = (zz >= 0 && zz < A.B) ? A.X + ((int64_t)zz * A.N + g) * n : nullptr;
                for (int q = lane; q < TA; q += 32) {
                    const int i = si * S + q / TS - 1, j = sj * S + q % TS - 1;
                    if (Xz && i >= 0 && i < A.ny && j >= 0 && j < A.nx) cp_async4(&ht[q], &Xz[(int64_t)i * A.nx + j]);
                    else ht[q] = 0.f;
                }
            }
        }
        cp_async_commit();
        // next super-voxel: claim its metadata while this one runs
        const int sv_n = sv_of(m + 1);
        if (sv_n >= 0) {
            const uint32_t *coff = A.col_off + ((int64_t)g * A.nsv + sv_n) * (S2 + 1);
            for (int k = lane; k <= S2; k += 32) cp_async4(&scoff[k], &coff[k]);
            const uint32_t *bd = A.band + (int64_t)A.nsv * v0 + (int64_t)sv_n * Vg;
            for (int v = lane; v < Vg; v += 32) cp_async4(&bdesc_n[v], &bd[v]);
        }
        cp_async_commit();
        // v (= 2 wbar - w from the FP64 consensus, or the caller's v) with
        // plain loads while the copies above are in flight
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float2 *vt2 = (float2 *)(chain(k) + Ly.vt2);
            const int64_t rb = (int64_t)(grp * K + k);
            for (int q = lane; q < count; q += 32) {
                const int t = tile_pixel(pl[q]);
                const int64_t s = (int64_t)(si * S + t / S) * A.nx + sj * S + t % S;
                const float vv = A.vexp ? A.vexp[(rb * A.N + g) * n + s]
                                        : (float)(2.0 * A.wbar[rb * n + s] - (double)A.w[(rb * A.N + g) * n + s]);
                vt2[q].x = vv * A.inv_s2;
            }
        }
        if (lane == 0) status_seen = *((volatile int *)A.status);
        cp_async_wait_all();
        __syncwarp();
        status_seen = __shfl_sync(FULL, status_seen, 0);
        count_n = 0;
        if (sv_n >= 0) count_n = build_list(sv_n, scoff, pl_n, cl_n);
        // a short super-voxel may leave ring slots free: start the next one's columns
        fill_ring(cl, cl_n);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint8_t *ch = chain(k);
            const float2 *beL = (const float2 *)(ch + Ly.beL);
            float *bsnap = (float *)(ch + Ly.bsnap);
            for (int f = lane; f < band_tot; f += 32) bsnap[f] = beL[f].x;
            float2 *vt2 = (float2 *)(ch + Ly.vt2);
            for (int q = lane; q < count; q += 32) vt2[q].y += A.inv_s2;
        }
        __syncwarp();
        if (status_seen != 0) {
            // another warp gave up: drain this warp's copies in flight and stop
            for (uint32_t q2 = seq; q2 < issued; ++q2) {
                uint32_t sp2 = 0;
                while (!mbar_try_wait(&bars[q2 & (kRing - 1)], (q2 / kRing) & 1u) && ++sp2 < kSpinLimit) {}
            }
            return;
        }

        // --- visit the pixels ------------------------------------------------
#pragma unroll 2
        for (int q = 0; q < count; ++q) {
            const uint32_t pq = pl[q];
            const int tc = (int)(pq & 0x1FFu);
            // the column that refills the slot this pixel frees (the ring
            // always has room for one once a column is consumed): the next
            // of the sequence, if its list is known; read now, off the
            // critical path
            const bool rf_any = issued - seq0 < (uint32_t)(count + count_n);
            uint2 rf = make_uint2(0u, 0u);
            if (rf_any) rf = list_entry(issued - seq0, cl, cl_n);
            if constexpr (K == 2) {
                // Two chains: half h (lanes 16h .. 16h+15) updates chain h
                // over the shared column, covering all its pairs; the control
                // flow, the column wait and refill and the reductions serve
                // both pixel updates.
                const int h = lane >> 4, hl = lane & 15;
                uint8_t *chh = chain(h);
                float *xth = (float *)(chh + Ly.xt);
                const float2 vq = ((const float2 *)(chh + Ly.vt2))[q];
                const float xs = xth[tc];
                const float d = xs - nb_half[tc];
                const float pbv = ((pq >> (9 + mbit)) & 1u) ? pb : 0.f;
                float pr2 = pbv * prior_weight(A, d);
                const float pr1 = pr2 * d;
                const float prox = fmaf(xs, A.inv_s2, -vq.x);   // (x - v) / sigma^2
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) pr2 += __shfl_xor_sync(FULL, pr2, o);
                pr2 = __shfl_sync(FULL, pr2, lane & 16);
                if (!wait_column()) return;
                const uint8_t *col = ring + (size_t)(seq & (kRing - 1)) * A.col_stride;
                const int nnz = *(const uint16_t *)col;
                const uint32_t *cidx2 = (const uint32_t *)(col + 4);
                const uint8_t *cval = col + col_idx_bytes(nnz);
                const int npairs = (nnz + 1) >> 1;
                const int lastp = max(npairs - 1, 0);
                constexpr int R2 = PR;   // rounds of 16 lanes
                uint32_t ib[R2];
                float2 av[R2];
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const int pe = r * 16 + hl;
                    const int pcl = min(pe, lastp);
                    const uint32_t i0 = cidx2[pcl];
                    const float2 a0 = ld_pair<T>(cval, pcl);
                    const bool ok = pe < npairs;
                    ib[r] = ok ? i0 : 0u;
                    av[r] = ok ? a0 : make_float2(0.f, 0.f);
                }
                float2 *beL = (float2 *)(chh + Ly.beL);
                float ex[R2][2], pa = 0.f, pc = 0.f;
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const float2 e0 = beL[ib[r] & 0xFFFFu], e1 = beL[ib[r] >> 16];
                    ex[r][0] = e0.x;
                    ex[r][1] = e1.x;
                    pa = fmaf(-av[r].x * e0.y, e0.x, pa);
                    pc = fmaf(-av[r].y * e1.y, e1.x, pc);
                }
                float p1 = (pa + pc) + pr1;
#pragma unroll
                for (int o = 8; o > 0; o >>= 1) p1 += __shfl_xor_sync(FULL, p1, o);
                // both halves have consumed the column: refill its slot
                ++seq;
                if (rf_any) {
                    if (lane == 0) issue(issued, col_src(rf), rf.y);
                    ++issued;
                }
                const float alpha = -(p1 + prox) * rcp_approx(vq.y + pr2);
                const int sink = A.max_band;
#pragma unroll
                for (int r = 0; r < R2; ++r) {
                    const int pe = r * 16 + hl;
                    const int d0 = pe < npairs ? (int)(ib[r] & 0xFFFFu) : sink;
                    const int d1 = 2 * pe + 1 < nnz ? (int)(ib[r] >> 16) : sink;
                    beL[d0].x = fmaf(-av[r].x, alpha, ex[r][0]);
                    beL[d1].x = fmaf(-av[r].y, alpha, ex[r][1]);
                }
                xth[tc] = xs + alpha;
                __syncwarp();
            } else {
            // prior through the surrogate weights (lane l: neighbour l), from
            // the X tiles only; its curvature is reduced here, before the
            // column is needed.  No branch: out-of-image neighbours and idle
            // lanes get weight 0.
            const float pbv = ((pq >> (9 + mbit)) & 1u) ? pb : 0.f;
            float xs[K], pr1[K], pr2[K], prox[K], t2[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float *xt = (const float *)(chain(k) + Ly.xt);
                const float2 vq = ((const float2 *)(chain(k) + Ly.vt2))[q];
                xs[k] = xt[tc];
                const float d = xs[k] - nbase[k][tc];
                pr2[k] = pbv * prior_weight(A, d);
                pr1[k] = pr2[k] * d;
                prox[k] = fmaf(xs[k], A.inv_s2, -vq.x);   // (x - v) / sigma^2
                t2[k] = vq.y;                             // theta2 + 1 / sigma^2
            }
#pragma unroll
            for (int o = 1; o < (NB26 ? 32 : 8); o <<= 1)
#pragma unroll
                for (int k = 0; k < K; ++k) pr2[k] += __shfl_xor_sync(FULL, pr2[k], o);
            if (!NB26) {
#pragma unroll
                for (int k = 0; k < K; ++k) pr2[k] = __shfl_sync(FULL, pr2[k], 0);
            }

            if (!wait_column()) return;
            const uint8_t *col = ring + (size_t)(seq & (kRing - 1)) * A.col_stride;
            const int nnz = *(const uint16_t *)col;
            const uint32_t *cidx2 = (const uint32_t *)(col + 4);
            const uint8_t *cval = col + col_idx_bytes(nnz);

            // data term of each chain: -sum A Lambda e in two interleaved
            // accumulators, plus the prior's gradient (lanes 0..7 / 0..25);
            // theta2 = sum A^2 Lambda is stored
            float alpha[K];
            if constexpr (PR > 0) {
                // pair loads without branches: lanes past the column's end
                // read its last pair (or pair 0 of an empty column, inside
                // the slot) and take (0, 0)
                const int npairs = (nnz + 1) >> 1;
                const int lastp = max(npairs - 1, 0);
                uint32_t ib[PR];
                float2 av[PR];
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int pe = r * 32 + lane;
                    const int pc = min(pe, lastp);
                    const uint32_t i0 = cidx2[pc];
                    const float2 a0 = ld_pair<T>(cval, pc);
                    const bool ok = pe < npairs;
                    ib[r] = ok ? i0 : 0u;
                    av[r] = ok ? a0 : make_float2(0.f, 0.f);
                }
                // pairs past the column's end are (0, 0) and add nothing;
                // every gather is issued back to back
                float ex[K][PR][2], pa[K], pc[K];
#pragma unroll
                for (int k = 0; k < K; ++k) { pa[k] = 0.f; pc[k] = 0.f; }
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int b0 = (int)(ib[r] & 0xFFFFu), b1 = (int)(ib[r] >> 16);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float2 *beL = (const float2 *)(chain(k) + Ly.beL);
                        const float2 e0 = beL[b0], e1 = beL[b1];
                        ex[k][r][0] = e0.x;
                        ex[k][r][1] = e1.x;
                        pa[k] = fmaf(-av[r].x * e0.y, e0.x, pa[k]);
                        pc[k] = fmaf(-av[r].y * e1.y, e1.x, pc[k]);
                    }
                }
                float p1[K];
#pragma unroll
                for (int k = 0; k < K; ++k) p1[k] = (pa[k] + pc[k]) + pr1[k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int k = 0; k < K; ++k) p1[k] += __shfl_xor_sync(FULL, p1[k], o);
                // Every lane's pairs have now been consumed (each loaded pair
                // feeds p1, and the full-warp reduction has joined all lanes),
                // so no read of the slot is outstanding: refill it now, before
                // the update.  Issuing right after the loads instead would let
                // a fast (L2-hit) copy overwrite the slot under reads still in
                // flight.
                ++seq;
                if (rf_any) {
                    if (lane == 0) issue(issued, col_src(rf), rf.y);
                    ++issued;
                }
                // the step's sign and zero set come from the numerator alone, so an
                // approximate reciprocal leaves the fixed point unchanged
#pragma unroll
                for (int k = 0; k < K; ++k) alpha[k] = -(p1[k] + prox[k]) * rcp_approx(t2[k] + pr2[k]);
                // update e: the entries of one column are distinct band positions;
                // stores past the column's end go to the sink entry (no branch)
                const int sink = A.max_band;
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int pe = r * 32 + lane;
                    const int d0 = pe < npairs ? (int)(ib[r] & 0xFFFFu) : sink;
                    const int d1 = 2 * pe + 1 < nnz ? (int)(ib[r] >> 16) : sink;
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float2 *beL = (float2 *)(chain(k) + Ly.beL);
                        beL[d0].x = fmaf(-av[r].x, alpha[k], ex[k][r][0]);
                        beL[d1].x = fmaf(-av[r].y, alpha[k], ex[k][r][1]);
                    }
                }
            } else {
                float2 *beL = (float2 *)(chain(0) + Ly.beL);
                float pa = 0.f, pc = 0.f;
                for (int pe = lane; 2 * pe < nnz; pe += 32) {
                    const uint32_t ib = cidx2[pe];
                    const float2 av = ld_pair<T>(cval, pe);
                    const float2 e0 = beL[ib & 0xFFFFu], e1 = beL[ib >> 16];
                    pa = fmaf(-av.x * e0.y, e0.x, pa);
                    pc = fmaf(-av.y * e1.y, e1.x, pc);
                }
                float p1 = (pa + pc) + pr1[0];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) p1 += __shfl_xor_sync(FULL, p1, o);
                alpha[0] = -(p1 + prox[0]) * rcp_approx(t2[0] + pr2[0]);
                for (int pe = lane; 2 * pe < nnz; pe += 32) {
                    const uint32_t ib = cidx2[pe];
                    const float2 av = ld_pair<T>(cval, pe);
                    const int b0 = (int)(ib & 0xFFFFu), b1 = (int)(ib >> 16);
                    beL[b0].x = fmaf(-av.x, alpha[0], beL[b0].x);
                    if (2 * pe + 1 < nnz) beL[b1].x = fmaf(-av.y, alpha[0], beL[b1].x);
                }
            }
            // X update: every lane holds alpha and stores the same value
#pragma unroll
            for (int k = 0; k < K; ++k) ((float *)(chain(k) + Ly.xt))[tc] = xs[k] + alpha[k];
            __syncwarp();
            if constexpr (PR == 0) {
                // the slot was read until the update above
                ++seq;
                if (rf_any) {
                    if (lane == 0) issue(issued, col_src(rf), rf.y);
                    ++issued;
                }
            }
            }
        }

        // --- write back: X tiles and the change of e --------------------------
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint8_t *ch = chain(k);
            const float *xt = (const float *)(ch + Ly.xt);
            float *Xg = Xk(k);
            for (int q = lane; q < S2; q += 32) {
                const int i = si * S + q / S, j = sj * S + q % S;
                if (i < A.ny && j < A.nx) Xg[(int64_t)i * A.nx + j] = xt[(q / S + 1) * TS + (q % S + 1)];
            }
            const float2 *beL = (const float2 *)(ch + Ly.beL);
            const float *bsnap = (const float *)(ch + Ly.bsnap);
            float2 *eL = eLk(k);
            for (int f = lane; f < band_tot; f += 32) {
                const float de = beL[f].x - bsnap[f];
                if (de != 0.f) atomicAdd(&eL[bglob[f]].x, de);
            }
        }
        __syncwarp();
        // hand the staged next-super-voxel state over; its successor's list
        // is built when it starts
        sv = sv_n;
        seq0 += count;
        count = count_n;
        count_n = 0;
        cur ^= 1;
    }
}

// Entries per column in rounds: one or four chains take pairs over 32 lanes
// (PR = ceil(max_nnz / 64) in {2, 3}; 0: any count, one chain); two chains
// take pairs over one 16-lane half (PR = ceil(max_nnz / 32) in {4, 5, 6}).
template <typename T, int S, bool CHAINS>
static sweep_fn sweep_lookup_s(int max_nnz, int K, bool nb26)
{
    const int r32 = (max_nnz + 63) / 64, r16 = (max_nnz + 31) / 32;
    if (nb26) {
        if (K != 1) return nullptr;
        if (r32 <= 2) return icd_sweep_kernel<T, 2, S, 1, true>;
        if (r32 <= 3) return icd_sweep_kernel<T, 3, S, 1, true>;
        return icd_sweep_kernel<T, 0, S, 1, true>;
    }
    if constexpr (CHAINS) {
        if (K == 2) {
            if (r16 <= 4) return icd_sweep_kernel<T, 4, S, 2, false>;
            if (r16 <= 5) return icd_sweep_kernel<T, 5, S, 2, false>;
            if (r16 <= 6) return icd_sweep_kernel<T, 6, S, 2, false>;
            return nullptr;
        }
        if (K == 4) {
            if (r32 <= 2) return icd_sweep_kernel<T, 2, S, 4, false>;
            if (r32 <= 3) return icd_sweep_kernel<T, 3, S, 4, false>;
            return nullptr;
        }
    }
    if (K != 1) return nullptr;
    if (r32 <= 2) return icd_sweep_kernel<T, 2, S, 1, false>;
    if (r32 <= 3) return icd_sweep_kernel<T, 3, S, 1, false>;
    return icd_sweep_kernel<T, 0, S, 1, false>;
}

// The sweep kernel for columns of at most max_nnz entries, super-voxel size
// S, K chains and the 8- or 26-neighbourhood; nullptr if that combination is
// not built.
template <typename T>
static sweep_fn sweep_lookup(int max_nnz, int S, int K, bool nb26)
{
    switch (S) {
    case 4: return sweep_lookup_s<T, 4, true>(max_nnz, K, nb26);
    case 8: return sweep_lookup_s<T, 8, true>(max_nnz, K, nb26);
    case 16: return sweep_lookup_s<T, 16, false>(max_nnz, K, nb26);
    default: return nullptr;
    }
}

__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f32(int max_nnz, int S, int K, bool nb26);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_bf16(int max_nnz, int S, int K, bool nb26);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f16(int max_nnz, int S, int K, bool nb26);
