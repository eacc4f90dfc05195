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
    float inv_sx2, inv_Tsx, qexp, qq;   // prior constants
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
//   boff:   max_views * 2                 band offset of each view (u16)
//   bview:  max_band * 2                  view of each band entry (u16)
//   coff:   2 * (S^2 + 1) * 4             column byte offsets, current and next super-voxel
//   tl:     2 * S^2 * 2                   non-empty pixels in visiting order, current and next
//   halo:   2 * (S+2)^2 * 4               X tiles of the slices below and above (volumes only)
// and per chain:
//   beL:    max_band * 8                  (e, Lambda) of the band, e kept current
//   bsnap:  max_band * 4                  e of the band when the super-voxel began
//   xt:     (S+2)^2 * 4                   X tile with one-pixel halo
//   vt:     S^2 * 4                       v tile
//   t2t:    S^2 * 4                       theta2 tile (data term of the coordinate curvature)
struct WarpSmem {
    size_t ring, bars, bdesc, boff, bview, coff, tl, halo, chain0, chain_size;
    size_t beL, bsnap, xt, vt, t2t;
    size_t total;
};

__host__ __device__ inline WarpSmem warp_smem_layout(int max_band, int col_stride, int S, int max_views, int K,
                                                     int halo)
{
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t S2 = (size_t)S * S, TA = (size_t)(S + 2) * (S + 2);
    WarpSmem L;
    size_t o = 0;
    L.ring = o;  o += r16((size_t)kRing * col_stride);
    L.bars = o;  o += r16(kRing * 8);
    L.bdesc = o; o += r16((size_t)2 * max_views * 4);
    L.boff = o;  o += r16((size_t)max_views * 2);
    L.bview = o; o += r16((size_t)max_band * 2);
    L.coff = o;  o += r16((size_t)2 * (S2 + 1) * 4);
    L.tl = o;    o += r16((size_t)2 * S2 * 2);
    L.halo = o;  o += halo ? r16(2 * TA * 4) : 0;
    L.chain0 = o;
    size_t c = 0;
    L.beL = c;   c += r16((size_t)max_band * 8);
    L.bsnap = c; c += r16((size_t)max_band * 4);
    L.xt = c;    c += r16(TA * 4);
    L.vt = c;    c += r16(S2 * 4);
    L.t2t = c;   c += r16(S2 * 4);
    L.chain_size = c;
    L.total = o + (size_t)K * c;
    return L;
}

// Surrogate weight rho'(D)/D of the prior potential (quadratic: 1/sigma_x^2;
// Q-GGMRF with p = 2: (2 + q a) / (2 sigma_x^2 (1 + a)^2), a = |D/(T sigma_x)|^(p-q)).
// It scales the prior's gradient, so its rounding moves the fixed point by
// a relative amount of the order of FP32 rounding only.
__device__ __forceinline__ float prior_weight(const SweepArgs &A, float d)
{
    if (A.prior == 0) return A.inv_sx2;
    const float a = __powf(fabsf(d * A.inv_Tsx), A.qexp);
    const float opa = 1.f + a;
    return __fdividef((2.f + A.qq * a) * 0.5f * A.inv_sx2, opa * opa);
}

// One warp runs K chains (reconstructions b0 .. b0+K-1 of one batch group,
// all on agent g) over a fixed sequence of super-voxels: slots c, c+C, c+2C,
// ... of the visiting order, where C warps serve the same (group, agent) -- so
// about C super-voxels of one agent of one reconstruction are in flight at a
// time.  Inside a super-voxel the pixels are visited in order; each pixel's
// column (a flat list of (band position, value) pairs, lane k taking the
// pairs k, k+32, ...) is streamed once by TMA for all K chains.  The next
// super-voxel's metadata and first columns are fetched while the current one
// is processed.  PR > 0: at most 64*PR entries per column, kept in registers
// between the reduction and the update, and the ring slot is refilled once
// they have been consumed; PR == 0: any count (K must be 1).
template <typename T, int PR, int S, int K>
__global__ void __launch_bounds__(256, 1) icd_sweep_kernel(SweepArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    constexpr int S2 = S * S, TS = S + 2, TA = TS * TS;
    static_assert(PR > 0 || K == 1, "uncached columns support one chain");
    static_assert((kRing & (kRing - 1)) == 0, "ring size is a power of two");
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const WarpSmem Ly = warp_smem_layout(A.max_band, A.col_stride, S, A.max_views, K, A.nb26);
    uint8_t *base = smem + wib * Ly.total;
    uint8_t *ring = base + Ly.ring;
    uint64_t *bars = (uint64_t *)(base + Ly.bars);
    uint32_t *bdesc2 = (uint32_t *)(base + Ly.bdesc);
    uint16_t *boff = (uint16_t *)(base + Ly.boff);
    uint16_t *bview = (uint16_t *)(base + Ly.bview);
    uint32_t *scoff2 = (uint32_t *)(base + Ly.coff);
    uint16_t *tl2 = (uint16_t *)(base + Ly.tl);
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
    // this lane's prior neighbour: lanes 0..7 the in-plane 8-neighbourhood,
    // or (volumes) lanes 0..25 the 26-neighbourhood
    int pdz = 0, pdi, pdj;
    float pb;
    if (A.nb26) {
        const int kk = lane < 13 ? lane : lane + 1;   // skip the centre of the 3x3x3
        pdz = kk / 9 - 1;
        pdi = (kk / 3) % 3 - 1;
        pdj = kk % 3 - 1;
        const int d2 = pdz * pdz + pdi * pdi + pdj * pdj;
        pb = lane < 26 ? A.pscale * A.b26[d2 - 1] : 0.f;
    } else {
        const int kk = lane < 4 ? lane : lane + 1;
        pdi = kk / 3 - 1;
        pdj = kk % 3 - 1;
        pb = lane < 8 ? A.pscale * ((pdi != 0 && pdj != 0) ? A.b_diag : A.b_edge) : 0.f;
    }
    const int nlanes = A.nb26 ? 26 : 8;
    const int zc = grp * K;   // slice of chain 0 (volumes run one chain per warp)
    const bool z_in = pdz == 0 || (zc + pdz >= 0 && zc + pdz < A.B);

    // chain k: reconstruction grp*K + k
    auto eLk = [&](int k) { return A.eL + (int64_t)(grp * K + k) * A.ne + (int64_t)v0 * A.D; };
    auto Xk = [&](int k) { return A.X + ((int64_t)(grp * K + k) * A.N + g) * n; };
    auto chain = [&](int k) { return chains + (size_t)k * Ly.chain_size; };

    // --- super-voxel metadata -------------------------------------------
    auto sv_of = [&](int m) {           // m-th super-voxel of this warp, -1 past the end
        const int slot = cidx + m * Cw;
        if (slot >= A.nsv) return -1;
        return A.sv_order[A.backward ? A.nsv - 1 - slot : slot];
    };
    // visiting list of a super-voxel from its column offsets; returns count
    auto build_list = [&](const uint32_t *sc, uint16_t *tl) {
        int count = 0;
        for (int k0 = 0; k0 < S2; k0 += 32) {
            const int k = k0 + lane;
            const int t = A.backward ? S2 - 1 - k : k;
            const bool ne = k < S2 && sc[t + 1] != sc[t];
            const unsigned m = __ballot_sync(FULL, ne);
            if (ne) tl[count + __popc(m & lt_mask)] = (uint16_t)t;
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
        for (int k = lane; k <= S2; k += 32) scoff2[k] = coff[k];
        const uint32_t *bd = A.band + (int64_t)A.nsv * v0 + (int64_t)sv * Vg;
        for (int v = lane; v < Vg; v += 32) bdesc2[v] = bd[v];
        __syncwarp();
    }
    int count = build_list(scoff2, tl2);
    const uint8_t *svcols = A.cols + A.sv_base[(int64_t)g * A.nsv + sv];
    uint32_t issued = 0, seq = 0;     // ring positions issued / consumed (per warp)
    if (lane == 0)
        for (int q = 0; q < min(count, kRing); ++q) {
            const int t = tl2[q];
            issue(issued + q, svcols + scoff2[t], scoff2[t + 1] - scoff2[t]);
        }
    issued += min(count, kRing);
    int cur = 0;
    int status_seen = 0;

    for (int m = 0; sv >= 0; ++m) {
        uint32_t *bdesc = bdesc2 + cur * A.max_views;
        uint32_t *scoff = scoff2 + cur * (S2 + 1);
        uint16_t *tl = tl2 + cur * S2;
        uint32_t *bdesc_n = bdesc2 + (cur ^ 1) * A.max_views;
        uint32_t *scoff_n = scoff2 + (cur ^ 1) * (S2 + 1);
        uint16_t *tl_n = tl2 + (cur ^ 1) * S2;
        const int si = sv / A.nsvx, sj = sv - si * A.nsvx;

        // --- band layout; band, X and theta2 tiles of every chain -----------
        const int band_tot = load_band_layout(bdesc, Vg, bdesc, boff, bview, lane);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint8_t *ch = chain(k);
            float2 *beL = (float2 *)(ch + Ly.beL);
            float *xt = (float *)(ch + Ly.xt);
            float *t2t = (float *)(ch + Ly.t2t);
            const float2 *eL = eLk(k);
            for (int f = lane; f < band_tot; f += 32) cp_async8(&beL[f], &eL[band_global(f, bdesc, boff, bview, A.D)]);
            const float *Xg = Xk(k);
            for (int q = lane; q < TA; q += 32) {
                const int i = si * S + q / TS - 1, j = sj * S + q % TS - 1;
                if (i >= 0 && i < A.ny && j >= 0 && j < A.nx) cp_async4(&xt[q], &Xg[(int64_t)i * A.nx + j]);
                else xt[q] = 0.f;
            }
            const float *t2g = A.theta2 + ((int64_t)(grp * K + k) * A.N + g) * n;
            for (int q = lane; q < S2; q += 32) {
                const int i = si * S + q / S, j = sj * S + q % S;
                if (i < A.ny && j < A.nx) cp_async4(&t2t[q], &t2g[(int64_t)i * A.nx + j]);
            }
        }
        if (A.nb26) {
            // X tiles of the neighbouring slices
            for (int h = 0; h < 2; ++h) {
                const int zz = zc + (h ? 1 : -1);
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
        const uint8_t *svcols_n = nullptr;
        if (sv_n >= 0) {
            svcols_n = A.cols + A.sv_base[(int64_t)g * A.nsv + sv_n];
            const uint32_t *coff = A.col_off + ((int64_t)g * A.nsv + sv_n) * (S2 + 1);
            for (int k = lane; k <= S2; k += 32) cp_async4(&scoff_n[k], &coff[k]);
            const uint32_t *bd = A.band + (int64_t)A.nsv * v0 + (int64_t)sv_n * Vg;
            for (int v = lane; v < Vg; v += 32) cp_async4(&bdesc_n[v], &bd[v]);
        }
        cp_async_commit();
        // v tile (v = 2 wbar - w, FP64 consensus; or the caller's v) with
        // plain loads while the copies above are in flight
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float *vt = (float *)(chain(k) + Ly.vt);
            const int64_t rb = (int64_t)(grp * K + k);
            for (int q = lane; q < S2; q += 32) {
                const int i = si * S + q / S, j = sj * S + q % S;
                float vv = 0.f;
                if (i < A.ny && j < A.nx) {
                    const int64_t s = (int64_t)i * A.nx + j;
                    vv = A.vexp ? A.vexp[(rb * A.N + g) * n + s]
                                : (float)(2.0 * A.wbar[rb * n + s] - (double)A.w[(rb * A.N + g) * n + s]);
                }
                vt[q] = vv;
            }
        }
        if (lane == 0) status_seen = *((volatile int *)A.status);
        cp_async_wait_all();
        __syncwarp();
        status_seen = __shfl_sync(FULL, status_seen, 0);
        int count_n = 0;
        if (sv_n >= 0) count_n = build_list(scoff_n, tl_n);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint8_t *ch = chain(k);
            const float2 *beL = (const float2 *)(ch + Ly.beL);
            float *bsnap = (float *)(ch + Ly.bsnap);
            for (int f = lane; f < band_tot; f += 32) bsnap[f] = beL[f].x;
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
        int nq = 0;   // columns of the next super-voxel issued so far
        for (int q = 0; q < count; ++q) {
            const int t = tl[q];
            const int ti = t / S, tj = t % S;
            const int i = si * S + ti, j = sj * S + tj;
            const int tc = (ti + 1) * TS + (tj + 1);
            // the column that refills the slot this pixel frees: column
            // q + kRing of this super-voxel, else the next one of the next
            // super-voxel (offsets read now, off the critical path)
            const bool rf_cur = q + kRing < count;
            const bool rf_any = rf_cur || nq < count_n;
            const uint8_t *rf_src = nullptr;
            uint32_t rf_bytes = 0;
            if (rf_any) {
                const int rt = rf_cur ? tl[q + kRing] : tl_n[nq];
                const uint32_t *rsc = rf_cur ? scoff : scoff_n;
                const uint32_t lo = rsc[rt];
                rf_bytes = rsc[rt + 1] - lo;
                rf_src = (rf_cur ? svcols : svcols_n) + lo;
            }
            // prior through the surrogate weights (lane l: neighbour l), from
            // the X tiles only; its curvature is reduced here, before the
            // column is needed
            float xs[K], pr1[K], pr2[K], prox[K], t2[K];
            const bool nb_in = lane < nlanes && z_in && i + pdi >= 0 && i + pdi < A.ny && j + pdj >= 0 &&
                               j + pdj < A.nx;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                const float *xt = (const float *)(chain(k) + Ly.xt);
                xs[k] = xt[tc];
                pr1[k] = 0.f;
                pr2[k] = 0.f;
                if (nb_in) {
                    const float *nt = pdz == 0 ? xt : (pdz < 0 ? halo_lo : halo_hi);
                    const float d = xs[k] - nt[tc + pdi * TS + pdj];
                    pr2[k] = pb * prior_weight(A, d);
                    pr1[k] = pr2[k] * d;
                }
                prox[k] = (xs[k] - ((const float *)(chain(k) + Ly.vt))[t]) * A.inv_s2;
                t2[k] = ((const float *)(chain(k) + Ly.t2t))[t];
            }
#pragma unroll
            for (int o = 1; o < 8; o <<= 1)
#pragma unroll
                for (int k = 0; k < K; ++k) pr2[k] += __shfl_xor_sync(FULL, pr2[k], o);
            if (A.nb26) {
#pragma unroll
                for (int o = 8; o < 32; o <<= 1)
#pragma unroll
                    for (int k = 0; k < K; ++k) pr2[k] += __shfl_xor_sync(FULL, pr2[k], o);
            } else {
#pragma unroll
                for (int k = 0; k < K; ++k) pr2[k] = __shfl_sync(FULL, pr2[k], 0);
            }

            const uint32_t stg = seq & (kRing - 1);
            const uint32_t parity = (seq / kRing) & 1u;
            uint32_t spins = 0;
            while (!mbar_try_wait(&bars[stg], parity)) {
                if (++spins > kSpinLimit) {
                    // give up: flag the host, then wait (bounded) for this
                    // warp's copies still in flight before leaving
                    if (lane == 0) atomicExch(A.status, kStatusTimeout);
                    for (uint32_t q2 = seq + 1; q2 < issued; ++q2) {
                        uint32_t sp2 = 0;
                        while (!mbar_try_wait(&bars[q2 & (kRing - 1)], (q2 / kRing) & 1u) && ++sp2 < kSpinLimit) {}
                    }
                    return;
                }
            }
            const uint8_t *col = ring + (size_t)stg * A.col_stride;
            const int nnz = *(const uint16_t *)col;
            const uint32_t *cidx2 = (const uint32_t *)(col + 4);
            const uint8_t *cval = col + col_idx_bytes(nnz);

            // data term of each chain: p1 = -sum A Lambda e (+ the prior's
            // gradient in lanes 0..7 / 0..25); theta2 = sum A^2 Lambda is stored
            float p1[K];
#pragma unroll
            for (int k = 0; k < K; ++k) p1[k] = pr1[k];
            float alpha[K];
            if constexpr (PR > 0) {
                uint32_t ib[PR];
                float2 av[PR];
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int pe = r * 32 + lane;
                    ib[r] = 0u;
                    av[r] = make_float2(0.f, 0.f);
                    if (2 * pe < nnz) {
                        ib[r] = cidx2[pe];
                        av[r] = ld_pair<T>(cval, pe);
                    }
                }
                float ex[K][PR][2];
                // no branch per round: pairs past the column's end are (0, 0)
                // and add nothing, and every gather is issued back to back
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int b0 = (int)(ib[r] & 0xFFFFu), b1 = (int)(ib[r] >> 16);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        const float2 *beL = (const float2 *)(chain(k) + Ly.beL);
                        const float2 e0 = beL[b0], e1 = beL[b1];
                        ex[k][r][0] = e0.x;
                        ex[k][r][1] = e1.x;
                        p1[k] = fmaf(-av[r].x * e0.y, e0.x, p1[k]);
                        p1[k] = fmaf(-av[r].y * e1.y, e1.x, p1[k]);
                    }
                }
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
                    if (lane == 0) issue(issued, rf_src, rf_bytes);
                    ++issued;
                    if (!rf_cur) ++nq;
                }
                // the step's sign and zero set come from the numerator alone, so a
                // fast division leaves the fixed point unchanged
#pragma unroll
                for (int k = 0; k < K; ++k) alpha[k] = -__fdividef(p1[k] + prox[k], t2[k] + pr2[k] + A.inv_s2);
                // update e: the entries of one column are distinct band positions
#pragma unroll
                for (int r = 0; r < PR; ++r) {
                    const int pe = r * 32 + lane;
                    const int b0 = (int)(ib[r] & 0xFFFFu), b1 = (int)(ib[r] >> 16);
#pragma unroll
                    for (int k = 0; k < K; ++k) {
                        float2 *beL = (float2 *)(chain(k) + Ly.beL);
                        if (2 * pe < nnz) beL[b0].x = fmaf(-av[r].x, alpha[k], ex[k][r][0]);
                        if (2 * pe + 1 < nnz) beL[b1].x = fmaf(-av[r].y, alpha[k], ex[k][r][1]);
                    }
                }
            } else {
                float2 *beL = (float2 *)(chain(0) + Ly.beL);
                for (int pe = lane; 2 * pe < nnz; pe += 32) {
                    const uint32_t ib = cidx2[pe];
                    const float2 av = ld_pair<T>(cval, pe);
                    const float2 e0 = beL[ib & 0xFFFFu], e1 = beL[ib >> 16];
                    p1[0] = fmaf(-av.x * e0.y, e0.x, p1[0]);
                    p1[0] = fmaf(-av.y * e1.y, e1.x, p1[0]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) p1[0] += __shfl_xor_sync(FULL, p1[0], o);
                alpha[0] = -__fdividef(p1[0] + prox[0], t2[0] + pr2[0] + A.inv_s2);
                for (int pe = lane; 2 * pe < nnz; pe += 32) {
                    const uint32_t ib = cidx2[pe];
                    const float2 av = ld_pair<T>(cval, pe);
                    const int b0 = (int)(ib & 0xFFFFu), b1 = (int)(ib >> 16);
                    beL[b0].x = fmaf(-av.x, alpha[0], beL[b0].x);
                    if (2 * pe + 1 < nnz) beL[b1].x = fmaf(-av.y, alpha[0], beL[b1].x);
                }
            }
            if (lane == 0) {
#pragma unroll
                for (int k = 0; k < K; ++k) ((float *)(chain(k) + Ly.xt))[tc] = xs[k] + alpha[k];
            }
            __syncwarp();
            if constexpr (PR == 0) {
                // the slot was read until the update above
                ++seq;
                if (rf_any) {
                    if (lane == 0) issue(issued, rf_src, rf_bytes);
                    ++issued;
                    if (!rf_cur) ++nq;
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
                if (de != 0.f) atomicAdd(&eL[band_global(f, bdesc, boff, bview, A.D)].x, de);
            }
        }
        __syncwarp();
        // the next super-voxel's first columns: those not issued yet
        if (sv_n >= 0) {
            while (nq < min(count_n, kRing) && (int)(issued - seq) < kRing) {
                if (lane == 0) {
                    const int t = tl_n[nq];
                    issue(issued, svcols_n + scoff_n[t], scoff_n[t + 1] - scoff_n[t]);
                }
                ++issued;
                ++nq;
            }
        }
        // hand the staged next-super-voxel state over
        sv = sv_n;
        svcols = svcols_n;
        count = count_n;
        cur ^= 1;
        // now exactly min(count, kRing) columns of the new super-voxel are in
        // flight, as the pixel loop's refill (column q + kRing) assumes
    }
}

template <typename T, int S>
static sweep_fn sweep_lookup_s(int pair_rounds, int K)
{
    if (pair_rounds <= 2)
        return K == 4 ? icd_sweep_kernel<T, 2, S, 4> : K == 2 ? icd_sweep_kernel<T, 2, S, 2> : icd_sweep_kernel<T, 2, S, 1>;
    if (pair_rounds <= 3)
        return K == 4 ? icd_sweep_kernel<T, 3, S, 4> : K == 2 ? icd_sweep_kernel<T, 3, S, 2> : icd_sweep_kernel<T, 3, S, 1>;
    return K == 1 ? icd_sweep_kernel<T, 0, S, 1> : nullptr;
}

// The sweep kernel for columns of at most 64 * pair_rounds entries (any
// count when pair_rounds > 3, one chain), super-voxel size S and K chains;
// nullptr if that combination is not built.
template <typename T>
static sweep_fn sweep_lookup(int pair_rounds, int S, int K)
{
    switch (S) {
    case 4: return sweep_lookup_s<T, 4>(pair_rounds, K);
    case 8: return sweep_lookup_s<T, 8>(pair_rounds, K);
    case 16: return K == 1 ? sweep_lookup_s<T, 16>(pair_rounds, 1) : nullptr;
    default: return nullptr;
    }
}

__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f32(int pair_rounds, int S, int K);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_bf16(int pair_rounds, int S, int K);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f16(int pair_rounds, int S, int K);
