// The ICD sweep of partial-update MACE: one pass of Algorithm 2 (iterative
// coordinate descent for the proximal map F_i(v_i; sigma), Eq. "ICDUpdate1")
// for every agent of every reconstruction of a batch, over the stored system
// matrix.  Instantiated per stored value type in sweep_<type>.cu.
//
// Work decomposition.  C warps serve each (batch group, agent) pair and stay
// resident; warp c takes the super-voxels c, c+C, c+2C, ... of the visiting
// order, so about C super-voxels of one agent are in flight.  A warp runs K
// chains: K reconstructions of the batch that share every column load (K = 2:
// two 16-lane halves, one per reconstruction).  Inside a chain, lane l owns
// the agent's views l, l + 32/K, l + 64/K, ...: for each pixel it reads its
// views' runs from the column (one header byte and the first two values per
// view), gathers their (e, Lambda) band entries, and after the step writes
// them back; the third values of three-channel runs form a short list that
// the lanes share.
//
// The super-voxel's band of (e, Lambda) lives in shared memory as rows t of
// vpad views, chains interleaved: entry (t, v) of chain k at float2 index
// (t vpad + v) K + k.  Lanes of one round touch views 16 apart in bank space,
// so a gather is conflict-free whatever the runs' offsets.  Columns stream in
// through a per-warp ring of TMA bulk copies; each column is decoded into
// registers one pixel ahead, so its slot is refilled at once and the next
// pixel's gathers only wait for the current pixel's update.
#pragma once

#include "common.cuh"

struct SweepArgs {
    const uint8_t *cols;
    const int64_t *sv_base;
    const uint32_t *col_off;
    const uint32_t *band;
    const int *view_off;
    const int32_t *sv_order;
    float2 *eL;                 // [B][V][D] (e, Lambda): error sinogram and weights
    float *X;
    const float *w;
    const double *wbar;
    const float *vexp;
    const float *theta2;        // [B][N][n]: sum over the agent's views of A_js^2 Lambda_j
    int *status;
    int B, N, nsv, nsvx, nx, ny, D, S;
    int64_t ne;
    int nwarps;                 // warps with work (the last block may have idle ones)
    int backward;
    int vpad, wmax, col_stride;
    float inv_s2, pscale;
    float inv_sx2, inv_Tsx, qexp, half_q_inv_sx2;   // prior constants (quadratic: inv_Tsx = 0)
    float b_edge, b_diag;       // 8-neighbourhood weights (face, diagonal)
    float b26[3];               // 26-neighbourhood weights by squared distance 1, 2, 3
    // deterministic mode: the C warps of a (group, agent) pair run their
    // super-voxels in lock-step phases (counter per pair, zero at launch);
    // changes of e go to the fixed-point accumulator, e is read as e + dacc
    unsigned *phase;
    unsigned long long *dacc;   // [B][V][D]
};

// Phase counter of a (group, agent) pair: every warp adds 1 when it has read
// a phase's state and 1 when it has written its changes.  Waits are bounded;
// on expiry they return false (the caller flags the host and leaves).
__device__ __forceinline__ void phase_arrive(unsigned *c)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c) : "memory");
}
__device__ __forceinline__ bool phase_wait(unsigned *c, unsigned target)
{
    uint32_t spins = 0;
    for (;;) {
        unsigned v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(c) : "memory");
        if ((int)(v - target) >= 0) return true;
        if (++spins > kSpinLimit) return false;
        __nanosleep(64);
    }
}

typedef void (*sweep_fn)(SweepArgs);

// Per-warp shared-memory layout (bytes, each part 16-aligned):
//   ring:   kRing * col_stride          column staging (TMA destination)
//   bars:   kRing * 8                   mbarriers
//   bdesc:  2 * vpad * 4                band descriptors (lo | len << 16), current and next super-voxel
//   coff:   (S^2 + 1) * 4               column byte offsets of the next super-voxel (staging)
//   pl:     2 * S^2 * 4                 per visited pixel: tile index | neighbour mask << 11
//                                       | pixel offset in the super-voxel << 20
//   cl:     2 * S^2 * 8                 per visited pixel: (column offset in 16-byte units, bytes)
//   halo:   2 K (S+2)^2 * 4             per chain, X tiles of the slices below and above (volumes only)
//   band:   (wmax bw K + 1) * 8         (e, Lambda), chains interleaved; the last entry is a
//                                       sink that idle lanes read and write with value 0
//   snap:   K wmax bw * 4               e of the band when the super-voxel began
//   xt:     K (S+2)^2 * 4               X tiles with a one-pixel halo
//   vt2:    K S^2 * 8                   per visited pixel (v / sigma^2, theta2 + 1 / sigma^2)
//   xch:    32                          a team's exchange slots (partial sums, flags, work items)
// bw: band row width, vpad for one warp per voxel; with W warps per voxel a
// warp keeps only its own views' entries, 32 ceil(vpad / 32 W) of them.
struct WarpSmem {
    size_t ring, bars, bdesc, coff, pl, cl, halo, band, snap, xt, vt2, xch;
    size_t total;
};

__host__ __device__ inline int band_width(int vpad, int W)
{
    return W == 1 ? vpad : 32 * ((vpad + 32 * W - 1) / (32 * W));
}

__host__ __device__ inline WarpSmem warp_smem_layout(int vpad, int wmax, int col_stride, int S, int K, bool halo,
                                                     int W = 1)
{
    const int bw = band_width(vpad, W);
    auto r16 = [](size_t b) { return (b + 15) & ~(size_t)15; };
    const size_t S2 = (size_t)S * S, TA = (size_t)(S + 2) * (S + 2);
    WarpSmem L;
    size_t o = 0;
    L.ring = o;  o += r16((size_t)kRing * col_stride);
    L.bars = o;  o += r16(kRing * 8);
    L.bdesc = o; o += r16((size_t)2 * vpad * 4);
    L.coff = o;  o += r16((S2 + 1) * 4);
    L.pl = o;    o += r16(2 * S2 * 4);
    L.cl = o;    o += r16(2 * S2 * 8);
    L.halo = o;  o += halo ? r16((size_t)2 * K * TA * 4) : 0;
    L.band = o;  o += r16(((size_t)wmax * bw * K + 1) * 8);
    L.snap = o;  o += r16((size_t)K * wmax * bw * 4);
    L.xt = o;    o += r16((size_t)K * TA * 4);
    L.vt2 = o;   o += r16((size_t)K * S2 * 8);
    L.xch = o;   o += 32;
    L.total = o;
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

// Surrogate weight rho'(D)/D of the prior potential (Q-GGMRF with p = 2:
// (2 + q a) / (2 sigma_x^2 (1 + a)^2), a = |D/(T sigma_x)|^(p-q), the power
// taken as 2^((p-q) log2 |D/(T sigma_x)|), a = 0 at D = 0).  Branch-free:
// the quadratic prior (weight 1/sigma_x^2) runs the same arithmetic with
// inv_Tsx = 0, so a = 0.
__device__ __forceinline__ float prior_weight(const SweepArgs &A, float d)
{
    const float a = ex2_approx(A.qexp * lg2_approx(fabsf(d * A.inv_Tsx)));
    const float r = rcp_approx(1.f + a);
    return fmaf(A.half_q_inv_sx2, a, A.inv_sx2) * r * r;
}

__device__ __forceinline__ float2 lds_f2(uint32_t a)
{
    float2 v;
    asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(a) : "memory");
    return v;
}
__device__ __forceinline__ void sts_f(uint32_t a, float v)
{
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

// One column decoded for one lane: for each owned view j the shared address
// of its run's first band entry (the second is one band row further) and
// the two values; for each share of the three-channel list the address and
// value of its third entry.  Idle lanes carry value 0: a share points at
// the sink, a view at entry (wmax - 1, 0) of chain 0, whose next row is the
// sink.  Row wmax - 1 holds no channel of any view (wmax is the widest band
// plus one), so every write there stores back the value read.
template <int R, int RO>
struct ColRegs {
    uint32_t addr[R];
    float a0[R], a1[R];
    uint32_t oaddr[RO];
    float a2[RO];
};
// The raw words of a column as read from its ring slot, before decoding.
template <int R, int RO>
struct ColRaw {
    uint32_t hb[R];
    float2 a[R];
    uint32_t code[RO];
    float a2[RO];
    int n3;
};

// Register cap: 128 keeps 16 warps per SM (shared memory allows about as
// many on the benchmark's configuration) without spills.
#ifndef MACE_SWEEP_MAXNREG
#define MACE_SWEEP_MAXNREG 128
#endif

// A team of W warps of one block sweeping the same super-voxels, the
// agent's views split between them (warp wi owns views 32 (wi + W j) + lane):
// each warp keeps its own views' band, the partial sums of a pixel's theta1
// are added in a fixed order through shared memory, so every warp of the
// team computes the same step and the same X tile.  xch0: shared address of
// the team's first warp's exchange slots; stride: bytes between the warps'
// regions; bar: the team's named barrier (1 + team index in the block).
struct TeamCtx {
    int wi, bar;
    uint32_t xch0, stride;
};

__device__ __forceinline__ void sts_u32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void team_barrier(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Per-warp set-up shared by the launches: ring barriers, and the band at
// zero (entries outside a super-voxel's band are only ever read and written
// with matrix value 0, so they stay finite whatever a previous super-voxel
// left there).
__device__ __forceinline__ void sweep_warp_init(uint8_t *base, const WarpSmem &Ly, int nband, int lane)
{
    uint64_t *bars = (uint64_t *)(base + Ly.bars);
    float2 *band = (float2 *)(base + Ly.band);
    if (lane == 0)
        for (int k = 0; k < kRing; ++k) mbar_init(&bars[k], 1);
    for (int f = lane; f <= nband; f += 32) band[f] = make_float2(0.f, 0.f);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();
}

// R: rounds of views per lane (R * 32/K >= the agent's views); RO: rounds of
// the three-channel list (RO * 32/K >= its longest).  NB26: the batch is the
// z-stack of one volume, 26-neighbourhood prior (with K = 2 each lane of a
// chain takes two of the 26 neighbours).  DET: deterministic mode (lock-step
// phases, fixed-point changes of e).  W: warps per super-voxel (a team).
// grp: the warp's (group, agent) pair is grp N + g; chain k updates
// reconstruction (slice) rbase + k rstride (rstride 2: two slices of one
// z parity).
template <typename T, int K, int R, int RO, bool NB26, bool DET, int W, class ARGS>
__device__ __forceinline__ bool sweep_work(ARGS A, uint8_t *base, const WarpSmem &Ly, const int grp, const int g,
                                           const int cidx, const int Cw, uint32_t &dec, uint32_t &issued,
                                           const TeamCtx &tm, const int rbase, const int rstride)
{
    static_assert(K == 1 || K == 2, "one or two chains per warp");
    static_assert(W == 1 || (W == 2 || W == 4) && K == 1 && R == 0 && !DET && !NB26,
                  "teams of 2 or 4 warps run the 2D decode-at-use sweep, one chain, free mode");
    static_assert((kRing & (kRing - 1)) == 0 && kRing >= 3, "ring size is a power of two >= 4");
    constexpr int LPC = 32 / K;                 // lanes per chain
    constexpr int LPCV = LPC * W;               // stride between a lane's views
    // R = 0: any number of views, each column decoded from its ring slot at
    // use (RR, RRO size the prefetch registers of the R > 0 kernels)
    constexpr int RR = R > 0 ? R : 1, RRO = RO > 0 ? RO : 1;
    constexpr int vb = (int)sizeof(T);
    const int S = A.S, S2 = S * S, TS = S + 2, TA = TS * TS;
    const int lS = 31 - __clz(S);               // S is a power of two
    const int lane = threadIdx.x & 31;
    uint8_t *ring = base + Ly.ring;
    uint64_t *bars = (uint64_t *)(base + Ly.bars);
    uint32_t *bdesc2 = (uint32_t *)(base + Ly.bdesc);
    uint32_t *scoff = (uint32_t *)(base + Ly.coff);
    uint32_t *pl2 = (uint32_t *)(base + Ly.pl);
    uint2 *cl2 = (uint2 *)(base + Ly.cl);
    float *const halo0 = (float *)(base + Ly.halo);   // chain k: below at 2k TA, above at (2k + 1) TA
    float2 *band = (float2 *)(base + Ly.band);
    float *snap = (float *)(base + Ly.snap);
    float *xt0 = (float *)(base + Ly.xt);
    float2 *vt20 = (float2 *)(base + Ly.vt2);

    const int vpad = A.vpad, wmax = A.wmax;
    const int bw = band_width(vpad, W);         // band row width (this warp's views)
    const int nrow = wmax * bw;                 // band entries of one chain
    const unsigned FULL = 0xffffffffu;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t n = (int64_t)A.nx * A.ny;
    const int pair = grp * A.N + g;             // (group, agent)
    const int v0 = A.view_off[g], Vg = A.view_off[g + 1] - v0;

    // lane roles in the pixel loop: chain h, index hl inside the chain's lanes
    const int h = K == 2 ? (lane >> 4) : 0;
    const int hl = K == 2 ? (lane & 15) : lane;
    const int hl_v = (W > 1 ? tm.wi * LPC : 0) + hl;     // this lane's first view
    const uint32_t band_s = smem_u32(band);
    const uint32_t sink_s = band_s + (uint32_t)nrow * K * 8u;
    const uint32_t tstr = (uint32_t)bw * K * 8u;        // bytes between band rows
    const int v01 = col_v01(Vg), ovc = col_ovc(Vg, vb);
    const uint32_t bdesc_s = smem_u32(bdesc2);
    const uint32_t snap0 = smem_u32(snap) + (uint32_t)(h * nrow + hl) * 4u;   // snapshot of entry (0, hl)
    const uint32_t sstr = (uint32_t)bw * 4u;            // bytes between snapshot rows
    // round j: view hl + LPC j, so the round's shared address and column
    // offsets are the first round's plus a constant (a lane past the agent's
    // views reads bytes of its ring slot or of the warp's next region, and
    // drops them)
    const uint32_t lbase0 = band_s + (uint32_t)(hl * K + h) * 8u;   // entry (0, hl)
    const uint32_t hoff0 = 2u + (uint32_t)hl;                        // view hl's header byte
    const uint32_t voff0 = (uint32_t)(v01 + 2 * vb * hl);           // view hl's value pair
    uint32_t vokm = 0;        // bit j: round j's view exists
#pragma unroll
    for (int j = 0; j < RR; ++j) vokm |= (hl + LPC * j < Vg ? 1u : 0u) << j;
    // tile rows of P lanes (P a power of two >= S + 2, at most 32)
    const int lP = TS <= 8 ? 3 : TS <= 16 ? 4 : 5;
    const int tr0 = lane >> lP, tc0 = lane & ((1 << lP) - 1), trs = 32 >> lP;

    // chain k: reconstruction (slice) rbase + k rstride
    auto rb_of = [&](int k) { return (int64_t)(rbase + k * rstride); };
    // this lane's prior neighbours: lanes 0..7 of each chain the in-plane
    // 8-neighbourhood; volumes: the 26-neighbourhood, lane l neighbour l with
    // one chain, lane l of a chain's 16 neighbours l and l + 16 with two
    // (NBL per lane); other lanes read the pixel itself with weight 0.
    // mbit: the neighbour's bit in a pixel's 3x3 in-image mask.
    constexpr int NBL = (NB26 && K == 2) ? 2 : 1;
    float *xth = xt0 + h * TA;                   // this lane's chain's X tile
    const float2 *vt2h = vt20 + h * S2;
    int mbit[NBL];
    float pb[NBL];
    const float *nb_tile[NBL];
    uint32_t nbt_s[NBL];
#pragma unroll
    for (int t = 0; t < NBL; ++t) {
        int pdz = 0, pdi = 0, pdj = 0;
        pb[t] = 0.f;
        if (NB26) {
            const int l = K == 2 ? hl + 16 * t : lane;
            if (l < 26) {
                const int kk = l < 13 ? l : l + 1;   // skip the centre of the 3x3x3
                pdz = kk / 9 - 1;
                pdi = (kk / 3) % 3 - 1;
                pdj = kk % 3 - 1;
                const int d2 = pdz * pdz + pdi * pdi + pdj * pdj;
                const int64_t zz = rb_of(h) + pdz;
                pb[t] = (zz >= 0 && zz < A.B) ? A.pscale * A.b26[d2 - 1] : 0.f;
            }
        } else if (hl < 8) {
            const int kk = hl < 4 ? hl : hl + 1;
            pdi = kk / 3 - 1;
            pdj = kk % 3 - 1;
            pb[t] = A.pscale * ((pdi != 0 && pdj != 0) ? A.b_diag : A.b_edge);
        }
        mbit[t] = (pdi + 1) * 3 + (pdj + 1);
        const float *tile = pdz == 0 ? xth : halo0 + (2 * h + (pdz < 0 ? 0 : 1)) * TA;
        nb_tile[t] = tile + pdi * TS + pdj;
        nbt_s[t] = smem_u32(nb_tile[t]);
    }
    const uint32_t xth_s = smem_u32(xth), vt2h_s = smem_u32(vt2h);
    const uint32_t ring_s = smem_u32(ring);
    // the prior's curvature and gradient at the pixel of tile index tc and
    // value xs, this lane's share (summed over the chain's lanes below); the
    // neighbours' values by tile pointer (nbv(t)) or shared address
    auto prior_terms = [&](uint32_t pq, float xs, auto nbv, float &pr2, float &pr1) {
        const float d0 = xs - nbv(0);
        const float w0 = (((pq >> (11 + mbit[0])) & 1u) ? pb[0] : 0.f) * prior_weight(A, d0);
        pr2 = w0;
        pr1 = w0 * d0;
#pragma unroll
        for (int t = 1; t < NBL; ++t) {
            const float d = xs - nbv(t);
            const float wgt = (((pq >> (11 + mbit[t])) & 1u) ? pb[t] : 0.f) * prior_weight(A, d);
            pr2 += wgt;
            pr1 = fmaf(wgt, d, pr1);
        }
    };
    float2 *const eLh = A.eL + rb_of(h) * A.ne + (int64_t)v0 * A.D;   // this lane's chain, agent g
    unsigned long long *const dacch = DET ? A.dacc + rb_of(h) * A.ne + (int64_t)v0 * A.D : nullptr;
    unsigned *const phase_c = DET ? A.phase + pair : nullptr;
    auto Xk = [&](int k) { return A.X + (rb_of(k) * A.N + g) * n; };

    // --- super-voxel metadata -------------------------------------------
    auto sv_of = [&](int m) {           // m-th super-voxel of this warp, -1 past the end
        const int slot = cidx + m * Cw;
        if (slot >= A.nsv) return -1;
        return A.sv_order[A.backward ? A.nsv - 1 - slot : slot];
    };
    // visiting list of super-voxel sv from its column offsets sc: per
    // non-empty pixel in visiting order its tile index, in-image neighbour
    // mask and pixel offset, and its column's offset and size; returns the
    // count
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
                const int ti = t >> lS, tj = t & (S - 1), i = bi + ti, j = bj + tj;
                uint32_t mask = 0;
#pragma unroll
                for (int di = -1; di <= 1; ++di)
#pragma unroll
                    for (int dj = -1; dj <= 1; ++dj)
                        if (i + di >= 0 && i + di < A.ny && j + dj >= 0 && j + dj < A.nx)
                            mask |= 1u << ((di + 1) * 3 + dj + 1);
                const int pos = count + __popc(m & lt_mask);
                pl[pos] = (uint32_t)((ti + 1) * TS + tj + 1) | mask << 11 | (uint32_t)t << 20;
                cl[pos] = make_uint2((uint32_t)((svoff + sc[t]) >> 4), sc[t + 1] - sc[t]);
            }
            count += __popc(m);
        }
        __syncwarp();
        return count;
    };
    // TMA of one column into ring stage idx % kRing, issued by lane 0 (all
    // lanes run the call; the others are predicated off, no branch)
    const uint64_t stream_policy = l2_evict_first_policy();
    auto issue = [&](uint32_t idx, const uint8_t *src, uint32_t bytes) {
        const uint32_t stg = idx & (kRing - 1);
        if (kDebug && !debug_ok(bytes >= 16 && bytes <= (uint32_t)A.col_stride && (bytes & 15u) == 0, A.status))
            bytes = 16;     // a safe copy: the column's first 16 bytes
        tma_load_1d_lane0(ring + (size_t)stg * A.col_stride, src, bytes, &bars[stg], lane, stream_policy);
    };

    int sv = sv_of(0);
    if (sv < 0) {
        if (DET && lane == 0)
            for (int p = 0; p < 2 * ((A.nsv + Cw - 1) / Cw); ++p) phase_arrive(A.phase + pair);
        return true;
    }
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
    // one after the other, over all its work items).  dec: columns decoded;
    // issued: columns whose copy has been started; seq0: sequence number of
    // the current super-voxel's first column.  A slot is refilled one column late: when column d is
    // decoded, the data of column d-1 has been used by the stores of the
    // pixel before, so its slot is free; at most kRing - 1 copies are in
    // flight beside the column held in registers.
    uint32_t seq0 = dec;      // (issued == dec: the previous item's columns are all decoded)
    int count_n = 0;
    int cur = 0;
    auto col_src = [&](uint2 c) { return A.cols + ((uint64_t)c.x << 4); };
    // column x of the sequence from the current (cl) or next (cl_n) list
    auto list_entry = [&](uint32_t x, const uint2 *cl, const uint2 *cl_n) {
        return x < (uint32_t)count ? cl[x] : cl_n[x - count];
    };
    auto fill_ring = [&](const uint2 *cl, const uint2 *cl_n) {
        while (issued - dec < (uint32_t)(kRing - 1) && issued - seq0 < (uint32_t)(count + count_n)) {
            const uint2 c = list_entry(issued - seq0, cl, cl_n);
            issue(issued, col_src(c), c.y);
            ++issued;
        }
    };
    fill_ring(cl2, cl2 + S2);
    // drain this warp's copies in flight (bounded) before leaving early
    auto drain = [&]() {
        for (uint32_t q2 = dec; q2 < issued; ++q2) {
            uint32_t sp2 = 0;
            while (!mbar_try_wait(&bars[q2 & (kRing - 1)], (q2 / kRing) & 1u) && ++sp2 < kSpinLimit) {}
        }
    };
    // wait for column dec; false when the bounded wait gave up (the host is
    // flagged and this warp's copies in flight are drained first)
    auto wait_column = [&]() {
        const uint32_t stg = dec & (kRing - 1);
        const uint32_t parity = (dec / kRing) & 1u;
        uint32_t spins = 0;
        while (!__all_sync(FULL, mbar_try_wait(&bars[stg], parity))) {
            if (++spins > kSpinLimit) {
                if (lane == 0) atomicExch(A.status, kStatusTimeout);
                drain();
                return false;
            }
        }
        return true;
    };
    // read column dec from its ring slot (first half of decoding: the loads)
    auto col_load = [&](ColRaw<RR, RRO> &w) {
        const uint8_t *col = ring + (size_t)(dec & (kRing - 1)) * A.col_stride;
        w.n3 = *(const uint16_t *)col;
        const uint8_t *ch = col + hoff0, *cv = col + voff0;
#pragma unroll
        for (int j = 0; j < RR; ++j) {
            w.hb[j] = ch[LPC * j];
            w.a[j] = ld_pair<T>(cv + 2 * vb * LPC * j, 0);
        }
        const int ovv = (ovc + 2 * w.n3 + 3) & ~3;
#pragma unroll
        for (int o = 0; o < RRO; ++o) {
            const int i = hl + LPC * o;
            const int il = i < w.n3 ? i : 0;
            w.code[o] = *(const uint16_t *)(col + ovc + 2 * il);
            w.a2[o] = ld_val<T>(col + ovv, il);
        }
    };
    // second half: band addresses and values; then the slot of the column
    // decoded before is refilled with the next column of the sequence
    auto col_finish = [&](const ColRaw<RR, RRO> &w, ColRegs<RR, RRO> &c, const uint2 *cl, const uint2 *cl_n) {
#pragma unroll
        for (int j = 0; j < RR; ++j) {
            bool ok = (vokm >> j) & 1u;
            if (kDebug && ok) ok = debug_ok((w.hb[j] & 63u) + 1u < (uint32_t)wmax, A.status);
            c.addr[j] = ok ? lbase0 + 256u * j + (w.hb[j] & 63u) * tstr : sink_s - tstr;
            c.a0[j] = ok ? w.a[j].x : 0.f;
            c.a1[j] = ok ? w.a[j].y : 0.f;
        }
#pragma unroll
        for (int o = 0; o < RRO; ++o) {
            bool ok = hl + LPC * o < w.n3;
            if (kDebug && ok) ok = debug_ok(w.code[o] < (uint32_t)(wmax * vpad), A.status);
            c.oaddr[o] = ok ? band_s + (w.code[o] * K + h) * 8u : sink_s;
            c.a2[o] = ok ? w.a2[o] : 0.f;
        }
        ++dec;
        if (issued - dec < (uint32_t)(kRing - 1) && issued - seq0 < (uint32_t)(count + count_n)) {
            const uint2 rf = list_entry(issued - seq0, cl, cl_n);
            issue(issued, col_src(rf), rf.y);
            ++issued;
        }
    };

    int status_seen = 0;
    // team exchange: every warp adds its value and flag; returns the OR of
    // the flags and the sum over the team's warps in warp order (the same
    // bits in every warp).  Slots alternate, so one barrier per exchange
    // keeps a slot from being rewritten before every warp has read it.
    uint32_t xpar = 0;
    auto team_sum = [&](float val, int flag, float &tot) -> int {
        const uint32_t mine = tm.xch0 + (uint32_t)tm.wi * tm.stride + xpar * 8u;
        if (lane == 0) {
            sts_f32(mine, val);
            sts_u32(mine + 4u, (uint32_t)flag);
        }
        team_barrier(tm.bar, 32 * W);
        float sum = 0.f;
        uint32_t any = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t a = tm.xch0 + (uint32_t)w * tm.stride + xpar * 8u;
            sum += lds_f32(a);
            any |= lds_u32(a + 4u);
        }
        xpar ^= 1u;
        tot = sum;
        return (int)any;
    };
    ColRegs<RR, RRO> cc, cn;
    bool have_cur = false;    // cc holds the current super-voxel's first column

    for (int m = 0; sv >= 0; ++m) {
        uint32_t *bdesc = bdesc2 + cur * vpad;
        const uint32_t *pl = pl2 + cur * S2;
        const uint2 *cl = cl2 + cur * S2;
        uint32_t *bdesc_n = bdesc2 + (cur ^ 1) * vpad;
        uint32_t *pl_n = pl2 + (cur ^ 1) * S2;
        uint2 *cl_n = cl2 + (cur ^ 1) * S2;
        const int si = sv / A.nsvx, sj = sv - si * A.nsvx;
        const int i0 = si * S, j0 = sj * S;

        // deterministic mode: this phase's reads wait for every warp of the
        // pair to have written the previous phase's changes
        if (DET && m > 0) {
            bool ok = true;
            if (lane == 0) ok = phase_wait(phase_c, 2u * (unsigned)Cw * (unsigned)m);
            if (!__shfl_sync(FULL, ok ? 1 : 0, 0)) {
                if (lane == 0) atomicExch(A.status, kStatusTimeout);
                drain();
                return false;
            }
            __threadfence();
        }
        // --- band (e, Lambda) of every chain, X tiles, theta2 ---------------
        // the lanes of chain h load and later flush the entries of chain h,
        // lane hl taking views hl, hl + 32/K, ... (the same lane for the same
        // global entry in every super-voxel, so a flushed change is seen by
        // the next load of that entry); e also goes into the snapshot
        // (deterministic mode: once the accumulated changes are added)
        for (int v = hl_v, jj = 0; v < Vg; v += LPCV, ++jj) {
            const uint32_t d = lds_u32(bdesc_s + cur * vpad * 4u + 4u * v);
            int len = (int)(d >> 16);
            if (kDebug && !debug_ok(len <= wmax && (int)(d & 0xFFFFu) + len <= A.D, A.status)) len = 0;
            const float2 *src = eLh + (int64_t)v * A.D + (d & 0xFFFFu);
            uint32_t ds = lbase0 + (uint32_t)jj * 256u, ss = snap0 + (uint32_t)(jj * LPC) * 4u;
            for (int t = 0; t < len; ++t) {
                cp_async8_s(ds, src + t);
                if (!DET) cp_async4_s(ss, src + t);
                ds += tstr;
                ss += sstr;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float *xt = xt0 + k * TA;
            float2 *vt2 = vt20 + k * S2;
            const float *Xg = Xk(k);
            for (int ti = tr0; ti < TS; ti += trs)
                for (int tj = tc0; tj < TS; tj += 32) {
                    const int i = i0 + ti - 1, j = j0 + tj - 1;
                    // deterministic mode: other warps' X through L2 (L1 may be stale)
                    if (i >= 0 && i < A.ny && j >= 0 && j < A.nx) {
                        if (DET) xt[ti * TS + tj] = __ldcg(&Xg[(int64_t)i * A.nx + j]);
                        else cp_async4(&xt[ti * TS + tj], &Xg[(int64_t)i * A.nx + j]);
                    } else {
                        xt[ti * TS + tj] = 0.f;
                    }
                }
            const float *t2g = A.theta2 + (rb_of(k) * A.N + g) * n;
            for (int q = lane; q < count; q += 32) {
                const int t = (int)(pl[q] >> 20);
                cp_async4(&vt2[q].y, &t2g[(int64_t)(i0 + (t >> lS)) * A.nx + j0 + (t & (S - 1))]);
            }
        }
        if (NB26) {
            // X tiles of each chain's neighbouring slices
            for (int hh = 0; hh < 2 * K; ++hh) {
                const int64_t zz = rb_of(hh >> 1) + ((hh & 1) ? 1 : -1);
                float *ht = halo0 + hh * TA;
                const float *Xz = (zz >= 0 && zz < A.B) ? A.X + ((int64_t)zz * A.N + g) * n : nullptr;
                for (int ti = tr0; ti < TS; ti += trs)
                    for (int tj = tc0; tj < TS; tj += 32) {
                        const int i = i0 + ti - 1, j = j0 + tj - 1;
                        if (Xz && i >= 0 && i < A.ny && j >= 0 && j < A.nx) {
                            if (DET) ht[ti * TS + tj] = __ldcg(&Xz[(int64_t)i * A.nx + j]);
                            else cp_async4(&ht[ti * TS + tj], &Xz[(int64_t)i * A.nx + j]);
                        } else {
                            ht[ti * TS + tj] = 0.f;
                        }
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
            float2 *vt2 = vt20 + k * S2;
            const int64_t rb = rb_of(k);
            for (int q = lane; q < count; q += 32) {
                const int t = (int)(pl[q] >> 20);
                const int64_t s = (int64_t)(i0 + (t >> lS)) * A.nx + j0 + (t & (S - 1));
                const float vv = A.vexp ? A.vexp[(rb * A.N + g) * n + s]
                                        : (float)(2.0 * A.wbar[rb * n + s] - (double)A.w[(rb * A.N + g) * n + s]);
                vt2[q].x = vv * A.inv_s2;
            }
        }
        if (lane == 0) status_seen = *((volatile int *)A.status);
        cp_async_wait_all();
        if (DET) {
            // e = e at launch + the changes accumulated so far; snapshot;
            // then this warp's reads of the phase are done
            for (int v = hl_v, jj = 0; v < Vg; v += LPCV, ++jj) {
                const uint32_t d = lds_u32(bdesc_s + cur * vpad * 4u + 4u * v);
                int len = (int)(d >> 16);
            if (kDebug && !debug_ok(len <= wmax && (int)(d & 0xFFFFu) + len <= A.D, A.status)) len = 0;
                const unsigned long long *da = dacch + (int64_t)v * A.D + (d & 0xFFFFu);
                uint32_t ds = lbase0 + (uint32_t)jj * 256u, ss = snap0 + (uint32_t)(jj * LPC) * 4u;
#pragma unroll 4
                for (int t = 0; t < len; ++t) {
                    const float e = lds_f32(ds) + efix_value(__ldcg(da + t));
                    sts_f32(ds, e);
                    sts_f32(ss, e);
                    ds += tstr;
                    ss += sstr;
                }
            }
            __syncwarp();
            if (lane == 0) phase_arrive(phase_c);
        }
        __syncwarp();
        status_seen = __shfl_sync(FULL, status_seen, 0);
        count_n = 0;
        if (sv_n >= 0) count_n = build_list(sv_n, scoff, pl_n, cl_n);
        // a short super-voxel may leave ring slots free: start the next one's columns
        fill_ring(cl, cl_n);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            float2 *vt2 = vt20 + k * S2;
            for (int q = lane; q < count; q += 32) vt2[q].y += A.inv_s2;
        }
        __syncwarp();
        int stop = status_seen != 0;
        if constexpr (W > 1) {
            float unused;
            stop = team_sum(0.f, stop, unused);     // the team stops together
        }
        if (stop) {
            // another warp gave up: drain this warp's copies in flight and stop
            drain();
            return false;
        }
        if (R > 0 && !have_cur && count > 0) {
            if (!wait_column()) return false;
            ColRaw<RR, RRO> w0;
            col_load(w0);
            col_finish(w0, cc, cl, cl_n);
            have_cur = true;
        }

        // --- visit the pixels ------------------------------------------------
        // one pixel with its column in c; the next column (this super-voxel's
        // or the next one's first) is decoded into c2 meanwhile.  False when a
        // bounded wait gave up.
        auto pixel = [&](int q, ColRegs<RR, RRO> &c, ColRegs<RR, RRO> &c2) {
            // gathers of this pixel's band entries (the previous pixel's
            // update is visible after its __syncwarp)
            float2 g0[RR], g1[RR], g2[RRO];
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                g0[j] = lds_f2(c.addr[j]);
                g1[j] = lds_f2(c.addr[j] + tstr);
            }
#pragma unroll
            for (int o = 0; o < RRO; ++o) g2[o] = lds_f2(c.oaddr[o]);
            // prior through the surrogate weights (a lane's neighbours, see
            // above), from the X tiles only.  No branch: out-of-image
            // neighbours and idle lanes get weight 0.
            const uint32_t pq = pl[q];
            const int tc = (int)(pq & 0x7FFu);
            const float2 vq = vt2h[q];
            const float xs = xth[tc];
            float pr2, pr1;
            prior_terms(pq, xs, [&](int t) { return nb_tile[t][tc]; }, pr2, pr1);
            const float prox = fmaf(xs, A.inv_s2, -vq.x);   // (x - v) / sigma^2
            if (NB26) {
#pragma unroll
                for (int o = 1; o < LPC; o <<= 1) pr2 += __shfl_xor_sync(FULL, pr2, o);
            } else {
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) pr2 += __shfl_xor_sync(FULL, pr2, o);
                pr2 = __shfl_sync(FULL, pr2, lane & ~(LPC - 1));
            }
            // data term: -sum A Lambda e over this lane's entries, plus the
            // prior's gradient; theta2 = sum A^2 Lambda is stored
            float pa = pr1, pc = 0.f;
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                pa = fmaf(-c.a0[j] * g0[j].y, g0[j].x, pa);
                pc = fmaf(-c.a1[j] * g1[j].y, g1[j].x, pc);
            }
#pragma unroll
            for (int o = 0; o < RRO; ++o) pa = fmaf(-c.a2[o] * g2[o].y, g2[o].x, pa);
            float p1 = pa + pc;
            const bool more = dec - seq0 < (uint32_t)(count + count_n);
            if (more) {
                if (!wait_column()) return false;
                ColRaw<RR, RRO> wn;
                col_load(wn);
                col_finish(wn, c2, cl, cl_n);
            }
#pragma unroll
            for (int o = LPC / 2; o > 0; o >>= 1) p1 += __shfl_xor_sync(FULL, p1, o);
            // the step's sign and zero set come from the numerator alone, so an
            // approximate reciprocal leaves the fixed point unchanged
            const float alpha = -(p1 + prox) * rcp_approx(vq.y + pr2);
            // update e: a lane's own views' entries, and its share of the
            // three-channel list (idle lanes write the zero sink with value 0)
#pragma unroll
            for (int j = 0; j < RR; ++j) {
                sts_f(c.addr[j], fmaf(-c.a0[j], alpha, g0[j].x));
                sts_f(c.addr[j] + tstr, fmaf(-c.a1[j], alpha, g1[j].x));
            }
#pragma unroll
            for (int o = 0; o < RRO; ++o) sts_f(c.oaddr[o], fmaf(-c.a2[o], alpha, g2[o].x));
            // X update: every lane of the chain stores the same value
            xth[tc] = xs + alpha;
            __syncwarp();
            return true;
        };
        // R = 0: one pixel, its column decoded from the ring slot as it is
        // used (views and list entries in run-time rounds, re-read for the
        // update); the slot of the column before is refilled at the start
        const uint32_t pl_s = smem_u32(pl);
        // three-channel list entry's band address; with a team, whether the
        // entry's view is this warp's
        auto ovf_addr = [&](uint32_t code, bool &own) -> uint32_t {
            if (kDebug && !debug_ok(code < (uint32_t)(wmax * vpad), A.status)) {
                own = false;
                return sink_s;
            }
            if constexpr (W == 1) {
                own = true;
                return band_s + (code * K + h) * 8u;
            } else {
                const uint32_t row = code / (uint32_t)vpad, v = code - row * (uint32_t)vpad;
                own = ((v >> 5) & (uint32_t)(W - 1)) == (uint32_t)tm.wi;
                return band_s + (row * (uint32_t)bw + (((v >> 5) / (uint32_t)W) << 5 | (v & 31u))) * 8u;
            }
        };
        auto pixel_any = [&](int q) {
            const bool okc = wait_column();
            if (!okc) {
                if constexpr (W > 1) {
                    float unused;
                    team_sum(0.f, 1, unused);    // tell the team at this pixel's exchange
                }
                return false;
            }
            const uint32_t col = ring_s + (dec & (kRing - 1)) * (uint32_t)A.col_stride;
            const int n3 = (int)lds_u16(col);
            const uint32_t ovv = col + (uint32_t)((ovc + 2 * n3 + 3) & ~3);
            ++dec;
            if (issued - dec < (uint32_t)(kRing - 1) && issued - seq0 < (uint32_t)(count + count_n)) {
                const uint2 rf = list_entry(issued - seq0, cl, cl_n);
                issue(issued, col_src(rf), rf.y);
                ++issued;
            }
            const uint32_t pq = lds_u32(pl_s + 4u * q);
            const uint32_t tc4 = (pq & 0x7FFu) * 4u;
            const float2 vq = lds_f2(vt2h_s + 8u * q);
            const float xs = lds_f32(xth_s + tc4);
            float pr2, pr1;
            prior_terms(pq, xs, [&](int t) { return lds_f32(nbt_s[t] + tc4); }, pr2, pr1);
            const float prox = fmaf(xs, A.inv_s2, -vq.x);
            if (NB26) {
#pragma unroll
                for (int o = 1; o < LPC; o <<= 1) pr2 += __shfl_xor_sync(FULL, pr2, o);
            } else {
#pragma unroll
                for (int o = 1; o < 8; o <<= 1) pr2 += __shfl_xor_sync(FULL, pr2, o);
                pr2 = __shfl_sync(FULL, pr2, lane & ~(LPC - 1));
            }
            const int nr = (Vg + LPCV - 1) / LPCV, nro = (n3 + LPC - 1) / LPC;
            // the prior's gradient enters once per team
            float pa = (W == 1 || tm.wi == 0) ? pr1 : 0.f, pc = 0.f;
            for (int j = 0; j < nr; ++j) {
                const int v = hl_v + LPCV * j;
                if (v < Vg && debug_ok((lds_u8(col + 2u + v) & 63u) + 1u < (uint32_t)wmax, A.status)) {
                    const float2 a = lds_pair<T>(col + v01 + 2u * vb * v);
                    const uint32_t ad = lbase0 + 256u * j + (lds_u8(col + 2u + v) & 63u) * tstr;
                    const float2 e0 = lds_f2(ad), e1 = lds_f2(ad + tstr);
                    pa = fmaf(-a.x * e0.y, e0.x, pa);
                    pc = fmaf(-a.y * e1.y, e1.x, pc);
                }
            }
            for (int o = 0; o < nro; ++o) {
                const int i = hl + LPC * o;
                if (i < n3) {
                    bool own;
                    const uint32_t ad = ovf_addr(lds_u16(col + ovc + 2u * i), own);
                    if (own) {
                        const float2 e2 = lds_f2(ad);
                        pa = fmaf(-lds_val<T>(ovv + vb * i) * e2.y, e2.x, pa);
                    }
                }
            }
            float p1 = pa + pc;
#pragma unroll
            for (int o = LPC / 2; o > 0; o >>= 1) p1 += __shfl_xor_sync(FULL, p1, o);
            if constexpr (W > 1) {
                float tot;
                if (team_sum(p1, 0, tot)) {
                    drain();
                    return false;
                }
                p1 = tot;
            }
            const float alpha = -(p1 + prox) * rcp_approx(vq.y + pr2);
            for (int j = 0; j < nr; ++j) {
                const int v = hl_v + LPCV * j;
                if (v < Vg && (!kDebug || (lds_u8(col + 2u + v) & 63u) + 1u < (uint32_t)wmax)) {
                    const float2 a = lds_pair<T>(col + v01 + 2u * vb * v);
                    const uint32_t ad = lbase0 + 256u * j + (lds_u8(col + 2u + v) & 63u) * tstr;
                    sts_f(ad, fmaf(-a.x, alpha, lds_f32(ad)));
                    sts_f(ad + tstr, fmaf(-a.y, alpha, lds_f32(ad + tstr)));
                }
            }
            for (int o = 0; o < nro; ++o) {
                const int i = hl + LPC * o;
                if (i < n3) {
                    bool own;
                    const uint32_t ad = ovf_addr(lds_u16(col + ovc + 2u * i), own);
                    if (own) sts_f(ad, fmaf(-lds_val<T>(ovv + vb * i), alpha, lds_f32(ad)));
                }
            }
            sts_f32(xth_s + tc4, xs + alpha);
            __syncwarp();
            return true;
        };
        int q = 0;
        if constexpr (R == 0) {
            for (; q < count; ++q)
                if (!pixel_any(q)) return false;
        } else if constexpr (R <= 3) {
            // two pixels per trip, the decoded columns alternating between
            // cc and cn (no register copy)
            for (; q + 1 < count; q += 2) {
                if (!pixel(q, cc, cn)) return false;
                if (!pixel(q + 1, cn, cc)) return false;
            }
        } else {
            for (; q + 1 < count; ++q) {
                if (!pixel(q, cc, cn)) return false;
                cc = cn;
            }
        }
        if (R > 0 && q < count) {
            if (!pixel(q, cc, cn)) return false;
            cc = cn;
        }
        // the next super-voxel's first column is decoded already when the
        // sequence went on past this one
        have_cur = dec - seq0 > (uint32_t)count;

        // deterministic mode: write only once every warp of the pair has read
        // this phase's state
        if (DET) {
            bool ok = true;
            if (lane == 0) ok = phase_wait(phase_c, 2u * (unsigned)Cw * (unsigned)m + (unsigned)Cw);
            if (!__shfl_sync(FULL, ok ? 1 : 0, 0)) {
                if (lane == 0) atomicExch(A.status, kStatusTimeout);
                drain();
                return false;
            }
        }
        // --- write back: X tiles (once per team) and the change of e ----------
#pragma unroll
        for (int k = 0; k < ((W == 1 || tm.wi == 0) ? K : 0); ++k) {
            const float *xt = xt0 + k * TA;
            float *Xg = Xk(k);
            for (int p = lane; p < S2; p += 32) {
                const int ti = p >> lS, tj = p & (S - 1);
                if (i0 + ti < A.ny && j0 + tj < A.nx)
                    Xg[(int64_t)(i0 + ti) * A.nx + j0 + tj] = xt[(ti + 1) * TS + tj + 1];
            }
        }
        for (int v = hl_v, jj = 0; v < Vg; v += LPCV, ++jj) {
            const uint32_t d = lds_u32(bdesc_s + cur * vpad * 4u + 4u * v);
            int len = (int)(d >> 16);
            if (kDebug && !debug_ok(len <= wmax && (int)(d & 0xFFFFu) + len <= A.D, A.status)) len = 0;
            float2 *eg = eLh + (int64_t)v * A.D + (d & 0xFFFFu);
            uint32_t ds = lbase0 + (uint32_t)jj * 256u, ss = snap0 + (uint32_t)(jj * LPC) * 4u;
            unsigned long long *da = dacch + (int64_t)v * A.D + (d & 0xFFFFu);
            for (int t = 0; t < len; ++t) {
                const float de = lds_f32(ds) - lds_f32(ss);
                if (DET) efix_add(da + t, de);
                else if (de != 0.f) atomicAdd(&eg[t].x, de);
                ds += tstr;
                ss += sstr;
            }
        }
        if (DET) {
            __threadfence();
            __syncwarp();
            if (lane == 0) phase_arrive(phase_c);
        }
        __syncwarp();
        // hand the staged next-super-voxel state over; its successor's list
        // is built when it starts
        sv = sv_n;
        seq0 += count;
        count = count_n;
        count_n = 0;
        cur ^= 1;
        if (sv < 0 && DET && lane == 0) {
            // phases past this warp's last super-voxel: nothing to read or
            // write, but the pair's counter counts every warp
            const int nph = (A.nsv + Cw - 1) / Cw;
            for (int p = m + 1; p < nph; ++p) {
                phase_arrive(phase_c);
                phase_arrive(phase_c);
            }
        }
    }
    return true;
}

// One warp per (group, agent, row of super-voxels), fixed at launch: the
// C warps of a pair are warps pair, pair + G N, pair + 2 G N, ...
template <typename T, int K, int R, int RO, bool NB26, bool DET>
__global__ void __maxnreg__(MACE_SWEEP_MAXNREG) icd_sweep_kernel(SweepArgs A)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const WarpSmem Ly = warp_smem_layout(A.vpad, A.wmax, A.col_stride, A.S, K, NB26);
    uint8_t *base = smem + (threadIdx.x >> 5) * Ly.total;
    sweep_warp_init(base, Ly, A.wmax * A.vpad * K, lane);
    const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (gw >= A.nwarps) return;
    const int G = A.B / K;
    const int pair = gw % (G * A.N);
    uint32_t dec = 0, issued = 0;
    const TeamCtx solo = {0, 0, 0u, 0u};
    sweep_work<T, K, R, RO, NB26, DET, 1, SweepArgs>(A, base, Ly, pair / A.N, pair % A.N, gw / (G * A.N),
                                                     A.nwarps / (G * A.N), dec, issued, solo, (pair / A.N) * K, 1);
}

// Work queue over (request, group, agent, row of super-voxels): every resident
// warp takes the next item from a counter until none is left, copies the
// item's request descriptor into its shared memory and runs the row.  Items
// are numbered row-fastest within a (group, agent) pair, so the C rows of a
// pair are taken by warps at about the same time, as in the fixed schedule,
// and a warp that finishes early takes more work (agents of uneven size).
// zpar >= 0: only the groups (slices) of that parity.
struct QueueArgs {
    const SweepArgs *table;     // per request, in device memory
    const int *offsets;         // [nreq + 1] first item of each request
    unsigned *counter;          // zero at launch
    int nreq, total, zpar;
    int vpad, wmax, col_stride, S;   // shared-memory layout: the largest of the requests
};

template <typename T, int K, int R, int RO, bool NB26, int W>
__global__ void __maxnreg__(MACE_SWEEP_MAXNREG) icd_sweep_queue_kernel(QueueArgs Q)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const WarpSmem Ly = warp_smem_layout(Q.vpad, Q.wmax, Q.col_stride, Q.S, K, NB26, W);
    const size_t per_warp = Ly.total + ((sizeof(SweepArgs) + 15) & ~(size_t)15);
    uint8_t *base = smem + warp * per_warp;
    SweepArgs *args = (SweepArgs *)(base + Ly.total);
    sweep_warp_init(base, Ly, Q.wmax * band_width(Q.vpad, W) * K, lane);
    // a team: W consecutive warps of the block; its first warp takes the
    // items and hands them over through its exchange slots (two, used in turn)
    TeamCtx tm;
    tm.wi = warp % W;
    tm.bar = 1 + warp / W;
    tm.stride = (uint32_t)per_warp;
    tm.xch0 = smem_u32(smem + (warp - tm.wi) * per_warp + Ly.xch);
    const uint32_t item_slot = tm.xch0 + 16u;
    uint32_t ipar = 0;
    uint32_t dec = 0, issued = 0;
    for (;;) {
        unsigned item = 0;
        if (lane == 0 && tm.wi == 0) item = atomicAdd(Q.counter, 1u);
        if constexpr (W > 1) {
            if (lane == 0 && tm.wi == 0) sts_u32(item_slot + 4u * ipar, item);
            team_barrier(tm.bar, 32 * W);
            item = lds_u32(item_slot + 4u * ipar);
            ipar ^= 1u;
        } else {
            item = __shfl_sync(0xffffffffu, item, 0);
        }
        if ((int)item >= Q.total) return;
        int r = 0;
        while (r + 1 < Q.nreq && (int)item >= Q.offsets[r + 1]) ++r;
        // this item's request descriptor, word by word
        const uint32_t *src = (const uint32_t *)(Q.table + r);
        for (int k = lane; k < (int)(sizeof(SweepArgs) / 4); k += 32) ((uint32_t *)args)[k] = src[k];
        __syncwarp();
        // the band back to zero: entries an item does not load are read with
        // matrix value 0, and a value left by another request's item (which
        // may have diverged) must not turn 0 x e into a NaN
        {
            float2 *band = (float2 *)(base + Ly.band);
            const int nband = Q.wmax * band_width(Q.vpad, W) * K;
            for (int f = lane; f <= nband; f += 32) band[f] = make_float2(0.f, 0.f);
            __syncwarp();   // before any lane's loads into the band
        }
        const SweepArgs &A = *args;
        const int local = (int)item - Q.offsets[r];
        const int Cw = A.nwarps;                 // rows of a pair in flight (the request's concurrency)
        const int pl = local / Cw, cidx = local - pl * Cw;
        const int grp = pl / A.N;
        const int g = pl - grp * A.N;
        // zpar >= 0: group grp holds the K slices zpar + 2 (K grp + k)
        const int rbase = Q.zpar >= 0 ? Q.zpar + 2 * K * grp : K * grp;
        const int rstride = Q.zpar >= 0 ? 2 : 1;
        if (!sweep_work<T, K, R, RO, NB26, false, W, const SweepArgs &>(A, base, Ly, grp, g, cidx, Cw, dec, issued,
                                                                          tm, rbase, rstride))
            return;
        __syncwarp();
    }
}

// Rounds of views per lane and of the three-channel list for an agent of at
// most max_views views and columns of at most max_n3 three-channel runs.
inline int sweep_rounds(int max_views, int K) { return (max_views + 32 / K - 1) / (32 / K); }
inline int sweep_ovf_rounds(int R, int K) { return (K == 2 || R >= 3) ? 2 : 1; }

template <typename T, int K, bool NB26, bool DET>
static sweep_fn sweep_lookup_k(int R)
{
    switch (R) {
    case 1: return icd_sweep_kernel<T, K, 1, (K == 2 ? 2 : 1), NB26, DET>;
    case 2: return icd_sweep_kernel<T, K, 2, (K == 2 ? 2 : 1), NB26, DET>;
    case 3: return icd_sweep_kernel<T, K, 3, 2, NB26, DET>;
    case 4: return icd_sweep_kernel<T, K, 4, 2, NB26, DET>;
    default: return icd_sweep_kernel<T, K, 0, 1, NB26, DET>;   // any view count
    }
}

// The sweep kernel for agents of at most max_views views with K chains, the
// 8- or 26-neighbourhood and the free or deterministic schedule (agents of
// more than four rounds of views run the kernel that decodes at use); nullptr
// if that combination is not built.
template <typename T>
static sweep_fn sweep_lookup(int max_views, int K, bool nb26, bool det)
{
    const int R = sweep_rounds(max_views, K);
    if (nb26) {
        if (K == 1) return det ? sweep_lookup_k<T, 1, true, true>(R) : sweep_lookup_k<T, 1, true, false>(R);
        if (K == 2) return det ? sweep_lookup_k<T, 2, true, true>(R) : sweep_lookup_k<T, 2, true, false>(R);
        return nullptr;
    }
    if (K == 1) return det ? sweep_lookup_k<T, 1, false, true>(R) : sweep_lookup_k<T, 1, false, false>(R);
    if (K == 2) return det ? sweep_lookup_k<T, 2, false, true>(R) : sweep_lookup_k<T, 2, false, false>(R);
    return nullptr;
}

typedef void (*sweep_queue_fn)(QueueArgs);

template <typename T, int K, bool NB26>
static sweep_queue_fn sweep_queue_lookup_r(int R)
{
    switch (R) {
    case 1: return icd_sweep_queue_kernel<T, K, 1, (K == 2 ? 2 : 1), NB26, 1>;
    case 2: return icd_sweep_queue_kernel<T, K, 2, (K == 2 ? 2 : 1), NB26, 1>;
    case 3: return icd_sweep_queue_kernel<T, K, 3, 2, NB26, 1>;
    case 4: return icd_sweep_queue_kernel<T, K, 4, 2, NB26, 1>;
    default: return icd_sweep_queue_kernel<T, K, 0, 1, NB26, 1>;
    }
}

// The queue-fed sweep for agents of at most max_views views and the 8- or
// 26-neighbourhood: one chain per warp, or (volumes) two slices of one z
// parity per warp; W = 2 or 4: teams of W warps per super-voxel (2D, one
// chain, decoding each column as it is used).
template <typename T>
static sweep_queue_fn sweep_queue_lookup(int max_views, bool nb26, int W, int K)
{
    if (K == 2) return (nb26 && W == 1) ? sweep_queue_lookup_r<T, 2, true>(sweep_rounds(max_views, 2)) : nullptr;
    if (W == 2 && !nb26) return icd_sweep_queue_kernel<T, 1, 0, 1, false, 2>;
    if (W == 4 && !nb26) return icd_sweep_queue_kernel<T, 1, 0, 1, false, 4>;
    if (W != 1) return nullptr;
    const int R = sweep_rounds(max_views, 1);
    return nb26 ? sweep_queue_lookup_r<T, 1, true>(R) : sweep_queue_lookup_r<T, 1, false>(R);
}

__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f32(int max_views, int K, bool nb26, bool det);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_bf16(int max_views, int K, bool nb26, bool det);
__attribute__((visibility("hidden"))) sweep_fn mace_sweep_kernel_f16(int max_views, int K, bool nb26, bool det);
__attribute__((visibility("hidden"))) sweep_queue_fn mace_sweep_queue_kernel_f32(int max_views, bool nb26, int W, int K);
__attribute__((visibility("hidden"))) sweep_queue_fn mace_sweep_queue_kernel_bf16(int max_views, bool nb26, int W, int K);
__attribute__((visibility("hidden"))) sweep_queue_fn mace_sweep_queue_kernel_f16(int max_views, bool nb26, int W, int K);
