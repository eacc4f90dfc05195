// GB300 (sm_103a) implementation of partial-update MACE CT reconstruction
// (Sridhar, Wang, Buzzard, Bouman, arXiv 1911.09278).  C ABI in include/mace.h.
//
// Per Mann iteration (Algorithm 1):
//   consensus_kernel   wbar = (1/N) sum_i w_i in FP64 (the operator G, Eq.
//                      "G_operators"), plus the final fixed-order reduction of
//                      the previous iteration's residual partials;
//   icd_sweep_kernel   K passes of Algorithm 2 per agent: X_i <- F~_i(v_i; X_i)
//                      with v_i = 2 wbar - w_i formed on the fly;
//   mann_kernel        w_i <- rho (2 X_i - v_i) + (1 - rho) w_i, FP64 partials of
//                      ||w^(k+1) - w^(k)||^2 and ||w^(k+1)||^2.
//
// The stored system matrix is voxel-column-major per super-voxel (an SxS tile
// of pixels): for every agent, super-voxel and pixel, a column holding the
// pixel's run (first channel, length, values) in each of the agent's views;
// the format is in common.cuh.  One warp owns one super-voxel at a time
// (sweep.cuh): it stages the super-voxel's band of the agent's error sinogram
// e_i and weights Lambda_i in shared memory, streams the columns in with TMA
// bulk copies into a per-warp ring, visits the pixels in order, and adds its
// change of e back to global memory at the end.
// This file holds the matrix builder, the other kernels and the host side.
#include <string.h>
#include <math.h>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "sweep.cuh"

// NVTX range over a host call (shown by Nsight Systems and ncu's NVTX
// filters; without a tool attached a push or pop costs a few nanoseconds)
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// ---------------------------------------------------------------------------
// error handling
// ---------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

#define CUDA_TRY(expr)                                                          \
    do {                                                                        \
        cudaError_t _e = (expr);                                                \
        if (_e != cudaSuccess)                                                  \
            return fail(MACE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
    } while (0)

extern "C" const char *mace_last_error(void) { return g_last_error.c_str(); }

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------
// ---------------------------------------------------------------------------
// geometry: strip-integral footprint of a square pixel (FP64, IEEE ops only)
// ---------------------------------------------------------------------------
struct GeoParams {
    int nx, ny, D;
    double dx, dd, off;
};

__device__ __forceinline__ double trap_cdf_dev(double u, double w1, double w2)
{
    double u1 = __dmul_rn(0.5, __dsub_rn(w2, w1));
    double u2 = __dmul_rn(0.5, __dadd_rn(w2, w1));
    double h = __ddiv_rn(1.0, w2);
    if (u <= -u2) return 0.0;
    if (u < -u1) {
        double d = __dadd_rn(u, u2);
        return __ddiv_rn(__dmul_rn(__dmul_rn(h, d), d), __dmul_rn(2.0, w1));
    }
    if (u <= u1) return __dmul_rn(h, __dadd_rn(__dmul_rn(0.5, w1), __dadd_rn(u, u1)));
    if (u < u2) {
        double d = __dsub_rn(u2, u);
        return __dsub_rn(1.0, __ddiv_rn(__dmul_rn(__dmul_rn(h, d), d), __dmul_rn(2.0, w1)));
    }
    return 1.0;
}

// Run of pixel (row i, col j) at view (ct, st): first channel and length
// (0..3, clipped to the detector); values in vals when non-null.
__device__ __forceinline__ int footprint_dev(const GeoParams &G, double ct, double st, int i, int j,
                                             int &c0, double *vals)
{
    double xc = __dmul_rn(__dsub_rn((double)j, __dmul_rn(0.5, (double)(G.nx - 1))), G.dx);
    double yc = __dmul_rn(__dsub_rn(__dmul_rn(0.5, (double)(G.ny - 1)), (double)i), G.dx);
    double t0 = __dadd_rn(__dmul_rn(xc, ct), __dmul_rn(yc, st));
    double qc = __dadd_rn(__ddiv_rn(__dsub_rn(t0, G.off), G.dd), __dmul_rn(0.5, (double)G.D));
    double a = __ddiv_rn(__dmul_rn(G.dx, fabs(ct)), G.dd);
    double b = __ddiv_rn(__dmul_rn(G.dx, fabs(st)), G.dd);
    double w1 = a < b ? a : b;
    double w2 = a < b ? b : a;
    double half = __dmul_rn(0.5, __dadd_rn(a, b));
    double lo = __dsub_rn(qc, half), hi = __dadd_rn(qc, half);
    int cf = (int)floor(lo);
    int cl = (int)ceil(hi) - 1;
    if (cf < 0) cf = 0;
    if (cl > G.D - 1) cl = G.D - 1;
    int L = cl - cf + 1;
    if (L < 0) L = 0;
    if (L > 3) L = 3;  // excluded by the host check on the pitches
    c0 = cf;
    if (vals) {
        double scale = __ddiv_rn(__dmul_rn(G.dx, G.dx), G.dd);
        for (int k = 0; k < L; ++k) {
            double c = (double)(cf + k);
            double hiu = __dsub_rn(__dadd_rn(c, 1.0), qc);
            double lou = __dsub_rn(c, qc);
            vals[k] = __dmul_rn(scale, __dsub_rn(trap_cdf_dev(hiu, w1, w2), trap_cdf_dev(lou, w1, w2)));
        }
    }
    return L;
}

// What the footprint of a pixel in one view needs, tabulated on the host in
// FP64 (the divisions stay off the GPU's FP64 units): the channel coordinate
// of pixel (i, j)'s centre is q00 + j cq - i sq, and the footprint is the
// trapezoid of the FP64 routine above with these breakpoints.
struct ViewGeo {
    double q00, cq, sq;
    float u1, u2;    // (w2 - w1) / 2, (w2 + w1) / 2
    float h, k2;     // plateau height 1 / w2; ramp factor h / (2 w1), 0 when w1 = 0
    float w1;        // the shorter of a = dx |cos| / dd and b = dx |sin| / dd
    float half;      // half the footprint width, (a + b) / 2
    float scale;     // dx^2 / dd
};

// ---------------------------------------------------------------------------
// system matrix
// ---------------------------------------------------------------------------
struct mace_sysmatrix {
    GeoParams geo;
    int nz;
    int V, N, S, nsvx, nsvy, nsv, S2;
    int max_views, max_col_bytes, max_n3 = 0;
    int vpad, wmax;                   // band rows in shared memory: vpad views, wmax rows
    mace_dtype dtype;
    int vbytes;                       // bytes per stored value
    cudaStream_t stream;
    std::vector<int> view_agent;      // [V]
    std::vector<int> agent_views;     // views grouped by agent (increasing m)
    std::vector<int> view_off;        // [N+1]
    std::vector<double> cosv, sinv;
    // device
    double2 *d_cs = nullptr;          // (cos, sin) per view in agent order
    ViewGeo *d_vgeo = nullptr;        // footprint constants per view in agent order
    int *d_view_off = nullptr;        // [N+1]
    uint32_t *d_band = nullptr;       // [nsv * V]: agent g block at nsv*view_off[g], (lo | len << 16)
    int64_t *d_sv_base = nullptr;     // [N * nsv] byte offset of the super-voxel block
    uint32_t *d_col_off = nullptr;    // [N * nsv * (S2 + 1)] byte offsets inside the block
    uint8_t *d_cols = nullptr;
    int64_t bytes_cols = 0, nnz = 0;
    std::vector<int64_t> agent_bytes;
};

__global__ void band_kernel(GeoParams G, const double2 *__restrict__ cs, const int *__restrict__ view_off,
                            int N, int S, int nsvx, int nsv, uint32_t *__restrict__ band)
{
    // one thread per (view in agent order, super-voxel); the view's agent block
    // of band[] starts at nsv * view_off[g]
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int V = view_off[N];
    if (tid >= (int64_t)V * nsv) return;
    int vg = (int)(tid / nsv);        // global index in agent order
    int sv = (int)(tid % nsv);
    int g = 0;
    while (view_off[g + 1] <= vg) ++g;
    int v = vg - view_off[g];
    int Vg = view_off[g + 1] - view_off[g];
    int si = sv / nsvx, sj = sv % nsvx;
    int lo = 1 << 30, hi = -1;
    for (int t = 0; t < S * S; ++t) {
        int i = si * S + t / S, j = sj * S + t % S;
        if (i >= G.ny || j >= G.nx) continue;
        int c0;
        int L = footprint_dev(G, cs[vg].x, cs[vg].y, i, j, c0, nullptr);
        if (L > 0) {
            lo = min(lo, c0);
            hi = max(hi, c0 + L - 1);
        }
    }
    uint32_t d = 0;
    if (hi >= lo) d = (uint32_t)lo | ((uint32_t)(hi - lo + 1) << 16);
    band[(int64_t)nsv * view_off[g] + (int64_t)sv * Vg + v] = d;
}

__global__ void colsize_kernel(GeoParams G, const double2 *__restrict__ cs, const int *__restrict__ view_off,
                               int N, int S, int nsvx, int nsv, int vbytes,
                               uint32_t *__restrict__ col_bytes_out, uint32_t *__restrict__ col_nnz,
                               uint32_t *__restrict__ col_n3)
{
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int S2 = S * S;
    if (tid >= (int64_t)N * nsv * S2) return;
    int g = (int)(tid / ((int64_t)nsv * S2));
    int rem = (int)(tid % ((int64_t)nsv * S2));
    int sv = rem / S2, t = rem % S2;
    int si = sv / nsvx, sj = sv % nsvx;
    int i = si * S + t / S, j = sj * S + t % S;
    if (i >= G.ny || j >= G.nx) { col_bytes_out[tid] = 0; col_nnz[tid] = 0; col_n3[tid] = 0; return; }
    int v0 = view_off[g], Vg = view_off[g + 1] - v0;
    int nz = 0, n3 = 0;
    for (int v = 0; v < Vg; ++v) {
        int c0;
        const int L = footprint_dev(G, cs[v0 + v].x, cs[v0 + v].y, i, j, c0, nullptr);
        nz += L;
        n3 += L == 3;
    }
    col_bytes_out[tid] = col_bytes(Vg, vbytes, n3);
    col_nnz[tid] = nz;
    col_n3[tid] = n3;
}

template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ float from_double<float>(double x) { return __double2float_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 from_double<__nv_bfloat16>(double x) { return __double2bfloat16(x); }
template <> __device__ __forceinline__ __half from_double<__half>(double x) { return __double2half(x); }

template <typename T>
__global__ void fill_kernel(GeoParams G, const double2 *__restrict__ cs, const int *__restrict__ view_off,
                            int N, int S, int nsvx, int nsv, int vpad, const uint32_t *__restrict__ band,
                            const int64_t *__restrict__ sv_base, const uint32_t *__restrict__ col_off,
                            uint8_t *__restrict__ cols)
{
    // one thread per column; the buffer is zeroed beforehand (padding)
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int S2 = S * S;
    if (tid >= (int64_t)N * nsv * S2) return;
    int g = (int)(tid / ((int64_t)nsv * S2));
    int rem = (int)(tid % ((int64_t)nsv * S2));
    int sv = rem / S2, t = rem % S2;
    int si = sv / nsvx, sj = sv % nsvx;
    int i = si * S + t / S, j = sj * S + t % S;
    if (i >= G.ny || j >= G.nx) return;
    int v0 = view_off[g], Vg = view_off[g + 1] - v0;
    const uint32_t *bd = band + (int64_t)nsv * v0 + (int64_t)sv * Vg;
    int64_t gsv = (int64_t)g * nsv + sv;
    uint8_t *col = cols + sv_base[gsv] + col_off[gsv * (S2 + 1) + t];
    const int vb = (int)sizeof(T);
    // pass 1: the three-channel count fixes where the third values go
    int n3 = 0;
    for (int v = 0; v < Vg; ++v) {
        int c0;
        n3 += footprint_dev(G, cs[v0 + v].x, cs[v0 + v].y, i, j, c0, nullptr) == 3;
    }
    *(uint16_t *)col = (uint16_t)n3;
    T *v01 = (T *)(col + col_v01(Vg));
    uint16_t *ovc = (uint16_t *)(col + col_ovc(Vg, vb));
    T *ov = (T *)(col + col_ovv(Vg, vb, n3));
    int k3 = 0;
    for (int v = 0; v < Vg; ++v) {
        double a[3];
        int c0;
        const int L = footprint_dev(G, cs[v0 + v].x, cs[v0 + v].y, i, j, c0, a);
        const int r = L > 0 ? c0 - (int)(bd[v] & 0xFFFFu) : 0;
        col[2 + v] = (uint8_t)(r | L << 6);
        v01[2 * v] = from_double<T>(L > 0 ? a[0] : 0.0);
        v01[2 * v + 1] = from_double<T>(L > 1 ? a[1] : 0.0);
        if (L == 3) {
            ovc[k3] = (uint16_t)((r + 2) * vpad + v);
            ov[k3] = from_double<T>(a[2]);
            ++k3;
        }
    }
}

static int check_geometry(const mace_geometry *g)
{
    if (!g) return fail(MACE_EINVAL, "geometry is NULL");
    if (g->nx < 1 || g->ny < 1 || g->nz < 1 || g->n_views < 1 || g->n_channels < 1)
        return fail(MACE_EINVAL, "geometry sizes must be positive");
    if (g->n_views > kMaxViews) return fail(MACE_EINVAL, "more than 4096 views");
    if (g->n_channels > 65535) return fail(MACE_EINVAL, "more than 65535 channels");
    if (!(g->pixel_pitch > 0) || !(g->channel_pitch > 0) || !std::isfinite(g->channel_offset))
        return fail(MACE_EINVAL, "pitches must be positive and finite");
    // runs of at most 3 channels: footprint width dx(|cos|+|sin|)/dd <= sqrt(2) dx/dd <= 2
    if (g->pixel_pitch * std::sqrt(2.0) > 2.0 * g->channel_pitch)
        return fail(MACE_EINVAL, "channel_pitch must be >= pixel_pitch / sqrt(2)");
    if (g->nz != 1) return fail(MACE_EINVAL, "only nz == 1 (2D) is supported");
    return MACE_OK;
}

extern "C" int mace_build_sysmatrix(const mace_geometry *geom, const mace_partition *part,
                                    mace_dtype dtype, int32_t sv_size, void *cuda_stream,
                                    mace_sysmatrix **out)
{
    NvtxRange nvtx_range("mace_build_sysmatrix");
    if (!out) return fail(MACE_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_geometry(geom);
    if (rc) return rc;
    if (!part || part->n_agents < 1 || part->n_agents > geom->n_views)
        return fail(MACE_EINVAL, "n_agents must be in [1, n_views]");
    if (sv_size != 4 && sv_size != 8 && sv_size != 16 && sv_size != 32)
        return fail(MACE_EINVAL, "sv_size must be 4, 8, 16 or 32");
    if (dtype != MACE_F32 && dtype != MACE_BF16 && dtype != MACE_F16)
        return fail(MACE_EINVAL, "unknown dtype");

    mace_sysmatrix *M = new mace_sysmatrix();
    M->geo = GeoParams{geom->nx, geom->ny, geom->n_channels, geom->pixel_pitch, geom->channel_pitch,
                       geom->channel_offset};
    M->nz = geom->nz;
    M->V = geom->n_views;
    M->N = part->n_agents;
    M->S = sv_size;
    M->S2 = sv_size * sv_size;
    M->nsvx = (geom->nx + sv_size - 1) / sv_size;
    M->nsvy = (geom->ny + sv_size - 1) / sv_size;
    M->nsv = M->nsvx * M->nsvy;
    M->dtype = dtype;
    M->vbytes = dtype == MACE_F32 ? 4 : 2;
    M->stream = (cudaStream_t)cuda_stream;
    M->view_agent.resize(M->V);
    for (int m = 0; m < M->V; ++m) {
        int g = part->view_agent ? part->view_agent[m] : m % M->N;
        if (g < 0 || g >= M->N) { delete M; return fail(MACE_EINVAL, "view_agent out of range"); }
        M->view_agent[m] = g;
    }
    M->view_off.assign(M->N + 1, 0);
    for (int m = 0; m < M->V; ++m) M->view_off[M->view_agent[m] + 1]++;
    for (int g = 0; g < M->N; ++g) {
        if (M->view_off[g + 1] == 0) { delete M; return fail(MACE_EINVAL, "an agent has no views"); }
        M->view_off[g + 1] += M->view_off[g];
    }
    M->agent_views.resize(M->V);
    {
        std::vector<int> fillp(M->view_off.begin(), M->view_off.end() - 1);
        for (int m = 0; m < M->V; ++m) M->agent_views[fillp[M->view_agent[m]]++] = m;
    }
    M->max_views = 0;
    for (int g = 0; g < M->N; ++g) M->max_views = std::max(M->max_views, M->view_off[g + 1] - M->view_off[g]);
    // view angles on the host (libm), in agent order
    M->cosv.resize(M->V);
    M->sinv.resize(M->V);
    std::vector<double2> cs(M->V);
    for (int m = 0; m < M->V; ++m) {
        double th = geom->view_angles ? geom->view_angles[m] : (double)m * M_PI / (double)M->V;
        if (!std::isfinite(th)) { delete M; return fail(MACE_EINVAL, "non-finite view angle"); }
        M->cosv[m] = cos(th);
        M->sinv[m] = sin(th);
    }
    for (int k = 0; k < M->V; ++k) cs[k] = make_double2(M->cosv[M->agent_views[k]], M->sinv[M->agent_views[k]]);

    auto cleanup = [&](int code, const std::string &msg) {
        mace_free_sysmatrix(M);
        return fail(code, msg);
    };
    cudaStream_t s = M->stream;
    const int64_t nband = (int64_t)M->nsv * M->V;
    const int64_t ncol = (int64_t)M->N * M->nsv * M->S2;
    std::vector<ViewGeo> vg(M->V);
    for (int k = 0; k < M->V; ++k) {
        const GeoParams &G = M->geo;
        const double ct = cs[k].x, st = cs[k].y;
        const double a = G.dx * fabs(ct) / G.dd, b = G.dx * fabs(st) / G.dd;
        const double w1 = std::min(a, b), w2 = std::max(a, b);
        const double xc = (0.0 - 0.5 * (double)(G.nx - 1)) * G.dx, yc = 0.5 * (double)(G.ny - 1) * G.dx;
        vg[k].q00 = (xc * ct + yc * st - G.off) / G.dd + 0.5 * (double)G.D;
        vg[k].cq = G.dx * ct / G.dd;
        vg[k].sq = G.dx * st / G.dd;
        vg[k].u1 = (float)(0.5 * (w2 - w1));
        vg[k].u2 = (float)(0.5 * (w2 + w1));
        vg[k].h = (float)(1.0 / w2);
        vg[k].k2 = w1 > 0.0 ? (float)(1.0 / (w2 * 2.0 * w1)) : 0.f;
        vg[k].w1 = (float)w1;
        vg[k].half = (float)(0.5 * (a + b));
        vg[k].scale = (float)(G.dx * G.dx / G.dd);
    }
    if (cudaMalloc(&M->d_vgeo, sizeof(ViewGeo) * M->V) != cudaSuccess ||
        cudaMalloc(&M->d_cs, sizeof(double2) * M->V) != cudaSuccess ||
        cudaMalloc(&M->d_view_off, sizeof(int) * (M->N + 1)) != cudaSuccess ||
        cudaMalloc(&M->d_band, sizeof(uint32_t) * nband) != cudaSuccess ||
        cudaMalloc(&M->d_sv_base, sizeof(int64_t) * M->N * M->nsv) != cudaSuccess ||
        cudaMalloc(&M->d_col_off, sizeof(uint32_t) * M->N * M->nsv * (M->S2 + 1)) != cudaSuccess)
        return cleanup(MACE_ENOMEM, "cudaMalloc failed for system-matrix metadata");
    if (cudaMemcpyAsync(M->d_cs, cs.data(), sizeof(double2) * M->V, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(M->d_vgeo, vg.data(), sizeof(ViewGeo) * M->V, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(M->d_view_off, M->view_off.data(), sizeof(int) * (M->N + 1), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return cleanup(MACE_ECUDA, "copy of view tables failed");

    band_kernel<<<(unsigned)((nband + 255) / 256), 256, 0, s>>>(M->geo, M->d_cs, M->d_view_off, M->N, M->S,
                                                               M->nsvx, M->nsv, M->d_band);
    uint32_t *d_bytes = nullptr, *d_nnz = nullptr, *d_n3 = nullptr;
    if (cudaMalloc(&d_bytes, sizeof(uint32_t) * ncol) != cudaSuccess ||
        cudaMalloc(&d_nnz, sizeof(uint32_t) * ncol) != cudaSuccess ||
        cudaMalloc(&d_n3, sizeof(uint32_t) * ncol) != cudaSuccess) {
        cudaFree(d_bytes);
        cudaFree(d_nnz);
        return cleanup(MACE_ENOMEM, "cudaMalloc failed for column sizes");
    }
    colsize_kernel<<<(unsigned)((ncol + 255) / 256), 256, 0, s>>>(M->geo, M->d_cs, M->d_view_off, M->N, M->S,
                                                                  M->nsvx, M->nsv, M->vbytes, d_bytes, d_nnz, d_n3);
    std::vector<uint32_t> h_bytes(ncol), h_nnz(ncol), h_n3(ncol), h_band(nband);
    cudaError_t ce = cudaMemcpyAsync(h_bytes.data(), d_bytes, sizeof(uint32_t) * ncol, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_nnz.data(), d_nnz, sizeof(uint32_t) * ncol, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_n3.data(), d_n3, sizeof(uint32_t) * ncol, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h_band.data(), M->d_band, sizeof(uint32_t) * nband, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(d_bytes);
    cudaFree(d_nnz);
    cudaFree(d_n3);
    if (ce != cudaSuccess) return cleanup(MACE_ECUDA, std::string("system-matrix size pass: ") + cudaGetErrorString(ce));

    // offsets (host prefix sums; a one-off cost per geometry)
    std::vector<int64_t> sv_base(M->N * M->nsv);
    std::vector<uint32_t> col_off((int64_t)M->N * M->nsv * (M->S2 + 1));
    int64_t total = 0;
    int max_len = 1;
    M->max_col_bytes = 16;
    M->agent_bytes.assign(M->N, 0);
    for (int g = 0; g < M->N; ++g) {
        int Vg = M->view_off[g + 1] - M->view_off[g];
        for (int sv = 0; sv < M->nsv; ++sv) {
            int64_t gsv = (int64_t)g * M->nsv + sv;
            sv_base[gsv] = total;
            uint32_t off = 0;
            for (int t = 0; t < M->S2; ++t) {
                col_off[gsv * (M->S2 + 1) + t] = off;
                uint32_t b = h_bytes[gsv * M->S2 + t];
                off += b;
                M->max_col_bytes = std::max<int>(M->max_col_bytes, (int)b);
                M->max_n3 = std::max<int>(M->max_n3, (int)h_n3[gsv * M->S2 + t]);
                M->nnz += h_nnz[gsv * M->S2 + t];
            }
            col_off[gsv * (M->S2 + 1) + M->S2] = off;
            total += off;
            M->agent_bytes[g] += off;
            const uint32_t *bd = h_band.data() + (int64_t)M->nsv * M->view_off[g] + (int64_t)sv * Vg;
            for (int v = 0; v < Vg; ++v) max_len = std::max(max_len, (int)(bd[v] >> 16));
        }
    }
    // band rows: one spare past the widest band (a run's second entry may sit
    // there); run offsets are stored in 6 bits
    if (max_len > kMaxRunOff - 1)
        return cleanup(MACE_EINVAL, "super-voxel band wider than 62 channels in a view; use a smaller sv_size");
    M->wmax = max_len + 1;
    M->vpad = (M->max_views + 15) & ~15;
    if ((int64_t)M->vpad * M->wmax > 65535)
        return cleanup(MACE_EINVAL, "super-voxel band of an agent larger than 65535 entries; use fewer views per agent");
    M->bytes_cols = total;
    if (cudaMalloc(&M->d_cols, total > 0 ? total : 16) != cudaSuccess)
        return cleanup(MACE_ENOMEM, "cudaMalloc failed for the system matrix (" + std::to_string(total) + " bytes)");
    ce = cudaMemcpyAsync(M->d_sv_base, sv_base.data(), sizeof(int64_t) * sv_base.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(M->d_col_off, col_off.data(), sizeof(uint32_t) * col_off.size(), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(M->d_cols, 0, total > 0 ? total : 16, s);
    if (ce != cudaSuccess) return cleanup(MACE_ECUDA, std::string("system-matrix upload: ") + cudaGetErrorString(ce));
    const unsigned fb = (unsigned)((ncol + 127) / 128);
    if (M->dtype == MACE_F32)
        fill_kernel<float><<<fb, 128, 0, s>>>(M->geo, M->d_cs, M->d_view_off, M->N, M->S, M->nsvx, M->nsv, M->vpad,
                                              M->d_band, M->d_sv_base, M->d_col_off, M->d_cols);
    else if (M->dtype == MACE_BF16)
        fill_kernel<__nv_bfloat16><<<fb, 128, 0, s>>>(M->geo, M->d_cs, M->d_view_off, M->N, M->S, M->nsvx, M->nsv,
                                                      M->vpad, M->d_band, M->d_sv_base, M->d_col_off, M->d_cols);
    else
        fill_kernel<__half><<<fb, 128, 0, s>>>(M->geo, M->d_cs, M->d_view_off, M->N, M->S, M->nsvx, M->nsv, M->vpad,
                                               M->d_band, M->d_sv_base, M->d_col_off, M->d_cols);
    ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    if (ce != cudaSuccess) return cleanup(MACE_ECUDA, std::string("system-matrix build: ") + cudaGetErrorString(ce));
    *out = M;
    return MACE_OK;
}

extern "C" int mace_sysmatrix_get_info(const mace_sysmatrix *M, mace_sysmatrix_info *info)
{
    if (!M || !info) return fail(MACE_EINVAL, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_voxels = (int64_t)M->geo.nx * M->geo.ny;
    info->n_agents = M->N;
    info->sv_size = M->S;
    info->n_sv = M->nsv;
    info->max_views = M->max_views;
    info->nnz = M->nnz;
    info->bytes_columns = M->bytes_cols;
    info->bytes_meta = (int64_t)M->nsv * M->V * 4 + (int64_t)M->N * M->nsv * (8 + 4 * (M->S2 + 1));
    for (int g = 0; g < M->N && g < 64; ++g) info->agent_bytes[g] = M->agent_bytes[g];
    return MACE_OK;
}

static float value_to_float(const uint8_t *p, mace_dtype dt)
{
    if (dt == MACE_F32) { float f; memcpy(&f, p, 4); return f; }
    uint16_t u; memcpy(&u, p, 2);
    if (dt == MACE_BF16) { uint32_t b = (uint32_t)u << 16; float f; memcpy(&f, &b, 4); return f; }
    // IEEE half -> float
    uint32_t sgn = (u >> 15) & 1, ex = (u >> 10) & 0x1F, man = u & 0x3FF;
    float f;
    if (ex == 0) f = std::ldexp((float)man, -24);
    else if (ex == 31) f = man ? NAN : INFINITY;
    else f = std::ldexp((float)(man | 0x400), (int)ex - 25);
    return sgn ? -f : f;
}

extern "C" int mace_sysmatrix_column(const mace_sysmatrix *M, int32_t g, int32_t i, int32_t j,
                                     int32_t *c0, int32_t *len, float *vals)
{
    if (!M || !c0 || !len || !vals) return fail(MACE_EINVAL, "NULL argument");
    if (g < 0 || g >= M->N || i < 0 || i >= M->geo.ny || j < 0 || j >= M->geo.nx)
        return fail(MACE_EINVAL, "column index out of range");
    int sv = (i / M->S) * M->nsvx + (j / M->S);
    int t = (i % M->S) * M->S + (j % M->S);
    int64_t gsv = (int64_t)g * M->nsv + sv;
    int Vg = M->view_off[g + 1] - M->view_off[g];
    int64_t base;
    uint32_t off[2];
    std::vector<uint32_t> bd(Vg);
    CUDA_TRY(cudaMemcpy(&base, M->d_sv_base + gsv, sizeof(int64_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(off, M->d_col_off + gsv * (M->S2 + 1) + t, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(bd.data(), M->d_band + (int64_t)M->nsv * M->view_off[g] + (int64_t)sv * Vg,
                        sizeof(uint32_t) * Vg, cudaMemcpyDeviceToHost));
    std::vector<uint8_t> col(off[1] - off[0]);
    if (!col.empty())
        CUDA_TRY(cudaMemcpy(col.data(), M->d_cols + base + off[0], col.size(), cudaMemcpyDeviceToHost));
    for (int v = 0; v < Vg; ++v) { c0[v] = 0; len[v] = 0; vals[3 * v] = vals[3 * v + 1] = vals[3 * v + 2] = 0.f; }
    if (col.empty()) return MACE_OK;
    const int vb = M->vbytes;
    uint16_t n3;
    memcpy(&n3, col.data(), 2);
    if (col_bytes(Vg, vb, n3) != col.size()) return fail(MACE_EINVAL, "stored column has an inconsistent size");
    const uint8_t *v01 = col.data() + col_v01(Vg);
    const uint8_t *ovc = col.data() + col_ovc(Vg, vb);
    const uint8_t *ov = col.data() + col_ovv(Vg, vb, n3);
    int k3 = 0;
    for (int v = 0; v < Vg; ++v) {
        const int hb = col[2 + v], r = hb & 63, L = hb >> 6;
        len[v] = L;
        if (L == 0) continue;
        const int lo = (int)(bd[v] & 0xFFFFu), blen = (int)(bd[v] >> 16);
        if (r + L > blen) return fail(MACE_EINVAL, "stored run leaves its super-voxel band");
        c0[v] = lo + r;
        vals[3 * v] = value_to_float(v01 + (size_t)(2 * v) * vb, M->dtype);
        if (L > 1) vals[3 * v + 1] = value_to_float(v01 + (size_t)(2 * v + 1) * vb, M->dtype);
        if (L == 3) {
            uint16_t code;
            memcpy(&code, ovc + 2 * k3, 2);
            if (k3 >= n3 || code != (uint16_t)((r + 2) * M->vpad + v))
                return fail(MACE_EINVAL, "stored three-channel list does not match the runs");
            vals[3 * v + 2] = value_to_float(ov + (size_t)k3 * vb, M->dtype);
            ++k3;
        }
    }
    if (k3 != n3) return fail(MACE_EINVAL, "stored three-channel list does not match the runs");
    return MACE_OK;
}

extern "C" void mace_free_sysmatrix(mace_sysmatrix *M)
{
    if (!M) return;
    cudaFree(M->d_cs);
    cudaFree(M->d_vgeo);
    cudaFree(M->d_view_off);
    cudaFree(M->d_band);
    cudaFree(M->d_sv_base);
    cudaFree(M->d_col_off);
    cudaFree(M->d_cols);
    delete M;
}

// ---------------------------------------------------------------------------
// reconstruction state
// ---------------------------------------------------------------------------
// Device memory that mace_consensus_noalloc writes the consensus images into
// before copying them to the host.  It is a file-scope array, so every GPU that
// loads this library holds it (4 MiB) until the process exits, and every call
// on that GPU shares it: the last call's images stay in it, and calls whose
// GPU work overlaps (different streams, or different host threads) race on
// it.  In host code its name is only a stand-in for the symbol; mace_init
// looks up the device address (cudaGetSymbolAddress, on the state's device)
// and keeps it in the state.
static constexpr int64_t kNoAllocFloats = (int64_t)1 << 20;
static __device__ __align__(256) float g_noalloc_images[kNoAllocFloats];


// One configuration of the queue-fed sweep for a set of matrices (one state,
// or the states of a group): the kernel for the most views per agent, and a
// shared-memory layout large enough for every one of them.
struct QueueLaunch {
    sweep_queue_fn fn = nullptr;
    int W = 1;                           // warps per super-voxel (a team)
    int K = 1;                           // chains per warp (two slices of a volume)
    int vpad = 0, wmax = 0, col_stride = 16, S = 4;
    int wpb = 1, blocks = 0;
    size_t smem = 0;
};

struct mace_state {
    const mace_sysmatrix *M;
    mace_params P;
    cudaStream_t stream;
    int B;                     // reconstructions in the batch (same geometry)
    int64_t n;                 // voxels of one image
    int64_t ne;                // error-sinogram entries of one reconstruction
    double sigma_abs;
    float2 *d_eL = nullptr;    // (e, Lambda) [B][agents: V_g][D]
    unsigned long long *d_dacc = nullptr;   // changes of e in fixed point (2^-40), same layout
    unsigned *d_phase = nullptr;            // deterministic sweeps: phase counter per (group, agent)
    float *d_y = nullptr;      // y, same layout
    float *d_w = nullptr;      // [B][N][n]
    float *d_X = nullptr;      // [B][N][n]
    float *d_vexp = nullptr;   // [B][N][n] explicit v (prox-pass entry point)
    float *d_theta2 = nullptr; // [B][N][n] sum_{k in J_g} A_ks^2 Lambda_k
    double *d_hbuf = nullptr;  // pnp: [2][B][n] the denoiser's input and its second iterate
    int h_iters = 0;           // pnp: Jacobi iterations of H (even)
    double h_c = 0.0;          // pnp: sigma^2 beta / sigma_x^2
    double *d_wbar = nullptr;  // [B][n]
    double *d_part = nullptr;  // [B][nblk_mann][2] residual partials
    float *noalloc_addr = nullptr;   // device address of g_noalloc_images on the state's device
    double *d_resid = nullptr; // [B][3]: dw2, ww2, r
    int *d_status = nullptr;   // device status word
    std::vector<int32_t> sv_order;   // super-voxel visiting order of a forward pass
    int32_t *d_sv_order = nullptr;
    // optional CUDA-event timing of the sweep launches
    // iterations captured once as a CUDA graph and replayed (explicit streams,
    // timing off); graph_failed: capture was refused, launch eagerly
    cudaGraphExec_t graph_exec = nullptr;
    // non-blocking status: pinned copy of d_resid (3 B doubles) and the
    // status word, and the event that marks its arrival
    double *h_poll = nullptr;
    cudaEvent_t poll_ev = nullptr;
    bool poll_pending = false;
    int graph_iters = 0;
    bool graph_failed = false;
    bool timing = false;
    std::vector<cudaEvent_t> ev;     // pairs (start, stop)
    int ev_used = 0;
    int nblk_mann = 0;
    int iters = 0;
    double last_resid = INFINITY;
    int sweep_warps = 0, sweep_wpb = 0, concurrency = 0, chains = 1;
    // work-queue schedule: descriptors (forward, backward, explicit v),
    // item offsets per z parity ([0, items] twice), item counter
    SweepArgs *d_qtab = nullptr;
    int *d_qoff = nullptr;
    unsigned *d_qcnt = nullptr;
    int q_items[2] = {0, 0};
    QueueLaunch q;
    int wpv = 1;                            // warps per super-voxel (the queue-fed sweep)
    size_t sweep_smem = 0, warp_smem = 0;
};

// --- consensus (G), Mann, residual ------------------------------------------
__global__ void consensus_kernel(const float *__restrict__ w, int B, int N, int64_t n, double *__restrict__ wbar,
                                 float *__restrict__ xout)
{
    // wbar[b][s] = (1/N) sum_g w[b][g][s], FP64, fixed agent order
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)B * n) return;
    int64_t b = k / n, s = k - b * n;
    const float *wb = w + b * N * n;
    double acc = 0.0;
    for (int g = 0; g < N; ++g) acc += (double)wb[(int64_t)g * n + s];
    double m = acc / (double)N;
    if (wbar) wbar[k] = m;
    if (xout) xout[k] = (float)m;
}

__global__ void __launch_bounds__(256) mann_kernel(float *__restrict__ w, const float *__restrict__ X,
                                                   const double *__restrict__ wbar, int N, int64_t n, float rho,
                                                   double *__restrict__ part)
{
    // blockIdx.y = reconstruction b
    __shared__ double sh[2][8];
    const int64_t b = blockIdx.y;
    float *wb = w + b * N * n;
    const float *Xb = X + b * N * n;
    const double *wbarb = wbar + b * n;
    double d2 = 0.0, w2 = 0.0;
    const int64_t total = (int64_t)N * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
        int64_t s = k % n;
        float wo = wb[k];
        float v = (float)(2.0 * wbarb[s] - (double)wo);
        float wn = rho * (2.f * Xb[k] - v) + (1.f - rho) * wo;
        wb[k] = wn;
        double d = (double)wn - (double)wo;
        d2 += d * d;
        w2 += (double)wn * (double)wn;
    }
    for (int o = 16; o > 0; o >>= 1) {
        d2 += __shfl_down_sync(0xffffffffu, d2, o);
        w2 += __shfl_down_sync(0xffffffffu, w2, o);
    }
    int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][wid] = d2; sh[1][wid] = w2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { a += sh[0][k]; c += sh[1][k]; }
        double *pb = part + 2 * (b * gridDim.x + blockIdx.x);
        pb[0] = a;
        pb[1] = c;
    }
}

__global__ void residual_kernel(const double *__restrict__ part, int nblk, int B, double *__restrict__ out)
{
    // block b: reconstruction b's block partials summed in a fixed order (a
    // strided per-thread sum, then a fixed tree), deterministic
    __shared__ double sh[2][256];
    const int b = blockIdx.x;
    if (b >= B) return;
    const double *pb = part + 2 * (int64_t)b * nblk;
    double a = 0.0, c = 0.0;
    for (int k = threadIdx.x; k < nblk; k += blockDim.x) { a += pb[2 * k]; c += pb[2 * k + 1]; }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = c;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        a = sh[0][0];
        c = sh[1][0];
        out[3 * b] = a;
        out[3 * b + 1] = c;
        out[3 * b + 2] = c > 0.0 ? sqrt(a / c) : sqrt(a);
    }
}

// --- error sinogram: e = y - A X ---------------------------------------------
// Per-warp shared memory of the kernels below: the super-voxel's band
// descriptors and one float per band entry (rows of vpad views).
struct AuxSmem {
    uint32_t *bdesc;
    float *acc;
};
__device__ __forceinline__ AuxSmem aux_smem(uint8_t *smem, int vpad, int wmax)
{
    uint8_t *base = smem + (threadIdx.x >> 5) * aux_warp_bytes(vpad, wmax);
    AuxSmem a;
    a.bdesc = (uint32_t *)base;
    a.acc = (float *)(base + ((size_t)vpad * 4 + 15) / 16 * 16);
    return a;
}

// Adds each band entry's accumulated value to the agent's accumulator of
// changes of e (fixed point: the warps' additions sum to the same value in
// any order).  Lane l takes views l, l + 32, ...
__device__ __forceinline__ void flush_band(const AuxSmem &a, int Vg, int vpad, int D, unsigned long long *dg, int lane)
{
    for (int v = lane; v < Vg; v += 32) {
        const uint32_t d = a.bdesc[v];
        const int lo = (int)(d & 0xFFFFu), len = (int)(d >> 16);
        for (int t = 0; t < len; ++t) efix_add(dg + (int64_t)v * D + lo + t, a.acc[t * vpad + v]);
    }
}

template <typename T>
__global__ void __launch_bounds__(256) forward_kernel(const uint8_t *__restrict__ cols, const int64_t *__restrict__ sv_base,
                                                      const uint32_t *__restrict__ col_off, const uint32_t *__restrict__ band,
                                                      const int *__restrict__ view_off, unsigned long long *__restrict__ dacc,
                                                      const float *__restrict__ X, int B, int N, int nsv, int nsvx, int S,
                                                      int nx, int ny, int D, int64_t ne, int vpad, int wmax)
{
    // one warp per (reconstruction, agent, super-voxel): accumulate -A x over
    // the super-voxel's columns in its band, then add the band to e (which
    // holds y on entry).  Lane l takes the runs of views l, l + 32, ... and
    // entries l, l + 32, ... of the three-channel list.
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const AuxSmem a = aux_smem(smem, vpad, wmax);
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= (int64_t)B * N * nsv) return;
    const int pair = (int)(item / nsv), sv = (int)(item % nsv);
    const int b = pair / N, g = pair - b * N;
    const int si = sv / nsvx, sj = sv % nsvx, S2 = S * S;
    const int v0 = view_off[g], Vg = view_off[g + 1] - v0;
    const int64_t gsv = (int64_t)g * nsv + sv;
    const uint8_t *svcols = cols + sv_base[gsv];
    const uint32_t *coff = col_off + gsv * (S2 + 1);
    const float *Xg = X + (int64_t)pair * nx * ny;
    const int vb = (int)sizeof(T), v01 = col_v01(Vg), ovc = col_ovc(Vg, vb);
    const uint32_t *bd = band + (int64_t)nsv * v0 + (int64_t)sv * Vg;
    for (int v = lane; v < Vg; v += 32) a.bdesc[v] = bd[v];
    for (int f = lane; f < wmax * vpad; f += 32) a.acc[f] = 0.f;
    __syncwarp();
    for (int t = 0; t < S2; ++t) {
        if (coff[t + 1] == coff[t]) continue;
        const int i = si * S + t / S, j = sj * S + t % S;
        const float xs = Xg[(int64_t)i * nx + j];
        if (xs == 0.f) continue;
        const uint8_t *col = svcols + coff[t];
        const int n3 = *(const uint16_t *)col;
        for (int v = lane; v < Vg; v += 32) {
            const int r = col[2 + v] & 63;
            const float2 av = ld_pair<T>(col + v01, v);
            a.acc[r * vpad + v] = fmaf(-av.x, xs, a.acc[r * vpad + v]);
            a.acc[(r + 1) * vpad + v] = fmaf(-av.y, xs, a.acc[(r + 1) * vpad + v]);
        }
        const uint8_t *ov = col + col_ovv(Vg, vb, n3);
        for (int k = lane; k < n3; k += 32) {
            const int code = ((const uint16_t *)(col + ovc))[k];
            a.acc[code] = fmaf(-ld_val<T>(ov, k), xs, a.acc[code]);
        }
        __syncwarp();
    }
    flush_band(a, Vg, vpad, D, dacc + (int64_t)b * ne + (int64_t)v0 * D, lane);
}

// The same product with A evaluated from the geometry instead of read from
// the stored columns: the periodic recompute that removes drift (Sec. II-C)
// then sees the exact projector even when the stored values are BF16/FP16.
// One warp per (reconstruction, agent, super-voxel); lane l takes views
// l, l + 32, ... of the agent, so the lanes write disjoint runs of the band.
// The projection of the super-voxel's first pixel is formed in FP64, the
// offsets inside the super-voxel and the trapezoid in FP32 (position error
// ~1e-6 channel).  Channels outside the stored band (values at round-off
// level on a footprint's edge) are dropped.
__device__ __forceinline__ float trap_cdf_f(float u, const ViewGeo &G)
{
    if (u <= -G.u2) return 0.f;
    if (u < -G.u1) {
        const float d = u + G.u2;
        return G.k2 * d * d;
    }
    if (u <= G.u1) return G.h * (0.5f * G.w1 + (u + G.u1));
    if (u < G.u2) {
        const float d = G.u2 - u;
        return 1.f - G.k2 * d * d;
    }
    return 1.f;
}

__global__ void __launch_bounds__(256) forward_geometry_kernel(const ViewGeo *__restrict__ vgeo,
                                                               const uint32_t *__restrict__ band,
                                                               const int *__restrict__ view_off,
                                                               unsigned long long *__restrict__ dacc,
                                                               const float *__restrict__ X, int B, int N, int nsv, int nsvx,
                                                               int S, int nx, int ny, int D, int64_t ne, int vpad, int wmax)
{
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const AuxSmem a = aux_smem(smem, vpad, wmax);
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= (int64_t)B * N * nsv) return;
    const int pair = (int)(item / nsv), sv = (int)(item % nsv);
    const int b = pair / N, g = pair - b * N;
    const int i0 = (sv / nsvx) * S, j0 = (sv % nsvx) * S, S2 = S * S;
    const int v0 = view_off[g], Vg = view_off[g + 1] - v0;
    const float *Xg = X + (int64_t)pair * nx * ny;
    const uint32_t *bd = band + (int64_t)nsv * v0 + (int64_t)sv * Vg;
    for (int v = lane; v < Vg; v += 32) a.bdesc[v] = bd[v];
    for (int f = lane; f < wmax * vpad; f += 32) a.acc[f] = 0.f;
    __syncwarp();
    for (int v = lane; v < Vg; v += 32) {
        const int lo_v = (int)(a.bdesc[v] & 0xFFFFu), len_v = (int)(a.bdesc[v] >> 16);
        if (len_v == 0) continue;
        const ViewGeo G = vgeo[v0 + v];
        const double q0 = fma((double)j0, G.cq, fma(-(double)i0, G.sq, G.q00));
        const double qb = floor(q0);
        const int qi = (int)qb;
        const float qf = (float)(q0 - qb), cqf = (float)G.cq, sqf = (float)G.sq;
        for (int t = 0; t < S2; ++t) {
            const int ti = t / S, tj = t - ti * S;
            if (i0 + ti >= ny || j0 + tj >= nx) continue;
            const float xs = Xg[(int64_t)(i0 + ti) * nx + j0 + tj];
            if (xs == 0.f) continue;
            const float q = qf + fmaf((float)tj, cqf, -(float)ti * sqf);
            const int cf = (int)floorf(q - G.half);
            float prev = trap_cdf_f((float)cf - q, G);
            for (int k = 0; k < 4; ++k) {
                const int c = cf + k;
                if ((float)c >= q + G.half) break;
                const float next = trap_cdf_f((float)(c + 1) - q, G);
                const int ch = qi + c;
                if (ch >= lo_v && ch < lo_v + len_v) {
                    float *ap = &a.acc[(ch - lo_v) * vpad + v];
                    *ap = fmaf(-G.scale * (next - prev), xs, *ap);
                }
                prev = next;
            }
        }
    }
    __syncwarp();
    flush_band(a, Vg, vpad, D, dacc + (int64_t)b * ne + (int64_t)v0 * D, lane);
}

__global__ void pack_kernel(const float *__restrict__ y, const float *__restrict__ lam, const int *__restrict__ agent_view,
                            int B, int V, int D, float2 *__restrict__ eL, float *__restrict__ yg)
{
    // agent-ordered row k of reconstruction b holds view agent_view[k]
    int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t per = (int64_t)V * D;
    if (tid >= (int64_t)B * per) return;
    int64_t b = tid / per, r = tid - b * per;
    int k = (int)(r / D), c = (int)(r % D);
    int m = agent_view[k];
    int64_t src = b * per + (int64_t)m * D + c;
    float yy = y[src];
    eL[tid] = make_float2(yy, lam[src]);
    yg[tid] = yy;
}

__global__ void reset_error_kernel(const float *__restrict__ yg, float2 *__restrict__ eL,
                                   unsigned long long *__restrict__ dacc, int64_t ne)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ne) {
        eL[k].x = yg[k];
        dacc[k] = 0ull;
    }
}

// e += the accumulated changes (one rounding per entry), accumulator cleared
__global__ void fold_error_kernel(float2 *__restrict__ eL, unsigned long long *__restrict__ dacc, int64_t ne)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < ne) {
        const unsigned long long q = dacc[k];
        if (q != 0ull) {
            eL[k].x += efix_value(q);
            dacc[k] = 0ull;
        }
    }
}

// Sum of m doubles in a fixed order (one block: strided partial sums, then a
// fixed tree), so the result does not depend on scheduling
__global__ void sum_fixed_kernel(const double *__restrict__ x, int64_t m, double *__restrict__ out)
{
    __shared__ double sh[1024];
    double a = 0.0;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) a += x[k];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

__global__ void broadcast_kernel(const double *__restrict__ wbar, float *__restrict__ X, int B, int N, int64_t n)
{
    // X[b][g][s] = wbar[b][s]
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (int64_t)B * N * n) return;
    int64_t b = k / ((int64_t)N * n);
    X[k] = (float)wbar[b * n + k % n];
}

__global__ void check_weights_kernel(const float *__restrict__ y, const float *__restrict__ lam, int64_t m, int *bad)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= m) return;
    float a = y[k], b = lam[k];
    if (!isfinite(a) || !isfinite(b) || b < 0.f) atomicOr(bad, 1);
}

template <typename T>
__global__ void theta2_kernel(const uint8_t *__restrict__ cols, const int64_t *__restrict__ sv_base,
                              const uint32_t *__restrict__ col_off, const uint32_t *__restrict__ band,
                              const int *__restrict__ view_off, const float2 *__restrict__ eL, int B, int N, int nsv,
                              int nsvx, int S, int nx, int ny, int D, int64_t ne, int vpad, int wmax,
                              float *__restrict__ theta2, double *__restrict__ part)
{
    // theta2[b][g][s] = sum_{k in J_g} A_ks^2 Lambda_k (the data term of the
    // coordinate curvature in Algorithm 2, constant over the iterations),
    // accumulated in FP64 and stored in FP32; zero for pixels without a
    // column.  part[item] = the FP64 sum over the warp's pixels (summed in a
    // fixed order afterwards, for the normalised sigma).  One warp per (b,
    // agent, super-voxel).
    extern __shared__ __align__(16) uint8_t smem[];
    const int lane = threadIdx.x & 31;
    const AuxSmem a = aux_smem(smem, vpad, wmax);
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= (int64_t)B * N * nsv) return;
    const int pair = (int)(item / nsv), sv = (int)(item % nsv), S2 = S * S;
    const int b = pair / N, g = pair - b * N;
    const int si = sv / nsvx, sj = sv % nsvx;
    const int v0 = view_off[g], Vg = view_off[g + 1] - v0;
    const int64_t gsv = (int64_t)g * nsv + sv;
    const uint32_t *coff = col_off + gsv * (S2 + 1);
    const float2 *lg = eL + (int64_t)b * ne + (int64_t)v0 * D;
    float *t2g = theta2 + (int64_t)pair * nx * ny;
    const int vb = (int)sizeof(T), v01 = col_v01(Vg), ovc = col_ovc(Vg, vb);
    const uint32_t *bd = band + (int64_t)nsv * v0 + (int64_t)sv * Vg;
    for (int v = lane; v < Vg; v += 32) a.bdesc[v] = bd[v];
    __syncwarp();
    double sum = 0.0;
    for (int t = 0; t < S2; ++t) {
        const int i = si * S + t / S, j = sj * S + t % S;
        if (i >= ny || j >= nx) continue;
        double acc = 0.0;
        if (coff[t + 1] != coff[t]) {
            const uint8_t *col = cols + sv_base[gsv] + coff[t];
            const int n3 = *(const uint16_t *)col;
            for (int v = lane; v < Vg; v += 32) {
                const int hb = col[2 + v], r = hb & 63, L = hb >> 6;
                const float2 av = ld_pair<T>(col + v01, v);
                const int64_t e0 = (int64_t)v * D + (a.bdesc[v] & 0xFFFFu) + r;
                if (L > 0) acc += (double)av.x * av.x * lg[e0].y;
                if (L > 1) acc += (double)av.y * av.y * lg[e0 + 1].y;
            }
            const uint8_t *ov = col + col_ovv(Vg, vb, n3);
            for (int k = lane; k < n3; k += 32) {
                const int code = ((const uint16_t *)(col + ovc))[k];
                const int v = code % vpad, row = code / vpad;
                const float a2 = ld_val<T>(ov, k);
                acc += (double)a2 * a2 * lg[(int64_t)v * D + (a.bdesc[v] & 0xFFFFu) + row].y;
            }
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        }
        if (lane == 0) t2g[(int64_t)i * nx + j] = (float)acc;
        sum += acc;
    }
    if (lane == 0) part[item] = sum;
}

// One Jacobi iteration of the plug-and-play denoiser H (Algorithm 3): the
// proximal map of the quadratic prior, x = (I + c B)^-1 v with
// (B x)_s = sum_r b_sr (x_s - x_r) (8-neighbourhood, b_sr ~ 1/distance summing
// to 1, out-of-image neighbours dropped, c = sigma^2 beta / sigma_x^2):
// x_s <- (v_s + c sum_r b_sr x_r) / (1 + c sum_r b_sr).  FP64.
__global__ void prior_prox_jacobi_kernel(const double *__restrict__ v, const double *__restrict__ xin,
                                         double *__restrict__ xout, int B, int nx, int ny, double c,
                                         double b_edge, double b_diag)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n = (int64_t)nx * ny;
    if (k >= (int64_t)B * n) return;
    const int64_t b = k / n, s = k - b * n;
    const int i = (int)(s / nx), j = (int)(s % nx);
    const double *xb = xin + b * n;
    double acc = 0.0, bs = 0.0;
    for (int di = -1; di <= 1; ++di)
        for (int dj = -1; dj <= 1; ++dj) {
            if (!di && !dj) continue;
            const int ii = i + di, jj = j + dj;
            if (ii < 0 || ii >= ny || jj < 0 || jj >= nx) continue;
            const double w = (di && dj) ? b_diag : b_edge;
            acc += w * xb[(int64_t)ii * nx + jj];
            bs += w;
        }
    xout[k] = (v[k] + c * acc) / (1.0 + c * bs);
}

__global__ void to_float_kernel(const double *__restrict__ x, float *__restrict__ out, int64_t m)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < m) out[k] = (float)x[k];
}

// Bounded-wait self test: one warp arms an mbarrier for bytes that are never
// sent and waits on it with the sweep's bounded spin (limit given); on expiry
// it records MACE_ETIMEOUT in the status word and returns, as the sweep does.
__global__ void wait_selftest_kernel(uint32_t spin_limit, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&bar, 16);
    }
    __syncwarp();
    uint32_t spins = 0;
    while (!mbar_try_wait(&bar, 0)) {
        if (++spins > spin_limit) {
            if (threadIdx.x == 0) atomicExch(status, kStatusTimeout);
            return;
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T>
static void launch_forward_t(mace_state *st, unsigned blocks)
{
    const mace_sysmatrix *M = st->M;
    const size_t sm = 8 * aux_warp_bytes(M->vpad, M->wmax);
    cudaFuncSetAttribute(forward_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    forward_kernel<T><<<blocks, 256, sm, st->stream>>>(M->d_cols, M->d_sv_base, M->d_col_off, M->d_band, M->d_view_off,
                                                       st->d_dacc, st->d_X, st->B, M->N, M->nsv, M->nsvx, M->S, M->geo.nx,
                                                       M->geo.ny, M->geo.D, st->ne, M->vpad, M->wmax);
}

// e_i = y_i - A_i X_i for every reconstruction and agent
static int launch_forward(mace_state *st)
{
    NvtxRange nvtx_range("e recompute");
    const mace_sysmatrix *M = st->M;
    int64_t items = (int64_t)st->B * M->N * M->nsv;
    unsigned blocks = (unsigned)((items * 32 + 255) / 256);
    int64_t tot = (int64_t)st->B * st->ne;
    reset_error_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st->stream>>>(st->d_y, st->d_eL, st->d_dacc, tot);
    // forward_geometry 0 (auto): from the geometry when the stored values are
    // rounded (BF16/FP16), from the stored values when they are FP32
    const bool geo = st->P.forward_geometry == 1 || (st->P.forward_geometry == 0 && M->dtype != MACE_F32);
    if (geo) {
        const size_t sm = 8 * aux_warp_bytes(M->vpad, M->wmax);
        cudaFuncSetAttribute(forward_geometry_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        forward_geometry_kernel<<<blocks, 256, sm, st->stream>>>(M->d_vgeo, M->d_band, M->d_view_off, st->d_dacc, st->d_X,
                                                                 st->B, M->N, M->nsv, M->nsvx, M->S, M->geo.nx,
                                                                 M->geo.ny, M->geo.D, st->ne, M->vpad, M->wmax);
    } else {
        switch (M->dtype) {
        case MACE_F32: launch_forward_t<float>(st, blocks); break;
        case MACE_BF16: launch_forward_t<__nv_bfloat16>(st, blocks); break;
        default: launch_forward_t<__half>(st, blocks); break;
        }
    }
    // e = y - A X: the products were summed in fixed point (any order)
    fold_error_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st->stream>>>(st->d_eL, st->d_dacc, tot);
    CUDA_TRY(cudaGetLastError());
    return MACE_OK;
}

static sweep_fn sweep_kernel_ptr(const mace_sysmatrix *M, int K, bool nb26, bool det)
{
    switch (M->dtype) {
    case MACE_F32: return mace_sweep_kernel_f32(M->max_views, K, nb26, det);
    case MACE_BF16: return mace_sweep_kernel_bf16(M->max_views, K, nb26, det);
    default: return mace_sweep_kernel_f16(M->max_views, K, nb26, det);
    }
}

// The sweep's arguments for this state (one pass, forward or backward, with
// v formed from the consensus or given explicitly).
static SweepArgs sweep_args(const mace_state *st, int backward, const float *vexp)
{
    const mace_sysmatrix *M = st->M;
    SweepArgs A;
    A.cols = M->d_cols;
    A.sv_base = M->d_sv_base;
    A.col_off = M->d_col_off;
    A.band = M->d_band;
    A.view_off = M->d_view_off;
    A.sv_order = st->d_sv_order;
    A.eL = st->d_eL;
    A.X = st->d_X;
    A.w = st->d_w;
    A.wbar = st->d_wbar;
    A.vexp = vexp;
    A.theta2 = st->d_theta2;
    A.status = st->d_status;
    A.B = st->B;
    A.N = M->N;
    A.nsv = M->nsv;
    A.nsvx = M->nsvx;
    A.nx = M->geo.nx;
    A.ny = M->geo.ny;
    A.D = M->geo.D;
    A.S = M->S;
    A.ne = st->ne;
    A.backward = backward;
    A.vpad = M->vpad;
    A.wmax = M->wmax;
    A.col_stride = (M->max_col_bytes + 15) & ~15;
    A.inv_s2 = (float)(1.0 / (st->sigma_abs * st->sigma_abs));
    A.pscale = st->P.pnp ? 0.f : (float)(st->P.beta / (double)M->N);
    if (st->P.pnp)   // data-only agents with proximal parameter sqrt(N) sigma (Algorithm 3)
        A.inv_s2 = (float)(1.0 / ((double)M->N * st->sigma_abs * st->sigma_abs));
    // prior weight constants: the quadratic prior runs the Q-GGMRF formula
    // with a = 0 (inv_Tsx = 0); a Q-GGMRF with q = p = 2 is the quadratic
    // rho(D) = D^2 / (4 sigma_x^2)
    const double isx2 = 1.0 / (st->P.sigma_x * st->P.sigma_x);
    const bool qg = st->P.prior == 1 && st->P.q < st->P.p;
    A.inv_sx2 = (float)((st->P.prior == 1 && !qg) ? 0.5 * isx2 : isx2);
    A.inv_Tsx = qg ? (float)(1.0 / (st->P.T * st->P.sigma_x)) : 0.f;
    A.qexp = qg ? (float)(st->P.p - st->P.q) : 1.f;
    A.half_q_inv_sx2 = qg ? (float)(0.5 * st->P.q * isx2) : 0.f;
    double bsum = 4.0 + 4.0 / std::sqrt(2.0);
    A.b_edge = (float)(1.0 / bsum);
    A.b_diag = (float)((1.0 / std::sqrt(2.0)) / bsum);
    double b3 = 6.0 + 12.0 / std::sqrt(2.0) + 8.0 / std::sqrt(3.0);
    A.b26[0] = (float)(1.0 / b3);
    A.b26[1] = (float)(1.0 / std::sqrt(2.0) / b3);
    A.b26[2] = (float)(1.0 / std::sqrt(3.0) / b3);
    // the fixed schedule's warp count; the work queue's rows per pair
    A.nwarps = st->P.schedule == 1 ? st->concurrency : st->sweep_warps;
    A.phase = st->d_phase;
    A.dacc = st->d_dacc;
    return A;
}

static int launch_sweep_queue(mace_state *st, int backward, const float *vexp);

static int launch_sweep(mace_state *st, int backward, const float *vexp)
{
    NvtxRange nvtx_range("ICD sweep");
    if (st->P.schedule == 1) return launch_sweep_queue(st, backward, vexp);
    const mace_sysmatrix *M = st->M;
    const SweepArgs A = sweep_args(st, backward, vexp);
    dim3 grid((st->sweep_warps + st->sweep_wpb - 1) / st->sweep_wpb), block(32 * st->sweep_wpb);
    const bool rec = st->timing && st->ev_used + 2 <= (int)st->ev.size();
    if (rec) CUDA_TRY(cudaEventRecord(st->ev[st->ev_used], st->stream));
    sweep_fn fn = sweep_kernel_ptr(M, st->chains, st->P.neighbourhood == 26, st->P.deterministic != 0);
    if (!fn) return fail(MACE_EINVAL, "no sweep kernel for this matrix");
    if (st->P.deterministic) {
        // lock-step phases need every warp of a pair resident at once: a
        // cooperative launch guarantees it; the changes of e are folded in
        // after the launch
        const int pairs = (st->B / st->chains) * M->N;
        CUDA_TRY(cudaMemsetAsync(st->d_phase, 0, sizeof(unsigned) * pairs, st->stream));
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = st->sweep_smem;
        cfg.stream = st->stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        CUDA_TRY(cudaLaunchKernelEx(&cfg, fn, A));
        const int64_t tot = (int64_t)st->B * st->ne;
        fold_error_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st->stream>>>(st->d_eL, st->d_dacc, tot);
    } else {
        fn<<<grid, block, st->sweep_smem, st->stream>>>(A);
    }
    if (rec) {
        CUDA_TRY(cudaEventRecord(st->ev[st->ev_used + 1], st->stream));
        st->ev_used += 2;
    }
    CUDA_TRY(cudaGetLastError());
    return MACE_OK;
}

// --- work-queue launches ------------------------------------------------------
static sweep_queue_fn queue_kernel_ptr(mace_dtype dt, int max_views, bool nb26, int W, int K)
{
    switch (dt) {
    case MACE_F32: return mace_sweep_queue_kernel_f32(max_views, nb26, W, K);
    case MACE_BF16: return mace_sweep_queue_kernel_bf16(max_views, nb26, W, K);
    default: return mace_sweep_queue_kernel_f16(max_views, nb26, W, K);
    }
}

// Warps per super-voxel of the queue-fed sweep: the caller's choice, else
// one.  (A team shortens each item's chain of pixel steps, but its warps hold
// more shared memory per view, so fewer items run at once: on the 512^2 and
// 1024^2 scans with 4 to 8 agents it won in some configurations and lost in
// others, so the choice is left to the caller and the autotuner.)
static int resolve_wpv(const mace_params &P)
{
    return P.warps_per_voxel > 0 ? P.warps_per_voxel : 1;
}

static int queue_configure(const mace_sysmatrix *const *Ms, int n, bool nb26, int W, QueueLaunch *L, int K = 1)
{
    L->W = W;
    L->K = K;
    int max_views = 1;
    for (int k = 0; k < n; ++k) {
        const mace_sysmatrix *M = Ms[k];
        if (M->dtype != Ms[0]->dtype) return fail(MACE_EINVAL, "a queue-fed launch needs one stored value type");
        if (M->bytes_cols >= ((int64_t)1 << 36)) return fail(MACE_EINVAL, "stored matrix larger than 64 GiB");
        max_views = std::max(max_views, M->max_views);
        L->vpad = std::max(L->vpad, M->vpad);
        L->wmax = std::max(L->wmax, M->wmax);
        L->col_stride = std::max(L->col_stride, (M->max_col_bytes + 15) & ~15);
        L->S = std::max(L->S, M->S);
    }
    int dev = 0, nsm = 0, max_smem = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const size_t per_warp = warp_smem_layout(L->vpad, L->wmax, L->col_stride, L->S, K, nb26, W).total +
                            ((sizeof(SweepArgs) + 15) & ~(size_t)15);
    if (per_warp > (size_t)max_smem)
        return fail(MACE_EINVAL, "super-voxel working set does not fit in shared memory; use a smaller sv_size");
    // the kernel with enough rounds of views per lane for every matrix; the
    // generic one (decoding each column as it is used) when a column's
    // three-channel list is longer than that kernel's rounds hold
    const int R = sweep_rounds(max_views, K);
    if (R <= 4)
        for (int k = 0; k < n; ++k)
            if (Ms[k]->max_n3 > sweep_ovf_rounds(R, K) * (32 / K)) max_views = 5 * 32 + 1;
    L->fn = queue_kernel_ptr(Ms[0]->dtype, max_views, nb26, W, K);
    if (!L->fn) return fail(MACE_EINVAL, "no queue-fed sweep kernel for this matrix and warps per voxel");
    CUDA_TRY(cudaFuncSetAttribute(L->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    // blocks of whole teams (at most 8 warps: team barriers 1..8)
    int best = 0;
    for (int w = W; w <= 8; w += W) {
        if (per_warp * w > (size_t)max_smem) break;
        int b = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, L->fn, 32 * w, per_warp * w));
        if (b * w > best) { best = b * w; L->wpb = w; L->blocks = b * nsm; }
    }
    if (best < 1) return fail(MACE_EINVAL, "the queue-fed sweep cannot be resident");
    L->smem = per_warp * L->wpb;
    return MACE_OK;
}

// One queue-fed launch over the items of a table of requests: every resident
// warp takes items until none is left (counter zeroed first, on the stream)
static int queue_run(const QueueLaunch &L, const SweepArgs *d_table, const int *d_off, unsigned *d_cnt, int nreq,
                     int total, int zpar, cudaStream_t s)
{
    if (total <= 0) return MACE_OK;
    CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(unsigned), s));
    QueueArgs Q;
    Q.table = d_table;
    Q.offsets = d_off;
    Q.counter = d_cnt;
    Q.nreq = nreq;
    Q.total = total;
    Q.zpar = zpar;
    Q.vpad = L.vpad;
    Q.wmax = L.wmax;
    Q.col_stride = L.col_stride;
    Q.S = L.S;
    L.fn<<<L.blocks, 32 * L.wpb, L.smem, s>>>(Q);
    CUDA_TRY(cudaGetLastError());
    return MACE_OK;
}

// items of one state for z parity p (volumes) or all groups (p < 0)
static int queue_items(const mace_state *st, int p)
{
    const int groups = (p < 0 ? st->B : (st->B - p + 1) / 2) / st->chains;
    return groups * st->M->N * st->concurrency;
}

static int launch_sweep_queue(mace_state *st, int backward, const float *vexp)
{
    const QueueLaunch &L = st->q;
    const bool nb26 = st->P.neighbourhood == 26;
    int rc = MACE_OK;
    const SweepArgs *tab = st->d_qtab + (backward ? 1 : 0);
    if (vexp) {
        // an explicit v (the single-pass entry point): its own descriptor,
        // written in stream order (the pageable source is staged at the call)
        const SweepArgs A = sweep_args(st, backward, vexp);
        CUDA_TRY(cudaMemcpyAsync(st->d_qtab + 2, &A, sizeof(SweepArgs), cudaMemcpyHostToDevice, st->stream));
        tab = st->d_qtab + 2;
    }
    const bool rec = st->timing && st->ev_used + 2 <= (int)st->ev.size();
    if (rec) CUDA_TRY(cudaEventRecord(st->ev[st->ev_used], st->stream));
    if (nb26) {
        // even slices, then odd: a slice's 26-neighbourhood is fixed while it
        // is updated (z-parity phases)
        for (int p = 0; p < 2 && rc == MACE_OK; ++p)
            rc = queue_run(L, tab, st->d_qoff + 2 * p, st->d_qcnt, 1, st->q_items[p], p, st->stream);
    } else {
        rc = queue_run(L, tab, st->d_qoff, st->d_qcnt, 1, st->q_items[0], -1, st->stream);
    }
    if (rc) return rc;
    if (rec) {
        CUDA_TRY(cudaEventRecord(st->ev[st->ev_used + 1], st->stream));
        st->ev_used += 2;
    }
    return MACE_OK;
}

// Set-up of the queue-fed schedule for one state: the launch configuration
// and the rows of super-voxels per (reconstruction, agent) pair
static int configure_queue(mace_state *st)
{
    const mace_sysmatrix *M = st->M;
    if (st->P.deterministic) return fail(MACE_EINVAL, "the deterministic mode runs the fixed schedule (schedule 0)");
    const mace_sysmatrix *Ms[1] = {M};
    // items per pair: `concurrency` rows (0 or -1: one per super-voxel row)
    int64_t C = st->P.concurrency > 0 ? st->P.concurrency : M->nsvy;
    C = std::max<int64_t>(1, std::min<int64_t>(C, M->nsv));
    st->concurrency = (int)C;
    st->wpv = resolve_wpv(st->P);
    // volumes: two slices of one z parity per warp when asked and every
    // parity class pairs up (a multiple of 4 slices)
    const bool nb26 = st->P.neighbourhood == 26;
    int K = (nb26 && st->P.chains >= 2 && st->B % 4 == 0) ? 2 : 1;
    int rc = queue_configure(Ms, 1, nb26, st->wpv, &st->q, K);
    if (rc && K == 2) {
        K = 1;
        rc = queue_configure(Ms, 1, nb26, st->wpv, &st->q, K);
    }
    if (rc) return rc;
    st->chains = K;
    st->sweep_warps = (int)std::min<int64_t>((int64_t)st->q.blocks * st->q.wpb,
                                             (int64_t)(st->B / K) * M->N * C * st->wpv);
    st->sweep_wpb = st->q.wpb;
    st->sweep_smem = st->q.smem;
    return MACE_OK;
}

// The queue's descriptors (forward and backward pass) and item offsets, in
// device memory; written once the super-voxel order is resident
static int queue_tables(mace_state *st)
{
    if (!st->d_qtab && (cudaMalloc(&st->d_qtab, 3 * sizeof(SweepArgs)) != cudaSuccess ||
                        cudaMalloc(&st->d_qoff, 4 * sizeof(int)) != cudaSuccess ||
                        cudaMalloc(&st->d_qcnt, sizeof(unsigned)) != cudaSuccess))
        return fail(MACE_ENOMEM, "cudaMalloc queue descriptors");
    const bool nb26 = st->P.neighbourhood == 26;
    st->q_items[0] = queue_items(st, nb26 ? 0 : -1);
    st->q_items[1] = nb26 ? queue_items(st, 1) : 0;
    const int off[4] = {0, st->q_items[0], 0, st->q_items[1]};
    const SweepArgs tab[2] = {sweep_args(st, 0, nullptr), sweep_args(st, 1, nullptr)};
    CUDA_TRY(cudaMemcpy(st->d_qoff, off, sizeof(off), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(st->d_qtab, tab, sizeof(tab), cudaMemcpyHostToDevice));
    return MACE_OK;
}

// Set-up of the fixed schedule: chains per warp, the kernel, the block size
// and C warps per (batch group, agent) pair, all resident
static int configure_fixed(mace_state *st)
{
    const mace_sysmatrix *M = st->M;
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    int nsm = 0, max_smem = 0;
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int col_stride = (M->max_col_bytes + 15) & ~15;
    // chains per warp: reconstructions of the batch (slices of a volume)
    // that share each column load (two when asked and the batch is even)
    const bool nb26 = st->P.neighbourhood == 26;
    int K = (st->P.chains >= 2 && st->B % 2 == 0) ? 2 : 1;
    sweep_fn fn = nullptr;
    for (;;) {
        st->warp_smem = warp_smem_layout(M->vpad, M->wmax, col_stride, M->S, K, nb26).total;
        const int R = sweep_rounds(M->max_views, K);
        const bool ovf_ok = R > 4 || M->max_n3 <= sweep_ovf_rounds(R, K) * (32 / K);
        fn = ovf_ok ? sweep_kernel_ptr(M, K, nb26, st->P.deterministic != 0) : nullptr;
        if (fn && st->warp_smem <= (size_t)max_smem) break;
        if (K == 1) break;
        K = 1;
    }
    if (!fn) return fail(MACE_EINVAL, "no sweep kernel for this matrix");
    if (st->warp_smem > (size_t)max_smem)
        return fail(MACE_EINVAL, "super-voxel working set does not fit in shared memory; use a smaller sv_size");
    st->chains = K;
    CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem));
    // block size (warps) that keeps the most warps resident per SM
    int wpb = 1, per_sm = 0, best = 0;
    for (int w = 1; w <= 8; ++w) {
        if (st->warp_smem * w > (size_t)max_smem) break;
        int b = 0;
        CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, 32 * w, st->warp_smem * w));
        if (b * w > best) { best = b * w; wpb = w; per_sm = b; }
    }
    if (per_sm < 1) per_sm = 1;
    // C warps per (batch group, agent): super-voxels of one agent of one
    // reconstruction in flight at a time; all warps resident
    const int64_t pairs = (int64_t)(st->B / K) * M->N;
    int64_t capacity = (int64_t)per_sm * nsm * wpb;
    int64_t C = capacity / pairs;
    if (C < 1) C = 1;
    if (st->P.concurrency > 0) C = std::min<int64_t>(C, st->P.concurrency);
    if (st->P.concurrency == -1) C = std::min<int64_t>(C, M->nsvy);   // one super-voxel row per warp
    C = std::min<int64_t>(C, M->nsv);
    int64_t warps = C * pairs;
    if (warps > capacity) return fail(MACE_EINVAL, "more (reconstruction, agent) pairs than resident warps; lower the batch");
    // whole blocks of wpb warps; the warps past C * pairs in the last block exit at once
    int w = (int)std::min<int64_t>(wpb, warps);
    st->sweep_wpb = w;
    st->sweep_smem = st->warp_smem * w;
    st->sweep_warps = (int)warps;
    st->concurrency = (int)C;
    return MACE_OK;
}

static int configure_sweep(mace_state *st)
{
    const mace_sysmatrix *M = st->M;
    // the sweep addresses columns in 16-byte units with 32 bits
    if (M->bytes_cols >= ((int64_t)1 << 36)) return fail(MACE_EINVAL, "stored matrix larger than 64 GiB");
    const bool queue = st->P.schedule == 1;
    int rc = queue ? configure_queue(st) : configure_fixed(st);
    if (rc) return rc;
    const int64_t C = st->concurrency;
    // super-voxel visiting order.  sv_order 0: the raster list of
    // super-voxels cut into C contiguous bands, interleaved so the C in flight
    // come from different bands (plain raster when C = 1); 1: a stride
    // permutation spreading consecutive super-voxels over the image.
    st->sv_order.resize(M->nsv);
    if (st->P.sv_order == 1) {
        int64_t p = std::max<int64_t>(1, (int64_t)llround(0.6180339887 * M->nsv));
        while (std::gcd<int64_t>(p, M->nsv) != 1) ++p;
        for (int k = 0; k < M->nsv; ++k) st->sv_order[k] = (int32_t)(((int64_t)k * p) % M->nsv);
    } else {
        std::vector<int> start(C + 1);
        for (int64_t b = 0; b <= C; ++b) start[b] = (int)((b * M->nsv) / C);
        int k = 0;
        for (int j = 0; k < M->nsv; ++j)
            for (int64_t b = 0; b < C; ++b)
                if (start[b] + j < start[b + 1]) st->sv_order[k++] = start[b] + j;
    }
    if (st->P.deterministic && !st->d_phase &&
        cudaMalloc(&st->d_phase, sizeof(unsigned) * (st->B / st->chains) * M->N) != cudaSuccess)
        return fail(MACE_ENOMEM, "cudaMalloc phase counters");
    if (!st->d_sv_order && cudaMalloc(&st->d_sv_order, sizeof(int32_t) * M->nsv) != cudaSuccess)
        return fail(MACE_ENOMEM, "cudaMalloc sv order");
    CUDA_TRY(cudaMemcpyAsync(st->d_sv_order, st->sv_order.data(), sizeof(int32_t) * M->nsv, cudaMemcpyHostToDevice,
                             st->stream));
    return queue ? queue_tables(st) : MACE_OK;
}

static int check_params(const mace_params *P)
{
    if (!P) return fail(MACE_EINVAL, "params is NULL");
    if (P->prior != 0 && P->prior != 1) return fail(MACE_EINVAL, "prior must be 0 (quadratic) or 1 (Q-GGMRF)");
    if (P->neighbourhood != 8 && P->neighbourhood != 26) return fail(MACE_EINVAL, "neighbourhood must be 8 or 26");
    if (!(P->beta >= 0) || !(P->sigma_x > 0) || !std::isfinite(P->beta) || !std::isfinite(P->sigma_x))
        return fail(MACE_EINVAL, "beta must be >= 0 and sigma_x > 0");
    if (P->prior == 1 && (P->p != 2.0 || !(P->q >= 1.0 && P->q <= 2.0) || !(P->T > 0)))
        return fail(MACE_EINVAL, "Q-GGMRF needs p == 2, 1 <= q <= 2, T > 0");
    if (!(P->sigma > 0) || !std::isfinite(P->sigma)) return fail(MACE_EINVAL, "sigma must be positive");
    if (P->sigma_mode != 0 && P->sigma_mode != 1) return fail(MACE_EINVAL, "sigma_mode must be 0 or 1");
    if (!(P->rho > 0 && P->rho < 1)) return fail(MACE_EINVAL, "rho must be in (0, 1)");
    if (P->sweeps_per_iter < 1 || P->sweeps_per_iter > 64) return fail(MACE_EINVAL, "sweeps_per_iter must be in [1, 64]");
    if (P->recompute_every < 0) return fail(MACE_EINVAL, "recompute_every must be >= 0");
    if (P->max_iter < 0) return fail(MACE_EINVAL, "max_iter must be >= 0");
    if (!(P->tol >= 0)) return fail(MACE_EINVAL, "tol must be >= 0");
    if (P->concurrency < -1) return fail(MACE_EINVAL, "concurrency must be >= -1");
    if (P->sv_order != 0 && P->sv_order != 1) return fail(MACE_EINVAL, "sv_order must be 0 or 1");
    if (P->chains != 0 && P->chains != 1 && P->chains != 2 && P->chains != 4)
        return fail(MACE_EINVAL, "chains must be 0, 1, 2 or 4");
    if (P->pnp != 0 && P->pnp != 1) return fail(MACE_EINVAL, "pnp must be 0 or 1");
    if (P->forward_geometry < 0 || P->forward_geometry > 2)
        return fail(MACE_EINVAL, "forward_geometry must be 0, 1 or 2");
    if (P->deterministic != 0 && P->deterministic != 1) return fail(MACE_EINVAL, "deterministic must be 0 or 1");
    if (P->schedule != 0 && P->schedule != 1) return fail(MACE_EINVAL, "schedule must be 0 or 1");
    if (P->schedule == 1 && P->deterministic)
        return fail(MACE_EINVAL, "the deterministic mode runs the fixed schedule (schedule 0)");
    if (P->warps_per_voxel != 0 && P->warps_per_voxel != 1 && P->warps_per_voxel != 2 && P->warps_per_voxel != 4)
        return fail(MACE_EINVAL, "warps_per_voxel must be 0 (automatic), 1, 2 or 4");
    if (P->warps_per_voxel > 1 && (P->schedule != 1 || P->neighbourhood == 26))
        return fail(MACE_EINVAL, "teams of warps per super-voxel run the 2D work-queue schedule (schedule 1)");
    if (P->pnp && (P->prior != 0 || P->neighbourhood != 8))
        return fail(MACE_EINVAL, "pnp needs the quadratic prior and the 8-neighbourhood");
    return MACE_OK;
}

extern "C" void mace_free_state(mace_state *st)
{
    if (!st) return;
    // work on the state's stream (and, through its event waits, the group
    // launches it took part in) ends before its memory goes
    cudaStreamSynchronize(st->stream);
    cudaFree(st->d_eL);
    cudaFree(st->d_dacc);
    cudaFree(st->d_phase);
    cudaFree(st->d_y);
    cudaFree(st->d_w);
    cudaFree(st->d_X);
    cudaFree(st->d_vexp);
    cudaFree(st->d_wbar);
    cudaFree(st->d_part);
    cudaFree(st->d_resid);
    cudaFree(st->d_theta2);
    cudaFree(st->d_hbuf);
    cudaFree(st->d_status);
    cudaFree(st->d_sv_order);
    cudaFree(st->d_qtab);
    cudaFree(st->d_qoff);
    cudaFree(st->d_qcnt);
    for (cudaEvent_t e : st->ev) cudaEventDestroy(e);
    if (st->graph_exec) cudaGraphExecDestroy(st->graph_exec);
    if (st->poll_ev) cudaEventDestroy(st->poll_ev);
    if (st->h_poll) cudaFreeHost(st->h_poll);
    delete st;
}

static int copy_in(void *dst, const void *src, size_t bytes, int is_dev, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (!is_dev) CUDA_TRY(cudaStreamSynchronize(s));
    return MACE_OK;
}

static int copy_out(void *dst, const void *src, size_t bytes, int is_dev, cudaStream_t s)
{
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, is_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!is_dev) CUDA_TRY(cudaStreamSynchronize(s));
    return MACE_OK;
}

// The consensus operator into d_wbar (FP64): G (Algorithm 1) = mean_i w_i, or
// G_H (Algorithm 3) = H(mean_i w_i) with H by h_iters Jacobi iterations from
// the mean; x_out (device, optional) receives it in FP32.
static int apply_consensus(mace_state *st, float *x_out)
{
    NvtxRange nvtx_range("consensus");
    const mace_sysmatrix *M = st->M;
    const int64_t Bn = (int64_t)st->B * st->n;
    const unsigned blocks = (unsigned)((Bn + 255) / 256);
    consensus_kernel<<<blocks, 256, 0, st->stream>>>(st->d_w, st->B, M->N, st->n, st->d_wbar,
                                                     st->P.pnp ? nullptr : x_out);
    if (st->P.pnp) {
        double *v = st->d_hbuf, *x2 = st->d_hbuf + Bn;
        CUDA_TRY(cudaMemcpyAsync(v, st->d_wbar, sizeof(double) * Bn, cudaMemcpyDeviceToDevice, st->stream));
        const double bsum = 4.0 + 4.0 / std::sqrt(2.0);
        for (int k = 0; k < st->h_iters; ++k)
            prior_prox_jacobi_kernel<<<blocks, 256, 0, st->stream>>>(v, (k & 1) ? x2 : st->d_wbar,
                                                                     (k & 1) ? st->d_wbar : x2, st->B, M->geo.nx,
                                                                     M->geo.ny, st->h_c, 1.0 / bsum,
                                                                     (1.0 / std::sqrt(2.0)) / bsum);
        if (x_out) to_float_kernel<<<blocks, 256, 0, st->stream>>>(st->d_wbar, x_out, Bn);
    }
    CUDA_TRY(cudaGetLastError());
    return MACE_OK;
}

// X^(0) = G(w^(0)) (Algorithm 1) or G_H(w^(0)) (Algorithm 3)
static int set_X_from_w(mace_state *st)
{
    const mace_sysmatrix *M = st->M;
    const int64_t Bn = (int64_t)st->B * st->n;
    int rc = apply_consensus(st, nullptr);
    if (rc) return rc;
    broadcast_kernel<<<(unsigned)((Bn * M->N + 255) / 256), 256, 0, st->stream>>>(st->d_wbar, st->d_X, st->B, M->N, st->n);
    CUDA_TRY(cudaGetLastError());
    return MACE_OK;
}

extern "C" int mace_init(const mace_sysmatrix *M, int32_t batch, const float *y, const float *weights,
                         int32_t ptr_is_device, const mace_params *params, const float *w0, void *cuda_stream,
                         mace_state **out)
{
    NvtxRange nvtx_range("mace_init");
    if (!out) return fail(MACE_EINVAL, "out is NULL");
    *out = nullptr;
    if (!M || !y || !weights) return fail(MACE_EINVAL, "NULL sysmatrix, y or weights");
    if (batch < 1 || batch > 4096) return fail(MACE_EINVAL, "batch must be in [1, 4096]");
    int rc = check_params(params);
    if (rc) return rc;
    mace_state *st = new mace_state();
    st->M = M;
    st->P = *params;
    st->B = batch;
    st->stream = (cudaStream_t)cuda_stream;
    st->n = (int64_t)M->geo.nx * M->geo.ny;
    st->ne = (int64_t)M->V * M->geo.D;
    const int64_t NN = (int64_t)batch * M->N * st->n;
    const int64_t m = (int64_t)batch * st->ne;
    auto bail = [&](int code, const std::string &msg) {
        mace_free_state(st);
        return fail(code, msg);
    };
    if (cudaMalloc(&st->d_eL, sizeof(float2) * m) != cudaSuccess ||
        cudaMalloc(&st->d_dacc, sizeof(unsigned long long) * m) != cudaSuccess ||
        cudaMalloc(&st->d_y, sizeof(float) * m) != cudaSuccess ||
        cudaMalloc(&st->d_w, sizeof(float) * NN) != cudaSuccess ||
        cudaMalloc(&st->d_X, sizeof(float) * NN) != cudaSuccess ||
        cudaMalloc(&st->d_theta2, sizeof(float) * NN) != cudaSuccess ||
        cudaMalloc(&st->d_wbar, sizeof(double) * batch * st->n) != cudaSuccess ||
        cudaMalloc(&st->d_resid, sizeof(double) * 3 * batch) != cudaSuccess ||
        cudaMalloc(&st->d_status, sizeof(int)) != cudaSuccess)
        return bail(MACE_ENOMEM, "cudaMalloc failed for the reconstruction state");
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t per = (int64_t)M->N * st->n;
    st->nblk_mann = (int)std::max<int64_t>(1, std::min<int64_t>(std::max(1, nsm * 4 / batch), (per + 255) / 256));
    if (cudaMalloc(&st->d_part, sizeof(double) * 2 * st->nblk_mann * batch) != cudaSuccess)
        return bail(MACE_ENOMEM, "cudaMalloc failed for residual partials");
    {
        // the no-allocation read-out's array on this device (looked up here,
        // outside any stream capture, with the state's device current)
        const cudaError_t e = cudaGetSymbolAddress((void **)&st->noalloc_addr, g_noalloc_images);
        if (e != cudaSuccess) return bail(MACE_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    cudaStream_t s = st->stream;
    // inputs: stage on the device, validate, pack agent-major
    float *d_yin = nullptr, *d_lin = nullptr;
    if (ptr_is_device) {
        d_yin = (float *)y;
        d_lin = (float *)weights;
    } else {
        if (cudaMalloc(&d_yin, sizeof(float) * m) != cudaSuccess || cudaMalloc(&d_lin, sizeof(float) * m) != cudaSuccess) {
            cudaFree(d_yin);
            return bail(MACE_ENOMEM, "cudaMalloc failed for input staging");
        }
        if (cudaMemcpyAsync(d_yin, y, sizeof(float) * m, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(d_lin, weights, sizeof(float) * m, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            cudaFree(d_yin);
            cudaFree(d_lin);
            return bail(MACE_ECUDA, "copy of y / weights failed");
        }
    }
    int *d_av = nullptr;
    int bad = 0;
    cudaError_t ce = cudaMalloc(&d_av, sizeof(int) * M->V);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(d_av, M->agent_views.data(), sizeof(int) * M->V, cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(st->d_status, 0, sizeof(int), s);
    if (ce == cudaSuccess) {
        check_weights_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_yin, d_lin, m, st->d_status);
        pack_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(d_yin, d_lin, d_av, batch, M->V, M->geo.D, st->d_eL,
                                                                st->d_y);
        ce = cudaMemcpyAsync(&bad, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(d_av);
    if (!ptr_is_device) { cudaFree(d_yin); cudaFree(d_lin); }
    if (ce != cudaSuccess) return bail(MACE_ECUDA, std::string("input packing: ") + cudaGetErrorString(ce));
    if (bad) return bail(MACE_EINVAL, "y and weights must be finite and weights >= 0");
    if (cudaMemsetAsync(st->d_status, 0, sizeof(int), s) != cudaSuccess) return bail(MACE_ECUDA, "memset status");
    // theta2 per (b, agent, pixel) and its mean; sigma in image units
    {
        double *d_t2 = nullptr;
        const int64_t t2items = (int64_t)batch * M->N * M->nsv;
        double h_t2 = 0.0;
        ce = cudaMalloc(&d_t2, sizeof(double) * (t2items + 1));
        if (ce == cudaSuccess) ce = cudaMemsetAsync(st->d_theta2, 0, sizeof(float) * NN, s);
        if (ce == cudaSuccess) {
            int64_t items = (int64_t)batch * M->N * M->nsv;
            const size_t sm = 8 * aux_warp_bytes(M->vpad, M->wmax);
            const unsigned tb = (unsigned)((items * 32 + 255) / 256);
            if (M->dtype == MACE_F32) {
                cudaFuncSetAttribute(theta2_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                theta2_kernel<float><<<tb, 256, sm, s>>>(M->d_cols, M->d_sv_base, M->d_col_off, M->d_band,
                                                         M->d_view_off, st->d_eL, batch, M->N, M->nsv, M->nsvx, M->S,
                                                         M->geo.nx, M->geo.ny, M->geo.D, st->ne, M->vpad, M->wmax,
                                                         st->d_theta2, d_t2);
            } else if (M->dtype == MACE_BF16) {
                cudaFuncSetAttribute(theta2_kernel<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                theta2_kernel<__nv_bfloat16><<<tb, 256, sm, s>>>(M->d_cols, M->d_sv_base, M->d_col_off, M->d_band,
                                                                 M->d_view_off, st->d_eL, batch, M->N, M->nsv, M->nsvx,
                                                                 M->S, M->geo.nx, M->geo.ny, M->geo.D, st->ne, M->vpad,
                                                                 M->wmax, st->d_theta2, d_t2);
            } else {
                cudaFuncSetAttribute(theta2_kernel<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
                theta2_kernel<__half><<<tb, 256, sm, s>>>(M->d_cols, M->d_sv_base, M->d_col_off, M->d_band,
                                                          M->d_view_off, st->d_eL, batch, M->N, M->nsv, M->nsvx, M->S,
                                                          M->geo.nx, M->geo.ny, M->geo.D, st->ne, M->vpad, M->wmax,
                                                          st->d_theta2, d_t2);
            }
            ce = cudaGetLastError();
            if (ce == cudaSuccess) {
                sum_fixed_kernel<<<1, 1024, 0, s>>>(d_t2, t2items, d_t2 + t2items);
                ce = cudaGetLastError();
            }
            if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_t2, d_t2 + t2items, sizeof(double), cudaMemcpyDeviceToHost, s);
        }
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        cudaFree(d_t2);
        if (ce != cudaSuccess) return bail(MACE_ECUDA, std::string("theta2: ") + cudaGetErrorString(ce));
        if (params->sigma_mode == 1) {
            double mean_t2 = h_t2 / ((double)batch * M->N * (double)st->n);
            if (!(mean_t2 > 0)) return bail(MACE_EINVAL, "all weights are zero");
            st->sigma_abs = params->sigma / std::sqrt(mean_t2);
        } else {
            st->sigma_abs = params->sigma;
        }
    }
    if (params->pnp) {
        // H: Jacobi for (I + c B) x = v contracts by c / (1 + c) per iteration
        // (sum_r b_sr <= 1); iterate to FP64 round-off, an even count
        st->h_c = st->sigma_abs * st->sigma_abs * params->beta / (params->sigma_x * params->sigma_x);
        const double q = st->h_c / (1.0 + st->h_c);
        int k = q > 0.0 ? (int)std::ceil(std::log(1e-15) / std::log(q)) : 1;
        k = std::max(2, std::min(1000, k + (k & 1)));
        st->h_iters = k;
        if (cudaMalloc(&st->d_hbuf, sizeof(double) * 2 * batch * st->n) != cudaSuccess)
            return bail(MACE_ENOMEM, "cudaMalloc failed for the denoiser buffers");
    }
    // w^(0), X^(0) = G(w^(0)), e = y - A X
    if (w0) {
        rc = copy_in(st->d_w, w0, sizeof(float) * NN, ptr_is_device, s);
        if (rc) { mace_free_state(st); return rc; }
    } else if (cudaMemsetAsync(st->d_w, 0, sizeof(float) * NN, s) != cudaSuccess) {
        return bail(MACE_ECUDA, "memset w");
    }
    rc = set_X_from_w(st);
    if (rc == MACE_OK) rc = launch_forward(st);
    if (rc) { mace_free_state(st); return rc; }
    rc = configure_sweep(st);
    if (rc) { mace_free_state(st); return rc; }
    ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return bail(MACE_ECUDA, std::string("init: ") + cudaGetErrorString(ce));
    *out = st;
    return MACE_OK;
}

extern "C" int mace_state_bytes(const mace_sysmatrix *M, int32_t batch, const mace_params *params,
                                int32_t ptr_is_device, int64_t *persistent, int64_t *peak)
{
    if (!M || !persistent || !peak) return fail(MACE_EINVAL, "NULL argument");
    if (batch < 1 || batch > 4096) return fail(MACE_EINVAL, "batch must be in [1, 4096]");
    const int rc = check_params(params);
    if (rc) return rc;
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // what mace_init allocates, call for call
    const int64_t n = (int64_t)M->geo.nx * M->geo.ny, B = batch;
    const int64_t m = B * (int64_t)M->V * M->geo.D, NN = B * M->N * n;
    const int64_t per = (int64_t)M->N * n;
    const int64_t nblk = std::max<int64_t>(1, std::min<int64_t>(std::max(1, nsm * 4 / batch), (per + 255) / 256));
    const int K = params->schedule == 0 ? ((params->chains >= 2 && batch % 2 == 0) ? 2 : 1)
                                        : ((params->neighbourhood == 26 && params->chains >= 2 && batch % 4 == 0) ? 2 : 1);
    int64_t p = m * (8 + 8 + 4)                 // (e, Lambda), changes of e, y
                + NN * 4 * 3                    // w, X, theta2
                + B * n * 8 + B * 3 * 8 + 4     // consensus, residuals, status
                + nblk * 2 * B * 8              // residual partials
                + (int64_t)M->nsv * 4;          // super-voxel order
    if (params->pnp) p += 2 * B * n * 8;
    if (params->deterministic) p += (B / K) * M->N * 4;
    if (params->schedule == 1) p += 3 * (int64_t)sizeof(SweepArgs) + 4 * 4 + 4;   // queue descriptors
    // transient during mace_init: input staging, the view map, theta2 partials
    const int64_t t = (ptr_is_device ? 0 : 2 * m * 4) + (int64_t)M->V * 4 + (B * M->N * M->nsv + 1) * 8;
    *persistent = p;
    *peak = p + t;
    return MACE_OK;
}

// The two halves of a Mann iteration around its ICD passes (Algorithm 1):
// the consensus G(w) before them; the Mann update, its residual and the
// periodic e recompute after them
static int iteration_pre(mace_state *st) { return apply_consensus(st, nullptr); }

static int iteration_post(mace_state *st)
{
    const mace_sysmatrix *M = st->M;
    mann_kernel<<<dim3(st->nblk_mann, st->B), 256, 0, st->stream>>>(st->d_w, st->d_X, st->d_wbar, M->N, st->n,
                                                                    (float)st->P.rho, st->d_part);
    residual_kernel<<<st->B, 256, 0, st->stream>>>(st->d_part, st->nblk_mann, st->B, st->d_resid);
    CUDA_TRY(cudaGetLastError());
    st->iters++;
    if (st->P.recompute_every > 0 && st->iters % st->P.recompute_every == 0) return launch_forward(st);
    return MACE_OK;
}

static int run_iteration(mace_state *st)
{
    NvtxRange nvtx_range("Mann iteration");
    int rc = iteration_pre(st);
    if (rc) return rc;
    for (int k = 0; k < st->P.sweeps_per_iter; ++k) {
        rc = launch_sweep(st, st->P.symmetric ? (k & 1) : 0, nullptr);
        if (rc) return rc;
    }
    return iteration_post(st);
}

// largest relative Mann residual over the batch from a host copy of d_resid
// ([B][3]) and the status word
static int parse_status(mace_state *st, const double *h, int status, double *r)
{
    if (status == kStatusTimeout) return fail(MACE_ETIMEOUT, "a device-side wait timed out");
    if (status == kStatusBounds)
        return fail(MACE_ECUDA, "a device-side bounds check failed (MACE_DEBUG build): stored matrix or state inconsistent");
    double worst = 0.0;
    for (int b = 0; b < st->B; ++b) {
        double rb = h[3 * b + 2];
        if (!std::isfinite(rb)) { worst = rb; break; }
        worst = std::max(worst, rb);
    }
    *r = worst;
    st->last_resid = worst;
    if (!std::isfinite(worst)) return fail(MACE_ENUMERIC, "non-finite Mann residual (divergence)");
    return MACE_OK;
}

static int read_status(mace_state *st, double *r)
{
    std::vector<double> h(3 * st->B);
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(h.data(), st->d_resid, sizeof(double) * 3 * st->B, cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaMemcpyAsync(&status, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    return parse_status(st, h.data(), status, r);
}

// One chunk of graph_iters iterations (a whole recompute period, starting
// right after a recompute) from the captured graph; the graph is captured
// on first use.  Returns 1 when capture is not possible (the caller then
// launches eagerly), else a MACE code.
static int graph_chunk(mace_state *st)
{
    if (!st->graph_exec) {
        const int saved = st->iters;
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(st->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            st->graph_failed = true;
            return 1;
        }
        int rc = MACE_OK;
        for (int k = 0; k < st->graph_iters && rc == MACE_OK; ++k) rc = run_iteration(st);
        cudaError_t ce = cudaStreamEndCapture(st->stream, &g);
        st->iters = saved;
        if (rc != MACE_OK || ce != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            cudaGetLastError();
            st->graph_failed = true;
            return 1;
        }
        ce = cudaGraphInstantiate(&st->graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            st->graph_exec = nullptr;
            cudaGetLastError();
            st->graph_failed = true;
            return 1;
        }
    }
    CUDA_TRY(cudaGraphLaunch(st->graph_exec, st->stream));
    st->iters += st->graph_iters;
    return MACE_OK;
}

extern "C" int mace_launch(mace_state *st, int32_t n_iters)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    if (n_iters < 0) return fail(MACE_EINVAL, "n_iters must be >= 0");
    st->graph_iters = st->P.recompute_every > 0 ? st->P.recompute_every : 10;
    int k = 0;
    while (k < n_iters) {
        const bool use_graph = st->stream != nullptr && !st->timing && !st->graph_failed &&
                               st->iters % st->graph_iters == 0 && n_iters - k >= st->graph_iters;
        if (use_graph) {
            const int rc = graph_chunk(st);
            if (rc == MACE_OK) {
                k += st->graph_iters;
                continue;
            }
            if (rc != 1) return rc;
        }
        const int rc = run_iteration(st);
        if (rc) return rc;
        ++k;
    }
    return MACE_OK;
}

extern "C" int mace_poll(mace_state *st, double *residual_out, int32_t *converged_out)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    double r = st->last_resid;
    if (st->iters > 0) {
        int rc = read_status(st, &r);
        if (rc) return rc;
    }
    if (residual_out) *residual_out = r;
    if (converged_out) *converged_out = r < st->P.tol ? 1 : 0;
    return MACE_OK;
}

extern "C" int mace_poll_async(mace_state *st)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    if (!st->h_poll) {
        // 3 B residual doubles, then one double's room for the status word
        if (cudaMallocHost(&st->h_poll, sizeof(double) * (3 * st->B + 1)) != cudaSuccess) {
            st->h_poll = nullptr;
            return fail(MACE_ENOMEM, "cudaMallocHost failed for the status copy");
        }
        CUDA_TRY(cudaEventCreateWithFlags(&st->poll_ev, cudaEventDisableTiming));
    }
    CUDA_TRY(cudaMemcpyAsync(st->h_poll, st->d_resid, sizeof(double) * 3 * st->B, cudaMemcpyDeviceToHost,
                             st->stream));
    CUDA_TRY(cudaMemcpyAsync(st->h_poll + 3 * st->B, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaEventRecord(st->poll_ev, st->stream));
    st->poll_pending = true;
    return MACE_OK;
}

extern "C" int mace_poll_ready(mace_state *st, double *residual_out, int32_t *converged_out, int32_t *ready_out)
{
    if (!st || !ready_out) return fail(MACE_EINVAL, "NULL argument");
    double r = st->last_resid;
    *ready_out = 1;
    if (st->poll_pending) {
        const cudaError_t q = cudaEventQuery(st->poll_ev);
        if (q == cudaErrorNotReady) {
            *ready_out = 0;
            return MACE_OK;
        }
        if (q != cudaSuccess) return fail(MACE_ECUDA, std::string("status copy: ") + cudaGetErrorString(q));
        st->poll_pending = false;
        int status = 0;
        memcpy(&status, st->h_poll + 3 * st->B, sizeof(int));
        if (st->iters > 0) {
            const int rc = parse_status(st, st->h_poll, status, &r);
            if (rc) return rc;
        }
    }
    if (residual_out) *residual_out = r;
    if (converged_out) *converged_out = r < st->P.tol ? 1 : 0;
    return MACE_OK;
}

extern "C" int mace_iterate(mace_state *st, int32_t n_iters, double *residual_out, int32_t *converged_out)
{
    int rc = mace_launch(st, n_iters);
    if (rc) return rc;
    return mace_poll(st, residual_out, converged_out);
}

// --- groups: several states' ICD passes in one queue-fed launch -------------
// Membership changes (mace_group_update) are stream-ordered: the new
// descriptors go through pinned staging (two slots, so the host does not
// wait for the upload it just queued) into device tables that later launches
// on the group's stream read; nothing synchronises the device.
struct mace_group {
    std::vector<mace_state *> members;
    cudaStream_t stream = nullptr;
    QueueLaunch q;
    int npass = 0;                       // largest sweeps_per_iter of the members
    SweepArgs *d_tab = nullptr;          // [npass][n] descriptors of each pass's requests
    int *d_off = nullptr;                // [npass][n + 1] first item of each request
    size_t cap_tab = 0, cap_off = 0;     // entries allocated
    unsigned *d_cnt = nullptr;
    std::vector<int> nreq, total;        // per pass
    cudaEvent_t done = nullptr;          // the group's work, for the members' streams
    std::vector<cudaEvent_t> ready;      // each member's earlier work, for the group's stream
    uint8_t *h_stage[2] = {nullptr, nullptr};
    size_t cap_stage[2] = {0, 0};
    cudaEvent_t staged[2] = {nullptr, nullptr};
    bool staged_used[2] = {false, false};
    int slot = 0;
};

static void group_free(mace_group *G)
{
    for (int k = 0; k < 2; ++k) {
        if (G->staged_used[k]) cudaEventSynchronize(G->staged[k]);
        if (G->h_stage[k]) cudaFreeHost(G->h_stage[k]);
        if (G->staged[k]) cudaEventDestroy(G->staged[k]);
    }
    if (G->d_tab) cudaFreeAsync(G->d_tab, G->stream);
    if (G->d_off) cudaFreeAsync(G->d_off, G->stream);
    if (G->d_cnt) cudaFreeAsync(G->d_cnt, G->stream);
    if (G->done) cudaEventDestroy(G->done);
    for (cudaEvent_t e : G->ready)
        if (e) cudaEventDestroy(e);
    delete G;
}

// Replace the members: check them, configure the launch, build the
// per-pass descriptor tables and queue their upload on the group's stream.
// On error the group keeps its previous members.
static int group_set(mace_group *G, mace_state *const *members, int n)
{
    if (!members) return fail(MACE_EINVAL, "NULL argument");
    if (n < 1 || n > 65536) return fail(MACE_EINVAL, "a group has 1 to 65536 members");
    std::vector<const mace_sysmatrix *> Ms(n);
    for (int k = 0; k < n; ++k) {
        const mace_state *st = members[k];
        if (!st) return fail(MACE_EINVAL, "NULL member");
        for (int j = 0; j < k; ++j)
            if (members[j] == st) return fail(MACE_EINVAL, "a state appears twice in the group");
        if (st->P.schedule != 1) return fail(MACE_EINVAL, "group members run the work-queue schedule (schedule 1)");
        if (st->P.neighbourhood == 26) return fail(MACE_EINVAL, "volumes (neighbourhood 26) are not grouped");
        Ms[k] = st->M;
    }
    // one team size for the launch: the smallest the members resolved (a
    // team runs the decode-at-use sweep, slower for agents of few views)
    int W = 4;
    for (int k = 0; k < n; ++k) W = std::min(W, members[k]->wpv);
    QueueLaunch q;
    int rc = queue_configure(Ms.data(), n, false, W, &q);
    if (rc) return rc;
    int npass = 0;
    for (int k = 0; k < n; ++k) npass = std::max(npass, members[k]->P.sweeps_per_iter);
    // pass p: the members with more than p passes per iteration, each in
    // its own direction (every second pass backward when symmetric)
    const size_t ntab = (size_t)npass * n, noff = (size_t)npass * (n + 1);
    const size_t tab_bytes = sizeof(SweepArgs) * ntab, bytes = tab_bytes + sizeof(int) * noff;
    std::vector<int> nreq(npass, 0), total(npass, 0);
    // staging slot: the one not used by the last update; its previous
    // upload (two updates ago) has long been queued
    const int slot = G->slot ^ 1;
    if (G->staged_used[slot]) CUDA_TRY(cudaEventSynchronize(G->staged[slot]));
    if (G->cap_stage[slot] < bytes) {
        if (G->h_stage[slot]) cudaFreeHost(G->h_stage[slot]);
        G->h_stage[slot] = nullptr;
        G->cap_stage[slot] = 0;
        if (cudaMallocHost(&G->h_stage[slot], bytes) != cudaSuccess) {
            G->h_stage[slot] = nullptr;
            return fail(MACE_ENOMEM, "cudaMallocHost group staging");
        }
        G->cap_stage[slot] = bytes;
    }
    SweepArgs *tab = (SweepArgs *)G->h_stage[slot];
    int *off = (int *)(G->h_stage[slot] + tab_bytes);
    // requests in decreasing order of an item's length (pixels of its share
    // of super-voxels times the agent's views): the longest items start
    // first and short ones fill in behind them, so a pass ends soon after
    // its longest item (a longest-first schedule)
    std::vector<int> order(n);
    std::vector<double> cost(n);
    for (int k = 0; k < n; ++k) {
        const mace_state *st = members[k];
        const mace_sysmatrix *M = st->M;
        order[k] = k;
        cost[k] = (double)M->nsv / st->concurrency * M->S2 * M->max_views;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    for (int p = 0; p < npass; ++p) {
        int r = 0, t = 0;
        for (int kk = 0; kk < n; ++kk) {
            const mace_state *st = members[order[kk]];
            if (st->P.sweeps_per_iter <= p) continue;
            tab[(size_t)p * n + r] = sweep_args(st, st->P.symmetric ? (p & 1) : 0, nullptr);
            off[(size_t)p * (n + 1) + r] = t;
            t += queue_items(st, -1);
            ++r;
        }
        for (int k = r; k <= n; ++k) off[(size_t)p * (n + 1) + k] = t;
        nreq[p] = r;
        total[p] = t;
    }
    // device tables, grown in stream order (launches before this point
    // still read the old ones)
    if (G->cap_tab < ntab) {
        if (G->d_tab) CUDA_TRY(cudaFreeAsync(G->d_tab, G->stream));
        G->d_tab = nullptr;
        G->cap_tab = 0;
        if (cudaMallocAsync((void **)&G->d_tab, sizeof(SweepArgs) * ntab, G->stream) != cudaSuccess)
            return fail(MACE_ENOMEM, "cudaMallocAsync group descriptors");
        G->cap_tab = ntab;
    }
    if (G->cap_off < noff) {
        if (G->d_off) CUDA_TRY(cudaFreeAsync(G->d_off, G->stream));
        G->d_off = nullptr;
        G->cap_off = 0;
        if (cudaMallocAsync((void **)&G->d_off, sizeof(int) * noff, G->stream) != cudaSuccess)
            return fail(MACE_ENOMEM, "cudaMallocAsync group offsets");
        G->cap_off = noff;
    }
    if (!G->d_cnt && cudaMallocAsync((void **)&G->d_cnt, sizeof(unsigned), G->stream) != cudaSuccess)
        return fail(MACE_ENOMEM, "cudaMallocAsync group counter");
    CUDA_TRY(cudaMemcpyAsync(G->d_tab, tab, tab_bytes, cudaMemcpyHostToDevice, G->stream));
    CUDA_TRY(cudaMemcpyAsync(G->d_off, off, sizeof(int) * noff, cudaMemcpyHostToDevice, G->stream));
    if (!G->staged[slot]) CUDA_TRY(cudaEventCreateWithFlags(&G->staged[slot], cudaEventDisableTiming));
    CUDA_TRY(cudaEventRecord(G->staged[slot], G->stream));
    G->staged_used[slot] = true;
    G->slot = slot;
    while ((int)G->ready.size() < n) {
        cudaEvent_t e = nullptr;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        G->ready.push_back(e);
    }
    G->members.assign(members, members + n);
    G->q = q;
    G->npass = npass;
    G->nreq = nreq;
    G->total = total;
    return MACE_OK;
}

extern "C" int mace_group_create(mace_state *const *members, int32_t n, void *cuda_stream, mace_group **out)
{
    if (!members || !out) return fail(MACE_EINVAL, "NULL argument");
    *out = nullptr;
    mace_group *G = new mace_group();
    G->stream = (cudaStream_t)cuda_stream;
    int rc = MACE_OK;
    if (cudaEventCreateWithFlags(&G->done, cudaEventDisableTiming) != cudaSuccess) rc = fail(MACE_ECUDA, "group event");
    if (rc == MACE_OK) rc = group_set(G, members, n);
    if (rc) {
        group_free(G);
        return rc;
    }
    *out = G;
    return MACE_OK;
}

extern "C" int mace_group_update(mace_group *G, mace_state *const *members, int32_t n)
{
    if (!G) return fail(MACE_EINVAL, "group is NULL");
    return group_set(G, members, n);
}

extern "C" int mace_group_launch(mace_group *G, int32_t n_iters)
{
    NvtxRange nvtx_range("group launch");
    if (!G) return fail(MACE_EINVAL, "group is NULL");
    if (n_iters < 0) return fail(MACE_EINVAL, "n_iters must be >= 0");
    if (n_iters == 0) return MACE_OK;
    const int n = (int)G->members.size();
    // the group's stream follows every member's earlier work
    for (int k = 0; k < n; ++k) {
        CUDA_TRY(cudaEventRecord(G->ready[k], G->members[k]->stream));
        CUDA_TRY(cudaStreamWaitEvent(G->stream, G->ready[k], 0));
    }
    // members enqueue on the group's stream for the length of the call
    std::vector<cudaStream_t> own(n);
    for (int k = 0; k < n; ++k) {
        own[k] = G->members[k]->stream;
        G->members[k]->stream = G->stream;
    }
    int rc = MACE_OK;
    for (int it = 0; it < n_iters && rc == MACE_OK; ++it) {
        for (int k = 0; k < n && rc == MACE_OK; ++k) rc = iteration_pre(G->members[k]);
        for (int p = 0; p < G->npass && rc == MACE_OK; ++p)
            rc = queue_run(G->q, G->d_tab + (size_t)p * n, G->d_off + (size_t)p * (n + 1), G->d_cnt, G->nreq[p],
                           G->total[p], -1, G->stream);
        for (int k = 0; k < n && rc == MACE_OK; ++k) rc = iteration_post(G->members[k]);
    }
    for (int k = 0; k < n; ++k) G->members[k]->stream = own[k];
    if (rc) return rc;
    // and every member's later work follows the group's
    CUDA_TRY(cudaEventRecord(G->done, G->stream));
    for (int k = 0; k < n; ++k) CUDA_TRY(cudaStreamWaitEvent(G->members[k]->stream, G->done, 0));
    return MACE_OK;
}

extern "C" int mace_group_free(mace_group *G)
{
    if (!G) return MACE_OK;
    group_free(G);
    return MACE_OK;
}

extern "C" int mace_set_timing(mace_state *st, int32_t enable, int32_t max_launches)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    if (enable && max_launches < 1) return fail(MACE_EINVAL, "max_launches must be >= 1");
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    st->ev_used = 0;
    st->timing = enable != 0;
    size_t need = enable ? (size_t)2 * max_launches : 0;
    while (st->ev.size() < need) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        st->ev.push_back(e);
    }
    return MACE_OK;
}

extern "C" int mace_get_timing(mace_state *st, double *sweep_ms, int32_t *launches)
{
    if (!st || !sweep_ms || !launches) return fail(MACE_EINVAL, "NULL argument");
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    double tot = 0.0;
    for (int k = 0; k + 1 < st->ev_used; k += 2) {
        float ms = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&ms, st->ev[k], st->ev[k + 1]));
        tot += ms;
    }
    *sweep_ms = tot;
    *launches = st->ev_used / 2;
    st->ev_used = 0;
    return MACE_OK;
}

extern "C" int mace_consensus(mace_state *st, float *x_out, int32_t ptr_is_device)
{
    if (!st || !x_out) return fail(MACE_EINVAL, "NULL argument");
    const int64_t Bn = (int64_t)st->B * st->n;
    float *d_x = ptr_is_device ? x_out : nullptr;
    if (!d_x && cudaMalloc(&d_x, sizeof(float) * Bn) != cudaSuccess) return fail(MACE_ENOMEM, "cudaMalloc x");
    const int rc = apply_consensus(st, d_x);
    cudaError_t ce = cudaSuccess;
    if (rc == MACE_OK && !ptr_is_device) {
        ce = cudaMemcpyAsync(x_out, d_x, sizeof(float) * Bn, cudaMemcpyDeviceToHost, st->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st->stream);
    }
    if (!ptr_is_device) cudaFree(d_x);
    if (rc) return rc;
    if (ce != cudaSuccess) return fail(MACE_ECUDA, std::string("consensus: ") + cudaGetErrorString(ce));
    return MACE_OK;
}

// ---------------------------------------------------------------------------
// Consensus image without any allocation
// ---------------------------------------------------------------------------
extern "C" int mace_consensus_noalloc(mace_state *st, float *x_out, int32_t ptr_is_device)
{
    if (!st || !x_out) return fail(MACE_EINVAL, "NULL argument");
    const int64_t Bn = (int64_t)st->B * st->n;
    float *d_x = x_out;
    if (!ptr_is_device) {
        if (Bn > kNoAllocFloats)
            return fail(MACE_EINVAL, "batch x image larger than the 1048576-float no-allocation buffer");
        d_x = st->noalloc_addr;
    }
    const int rc = apply_consensus(st, d_x);
    if (rc) return rc;
    if (!ptr_is_device) {
        CUDA_TRY(cudaMemcpyAsync(x_out, d_x, sizeof(float) * Bn, cudaMemcpyDeviceToHost, st->stream));
        CUDA_TRY(cudaStreamSynchronize(st->stream));
    }
    return MACE_OK;
}

extern "C" int mace_reconstruct(mace_state *st, float *x_out, int32_t ptr_is_device, int32_t *iters_out,
                                double *residual_out)
{
    NvtxRange nvtx_range("mace_reconstruct");
    if (!st || !x_out) return fail(MACE_EINVAL, "NULL argument");
    const int check = 10;
    double r = st->last_resid;
    int run = 0;
    bool conv = false;
    while (run < st->P.max_iter) {
        int chunk = std::min(check, st->P.max_iter - run);
        int32_t c = 0;
        int rc = mace_iterate(st, chunk, &r, &c);
        if (rc) return rc;
        run += chunk;
        if (c) { conv = true; break; }
    }
    int rc = mace_consensus(st, x_out, ptr_is_device);
    if (rc) return rc;
    if (iters_out) *iters_out = run;
    if (residual_out) *residual_out = r;
    if (!conv) return fail(MACE_ENOTCONVERGED, "max_iter reached before tol");
    return MACE_OK;
}

extern "C" int mace_get_state(mace_state *st, float *w, float *X, int32_t ptr_is_device)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    size_t bytes = sizeof(float) * st->B * st->M->N * st->n;
    if (w) { int rc = copy_out(w, st->d_w, bytes, ptr_is_device, st->stream); if (rc) return rc; }
    if (X) { int rc = copy_out(X, st->d_X, bytes, ptr_is_device, st->stream); if (rc) return rc; }
    return MACE_OK;
}

extern "C" int mace_set_state(mace_state *st, const float *w, const float *X, int32_t ptr_is_device)
{
    if (!st || !w || !X) return fail(MACE_EINVAL, "NULL argument");
    size_t bytes = sizeof(float) * st->B * st->M->N * st->n;
    int rc = copy_in(st->d_w, w, bytes, ptr_is_device, st->stream);
    if (!rc) rc = copy_in(st->d_X, X, bytes, ptr_is_device, st->stream);
    if (!rc) rc = launch_forward(st);
    if (!rc) {
        st->last_resid = INFINITY;
        CUDA_TRY(cudaStreamSynchronize(st->stream));
    }
    return rc;
}

extern "C" int mace_prox_pass(mace_state *st, const float *v, int32_t ptr_is_device, int32_t backward)
{
    if (!st || !v) return fail(MACE_EINVAL, "NULL argument");
    size_t bytes = sizeof(float) * st->B * st->M->N * st->n;
    if (!st->d_vexp && cudaMalloc(&st->d_vexp, bytes) != cudaSuccess) return fail(MACE_ENOMEM, "cudaMalloc v");
    int rc = copy_in(st->d_vexp, v, bytes, ptr_is_device, st->stream);
    if (!rc) rc = launch_sweep(st, backward ? 1 : 0, st->d_vexp);
    if (!rc) {
        int status = 0;
        CUDA_TRY(cudaMemcpyAsync(&status, st->d_status, sizeof(int), cudaMemcpyDeviceToHost, st->stream));
        CUDA_TRY(cudaStreamSynchronize(st->stream));
        if (status == kStatusTimeout) return fail(MACE_ETIMEOUT, "a device-side wait timed out");
        if (status == kStatusBounds)
            return fail(MACE_ECUDA, "a device-side bounds check failed (MACE_DEBUG build): stored matrix or state inconsistent");
    }
    return rc;
}

extern "C" int64_t mace_error_size(const mace_state *st) { return st ? (int64_t)st->B * st->ne : -1; }

extern "C" int mace_get_visit_order(const mace_state *st, int64_t *order)
{
    if (!st || !order) return fail(MACE_EINVAL, "NULL argument");
    const mace_sysmatrix *M = st->M;
    int64_t k = 0;
    for (int q = 0; q < M->nsv; ++q) {
        int sv = st->sv_order[q], si = sv / M->nsvx, sj = sv % M->nsvx;
        for (int t = 0; t < M->S2; ++t) {
            int i = si * M->S + t / M->S, j = sj * M->S + t % M->S;
            if (i < M->geo.ny && j < M->geo.nx) order[k++] = (int64_t)i * M->geo.nx + j;
        }
    }
    return MACE_OK;
}

extern "C" int mace_get_error(mace_state *st, float *e, int32_t ptr_is_device)
{
    if (!st || !e) return fail(MACE_EINVAL, "NULL argument");
    // strided copy of the .x components
    CUDA_TRY(cudaMemcpy2DAsync(e, sizeof(float), st->d_eL, sizeof(float2), sizeof(float), (size_t)st->B * st->ne,
                               ptr_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st->stream));
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    return MACE_OK;
}

extern "C" int mace_recompute_error(mace_state *st)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    int rc = launch_forward(st);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(st->stream));
    return MACE_OK;
}

extern "C" int mace_wait_selftest(uint32_t spin_limit, void *cuda_stream)
{
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int *d = nullptr, h = 0;
    CUDA_TRY(cudaMalloc(&d, sizeof(int)));
    cudaError_t ce = cudaMemsetAsync(d, 0, sizeof(int), s);
    if (ce == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, s>>>(spin_limit, d);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    cudaFree(d);
    if (ce != cudaSuccess) return fail(MACE_ECUDA, std::string("wait self test: ") + cudaGetErrorString(ce));
    if (h == kStatusTimeout) return fail(MACE_ETIMEOUT, "a device-side wait timed out");
    if (h == kStatusBounds)
        return fail(MACE_ECUDA, "a device-side bounds check failed (MACE_DEBUG build): stored matrix or state inconsistent");
    return MACE_OK;
}

extern "C" int mace_get_launch_info(const mace_state *st, int32_t *schedule, int32_t *warps_per_voxel,
                                    int32_t *warps)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    if (schedule) *schedule = st->P.schedule;
    if (warps_per_voxel) *warps_per_voxel = st->P.schedule == 1 ? st->wpv : 1;
    if (warps) *warps = st->sweep_warps;
    return MACE_OK;
}

extern "C" int mace_get_stats(const mace_state *st, int32_t *iters, double *sigma_abs, double *last_residual,
                              int32_t *concurrency, int32_t *chains)
{
    if (!st) return fail(MACE_EINVAL, "state is NULL");
    if (concurrency) *concurrency = st->concurrency;
    if (chains) *chains = st->chains;
    if (iters) *iters = st->iters;
    if (sigma_abs) *sigma_abs = st->sigma_abs;
    if (last_residual) *last_residual = st->last_resid;
    return MACE_OK;
}
