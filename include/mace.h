/*
 * mace.h -- C ABI of the GB300 library for partial-update MACE CT
 * reconstruction (Sridhar, Wang, Buzzard, Bouman, arXiv 1911.09278).
 *
 * The problem (Sec. II-A, Eqs. "MAP est", "global_obj", "local_obj"):
 *   x* = argmin_x  sum_k 1/2 ||y_k - A_k x||^2_{Lambda_k} + beta h(x),
 * split over N view subsets J_i (interleaved by default: J_i = {m : m mod N
 * = i}, 0-based) into agents f_i = sum_{k in J_i} ... + (beta/N) h(x).
 * Each agent's proximal map F_i (Eq. "prox_F") is replaced by its partial
 * update F~_i(v; X_i) (Algorithm 2: ICD passes from the state X_i), and the
 * Mann iteration of T = (2F - I)(2G - I) (Eqs. "w*_fixed_pt", "Mann") is run
 * as Algorithm 1:  v = (2G - I) w;  X = F~(v; X);  w <- rho (2X - v) +
 * (1 - rho) w;  solution x* = mean_i w_i.
 *
 * Conventions for every entry point:
 *   - Return value 0 on success, a negative MACE_E* code on failure; the
 *     message of the last failure on the calling thread is mace_last_error().
 *   - Handles are opaque and owned by the library; free them with the
 *     matching mace_free_* call.  A state borrows its system matrix, which
 *     must outlive every state built on it.
 *   - All device work is ordered on the CUDA stream given at creation (NULL
 *     = the legacy default stream).  Entry points that return host values
 *     synchronise that stream.
 *   - Image arrays are [nz][ny][nx] row-major (row 0 at the top); sinogram
 *     arrays are [nz][n_views][n_channels]; stacked agent images are
 *     [n_agents][nz*ny*nx].  All are float32.
 *   - ptr_is_device != 0 means the pointer is CUDA device memory read or
 *     written on the state's stream; otherwise it is host memory and the call
 *     copies synchronously.  Input pointers are only read during the call.
 *
 * The GPU never faults on bad input: arguments are checked on the host and
 * device-side waits are bounded (MACE_ETIMEOUT).
 */
#ifndef MACE_H
#define MACE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MACE_OK               0
#define MACE_EINVAL          -1   /* bad argument, shape or parameter       */
#define MACE_ENOMEM          -2   /* device or host allocation failed       */
#define MACE_ECUDA           -3   /* a CUDA runtime call failed             */
#define MACE_ENOTCONVERGED   -4   /* max_iter reached before tol            */
#define MACE_ETIMEOUT        -5   /* a bounded device-side wait expired     */
#define MACE_ENUMERIC        -6   /* non-finite residual (divergence)       */

typedef struct mace_sysmatrix mace_sysmatrix;
typedef struct mace_state mace_state;

/* Scanner geometry (Sec. II-A; the paper fixes parallel-beam views over
 * 180 degrees, Sec. IV, but not the projector).  Parallel beam; square
 * pixels of pitch pixel_pitch with pixel (row i, col j) centred at
 * ((j - (nx-1)/2) dx, ((ny-1)/2 - i) dx); channel c covers detector
 * coordinate t in [(c - n_channels/2) dd + off, (c + 1 - n_channels/2) dd +
 * off).  A[c, s] for view angle theta is the strip integral of pixel s over
 * channel c divided by dd (t = x cos theta + y sin theta).
 * view_angles: host array of n_views radians, or NULL for m pi / n_views.
 * nz > 1 is a stack of slices sharing the 2D matrix. */
typedef struct {
    int32_t nx, ny, nz;
    int32_t n_views, n_channels;
    double pixel_pitch, channel_pitch, channel_offset;
    const double *view_angles;
} mace_geometry;

/* View partition J_1..J_N (Sec. II-A, footnote: any partition).
 * view_agent: host array of n_views agent indices in [0, n_agents), or NULL
 * for interleaved subsets m mod n_agents.  Every agent needs >= 1 view. */
typedef struct {
    int32_t n_agents;
    const int32_t *view_agent;
} mace_partition;

typedef enum { MACE_F32 = 0, MACE_BF16 = 1, MACE_F16 = 2 } mace_dtype;

/* Prior, agent and solver parameters.
 *   prior 0: quadratic, rho(D) = D^2 / (2 sigma_x^2) (the x^T B x prior of
 *            Theorem 2, with h = 1/2 x^T B x);
 *   prior 1: Q-GGMRF, rho(D) = (D^2/(2 sigma_x^2)) / (1 + |D/(T sigma_x)|^(p-q)),
 *            p must be 2 (the paper cites the prior without defining it).
 *   h(x) = sum over neighbour pairs of b_sr rho(x_s - x_r), b_sr ~ 1/distance
 *   over the neighbourhood, normalised to sum 1.  neighbourhood 8: in-plane;
 *   neighbourhood 26: the batch of mace_init is the z-stack of ONE volume
 *   (batch element b is slice z = b, all slices share the 2D matrix) and the
 *   prior couples neighbouring slices; with schedule 0 all slices are
 *   updated at once, each reading its neighbour slices as they were when its
 *   super-voxel began; with schedule 1 even slices are swept first, then odd
 *   ones (see schedule).
 *   sigma: the proximal parameter of Eq. "prox_F"; sigma_mode 0 takes it in
 *   image units, 1 scales it by 1/sqrt(mean_{i,s} sum_{k in J_i} A^2 Lambda).
 *   rho in (0, 1): Mann parameter (Eq. "Mann").
 *   sweeps_per_iter >= 1 ICD passes per Mann iteration; symmetric != 0 runs
 *   every second pass in reverse voxel order.
 *   recompute_every > 0: e_i = y_i - A_i X_i is recomputed from scratch every
 *   that many iterations (removes float drift); 0 never.
 *   max_iter, tol: mace_reconstruct stops when the relative Mann residual
 *   ||w^(k+1) - w^(k)|| / ||w^(k+1)|| (FP64) falls below tol.
 *   concurrency: super-voxels of one agent updated at the same time (0 =
 *   every warp the GPU holds; 1 = one at a time, the serial ICD order;
 *   -1 = one per row of super-voxels, so with sv_order 0 each warp sweeps
 *   one row and the rows advance side by side -- on the 512^2 workload
 *   this converges in the fewest iterations of the settings measured).
 *   Always capped by the warps the GPU holds.
 *   sv_order: 0 visits super-voxels in raster order cut into `concurrency`
 *   bands that run side by side (plain raster when concurrency is 1);
 *   1 a stride permutation spreading consecutive super-voxels apart.
 *   Pixels inside a super-voxel are visited in raster order.
 *   chains: reconstructions of a batch (slices of a volume) one warp updates
 *   together, sharing every column load (0 or 1: one; 2 or 4: two, the warp
 *   then working as two 16-lane halves, one per reconstruction; schedule 0:
 *   when the batch is even, slices 2k and 2k + 1; schedule 1: volumes only,
 *   when the slice count is a multiple of 4, two slices of one z parity,
 *   z and z + 2).  Results do not depend on it.
 *   pnp: 0 = Algorithm 1 (the prior inside every agent, weight beta/N);
 *   1 = Algorithm 3 (Sec. III, MACE with a plug-and-play prior): the agents
 *   hold the data terms only and use proximal parameter sqrt(N) sigma; the
 *   consensus operator is G_H(w) = H(mean_i w_i) for every agent, and the
 *   solution is H(mean_i w_i).  H is the proximal map of the prior beta h at
 *   sigma, H(v) = (I + sigma^2 beta B)^-1 v for the quadratic prior (the only
 *   one accepted with pnp = 1, 8-neighbourhood), solved in FP64 by Jacobi
 *   iterations to round-off.  H is firmly non-expansive, so by Theorem 3 and
 *   Lemma 2 the fixed point is the MAP image of the whole cost.
 *   forward_geometry: how the periodic recompute e_i = y_i - A_i X_i (and
 *   the initial one) gets A_i.  1 = it evaluates A_i's strip-integral
 *   footprints from the geometry (the super-voxel's projection in FP64, the
 *   rest in FP32), so with BF16/FP16 stored values the recompute still sees
 *   the exact projector; 2 = it reads the stored values; 0 (default) = 1
 *   for BF16/FP16 stored values, 2 for FP32.  The ICD updates keep using
 *   the stored values; with the geometry recompute the fixed point matches
 *   the exact MAP image more closely than that of the rounded matrix.
 *   deterministic: 0 = the super-voxels of an agent in flight run freely:
 *   each reads the error sinogram when it starts and adds its change back
 *   when it ends (float atomics), so the result depends on the GPU's
 *   scheduling at the level of float rounding; 1 = they advance in lock-step
 *   phases (a phase is one super-voxel per warp: all of a phase's reads come
 *   before any of its writes, all its writes before the next phase's reads)
 *   and the changes are summed in 64-bit fixed point, so every run, alone or
 *   beside other work, eagerly or from a captured graph, gives the same bits.
 *   The e recompute and the initial normalisation are order-independent in
 *   both modes.
 *   schedule: how warps get super-voxels.  0 (fixed) = C warps per
 *   (reconstruction, agent) pair, every one resident for the whole pass,
 *   warp c taking the c-th of every C super-voxels of its pair's order (C
 *   from concurrency, capped so that every pair fits on the GPU at once);
 *   1 (work queue) = a persistent grid of every resident warp takes work
 *   items from a counter, an item being one of `concurrency` interleaved
 *   shares of one pair's order (0 or -1: one per row of super-voxels), so
 *   any number of pairs runs, a warp that finishes early takes more work,
 *   and slices of a volume (neighbourhood 26) are swept even ones first,
 *   then odd ones, each reading neighbour slices that are not being
 *   updated.  Schedule 1 runs one chain per warp and the free mode
 *   (deterministic 0).
 *   warps_per_voxel (schedule 1, neighbourhood 8): 1, 2 or 4 warps of one
 *   block sweep the same super-voxels together, each holding its share of
 *   the agent's views (views 32 (w + W j) + lane of warp w) and its share of
 *   the error-sinogram band; a pixel's theta1 is the sum of the warps'
 *   partial sums, added in warp order through shared memory, so every warp
 *   takes the same step (Algorithm 2 is unchanged).  For agents with many
 *   views: fewer views per warp, but more shared memory per view, so fewer
 *   super-voxels at a time; which wins depends on the scan (the autotuner
 *   measures it).  0 = 1.  A group runs the smallest of its members'. */
typedef struct {
    int32_t prior;
    int32_t neighbourhood;
    double beta, sigma_x, p, q, T;
    double sigma;
    int32_t sigma_mode;
    double rho;
    int32_t sweeps_per_iter;
    int32_t symmetric;
    int32_t recompute_every;
    int32_t max_iter;
    double tol;
    int32_t concurrency;
    int32_t sv_order;
    int32_t chains;
    int32_t pnp;
    int32_t forward_geometry;
    int32_t deterministic;
    int32_t schedule;
    int32_t warps_per_voxel;
} mace_params;

/* Sizes of a built system matrix (for memory accounting, Table 3). */
typedef struct {
    int64_t n_voxels;        /* nx*ny (one slice)                          */
    int32_t n_agents, sv_size, n_sv;   /* super-voxels per agent             */
    int32_t max_views;       /* largest |J_i|                              */
    int64_t nnz;             /* stored non-zeros over all agents           */
    int64_t bytes_columns;   /* headers + values + padding                 */
    int64_t bytes_meta;      /* offsets and band descriptors               */
    int64_t agent_bytes[64]; /* column bytes of agents 0..63               */
} mace_sysmatrix_info;

/* Build the stored system matrix (the paper precomputes and stores A,
 * Sec. I and Table 3) for every agent: voxel-column-major per super-voxel
 * (sv_size x sv_size pixel tiles), per view a run (first channel, length
 * 0..3, values): one header byte per (pixel, view) holding the run's length
 * and its first channel relative to the super-voxel's band in that view,
 * the first two values per view, and the third values of three-channel runs
 * in a short list.  dtype selects the stored value type.  Runs on the GPU
 * on cuda_stream (a cudaStream_t or NULL).  *out receives the handle.
 * Errors: MACE_EINVAL (sizes, angles, partition, sv_size not 4, 8, 16 or
 * 32, more than 4096 views, a super-voxel band wider than 62 channels in a
 * view), MACE_ENOMEM, MACE_ECUDA. */
int mace_build_sysmatrix(const mace_geometry *geom, const mace_partition *part,
                         mace_dtype dtype, int32_t sv_size, void *cuda_stream,
                         mace_sysmatrix **out);

int mace_sysmatrix_get_info(const mace_sysmatrix *sm, mace_sysmatrix_info *info);

/* Decode the stored column of pixel (row i, col j) for agent g: for each of
 * the agent's views (increasing m) the first channel, run length and values
 * (widened to float).  c0, len: [|J_g|]; vals: [3 |J_g|], zero-padded.
 * Host arrays; copies a few hundred bytes from the device. */
int mace_sysmatrix_column(const mace_sysmatrix *sm, int32_t g, int32_t i, int32_t j,
                          int32_t *c0, int32_t *len, float *vals);

/* Create a reconstruction state for a batch of `batch` independent
 * reconstructions that share the system matrix (same geometry and
 * partition, different data).  Copies y and weights (Lambda, the inverse
 * noise variances), [batch][nz][n_views][n_channels], into agent-major device
 * layout, sets w^(0) = w0 (NULL = 0; [batch][n_agents][n] float32), X^(0) =
 * G(w^(0)) (Algorithm 1 initialisation) and e_i = y_i - A_i X_i.  Work is
 * ordered on cuda_stream.  All arrays of a state below carry the leading
 * batch dimension.
 * Errors: MACE_EINVAL (batch not in [1, 4096], parameters out of range,
 * non-finite or negative weights), MACE_ENOMEM, MACE_ECUDA. */
int mace_init(const mace_sysmatrix *sm, int32_t batch, const float *y, const float *weights,
              int32_t ptr_is_device, const mace_params *params, const float *w0,
              void *cuda_stream, mace_state **out);

/* Device memory a state of `batch` reconstructions on this matrix with these
 * parameters takes: *persistent = the bytes mace_init allocates and keeps
 * until mace_free_state; *peak = that plus its transient buffers during
 * mace_init (input staging when ptr_is_device == 0, per-super-voxel
 * partial sums).  For admission control by a server (Sec. IV serves no
 * requests; this is the library's own accounting).  mace_prox_pass
 * allocates one more [batch][n_agents][n] float32 array on first use, not
 * counted here.  Errors: MACE_EINVAL (as mace_init's parameter checks). */
int mace_state_bytes(const mace_sysmatrix *sm, int32_t batch, const mace_params *params,
                     int32_t ptr_is_device, int64_t *persistent, int64_t *peak);

/* Run n_iters Mann iterations of Algorithm 1 on every reconstruction of the
 * batch.  residual_out (may be NULL) receives the largest relative Mann
 * residual over the batch at the last iteration (FP64); converged_out (may
 * be NULL) is set to 1 once it is below params.tol.
 * Errors: MACE_ENUMERIC when the residual is not finite, MACE_ETIMEOUT,
 * MACE_ECUDA. */
int mace_iterate(mace_state *st, int32_t n_iters, double *residual_out,
                 int32_t *converged_out);

/* Asynchronous form of mace_iterate: mace_launch enqueues n_iters
 * iterations on the state's stream and returns without waiting; mace_poll
 * waits for the stream and reports the last residual (as mace_iterate).
 * States on different streams then run on the GPU at the same time. */
int mace_launch(mace_state *st, int32_t n_iters);
int mace_poll(mace_state *st, double *residual_out, int32_t *converged_out);

/* Non-blocking status.  mace_poll_async enqueues on the state's stream,
 * after the iterations launched so far, a copy of the batch's Mann
 * residuals and the device status word into host memory the state owns,
 * and records an event; it returns at once.  mace_poll_ready never waits:
 * *ready_out = 0 while that copy is in flight; once it has landed,
 * *ready_out = 1 and residual_out / converged_out are set as by mace_poll
 * (a caller may launch further iterations meanwhile: the status is the one
 * at the point mace_poll_async was called).  Without a pending
 * mace_poll_async, *ready_out = 1 with the last known residual.
 * Errors: as mace_poll (MACE_ENUMERIC, MACE_ETIMEOUT, MACE_ECUDA). */
int mace_poll_async(mace_state *st);
int mace_poll_ready(mace_state *st, double *residual_out, int32_t *converged_out, int32_t *ready_out);

/* Iterate until the residual is below params.tol or params.max_iter
 * iterations have run (checking every 10 iterations), then write the
 * consensus images x* = mean_i w_i (Algorithm 1 output) to x_out
 * ([batch][nz][ny][nx]).
 * Returns MACE_ENOTCONVERGED (x_out still written) if max_iter was hit. */
int mace_reconstruct(mace_state *st, float *x_out, int32_t ptr_is_device,
                     int32_t *iters_out, double *residual_out);

/* Consensus image mean_i w_i of the current state, without iterating. */
int mace_consensus(mace_state *st, float *x_out, int32_t ptr_is_device);

/* mace_consensus without any device allocation, for callers that may not
 * allocate GPU memory after start-up: a service that reserves all device
 * memory once and forbids allocation on its per-scan path (cudaMalloc can
 * synchronise the device and fragment a fixed budget), or code that runs
 * under another framework whose caching allocator owns the free memory.
 * The paper has no counterpart; it only reads the result out.
 * With ptr_is_device != 0 the images go straight to x_out.  With host x_out
 * they pass through a 4 MiB device array inside the library (at most
 * 1048576 floats = batch * nz * ny * nx; larger requests return MACE_EINVAL).
 * That array belongs to the library for the life of the process on every
 * GPU that loads it, and all calls on one GPU share it: calls whose GPU work
 * overlaps (other streams or host threads) race on it.  mace_init looks up
 * the array's device address (cudaGetSymbolAddress) and keeps it in the
 * state, so this call does no set-up of its own.  Calls no allocator. */
int mace_consensus_noalloc(mace_state *st, float *x_out, int32_t ptr_is_device);

/* Checkpoint / resume: the complete algorithm state is (w, X) (Eq.
 * "PUCEupdate"); e_i is recomputed from X on mace_set_state.  w, X:
 * [batch][n_agents][n] float32 (either may be NULL in get_state). */
int mace_get_state(mace_state *st, float *w, float *X, int32_t ptr_is_device);
int mace_set_state(mace_state *st, const float *w, const float *X, int32_t ptr_is_device);

/* One partial-update pass X_i <- F~_i(v_i; X_i) (Algorithm 2) for every
 * agent with the given v ([batch][n_agents][n] float32), without touching w.
 * backward != 0 visits voxels in reverse order.  For testing the agent
 * update in isolation. */
int mace_prox_pass(mace_state *st, const float *v, int32_t ptr_is_device, int32_t backward);

/* The pixel visiting order of a forward ICD pass of this state (raster
 * indices i*nx + j, nx*ny entries); a backward pass visits it from the end.
 * With params.concurrency = 1 each agent's pass is exactly Algorithm 2 in
 * this order. */
int mace_get_visit_order(const mace_state *st, int64_t *order);

/* Error sinograms e_i in agent-local layout: agent g's block is
 * [nz][|J_g|][n_channels], agents concatenated in order, reconstructions
 * concatenated; mace_error_size gives the total count. */
int mace_get_error(mace_state *st, float *e, int32_t ptr_is_device);
int64_t mace_error_size(const mace_state *st);

/* Recompute e_i = y_i - A_i X_i from scratch. */
int mace_recompute_error(mace_state *st);

/* Iterations run so far, the proximal sigma in image units, the last
 * residual, the super-voxels of one agent in flight per pass and the
 * reconstructions one warp updates together. */
int mace_get_stats(const mace_state *st, int32_t *iters, double *sigma_abs,
                   double *last_residual, int32_t *concurrency, int32_t *chains);

/* The sweep's launch configuration: params.schedule, the warps per
 * super-voxel in use (1 for schedule 0) and the warps the sweep launches
 * (schedule 0) or keeps resident (schedule 1).  Any pointer may be NULL. */
int mace_get_launch_info(const mace_state *st, int32_t *schedule, int32_t *warps_per_voxel, int32_t *warps);

/* Groups: the Mann iterations of several states (different scans,
 * geometries and parameters; params.schedule = 1, neighbourhood 8, one
 * stored value type) advanced together, the ICD passes of all of them in
 * one queue-fed launch per pass, so a small reconstruction does not hold
 * the GPU alone and warps that finish one state's work take another's.
 * mace_group_create takes the member states (not owned; each must outlive
 * the group and belong to no group launch in flight on another stream)
 * and the CUDA stream (NULL = legacy default) the group enqueues on.
 * mace_group_launch enqueues n_iters Mann iterations of every member
 * (Algorithm 1 per member; each member's iterates are those of
 * mace_launch on it alone, up to the order of float additions); the group's
 * stream first waits for each member's stream, and each member's stream
 * then waits for the group's, so mace_poll / mace_poll_async /
 * mace_consensus on a member see the group's iterations.  Returns without
 * waiting.  mace_group_update replaces the members (a server admitting and
 * retiring requests): stream-ordered, it neither waits for the group's work
 * in flight nor synchronises the device; on error the group keeps its
 * previous members.  mace_group_free releases the group's descriptors (not
 * the members).  Errors: MACE_EINVAL (schedule 0 or volume members, a
 * member twice, mixed value types, n outside [1, 65536]), MACE_ENOMEM,
 * MACE_ECUDA. */
typedef struct mace_group mace_group;
int mace_group_create(mace_state *const *members, int32_t n, void *cuda_stream, mace_group **out);
int mace_group_update(mace_group *group, mace_state *const *members, int32_t n);
int mace_group_launch(mace_group *group, int32_t n_iters);
int mace_group_free(mace_group *group);

/* CUDA-event timing of the ICD sweep launches on the state's stream:
 * mace_set_timing(st, 1, max_launches) starts recording (up to max_launches
 * launches); mace_get_timing returns the summed device time in ms and the
 * number of launches recorded since, then restarts the count. */
int mace_set_timing(mace_state *st, int32_t enable, int32_t max_launches);
int mace_get_timing(mace_state *st, double *sweep_ms, int32_t *launches);

/* Failure detection without a GPU fault: launch one warp that waits on a
 * barrier nothing completes, with the sweep's bounded wait cut to spin_limit
 * polls; returns MACE_ETIMEOUT (the kernel records it and exits, the context
 * stays usable).  Not part of the paper's method. */
int mace_wait_selftest(uint32_t spin_limit, void *cuda_stream);

void mace_free_state(mace_state *st);
void mace_free_sysmatrix(mace_sysmatrix *sm);
const char *mace_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MACE_H */
