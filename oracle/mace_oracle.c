/*
 * FP64 CPU oracle for partial-update MACE CT reconstruction
 * (Sridhar, Wang, Buzzard, Bouman, "Distributed Iterative CT Reconstruction
 * using Multi-Agent Consensus Equilibrium", arXiv 1911.09278).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously-correct
 * reference that the CUDA library is checked against.  It shares no code with
 * the CUDA path; only the test suite, the smoke check and the benchmark's CPU
 * baseline may load it.
 *
 * Everything is double precision, written in the order the paper states it:
 *   - MAP cost f(x) = sum_k 1/2 ||y_k - A_k x||^2_{Lambda_k} + beta h(x)
 *     (Sec. II-A, Eq. "global_obj"), split over interleaved view subsets J_i
 *     into f_i = sum_{k in J_i} ... + (beta/N) h(x)  (Eq. "local_obj").
 *   - ICD partial update of the proximal map F_i (Algorithm 2): one pass of
 *     exact coordinate minimisation of f_i(z) + ||z - v||^2 / (2 sigma^2).
 *   - Partial-update MACE (Algorithm 1): v = (2G - I) w; X = F~(v; X);
 *     w <- rho (2X - v) + (1 - rho) w; solution x* = mean_i w_i.
 *   - Centralised MAP by plain ICD (the single-node method of Sec. IV-A).
 *   - Partial-update MACE with a plug-and-play denoiser (Sec. III,
 *     Algorithm 3): agents hold the data terms only and use proximal
 *     parameter sqrt(N) sigma; the consensus operator is
 *     G_H(w) = H(mean_i w_i) for every agent; the solution is H(mean_i w_i).
 *     H here is the proximal map of beta h at sigma, computed to convergence.
 *
 * Readings of things the paper leaves open (the paper cites but does not
 * define the projector, the Q-GGMRF prior and the stopping rule):
 *   - Projector: parallel beam, square pixels of pitch dx, channels of pitch
 *     dd.  A[c, s] is the strip integral of pixel s over channel c divided by
 *     dd: the pixel's projection is a trapezoid of unit area with widths
 *     dx|cos t|/dd and dx|sin t|/dd (in channel units), integrated exactly over
 *     the channel.  Channel c holds the edge coordinate interval [c, c+1).
 *   - Prior: h(x) = sum over unordered neighbour pairs {s,r} of
 *     b_sr rho(x_s - x_r); b_sr proportional to 1/distance over the 8 (2D) or
 *     26 (3D) neighbourhood, normalised to sum 1 over the full neighbourhood,
 *     out-of-volume neighbours dropped.  Quadratic: rho = D^2/(2 sx^2).
 *     Q-GGMRF (p = 2): rho = (D^2/(2 sx^2)) / (1 + |D/(T sx)|^(p-q)).
 *   - Coordinate minimisation for Q-GGMRF uses the symmetric tangent
 *     quadratic surrogate, weight rho'(D)/D, whose step is zero exactly when
 *     the coordinate derivative is zero, so Lemma B.1 and the fixed point of
 *     Algorithm 1 (Theorem 1) are unchanged.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL -1
#define OR_ENOMEM -2

typedef struct {
    int32_t nx, ny, nz;             /* image columns, rows, slices           */
    int32_t n_views, n_channels;    /* views over [0, pi), detector channels */
    double pixel_pitch;             /* dx                                    */
    double channel_pitch;           /* dd                                    */
    double channel_offset;          /* detector centre offset (same units)   */
    const double *cos_t, *sin_t;    /* [n_views]                             */
    const double *y, *lam;          /* [nz][n_views][n_channels]             */
    int32_t n_agents;
    const int32_t *view_agent;      /* [n_views], agent owning each view     */
    int32_t prior;                  /* 0 quadratic, 1 Q-GGMRF                */
    int32_t neighbourhood;          /* 8 (in-plane) or 26 (3D)               */
    double beta, sigma_x, p, q, T;
} or_problem;

int or_version(void) { return 4; }

/* ---------------------------------------------------------------------- */
/* View angles theta_m = m pi / N_theta (Sec. IV: views uniform over 180 deg) */
void or_angles(int32_t n_views, double *cos_t, double *sin_t)
{
    for (int32_t m = 0; m < n_views; ++m) {
        double th = (double)m * M_PI / (double)n_views;
        cos_t[m] = cos(th);
        sin_t[m] = sin(th);
    }
}

/* CDF of the unit-area trapezoid with widths w1 <= w2 (channel units),
 * centred at 0, evaluated at u. */
static double trap_cdf(double u, double w1, double w2)
{
    double u1 = 0.5 * (w2 - w1);
    double u2 = 0.5 * (w2 + w1);
    double h = 1.0 / w2;
    if (u <= -u2) return 0.0;
    if (u < -u1) { double d = u + u2; return h * d * d / (2.0 * w1); }
    if (u <= u1) return h * (0.5 * w1 + (u + u1));
    if (u < u2) { double d = u2 - u; return 1.0 - h * d * d / (2.0 * w1); }
    return 1.0;
}

/* Column entry of pixel (row i, col j) for view m: first channel, run
 * length (0..3) and values.  Returns the run length. */
int32_t or_footprint(const or_problem *P, int32_t m, int32_t i, int32_t j,
                     int32_t *c0_out, double *vals)
{
    double dx = P->pixel_pitch, dd = P->channel_pitch;
    double ct = P->cos_t[m], st = P->sin_t[m];
    double xc = ((double)j - 0.5 * (double)(P->nx - 1)) * dx;
    double yc = (0.5 * (double)(P->ny - 1) - (double)i) * dx;
    double t0 = xc * ct + yc * st;
    double qc = (t0 - P->channel_offset) / dd + 0.5 * (double)P->n_channels;
    double a = dx * fabs(ct) / dd;
    double b = dx * fabs(st) / dd;
    double w1 = a < b ? a : b;
    double w2 = a < b ? b : a;
    double half = 0.5 * (a + b);
    double lo = qc - half, hi = qc + half;
    int32_t cf = (int32_t)floor(lo);
    int32_t cl = (int32_t)ceil(hi) - 1;
    if (cf < 0) cf = 0;
    if (cl > P->n_channels - 1) cl = P->n_channels - 1;
    int32_t L = cl - cf + 1;
    if (L < 0) L = 0;
    double scale = dx * dx / dd;
    for (int32_t k = 0; k < L; ++k) {
        double c = (double)(cf + k);
        vals[k] = scale * (trap_cdf(c + 1.0 - qc, w1, w2) - trap_cdf(c - qc, w1, w2));
    }
    *c0_out = cf;
    return L;
}

/* Dense system matrix of one slice, rows (view m, channel c), columns raster
 * pixels.  out is [n_views * n_channels][nx * ny], zero-filled here. */
void or_dense_A(const or_problem *P, double *out)
{
    int64_t n = (int64_t)P->nx * P->ny;
    memset(out, 0, sizeof(double) * (size_t)(n * P->n_views * P->n_channels));
    for (int32_t m = 0; m < P->n_views; ++m)
        for (int32_t i = 0; i < P->ny; ++i)
            for (int32_t j = 0; j < P->nx; ++j) {
                int32_t c0; double v[3];
                int32_t L = or_footprint(P, m, i, j, &c0, v);
                for (int32_t k = 0; k < L; ++k)
                    out[((int64_t)m * P->n_channels + c0 + k) * n + (int64_t)i * P->nx + j] = v[k];
            }
}

/* ---------------------------------------------------------------------- */
/* Prior: neighbour offsets and normalised weights b_sr. */
typedef struct { int dz, di, dj; double b; } nbr_t;

static int make_nbrs(int32_t neighbourhood, nbr_t *nb)
{
    int cnt = 0; double tot = 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int di = -1; di <= 1; ++di)
            for (int dj = -1; dj <= 1; ++dj) {
                if (!dz && !di && !dj) continue;
                if (neighbourhood == 8 && dz) continue;
                double d2 = (double)(dz * dz + di * di + dj * dj);
                nb[cnt].dz = dz; nb[cnt].di = di; nb[cnt].dj = dj;
                nb[cnt].b = 1.0 / sqrt(d2);
                tot += nb[cnt].b;
                ++cnt;
            }
    for (int k = 0; k < cnt; ++k) nb[k].b /= tot;
    return cnt;
}

/* rho'(D)/D: the surrogate weight (exact for the quadratic prior). */
static double prior_weight(const or_problem *P, double d)
{
    double s2 = P->sigma_x * P->sigma_x;
    if (P->prior == 0) return 1.0 / s2;
    double a = pow(fabs(d / (P->T * P->sigma_x)), P->p - P->q);
    return (2.0 + P->q * a) / (2.0 * s2 * (1.0 + a) * (1.0 + a));
}

static double prior_rho(const or_problem *P, double d)
{
    double s2 = P->sigma_x * P->sigma_x;
    double quad = d * d / (2.0 * s2);
    if (P->prior == 0) return quad;
    return quad / (1.0 + pow(fabs(d / (P->T * P->sigma_x)), P->p - P->q));
}

/* ---------------------------------------------------------------------- */
/* Views of agent g in increasing m (interleaved subsets J_i, Sec. II-A).
 * g < 0 selects every view (the centralised problem). */
static int32_t agent_views(const or_problem *P, int32_t g, int32_t *views)
{
    int32_t cnt = 0;
    for (int32_t m = 0; m < P->n_views; ++m)
        if (g < 0 || P->view_agent[m] == g) views[cnt++] = m;
    return cnt;
}

int32_t or_agent_views(const or_problem *P, int32_t g, int32_t *views)
{
    return agent_views(P, g, views);
}

/* e = y_J - A_J x for the views of agent g; e is [nz][|J|][n_channels]. */
void or_error_sinogram(const or_problem *P, int32_t g, const double *x, double *e)
{
    int32_t *views = (int32_t *)malloc(sizeof(int32_t) * (size_t)P->n_views);
    int32_t V = agent_views(P, g, views);
    int64_t D = P->n_channels, plane = (int64_t)P->nx * P->ny;
    for (int32_t z = 0; z < P->nz; ++z)
        for (int32_t vl = 0; vl < V; ++vl) {
            int32_t m = views[vl];
            double *ev = e + ((int64_t)z * V + vl) * D;
            const double *yv = P->y + ((int64_t)z * P->n_views + m) * D;
            for (int64_t c = 0; c < D; ++c) ev[c] = yv[c];
            for (int32_t i = 0; i < P->ny; ++i)
                for (int32_t j = 0; j < P->nx; ++j) {
                    double xs = x[z * plane + (int64_t)i * P->nx + j];
                    int32_t c0; double a[3];
                    int32_t L = or_footprint(P, m, i, j, &c0, a);
                    for (int32_t k = 0; k < L; ++k) ev[c0 + k] -= a[k] * xs;
                }
        }
    free(views);
}

/* theta2_s = sum_{k in J, c} A^2 Lambda for every voxel (the data part of the
 * diagonal of H_i, Theorem 2 proof). */
void or_theta2(const or_problem *P, int32_t g, double *out)
{
    int32_t *views = (int32_t *)malloc(sizeof(int32_t) * (size_t)P->n_views);
    int32_t V = agent_views(P, g, views);
    int64_t D = P->n_channels, plane = (int64_t)P->nx * P->ny;
    for (int32_t z = 0; z < P->nz; ++z)
        for (int32_t i = 0; i < P->ny; ++i)
            for (int32_t j = 0; j < P->nx; ++j) {
                double t2 = 0.0;
                for (int32_t vl = 0; vl < V; ++vl) {
                    int32_t m = views[vl], c0; double a[3];
                    int32_t L = or_footprint(P, m, i, j, &c0, a);
                    const double *lv = P->lam + ((int64_t)z * P->n_views + m) * D;
                    for (int32_t k = 0; k < L; ++k) t2 += a[k] * a[k] * lv[c0 + k];
                }
                out[z * plane + (int64_t)i * P->nx + j] = t2;
            }
    free(views);
}

/* One ICD pass (Algorithm 2) for agent g (g < 0: all views).
 *   prox != 0: minimise f_i(z) + ||z - v||^2/(2 sigma^2) coordinate-wise;
 *   prox == 0: minimise the cost alone (centralised ICD), v unused.
 * pscale multiplies h (beta/N for an agent, beta for the centralised cost).
 * order: voxel visiting order (NULL = raster).  x and e are updated in
 * place; e must equal y_J - A_J x on entry.  Returns sum of alpha^2. */
static double icd_sweep_dir(const or_problem *P, int32_t g, int32_t prox, double sigma,
                            double pscale, const int64_t *order, int32_t backward,
                            const double *v, double *x, double *e);

double or_icd_sweep(const or_problem *P, int32_t g, int32_t prox, double sigma,
                    double pscale, const int64_t *order, const double *v,
                    double *x, double *e)
{
    return icd_sweep_dir(P, g, prox, sigma, pscale, order, 0, v, x, e);
}

/* backward != 0 visits the order from its end (the second half of a
 * symmetric ICD pass). */
static double icd_sweep_dir(const or_problem *P, int32_t g, int32_t prox, double sigma,
                            double pscale, const int64_t *order, int32_t backward,
                            const double *v, double *x, double *e)
{
    int32_t *views = (int32_t *)malloc(sizeof(int32_t) * (size_t)P->n_views);
    int32_t V = agent_views(P, g, views);
    nbr_t nb[26];
    int nnb = make_nbrs(P->neighbourhood, nb);
    int64_t D = P->n_channels, plane = (int64_t)P->nx * P->ny;
    int64_t n = plane * P->nz;
    double inv_s2 = prox ? 1.0 / (sigma * sigma) : 0.0;
    double sum_a2 = 0.0;
    int32_t *c0s = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    int32_t *Ls = (int32_t *)malloc(sizeof(int32_t) * (size_t)V);
    double *as = (double *)malloc(sizeof(double) * 3 * (size_t)V);
    for (int64_t tt = 0; tt < n; ++tt) {
        int64_t t = backward ? n - 1 - tt : tt;
        int64_t s = order ? order[t] : t;
        int32_t z = (int32_t)(s / plane);
        int32_t i = (int32_t)((s % plane) / P->nx);
        int32_t j = (int32_t)(s % P->nx);
        /* data term: theta1 = -sum A Lambda e, theta2 = sum A^2 Lambda */
        double th1 = 0.0, th2 = 0.0;
        for (int32_t vl = 0; vl < V; ++vl) {
            int32_t m = views[vl];
            Ls[vl] = or_footprint(P, m, i, j, &c0s[vl], &as[3 * vl]);
            const double *lv = P->lam + ((int64_t)z * P->n_views + m) * D;
            const double *ev = e + ((int64_t)z * V + vl) * D;
            for (int32_t k = 0; k < Ls[vl]; ++k) {
                double a = as[3 * vl + k];
                double l = lv[c0s[vl] + k];
                th1 -= a * l * ev[c0s[vl] + k];
                th2 += a * a * l;
            }
        }
        /* prior term through the surrogate weights at the current state */
        double gp = 0.0, hp = 0.0;
        for (int k = 0; k < nnb; ++k) {
            int32_t zz = z + nb[k].dz, ii = i + nb[k].di, jj = j + nb[k].dj;
            if (zz < 0 || zz >= P->nz || ii < 0 || ii >= P->ny || jj < 0 || jj >= P->nx)
                continue;
            double d = x[s] - x[zz * plane + (int64_t)ii * P->nx + jj];
            double wgt = nb[k].b * prior_weight(P, d);
            gp += wgt * d;
            hp += wgt;
        }
        gp *= pscale; hp *= pscale;
        double num = th1 + gp + (prox ? (x[s] - v[s]) * inv_s2 : 0.0);
        double den = th2 + hp + inv_s2;
        double alpha = den > 0.0 ? -num / den : 0.0;
        x[s] += alpha;
        sum_a2 += alpha * alpha;
        for (int32_t vl = 0; vl < V; ++vl) {
            double *ev = e + ((int64_t)z * V + vl) * D;
            for (int32_t k = 0; k < Ls[vl]; ++k) ev[c0s[vl] + k] -= as[3 * vl + k] * alpha;
        }
    }
    free(as); free(Ls); free(c0s); free(views);
    return sum_a2;
}

/* ---------------------------------------------------------------------- */
/* MAP cost f(x) (Eq. "global_obj") and its gradient. */
double or_cost(const or_problem *P, const double *x)
{
    int64_t D = P->n_channels, plane = (int64_t)P->nx * P->ny;
    int64_t ne = (int64_t)P->nz * P->n_views * D;
    double *e = (double *)malloc(sizeof(double) * (size_t)ne);
    or_error_sinogram(P, -1, x, e);
    double data = 0.0;
    for (int64_t k = 0; k < ne; ++k) data += 0.5 * P->lam[k] * e[k] * e[k];
    free(e);
    nbr_t nb[26];
    int nnb = make_nbrs(P->neighbourhood, nb);
    double h = 0.0;
    for (int32_t z = 0; z < P->nz; ++z)
        for (int32_t i = 0; i < P->ny; ++i)
            for (int32_t j = 0; j < P->nx; ++j)
                for (int k = 0; k < nnb; ++k) {
                    int32_t zz = z + nb[k].dz, ii = i + nb[k].di, jj = j + nb[k].dj;
                    if (zz < 0 || zz >= P->nz || ii < 0 || ii >= P->ny || jj < 0 || jj >= P->nx)
                        continue;
                    /* every unordered pair is visited twice */
                    double d = x[z * plane + (int64_t)i * P->nx + j] - x[zz * plane + (int64_t)ii * P->nx + jj];
                    h += 0.5 * nb[k].b * prior_rho(P, d);
                }
    return data + P->beta * h;
}

void or_gradient(const or_problem *P, const double *x, double *grad)
{
    int64_t D = P->n_channels, plane = (int64_t)P->nx * P->ny;
    int64_t ne = (int64_t)P->nz * P->n_views * D;
    double *e = (double *)malloc(sizeof(double) * (size_t)ne);
    or_error_sinogram(P, -1, x, e);
    nbr_t nb[26];
    int nnb = make_nbrs(P->neighbourhood, nb);
    for (int32_t z = 0; z < P->nz; ++z)
        for (int32_t i = 0; i < P->ny; ++i)
            for (int32_t j = 0; j < P->nx; ++j) {
                int64_t s = z * plane + (int64_t)i * P->nx + j;
                double g = 0.0;
                for (int32_t m = 0; m < P->n_views; ++m) {
                    int32_t c0; double a[3];
                    int32_t L = or_footprint(P, m, i, j, &c0, a);
                    int64_t row = ((int64_t)z * P->n_views + m) * D;
                    for (int32_t k = 0; k < L; ++k)
                        g -= a[k] * P->lam[row + c0 + k] * e[row + c0 + k];
                }
                double gp = 0.0;
                for (int k = 0; k < nnb; ++k) {
                    int32_t zz = z + nb[k].dz, ii = i + nb[k].di, jj = j + nb[k].dj;
                    if (zz < 0 || zz >= P->nz || ii < 0 || ii >= P->ny || jj < 0 || jj >= P->nx)
                        continue;
                    double d = x[s] - x[zz * plane + (int64_t)ii * P->nx + jj];
                    gp += nb[k].b * prior_weight(P, d) * d;
                }
                grad[s] = g + P->beta * gp;
            }
    free(e);
}

/* ---------------------------------------------------------------------- */
/* Centralised MAP by plain ICD (all views, no proximal term), starting from
 * x (in/out).  Stops when ||dx|| / ||x|| < tol or after max_sweeps. */
int32_t or_central_icd(const or_problem *P, double *x, int32_t max_sweeps, double tol,
                       const int64_t *order, double *resid_out)
{
    int64_t n = (int64_t)P->nx * P->ny * P->nz;
    int64_t ne = (int64_t)P->nz * P->n_views * P->n_channels;
    double *e = (double *)malloc(sizeof(double) * (size_t)ne);
    if (!e) return OR_ENOMEM;
    or_error_sinogram(P, -1, x, e);
    double r = INFINITY;
    int32_t it = 0;
    while (it < max_sweeps) {
        double da2 = or_icd_sweep(P, -1, 0, 1.0, P->beta, order, NULL, x, e);
        ++it;
        double xx = 0.0;
        for (int64_t s = 0; s < n; ++s) xx += x[s] * x[s];
        r = xx > 0.0 ? sqrt(da2 / xx) : sqrt(da2);
        if (r < tol) break;
    }
    if (resid_out) *resid_out = r;
    free(e);
    return it;
}

/* ---------------------------------------------------------------------- */
/* Partial-update MACE, Algorithm 1.
 *   w (in/out, [N][n]): initial w^(0) on entry (the paper allows any value);
 *   X (in/out, [N][n]): if init_X != 0, X^(0) = G(w^(0)) is formed here;
 *   sweeps: ICD passes per agent per iteration (1 = Algorithm 2 as printed;
 *           a large value with inner_tol > 0 approximates exact MACE, i.e.
 *           F_i solved to convergence at every Mann step);
 *   order:  voxel visiting order (NULL = raster);
 *   xbar (out, [n]): consensus solution mean_i w_i;
 *   resid_hist (optional, [max_iter]): r_k = ||w^(k+1) - w^(k)|| / ||w^(k+1)||.
 * Returns the number of iterations run (or a negative error). */
int32_t or_mace(const or_problem *P, double sigma, double rho, int32_t sweeps,
                int32_t symmetric, double inner_tol, int32_t max_iter, double tol, const int64_t *order,
                int32_t init_X, double *w, double *X, double *xbar,
                double *resid_hist, double *resid_out, int32_t n_threads,
                const double *xref, double *nrmse_hist)
{
    int32_t N = P->n_agents;
    int64_t n = (int64_t)P->nx * P->ny * P->nz;
    if (N < 1 || n < 1 || sigma <= 0.0 || rho <= 0.0 || rho >= 1.0 + 1e-15) return OR_EINVAL;
    int32_t *nv = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    for (int32_t m = 0; m < P->n_views; ++m) {
        if (P->view_agent[m] < 0 || P->view_agent[m] >= N) { free(nv); return OR_EINVAL; }
        nv[P->view_agent[m]]++;
    }
    double **e = (double **)calloc((size_t)N, sizeof(double *));
    double *v = (double *)malloc(sizeof(double) * (size_t)(N * n));
    double *wbar = (double *)malloc(sizeof(double) * (size_t)n);
    for (int32_t g = 0; g < N; ++g)
        e[g] = (double *)malloc(sizeof(double) * (size_t)((int64_t)P->nz * nv[g] * P->n_channels) + 8);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    /* X^(0) = G(w^(0)) */
    if (init_X) {
        for (int64_t s = 0; s < n; ++s) {
            double acc = 0.0;
            for (int32_t g = 0; g < N; ++g) acc += w[g * n + s];
            wbar[s] = acc / (double)N;
        }
        for (int32_t g = 0; g < N; ++g) memcpy(X + g * n, wbar, sizeof(double) * (size_t)n);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t g = 0; g < N; ++g) or_error_sinogram(P, g, X + g * n, e[g]);

    double r = INFINITY;
    int32_t k = 0;
    double pscale = P->beta / (double)N;
    while (k < max_iter) {
        /* v = (2G - I) w */
        for (int64_t s = 0; s < n; ++s) {
            double acc = 0.0;
            for (int32_t g = 0; g < N; ++g) acc += w[g * n + s];
            wbar[s] = acc / (double)N;
        }
        for (int32_t g = 0; g < N; ++g)
            for (int64_t s = 0; s < n; ++s) v[g * n + s] = 2.0 * wbar[s] - w[g * n + s];
        /* X = F~(v; X): each agent independently (the parallel operator F) */
        #pragma omp parallel for schedule(dynamic, 1)
        for (int32_t g = 0; g < N; ++g) {
            for (int32_t sw = 0; sw < sweeps; ++sw) {
                double da2 = icd_sweep_dir(P, g, 1, sigma, pscale, order,
                                           symmetric && (sw & 1), v + g * n, X + g * n, e[g]);
                if (inner_tol > 0.0) {
                    double xx = 0.0;
                    for (int64_t s = 0; s < n; ++s) xx += X[g * n + s] * X[g * n + s];
                    if (da2 <= inner_tol * inner_tol * (xx > 0.0 ? xx : 1.0)) break;
                }
            }
        }
        /* w <- rho (2X - v) + (1 - rho) w, and the relative Mann residual */
        double dw2 = 0.0, ww2 = 0.0;
        for (int64_t t = 0; t < N * n; ++t) {
            double wn = rho * (2.0 * X[t] - v[t]) + (1.0 - rho) * w[t];
            double d = wn - w[t];
            dw2 += d * d;
            ww2 += wn * wn;
            w[t] = wn;
        }
        r = ww2 > 0.0 ? sqrt(dw2 / ww2) : sqrt(dw2);
        if (resid_hist) resid_hist[k] = r;
        if (xref && nrmse_hist) {
            /* NRMSE of the current consensus mean_i w_i against xref (Sec. IV-A) */
            double num = 0.0, den = 0.0;
            for (int64_t s = 0; s < n; ++s) {
                double acc = 0.0;
                for (int32_t g = 0; g < N; ++g) acc += w[g * n + s];
                double d = acc / (double)N - xref[s];
                num += d * d;
                den += xref[s] * xref[s];
            }
            nrmse_hist[k] = den > 0.0 ? sqrt(num / den) : sqrt(num);
        }
        ++k;
        if (r < tol) break;
    }
    /* x* = mean_i w_i */
    for (int64_t s = 0; s < n; ++s) {
        double acc = 0.0;
        for (int32_t g = 0; g < N; ++g) acc += w[g * n + s];
        xbar[s] = acc / (double)N;
    }
    if (resid_out) *resid_out = r;
    for (int32_t g = 0; g < N; ++g) free(e[g]);
    free(e); free(v); free(wbar); free(nv);
    return k;
}

/* ---------------------------------------------------------------------- */
/* Proximal map of the prior: x = argmin_z beta h(z) + ||z - v||^2 / (2 sigma^2),
 * by exact coordinate minimisation (Gauss-Seidel in raster order) repeated
 * until ||dx|| <= tol ||x||, from x = v.  For the quadratic prior each step is
 * the exact 1-D minimiser; for Q-GGMRF the surrogate step, which is zero
 * exactly where the coordinate derivative is (so the limit is the prox).
 * Returns the number of passes. */
int32_t or_prior_prox(const or_problem *P, double sigma, const double *v, double *x, int32_t max_pass,
                      double tol)
{
    int64_t plane = (int64_t)P->nx * P->ny, n = plane * P->nz;
    nbr_t nb[26];
    int nnb = make_nbrs(P->neighbourhood, nb);
    double inv_s2 = 1.0 / (sigma * sigma);
    memcpy(x, v, sizeof(double) * (size_t)n);
    int32_t pass = 0;
    while (pass < max_pass) {
        double da2 = 0.0, xx = 0.0;
        for (int64_t s = 0; s < n; ++s) {
            int32_t z = (int32_t)(s / plane);
            int32_t i = (int32_t)((s % plane) / P->nx);
            int32_t j = (int32_t)(s % P->nx);
            double gp = 0.0, hp = 0.0;
            for (int k = 0; k < nnb; ++k) {
                int32_t zz = z + nb[k].dz, ii = i + nb[k].di, jj = j + nb[k].dj;
                if (zz < 0 || zz >= P->nz || ii < 0 || ii >= P->ny || jj < 0 || jj >= P->nx)
                    continue;
                double d = x[s] - x[zz * plane + (int64_t)ii * P->nx + jj];
                double wgt = nb[k].b * prior_weight(P, d);
                gp += wgt * d;
                hp += wgt;
            }
            double num = P->beta * gp + (x[s] - v[s]) * inv_s2;
            double den = P->beta * hp + inv_s2;
            double alpha = -num / den;
            x[s] += alpha;
            da2 += alpha * alpha;
        }
        for (int64_t s = 0; s < n; ++s) xx += x[s] * x[s];
        ++pass;
        if (da2 <= tol * tol * (xx > 0.0 ? xx : 1.0)) break;
    }
    return pass;
}

/* Partial-update MACE with a plug-and-play prior, Algorithm 3:
 *   v = (2 G_H - I) w, G_H(w) = H(mean_i w_i) for every agent;
 *   X = F~(v; sqrt(N) sigma, X): `sweeps` ICD passes of each agent's data
 *       term only (beta = 0), symmetric as in or_mace;
 *   w <- rho (2X - v) + (1 - rho) w;
 *   solution x* = H(mean_i w_i).
 * H is or_prior_prox(sigma) solved to h_tol.  Arguments as in or_mace;
 * init_X != 0 forms X^(0) = G_H(w^(0)). */
int32_t or_pnp_mace(const or_problem *P, double sigma, double rho, int32_t sweeps, int32_t symmetric,
                    int32_t max_iter, double tol, const int64_t *order, int32_t init_X, double h_tol,
                    double *w, double *X, double *xstar, double *resid_hist, double *resid_out,
                    int32_t n_threads)
{
    int32_t N = P->n_agents;
    int64_t n = (int64_t)P->nx * P->ny * P->nz;
    if (N < 1 || n < 1 || sigma <= 0.0 || rho <= 0.0 || rho >= 1.0) return OR_EINVAL;
    int32_t *nv = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    for (int32_t m = 0; m < P->n_views; ++m) {
        if (P->view_agent[m] < 0 || P->view_agent[m] >= N) { free(nv); return OR_EINVAL; }
        nv[P->view_agent[m]]++;
    }
    double **e = (double **)calloc((size_t)N, sizeof(double *));
    double *v = (double *)malloc(sizeof(double) * (size_t)(N * n));
    double *wbar = (double *)malloc(sizeof(double) * (size_t)n);
    double *hx = (double *)malloc(sizeof(double) * (size_t)n);
    for (int32_t g = 0; g < N; ++g)
        e[g] = (double *)malloc(sizeof(double) * (size_t)((int64_t)P->nz * nv[g] * P->n_channels) + 8);
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#else
    (void)n_threads;
#endif
    const double sigma_f = sqrt((double)N) * sigma;
    /* G_H(w): mean over agents, then the denoiser */
    #define PNP_GH()                                                           \
        do {                                                                   \
            for (int64_t s = 0; s < n; ++s) {                                  \
                double acc = 0.0;                                              \
                for (int32_t g = 0; g < N; ++g) acc += w[g * n + s];           \
                wbar[s] = acc / (double)N;                                     \
            }                                                                  \
            or_prior_prox(P, sigma, wbar, hx, 100000, h_tol);                  \
        } while (0)
    if (init_X) {
        PNP_GH();
        for (int32_t g = 0; g < N; ++g) memcpy(X + g * n, hx, sizeof(double) * (size_t)n);
    }
    #pragma omp parallel for schedule(dynamic, 1)
    for (int32_t g = 0; g < N; ++g) or_error_sinogram(P, g, X + g * n, e[g]);

    double r = INFINITY;
    int32_t k = 0;
    while (k < max_iter) {
        PNP_GH();
        for (int32_t g = 0; g < N; ++g)
            for (int64_t s = 0; s < n; ++s) v[g * n + s] = 2.0 * hx[s] - w[g * n + s];
        #pragma omp parallel for schedule(dynamic, 1)
        for (int32_t g = 0; g < N; ++g)
            for (int32_t sw = 0; sw < sweeps; ++sw)
                icd_sweep_dir(P, g, 1, sigma_f, 0.0, order, symmetric && (sw & 1), v + g * n, X + g * n, e[g]);
        double dw2 = 0.0, ww2 = 0.0;
        for (int64_t t = 0; t < N * n; ++t) {
            double wn = rho * (2.0 * X[t] - v[t]) + (1.0 - rho) * w[t];
            double d = wn - w[t];
            dw2 += d * d;
            ww2 += wn * wn;
            w[t] = wn;
        }
        r = ww2 > 0.0 ? sqrt(dw2 / ww2) : sqrt(dw2);
        if (resid_hist) resid_hist[k] = r;
        ++k;
        if (r < tol) break;
    }
    PNP_GH();
    memcpy(xstar, hx, sizeof(double) * (size_t)n);
    #undef PNP_GH
    if (resid_out) *resid_out = r;
    for (int32_t g = 0; g < N; ++g) free(e[g]);
    free(e); free(v); free(wbar); free(hx); free(nv);
    return k;
}
