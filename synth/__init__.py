"""Seeded synthetic parallel-beam CT inputs.

This module generates INPUTS only: it holds none of the reconstruction
method's arithmetic (no system matrix, no ICD, no MACE).  Both the CUDA
library's tests and the FP64 oracle consume what it produces.

* Phantom: a sum of random ellipses (centres in a disc, random semi-axes,
  orientation and value), scaled so its maximum equals ``mu_max``.
* Sinogram: the exact analytic strip-averaged line integral of that ellipse
  phantom (closed form, not A x): for every view angle and channel, the chord
  length of each ellipse integrated over the channel's width.  The data are
  therefore not generated by the system matrix the reconstruction uses.
* Measurement model: counts k ~ Poisson(I0 exp(-p)), y = -log(max(k,1)/I0),
  weights Lambda = k (the inverse-variance weight of the post-log data).
* Random numbers: a counter-based SplitMix64 stream (Steele, Lea, Flood,
  "Fast splittable pseudorandom number generators", OOPSLA 2014), so the
  same seed gives the same inputs on any host; Poisson variates by the PTRS
  transformed-rejection method (Hormann, "The transformed rejection method
  for generating Poisson random variables", 1993) for large means and
  sequential inversion for small means.
"""
import math

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def _splitmix64(x):
    """SplitMix64 finaliser applied to uint64 counters (vectorised)."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


class CounterRNG:
    """uniform(stream, index) in [0, 1): a pure function of (seed, stream, index)."""

    def __init__(self, seed):
        self.seed = np.uint64(seed)

    def uniform(self, stream, index):
        idx = np.asarray(index, dtype=np.uint64)
        with np.errstate(over="ignore"):
            key = _splitmix64(self.seed * np.uint64(0x632BE59BD9B4E019)
                              + np.uint64(stream) * np.uint64(0xD1B54A32D192ED03))
            z = _splitmix64(key ^ (idx * np.uint64(0x9E3779B97F4A7C15)))
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def poisson(rng, lam, stream):
    """Poisson variates with means lam (any shape), one per element."""
    lam = np.asarray(lam, dtype=np.float64)
    flat = lam.ravel()
    out = np.zeros(flat.shape, np.int64)
    idx = np.arange(flat.size, dtype=np.uint64)
    small = flat < 10.0
    # sequential inversion for small means
    if small.any():
        li = flat[small]
        u = rng.uniform(stream, idx[small] * np.uint64(64))
        k = np.zeros(li.shape, np.int64)
        p = np.exp(-li)
        F = p.copy()
        for kk in range(1, 200):
            more = u > F
            if not more.any():
                break
            k[more] = kk
            p = p * li / kk
            F = F + p
        out[small] = k
    # PTRS for large means
    big = np.nonzero(~small)[0]
    lb = flat[big]
    slam = np.sqrt(lb)
    loglam = np.log(lb)
    b = 0.931 + 2.53 * slam
    a = -0.059 + 0.02483 * b
    invalpha = 1.1239 + 1.1328 / (b - 3.4)
    vr = 0.9277 - 3.6224 / (b - 2.0)
    pending = np.arange(big.size)
    attempt = 0
    lgam = np.vectorize(math.lgamma, otypes=[np.float64])
    while pending.size and attempt < 1000:
        ctr = idx[big[pending]] * np.uint64(64) + np.uint64(2 * attempt + 1)
        U = rng.uniform(stream, ctr) - 0.5
        V = rng.uniform(stream, ctr + np.uint64(1))
        us = 0.5 - np.abs(U)
        ap, bp, lp = a[pending], b[pending], lb[pending]
        k = np.floor((2.0 * ap / us + bp) * U + lp + 0.43)
        acc = (us >= 0.07) & (V <= vr[pending])
        rej = (k < 0) | ((us < 0.013) & (V > us))
        test = ~acc & ~rej
        if test.any():
            kt = k[test]
            lhs = (np.log(V[test]) + np.log(invalpha[pending][test])
                   - np.log(ap[test] / (us[test] * us[test]) + bp[test]))
            rhs = -lp[test] + kt * loglam[pending][test] - lgam(kt + 1.0)
            ok = np.zeros(test.shape, bool)
            ok[np.nonzero(test)[0][lhs <= rhs]] = True
            acc = acc | ok
        out[big[pending[acc]]] = k[acc].astype(np.int64)
        pending = pending[~acc]
        attempt += 1
    if pending.size:
        raise RuntimeError("Poisson sampler did not terminate")
    return out.reshape(lam.shape)


def ellipses(seed, n, mu_max, count=12):
    """Random ellipse parameters (x0, y0, a, b, phi, value), pixel units with the
    image centred at the origin; values scaled so the phantom max is mu_max."""
    rng = CounterRNG(seed)
    u = rng.uniform(1, np.arange(6 * count)).reshape(count, 6)
    r = 0.4 * n * np.sqrt(u[:, 0])
    ang = 2.0 * np.pi * u[:, 1]
    x0, y0 = r * np.cos(ang), r * np.sin(ang)
    a = n * (0.05 + 0.25 * u[:, 2])
    b = n * (0.05 + 0.25 * u[:, 3])
    phi = np.pi * u[:, 4]
    val = mu_max * (0.1 + 0.4 * u[:, 5])
    E = np.stack([x0, y0, a, b, phi, val], axis=1)
    peak = phantom_image(E, n, supersample=2).max()
    if peak > 0:
        E[:, 5] *= mu_max / peak
    return E


def phantom_image(E, n, supersample=1):
    """Point-sampled phantom on the n x n pixel grid (row 0 at the top)."""
    ss = int(supersample)
    off = (np.arange(ss) + 0.5) / ss - 0.5
    xs = (np.arange(n) - 0.5 * (n - 1))[None, :, None, None] + off[None, None, None, :]
    ys = (0.5 * (n - 1) - np.arange(n))[:, None, None, None] + off[None, None, :, None]
    img = np.zeros((n, n, ss, ss))
    for x0, y0, a, b, phi, val in E:
        c, s = math.cos(phi), math.sin(phi)
        dx, dy = xs - x0, ys - y0
        u = (dx * c + dy * s) / a
        v = (-dx * s + dy * c) / b
        img += val * ((u * u + v * v) <= 1.0)
    return img.mean(axis=(2, 3))


def sinogram(E, n_views, n_channels, channel_pitch=1.0, channel_offset=0.0,
             view_angles=None):
    """Channel-averaged line integrals of the ellipse phantom: [n_views, n_channels]."""
    if view_angles is None:
        view_angles = np.arange(n_views) * np.pi / n_views
    th = np.asarray(view_angles, np.float64)[:, None]
    tc = (np.arange(n_channels) - 0.5 * (n_channels - 1)) * channel_pitch + channel_offset
    lo, hi = (tc - 0.5 * channel_pitch)[None, :], (tc + 0.5 * channel_pitch)[None, :]
    ct, st = np.cos(th), np.sin(th)
    out = np.zeros((len(view_angles), n_channels))
    for x0, y0, a, b, phi, val in E:
        s2 = a * a * np.cos(th - phi) ** 2 + b * b * np.sin(th - phi) ** 2
        s = np.sqrt(s2)
        centre = x0 * ct + y0 * st

        def prim(tau):
            t = np.clip(tau, -s, s)
            return 0.5 * (t * np.sqrt(np.maximum(s2 - t * t, 0.0)) + s2 * np.arcsin(t / s))

        out += val * (2.0 * a * b / s2) * (prim(hi - centre) - prim(lo - centre)) / channel_pitch
    return out


def measurements(p, I0, rng, stream=7):
    """Poisson transmission counts -> (y, Lambda) as float32 arrays."""
    k = poisson(rng, I0 * np.exp(-p), stream)
    y = -np.log(np.maximum(k, 1).astype(np.float64) / I0)
    return y.astype(np.float32), k.astype(np.float32)


def interleaved_partition(n_views, n_agents):
    """J_i = {m : m mod N = i} with 0-based views and agents."""
    return (np.arange(n_views) % n_agents).astype(np.int32)


def uneven_partition(seed, n_views, n_agents, lo, hi):
    """Seeded per-agent view counts in [lo, hi] summing to n_views, assigned by
    smooth weighted round-robin so each agent's views span the half circle."""
    rng = CounterRNG(seed)
    u = rng.uniform(3, np.arange(n_agents))
    c = np.floor(lo + (hi - lo + 1) * u).astype(np.int64).clip(lo, hi)
    i = 0
    while c.sum() != n_views:
        j = i % n_agents
        if c.sum() < n_views and c[j] < hi:
            c[j] += 1
        elif c.sum() > n_views and c[j] > lo:
            c[j] -= 1
        i += 1
        if i > 100 * n_agents * (hi - lo + 1):
            raise ValueError("infeasible uneven partition")
    assigned = np.zeros(n_agents, np.int64)
    va = np.empty(n_views, np.int32)
    for m in range(n_views):
        deficit = c * (m + 1) / n_views - assigned
        g = int(np.argmax(deficit))
        va[m] = g
        assigned[g] += 1
    return va


def prior_sigma_x(lam, n_views, frac=0.1):
    """sigma_x such that beta/sigma_x^2 (beta = 1) is about `frac` of the
    typical data-Hessian diagonal, N_theta * E[sum A^2] * mean(Lambda), with
    E[sum A^2] taken as 1/2 for unit pixels on unit channels."""
    inv = frac * 0.5 * n_views * float(np.mean(lam))
    return 1.0 / math.sqrt(inv)


CONFIGS = {
    # 64^2, 90 views, 95 channels, 4 interleaved agents, quadratic prior
    "cfg1": dict(n=64, n_views=90, n_channels=95, I0=1e4, mu_max=0.02, n_agents=4,
                 prior="quadratic", seed=1, noise_seed=101, prior_frac=1.0),
    # 512^2, 720 views, 725 channels, 16 agents x 45 views, Q-GGMRF
    "cfg2": dict(n=512, n_views=720, n_channels=725, I0=2e4, mu_max=0.02 * 64 / 512,
                 n_agents=16, prior="qggmrf", seed=2, noise_seed=102, prior_frac=1.0),
    # the benchmark batch's second scan (phantom and noise seeds + 7); the
    # batch shares one prior scale, set from the first scan's weights
    "cfg2_scan1": dict(n=512, n_views=720, n_channels=725, I0=2e4, mu_max=0.02 * 64 / 512,
                       n_agents=16, prior="qggmrf", seed=9, noise_seed=109, prior_frac=1.0,
                       prior_scale_from="cfg2"),
}


def ellipsoids(seed, n, nz, mu_max, count=12):
    """Random ellipsoids (x0, y0, z0, a, b, c, phi, value) in pixel units, the
    volume centred at the origin (slices at z = k - (nz-1)/2), axis c along z;
    values scaled so the volume's maximum is mu_max."""
    rng = CounterRNG(seed)
    u = rng.uniform(2, np.arange(8 * count)).reshape(count, 8)
    r = 0.4 * n * np.sqrt(u[:, 0])
    ang = 2.0 * np.pi * u[:, 1]
    x0, y0 = r * np.cos(ang), r * np.sin(ang)
    z0 = (u[:, 2] - 0.5) * 0.8 * nz
    a = n * (0.05 + 0.25 * u[:, 3])
    b = n * (0.05 + 0.25 * u[:, 4])
    c = nz * (0.2 + 0.5 * u[:, 5])
    phi = np.pi * u[:, 6]
    val = mu_max * (0.1 + 0.4 * u[:, 7])
    Q = np.stack([x0, y0, z0, a, b, c, phi, val], axis=1)
    peak = max(phantom_image(slice_ellipses(Q, z, nz), n, supersample=2).max() for z in range(nz))
    if peak > 0:
        Q[:, 7] *= mu_max / peak
    return Q


def slice_ellipses(Q, z, nz):
    """Cross-section of the ellipsoids with slice z: ellipses (x0, y0, a, b, phi, value)."""
    zc = z - 0.5 * (nz - 1)
    out = []
    for x0, y0, z0, a, b, c, phi, val in Q:
        t = (zc - z0) / c
        if abs(t) < 1.0:
            f = math.sqrt(1.0 - t * t)
            out.append([x0, y0, a * f, b * f, phi, val])
    return np.array(out).reshape(-1, 6)


def make_volume(n, nz, n_views, n_channels, I0, mu_max, seed, noise_seed, **_):
    """Ellipsoid phantom -> per-slice analytic sinograms -> Poisson data:
    y, lam [nz, n_views, n_channels] float32 (parallel beam, one 2D geometry
    for every slice)."""
    Q = ellipsoids(seed, n, nz, mu_max)
    ys, ls = [], []
    for z in range(nz):
        E = slice_ellipses(Q, z, nz)
        p = sinogram(E, n_views, n_channels) if len(E) else np.zeros((n_views, n_channels))
        y, lam = measurements(p, I0, CounterRNG(noise_seed * 1000 + z))
        ys.append(y)
        ls.append(lam)
    return dict(y=np.stack(ys), lam=np.stack(ls), ellipsoids=Q)


def make_case(n, n_views, n_channels, I0, mu_max, seed, noise_seed, nz=1, **_):
    """Phantom -> analytic sinogram -> Poisson data for nz identical-geometry
    slices (each slice its own phantom seed offset).  Returns dict with y, lam
    ([nz, n_views, n_channels] float32) and the phantom parameters."""
    ys, ls, Es = [], [], []
    for z in range(nz):
        E = ellipses(seed * 1000 + z, n, mu_max)
        p = sinogram(E, n_views, n_channels)
        y, lam = measurements(p, I0, CounterRNG(noise_seed * 1000 + z))
        ys.append(y)
        ls.append(lam)
        Es.append(E)
    return dict(y=np.stack(ys), lam=np.stack(ls), ellipses=Es)
