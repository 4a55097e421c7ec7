"""Seeded synthetic common-receiver gathers (inputs only; no operator arithmetic).

This module serves both the CUDA path and the FP64 oracle with identical,
seeded inputs.  It draws hyperbolic events, renders them with an analytic
Ricker wavelet at the exact fractional traveltime (no inverse crime), and
forms a pseudo-deblended gather: the wanted source plus interfering sources
whose traces carry random firing delays (source dithering, ch. 2 blending
b = Gamma D and pseudo-deblending D~ = Gamma^T b), so that the interference is
incoherent in the receiver gather (ch. 2, ch. 4 "Synthetic data example").

Config recipes (seed = 1000 * config + gather):
  c1  1 gather, nt 256 @ 4 ms, nx 64 @ 12.5 m; 4 reflections tau ~ U[0.2,0.8] s,
      apex ~ U[line], v ~ U[1500,3000], A ~ N(1,0.3), 20 Hz Ricker; one
      interfering source (an independent 4-event gather) with per-trace delays
      ~ U[0,0.5] s, scaled to 3x the signal peak.  Scan: 8 velocities.
  c2  64 gathers, nt 1024, nx 256; 10-30 events, tau ~ U[0.2,3.5] s,
      v ~ U[1400,3500], 25 Hz; 2 interfering sources, delays ~ U[0,1] s,
      peak ratio per source ~ U[1,10].  Scan: 32 velocities.
  c3  16 gathers, nt 1024, nx 256; 40 diffractions t = tau0 + sqrt(tau^2+h^2)
      with tau0 ~ U[0,0.4] s, tau ~ U[0.2,3.0] s, plus 5 reflections; 50% of
      traces removed.  Scan: 24 velocities x 16 asymptote shifts.
  c4  uneven gathers, nx ~ U{96..480}, nt 1500; 5-40 events; 3 interfering
      sources with delays ~ U[0,1.5] s.  Scan: 24 velocities.
  c5  warm-start training and evaluation gathers, nt 1024, nx 256: the c3
      signal (5 reflections + 40 diffractions, tau0 ~ U[0,0.4] s) blended as
      in c2 (2 interfering sources of 5 events, delays ~ U[0,1] s, peak
      ratio ~ U[1,10]).  Scan: 24 velocities, tau0 = {0}.  Smaller nt / nx
      keep the recipe with the time ranges clipped to the record.
"""
import numpy as np

DT = 0.004
DX = 12.5


def rng_for(config, gather):
    return np.random.Generator(np.random.PCG64(1000 * int(config) + int(gather)))


def ricker(t, f_peak):
    a = (np.pi * f_peak * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def draw_events(rng, n, nx, dx, tau_range, v_range, t0_range=None, amp=(1.0, 0.3)):
    ev = dict(
        tau=rng.uniform(*tau_range, size=n),
        xa=rng.uniform(0.0, (nx - 1) * dx, size=n),
        v=rng.uniform(*v_range, size=n),
        A=rng.normal(amp[0], amp[1], size=n),
        t0=np.zeros(n) if t0_range is None else rng.uniform(*t0_range, size=n),
    )
    return ev


def render(ev, nt, nx, dt, dx, f_peak):
    """Sum of A * ricker(t - (t0 + sqrt(tau^2 + ((x - xa)/v)^2))) over events.

    Each wavelet is evaluated within +-2/f_peak of its arrival, where the
    Ricker envelope exp(-(pi f t)^2) has decayed below 1e-17."""
    x = np.arange(nx) * dx
    d = np.zeros((nx, nt))
    half = int(np.ceil(2.0 / (f_peak * dt))) + 1
    win = np.arange(-half, half + 1)
    rows = np.arange(nx)[:, None]
    for tau, xa, v, A, t0 in zip(ev["tau"], ev["xa"], ev["v"], ev["A"], ev["t0"]):
        tx = t0 + np.sqrt(tau * tau + ((x - xa) / v) ** 2)
        idx = np.rint(tx / dt).astype(np.int64)[:, None] + win[None, :]
        ok = (idx >= 0) & (idx < nt)
        vals = A * ricker(idx * dt - tx[:, None], f_peak)
        np.add.at(d, (np.broadcast_to(rows, idx.shape)[ok], idx[ok]), vals[ok])
    return d


def dither(rng, g, max_delay, dt):
    """Delay every trace of an interfering gather by its own random firing
    time (sample-rounded, zero-filled): the pseudo-deblended view of a
    dithered source in a receiver gather."""
    nx, nt = g.shape
    out = np.zeros_like(g)
    lag = np.rint(rng.uniform(0.0, max_delay, size=nx) / dt).astype(int)
    for j in range(nx):
        s = lag[j]
        if s < nt:
            out[j, s:] = g[j, :nt - s]
    return out


def velocity_scan(vmin, vmax, nv):
    return np.linspace(vmin, vmax, nv).astype(np.float32)


def _gather(rng, nt, nx, n_ev, tau_range, v_range, f_peak, n_src, max_delay,
            ratio, diffr=0, t0_range=None, dt=DT, dx=DX):
    ev = draw_events(rng, n_ev, nx, dx, tau_range, v_range)
    clean = render(ev, nt, nx, dt, dx, f_peak)
    if diffr:
        evd = draw_events(rng, diffr, nx, dx, tau_range, v_range, t0_range=t0_range)
        clean = clean + render(evd, nt, nx, dt, dx, f_peak)
    peak = np.max(np.abs(clean))
    blended = clean.copy()
    for _ in range(n_src):
        evi = draw_events(rng, n_ev, nx, dx, tau_range, v_range)
        gi = dither(rng, render(evi, nt, nx, dt, dx, f_peak), max_delay, dt)
        r = ratio if np.isscalar(ratio) else rng.uniform(*ratio)
        pk = np.max(np.abs(gi))
        if pk > 0:
            blended += gi * (r * peak / pk)
    return clean, blended


def config1(gather=0):
    """c1: (clean, blended, velocities) for one 256 x 64 gather."""
    rng = rng_for(1, gather)
    nt, nx = 256, 64
    clean, blended = _gather(rng, nt, nx, 4, (0.2, 0.8), (1500.0, 3000.0), 20.0,
                             1, 0.5, 3.0)
    return dict(nt=nt, nx=nx, dt=DT, dx=DX, clean=clean, blended=blended,
                velocities=velocity_scan(1500.0, 3000.0, 8), t0s=np.zeros(1, np.float32),
                f_peak=20.0)


def config2(n_gathers=64, nt=1024, nx=256, nv=32):
    """c2: batch of pseudo-deblended gathers [B][nx][nt] and their clean versions."""
    clean = np.zeros((n_gathers, nx, nt))
    blended = np.zeros((n_gathers, nx, nt))
    for g in range(n_gathers):
        rng = rng_for(2, g)
        n_ev = int(rng.integers(10, 31))
        c, b = _gather(rng, nt, nx, n_ev, (0.2, min(3.5, 0.85 * nt * DT)),
                       (1400.0, 3500.0), 25.0, 2, 1.0, (1.0, 10.0))
        clean[g], blended[g] = c, b
    return dict(nt=nt, nx=nx, dt=DT, dx=DX, clean=clean, blended=blended,
                velocities=velocity_scan(1400.0, 3500.0, nv), t0s=np.zeros(1, np.float32),
                f_peak=25.0)


def config3(n_gathers=16, nt=1024, nx=256, nv=24, nt0=16, keep=0.5):
    """c3: diffraction gathers with half of the traces removed (mask [B][nx])."""
    clean = np.zeros((n_gathers, nx, nt))
    mask = np.zeros((n_gathers, nx), dtype=np.float32)
    for g in range(n_gathers):
        rng = rng_for(3, g)
        c, _ = _gather(rng, nt, nx, 5, (0.2, min(3.0, 0.75 * nt * DT)), (1400.0, 3500.0),
                       25.0, 0, 0.0, 0.0, diffr=40, t0_range=(0.0, 0.4))
        clean[g] = c
        keep_idx = rng.permutation(nx)[: int(round(keep * nx))]
        mask[g, keep_idx] = 1.0
    observed = clean * mask[:, :, None]
    return dict(nt=nt, nx=nx, dt=DT, dx=DX, clean=clean, observed=observed, mask=mask,
                velocities=velocity_scan(1400.0, 3500.0, nv),
                t0s=np.linspace(0.0, 0.4, nt0).astype(np.float32), f_peak=25.0)


def config5_gather(g, nt=1024, nx=256):
    """c5 gather g: (clean, pseudo-deblended), both [nx][nt]."""
    rng = rng_for(5, g)
    return _gather(rng, nt, nx, 5, (0.2, min(3.0, 0.75 * nt * DT)), (1400.0, 3500.0), 25.0,
                   2, min(1.0, 0.25 * nt * DT), (1.0, 10.0), diffr=40, t0_range=(0.0, 0.4))


def _c5_job(args):
    g, nt, nx = args
    c, b = config5_gather(g, nt, nx)
    return c.astype(np.float32), b.astype(np.float32)


def _c1_job(args):
    c = config1(args[0])
    return c["clean"], c["blended"]


def config5(gathers, nt=1024, nx=256, processes=0):
    """c5 gathers for the seeds in `gathers`: dict with clean / blended
    [len][nx][nt] (float32), velocities and t0s.  processes > 1 renders them
    in a pool of that many 'spawn' workers."""
    gathers = list(gathers)
    clean = np.zeros((len(gathers), nx, nt), np.float32)
    blended = np.zeros_like(clean)
    jobs = [(g, nt, nx) for g in gathers]
    if processes and processes > 1 and len(gathers) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map(_c5_job, jobs, chunksize=max(1, len(jobs) // (4 * processes)))
    else:
        res = [_c5_job(j) for j in jobs]
    for i, (c, b) in enumerate(res):
        clean[i], blended[i] = c, b
    return dict(nt=nt, nx=nx, dt=DT, dx=DX, clean=clean, blended=blended,
                velocities=velocity_scan(1400.0, 3500.0, 24), t0s=np.zeros(1, np.float32),
                f_peak=25.0)


def config4_sizes(n_gathers=2000):
    """c4: per-gather trace counts nx ~ U{96..480}."""
    rng = rng_for(4, 0)
    return rng.integers(96, 481, size=n_gathers)


def config4_gather(g, nx, nt=1500):
    rng = rng_for(4, g + 1)
    n_ev = int(rng.integers(5, 41))
    return _gather(rng, nt, int(nx), n_ev, (0.2, 0.85 * nt * DT), (1400.0, 3500.0), 25.0,
                   3, 1.5, (1.0, 10.0))


def _c4_job(args):
    g, nx, nt = args
    c, b = config4_gather(g, nx, nt)
    return c.astype(np.float32), b.astype(np.float32)


def config4(gathers, nxs, nt=1500, processes=0):
    """c4 gathers for the seeds in `gathers` with trace counts `nxs`: dict with
    packed clean / blended float32 arrays (gather g is [nx_g][nt] at offset
    nt * sum_{h<g} nx_h), velocities (24) and f_peak.  processes > 1 renders
    them in a pool of that many 'spawn' workers."""
    gathers, nxs = list(gathers), [int(n) for n in nxs]
    jobs = [(g, nx, nt) for g, nx in zip(gathers, nxs)]
    if processes and processes > 1 and len(jobs) > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map(_c4_job, jobs, chunksize=max(1, len(jobs) // (4 * processes)))
    else:
        res = [_c4_job(j) for j in jobs]
    return dict(nt=nt, nxs=nxs, dt=DT, dx=DX,
                clean=np.concatenate([c.ravel() for c, _ in res]),
                blended=np.concatenate([b.ravel() for _, b in res]),
                velocities=velocity_scan(1400.0, 3500.0, 24), t0s=np.zeros(1, np.float32),
                f_peak=25.0)


def random_model(rng, shape, sparsity=None):
    """Random test vector (optionally sparse) for operator parity checks."""
    x = rng.standard_normal(shape)
    if sparsity is not None:
        x *= rng.random(shape) < sparsity
    return x
