"""Benchmark of the Stolt-ASHRT robust deblending hot path on GB300.

Workload (one step): robust IRLS deblending (p = q = 1, 8 outer x 30 CGLS
iterations, Ricker wavelet C at 25 Hz) of a batch of 64 synthetic
pseudo-deblended common-receiver gathers, nt = 1024 @ 4 ms, nx = 256 @ 12.5 m,
Radon scan of 32 velocities x 256 apexes.  Every operator application is a
Stolt-ASHRT forward or adjoint over the whole batch.

value = gather-level forward+adjoint operator pairs per second over all ranks
(pairs = batch x (forward applies + adjoint applies) / 2 per step), measured
with inputs resident in HBM; `gathers_per_s` is deblended gathers per second;
`e2e` is the same metric through the public API with host buffers (pinned
host -> device copy of the gathers, device -> host copy of the recovered
gathers, every step).  `--impl reference` times the FP64 CPU oracle (the
reference arm of this method) on a bounded sample of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NT, NX, NV, B = 1024, 256, 32, 64
DT, DX = 0.004, 12.5
N_OUTER, N_CG = 8, 30
F_PEAK = 25.0
METRIC = "Stolt-ASHRT fwd+adj pairs/s (robust IRLS deblend, 64 gathers 1024x256, 32 velocities)"
UNIT = "gather fwd+adj pairs/s"


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--mode", default="deblend", choices=["deblend", "ops", "unet", "td", "fista",
                                                         "cube", "c1", "c3", "c4", "irregular"],
                    help="ops: forward+adjoint operator pairs only; unet: warm-start U-Net "
                         "inference; td: time-domain (hyperbolic summation) pair against the "
                         "Stolt pair on the same gathers; fista: l2-l1 interpolation by FISTA "
                         "on the gathers with 4 of 5 traces removed; cube: blending, "
                         "pseudo-deblending, sorting and the deblend of a 256-shot x 64-receiver "
                         "cube; c1: the one-gather robust solve (5 x 20) on the GPU, by the "
                         "FP64 oracle and by the scipy.fft operator on the host cores; c3: the "
                         "AASHRT pair with 24 velocities x 16 asymptote "
                         "shifts on 16 gathers with half the traces removed, and their FISTA "
                         "interpolation; c4: 2000 gathers of uneven width (nx 96..480, nt "
                         "1500) deblended through the batch layer, recorded graphs against "
                         "direct launches; irregular: the operator pair and the deblend "
                         "of the workload's gathers recorded at jittered trace positions "
                         "against the same on the regular grid (profiling aids and workload "
                         "runs, not the bench "
                         "line)")
    ap.add_argument("--gathers", type=int, default=2000, help="c4: number of gathers")
    ap.add_argument("--irls", type=int, nargs=2, default=[3, 10],
                    help="c4: IRLS outer and CG iterations")
    ap.add_argument("--batch", type=int, default=B,
                    help="gathers per call (the deblend workload is 64; smaller batches are "
                         "for profiling captures)")
    ap.add_argument("--variant", type=int, default=0,
                    help="deblend mode: row-kernel variant 1..9 instead of the autotuner's "
                         "choice (profiling captures skip the autotuner's launches this way)")
    ap.add_argument("--rows-variant", type=int, default=0,
                    help="ops mode: row-kernel variant 1..9 (0: the plan's default; see "
                         "ashrt_plan_set_variant)")
    return ap.parse_args()


def _config(extra=None, batch=B):
    c = {"workload": "robust IRLS deblend, %d gathers x (nt 1024 @ 4 ms, nx 256 @ 12.5 m), "
                     "32 velocities x 256 apexes, IRLS 8 x 30, p = q = 1, 25 Hz wavelet" % batch,
         "gathers_per_step": batch, "nt": NT, "nx": NX, "nv": NV, "irls": [N_OUTER, N_CG],
         "padded": [2048, 512], "l2": "inputs larger than L2 (model 2.1 GB per vector)",
         "parallelism": "replicas (gathers are independent; no collective)"}
    if extra:
        c.update(extra)
    return c


# ---------------------------------------------------------------------------
# algorithmic work per gather: FFT flops 5 N log2 N per complex length-N transform
# (half for real input), 16 flops per mapped bin for the 2-tap complex map
def _fft_flops(n):
    return 5.0 * n * (n.bit_length() - 1)


def algorithmic(nt=NT, nx=NX, P=NV, Nt=2048, Nx=512):
    lh = Nx // 2 + 1
    rows = (P + 1) * lh * _fft_flops(Nt) + 16.0 * P * Nt * lh          # one row kernel launch, per gather
    xcols = (P + 1) * nt * 0.5 * _fft_flops(Nx)                         # both trace-axis kernels, per gather
    pair_flops = 2.0 * (rows + xcols)
    pair_bytes = 2.0 * 4.0 * nt * nx * (P + 1)
    return dict(rows_flops=rows, pair_flops=pair_flops, pair_bytes=pair_bytes,
                rows_bytes=4.0 * 2 * lh * nt * (P + 1))


def xfft_model_bytes(kernel, B, nt=NT, nx=NX, P=NV, Nx=512, n_outer=None, n_cg=None):
    """Algorithmic HBM bytes of the model-side trace-axis launches of one
    deblend step (mu = 0, fused CG path), averaged per launch: the FP32 model-
    sized streams each launch must move once and the half spectrum X it writes
    or reads.  Per outer iteration the r2c runs n_cg CG forwards and one
    plain reconstruction forward (reads m, writes X).  CG forward it reads
    p~_{it-1} and s~ and writes p~_it and X; the model takes its updates two
    at a time on odd iterations, which also read and write m and, from it = 3
    on, read p~_{it-2}.  The c2r runs n_cg weighted adjoints (reads X and
    W_m^-1, writes s~)."""
    n_outer = N_OUTER if n_outer is None else n_outer
    n_cg = N_CG if n_cg is None else n_cg
    S = 4.0 * nx * nt * P                       # one model-sized FP32 stream, per gather
    X = 8.0 * (Nx // 2 + 1) * nt * P            # the half spectrum, per gather
    if kernel == "xfft_r2c":
        per_outer = S + X
        for it in range(n_cg):
            streams = 3                                  # p~_{it-1}, s~ in; p~_it out
            if it & 1:
                streams += 2 + (1 if it >= 3 else 0)     # m in and out; p~_{it-2} in
            per_outer += streams * S + X
        launches = n_cg + 1
    else:
        per_outer = n_cg * (X + 2 * S)
        launches = n_cg
    return B * per_outer / launches


def _peaks():
    p = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
    except OSError:
        pass
    hbm = p.get("hbm_gbs")
    return dict(hbm_gbs=hbm if hbm else 6800.0, hbm_src="measured" if hbm else "fallback",
                sm_max_mhz=p.get("sm_max_mhz", 2070.0))


# Source files of each timed kernel class: the committed DRAM-traffic figures
# (profiles/dram_traffic.md) hold for the sources they were captured from.
KERNEL_SOURCES = {
    "stolt_adj_rows": ["stolt_adj.cu", "stolt_r16.cu", "stolt_r16s.cu", "stolt_r16.cuh",
                       "stolt_common.cuh", "common.cuh"],
    "stolt_fwd_rows": ["stolt_r16.cu", "stolt_fwd.cu", "stolt_r16s.cu", "stolt_r16.cuh",
                       "stolt_common.cuh", "common.cuh"],
    "xfft_r2c": ["xfft.cu", "tma.cu", "tma.cuh", "common.cuh"],
    "xfft_c2r": ["xfft.cu", "common.cuh"],
}
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.md")


def source_hash(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1711_10214_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def measured_traffic(kernel, gathers, variant=(9, 16)):
    """DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch
    of `kernel` over `gathers` gathers, scaled from the committed ncu capture
    in profiles/dram_traffic.md (rows: | kernel | gathers per launch | bytes
    per launch | source hash | variant | ...), the variant being the plan's
    rows_minb/xfft_cols.  None when there is no capture of the kernel's
    current sources in the variant that ran."""
    try:
        with open(TRAFFIC_FILE) as f:
            rows = [ln.split("|")[1:-1] for ln in f if ln.startswith("| ")]
    except OSError:
        return None, None
    want = source_hash(kernel)
    for r in rows:
        r = [x.strip() for x in r]
        if len(r) >= 5 and r[0] == kernel and r[3] == want and r[4] == "%d/%d" % tuple(variant):
            try:
                return float(r[2]) / float(r[1]) * gathers, want
            except ValueError:
                continue
    return None, want


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def whole_job_rate(t_local, units_per_rank, world, dist=None, device=None):
    """Slowest rank's time and the whole job's rate: every rank processed
    units_per_rank units in its own t_local seconds; the job took the max over
    ranks (one all-reduce when distributed)."""
    t = float(t_local)
    if dist is not None and world > 1:
        import torch
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return t, world * units_per_rank / t


def cpu_baseline_sample():
    """The FP64 oracle (numpy, naive DFTs) on one gather of the workload: one
    forward + one adjoint with all 32 velocities, timed on the host cores."""
    import numpy as np

    from oracle import stolt
    from paper_1711_10214_gb300 import synth
    v = synth.velocity_scan(1400.0, 3500.0, NV)
    g = stolt.Geometry(NT, NX, DT, DX, v, wavelet_peak_hz=F_PEAK)
    rng = np.random.default_rng(0)
    m = rng.standard_normal(g.model_shape)
    d = rng.standard_normal(g.data_shape)
    t0 = time.perf_counter()
    stolt.forward(g, m)
    stolt.adjoint(g, d)
    dt = time.perf_counter() - t0
    cores = os.cpu_count()
    return dict(value=1.0 / dt, unit=UNIT, cores=cores, kind="oracle",
                sample="1 gather, 1 forward + 1 adjoint (32 velocities, nt 1024, nx 256), "
                       "FP64 numpy naive-DFT oracle; %.1f s" % dt)


class ScipyStolt:
    """The Stolt ASHRT pair as a CPU program on scipy.fft: the fair CPU
    baseline of the measurement (the same operator as the GPU path and the
    oracle, with fast transforms instead of the oracle's naive DFTs, all host
    cores as scipy.fft workers, FP64 or FP32).  Layouts and readings as the
    library's: real x-transform to the half spectrum (pad nx -> Nx), complex
    t-transform (pad nt -> Nt), 2-tap linear interpolation in the w index at
    u = sgn(k) sqrt(k^2 - a^2) inside the cone k^2 > a^2 (taps on the w-Nyquist
    bin weigh 0), exp(-i w tau0) asymptote phase, Ricker amplitude spectrum
    W(f) = (f/fp)^2 exp(1 - (f/fp)^2), the adjoint as the exact transpose."""

    def __init__(self, nt, nx, dt, dx, velocities, t0s=(0.0,), wavelet_peak_hz=0.0,
                 dtype="float64", workers=None):
        import numpy as np
        self.np = np
        self.nt, self.nx, self.dt, self.dx = nt, nx, dt, dx
        self.Nt = 1 << max(6, (2 * nt - 1).bit_length())
        self.Nx = 1 << max(4, (2 * nx - 1).bit_length())
        self.Lh = self.Nx // 2 + 1
        self.rdt = np.dtype(dtype)
        self.cdt = np.result_type(self.rdt, np.complex64)
        self.workers = workers or os.cpu_count()
        v = np.asarray(velocities, np.float32).astype(np.float64)
        t0 = np.asarray(t0s, np.float32).astype(np.float64)
        Nt, Nx, H = self.Nt, self.Nx, self.Nt // 2
        k = np.arange(Nt)
        ks = np.where(k <= H, k, k - Nt).astype(np.float64)
        f = np.abs(ks) / (Nt * dt)
        W = np.ones(Nt)
        if wavelet_peak_hz > 0:
            z = (f / wavelet_peak_hz) ** 2
            W = z * np.exp(1.0 - z)
        W[H] = 0.0
        self.W = W
        self.phase = [np.exp(-2j * np.pi * ks * tj / (Nt * dt)).astype(self.cdt) for tj in t0]
        # per velocity: flat source / target indices and weights of the map on [Lh, Nt]
        self.taps = []
        rows = np.arange(self.Lh)[:, None]
        for vi in v:
            a = ((vi * np.arange(self.Lh, dtype=np.float64)) * float(Nt)) * dt / (float(Nx) * dx)
            a2 = (a * a)[:, None]
            cone = (ks[None, :] ** 2 > a2) & (k[None, :] != H)
            u = np.where(cone, np.sign(ks)[None, :] * np.sqrt(np.maximum(ks[None, :] ** 2 - a2, 0)),
                         0.0)
            k0 = np.floor(u)
            fr = u - k0
            i0 = np.mod(k0.astype(np.int64), Nt)
            i1 = np.mod(k0.astype(np.int64) + 1, Nt)
            w0 = np.where(cone & (i0 != H), 1.0 - fr, 0.0)
            w1 = np.where(cone & (i1 != H), fr, 0.0)
            src0 = (rows * Nt + i0).ravel()
            src1 = (rows * Nt + i1).ravel()
            self.taps.append((src0, src1, w0.ravel().astype(self.rdt), w1.ravel().astype(self.rdt)))

    def _spec(self, x):
        import scipy.fft as sf
        Xh = sf.rfft(x, n=self.Nx, axis=-2, workers=self.workers)
        return sf.fft(Xh, n=self.Nt, axis=-1, workers=self.workers)

    def forward(self, m):
        """m [nt0][nv][nx][nt] -> d [nx][nt]."""
        import scipy.fft as sf
        np = self.np
        nt0, nv = m.shape[:2]
        M = self._spec(m.astype(self.rdt, copy=False)).reshape(nt0, nv, -1)
        D = np.zeros(self.Lh * self.Nt, self.cdt)
        for j in range(nt0):
            Dj = np.zeros_like(D)
            for i in range(nv):
                s0, s1, w0, w1 = self.taps[i]
                Dj += w0 * M[j, i][s0] + w1 * M[j, i][s1]
            D += Dj * np.tile(self.phase[j], self.Lh)
        D = D.reshape(self.Lh, self.Nt) * self.W[None, :].astype(self.rdt)
        y = sf.ifft(D, axis=-1, workers=self.workers)[:, :self.nt]
        return sf.irfft(y, n=self.Nx, axis=0, workers=self.workers)[:self.nx]

    def adjoint(self, d, nt0, nv):
        """d [nx][nt] -> m [nt0][nv][nx][nt], the exact transpose of forward."""
        import scipy.fft as sf
        np = self.np
        Dh = (self._spec(d.astype(self.rdt, copy=False)) * self.W[None, :].astype(self.rdt)).ravel()
        n = self.Lh * self.Nt
        out = np.empty((nt0, nv, self.nx, self.nt), self.rdt)
        for j in range(nt0):
            Dj = Dh * np.tile(np.conj(self.phase[j]), self.Lh)
            for i in range(nv):
                s0, s1, w0, w1 = self.taps[i]
                re = np.bincount(s0, w0 * Dj.real, n) + np.bincount(s1, w1 * Dj.real, n)
                im = np.bincount(s0, w0 * Dj.imag, n) + np.bincount(s1, w1 * Dj.imag, n)
                Mi = (re + 1j * im).astype(self.cdt).reshape(self.Lh, self.Nt)
                # the 1/(Nt Nx) of the pair sits in the inverse transforms here;
                # the half spectrum is Hermitian in k_x, so the real inverse
                # transform gives the synthesis over both signs of k_x
                y = sf.ifft(Mi, axis=-1, workers=self.workers)[:, :self.nt]
                out[j, i] = sf.irfft(y, n=self.Nx, axis=0, workers=self.workers)[:self.nx]
        return out


def cpu_fft_baseline(nt=NT, nx=NX, nv=NV, reps=2):
    """The scipy.fft Stolt pair (ScipyStolt) on one gather of the workload,
    FP64 and FP32, best of `reps` forward + adjoint pairs, all host cores."""
    import numpy as np

    from paper_1711_10214_gb300 import synth
    v = synth.velocity_scan(1400.0, 3500.0, nv)
    rng = np.random.default_rng(0)
    m = rng.standard_normal((1, nv, nx, nt))
    d = rng.standard_normal((nx, nt))
    out = {}
    for dt_ in ("float64", "float32"):
        op = ScipyStolt(nt, nx, DT, DX, v, wavelet_peak_hz=F_PEAK, dtype=dt_)
        best = 1e30
        for _ in range(reps):
            t0 = time.perf_counter()
            op.forward(m)
            op.adjoint(d, 1, nv)
            best = min(best, time.perf_counter() - t0)
        out[dt_] = {"pairs_per_s": 1.0 / best, "s_per_pair": best}
    return {"kind": "scipy.fft Stolt pair (same operator, fast transforms)",
            "cores": os.cpu_count(), "workload": "1 gather, nt %d, nx %d, %d velocities" % (nt, nx, nv),
            "f64": out["float64"], "f32": out["float32"]}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    for i in range(args.warmup + args.steps):
        r = cpu_baseline_sample()
        if i >= args.warmup:
            vals.append(r["value"])
    value = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": _config({"reference_step": "1 gather fwd+adj pair (bounded sample)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["cores"], "kind": "oracle",
                             "sample": r["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    dev = torch.device("cuda", local)
    B = args.batch
    c = synth.config2(B, NT, NX, NV)
    d_host = torch.from_numpy(c["blended"].astype(np.float32)).pin_memory()
    drec_host = torch.empty_like(d_host).pin_memory()
    d = d_host.to(dev)
    plan = ashrt.Plan(NT, NX, DT, DX, c["velocities"], wavelet_peak_hz=F_PEAK, max_batch=B,
                      with_solver=True)
    m = torch.empty((B,) + plan.model_shape, device=dev)
    drec = torch.empty_like(d)
    stream = torch.cuda.current_stream(dev)
    # direct launches (not the recorded graph): the roofline needs each kernel
    # bracketed by CUDA events inside the timed region
    kw = dict(p=1.0, q=1.0, n_outer=N_OUTER, n_cg=N_CG)
    if args.variant:
        plan.set_variant(args.variant, 16)
        variant = (args.variant, 16)
    else:
        variant = plan.autotune(batch=B, cache_path=os.environ.get(
            "ASHRT_TUNE_CACHE", "/tmp/ashrt_autotune.jsonl"))
    # FP32 FMA peak of this device, measured with its own clock record
    pclk = ClockSampler(local)
    pclk.start()
    fp32_peak, n_sm = ashrt.fp32_peak(iters=100000, reps=5, stream=stream)
    peak_clk = pclk.stop()

    for _ in range(args.warmup):
        reps = plan.deblend(d, m, drec, batch=B, stream=stream, **kw)
    torch.cuda.synchronize(dev)
    pairs_per_step = B * (reps[0]["applies_fwd"] + reps[0]["applies_adj"]) / 2.0

    clocks = ClockSampler(local)
    clocks.start()
    ashrt.profile_read()
    ashrt.profile_enable(True)
    launches0 = ashrt.kernel_launches()
    barrier()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        reps = plan.deblend(d, m, drec, batch=B, stream=stream, **kw)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    launches = ashrt.kernel_launches() - launches0
    ashrt.profile_enable(False)
    prof = ashrt.profile_read()
    clk = clocks.stop()
    t, value = whole_job_rate(e0.elapsed_time(e1) / 1000.0, pairs_per_step * args.steps, world,
                              dist, dev)

    # end to end through the public API with host buffers
    e2e_steps = max(1, min(args.steps, 3))
    barrier()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        d.copy_(d_host, non_blocking=True)
        plan.deblend(d, m, drec, batch=B, stream=stream, **kw)
        drec_host.copy_(drec, non_blocking=True)
        torch.cuda.synchronize(dev)
    barrier()
    te, e2e = whole_job_rate(time.perf_counter() - t0, pairs_per_step * e2e_steps, world, dist,
                             dev)

    # deblending quality of the batch (ch. 4 Eqs ch4_Qpd, ch4_Qr), FP64 on the device
    clean = torch.from_numpy(c["clean"].astype(np.float32)).to(dev)
    sums = torch.empty((B, 2), dtype=torch.float64, device=dev)
    q_pd = ashrt.quality_db(clean, d, sums, stream=stream)
    q_r = ashrt.quality_db(clean, drec, sums, stream=stream)

    if rank != 0:
        return
    alg = algorithmic()
    pk = _peaks()
    dom = max(("stolt_fwd_rows", "stolt_adj_rows", "xfft_r2c", "xfft_c2r"),
              key=lambda k: prof[k][0])
    ms, cnt = prof[dom]
    per_launch_s = ms / 1000.0 / max(cnt, 1)
    derived_peak = n_sm * 128 * 2 * pk["sm_max_mhz"] * 1e6 / 1e12   # FP32 lanes x FMA x max clock
    traffic, src_hash = measured_traffic(dom, B, variant)
    if dom.startswith("stolt"):
        achieved = alg["rows_flops"] * B / per_launch_s / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": fp32_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp32_peak, "traffic": traffic,
                    "peak_src": "measured: ashrt_fp32_peak (independent FMA chains on all %d "
                                "SMs, best of 5 launches), median SM clock %s MHz during it"
                                % (n_sm, peak_clk.get("sm_mhz")),
                    "derived_peak": derived_peak,
                    "traffic_src": "profiles/dram_traffic.md, sources %s" % src_hash}
    else:
        byts = xfft_model_bytes(dom, B)
        achieved = byts / per_launch_s / 1e9
        roofline = {"kernel": dom + " (model side)", "bound": "hbm", "achieved": achieved,
                    "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": achieved / pk["hbm_gbs"],
                    "traffic": traffic, "algorithmic_bytes_per_launch": byts,
                    "peak_src": "MEASURED_PEAKS.json hbm_gbs (copy)" if pk["hbm_src"] == "measured"
                                else "fallback 6800 GB/s",
                    "traffic_src": "profiles/dram_traffic.md (one CG-fused launch), sources %s"
                                   % src_hash,
                    "fp32_peak_measured": fp32_peak}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000.0 * t / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": _config(batch=B),
        "gathers_per_s": world * B * args.steps / t,
        "hbm_fraction_pair": {"algorithmic_bytes_per_pair": alg["pair_bytes"],
                              "achieved_gbs": value / world * alg["pair_bytes"] / 1e9,
                              "peak_gbs": pk["hbm_gbs"], "peak_src": pk["hbm_src"]},
        "roofline": roofline,
        "roofline_trace_axis": {
            k: {"bound": "hbm", "achieved": xfft_model_bytes(k, B) / (prof[k][0] / 1000.0 /
                                                                    max(prof[k][1], 1)) / 1e9,
                "unit": "GB/s", "peak": pk["hbm_gbs"],
                "frac": xfft_model_bytes(k, B) / (prof[k][0] / 1000.0 / max(prof[k][1], 1))
                        / 1e9 / pk["hbm_gbs"],
                "algorithmic_bytes_per_launch": xfft_model_bytes(k, B),
                "traffic": measured_traffic(k, B, variant)[0]}
            for k in ("xfft_r2c", "xfft_c2r")},
        "quality": {"q_pd_db_mean": float(np.mean(q_pd)), "q_r_db_mean": float(np.mean(q_r)),
                    "q_improvement_db_mean": float(np.mean(np.asarray(q_r) - np.asarray(q_pd))),
                    "q_r_db_min": float(np.min(q_r)),
                    "what": "Q = 10 log10(|clean|^2 / |clean - x|^2) per gather, x = input "
                            "(Q_PD) or deblended (Q_R), FP64 device reduction"},
        "kernel_ms": {k: {"total_ms": v[0], "launches": v[1]} for k, v in prof.items()},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": int(d_host.numel() * 4),
                "d2h_bytes_per_step": int(drec_host.numel() * 4)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "gpu": torch.cuda.get_device_name(dev),
        "autotuned_variant": {"rows_minb": variant[0], "xfft_cols": variant[1]},
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
        line["cpu_fft_baseline"] = cpu_fft_baseline()
    print(json.dumps(line), flush=True)


def run_ops(args):
    """Operator pairs only, at the workload's gather size (not the bench line)."""
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    nb = args.batch
    v = synth.velocity_scan(1400.0, 3500.0, NV)
    plan = ashrt.Plan(NT, NX, DT, DX, v, wavelet_peak_hz=F_PEAK, max_batch=nb)
    if args.rows_variant:
        plan.set_variant(args.rows_variant, 16)
    g = torch.Generator(device=dev).manual_seed(0)
    m = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
    d = torch.randn((nb, NX, NT), device=dev, generator=g)
    for _ in range(args.warmup):
        plan.forward(m, d, batch=nb)
        plan.adjoint(d, m, batch=nb)
    torch.cuda.synchronize()
    ashrt.profile_read()
    ashrt.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.forward(m, d, batch=nb)
        plan.adjoint(d, m, batch=nb)
    e1.record()
    torch.cuda.synchronize()
    ashrt.profile_enable(False)
    prof = ashrt.profile_read()
    t = e0.elapsed_time(e1) / 1000.0
    print(json.dumps({"mode": "ops", "batch": nb, "rows_variant": args.rows_variant or "default",
                      "pairs_per_s": nb * args.steps / t,
                      "ms_per_pair_call": 1000.0 * t / args.steps,
                      "kernel_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in prof.items()}}),
          flush=True)


def _unet_flops(H, W, cout, ch=(16, 48, 96, 192)):
    """Multiply-add flops of one U-Net forward on an H x W image (2 per MAC)."""
    c0, c1, c2, c3 = ch
    layers = [(1, c0, 3, 1), (c0, c0, 3, 1), (c0, c1, 3, 4), (c1, c1, 3, 4), (c1, c2, 3, 16),
              (c2, c2, 3, 16), (c2, c3, 3, 64), (c3, c3, 3, 64), (c3 + c2, c2, 3, 16),
              (c2, c2, 3, 16), (c2 + c1, c1, 3, 4), (c1, c1, 3, 4), (c1 + c0, c0, 3, 1),
              (c0, c0, 3, 1), (c0, cout, 1, 1)]
    return sum(2.0 * ci * co * k * k * H * W / div for ci, co, k, div in layers)


def run_unet(args):
    """Warm-start U-Net inference on 256 x 1024 gathers, 25 output channels (the
    c5 warm start's network; a profiling aid, not the bench line)."""
    import torch

    from paper_1711_10214_gb300 import ashrt
    dev = torch.device("cuda", 0)
    nb, H, W, cout = args.batch, NX, NT, 25
    net = ashrt.UNet(H, W, cout, max_batch=nb)
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.randn((nb, H, W), device=dev, generator=g)
    y = torch.empty((nb, cout, H, W), device=dev)
    for _ in range(args.warmup):
        net.forward(x, y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        net.forward(x, y)
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1000.0 / args.steps
    f = _unet_flops(H, W, cout) * nb
    print(json.dumps({"mode": "unet", "batch": nb, "ms_per_image": 1000.0 * t / nb,
                      "images_per_s": nb / t, "tflops": f / t / 1e12,
                      "gflop_per_image": f / nb / 1e9}), flush=True)
    net.close()


def run_td(args):
    """The thesis's ch. 5 speed comparison on one GPU: time-domain ASHRT
    (hyperbolic summation) against the Stolt form, forward + adjoint pairs on
    the same gathers (not the bench line)."""
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    nb = args.batch
    v = synth.velocity_scan(1400.0, 3500.0, NV)
    plan = ashrt.Plan(NT, NX, DT, DX, v, max_batch=nb)
    g = torch.Generator(device=dev).manual_seed(0)
    m = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
    d = torch.randn((nb, NX, NT), device=dev, generator=g)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    ms = {
        "td_forward": timed(lambda: ashrt.td_forward(NT, NX, DT, DX, v, m, d, batch=nb)),
        "td_adjoint": timed(lambda: ashrt.td_adjoint(NT, NX, DT, DX, v, d, m, batch=nb)),
        "stolt_forward": timed(lambda: plan.forward(m, d, batch=nb)),
        "stolt_adjoint": timed(lambda: plan.adjoint(d, m, batch=nb)),
    }
    td = ms["td_forward"] + ms["td_adjoint"]
    st = ms["stolt_forward"] + ms["stolt_adjoint"]
    print(json.dumps({"mode": "td", "batch": nb, "nt": NT, "nx": NX, "nv": NV,
                      "ms_per_call": ms, "td_pairs_per_s": nb * 1000.0 / td,
                      "stolt_pairs_per_s": nb * 1000.0 / st, "stolt_speedup": td / st}),
          flush=True)
    plan.close()


def run_fista(args):
    """FISTA interpolation (ch. 6 "Sparse inversion") on the workload's
    gathers with one trace in five kept: 20 power-method and 30 FISTA
    iterations per call (not the bench line)."""
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    nb = args.batch
    c = synth.config2(nb, NT, NX, NV)
    d = torch.from_numpy(c["blended"].astype("float32")).to(dev)
    plan = ashrt.Plan(NT, NX, DT, DX, c["velocities"], wavelet_peak_hz=F_PEAK, max_batch=nb,
                      with_solver=True)
    mask = torch.zeros((nb, NX), device=dev)
    mask[:, ::5] = 1.0
    g = torch.Generator(device=dev).manual_seed(0)
    v0 = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
    m = torch.empty((nb,) + plan.model_shape, device=dev)
    drec = torch.empty_like(d)
    n_iter, n_power = 30, 20
    for _ in range(args.warmup):
        plan.fista(d, m, v0, drec=drec, mask=mask, batch=nb, mu=0.01, n_iter=n_iter,
                   n_power=n_power)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.fista(d, m, v0, drec=drec, mask=mask, batch=nb, mu=0.01, n_iter=n_iter,
                   n_power=n_power)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    pairs = n_iter + n_power + 1.0 / 2.0          # + the reconstruction forward
    print(json.dumps({"mode": "fista", "batch": nb, "n_iter": n_iter, "n_power": n_power,
                      "ms_per_call": ms, "gathers_per_s": nb * 1000.0 / ms,
                      "pairs_per_s": nb * pairs * 1000.0 / ms}), flush=True)
    plan.close()


def run_cube(args):
    """The acquisition model around the solve on a whole cube: 256 shots x 64
    receivers x 1024 samples of three flat reflectors, fired every 512
    samples with up to 256 samples of dither; blend, pseudo-deblend, sort to
    64 receiver gathers (the bench workload's size), robust deblend (8 x 30),
    sort back (not the bench line)."""
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    ns, nr, nt = 256, NX // 4, NT
    dev = torch.device("cuda", 0)
    xs = np.arange(ns) * DX
    xr = (np.arange(nr) * 4 + 2) * DX
    t = np.arange(nt) * DT
    D = np.zeros((ns, nr, nt), np.float32)
    for tau, v, A in ((0.3, 1600.0, 1.0), (0.8, 2000.0, -0.7), (1.4, 2400.0, 0.6),
                      (2.2, 2800.0, 0.5)):
        tt = np.sqrt(tau * tau + ((xs[:, None] - xr[None, :]) / v) ** 2)
        D += (A * synth.ricker(t[None, None, :] - tt[:, :, None], F_PEAK)).astype(np.float32)
    rng = np.random.default_rng(0)
    fire = (np.arange(ns) * (nt // 2) + rng.integers(0, nt // 4, ns)).astype(np.int32)
    nb = int(fire.max()) + nt
    Dd, fd = torch.from_numpy(D).to(dev), torch.from_numpy(fire).to(dev)
    b = torch.empty((nr, nb), device=dev)
    Dt = torch.empty_like(Dd)
    crg = torch.empty((nr, ns, nt), device=dev)
    rec_crg = torch.empty_like(crg)
    rec = torch.empty_like(Dd)
    plan = ashrt.Plan(nt, ns, DT, DX, synth.velocity_scan(1400.0, 3500.0, NV),
                      wavelet_peak_hz=F_PEAK, max_batch=nr, with_solver=True)
    m = torch.empty((nr,) + plan.model_shape, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    stages = ("blend", "pseudo_deblend", "sort_to_receivers", "deblend", "sort_to_shots")
    for rep in range(2):                      # the first pass warms everything up
        ev[0].record()
        ashrt.blend(Dd, fd, b)
        ev[1].record()
        ashrt.pseudo_deblend(b, fd, Dt)
        ev[2].record()
        ashrt.sort_gathers(Dt, crg)
        ev[3].record()
        plan.deblend(crg, m, rec_crg, batch=nr, p=1.0, q=1.0, n_outer=N_OUTER, n_cg=N_CG)
        ev[4].record()
        ashrt.sort_gathers(rec_crg, rec)
        ev[5].record()
        torch.cuda.synchronize()
    ms = {k: ev[i].elapsed_time(ev[i + 1]) for i, k in enumerate(stages)}

    def q_db(ref, x):
        return float(10.0 * torch.log10((ref.double() ** 2).sum() /
                                        ((ref.double() - x.double()) ** 2).sum()))

    print(json.dumps({"mode": "cube", "shots": ns, "receivers": nr, "nt": nt, "record": nb,
                      "ms": ms, "q_pseudo_deblended_db": q_db(Dd, Dt),
                      "q_deblended_db": q_db(Dd, rec)}), flush=True)
    plan.close()


def run_c1(args):
    """c1 workload: one 256 x 64 gather, 8 velocities, IRLS 5 x 20 (p = q = 1,
    20 Hz wavelet): the GPU solve, the FP64 oracle solve and the same solve on
    the scipy.fft operator (FP64 and FP32), timed; Q of each."""
    import numpy as np
    import torch

    from oracle import irls, stolt
    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    c = synth.config1(0)
    nt, nx, v, fp = c["nt"], c["nx"], c["velocities"], c["f_peak"]
    kw = dict(p=1.0, q=1.0, n_outer=5, n_cg=20)
    plan = ashrt.Plan(nt, nx, DT, DX, v, wavelet_peak_hz=fp, with_solver=True)
    d = torch.from_numpy(c["blended"][None].astype(np.float32)).to(dev)
    m = torch.empty((1,) + plan.model_shape, device=dev)
    drec = torch.empty_like(d)
    for _ in range(args.warmup):
        reps = plan.deblend(d, m, drec, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        reps = plan.deblend(d, m, drec, **kw)
    torch.cuda.synchronize()
    t_gpu = (time.perf_counter() - t0) / args.steps
    pairs = (reps[0]["applies_fwd"] + reps[0]["applies_adj"]) / 2.0
    q_gpu = float(irls.q_db(c["clean"], drec[0].cpu().numpy()))
    g = stolt.Geometry(nt, nx, DT, DX, v, wavelet_peak_hz=fp)
    d64 = c["blended"].astype(np.float32).astype(np.float64)
    t0 = time.perf_counter()
    _, rep_o = irls.irls(lambda x: stolt.forward(g, x), lambda r: stolt.adjoint(g, r), d64, **{
        k: int(v_) if k.startswith("n_") else v_ for k, v_ in kw.items()})
    t_or = time.perf_counter() - t0
    out = {"mode": "c1", "nt": nt, "nx": nx, "nv": len(v), "irls": [5, 20],
           "gpu": {"s_per_solve": t_gpu, "gathers_per_s": 1.0 / t_gpu,
                   "pairs_per_s": pairs / t_gpu, "q_db": q_gpu},
           "oracle": {"s_per_solve": t_or, "q_db": float(irls.q_db(c["clean"], rep_o["d_model"])),
                      "cores": os.cpu_count()},
           "q_pd_db": float(irls.q_db(c["clean"], c["blended"]))}
    for dt_ in ("float64", "float32"):
        op = ScipyStolt(nt, nx, DT, DX, v, wavelet_peak_hz=fp, dtype=dt_)
        t0 = time.perf_counter()
        _, rep_s = irls.irls(lambda x: op.forward(x), lambda r: op.adjoint(r, 1, len(v)), d64,
                             n_outer=5, n_cg=20, p=1, q=1)
        ts = time.perf_counter() - t0
        out["cpu_fft_" + dt_] = {"s_per_solve": ts, "q_db": float(irls.q_db(c["clean"],
                                                                            rep_s["d_model"])),
                                 "cores": os.cpu_count()}
    print(json.dumps(out), flush=True)
    plan.close()


def run_irregular(args):
    """The workload's gathers (64 x nt 1024, 32 velocities, 256 apexes)
    recorded at 256 jittered trace positions (x_j = (j + U(-0.45, 0.45)) dx):
    forward + adjoint pairs and the 8 x 30 robust deblend on the irregular
    plan (data-side x transforms as DFTs at the traces) against the regular
    plan on the same sizes."""
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    nb = args.batch
    v = synth.velocity_scan(1400.0, 3500.0, NV)
    rng = np.random.default_rng(0)
    x = (np.arange(NX) + rng.uniform(-0.45, 0.45, NX)) * DX
    c = synth.config2(nb, NT, NX, NV)
    d = torch.from_numpy(c["blended"].astype(np.float32)).to(dev)
    out = {"mode": "irregular", "batch": nb, "nt": NT, "nx": NX, "nr": NX, "nv": NV}
    for name, tx in (("regular", None), ("irregular", x)):
        plan = ashrt.Plan(NT, NX, DT, DX, v, wavelet_peak_hz=F_PEAK, max_batch=nb,
                          with_solver=True, trace_x=tx)
        g = torch.Generator(device=dev).manual_seed(0)
        m = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
        dd = torch.empty_like(d)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for _ in range(args.warmup):
            plan.forward(m, dd, batch=nb)
            plan.adjoint(dd, m, batch=nb)
        torch.cuda.synchronize()
        ashrt.profile_read()
        ashrt.profile_enable(True)
        e0.record()
        for _ in range(args.steps):
            plan.forward(m, dd, batch=nb)
            plan.adjoint(dd, m, batch=nb)
        e1.record()
        torch.cuda.synchronize()
        ashrt.profile_enable(False)
        prof = ashrt.profile_read()
        t = e0.elapsed_time(e1) / 1000.0 / args.steps
        drec = torch.empty_like(d)
        plan.deblend(d, m, drec, batch=nb, p=1.0, q=1.0, n_outer=N_OUTER, n_cg=N_CG)
        torch.cuda.synchronize()
        e0.record()
        reps = plan.deblend(d, m, drec, batch=nb, p=1.0, q=1.0, n_outer=N_OUTER, n_cg=N_CG)
        e1.record()
        torch.cuda.synchronize()
        td = e0.elapsed_time(e1) / 1000.0
        out[name] = {"pairs_per_s": nb / t, "ms_per_pair_call": 1000.0 * t,
                     "kernel_ms_per_launch": {k: w[0] / max(w[1], 1) for k, w in prof.items()},
                     "deblend_s": td, "deblend_gathers_per_s": nb / td,
                     "deblend_pairs_per_s": nb * (reps[0]["applies_fwd"] +
                                                  reps[0]["applies_adj"]) / 2.0 / td}
        plan.close()
    out["irregular_over_regular_time"] = (out["regular"]["pairs_per_s"] /
                                          out["irregular"]["pairs_per_s"])
    print(json.dumps(out), flush=True)


def run_c3(args):
    """c3 workload: AASHRT (24 velocities x 16 asymptote shifts = 384 panels)
    on 16 gathers of nt 1024 x nx 256 with half of the traces removed (the
    trace mask S), the velocity sum and phase shift fused in the row kernels;
    forward + adjoint pairs, then the FISTA interpolation of the gathers (ch. 6
    "Sparse inversion", 20 power + 30 FISTA iterations) with Q of the
    interpolated gathers against the complete ones."""
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    nb = min(args.batch, 16)
    c = synth.config3(nb)
    plan = ashrt.Plan(NT, NX, DT, DX, c["velocities"], t0s=c["t0s"], wavelet_peak_hz=F_PEAK,
                      max_batch=nb, with_solver=True)
    mask = torch.from_numpy(c["mask"]).to(dev)
    obs = torch.from_numpy(c["observed"].astype(np.float32)).to(dev)
    clean = torch.from_numpy(c["clean"].astype(np.float32)).to(dev)
    g = torch.Generator(device=dev).manual_seed(0)
    m = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
    d = torch.empty_like(obs)
    for _ in range(args.warmup):
        plan.forward(m, d, mask=mask, batch=nb)
        plan.adjoint(d, m, mask=mask, batch=nb)
    torch.cuda.synchronize()
    ashrt.profile_read()
    ashrt.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        plan.forward(m, d, mask=mask, batch=nb)
        plan.adjoint(d, m, mask=mask, batch=nb)
    e1.record()
    torch.cuda.synchronize()
    ashrt.profile_enable(False)
    prof = ashrt.profile_read()
    t = e0.elapsed_time(e1) / 1000.0 / args.steps
    P = plan.P
    alg = algorithmic(P=P)
    v0 = torch.randn((nb,) + plan.model_shape, device=dev, generator=g)
    drec = torch.empty_like(obs)
    e0.record()
    plan.fista(obs, m, v0, drec=drec, mask=mask, batch=nb, mu=0.01, n_iter=30, n_power=20)
    e1.record()
    torch.cuda.synchronize()
    t_f = e0.elapsed_time(e1) / 1000.0
    sums = torch.empty((nb, 2), dtype=torch.float64, device=dev)
    q_obs = ashrt.quality_db(clean, obs, sums)
    q_rec = ashrt.quality_db(clean, drec, sums)
    print(json.dumps({
        "mode": "c3", "gathers": nb, "panels": P, "nt": NT, "nx": NX,
        "traces_kept": float(c["mask"].mean()), "pairs_per_s": nb / t,
        "ms_per_pair_call": 1000.0 * t,
        "kernel_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in prof.items()},
        "pair_tflops": alg["pair_flops"] * nb / t / 1e12,
        "pair_algorithmic_gbs": alg["pair_bytes"] * nb / t / 1e9,
        "fista": {"n_power": 20, "n_iter": 30, "s": t_f, "gathers_per_s": nb / t_f,
                  "q_observed_db_mean": float(np.mean(q_obs)),
                  "q_interpolated_db_mean": float(np.mean(q_rec))}}), flush=True)
    plan.close()


def run_c4(args):
    """c4 workload: gathers of uneven width (nx ~ U{96..480}, nt 1500, 5-40
    events, three dithered interfering sources, 24 velocities, 25 Hz) deblended
    through the batch layer: classes per padded width Nx, each class streamed
    through a resident pool of 64 gathers with the autotuned row kernels; the
    whole pass with recorded graphs (use_graph) and with direct launches."""
    import numpy as np
    import torch

    from paper_1711_10214_gb300 import ashrt, synth
    dev = torch.device("cuda", 0)
    n, nt = args.gathers, 1500
    nxs = synth.config4_sizes(n)
    t0 = time.perf_counter()
    c = synth.config4(range(n), nxs, nt=nt, processes=os.cpu_count())
    t_gen = time.perf_counter() - t0
    b = ashrt.Batch(nt, nxs, DT, DX, c["velocities"], wavelet_peak_hz=F_PEAK, max_resident=64,
                    with_solver=True)
    b.autotune(os.environ.get("ASHRT_TUNE_CACHE", "/tmp/ashrt_autotune.jsonl"))
    d = torch.from_numpy(c["blended"]).to(dev)
    clean = torch.from_numpy(c["clean"]).to(dev)
    m = torch.empty(b.model_elems, device=dev)
    drec = torch.empty_like(d)
    no, ncg = args.irls
    kw = dict(p=1.0, q=1.0, n_outer=no, n_cg=ncg)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def run(graph):
        ev[0].record()
        reps = b.deblend(d, m, drec, use_graph=graph, **kw)
        ev[1].record()
        torch.cuda.synchronize()
        return ev[0].elapsed_time(ev[1]) / 1000.0, reps

    run(1)                                        # records the class graphs, loads kernels
    l0 = ashrt.kernel_launches()
    t_graph, reps = run(1)
    l1 = ashrt.kernel_launches()
    t_direct, _ = run(0)
    pairs = sum((r["applies_fwd"] + r["applies_adj"]) / 2.0 for r in reps)
    sums = torch.empty((n, 2), dtype=torch.float64, device=dev)
    off = 0
    for g, nx in enumerate(nxs):
        k = int(nx) * nt
        ashrt.quality_db(clean[off:off + k], d[off:off + k], sums[g], batch=1, n=k, sync=False)
        off += k
    s_pd = sums.cpu().numpy().copy()
    off = 0
    for g, nx in enumerate(nxs):
        k = int(nx) * nt
        ashrt.quality_db(clean[off:off + k], drec[off:off + k], sums[g], batch=1, n=k, sync=False)
        off += k
    s_r = sums.cpu().numpy()
    q_pd = 10 * np.log10(s_pd[:, 0] / s_pd[:, 1])
    q_r = 10 * np.log10(s_r[:, 0] / s_r[:, 1])
    widths = np.array([2 ** int(np.ceil(np.log2(2 * x))) for x in nxs])
    print(json.dumps({
        "mode": "c4", "gathers": n, "nt": nt, "nx_range": [int(nxs.min()), int(nxs.max())],
        "nv": 24, "irls": [no, ncg], "classes": b.n_classes,
        "gathers_per_class_Nx": {str(w): int((widths == w).sum()) for w in np.unique(widths)},
        "resident_pool": 64, "device_bytes_held": b.workspace_bytes,
        "graph": {"s": t_graph, "gathers_per_s": n / t_graph, "pairs_per_s": pairs / t_graph,
                  "launches": l1 - l0},
        "direct": {"s": t_direct, "gathers_per_s": n / t_direct, "pairs_per_s": pairs / t_direct},
        "graph_over_direct_speedup": t_direct / t_graph,
        "q_pd_db_mean": float(np.mean(q_pd)), "q_r_db_mean": float(np.mean(q_r)),
        "q_improvement_db_mean": float(np.mean(q_r - q_pd)),
        "generation_s": t_gen}), flush=True)
    b.close()


def main():
    args = _args()
    if args.mode == "c1":
        run_c1(args)
        return
    if args.mode == "irregular":
        run_irregular(args)
        return
    if args.mode == "c3":
        run_c3(args)
        return
    if args.mode == "c4":
        run_c4(args)
        return
    if args.mode == "cube":
        run_cube(args)
        return
    if args.mode == "fista":
        run_fista(args)
        return
    if args.mode == "td":
        run_td(args)
        return
    if args.mode == "ops":
        run_ops(args)
        return
    if args.mode == "unet":
        run_unet(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
