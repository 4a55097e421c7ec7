"""Learned warm start of the robust deblending solve.

The thesis starts every IRLS solve cold (m = 0, W_r = W_m = I at the first
outer iteration, ch. 4).  Here a U-Net (``ashrt_unet_*`` in the library)
learns, from pairs the cold solve itself produces, to map a pseudo-deblended
gather to (a) an initial Radon model m0 and (b) initial residual weights W_r0;
the solve then starts from them (``irls_opts.m0_dev`` / ``wr0_dev``).  The cold
solve stays the reference: the warm start is measured by the operator applies
and gathers/s it needs to reach the cold solve's deblending quality within a
stated margin (0.1 dB of Q).

Everything on the device runs in the library's kernels; this module only
orders the calls: render gathers on the host (a process pool), solve cold in
chunks, turn each solve into targets, train online (every pair is used for a
few minibatch steps right after it is solved, then dropped, so memory stays
bounded however many pairs are used), and evaluate warm against cold on a
disjoint set of gathers over a ladder of iteration budgets.
"""
import argparse
import json
import math
import os
import time

import numpy as np

from . import ashrt, synth

# (n_outer, n_cg) iteration budgets of the evaluation ladder, smallest first
BUDGETS = [(1, 5), (1, 10), (1, 20), (1, 30), (2, 15), (2, 30), (3, 30), (4, 30), (5, 30),
           (6, 30), (8, 30)]
REFERENCE = (8, 30)
TEST_SEED0 = 1_000_000


class Source:
    """Seeded gathers of one recipe: c5 (any nt, nx; 24 velocities, 25 Hz)
    or c1 (nt 256, nx 64; 8 velocities, 20 Hz)."""

    def __init__(self, name="c5", nt=1024, nx=256):
        if name == "c1":
            c = synth.config1(0)
            self.job, self.nt, self.nx = synth._c1_job, c["nt"], c["nx"]
        elif name == "c5":
            c = synth.config5([0], nt=nt, nx=nx)
            self.job, self.nt, self.nx = synth._c5_job, nt, nx
        else:
            raise ValueError("unknown gather source %r" % name)
        self.name, self.velocities, self.f_peak = name, c["velocities"], c["f_peak"]

    def args(self, ids):
        return [(g, self.nt, self.nx) for g in ids]


def q_db(clean, rec):
    """Deblending quality Q = 10 log10(||clean||^2 / ||clean - rec||^2) per gather (ch. 4)."""
    c = clean.reshape(clean.shape[0], -1).astype(np.float64)
    r = rec.reshape(rec.shape[0], -1).astype(np.float64)
    return 10.0 * np.log10(np.sum(c * c, 1) / np.maximum(np.sum((c - r) ** 2, 1), 1e-300))


class WarmStart:
    """A plan with the solver plus a U-Net for one gather size."""

    def __init__(self, nt, nx, velocities, dt=synth.DT, dx=synth.DX, chunk=64, train_batch=8,
                 wavelet_peak_hz=25.0, p=1.0, q=1.0, params=None, source=None, w_weight=0.75):
        import torch
        self.torch = torch
        self.dev = torch.device("cuda:0")
        self.nt, self.nx, self.chunk, self.tb = nt, nx, chunk, train_batch
        self.source = source or Source("c5", nt, nx)
        self.p, self.q = p, q
        self.plan = ashrt.Plan(nt, nx, dt, dx, velocities, max_batch=chunk, with_solver=True,
                               wavelet_peak_hz=wavelet_peak_hz)
        self.P = int(np.prod(self.plan.model_shape[:-2]))
        self.net = ashrt.UNet(nx, nt, self.P + 1, max_batch=max(chunk, train_batch),
                              params=params)
        B = chunk
        self.d = torch.empty((B, nx, nt), device=self.dev)
        self.m = torch.empty((B,) + tuple(self.plan.model_shape), device=self.dev)
        self.drec = torch.empty((B, nx, nt), device=self.dev)
        self.wr = torch.empty((B, nx, nt), device=self.dev)
        self.m0 = torch.empty_like(self.m)
        self.wr0 = torch.empty_like(self.wr)
        self.t = torch.empty((B, self.P + 1, nx, nt), device=self.dev)
        self.lam = None
        self.w_weight = w_weight

    def upload(self, blended):
        n = blended.shape[0]
        self.d[:n].copy_(self.torch.from_numpy(np.ascontiguousarray(blended, np.float32)))
        return n

    def solve(self, n, n_outer, n_cg, warm=None, wr_out=False):
        """Robust solve of the first n uploaded gathers; warm = None (cold),
        "w" (predicted W_r0 only) or "mw" (predicted m0 and W_r0)."""
        kw = dict(p=self.p, q=self.q, n_outer=n_outer, n_cg=n_cg)
        if warm:
            self.net.predict(self.d, self.m0 if "m" in warm else None, self.wr0, n=n, p=self.p)
            kw.update(wr0=self.wr0)
            if "m" in warm:
                kw.update(m0=self.m0)
        return self.plan.deblend(self.d, self.m, self.drec, batch=n,
                                 wr_out=self.wr if wr_out else None, **kw)

    def train_chunk(self, n, lr, passes=1, rng=None):
        """Targets from the last cold solve of n gathers, then `passes` epochs
        of minibatch Adam steps over them (contiguous minibatches of the
        chunk, whose gathers are independent draws, in random order);
        returns the mean loss."""
        self.net.targets(self.d, self.m, self.wr, self.t, n=n, p=self.p)
        if self.lam is None:
            # per-group weights from the first gathers' targets: variance-
            # normalised errors, log W_r weighted w_weight, the panels the rest
            tv = self.t[:min(n, 4)].cpu().numpy().astype(np.float64)
            vm, vw = tv[:, :self.P].var(), tv[:, self.P].var()
            ww = self.w_weight
            self.lam = np.array([(1.0 - ww) / (self.P * max(vm, 1e-30))] * self.P
                                + [ww / max(vw, 1e-30)], np.float32)
        rng = rng or np.random.default_rng(0)
        losses = []
        starts = list(range(0, n - self.tb + 1, self.tb))
        for _ in range(passes):
            for s in rng.permutation(starts):
                losses.append(self.net.train_step(self.d[s:s + self.tb], self.t[s:s + self.tb],
                                                  lr, channel_weight=self.lam))
        return float(np.mean(losses)) if losses else float("nan")

    def close(self):
        self.plan.close()
        self.net.close()


def _lr(step, total, lr0, lr1):
    return lr1 + 0.5 * (lr0 - lr1) * (1.0 + math.cos(math.pi * min(step / max(total, 1), 1.0)))


def train(ws, n_train, processes=8, passes=2, lr0=1e-3, lr1=1e-4, log=None, epochs=1):
    """Online training on gathers 0..n_train-1 of the plan's source: render,
    cold-solve at the reference budget, train `passes` times over each chunk;
    `epochs` > 1 repeats the whole sequence (re-rendering and re-solving, so
    memory stays bounded).  Returns a summary dict."""
    import multiprocessing as mp
    src = ws.source
    chunks = [list(range(s, min(s + ws.chunk, n_train))) for s in range(0, n_train, ws.chunk)]
    chunks = chunks * max(1, int(epochs))
    pool = mp.get_context("spawn").Pool(processes) if processes > 1 else None
    rng = np.random.default_rng(7)

    def render(ids):
        return [src.job(a) for a in src.args(ids)]

    t_solve = t_train = 0.0
    hist = []
    nxt = pool.map_async(src.job, src.args(chunks[0])) if pool else None
    for ci, ids in enumerate(chunks):
        res = nxt.get(timeout=900) if pool else render(ids)
        if pool and ci + 1 < len(chunks):
            nxt = pool.map_async(src.job, src.args(chunks[ci + 1]))
        n = ws.upload(np.stack([b for _, b in res]))
        t0 = time.perf_counter()
        ws.solve(n, *REFERENCE, wr_out=True)
        ws.torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss = ws.train_chunk(n, _lr(ci, len(chunks), lr0, lr1), passes=passes, rng=rng)
        ws.torch.cuda.synchronize()
        t2 = time.perf_counter()
        t_solve += t1 - t0
        t_train += t2 - t1
        hist.append(loss)
        if log:
            log("chunk %d/%d loss %.4f solve %.1fs train %.1fs" % (ci + 1, len(chunks), loss,
                                                                  t1 - t0, t2 - t1))
    if pool:
        pool.close()
        pool.join()
    return dict(n_train=n_train, passes=passes, epochs=epochs, chunk=ws.chunk, train_batch=ws.tb,
                solve_s=t_solve, train_s=t_train, loss_first=hist[0], loss_last=hist[-1],
                loss_history=hist)


def evaluate(ws, n_test, processes=8, budgets=BUDGETS, margin_db=0.1,
             arms=("cold", "warm_w", "warm_mw"), warm_budgets=None):
    """Cold and warm solves of gathers TEST_SEED0.. (disjoint from training)
    over the budget ladder.  Arms: cold; warm_w (predicted W_r0, m = 0);
    warm_mw (predicted m0 and W_r0).

    For each budget: mean Q = Q_R - Q_PD (the improvement over the
    pseudo-deblended gather, ch. 4), operator applies per gather (forward +
    adjoint, including the warm start's residual apply), and gathers/s (device
    time of prediction + solve).  The target is the cold reference budget's
    mean Q minus margin_db; each arm's answer is its cheapest budget that
    reaches it.  warm_budgets (optional) is a shorter ladder for the warm
    arms.
    """
    import multiprocessing as mp
    src = ws.source
    ids = list(range(TEST_SEED0, TEST_SEED0 + n_test))
    if processes > 1:
        with mp.get_context("spawn").Pool(processes) as pool:
            res = pool.map_async(src.job, src.args(ids)).get(timeout=900)
    else:
        res = [src.job(a) for a in src.args(ids)]
    clean = np.stack([c for c, _ in res])
    blended = np.stack([b for _, b in res])
    q_pd = q_db(clean, blended)
    torch = ws.torch
    out = {arm: [] for arm in arms}
    for arm in arms:
        ladder = budgets if (arm == "cold" or warm_budgets is None) else warm_budgets
        for (no, nc) in ladder:
            qs, applies, secs = [], 0, 0.0
            for s in range(0, n_test, ws.chunk):
                n = ws.upload(blended[s:s + ws.chunk])
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                reps = ws.solve(n, no, nc, warm=arm[5:] if arm.startswith("warm") else None)
                e1.record()
                torch.cuda.synchronize()
                secs += e0.elapsed_time(e1) / 1e3
                applies += sum(r["applies_fwd"] + r["applies_adj"] for r in reps)
                qs.extend((q_db(clean[s:s + n], ws.drec[:n].cpu().numpy()) - q_pd[s:s + n]).tolist())
            out[arm].append(dict(n_outer=no, n_cg=nc, q_db=float(np.mean(qs)),
                                 applies=applies / n_test, gathers_per_s=n_test / secs))
    ref = [r for r in out["cold"] if (r["n_outer"], r["n_cg"]) == REFERENCE][0]
    target = ref["q_db"] - margin_db
    out["q_cold_ref_db"] = ref["q_db"]
    out["q_target_db"] = target
    for arm in arms:
        ok = [r for r in out[arm] if r["q_db"] >= target]
        out[arm + "_reach"] = min(ok, key=lambda r: r["applies"]) if ok else None
    out["n_test"] = n_test
    out["q_pd_db"] = float(q_pd.mean())
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="train and evaluate the learned warm start (c5)")
    ap.add_argument("--source", default="c5")
    ap.add_argument("--epochs", type=int, default=1)
    ap.add_argument("--nt", type=int, default=1024)
    ap.add_argument("--nx", type=int, default=256)
    ap.add_argument("--train", type=int, default=2048)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--passes", type=int, default=6)
    ap.add_argument("--chunk", type=int, default=64)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--w-weight", type=float, default=0.75)
    ap.add_argument("--processes", type=int, default=min(12, os.cpu_count() or 1))
    ap.add_argument("--out", default=None)
    ap.add_argument("--save-params", default=None)
    ap.add_argument("--warm-budgets", default=None,
                    help="ladder of the warm arms (default: --budgets)")
    ap.add_argument("--arms", default="cold,warm_w,warm_mw")
    ap.add_argument("--budgets", default=None,
                    help="evaluation ladder as outer x CG pairs, e.g. 1x5,8x30 "
                         "(default: the full ladder; it must contain 8x30)")
    a = ap.parse_args(argv)
    import multiprocessing as mp
    mp.get_context("spawn")
    src = Source(a.source, a.nt, a.nx)
    ws = WarmStart(src.nt, src.nx, src.velocities, chunk=a.chunk, train_batch=a.batch,
                   wavelet_peak_hz=src.f_peak, source=src, w_weight=a.w_weight)
    log = lambda s: print(s, flush=True)
    t0 = time.perf_counter()
    tr = train(ws, a.train, processes=a.processes, passes=a.passes, lr0=a.lr, log=log,
               epochs=a.epochs)
    tr["wall_s"] = time.perf_counter() - t0
    budgets = BUDGETS
    if a.budgets:
        budgets = [tuple(int(v) for v in b.split("x")) for b in a.budgets.split(",")]
        if REFERENCE not in budgets:
            raise SystemExit("--budgets must contain the reference budget 8x30")
    parse = lambda txt: [tuple(int(v) for v in b.split("x")) for b in txt.split(",")]
    ev = evaluate(ws, a.test, processes=a.processes, budgets=budgets,
                  arms=tuple(a.arms.split(",")),
                  warm_budgets=parse(a.warm_budgets) if a.warm_budgets else None)
    res = dict(config=dict(workload="%s warm start" % src.name, nt=src.nt, nx=src.nx,
                           nv=len(src.velocities), params=ws.net.n_params), train=tr, eval=ev)
    print(json.dumps({k: v for k, v in ev.items() if k.endswith("reach") or k.startswith("q_")}))
    if a.out:
        with open(a.out, "w") as f:
            json.dump(res, f, indent=1)
    if a.save_params:
        np.save(a.save_params, ws.net.params())
    ws.close()
    return res


if __name__ == "__main__":
    main()
