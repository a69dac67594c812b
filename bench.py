"""Throughput benchmark: PD and FD L-MMSE equalization on GB300.

One step = PD equalization and FD equalization of the same batch (B=256
antennas, U=16 users, C=8 clusters, 1200 subcarriers x 14 OFDM symbols, 16-QAM,
i.i.d. Rayleigh, 10 dB, LLRs on): every stage of the hot path runs once per
architecture.  The metric counts equalized symbols (subcarrier x symbol x user)
of both architectures per second.

The same JSON line carries the other workloads as extra keys (each timed the
same way, with its own accuracy against the FP64 oracle on sampled subcarriers):
``correlated`` (B=256, U=32, C=16, 3300 x 14, 64-QAM, r = 0.7, 15 dB: FP32
against FP16x3 with and without refinement), ``training`` (one forward +
adjoint step of the differentiable FD form, B=128, U=16, C=8, 8 x 1024
subcarriers, QPSK, 10 dB) and ``uneven`` (4096 instances of mixed size).

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "equalized symbols/s (subcarrier x symbol x user), PD + FD L-MMSE"
UNIT = "symbols/s"
WORKLOAD = dict(B=256, U=16, C=8, n_sc=1200, n_sym=14, bits=4, snr_db=10.0)
CORRELATED = dict(B=256, U=32, C=16, n_sc=3300, n_sym=14, bits=6, snr_db=15.0, corr_r=0.7)
TRAINING = dict(B=128, U=16, C=8, n_sc=8 * 1024, n_sym=1, bits=2, snr_db=10.0)
# Paper, Table I (L-MMSE, B=256, C=8 on 8 V100): PD 0.856 ms, FD 0.751 ms for
# 16*1200*14 symbols each; symbols/s of one PD + one FD pass of the batch.
PAPER_SYMBOLS_PER_S = 2 * 16 * 1200 * 14 / (0.856e-3 + 0.751e-3)
L2_BYTES = 129 * 1024 * 1024
LAMA_ITERS = 8              # LAMA iterations of the equalizer-variant lines
FALLBACK_HBM_GBS = 6800.0
PRECISIONS = ("fp32", "tf32x3", "bf16x3", "fp16x3")
DTYPE = {"fp32": "f32", "tf32x3": "tf32x3+f32", "bf16x3": "bf16x3+f32", "fp16x3": "fp16x3+f32"}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def _source_digest():
    """Digest of the CUDA sources: DRAM counters taken from another build are stale."""
    import glob
    import hashlib
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(ROOT, "paper_1808_04473_gb300", "csrc", "*"))):
        with open(f, "rb") as fh:
            h.update(os.path.basename(f).encode() + fh.read())
    return h.hexdigest()[:16]


def _ncu_traffic():
    """Per-launch DRAM bytes (read + write) from the committed ncu summary, if it
    was taken on the current sources; otherwise {} (the JSON reports null)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return {}
    return d.get("kernels", {}) if d.get("source_digest") == _source_digest() else {}


def max_over_ranks(x: float, device) -> float:
    """The maximum of ``x`` over the ranks of the default process group: the job's
    timed region ends with its slowest rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank_step: float, world: int, steps: int, ms: float) -> float:
    """Whole-job throughput: the units every rank processed in ``steps`` steps over
    the (max-over-ranks) time of the timed region, per second."""
    return world * units_per_rank_step * steps / (ms * 1e-3)


def input_bytes(B, U, n_sc, n_sym):
    """HBM bytes the local preprocessing must read: H and y (complex64)."""
    return n_sc * 8 * (B * U + B * n_sym)


def solve_flops(U, n_sym, C):
    """Algorithmic real flops of one subcarrier's solve stage (independent of the
    method used): per system a Cholesky factorization 4U^3/3, the diagonal of the
    inverse 4U^3/3 and two triangular solves with n_sym right-hand sides 8U^2 n_sym."""
    return C * (8.0 * U ** 3 / 3.0 + 8.0 * U * U * n_sym)


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


ORACLE_CHUNK = 40           # subcarriers per oracle call of the CPU legs


def _time_oracle(budget_s: float, seed: int = 99):
    """The FP64 oracle as it stands on chunks of the headline workload (generation
    excluded): PD and FD with their LLRs, what the GPU step computes.  Returns
    (symbols/s, subcarriers done, seconds spent)."""
    from oracle import llr as ollr
    from oracle import lmmse
    from paper_1808_04473_gb300 import synth
    w = WORKLOAD
    p = synth.make_problem(w["B"], w["U"], w["C"], ORACLE_CHUNK, w["n_sym"], snr_db=w["snr_db"], bits=w["bits"],
                           seed=seed)
    done, spent = 0, 0.0
    while spent < budget_s:
        t = time.perf_counter()
        for f in (lmmse.equalize_pd, lmmse.equalize_fd):
            o = f(p.H, p.y, p.N0, p.Es, p.C)
            ollr.maxlog_llr(o["z"], o["sigma2"][:, None, :], w["bits"], p.Es)
        spent += time.perf_counter() - t
        done += ORACLE_CHUNK
    return 2 * w["U"] * w["n_sym"] * done / spent, done, spent


def numpy32_equalize(H, y, N0: float, Es: float, C: int, fd: bool):
    """CPU throughput baseline (not the oracle): the L-MMSE path in FP32 NumPy,
    batched over subcarriers -- Gram matrices and matched filters by batched
    products, Cholesky factors by ``np.linalg.cholesky``, the diagonal of the
    inverse and the estimates by ``np.linalg.solve`` on the factors, unbiased
    pairs, and for FD the optimal fusion.  Returns (z [n_sc][n_sym][U], sigma2)."""
    import numpy as np
    n_sc, U, B = H.shape
    rho = np.float32(N0 / Es)
    eye = np.eye(U, dtype=np.complex64)
    S = B // C
    parts = [(c * S, (c + 1) * S) for c in range(C)] if fd else [(0, B)]
    num = np.zeros((n_sc, U, y.shape[1]), np.complex64)
    den = np.zeros((n_sc, U), np.float32)
    for b0, b1 in parts:
        Hc = H[:, :, b0:b1]                                   # [n_sc][U][S]
        G = Hc.conj() @ Hc.transpose(0, 2, 1) + rho * eye     # G + rho I
        b = Hc.conj() @ y[:, :, b0:b1].transpose(0, 2, 1)     # [n_sc][U][n_sym]
        L = np.linalg.cholesky(G)
        Li = np.linalg.solve(L, np.broadcast_to(eye, G.shape))
        A_diag = np.einsum("kij,kij->kj", Li.conj(), Li).real   # diag of L^-H L^-1
        x = np.linalg.solve(L.conj().transpose(0, 2, 1), np.linalg.solve(L, b))
        mu = np.maximum(1.0 - rho * A_diag, 0.0)
        w = mu / A_diag                                       # Es / unbiased variance, N0 cancelled
        num += x / A_diag[:, :, None]
        den += w
    z = num / den[:, :, None]
    return z.transpose(0, 2, 1), N0 / den


def _time_numpy32(budget_s: float, seed: int = 99):
    from paper_1808_04473_gb300 import synth
    w = WORKLOAD
    p = synth.make_problem(w["B"], w["U"], w["C"], 4 * ORACLE_CHUNK, w["n_sym"], snr_db=w["snr_db"],
                           bits=w["bits"], seed=seed)
    done, spent = 0, 0.0
    while spent < budget_s:
        t = time.perf_counter()
        for fd in (False, True):
            numpy32_equalize(p.H, p.y, p.N0, p.Es, p.C, fd)
        spent += time.perf_counter() - t
        done += 4 * ORACLE_CHUNK
    return 2 * w["U"] * w["n_sym"] * done / spent, done, spent


def _cpu_worker(job):
    kind, budget_s, seed = job
    f = _time_oracle if kind == "oracle" else _time_numpy32
    _, done, spent = f(budget_s, seed)
    return done, spent


def _single_thread_env():
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    for k in keys:
        os.environ[k] = "1"
    return saved


def _restore_env(saved):
    for k, v in saved.items():
        if v is None:
            os.environ.pop(k, None)
        else:
            os.environ[k] = v


def _time_cpu_all_cores(kind: str, budget_s: float):
    """One single-threaded process per host core (a spawned pool: safe after CUDA
    initialization), each timing its own chunks of the headline workload for
    about budget_s seconds.  Returns (symbols/s over the slowest worker's time,
    subcarriers done, workers)."""
    import multiprocessing as mp
    workers = os.cpu_count() or 1
    saved = _single_thread_env()
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            res = pool.map(_cpu_worker, [(kind, budget_s, 99 + i) for i in range(workers)])
    finally:
        _restore_env(saved)
    done = sum(r[0] for r in res)
    spent = max(r[1] for r in res)
    w = WORKLOAD
    return 2 * w["U"] * w["n_sym"] * done / spent, done, workers


def run_reference(args, rank, world):
    """The oracle as it stands on the host cores: one single-threaded process per
    core (a spawned pool, created once); each step every worker times oracle
    chunks of the workload (PD and FD with their LLRs) for a bounded slice of
    time (at least one chunk), so that the whole --steps K --warmup W run takes
    about two minutes."""
    if rank != 0:
        return
    import multiprocessing as mp
    workers = os.cpu_count() or 1
    budget = max(0.01, min(30.0, 120.0 / max(1, args.steps + args.warmup)))
    saved = _single_thread_env()
    rates, samples, spent_all = [], 0, 0.0
    w = WORKLOAD
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            for step in range(args.warmup + args.steps):
                res = pool.map(_cpu_worker, [("oracle", budget, 99 + i + 1000 * step) for i in range(workers)])
                if step < args.warmup:
                    continue
                done = sum(r[0] for r in res)
                spent = max(r[1] for r in res)
                rates.append(2 * w["U"] * w["n_sym"] * done / spent)
                samples += done
                spent_all += spent
    finally:
        _restore_env(saved)
    value = statistics.median(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * 2 * w["U"] * w["n_sym"] * w["n_sc"] / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "B=256 U=16 C=8 1200sc x 14sym 16-QAM Rayleigh 10dB, PD+FD, LLRs",
                   "sample": f"FP64 oracle (z, sigma^2 and LLRs) on {ORACLE_CHUNK}-subcarrier chunks, {workers} "
                             f"single-threaded processes, ~{budget:.2f} s of oracle work per process per timed step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle",
                         "sample": f"{samples} subcarriers over {args.steps} steps ({spent_all:.1f} s of oracle "
                                   f"time per process)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _errors(g, o):
    """[max over subcarriers of ||g - o|| / ||o||, max over entries of |g - o| / max(|o|, rms of the
    subcarrier)] -- the two measures of the parity tests."""
    import numpy as np
    g = np.asarray(g).reshape(g.shape[0], -1).astype(np.complex128)
    o = np.asarray(o).reshape(o.shape[0], -1).astype(np.complex128)
    nrm = np.linalg.norm(g - o, axis=1) / np.maximum(np.linalg.norm(o, axis=1), 1e-30)
    rms = np.sqrt(np.mean(np.abs(o) ** 2, axis=1, keepdims=True))
    ent = np.abs(g - o) / np.maximum(np.abs(o), np.maximum(rms, 1e-30))
    return [float(nrm.max()), float(ent.max())]


def _accuracy(p, outs, idx, archs):
    """Errors of the outputs of input set 0 against the FP64 oracle on sampled subcarriers."""
    import numpy as np
    from oracle import lmmse
    res = {}
    for a in archs:
        f = lmmse.equalize_pd if a == 0 else lmmse.equalize_fd
        o = f(p.H[idx], p.y[idx], float(np.float32(p.N0)), p.Es, p.C, "unbiased")
        z = outs[a]["z"][idx].cpu().numpy()
        s2 = outs[a]["s2"][idx].cpu().numpy()
        res["pd" if a == 0 else "fd"] = {"z": _errors(z, o["z"]), "sigma2": _errors(s2, o["sigma2"])}
    return res


UNEVEN = dict(n_inst=4096, seed=77)


class Runner:
    """What every GPU leg shares: torch, the binding, the device, the rank layout."""

    def __init__(self, args, rank, world, local_rank):
        import torch

        from paper_1808_04473_gb300 import build as fbuild
        from paper_1808_04473_gb300 import ffeq
        self.args, self.rank, self.world = args, rank, world
        self.torch, self.ffeq = torch, ffeq
        torch.cuda.set_device(local_rank)
        self.local_rank = local_rank
        self.dev = torch.device("cuda", local_rank)
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl", device_id=self.dev)
        fbuild.build()
        ffeq.lib()
        self.PREC = {"fp32": ffeq.FP32, "tf32x3": ffeq.TF32X3, "bf16x3": ffeq.BF16X3, "fp16x3": ffeq.FP16X3}

    def barrier(self):
        if self.world > 1:
            import torch.distributed as dist
            dist.barrier()

    def rotating_sets(self, *arrays):
        """Device copies of the inputs, enough of them that the rotating working set
        exceeds 4x L2 (at least 2): every step reads cold inputs."""
        torch = self.torch
        nbytes = sum(a.nbytes for a in arrays)
        n_sets = max(2, -(-4 * L2_BYTES // nbytes))
        first = [torch.from_numpy(a).to(self.dev) for a in arrays]
        sets = [first] + [[t.clone() for t in first] for _ in range(n_sets - 1)]
        return [list(col) for col in zip(*sets)], n_sets, nbytes


def soak(replay, seconds: float, torch):
    """Replay step graphs for about `seconds` (untimed) so that the clock samples
    taken next to the timed region are under load."""
    t_end = time.perf_counter() + seconds
    i = 0
    while time.perf_counter() < t_end:
        for _ in range(16):
            replay(i)
            i += 1
        torch.cuda.synchronize()


STEP_SHAPES = ((7, 0), (6, 0), (5, 0), (4, 0), (2, 0), (1, 0))   # launch shapes tried together for a whole step
FUSED_SHAPE = 6          # the contraction and the solve in one launch (include/ffeq.h tuning)


def equalize_steps(R, shape, Hs, ys, N0, Es, *, precision, bits, K, warmup, equalizer=0, refine=0,
                   refine_fp64=0, pinned=None, breakdown=False, sampler=None, soak_s=0.0, concurrent=False,
                   tune_step=False, tune_schedule=False):
    """K steps of PD then FD equalization; each step is captured once per rotating
    input set as a CUDA graph (what a serving loop replays per frame) and the
    timed region replays K graphs, bracketed by CUDA events on the replay stream.
    Without refinement a step is the local-preprocessing kernel and the
    fusion / equalization kernel per architecture (the latter launched with
    programmatic dependent launch); with refinement it is ffeq_equalize per
    architecture.  breakdown: a separate pass replays graphs of one kernel each
    (that kernel alone, on the rotating input sets) for per-kernel device times.
    concurrent: PD and FD as two branches of the captured step (a second stream
    forked from and joined to the replay stream), so that one architecture's
    kernels can run while the other's hold fewer SMs.
    tune_step: after each plan's own autotuning, time the whole captured step for
    every pair of contraction shapes in STEP_SHAPES, sequential and concurrent,
    and keep the fastest (setup, outside the timed region): the best shape of a
    plan alone is not always the best one next to the other plan's kernels.
    tune_schedule: keep each plan's own tuning and choose only between the
    sequential and the concurrent step by timing both.
    Leaves the outputs of input set 0 in `outs`."""
    torch, ffeq, dev = R.torch, R.ffeq, R.dev
    B, U, C, n_sc, n_sym = shape
    iters = LAMA_ITERS if equalizer == ffeq.LAMA else 0
    archs = (ffeq.PD, ffeq.FD)
    plans = {a: ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=a, precision=R.PREC[precision], llr_bits=bits,
                                      refine=refine, refine_fp64=refine_fp64, equalizer=equalizer,
                                      lama_iters=iters) for a in archs}
    nb = {a: ffeq.ffeq_workspace_size(x) for a, x in plans.items()}
    ws = {a: torch.empty(max(nb[a], 16), dtype=torch.uint8, device=dev) for a in plans}
    s2_shape = (n_sc, n_sym, U) if equalizer == ffeq.LAMA else (n_sc, U)
    outs = {a: dict(z=torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=dev),
                    s2=torch.empty(s2_shape, dtype=torch.float32, device=dev),
                    llr=torch.empty((n_sc, n_sym, U, bits), dtype=torch.float32, device=dev) if bits else None)
            for a in archs}
    n_sets = len(Hs)
    stream = torch.cuda.current_stream(dev)
    for a in plans:                  # launch shape chosen by timing (outside the timed region)
        o = outs[a]
        if pinned:
            ffeq.ffeq_plan_set_tuning(plans[a], pinned[2 * a:2 * a + 2])
        else:
            # Over the rotating input sets: every timed call reads cold inputs, as the steps do.
            ffeq.ffeq_plan_autotune_sets(plans[a], Hs, ys, N0, Es, o["z"], o["s2"], o["llr"], None, ws[a], nb[a],
                                         stream, 2 * n_sets)
    cap = torch.cuda.Stream(dev)
    split = refine == 0

    def launch(a, i, which, stream=None):
        # "step": the whole equalization call (one fused launch, or the
        # contraction then the solve kernel); "local" / "fuse": one stage alone.
        o = outs[a]
        st = cap if stream is None else stream
        if not split or which == "step":
            ffeq.ffeq_equalize(plans[a], Hs[i], ys[i], N0, Es, o["z"], o["s2"], o["llr"], None, ws[a], nb[a], st)
        elif which == "local":
            ffeq.ffeq_local_preprocess(plans[a], Hs[i], ys[i], ws[a], nb[a], st)
        else:
            ffeq.ffeq_fuse_equalize(plans[a], ws[a], nb[a], N0, Es, o["z"], o["s2"], o["llr"], None, st)

    def capture(fn):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            fn()
        return g

    cap2 = torch.cuda.Stream(dev)

    def whole_step(i):
        if not concurrent:
            for a in archs:
                launch(a, i, "step")
            return
        fork, join = torch.cuda.Event(), torch.cuda.Event()
        fork.record(cap)
        cap2.wait_event(fork)
        launch(archs[0], i, "step")
        launch(archs[1], i, "step", cap2)     # the second architecture on the forked stream
        join.record(cap2)
        cap.wait_event(join)

    def time_steps(graphs, reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(cap):
            for i in range(n_sets):
                graphs[i].replay()
            e0.record(cap)
            for k in range(reps):
                graphs[k % n_sets].replay()
            e1.record(cap)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    torch.cuda.synchronize()
    with torch.cuda.stream(cap):
        for i in range(2):           # eager warm-up before capture
            for a in archs:
                launch(a, i % n_sets, "step")
    cap.synchronize()
    schedule = {"concurrent": concurrent}
    if tune_step and not pinned:
        best = None
        for tp in STEP_SHAPES:
            for tf in STEP_SHAPES:
                try:
                    ffeq.ffeq_plan_set_tuning(plans[archs[0]], tp)
                    ffeq.ffeq_plan_set_tuning(plans[archs[1]], tf)
                except ffeq.FfeqError:
                    continue
                with torch.cuda.stream(cap):
                    for a in archs:          # first use of a shape outside capture
                        launch(a, 0, "step")
                for conc in (False, True):
                    concurrent = conc
                    gs = [capture(lambda i=i: whole_step(i)) for i in range(n_sets)]
                    t = time_steps(gs, 4 * n_sets)
                    del gs
                    if best is None or t < best[0]:
                        best = (t, tp, tf, conc)
        _, tp, tf, concurrent = best
        ffeq.ffeq_plan_set_tuning(plans[archs[0]], tp)
        ffeq.ffeq_plan_set_tuning(plans[archs[1]], tf)
        schedule = {"concurrent": concurrent, "chosen_by": "whole-step timing over contraction shape pairs"}
        with torch.cuda.stream(cap):
            for a in archs:
                launch(a, 0, "step")
        cap.synchronize()
    elif tune_schedule and not pinned:
        best = None
        for conc in (False, True):
            concurrent = conc
            gs = [capture(lambda i=i: whole_step(i)) for i in range(n_sets)]
            t = time_steps(gs, 2 * n_sets)
            del gs
            if best is None or t < best[0]:
                best = (t, conc)
        concurrent = best[1]
        schedule = {"concurrent": concurrent, "chosen_by": "whole-step timing, sequential against concurrent"}
    steps = [capture(lambda i=i: whole_step(i)) for i in range(n_sets)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if sampler is not None:          # clocks: sampled from the load phase through the timed region
        sampler.__enter__()
    with torch.cuda.stream(cap):
        if soak_s > 0:
            soak(lambda i: steps[i % n_sets].replay(), soak_s, torch)
        for i in range(warmup):
            steps[i % n_sets].replay()
    torch.cuda.synchronize()
    R.barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")      # profiling filter: ncu --nvtx --nvtx-include "timed/"
    with torch.cuda.stream(cap):
        start.record(cap)
        for k in range(K):
            steps[k % n_sets].replay()
        end.record(cap)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.__exit__(None, None, None)
    R.barrier()
    ms = start.elapsed_time(end)
    kern = {}
    fused = {a: ffeq.ffeq_plan_get_tuning(plans[a])[0] == FUSED_SHAPE for a in archs}
    if breakdown and split:
        # Each stage alone (with a fused plan, "local" and "fuse" are the separate
        # kernels the fused launch replaces, its contraction with a ring of 2),
        # and a fused plan's one launch.
        Kb = max(8, min(K, 200))
        items = []
        for a, tag in ((ffeq.PD, "pd"), (ffeq.FD, "fd")):
            items += [(f"{tag}_local", a, "local"), (f"{tag}_fuse", a, "fuse")]
            if fused[a]:
                items.append((f"{tag}_fused", a, "step"))
        def both_locals(i):
            # The two contractions as the concurrent step runs them (two graph
            # branches), without the solves: the Gram stage of the step.
            fork, join = torch.cuda.Event(), torch.cuda.Event()
            fork.record(cap)
            cap2.wait_event(fork)
            launch(archs[0], i, "local")
            launch(archs[1], i, "local", cap2)
            join.record(cap2)
            cap.wait_event(join)

        if concurrent:
            items.append(("gram_stage_concurrent", None, "both"))
        for name, a, which in items:
            gs = [capture(lambda i=i: both_locals(i) if which == "both" else launch(a, i, which))
                  for i in range(n_sets)]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(cap):
                for i in range(n_sets):
                    gs[i].replay()
                e0.record(cap)
                for k in range(Kb):
                    gs[k % n_sets].replay()
                e1.record(cap)
            torch.cuda.synchronize()
            kern[name] = e0.elapsed_time(e1) / Kb
            del gs
    # Leave the outputs of input set 0 (the accuracy checks read them).
    with torch.cuda.stream(cap):
        steps[0].replay()
    torch.cuda.synchronize()
    del steps
    if R.world > 1:
        ms = max_over_ranks(ms, dev)
    assert ffeq.ffeq_device_status() == 0
    for a in outs:
        assert torch.isfinite(torch.view_as_real(outs[a]["z"])).all().item()
    launches = sum(1 if fused[a] else (2 if split else 1) for a in archs)   # per step, without refinement
    return dict(ms=ms, kern=kern, plans=plans, outs=outs, schedule=schedule, fused=fused, launches=launches)


def e2e_steps(R, plans, p, shape, bits, K):
    """End to end from pinned host memory through the public device entry point.

    One step takes one received block (H, y) from pinned host memory to the GPU
    (one upload: PD and FD equalize the same block), runs ffeq_equalize for both
    architectures with the tuning the device-timed step uses, and reads z,
    sigma^2 and the LLRs of both back into pinned host memory.  Two lanes
    (device inputs, workspaces and outputs, one stream each) alternate over the
    steps, so the upload of step k + 1 overlaps the kernels and the read-back of
    step k, as a receiver streaming blocks would run it; every step's copies lie
    inside the timed region (host clock, synchronized on both sides).  Two host
    input sets alternate.  The last two steps' host outputs are checked bit for
    bit against ffeq_equalize on device copies of the same inputs."""
    torch, ffeq, dev = R.torch, R.ffeq, R.dev
    B, U, C, n_sc, n_sym = shape
    Hh = [torch.from_numpy(p.H).pin_memory() for _ in range(2)]
    yh = [torch.from_numpy(p.y).pin_memory() for _ in range(2)]
    Hh[1].mul_(-1)               # a second block (the same channel and signal, negated)
    yh[1].mul_(-1)
    archs = (ffeq.PD, ffeq.FD)
    nb = {a: ffeq.ffeq_workspace_size(plans[a]) for a in archs}

    def outs(pin):
        mk = (lambda *sh, dt: torch.empty(sh, dtype=dt).pin_memory()) if pin else \
             (lambda *sh, dt: torch.empty(sh, dtype=dt, device=dev))
        return {a: dict(z=mk(n_sc, n_sym, U, dt=torch.complex64), s2=mk(n_sc, U, dt=torch.float32),
                        llr=mk(n_sc, n_sym, U, bits, dt=torch.float32)) for a in archs}

    lanes = [dict(st=torch.cuda.Stream(dev), H=torch.empty_like(Hh[0], device=dev),
                  y=torch.empty_like(yh[0], device=dev),
                  ws={a: torch.empty(max(nb[a], 16), dtype=torch.uint8, device=dev) for a in archs},
                  dout=outs(False), hout=outs(True)) for _ in range(2)]

    def step(k):
        ln = lanes[k % 2]
        st = ln["st"]
        with torch.cuda.stream(st):
            ln["H"].copy_(Hh[k % 2], non_blocking=True)
            ln["y"].copy_(yh[k % 2], non_blocking=True)
            for a in archs:
                o = ln["dout"][a]
                ffeq.ffeq_equalize(plans[a], ln["H"], ln["y"], p.N0, p.Es, o["z"], o["s2"], o["llr"], None,
                                   ln["ws"][a], nb[a], st)
            for a in archs:
                for key in ("z", "s2", "llr"):
                    ln["hout"][a][key].copy_(ln["dout"][a][key], non_blocking=True)

    for k in range(4):
        step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(K):
        step(k)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / K
    assert ffeq.ffeq_device_status() == 0
    # The host outputs of the last two steps against a plain device call on the same block.
    for k in (K - 2, K - 1):
        ln = lanes[k % 2]
        ref = outs(False)
        Hd, yd = Hh[k % 2].to(dev), yh[k % 2].to(dev)
        for a in archs:
            ffeq.ffeq_equalize(plans[a], Hd, yd, p.N0, p.Es, ref[a]["z"], ref[a]["s2"], ref[a]["llr"], None,
                               ln["ws"][a], nb[a], torch.cuda.current_stream(dev))
        torch.cuda.synchronize()
        for a in archs:
            for key in ("z", "s2", "llr"):
                got, want = ln["hout"][a][key], ref[a][key].cpu()
                if got.is_complex():
                    got, want = torch.view_as_real(got), torch.view_as_real(want)
                assert torch.equal(got.view(torch.int32), want.view(torch.int32)), (a, key)
    in_bytes = p.H.nbytes + p.y.nbytes
    out_bytes = 2 * (n_sc * n_sym * U * 8 + n_sc * U * 4 + n_sc * n_sym * U * bits * 4)
    return {"value": R.world * 2 * U * n_sc * n_sym / dt, "unit": UNIT, "steps": K, "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": in_bytes, "d2h_bytes_per_step": out_bytes,
            "path": "pinned host block -> device (one upload, both architectures), ffeq_equalize for PD and FD, "
                    "outputs -> pinned host; two lanes on two streams so that one step's upload overlaps the "
                    "previous step's kernels; host clock around the steps, synchronized on both sides; outputs "
                    "checked bit for bit against the device entry point"}


def uneven_line(R, K, warmup, precision, sampler=None):
    """One step = PD and FD equalization of 4096 instances of uneven size (U 4..32,
    B 64/128/256, C 1..16, 1..14 symbols, 5..20 dB, 16-QAM) through the batch
    ABI, replayed from one CUDA graph per input set; inputs rotate over sets
    larger than L2 in total."""
    import numpy as np
    torch, ffeq, dev = R.torch, R.ffeq, R.dev
    from paper_1808_04473_gb300 import synth
    ps = synth.make_uneven(UNEVEN["n_inst"], seed=UNEVEN["seed"] + R.rank)
    specs = [(p.B, p.U, p.C, p.n_sc, p.n_sym, p.N0, p.Es) for p in ps]
    symbols = sum(p.U * p.n_sym * p.n_sc for p in ps)
    stream = torch.cuda.Stream(dev)
    runs = {}
    for a in (ffeq.PD, ffeq.FD):
        cfg, inst = ffeq.pack_batch(specs, arch=a, precision=R.PREC[precision], llr_bits=4, with_info=False)
        H = np.zeros(cfg.h_elems, np.complex64)
        y = np.zeros(cfg.y_elems, np.complex64)
        for p, it in zip(ps, inst):
            H[it.h_off:it.h_off + p.H.size] = p.H.ravel()
            y[it.y_off:it.y_off + p.y.size] = p.y.ravel()
        b = ffeq.ffeq_batch_create(cfg, inst)
        nb = ffeq.ffeq_batch_workspace_size(b)
        runs[a] = dict(b=b, nb=nb, ws=torch.empty(nb, dtype=torch.uint8, device=dev),
                       H=torch.from_numpy(H).to(dev), y=torch.from_numpy(y).to(dev),
                       z=torch.empty(cfg.z_elems, dtype=torch.complex64, device=dev),
                       s2=torch.empty(cfg.sigma2_elems, dtype=torch.float32, device=dev),
                       llr=torch.empty(cfg.llr_elems, dtype=torch.float32, device=dev), cfg=cfg)
    in_bytes = sum(r["H"].numel() * 8 + r["y"].numel() * 8 for r in runs.values()) // 2
    n_sets = max(2, -(-4 * L2_BYTES // (2 * in_bytes)))
    for r in runs.values():
        r["Hs"] = [r["H"]] + [r["H"].clone() for _ in range(n_sets - 1)]
        r["ys"] = [r["y"]] + [r["y"].clone() for _ in range(n_sets - 1)]
    with torch.cuda.stream(stream):
        for r in runs.values():
            ffeq.ffeq_batch_autotune(r["b"], r["H"], r["y"], r["z"], r["s2"], r["llr"], None, r["ws"], r["nb"],
                                     stream, 5)
        for i in range(n_sets):
            for r in runs.values():          # warm-up (and table upload) outside capture
                ffeq.ffeq_batch_equalize(r["b"], r["Hs"][i], r["ys"][i], r["z"], r["s2"], r["llr"], None, r["ws"],
                                         r["nb"], stream)
        stream.synchronize()
        stream2 = torch.cuda.Stream(dev)

        def step(i, concurrent):
            # PD then FD on one stream, or the two batches as two graph branches
            # (each batch forks its own groups onto its side streams).
            rs = list(runs.values())
            if not concurrent:
                for r in rs:
                    ffeq.ffeq_batch_equalize(r["b"], r["Hs"][i], r["ys"][i], r["z"], r["s2"], r["llr"], None,
                                             r["ws"], r["nb"], stream)
                return
            fork, join = torch.cuda.Event(), torch.cuda.Event()
            fork.record(stream)
            stream2.wait_event(fork)
            for r, st in ((rs[0], stream), (rs[1], stream2)):
                ffeq.ffeq_batch_equalize(r["b"], r["Hs"][i], r["ys"][i], r["z"], r["s2"], r["llr"], None,
                                         r["ws"], r["nb"], st)
            join.record(stream2)
            stream.wait_event(join)

        def capture_all(concurrent):
            gs = []
            for i in range(n_sets):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    step(i, concurrent)
                gs.append(g)
            return gs

        # Schedule chosen by timing both (setup, outside the timed region).
        best = None
        for conc in (False, True):
            gs = capture_all(conc)
            for i in range(n_sets):
                gs[i].replay()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for k in range(4 * n_sets):
                gs[k % n_sets].replay()
            e1.record(stream)
            stream.synchronize()
            t = e0.elapsed_time(e1)
            if best is None or t < best[0]:
                best = (t, conc, gs)
            else:
                del gs
        _, concurrent, graphs = best
        if sampler is not None:
            sampler.__enter__()
            soak(lambda i: graphs[i % n_sets].replay(), 1.0, torch)
        for i in range(warmup):
            graphs[i % n_sets].replay()
        stream.synchronize()
        R.barrier()
        torch.cuda.synchronize()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed")
        start.record(stream)
        for k in range(K):
            graphs[k % n_sets].replay()
        end.record(stream)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.__exit__(None, None, None)
    ms = start.elapsed_time(end)
    if R.world > 1:
        ms = max_over_ranks(ms, dev)
    assert ffeq.ffeq_device_status() == 0
    value = job_rate(2 * symbols, R.world, K, ms)
    out_bytes = sum(r["z"].numel() * 8 + r["s2"].numel() * 4 + r["llr"].numel() * 4 for r in runs.values())
    alg = 2 * in_bytes + out_bytes
    hbm_peak, peak_src = _peaks()
    achieved = alg / (ms / K * 1e-3) / 1e9
    launches = sum(2 * ffeq.ffeq_batch_groups(r["b"]) for r in runs.values())   # kernels (the memset is not one)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": R.world, "steps": K, "warmup": warmup,
        "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": DTYPE[precision], "data": "synthetic",
        "config": {"workload": f"uneven batch: {UNEVEN['n_inst']} instances, U 4..32, B 64/128/256, C 1..16, "
                               "1..14 sym, 5..20 dB, 16-QAM, PD+FD, LLRs, CUDA-graph replay",
                   "precision": precision,
                   "l2": f"rotating {n_sets} input sets ({n_sets * in_bytes / 2**20:.0f} MiB > L2)",
                   "parallelism": f"replicas x{R.world}"},
        "tuning": {("pd" if a == ffeq.PD else "fd"): ffeq.ffeq_batch_get_tuning(r["b"]) for a, r in runs.items()},
        "schedule": {"mode": "concurrent" if concurrent else "sequential",
                     "chosen_by": "timing PD and FD in sequence and as two graph branches"},
        "roofline": {"kernel": "whole step (memset + per-group gram_kernel and solve_fuse_kernel)", "bound": "hbm",
                     "achieved": achieved, "peak": hbm_peak, "peak_source": f"{peak_src} (STREAM-style copy)",
                     "unit": "GB/s", "frac": achieved / hbm_peak, "traffic": None,
                     "algorithmic_bytes_per_step": alg},
        "gpu_launches": launches * K,
    }
    return line


def run_correlated(R, K, warmup):
    """The correlated workload: B=256, U=32, C=16 (S=16 < U), 3300 x 14, 64-QAM,
    receive correlation r = 0.7, 15 dB.  One step = PD + FD.  Arms: FP32 and FP16x3
    preprocessing without refinement, and each with one refinement step whose
    residual is FP64 for the systems with condition estimate > 1e4 (the
    configuration); each arm's errors against the FP64 oracle on 8 sampled
    subcarriers."""
    import numpy as np
    from paper_1808_04473_gb300 import synth
    w = CORRELATED
    shape = (w["B"], w["U"], w["C"], w["n_sc"], w["n_sym"])
    p = synth.make_problem(*shape, snr_db=w["snr_db"], bits=w["bits"], seed=3300 + R.rank, corr_r=w["corr_r"])
    (Hs, ys), n_sets, in_bytes = R.rotating_sets(p.H, p.y)
    idx = np.linspace(0, w["n_sc"] - 1, 8).astype(int)
    symbols = 2 * w["U"] * w["n_sc"] * w["n_sym"]
    arms = {}
    for name, prec, refine in (("fp32", "fp32", 0), ("fp16x3", "fp16x3", 0),
                               ("fp32+refine1(fp64>1e4)", "fp32", 1), ("fp16x3+refine1(fp64>1e4)", "fp16x3", 1)):
        r = equalize_steps(R, shape, Hs, ys, p.N0, p.Es, precision=prec, bits=w["bits"], K=K, warmup=warmup,
                           refine=refine, refine_fp64=1 if refine else 0, tune_schedule=True)
        arms[name] = {"value": job_rate(symbols, R.world, K, r["ms"]), "ms_per_step": r["ms"] / K, "steps": K,
                      "schedule": r["schedule"],
                      "error_vs_oracle": _accuracy(p, r["outs"], idx, (0, 1)) if R.rank == 0 else None}
        del r
    return {"workload": "B=256 U=32 C=16 3300sc x 14sym 64-QAM, exponential correlation r=0.7, 15dB, PD+FD, LLRs",
            "unit": UNIT, "l2": f"rotating {n_sets} input sets ({n_sets * in_bytes / 2**20:.0f} MiB > L2)",
            "error_metric": "[max over 8 sampled subcarriers of ||x - x_oracle|| / ||x_oracle||, max entry "
                            "|x - x_oracle| / max(|x_oracle|, rms of its subcarrier)]",
            "arms": arms}


def lama_flops(U, bits, T):
    """Algorithmic FP32 flops of LAMA per received vector and cluster: T products
    G s of 8 U^2 flops and T - 1 denoiser steps of U (2 * 2^(b/2) * 6 + 10) flops
    (per PAM level and axis: distance, exponent scaling, weight sums, first and
    second moments; then the moments and the update)."""
    levels = 2 ** (bits // 2)
    return T * 8 * U * U + (T - 1) * U * (2 * levels * 6 + 10)


def lama_roofline(kern, U, C, n_sc, n_sym, bits):
    """FP32 ALU roofline of the PD and FD LAMA kernels from their breakdown times."""
    roof = {}
    for tag, Ceff in (("pd", 1), ("fd", C)):
        flops = lama_flops(U, bits, LAMA_ITERS) * n_sc * Ceff * n_sym
        ach = flops / (kern[f"{tag}_fuse"] * 1e-3) / 1e12
        roof[tag] = {"kernel": f"lama_kernel ({tag.upper()}, T = {LAMA_ITERS})", "bound": "alu", "achieved": ach,
                     "peak": FP32_ALU_TFLOPS, "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz",
                     "unit": "TFLOP/s", "frac": ach / FP32_ALU_TFLOPS, "algorithmic_flops_per_launch": flops,
                     "kernel_ms": kern[f"{tag}_fuse"]}
    return roof


def run_lama(R, K, warmup, pinned):
    """The headline shape with LAMA (Sec. III-B, LAMA_ITERS iterations) in place
    of L-MMSE: the step the default line's `equalizers.lama` key times, as a line
    of its own with the LAMA kernels' FP32 ALU roofline (a profiling target)."""
    import numpy as np
    from paper_1808_04473_gb300 import synth
    ffeq = R.ffeq
    w = WORKLOAD
    B, U, C, n_sc, n_sym, bits = w["B"], w["U"], w["C"], w["n_sc"], w["n_sym"], w["bits"]
    shape = (B, U, C, n_sc, n_sym)
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=w["snr_db"], bits=bits, seed=12345 + R.rank)
    (Hs, ys), n_sets, in_bytes = R.rotating_sets(p.H, p.y)
    r = equalize_steps(R, shape, Hs, ys, p.N0, p.Es, precision="bf16x3", bits=bits, K=K, warmup=warmup,
                       equalizer=ffeq.LAMA, pinned=pinned, breakdown=True, concurrent=True,
                       tune_step=pinned is None)
    kern = r["kern"]
    roof = lama_roofline(kern, U, C, n_sc, n_sym, bits)
    symbols = 2 * U * n_sc * n_sym
    return {"workload": f"B={B} U={U} C={C} {n_sc}sc x {n_sym}sym 16-QAM Rayleigh 10dB, PD+FD LAMA "
                        f"(T = {LAMA_ITERS}), LLRs",
            "value": job_rate(symbols, R.world, K, r["ms"]), "unit": UNIT, "ms_per_step": r["ms"] / K,
            "steps": K, "l2": f"rotating {n_sets} input sets ({n_sets * in_bytes / 2**20:.0f} MiB > L2)",
            "kernels_ms": kern, "schedule": r["schedule"],
            "tuning": {("pd" if a == ffeq.PD else "fd"): list(ffeq.ffeq_plan_get_tuning(pl))
                       for a, pl in r["plans"].items()},
            "roofline": roof}


def run_training(R, K, warmup):
    """One training step of the differentiable FD form: ffeq_fd_train_forward and
    ffeq_fd_train_backward on B=128, U=16, C=8, 8 draws x 1024 subcarriers, QPSK,
    10 dB (one symbol per draw), with per-cluster rho_c = N0/Es and fusion weights
    1/C; the upstream gradient dL/dz is that of the MSE against the sent symbols,
    formed once from the first forward pass (an input of the adjoint)."""
    import numpy as np
    torch, ffeq, dev = R.torch, R.ffeq, R.dev
    from paper_1808_04473_gb300 import synth
    w = TRAINING
    B, U, C, n_sc, n_sym = w["B"], w["U"], w["C"], w["n_sc"], w["n_sym"]
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=w["snr_db"], bits=w["bits"], seed=1024 + R.rank)
    (Hs, ys), n_sets, in_bytes = R.rotating_sets(p.H, p.y)
    rho = torch.full((C,), p.N0 / p.Es, dtype=torch.float32, device=dev)
    nu = torch.full((C, U), 1.0 / C, dtype=torch.float32, device=dev)
    plan = ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ffeq.FD)
    nb = ffeq.ffeq_fd_train_workspace_size(plan)
    ws = torch.empty(nb, dtype=torch.uint8, device=dev)
    z = torch.empty((n_sc, n_sym, U), dtype=torch.complex64, device=dev)
    # The contraction shape of the plan, chosen by timing (setup, untimed).
    s2t = torch.empty((n_sc, U), dtype=torch.float32, device=dev)
    ffeq.ffeq_plan_autotune_sets(plan, Hs, ys, p.N0, p.Es, z, s2t, None, None, ws, nb,
                                 torch.cuda.current_stream(dev), 2 * n_sets)
    gH, gy = torch.empty_like(Hs[0]), torch.empty_like(ys[0])
    grho, gnu = torch.empty_like(rho), torch.empty_like(nu)
    cap = torch.cuda.Stream(dev)
    with torch.cuda.stream(cap):
        ffeq.ffeq_fd_train_forward(plan, Hs[0], ys[0], rho, nu, z, ws, nb, cap)
    cap.synchronize()
    s = torch.from_numpy(p.s.astype(np.complex64)).to(dev)
    gz = (2.0 / z.numel()) * (z - s)

    def step(i):
        ffeq.ffeq_fd_train_forward(plan, Hs[i], ys[i], rho, nu, z, ws, nb, cap)
        ffeq.ffeq_fd_train_backward(plan, Hs[i], ys[i], rho, nu, gz, gH, gy, grho, gnu, ws, nb, cap)

    with torch.cuda.stream(cap):
        for i in range(2):
            step(i % n_sets)
    cap.synchronize()
    graphs = []
    for i in range(n_sets):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            step(i)
        graphs.append(g)
    with torch.cuda.stream(cap):
        for i in range(warmup):
            graphs[i % n_sets].replay()
    torch.cuda.synchronize()
    R.barrier()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(cap):
        start.record(cap)
        for k in range(K):
            graphs[k % n_sets].replay()
        end.record(cap)
        graphs[0].replay()                   # leave the outputs of input set 0
    torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    if R.world > 1:
        ms = max_over_ranks(ms, dev)
    assert ffeq.ffeq_device_status() == 0
    out = {"workload": "differentiable FD, B=128 U=16 C=8, 8 draws x 1024 subcarriers x 1 sym, QPSK, 10dB: "
                       "forward + adjoint (dL/dH, dL/dy, dL/drho_c, dL/dnu)",
           "tuning": list(ffeq.ffeq_plan_get_tuning(plan)),
           "value": job_rate(U * n_sc * n_sym, R.world, K, ms), "unit": UNIT, "ms_per_step": ms / K, "steps": K,
           "l2": f"rotating {n_sets} input sets ({n_sets * in_bytes / 2**20:.0f} MiB > L2)"}
    # HBM roofline of the step: forward reads H, y and writes z; the adjoint reads
    # H, y, dL/dz and writes dL/dH, dL/dy (complex64).
    alg = n_sc * (24 * (B * U + B * n_sym) + 24 * U * n_sym)
    hbm_peak, peak_src = _peaks()
    achieved = alg / (ms / K * 1e-3) / 1e9
    out["roofline"] = {"kernel": "whole step (contraction, train_forward, adjoint kernels)", "bound": "hbm",
                       "achieved": achieved, "peak": hbm_peak, "peak_source": f"{peak_src} (STREAM-style copy)",
                       "unit": "GB/s", "frac": achieved / hbm_peak, "algorithmic_bytes_per_step": alg}
    # The FD estimate with the paper's optimal weights (ffeq_equalize) and its adjoint
    # through the weight rule (ffeq_fd_optimal_backward), the same upstream gradient.
    oplan = ffeq.ffeq_plan_create(B, U, C, n_sc, n_sym, arch=ffeq.FD)
    onb = ffeq.ffeq_workspace_size(oplan)
    ows = torch.empty(onb, dtype=torch.uint8, device=dev)
    bnb = ffeq.ffeq_fd_optimal_workspace_size(oplan)
    bws = torch.empty(bnb, dtype=torch.uint8, device=dev)
    zo = torch.empty_like(z)
    s2o = torch.empty((n_sc, U), dtype=torch.float32, device=dev)
    ffeq.ffeq_plan_set_tuning(oplan, ffeq.ffeq_plan_get_tuning(plan))

    def ostep(i):
        ffeq.ffeq_equalize(oplan, Hs[i], ys[i], p.N0, p.Es, zo, s2o, None, None, ows, onb, cap)
        ffeq.ffeq_fd_optimal_backward(oplan, Hs[i], ys[i], p.N0, p.Es, gz, gH, gy, bws, bnb, cap)

    with torch.cuda.stream(cap):
        for i in range(2):
            ostep(i % n_sets)
    cap.synchronize()
    ographs = []
    for i in range(n_sets):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=cap):
            ostep(i)
        ographs.append(g)
    with torch.cuda.stream(cap):
        for i in range(warmup):
            ographs[i % n_sets].replay()
    torch.cuda.synchronize()
    R.barrier()
    with torch.cuda.stream(cap):
        start.record(cap)
        for k in range(K):
            ographs[k % n_sets].replay()
        end.record(cap)
    torch.cuda.synchronize()
    oms = start.elapsed_time(end)
    if R.world > 1:
        oms = max_over_ranks(oms, dev)
    assert ffeq.ffeq_device_status() == 0
    out["optimal_weights"] = {
        "step": "ffeq_equalize (FD, Lemma 1 weights) + ffeq_fd_optimal_backward (dL/dH, dL/dy through the "
                "weight rule)", "value": job_rate(U * n_sc * n_sym, R.world, K, oms), "unit": UNIT,
        "ms_per_step": oms / K, "steps": K}
    with torch.cuda.stream(cap):
        graphs[0].replay()                   # leave the free-weight outputs of input set 0
    torch.cuda.synchronize()
    if R.rank == 0:
        from oracle import adjoint
        idx = np.linspace(0, n_sc - 1, 8).astype(int)
        r64 = np.full(C, p.N0 / p.Es)
        n64 = np.full((C, U), 1.0 / C)
        z0, _ = adjoint.fd_train_forward(p.H[idx], p.y[idx], r64.astype(np.float32).astype(np.float64),
                                         n64.astype(np.float32).astype(np.float64))
        gzs = gz[idx].cpu().numpy().astype(np.complex128)
        oH, oy, _, _ = adjoint.fd_train_backward(p.H[idx], p.y[idx], r64.astype(np.float32).astype(np.float64),
                                                 n64.astype(np.float32).astype(np.float64), gzs)
        out["error_vs_oracle"] = {"z": _errors(z[idx].cpu().numpy(), z0), "gH": _errors(gH[idx].cpu().numpy(), oH),
                                  "gy": _errors(gy[idx].cpu().numpy(), oy), "subcarriers": len(idx)}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ffeq", choices=["ffeq", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline step only (no FP32 comparison, equalizer variants, correlated, training or "
                         "uneven lines)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--concurrent", type=int, default=0,
                    help="1: PD and FD as two concurrent branches of each captured step")
    ap.add_argument("--precision", default="bf16x3", choices=PRECISIONS,
                    help="arithmetic of the local preprocessing (solve and fusion are FP32)")
    ap.add_argument("--tuning", default=None,
                    help="pin the contraction shapes instead of autotuning: PD_SHAPE,PD_STAGES,FD_SHAPE,FD_STAGES "
                         "(values of ffeq_plan_set_tuning; for reproducible profiles)")
    ap.add_argument("--workload", default="ofdm", choices=["ofdm", "uneven", "correlated", "training", "lama"],
                    help="ofdm: the headline B=256 U=16 C=8 1200x14 step (other workloads as extra keys); "
                         "uneven / correlated / training / lama: that workload's line alone")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    R = Runner(args, rank, world, local_rank)
    if args.workload != "ofdm":
        if args.workload == "uneven":
            line = uneven_line(R, args.steps, args.warmup, args.precision, ClockSampler(local_rank))
        elif args.workload == "correlated":
            line = run_correlated(R, args.steps, args.warmup)
        elif args.workload == "lama":
            line = run_lama(R, args.steps, args.warmup,
                            [int(v) for v in args.tuning.split(",")] if args.tuning else None)
        else:
            line = run_training(R, args.steps, args.warmup)
        if rank == 0:
            print(json.dumps(line), flush=True)
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return

    import numpy as np
    torch, ffeq, dev = R.torch, R.ffeq, R.dev
    from paper_1808_04473_gb300 import synth

    w = WORKLOAD
    B, U, C, n_sc, n_sym, bits = w["B"], w["U"], w["C"], w["n_sc"], w["n_sym"], w["bits"]
    shape = (B, U, C, n_sc, n_sym)
    p = synth.make_problem(B, U, C, n_sc, n_sym, snr_db=w["snr_db"], bits=bits, seed=12345 + rank)
    (Hs, ys), n_sets, in_bytes = R.rotating_sets(p.H, p.y)
    pinned = [int(v) for v in args.tuning.split(",")] if args.tuning else None
    idx = np.linspace(0, n_sc - 1, 12).astype(int)
    do_cpu = rank == 0 and not args.no_cpu_baseline

    K = args.steps
    clk = ClockSampler(local_rank)
    head = equalize_steps(R, shape, Hs, ys, p.N0, p.Es, precision=args.precision, bits=bits, K=K,
                          warmup=args.warmup, pinned=pinned, breakdown=True, sampler=clk, soak_s=1.0,
                          concurrent=bool(args.concurrent), tune_step=not args.tuning)
    elapsed_ms, kern, plans, schedule = head["ms"], head["kern"], head["plans"], head["schedule"]
    fused, launches = head["fused"], head["launches"]
    accuracy = _accuracy(p, head["outs"], idx, (0, 1)) if do_cpu else None
    if accuracy is not None:
        accuracy["subcarriers"] = len(idx)
        accuracy["metric"] = ("[max over sampled subcarriers of ||x - x_oracle|| / ||x_oracle||, max entry "
                              "|x - x_oracle| / max(|x_oracle|, rms of its subcarrier)]")
    symbols_per_step = 2 * U * n_sc * n_sym
    value = job_rate(symbols_per_step, world, K, elapsed_ms)
    del head

    fp32_cmp = None
    if args.precision != "fp32" and not args.no_extras:
        Kc = max(5, K // 4)
        r32 = equalize_steps(R, shape, Hs, ys, p.N0, p.Es, precision="fp32", bits=bits, K=Kc, warmup=args.warmup,
                             breakdown=True, tune_step=True)
        fp32_cmp = {"value": job_rate(symbols_per_step, world, Kc, r32["ms"]), "ms_per_step": r32["ms"] / Kc,
                    "steps": Kc, "kernels_ms": r32["kern"], "schedule": r32["schedule"],
                    "tuning": {("pd" if a == ffeq.PD else "fd"): list(ffeq.ffeq_plan_get_tuning(pl))
                               for a, pl in r32["plans"].items()},
                    "error_vs_oracle": _accuracy(p, r32["outs"], idx, (0, 1)) if do_cpu else None}
        del r32

    # ---- the same step with the ZF and MRC equalizers of Sec. III-A and LAMA (Sec. III-B,
    # LAMA_ITERS iterations) in place of L-MMSE (same contraction)
    variants = {}
    if not args.tuning and not args.no_extras:
        Kv = max(5, K // 4)
        for name, eq in (("zf", ffeq.ZF), ("mrc", ffeq.MRC), ("lama", ffeq.LAMA)):
            rv = equalize_steps(R, shape, Hs, ys, p.N0, p.Es, precision=args.precision, bits=bits, K=Kv,
                                warmup=args.warmup, equalizer=eq, breakdown=True, tune_step=True)
            variants[name] = {"value": job_rate(symbols_per_step, world, Kv, rv["ms"]), "ms_per_step": rv["ms"] / Kv,
                              "steps": Kv, "kernels_ms": rv["kern"], "schedule": rv["schedule"]}
            if eq == ffeq.LAMA:
                variants[name]["roofline"] = lama_roofline(rv["kern"], U, C, n_sc, n_sym, bits)
            del rv

    # ---- end to end from pinned host memory (the headline e2e number), and through
    # the host-buffer entry point (context)
    e2e = e2e_steps(R, plans, p, shape, bits, max(3, min(K, 50)))
    stream = torch.cuda.current_stream(dev)
    Hh = torch.from_numpy(p.H).pin_memory()
    yh = torch.from_numpy(p.y).pin_memory()
    stage_bytes = max(ffeq.ffeq_host_staging_size(pl) for pl in plans.values())
    staging = torch.empty(stage_bytes, dtype=torch.uint8, device=dev)
    host_out = {a: dict(z=torch.empty((n_sc, n_sym, U), dtype=torch.complex64).pin_memory(),
                        s2=torch.empty((n_sc, U), dtype=torch.float32).pin_memory(),
                        llr=torch.empty((n_sc, n_sym, U, bits), dtype=torch.float32).pin_memory())
                for a in plans}

    def host_step():
        for a in (ffeq.PD, ffeq.FD):
            o = host_out[a]
            ffeq.ffeq_equalize_host(plans[a], Hh, yh, p.N0, p.Es, o["z"], o["s2"], o["llr"], None, staging,
                                    stage_bytes, stream)

    for _ in range(2):
        host_step()
    Ke = max(3, min(K, 20))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(Ke):
        host_step()
    host_s = (time.perf_counter() - t0) / Ke
    out_bytes = n_sc * n_sym * U * 8 + n_sc * U * 4 + n_sc * n_sym * U * bits * 4
    e2e_host_entry = {"value": world * symbols_per_step / host_s, "unit": UNIT, "steps": Ke,
                      "h2d_bytes_per_step": 2 * in_bytes, "d2h_bytes_per_step": 2 * out_bytes,
                      "path": "ffeq_equalize_host once per architecture: the kernels read H and y and write the "
                              "outputs in pinned host memory in place (each architecture reads the inputs)"}
    del staging, Hh, yh, host_out

    # ---- the other workloads (extra keys)
    extras = {}
    if world == 1 and not args.no_extras and not args.tuning:
        Kx = max(5, min(K // 10, 100))
        extras["correlated"] = run_correlated(R, Kx, args.warmup)
        extras["training"] = run_training(R, max(5, min(K // 10, 200)), args.warmup)
        u = uneven_line(R, max(5, min(K // 10, 200)), args.warmup, args.precision)
        extras["uneven"] = {k: u[k] for k in ("value", "unit", "ms_per_step", "steps", "config", "roofline",
                                              "tuning", "schedule")}

    # ---- roofline of the dominant kernel (and of the Gram stage)
    hbm_peak, peak_src = _peaks()
    traffic = _ncu_traffic()

    def gram_roof(name):
        alg = input_bytes(B, U, n_sc, n_sym)
        achieved = alg / (kern[name] * 1e-3) / 1e9
        if name.endswith("fused"):
            kname = (f"gram_ws_kernel<{args.precision}, fused> ({name[:2].upper()} contraction + solve + fusion "
                     f"+ LLRs, one launch)")
        else:
            kname = f"gram_kernel<{args.precision}> ({name[:2].upper()} local preprocessing)"
        return {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                "peak_source": f"{peak_src} (STREAM-style copy)", "unit": "GB/s", "frac": achieved / hbm_peak,
                "traffic": traffic.get(f"{args.precision}:{name}"), "algorithmic_bytes_per_launch": alg,
                "kernel_ms": kern[name]}

    def solve_roof(name):
        flops = solve_flops(U, n_sym, C if name.startswith("fd") else 1) * n_sc
        achieved = flops / (kern[name] * 1e-3) / 1e12
        return {"kernel": f"solve kernel ({name[:2].upper()} solve + fusion + LLRs)", "bound": "alu",
                "achieved": achieved, "peak": FP32_ALU_TFLOPS,
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz", "unit": "TFLOP/s",
                "frac": achieved / FP32_ALU_TFLOPS, "traffic": traffic.get(f"{args.precision}:{name}"),
                "algorithmic_flops_per_launch": flops, "kernel_ms": kern[name]}

    # The step's own kernels: a fused plan's one launch, else its two stages.
    step_kernels = []
    for tag, a in (("pd", ffeq.PD), ("fd", ffeq.FD)):
        step_kernels += [f"{tag}_fused"] if fused[a] else [f"{tag}_local", f"{tag}_fuse"]
    dom = max(step_kernels, key=kern.get)
    roof = solve_roof(dom) if dom.endswith("_fuse") else gram_roof(dom)

    gram_stage = {"pd": gram_roof("pd_local"), "fd": gram_roof("fd_local")}
    if "gram_stage_concurrent" in kern:
        # Both contractions together, as the step's two branches run them.
        alg2 = 2 * input_bytes(B, U, n_sc, n_sym)
        ach2 = alg2 / (kern["gram_stage_concurrent"] * 1e-3) / 1e9
        gram_stage["pd+fd concurrent"] = {
            "kernels": "PD and FD contractions as two graph branches (the step without its solves)",
            "bound": "hbm", "achieved": ach2, "peak": hbm_peak, "peak_source": f"{peak_src} (STREAM-style copy)",
            "unit": "GB/s", "frac": ach2 / hbm_peak, "algorithmic_bytes": alg2,
            "ms": kern["gram_stage_concurrent"]}

    def arch_ms(tag, a):
        return kern[f"{tag}_fused"] if fused[a] else kern[f"{tag}_local"] + kern[f"{tag}_fuse"]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": elapsed_ms / K, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": value / PAPER_SYMBOLS_PER_S,
        "dtype": DTYPE[args.precision], "data": "synthetic",
        "config": {"workload": "B=256 U=16 C=8 1200sc x 14sym 16-QAM Rayleigh 10dB, PD+FD, LLRs",
                   "precision": args.precision,
                   "l2": f"rotating {n_sets} input sets ({n_sets * in_bytes / 2**20:.0f} MiB > L2)",
                   "parallelism": f"replicas x{world}"},
        "kernels_ms": kern,
        "tuning": {("pd" if a == ffeq.PD else "fd"): list(ffeq.ffeq_plan_get_tuning(pl)) for a, pl in plans.items()},
        "schedule": schedule,
        "per_arch_symbols_per_s": {"pd": U * n_sc * n_sym / (arch_ms("pd", ffeq.PD) * 1e-3),
                                   "fd": U * n_sc * n_sym / (arch_ms("fd", ffeq.FD) * 1e-3)},
        "roofline": roof,
        "roofline_gram_stage": gram_stage,
        "roofline_solve_stage": {"pd": solve_roof("pd_fuse"), "fd": solve_roof("fd_fuse")},
        "fp32_same_gpu": fp32_cmp,
        "equalizers": variants or None,
        "accuracy": accuracy,
        "e2e": e2e,
        "e2e_host_entry": e2e_host_entry,
        "gpu_launches": launches * K,
    }
    line.update(extras)
    clocks = clk.summary()
    if clocks:
        clocks["window"] = "1 s of step replays directly before the timed region, then the timed region"
        line["clocks"] = clocks
    if do_cpu and world == 1:
        r, n, cores = _time_cpu_all_cores("oracle", args.cpu_seconds)
        line["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n} subcarriers of the same workload, PD+FD with LLRs, one "
                                          f"single-threaded process per core for ~{args.cpu_seconds:.0f} s"}
        r2, n2, cores2 = _time_cpu_all_cores("numpy32", max(2.0, args.cpu_seconds / 3))
        line["cpu_baseline_numpy_fp32"] = {
            "value": r2, "unit": UNIT, "cores": cores2, "kind": "batched FP32 NumPy (Cholesky / solve)",
            "sample": f"{n2} subcarriers of the same workload, PD+FD z and sigma^2 (no LLRs), one single-threaded "
                      f"process per core for ~{max(2.0, args.cpu_seconds / 3):.0f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
