#!/usr/bin/env python
"""Throughput of the SPGM hot path (A_B s, A_B^H r, gradient step, prox) on one GB300.

Workload (default, --workload large): 32 TX + 32 RX boundary array on a 0.4 m
aperture (1024 pairs), 128 equally spaced frequencies 70-80 GHz (M = 131072),
128 x 128 x 64 voxels (N = 1048576), minibatches of 64 pairs x 128 frequencies.
One step = one SPGM epoch = 16 minibatch iterations, each a forward A_B s with
the residual, an adjoint A_B^H r fused with the gradient step and the prox.
--workload mid is the 16 + 16 array, 64 frequencies, 64 x 64 x 32 voxels and
16-pair minibatches; --workload batched48 the 48 uneven scenes alone.

Metric: (measurement row, voxel) element pairs processed per second by the
forward and the adjoint, in units of 1e9: each epoch touches 2 * M * N pairs
(2.75e11 on the large workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica (its own scene) and rank
0 prints one JSON line with the whole-job throughput.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "G (meas,voxel) pairs/s for A_B s + A_B^H r; SPGM time to oracle NMSE"
UNIT = "G pairs/s"
# Algorithmic work per (row, voxel) element: one complex multiply-accumulate plus
# one complex phasor step of the frequency recurrence = 8 FP32 FMA-pipe
# lane-instructions, counted as 16 flops (an FMA-pipe instruction = 2 flops).
FLOPS_PER_PAIR = 16.0          # direct recurrence: flops per (row, voxel) element
FP32_LANES_PER_SM = 128
CHEB_GEOM_OPS = 42             # expansion: FP32/SFU ops of geometry and base phase per (pair, voxel)


def cheb_flops_per_pair_voxel(L, K, block=128):
    """Algorithmic FP32 work of the expansion operator per (pair, voxel), each FMA-pipe operation counted as
    2 flops: L Chebyshev recurrence steps with a complex-by-real accumulation (3L FMAs); per (pair, block),
    spread over the block's voxels (128 for a tile, 256 for the adjoint's two-tile blocks), the expansion
    over half the band with its mirror (K L FMAs: the band-centred table has b_l(K-1-k) = (-1)^l b_l(k)),
    the even/odd fold (2K adds) and the block phasor (a complex multiply and a recurrence step per
    frequency, 8K); and the geometry (two distances, amplitude, base phase: CHEB_GEOM_OPS ops)."""
    return 2.0 * (3 * L + (K * L + 10.0 * K) / float(block) + CHEB_GEOM_OPS)
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=10.0, help="bound on the CPU-baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "tc_bf16x3", "tc_fp16x3"],
                    help="adjoint arithmetic: CUDA-core FP32 or tensor-core split precision")
    ap.add_argument("--nonuniform", action="store_true",
                    help="jitter the frequencies off the uniform grid (general-frequency kernels)")
    ap.add_argument("--study-rho", type=float, nargs="+", default=[0.3, 0.1, 0.03],
                    help="paper_like study: step sizes as eta * L")
    ap.add_argument("--algorithm", default="auto", choices=["auto", "direct", "chebyshev"],
                    help="FP32 operator algorithm for equally spaced frequencies")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default forward launch shape")
    ap.add_argument("--forward-shape", default=None, metavar="T,G,P,C",
                    help="apply this expansion-forward launch shape (threads, lanes per group, pairs per CTA, "
                         "chunks) instead of autotuning, e.g. one an earlier run printed")
    ap.add_argument("--study", default=None, choices=["paper_like", "time_to_nmse"],
                    help="run a study instead of the bench line: the Sec. V PGM vs SPGM comparison on a "
                         "paper-shaped scene, or SPGM time to the oracle's NMSE (small and mid workloads)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra legs of the default run (48 uneven scenes, time to the oracle's NMSE)")
    ap.add_argument("--workload", default="large", choices=["mid", "large", "batched48"],
                    help="mid = the headline workload; large = 32 TX x 32 RX, K = 128, N = 1048576; "
                         "batched48 = 48 uneven scenes per epoch through one CUDA graph")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def ranks_max(x: float, device="cpu") -> float:
    """Maximum of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(pairs_per_step: float, steps: int, world: int, max_seconds: float) -> float:
    """Whole-job G pairs/s: every rank runs its own replica of the same workload (weak scaling)."""
    return pairs_per_step * steps * world / max_seconds / 1e9


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ---------------------------------------------------------------------------
# clocks sampler (nvidia-smi during the timed region)
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.samples = []
        self.proc = None
        self.marks = []

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.perf_counter(), line.strip()))

    def mark(self):
        self.marks.append(time.perf_counter())

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.samples:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((t, float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        t0, t1 = (self.marks[0], self.marks[-1]) if len(self.marks) >= 2 else (rows[0][0], rows[-1][0])
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in inside for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# ---------------------------------------------------------------------------
def build_problem(torch, ctx, w, seed_offset):
    """Scene, noisy measurements y = A s + w (GPU forward), SPGM step and lambda (GPU).

    The step is 1 / max(L, L_B): L = lambda_max(A^H A)/M (50 power iterations) and L_B the largest
    minibatch constant lambda_max(A_B^H A_B)/B over the minibatches of the first epoch (20 power
    iterations each); a step of 1/L alone can make SPGM diverge where a few pairs' L_B exceeds 2L.
    Returns y, eta, lambda, L, L_B."""
    import numpy as np
    from paper_2509_00774_gb300 import inputs as I
    geom = w.geom
    ctx.set_geometry(geom)
    dev = torch.device("cuda", ctx.device)
    s_true = torch.from_numpy(w.scene_vector().astype(np.complex64)).to(dev)
    all_pairs = torch.arange(geom.P, dtype=torch.int32, device=dev)
    clean = ctx.forward(all_pairs, s_true)
    g = torch.from_numpy(I.complex_gaussian(geom.M, w.seeds["noise"] + seed_offset).astype(np.complex64)).to(dev)
    sigma = float(torch.sqrt(torch.mean(clean.abs() ** 2) / 10 ** (w.snr_db / 10)))
    y = clean + sigma * g
    v0 = torch.from_numpy(I.complex_gaussian(geom.N, w.seeds["power"]).astype(np.complex64)).to(dev)
    L = ctx.power_iteration(v0, 50)
    perm0 = torch.from_numpy(I.epoch_permutation(geom.P, w.seeds["perm"] + 1000 * seed_offset, 0)
                             .astype(np.int32)).to(dev)
    LB = ctx.spgm_lipschitz(perm0, w.pairs_per_batch, v0, 20)
    lam = 0.05 * ctx.lambda_max(y)
    return y, 1.0 / max(L, LB), lam, L, LB


KERNEL_SOURCES = {"fwd_cheb_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "cheb_device.cuh", "op_cheb.cu"),
                  "adj_cheb_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "cheb_device.cuh", "op_cheb.cu"),
                  "adj_cheb_tc_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "cheb_device.cuh", "tc_ptx.cuh",
                                         "op_cheb_tc.cu"),
                  "fwd_cheb_tc_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "cheb_device.cuh", "tc_ptx.cuh",
                                         "op_cheb_tc_fwd.cu"),
                  "fwd_partial_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "op_forward.cu"),
                  "adj_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "op_adjoint.cu"),
                  "adj_tc_kernel": ("nfm_device.cuh", "nfm_kernels.cuh", "tc_ptx.cuh", "op_adjoint_tc.cu")}


def traffic_for(kernel, workload, pairs_per_batch):
    """DRAM bytes per launch from the committed ncu summary of this workload and minibatch size, if the
    kernel's sources are unchanged since the capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f).get("workloads", {}).get(workload, {})
    k = d.get("kernels", {}).get(kernel, {})
    if not k or d.get("pairs_per_batch") != pairs_per_batch or k.get("sources_sha256") != sources_digest(kernel):
        return None
    return k.get("dram_bytes_per_launch")


def sources_digest(kernel):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2509_00774_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    return h.hexdigest()


def prox_stream_gbs(torch, ctx, dev, stream, n=1 << 26, reps=10):
    """HBM rate of the stand-alone gradient-step + prox kernel (the autograd op; inside SPGM the same
    update is the adjoint's epilogue): 24 bytes per element (read s and g, write out), a 1.5 GB
    stream, CUDA events on the context stream, best of `reps` launches."""
    s = torch.randn(n, dtype=torch.complex64, device=dev)
    g = torch.randn(n, dtype=torch.complex64, device=dev)
    out = torch.empty_like(s)
    for _ in range(3):
        ctx.prox_step(s, g, 0.5, 0.3, out)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        ctx.prox_step(s, g, 0.5, 0.3, out)
        e1.record(stream)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    del s, g, out
    return {"kernel": "prox_step_vec_kernel", "elements": n, "bytes_per_element": 24,
            "achieved_gbs": 24.0 * n / best / 1e9, "us_per_launch": best * 1e6}


ORACLE_STEP_ELEMS = 1.0e9      # (row, voxel) pairs of one sampled oracle step (about 1-2 s on 16 cores)


def sample_pairs(w):
    """Pairs per sampled oracle step: the whole minibatch when its forward + adjoint stays within
    ORACLE_STEP_ELEMS element evaluations, else the first pairs of it (the metric counts pairs)."""
    per_pair = 2.0 * w.geom.K * w.geom.N
    return max(1, min(w.pairs_per_batch, int(ORACLE_STEP_ELEMS // per_pair)))


def cpu_baseline(w, y_np, eta, lam, seconds):
    """Time the FP64 oracle on SPGM minibatch steps of the same workload (bounded sample: a step holds the
    first sample_pairs(w) pairs of each minibatch)."""
    import numpy as np
    import oracle
    from paper_2509_00774_gb300 import inputs as I
    oracle.build()
    o = oracle.Oracle(w.geom)
    cores = oracle.get_threads()
    perm = I.epoch_permutation(w.geom.P, w.seeds["perm"], 0)
    bp = w.pairs_per_batch
    sp = sample_pairs(w)
    s = np.zeros(w.geom.N, dtype=np.complex128)
    done = 0
    t0 = time.perf_counter()
    while True:
        c = done % (w.geom.P // bp)
        s = o.spgm_step(y_np, s, perm[c * bp:c * bp + sp], eta, lam)
        done += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    pairs = done * 2.0 * sp * w.geom.K * w.geom.N
    return {"value": pairs / dt / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{done} SPGM step(s) on {sp} of the {bp} pairs of a minibatch of the workload ({w.geom.K} "
                      f"freqs x {w.geom.N} voxels, forward + adjoint + prox) in FP64 on {cores} host threads, "
                      f"{dt:.1f} s"}


def time_to_oracle_nmse(include_mid=False, tols=(1e-1, 3e-2, 1e-2, 1e-3, 1e-4), max_epochs=12000, block=100):
    """Time for each GPU form to bring its iterate within NMSE tol of the FP64 oracle's minimiser of Eq. 3.

    Small workload (4 TX x 4 RX, 16 freqs, 16x16x8 voxels, 4 pairs per minibatch): y, L (50 power
    iterations) and lambda from the oracle; the reference s* is the oracle's minimiser of Eq. 3
    (accelerated proximal gradient on the dense A, 10000 iterations, KKT residual reported).  SPGM uses
    eta = 1/L_B, L_B the largest minibatch constant over every possible 4-pair minibatch (a step of 1/L
    diverges here); PGM uses 1/L.  Every form runs the expansion operator (forward shape autotuned) from
    s = 0 for up to max_epochs epochs with CUDA events around each block of `block` epochs; the NMSE to
    s* is read at block ends, so epochs and times to each tolerance have a resolution of one block.
    Forms: SPGM in FP32, with the BF16x3 and FP16x3 tensor-core adjoint, PGM in FP32, and SPGM of 8
    scenes (other seeds, each with its own s*) in one CUDA graph per epoch (time per scene).  Each form
    is also compared with the oracle's own SPGM iterate after 30 epochs (the same algorithm and step):
    that NMSE is the parity at the same accuracy.  With include_mid, the mid workload's first 3 epochs
    (eta from the oracle's bound ||A||_F^2/M) are compared with the oracle's iterate the same way.
    """
    import dataclasses
    import itertools
    import numpy as np
    import torch
    import oracle
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import metrics
    from paper_2509_00774_gb300 import workloads as W
    from paper_2509_00774_gb300.nfmimo import Batch, Context
    oracle.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    n_blocks = max_epochs // block

    def problem(w):
        o = oracle.Oracle(w.geom)
        y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
        y = y.astype(np.complex64).astype(np.complex128)
        L = o.power_iteration(I.complex_gaussian(o.N, w.seeds["power"]), 50)
        lam = float(np.float32(0.05 * o.lambda_max(y)))
        s_star, kkt = o.minimiser_dense(y, lam, L, 10000)
        return o, y, L, lam, s_star, kkt

    def minibatch_L_max(o, bp):
        A = o.dense(np.arange(o.M), np.arange(o.N))
        G = A @ A.conj().T
        best = 0.0
        for pairs in itertools.combinations(range(o.P), bp):
            rows = o.rows_of_pairs(pairs)
            best = max(best, float(np.linalg.eigvalsh(G[np.ix_(rows, rows)])[-1]) / rows.size)
        return best

    def oracle_spgm(o, w, y, eta, lam, epochs):
        s = np.zeros(o.N, dtype=np.complex128)
        t0 = time.perf_counter()
        for e in range(epochs):
            s = o.spgm_epoch(y, s, I.epoch_permutation(o.P, w.seeds["perm"], e), w.pairs_per_batch, eta, lam)
        return s, time.perf_counter() - t0

    def summarise(ms_blocks, nmse_blocks, extra):
        out = dict(extra)
        for tol in tols:
            hit = next((b for b, x in enumerate(nmse_blocks) if x <= tol), None)
            out[f"nmse<={tol:g}"] = None if hit is None else {"epochs": (hit + 1) * block,
                                                              "ms": float(sum(ms_blocks[:hit + 1]))}
        out.update({"epochs_run": len(ms_blocks) * block, "ms_all": float(sum(ms_blocks)),
                    "final_nmse_to_minimiser": nmse_blocks[-1]})
        return out

    def make_ctx(g, precision, bp):
        c = Context(dev.index)
        c.set_precision(precision)
        c.set_geometry(g)
        c.set_algorithm("chebyshev")
        c.autotune(bp)
        return c

    def run_form(w, y, s_star, s_orc30, eta, lam, precision="fp32", pgm=False):
        g = w.geom
        ctx = make_ctx(g, precision, w.pairs_per_batch)
        y_d = torch.from_numpy(y.astype(np.complex64)).to(dev)
        star = torch.from_numpy(s_star.astype(np.complex64)).to(dev)
        orc = torch.from_numpy(s_orc30.astype(np.complex64)).to(dev)
        perms = torch.from_numpy(np.stack([I.epoch_permutation(g.P, w.seeds["perm"], e)
                                           for e in range(max_epochs)]).astype(np.int32)).to(dev)
        bp = w.pairs_per_batch

        def epoch(s, e):
            if pgm:
                ctx.pgm_step(y_d, s, eta, lam)
            else:
                ctx.spgm_epoch(y_d, s, perms[e], bp, eta, lam)

        scratch = torch.zeros(g.N, dtype=torch.complex64, device=dev)
        for e in range(3):
            epoch(scratch, e)
        s = torch.zeros(g.N, dtype=torch.complex64, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_blocks)]
        errs = []
        track = None
        torch.cuda.synchronize()
        for b in range(n_blocks):
            ev[2 * b].record()
            for e in range(b * block, (b + 1) * block):
                epoch(s, e)
                if e == 29 and not pgm:
                    track = torch.sum((s - orc).abs() ** 2) / torch.sum(orc.abs() ** 2)
            ev[2 * b + 1].record()
            errs.append(torch.sum((s - star).abs() ** 2) / torch.sum(star.abs() ** 2))
        torch.cuda.synchronize()
        ms = [ev[2 * b].elapsed_time(ev[2 * b + 1]) for b in range(n_blocks)]
        nm = [float(x) for x in errs]
        ctx.close()
        extra = {"step": eta, "operator": "chebyshev"}
        if track is not None:
            extra["nmse_to_oracle_spgm_at_30_epochs"] = float(track)
        return summarise(ms, nm, extra)

    w = W.small_T4R4_K16_16x16x8()
    t0 = time.perf_counter()
    o, y, L, lam, s_star, kkt = problem(w)
    t_orc = time.perf_counter() - t0
    LB = minibatch_L_max(o, w.pairs_per_batch)
    eta_s = float(np.float32(1.0 / LB))
    eta_p = float(np.float32(1.0 / L))
    s_orc30, t_orc30 = oracle_spgm(o, w, y, eta_s, lam, 30)
    small = {"workload": w.name, "pairs_per_batch": w.pairs_per_batch, "L": L, "L_B_max": LB, "lambda": lam,
             "reference": "oracle minimiser of Eq. 3 (FISTA on the dense A, 10000 iterations, FP64)",
             "reference_kkt": kkt, "reference_s": t_orc, "oracle_spgm_30_epochs_s": t_orc30,
             "oracle_cores": oracle.get_threads(), "block": block}
    for prec in ("fp32", "tc_bf16x3", "tc_fp16x3"):
        small["spgm_" + prec] = run_form(w, y, s_star, s_orc30, eta_s, lam, precision=prec)
    small["pgm_fp32"] = run_form(w, y, s_star, s_orc30, eta_p, lam, pgm=True)
    # batched form: 8 scenes of the same geometry with their own seeds, one graph per epoch
    scenes = [dataclasses.replace(w, seeds={"scene": 50 + 4 * i, "noise": 51 + 4 * i, "perm": 52 + 4 * i,
                                            "power": 53 + 4 * i}) for i in range(8)]
    probs = [problem(x) for x in scenes]
    LBs = [minibatch_L_max(p[0], w.pairs_per_batch) for p in probs]
    ctxs = [make_ctx(x.geom, "fp32", w.pairs_per_batch) for x in scenes]
    batch = Batch(ctxs)
    ys = [torch.from_numpy(p[1].astype(np.complex64)).to(dev) for p in probs]
    stars = [torch.from_numpy(p[4].astype(np.complex64)).to(dev) for p in probs]
    perm_all = [torch.from_numpy(np.stack([I.epoch_permutation(w.geom.P, x.seeds["perm"], e)
                                           for e in range(max_epochs)]).astype(np.int32)).to(dev) for x in scenes]
    perm_bufs = [torch.empty(w.geom.P, dtype=torch.int32, device=dev) for _ in scenes]
    bps = [w.pairs_per_batch] * len(scenes)
    etas = [float(np.float32(1.0 / x)) for x in LBs]
    lams = [p[3] for p in probs]
    scratch = [torch.zeros(w.geom.N, dtype=torch.complex64, device=dev) for _ in scenes]
    for e in range(3):
        for pb, pa in zip(perm_bufs, perm_all):
            pb.copy_(pa[e])
        batch.spgm_epoch(ys, scratch, perm_bufs, bps, etas, lams)
    ss = [torch.zeros(w.geom.N, dtype=torch.complex64, device=dev) for _ in scenes]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * n_blocks)]
    errs = []
    torch.cuda.synchronize()
    for b in range(n_blocks):
        ev[2 * b].record()
        for e in range(b * block, (b + 1) * block):
            for pb, pa in zip(perm_bufs, perm_all):
                pb.copy_(pa[e])
            batch.spgm_epoch(ys, ss, perm_bufs, bps, etas, lams)
        ev[2 * b + 1].record()
        errs.append(torch.stack([torch.sum((x - st).abs() ** 2) / torch.sum(st.abs() ** 2)
                                 for x, st in zip(ss, stars)]).max())
    torch.cuda.synchronize()
    ms = [ev[2 * b].elapsed_time(ev[2 * b + 1]) / len(scenes) for b in range(n_blocks)]
    small["spgm_batched_fp32_8_scenes"] = summarise(ms, [float(x) for x in errs],
                                                   {"time": "per scene (8 scenes per graph; worst NMSE of the 8)",
                                                    "reference_kkt_max": max(p[5] for p in probs)})
    batch.close()
    for c in ctxs:
        c.close()
    out = {"tolerances": list(tols), "small": small}
    if include_mid:
        w = W.mid_T16R16_K64_64x64x32()
        o = oracle.Oracle(w.geom)
        y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
        y = y.astype(np.complex64).astype(np.complex128)
        eta = float(np.float32(1.0 / o.frobenius_bound()))
        lam = float(np.float32(0.05 * o.lambda_max(y)))
        s_ref, t_orc = oracle_spgm(o, w, y, eta, lam, 3)
        mid = {"workload": w.name, "epochs": 3, "pairs_per_batch": w.pairs_per_batch, "oracle_s": t_orc,
               "oracle_cores": oracle.get_threads(),
               "reference": "oracle SPGM iterate after the same 3 epochs (the minimiser is out of the oracle's reach)",
               "step": "1/L_F, L_F = ||A||_F^2/M (oracle closed form; bounds every minibatch constant)"}
        for prec in ("fp32", "tc_bf16x3", "tc_fp16x3"):
            ctx = make_ctx(w.geom, prec, w.pairs_per_batch)
            y_d = torch.from_numpy(y.astype(np.complex64)).to(dev)
            s = torch.zeros(w.geom.N, dtype=torch.complex64, device=dev)
            perms = [torch.from_numpy(I.epoch_permutation(w.geom.P, w.seeds["perm"], e).astype(np.int32)).to(dev)
                     for e in range(3)]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for e in range(3):
                ctx.spgm_epoch(y_d, s, perms[e], w.pairs_per_batch, eta, lam)
            e1.record()
            torch.cuda.synchronize()
            mid[prec] = {"ms_3_epochs": e0.elapsed_time(e1), "nmse_to_oracle": metrics.nmse(s.cpu().numpy(), s_ref)}
            ctx.close()
        out["mid"] = mid
    return out


def run_reference(args):
    """The oracle arm: the FP64 CPU oracle on the same workload, one minibatch step per step."""
    import numpy as np
    import oracle
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import workloads as W
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = W.large_T32R32_K128_128x128x64() if args.workload == "large" else W.mid_T16R16_K64_64x64x32()
    oracle.build()
    o = oracle.Oracle(w.geom)
    cores = oracle.get_threads()
    y = I.add_noise(o.forward_sparse(w.scene_vector()), I.complex_gaussian(o.M, w.seeds["noise"]), w.snr_db)
    eta, lam = 1.0 / 70.0, 0.05 * 1e-3
    perm = I.epoch_permutation(o.P, w.seeds["perm"], 0)
    bp = w.pairs_per_batch
    sp = sample_pairs(w)
    s = np.zeros(o.N, dtype=np.complex128)
    n_chunks = o.P // bp
    for i in range(args.warmup):
        c = i % n_chunks
        s = o.spgm_step(y, s, perm[c * bp:c * bp + sp], eta, lam)
    t0 = time.perf_counter()
    for i in range(args.steps):
        c = (args.warmup + i) % n_chunks
        s = o.spgm_step(y, s, perm[c * bp:c * bp + sp], eta, lam)
    dt = time.perf_counter() - t0
    per_step = 2.0 * sp * o.K * o.N
    value = per_step * args.steps / dt / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "T": o.T, "R": o.R, "K": o.K, "N": o.N, "M": o.M, "pairs_per_batch": bp,
                   "minibatches_per_step": 1,
                   "step": f"one SPGM step on {sp} of the {bp} pairs of a minibatch ({o.K} freqs, forward + adjoint "
                           f"+ prox) in FP64",
                   "parallelism": f"{cores} host threads (OpenMP)"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} SPGM steps on {sp} of the {bp} pairs of a minibatch each, "
                                   f"{cores} host threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2509_00774_gb300 import build as nb
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import workloads as W
    from paper_2509_00774_gb300.nfmimo import Context

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    nb.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    w = W.mid_T16R16_K64_64x64x32() if args.workload == "mid" else W.large_T32R32_K128_128x128x64()
    if args.nonuniform:
        f = w.geom.freq
        step = (f[-1] - f[0]) / (f.size - 1)
        w.geom.freq = f + np.random.default_rng(5).uniform(-0.3, 0.3, f.size) * step
    geom = w.geom
    with torch.cuda.stream(stream):
        ctx = Context(local, stream=stream)
        ctx.set_precision(args.precision)
        ctx.set_algorithm(args.algorithm)
        y, eta, lam, L_full, L_B = build_problem(torch, ctx, w, seed_offset=rank)
        algo, cheb_L, cheb_zmax = ctx.algorithm_info()
        shape = None
        if algo == "chebyshev" and args.forward_shape:
            t, g, p, c = (int(x) for x in args.forward_shape.split(","))
            shape = {"algorithm": "chebyshev", "threads": t, "lanes_per_group": g, "pairs_per_cta": p, "chunks": c}
            ctx.set_forward_shape(w.pairs_per_batch, shape)
        elif algo == "chebyshev" and not args.no_autotune:
            shape = ctx.autotune(w.pairs_per_batch)
        if shape is not None:
            algo = shape["algorithm"]          # with "auto" the tuner may keep the direct recurrence
        E = args.warmup + args.steps
        perms = np.stack([I.epoch_permutation(geom.P, w.seeds["perm"] + 1000 * rank, e) for e in range(E)])
        perms_d = torch.from_numpy(perms.astype(np.int32)).to(dev)
        s = torch.zeros(geom.N, dtype=torch.complex64, device=dev)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
        bp = w.pairs_per_batch
        for e in range(args.warmup):
            ctx.spgm_epoch(y, s, perms_d[e], bp, eta, lam)
        torch.cuda.synchronize()
        props = torch.cuda.get_device_properties(dev)
        uuid = str(getattr(props, "uuid", "") or "")
        sampler = ClockSampler(("GPU-" + uuid) if uuid and not uuid.startswith("GPU-") else uuid)
        sampler.start()
        time.sleep(0.3)
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        sampler.mark()
        for k in range(args.steps):
            flush.fill_(float(k))                  # L2 flush, outside the timed events
            starts[k].record(stream)
            ctx.spgm_epoch(y, s, perms_d[args.warmup + k], bp, eta, lam)
            ends[k].record(stream)
        torch.cuda.synchronize()
        sampler.mark()
        # kernel timing pass: the same epochs with every kernel bracketed by events
        # (kept out of the timed region above because the events add gaps)
        ctx.profile_enable(True)
        ctx.profile_report()
        prof_steps = max(1, min(args.steps, 20))
        for k in range(prof_steps):
            flush.fill_(float(k))
            ctx.spgm_epoch(y, s, perms_d[args.warmup + k], bp, eta, lam)
        prof = ctx.profile_report()
        ctx.profile_enable(False)
        hbm = prox_stream_gbs(torch, ctx, dev, stream)
        time.sleep(0.25)
        sampler.stop()
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        total_ms = ranks_max(float(sum(step_ms)), dev)
        pairs_per_step = 2.0 * geom.M * geom.N
        value = job_throughput(pairs_per_step, args.steps, world, total_ms * 1e-3)

        # end to end through the host-buffer entry point (copies inside the timed region)
        y_host = torch.empty(geom.M, dtype=torch.complex64, pin_memory=True)
        y_host.copy_(y)
        s_host = torch.zeros(geom.N, dtype=torch.complex64, pin_memory=True)
        perms_host = torch.from_numpy(perms.astype(np.int32)).pin_memory()
        for e in range(min(args.warmup, 2)):
            ctx.spgm_epochs_host(y_host, s_host, perms_host[e:e + 1], bp, eta, lam)
        e2e_steps = max(1, min(args.steps, 50))
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            ctx.spgm_epochs_host(y_host, s_host, perms_host[k % E:k % E + 1], bp, eta, lam)
        e2e_s = ranks_max(time.perf_counter() - t0, dev)
        e2e_value = job_throughput(pairs_per_step, e2e_steps, world, e2e_s)
        h2d = geom.M * 8 + geom.N * 8 + geom.P * 4
        d2h = geom.N * 8

    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peaks, peak_src = measured_peaks()
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12
    kernels = {}
    elems = bp * geom.K * geom.N        # (row, voxel) pairs per forward / adjoint launch
    cheb = algo == "chebyshev"
    # the FP32 expansion operator may run over blocks of two tiles (256 voxels) with their own expansion
    blk_L, blk_V = ctx.expansion_info() if cheb and args.precision == "fp32" else (cheb_L, 128)
    flops_fwd = cheb_flops_per_pair_voxel(blk_L, geom.K, blk_V) if cheb else None
    flops_adj = flops_fwd
    for kind, (ms, n) in prof.items():
        if n == 0:
            continue
        avg_ms = ms / n
        entry = {"launches": n, "total_ms": ms, "avg_us": avg_ms * 1e3}
        if kind in ("forward_partial", "adjoint") and (cheb or kind == "forward_partial" or args.precision == "fp32"):
            flops_per_launch = ((flops_fwd if kind == "forward_partial" else flops_adj) * bp * geom.N if cheb
                                else FLOPS_PER_PAIR * elems)
            tf = flops_per_launch / (avg_ms * 1e-3) / 1e12
            entry.update({"gpairs_per_s": elems / (avg_ms * 1e-3) / 1e9, "tflops": tf,
                          "direct_equivalent_tflops": FLOPS_PER_PAIR * elems / (avg_ms * 1e-3) / 1e12})
        elif kind == "adjoint":
            entry.update({"gpairs_per_s": elems / (avg_ms * 1e-3) / 1e9,
                          "tflops": FLOPS_PER_PAIR * elems / (avg_ms * 1e-3) / 1e12})
        kernels[kind] = entry
    dom = max(("forward_partial", "adjoint"), key=lambda k: kernels.get(k, {}).get("total_ms", 0.0))
    dk = kernels[dom]
    kname = {"forward_partial": ("fwd_cheb_kernel" if args.precision == "fp32" else "fwd_cheb_tc_kernel") if cheb
             else "fwd_partial_kernel",
             "adjoint": ("adj_cheb_kernel" if cheb else "adj_kernel") if args.precision == "fp32"
             else ("adj_cheb_tc_kernel" if cheb else "adj_tc_kernel")}[dom]
    if cheb:
        wL, wB = blk_L, blk_V
        work = (f"{cheb_flops_per_pair_voxel(wL, geom.K, wB):.0f} flops per (pair, voxel) = 2 x (3L "
                f"recurrence/accumulate FMAs + (KL + 10K)/{wB} mirror-folded expansion and block-phasor ops + "
                f"{CHEB_GEOM_OPS} geometry ops), L = {wL}, K = {geom.K}, {wB}-voxel blocks; "
                f"{bp * geom.N} (pair, voxel) = {elems} (row, voxel) per launch" +
                ("" if args.precision == "fp32" else
                 "; the expansion contraction runs on tcgen05, the rest on the FP32 lanes"))
    else:
        work = (f"{FLOPS_PER_PAIR:.0f} flops = 8 FP32 FMA-pipe lane-instructions (complex MAC + phasor step) "
                f"per (row, voxel) pair, {elems} pairs per launch")
    roofline = {"bound": "alu", "kernel": kname, "achieved": dk["tflops"], "peak": fp32_peak_tflops,
                "unit": "TFLOP/s", "frac": dk["tflops"] / fp32_peak_tflops,
                "traffic": None if args.nonuniform else traffic_for(kname, w.name, bp),
                "peak_source": f"FP32 FMA lanes: {props.multi_processor_count} SMs x {FP32_LANES_PER_SM} x 2 flops x "
                               f"{sm_mhz:.0f} MHz (sm_max_mhz, {peak_src})",
                "work": work,
                "timing": f"CUDA events around every launch over {prof_steps} epochs run right after the timed region"}
    launches = sum(kernels.get(k, {}).get("launches", 0) for k in ("forward_partial", "forward_reduce", "adjoint"))
    launches = launches * args.steps // prof_steps      # per timed region (same kernels every epoch)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name + ("_jittered_freqs" if args.nonuniform else ""), "T": geom.T, "R": geom.R, "K": geom.K, "N": geom.N, "M": geom.M,
                   "pairs_per_batch": bp, "minibatches_per_step": geom.P // bp, "step": "one SPGM epoch",
                   "operator": (f"fp32 cuda-core block-local Chebyshev expansion, L = {blk_L} over {blk_V}-voxel "
                                f"blocks" if cheb else
                                "forward: fp32 cuda-core three-term phasor recurrence; adjoint: fp32 cuda-core Horner") +
                               ("" if args.precision == "fp32" else
                                f"; expansion contractions of the forward{' and the adjoint' if cheb else ''} on "
                                f"tcgen05, {args.precision[3:]} split, FP32 accumulate in TMEM"),
                   "forward_launch_shape": shape,
                   "l2": "256 MiB buffer written between timed steps, outside the timed events",
                   "eta": eta, "lambda": lam, "L": L_full, "L_B_max_epoch0": L_B,
                   "step_rule": "eta = 1/max(L, L_B)", "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "kernels": kernels,
        "update_prox_hbm": dict(hbm, peak_gbs=float(peaks.get("hbm_gbs", 6800.0)),
                                frac=hbm["achieved_gbs"] / float(peaks.get("hbm_gbs", 6800.0)),
                                peak_source=peak_src),
        "gpu_launches": launches,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps, "api": "nfm_spgm_epochs_host (pinned host buffers)"},
        "clocks": sampler.summary(),
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, y.cpu().numpy().astype(np.complex128), eta, lam, args.cpu_seconds)
    if world == 1 and not args.no_extras and not args.nonuniform:
        ctx.close()
        line["batched48"] = batched48_leg(args, min(args.steps, 10), 3)
        line["time_to_oracle_nmse"] = time_to_oracle_nmse(include_mid=True)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_batched(args):
    """48 uneven scenes (grids 32..96, 8..24 TX/RX, 32..96 freqs), one SPGM epoch of all per step."""
    line = batched48_leg(args, args.steps, args.warmup)
    print(json.dumps(line), flush=True)


def batched48_leg(args, steps, warmup):
    """The 48-scene batched SPGM timed over `steps` epochs in both batch modes (a graph branch per scene, and
    the fused launches over all scenes per step index); returns the line of the faster, the other under
    config["other_mode"]."""
    lines = {}
    for mode in ("branches", "fused"):
        try:
            lines[mode] = batched48_mode(args, steps, warmup, mode)
        except Exception as ex:          # a scene set the fused mode cannot run (expansion longer than 20 terms)
            lines[mode] = {"unavailable": str(ex)[:200]}
    ok = [m for m in lines if "value" in lines[m]]
    best = max(ok, key=lambda m: lines[m]["value"])
    line = lines[best]
    other = [m for m in lines if m != best][0]
    o = lines[other]
    line["config"]["other_mode"] = ({"mode": other, "value": o["value"], "ms_per_step": o["ms_per_step"]}
                                    if "value" in o else {"mode": other, **o})
    return line


def batched48_mode(args, steps, warmup, mode):
    """The 48-scene batched SPGM in one batch mode (one CUDA graph per epoch)."""
    import numpy as np
    import torch
    from paper_2509_00774_gb300 import build as nb
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import workloads as W
    from paper_2509_00774_gb300.nfmimo import Batch, Context
    nb.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream(device=dev)
    ws = [W.batched_scene(i) for i in range(48)]
    E = warmup + steps
    with torch.cuda.stream(stream):
        ctxs, ys, ss, perm_bufs, perm_all, etas, lams = [], [], [], [], [], [], []
        for w in ws:
            g = w.geom
            c = Context(0, stream=stream)
            c.set_precision(args.precision)
            c.set_algorithm(args.algorithm)
            c.set_geometry(g)
            allp = torch.arange(g.P, dtype=torch.int32, device=dev)
            clean = c.forward(allp, torch.from_numpy(w.scene_vector().astype(np.complex64)).to(dev))
            noise = torch.from_numpy(I.complex_gaussian(g.M, w.seeds["noise"]).astype(np.complex64)).to(dev)
            sigma = float(torch.sqrt(torch.mean(clean.abs() ** 2) / 10 ** (w.snr_db / 10)))
            y = clean + sigma * noise
            v0 = torch.from_numpy(I.complex_gaussian(g.N, w.seeds["power"]).astype(np.complex64)).to(dev)
            L = c.power_iteration(v0, 10)
            ctxs.append(c)
            ys.append(y)
            ss.append(torch.zeros(g.N, dtype=torch.complex64, device=dev))
            perm_all.append(torch.from_numpy(np.stack([I.epoch_permutation(g.P, w.seeds["perm"], e)
                                                       for e in range(E)]).astype(np.int32)).to(dev))
            perm_bufs.append(torch.empty(g.P, dtype=torch.int32, device=dev))
            etas.append(1.0 / L)
            lams.append(0.05 * c.lambda_max(y))
            if not args.no_autotune and c.algorithm_info()[0] == "chebyshev":
                c.autotune(w.pairs_per_batch)
        bps = [w.pairs_per_batch for w in ws]
        batch = Batch(ctxs, stream=stream)
        batch.set_mode(mode)
        flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

        def set_perms(e):
            for pb, pa in zip(perm_bufs, perm_all):
                pb.copy_(pa[e])

        for e in range(warmup):
            set_perms(e)
            batch.spgm_epoch(ys, ss, perm_bufs, bps, etas, lams)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for k in range(steps):
            set_perms(warmup + k)
            flush.fill_(float(k))
            starts[k].record(stream)
            batch.spgm_epoch(ys, ss, perm_bufs, bps, etas, lams)
            ends[k].record(stream)
        torch.cuda.synchronize()
        total_ms = float(sum(a.elapsed_time(b) for a, b in zip(starts, ends)))
    pairs = sum(2.0 * w.geom.M * w.geom.N for w in ws)
    line = {"metric": METRIC, "value": pairs * steps / (total_ms * 1e-3) / 1e9, "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": total_ms / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched48_uneven", "scenes": len(ws), "pairs_per_step": pairs,
                       "mode": mode,
                       "step": ("one SPGM epoch of all 48 scenes (one CUDA graph, a branch per scene)" if mode == "branches"
                                else "one SPGM epoch of all 48 scenes (one CUDA graph; per step index one forward, one "
                                     "reduction and one adjoint launch over every scene with a minibatch left)"),
                       "precision": args.precision, "l2": "256 MiB buffer written between timed steps"}}
    batch.close()
    for c in ctxs:
        c.close()
    return line


def run_paper_like(args):
    """Synthetic analogue of the paper's Sec. V study (Figs. 1-4) on a scene of the measured data
    set's shape (16 TX x 9 RX spirals, 11 frequencies 4-16 GHz, 61 x 61 x 21 voxels).

    PGM and SPGM with Cartesian minibatches (#f, #Tx, #Rx) run until the change in reflectivity
    magnitudes relative to the peak magnitude, max_n | |s_n(k+1)| - |s_n(k)| | / max_n |s_n(k+1)|,
    drops below 1e-3 (relative, since the synthetic data's scale is not the measured set's).  The
    statistic is taken once every c iterations (c = ceil(M / B), about one pass over the rows)
    over that chunk's last iteration and read one chunk later, so a run stops at most 2c - 1
    iterations after the rule first holds.  PSNR over
    normalised magnitudes against the PGM reconstruction, as in Fig. 4, and against PGM run to a
    relative change of 1e-6 (the fixed point); PGM* is PGM stopped at the (4, 4, 3) run's wall
    time, as in Fig. 1(e).  Device microseconds per iteration are timed separately, without checks.  The minibatch draws are generated before the
    timed region (they are inputs); wall time covers the GPU work and its launches."""
    import numpy as np
    import torch
    from paper_2509_00774_gb300 import build as nb
    from paper_2509_00774_gb300 import inputs as I
    from paper_2509_00774_gb300 import metrics
    from paper_2509_00774_gb300 import workloads as W
    from paper_2509_00774_gb300.nfmimo import Context
    nb.build()
    dev = torch.device("cuda", 0)
    w = W.paper_like_T16R9_K11_61x61x21()
    g = w.geom
    ctx = Context(0)
    ctx.set_geometry(g)
    allp = torch.arange(g.P, dtype=torch.int32, device=dev)
    clean = ctx.forward(allp, torch.from_numpy(w.scene_vector().astype(np.complex64)).to(dev))
    noise = torch.from_numpy(I.complex_gaussian(g.M, w.seeds["noise"]).astype(np.complex64)).to(dev)
    y = clean + float(torch.sqrt(torch.mean(clean.abs() ** 2) / 10 ** (w.snr_db / 10))) * noise
    L = ctx.power_iteration(torch.from_numpy(I.complex_gaussian(g.N, 3).astype(np.complex64)).to(dev), 50)
    lam = 0.05 * ctx.lambda_max(y)
    tol = 1e-3
    comps = [(4, 4, 3), (1, 4, 3), (2, 4, 3), (4, 8, 6), (11, 4, 3), (11, 16, 9)]
    out = {"study": "pgm_vs_spgm_cartesian", "workload": w.name, "M": g.M, "N": g.N, "L": L,
           "lambda": lam, "tol_magnitude_change": tol, "runs": []}

    def solve(eta, comp, max_iters, fixed_iters=None, tol_override=None):
        nf, ntx, nrx = comp
        full = comp == (g.K, g.T, g.R)
        B = nf * ntx * nrx
        c = 1 if full else -(-g.M // B)
        n_draw = 0 if full else min(max_iters, 1 << 16)
        if not full:
            draws = [I.cartesian_minibatch(g.T, g.R, g.K, ntx, nrx, nf, seed=13, it=i) for i in range(n_draw)]
            pairs = torch.from_numpy(np.stack([d[0] for d in draws])).to(dev)
            masks = torch.from_numpy(np.stack([d[1] for d in draws])).to(dev)
        s = torch.zeros(g.N, dtype=torch.complex64, device=dev)
        prev = torch.empty_like(s)
        stat = torch.empty(2, dtype=torch.float32, pin_memory=True)
        ev = [torch.cuda.Event(), torch.cuda.Event()]
        limit = fixed_iters if fixed_iters is not None else (max_iters if full else n_draw)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = 0
        chunk = 0
        change = float("inf")
        while k < limit:
            n = min(c, limit - k)
            for j in range(n):
                if j == n - 1 and fixed_iters is None:
                    prev.copy_(s)
                if full:
                    ctx.pgm_step(y, s, eta, lam)
                else:
                    ctx.spgm_step_freqs(y, s, pairs[k], masks[k], eta, lam, n_freq=nf)
                k += 1
            if fixed_iters is None:
                # relative change of the chunk's last iteration, copied back without a stall; the
                # previous chunk's value is read while this chunk runs (the run stops one chunk late)
                m = s.abs()
                rel = (m - prev.abs()).abs().max() / m.max().clamp_min(1e-30)
                stat[chunk % 2].copy_(rel, non_blocking=True)
                ev[chunk % 2].record()
                if chunk > 0:
                    ev[(chunk - 1) % 2].synchronize()
                    change = float(stat[(chunk - 1) % 2])
                    if change < (tol if tol_override is None else tol_override):
                        break
                chunk += 1
        torch.cuda.synchronize()
        return s.cpu().numpy(), time.perf_counter() - t0, k, change

    def device_us_per_iter(eta, comp, n):
        """Device time of n back-to-back iterations (no termination checks), CUDA events."""
        nf, ntx, nrx = comp
        full = comp == (g.K, g.T, g.R)
        if not full:
            draws = [I.cartesian_minibatch(g.T, g.R, g.K, ntx, nrx, nf, seed=29, it=i) for i in range(n)]
            pairs = torch.from_numpy(np.stack([d[0] for d in draws])).to(dev)
            masks = torch.from_numpy(np.stack([d[1] for d in draws])).to(dev)
        s = torch.zeros(g.N, dtype=torch.complex64, device=dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for i in range(n):
            if full:
                ctx.pgm_step(y, s, eta, lam)
            else:
                ctx.spgm_step_freqs(y, s, pairs[i], masks[i], eta, lam, n_freq=nf)
        e1.record()
        torch.cuda.synchronize()
        return 1e3 * e0.elapsed_time(e1) / n

    pgm_comp = (g.K, g.T, g.R)
    for comp in comps:                      # warm-up: module loading and first launches
        solve(0.1 / L, comp, 8, fixed_iters=4)
    out["device_us_per_iteration"] = {
        "x".join(map(str, comp)): device_us_per_iter(0.1 / L, comp, 200 if comp == pgm_comp else 2000)
        for comp in comps}
    for rho in args.study_rho:
        eta = rho / L
        s_fp, _, k_fp, ch_fp = solve(eta, pgm_comp, 40000, tol_override=1e-6)
        s_pgm, t_pgm, k_pgm, ch_pgm = solve(eta, pgm_comp, 200000)
        row = {"eta_times_L": rho, "eta": eta, "alpha": eta * lam,
               "pgm_fixed_point": {"iterations": k_fp, "last_change": ch_fp, "tol": 1e-6},
               "pgm": {"iterations": k_pgm, "seconds": t_pgm, "last_change": ch_pgm,
                       "psnr_vs_fixed_point_db": metrics.psnr_magnitude(s_pgm, s_fp)}, "spgm": []}
        t443 = None
        for comp in comps[:-1]:
            s_, t_, k_, ch_ = solve(eta, comp, 1 << 16)
            row["spgm"].append({"composition_f_tx_rx": list(comp), "B": comp[0] * comp[1] * comp[2],
                                "iterations": k_, "seconds": t_, "last_change": ch_,
                                "converged": ch_ < tol, "speedup_vs_pgm": t_pgm / t_,
                                "psnr_vs_pgm_db": metrics.psnr_magnitude(s_, s_pgm),
                                "psnr_vs_fixed_point_db": metrics.psnr_magnitude(s_, s_fp)})
            if comp == (4, 4, 3):
                t443 = t_
        k_star = max(1, int(k_pgm * t443 / t_pgm))
        s_star, t_star, _, _ = solve(eta, pgm_comp, k_star, fixed_iters=k_star)
        row["pgm_star"] = {"iterations": k_star, "seconds": t_star,
                           "psnr_vs_pgm_db": metrics.psnr_magnitude(s_star, s_pgm)}
        out["runs"].append(row)
        print(json.dumps(row), flush=True)
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.study == "paper_like":
        run_paper_like(args)
        return
    if args.study == "time_to_nmse":
        from paper_2509_00774_gb300 import build as nb
        nb.build()
        print(json.dumps(time_to_oracle_nmse(include_mid=True)), flush=True)
        return
    if args.workload == "batched48" and args.impl != "reference":
        run_batched(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
