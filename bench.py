"""Benchmark of the particle-particle ladder term on GB300.

One step = one pass of the whole path on one molecule's inputs already in HBM:
tau assembly, operand slicing / pair packing, the ladder kernels (the fused
kernel, or the storing and GEMM2 passes of the two-pass form, as the plan or
the autotuner's cache chooses; --form forces one), the unpacking of R, and the
FP64 ladder energy.  The headline metric is ladder TFLOP/s (algorithmic flops
of the symmetric/antisymmetric scheme / time) on the mid-size workload (o=34,
v=400, N_aux=1600) of the tensor-core mode that meets both tolerances, R to
1e-6 and |dE_L| <= 1 microhartree: the error-free split (LADDER_OZAKI, five
fixed-point BF16 slices).  BF16X6 (meets the R tolerance only), its one-kernel
fused form, BF16X3 and the FP64 path are timed on the same workload and
reported beside it, each with its measured |dE_L| and tolerance verdicts.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--dressed] [--lambda-only] [--backward] [--triples] [--tuning k=v,...]

--dressed also times the t1-dressed term (Eq. pp-Ladder-2), --lambda-only
the paper's lambda-only contraction (the ablation of the +- split) and
--backward the adjoint (dE/dtau, dE/dB) and --triples the perturbative
triples energy E(T), one step each on the same workload, under "others";
--tuning overrides the timed plan's launch parameters.

Under torchrun each rank runs its own replica of the workload on its own GPU
(the ladder term of one molecule is one GPU's work); value = all ranks' flops
/ max-over-ranks time.  --impl reference times the plain FP64 CPU oracle on a
bounded sample of the same workload (host cores) and prints the same line.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic  # noqa: E402

METRIC = "ladder TFLOP/s & ms/call, split-BF16 vs FP64 GPU path at |dE_L|<=1 uEh"
DEFAULT_WORKLOAD = "mid_o34_v400_n1600"
PRODUCTS = {"bf16x3": 3, "bf16x6": 6, "fp64": 1}
TOL_R = 1e-6      # relative Frobenius error of R, split modes
TOL_E = 1e-6      # |dE_L| in Hartree


def _ppos(n):
    return n * (n + 1) // 2


def xsym_pairs(v):
    """(row tile, column block pair) tile products of the symmetric-B form's
    distinct-tile pass: row tiles (iA, kk >= 2 iA) of 8-blocks, each against
    the column block pairs from its first row block pair on."""
    nb = (v + 15) // 16 * 2
    nbp = _ppos(nb)
    return sum(nbp - (_ppos(kk) + 2 * iA) for iA in range(nb // 2) for kk in range(2 * iA, nb))


def xsym_flops(v, naux):
    """Multiply-add flops of the distinct-tile pass per slice product: 128 x 64
    tiles over N_aux (the halves it computes but does not store included)."""
    return 2.0 * xsym_pairs(v) * 128 * 64 * naux


def vform_bytes(v, S):
    """Algorithmic bytes of the V+- formation: the distinct tiles read once
    (64 x 64 double-single each) and the S-slice V+- planes and their row
    scales written for every (ab tile, block pair)."""
    nb = (v + 15) // 16 * 2
    nbp = _ppos(nb)
    ntiles = sum(nb - 2 * i for i in range(nb // 2))
    return nbp * (nbp + 1) / 2 * 4096 * 8 + ntiles * nbp * 2 * (S * 128 * 64 * 2 + 128 * 4)


def products(mode, tun):
    """Slice products per multiply-add of a mode (issued tensor flops / F_alg)."""
    if mode == "ozaki":
        S = tun["oz_slices"]
        return S * (S + 1) // 2
    return PRODUCTS[mode]


def fp64_peak(dev):
    """FP64 DGEMM rate of this GPU (torch.matmul float64, n = 8192, best of
    3 after a warm-up), the roofline of the plain FP64 path."""
    import torch
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    c = a @ b
    torch.cuda.synchronize()
    best = None
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    del a, b, c
    torch.cuda.empty_cache()
    return {"tflops": 2.0 * n ** 3 / (best * 1e-3) / 1e12, "how": "torch.matmul float64 %d^3, best of 3" % n}
# FP32 CUDA-core peak of one GB300, from the unit counts and the maximum SM
# clock: 152 SMs x 128 FP32 lanes x 2 flops (FMA) x 2.07 GHz
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

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
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle
def oracle_sample(x, seconds_target: float):
    """Time the plain oracle on a bounded sample of (a, b) columns; return
    (seconds the full term would take at the sample's rate, the sample's own
    seconds, its description, threads, the sampled fraction of columns)."""
    import oracle
    tau = oracle.tau(x.t1, x.t2)
    nthr = oracle.threads()
    v = x.v
    rng = np.random.default_rng(0)
    # calibrate with one column per thread, then size the sample
    n0 = max(1, nthr)
    pa, pb = rng.integers(0, v, n0), rng.integers(0, v, n0)
    t = time.perf_counter()
    oracle.ladder_pairs(x.B, tau, pa, pb)
    dt = time.perf_counter() - t
    n = max(n0, int(n0 * seconds_target / max(dt, 1e-6)))
    n = min(n, v * v)
    pa, pb = rng.integers(0, v, n), rng.integers(0, v, n)
    t = time.perf_counter()
    oracle.ladder_pairs(x.B, tau, pa, pb)
    dt = time.perf_counter() - t
    full = dt * (v * v) / n
    return full, dt, "%d of %d (a,b) columns of R (all i,j), %.1f s" % (n, v * v, dt), nthr, n / (v * v)


def tuned_for(w, mode):
    """The autotuner's cached launch parameters for this shape and mode, if any."""
    if mode == "fp64":
        return None
    from paper_1810_08142_gb300 import tune
    return tune.lookup_mode(w.o, w.v, w.naux, mode)


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def ragged_parity(Rs, E):
    """Every member's E_L and four R columns against the stored oracle values
    (tests/golden/ragged48.json), or None where that file is absent."""
    path = os.path.join(ROOT, "tests", "golden", "ragged48.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        gold = json.load(f)["molecules"]
    Eh = E.cpu().numpy()
    dE, rel = [], []
    for k, g in enumerate(gold):
        cols = np.array(g["R_cols"])
        got = np.stack([Rs[k][:, :, a, b].cpu().numpy() for a, b in zip(g["pairs_a"], g["pairs_b"])])
        rel.append(float(np.linalg.norm(got - cols) / np.linalg.norm(cols)))
        dE.append(abs(float(Eh[k]) - g["E_L"]))
    return {"max_dE_L": max(dE), "molecules_dE_L_tol_met": sum(d <= TOL_E for d in dE),
            "max_rel_fro_sampled_cols": max(rel), "dE_L_tol": TOL_E, "dE_L_tol_met": max(dE) <= TOL_E}


def ragged_measure(steps, warmup, mode="bf16x6", fp64=True):
    """The 48-molecule ragged batch: one graph-replayed batched step
    (ladder_step_batched: tau, the ladder and E_L of every molecule), in
    BF16X6 with each member's autotuned launch parameters (against the plan's
    own rules) or in the error-free mode, and (fp64=True) 48 separate FP64
    steps, all on inputs in HBM; parity of the last step against the stored
    oracle values."""
    import torch
    import paper_1810_08142_gb300 as lad
    mols = synthetic.ragged_batch()
    F = sum(synthetic.falg(x.o, x.v, x.naux) for x in mols)
    dev = torch.device("cuda", 0)
    Bs, t1s, t2s = ([torch.from_numpy(getattr(x, a)).to(dev) for x in mols] for a in ("B", "t1", "t2"))
    taus = [torch.empty_like(t) for t in t2s]
    Rs = [torch.empty_like(t) for t in t2s]
    E = torch.empty(len(mols), dtype=torch.float64, device=dev)
    shapes = [(x.o, x.v, x.naux) for x in mols]

    def timed(batch):
        for _ in range(warmup):
            batch.step(Bs, t1s, t2s, taus, Rs, E)
        torch.cuda.synchronize()
        batch.check_device()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            batch.step(Bs, t1s, t2s, taus, Rs, E)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    tuned = mode == "bf16x6"
    # the error-free batch uses each member's a <-> c symmetry of B (the
    # generator's B has it), and its general form is timed beside it
    sym = mode == "ozaki"
    batch = lad.LadderBatch(shapes, mode="tuned" if tuned else mode, sym_b=sym)
    ms = timed(batch)
    parity = ragged_parity(Rs, E)
    ntuned = sum(t is not None for t in batch.tunings)
    ntwo = sum(bool(t and t["two_pass"]) for t in batch.tunings)
    batch.close()
    del batch
    torch.cuda.empty_cache()
    default_ms = general_ms = None
    if tuned or sym:
        b2 = lad.LadderBatch(shapes, mode=mode)
        if tuned:
            default_ms = timed(b2)
        else:
            general_ms = timed(b2)
        b2.close()
        del b2
        torch.cuda.empty_cache()
    out = {"mode": mode, "ms_per_step": ms, "tflops": F / (ms * 1e-3) / 1e12, "molecules": len(mols),
           "falg_total": F, "parity": parity,
           "call": "ladder_step_batched (tau, ladder, E_L per molecule, one CUDA graph)",
           "tuning": "per-member autotuned (cache)" if tuned else "plan defaults",
           "members_tuned": ntuned if tuned else 0, "members_two_pass": ntwo if tuned else None,
           "plan_defaults": None if default_ms is None else
           {"ms_per_step": default_ms, "tflops": F / (default_ms * 1e-3) / 1e12},
           "sym_b": sym, "general_form": None if general_ms is None else
           {"ms_per_step": general_ms, "tflops": F / (general_ms * 1e-3) / 1e12}}
    if fp64:
        plans = [lad.Ladder(x.o, x.v, x.naux, mode="fp64") for x in mols]
        Es = [torch.empty((), dtype=torch.float64, device=dev) for _ in mols]

        def fp64_steps():
            for L, B, t1, t2, tau, R, e in zip(plans, Bs, t1s, t2s, taus, Rs, Es):
                lad.ladder_tau(L.plan, t1, t2, tau)
                lad.ladder_apply(L.plan, B, tau, R)
                lad.ladder_energy(L.plan, R, t2, e)

        fp64_steps()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record()
        fp64_steps()
        f1.record()
        torch.cuda.synchronize()
        fms = f0.elapsed_time(f1)
        out["fp64_48_launches"] = {"ms_per_step": fms, "tflops": F / (fms * 1e-3) / 1e12,
                                   "launches": len(mols), "speedup": fms / ms}
        for L in plans:
            L.close()
    return out


def run_ragged(args):
    """--workload ragged48: the batch as the line's headline."""
    mode = args.mode if args.mode in ("ozaki", "bf16x6", "bf16x3") else "ozaki"
    r = ragged_measure(args.steps, args.warmup, mode, fp64=not args.no_fp64)
    line = {"metric": METRIC, "value": r["tflops"], "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16 fixed-point x5 slices, exact FP32 windows" if mode == "ozaki"
                      else mode + "-split"),
            "data": "synthetic",
            "config": {"workload": "ragged48", "mode": mode, "molecules": r["molecules"],
                       "falg_total": r["falg_total"], "tuning": r["tuning"], "members_tuned": r["members_tuned"],
                       "members_two_pass": r["members_two_pass"], "call": r["call"], "sym_b": r["sym_b"]},
            "parity": r["parity"],
            "others": {"fp64_48_launches": r.get("fp64_48_launches"), "plan_defaults": r["plan_defaults"],
                       "general_form": r["general_form"]}}
    print(json.dumps(line), flush=True)
    return 0


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# dominant kernel, from an ncu capture of the same kernel build on the same
# workload and tuning.  A configuration not listed here reports traffic null.
TRAFFIC = {
    ("mid_o34_v400_n1600", "bf16x6", "pass1", (4, 2, 7, 128)): 705.02e9 + 81.46e9,
    ("mid_o34_v400_n1600", "bf16x6", "pass2", (4, 2, 7, 128)): 278.50e9 + 11.65e9,
}


class Replicas:
    """Rank bookkeeping of a replica run: one process per GPU (torchrun sets
    WORLD_SIZE / RANK / LOCAL_RANK), no collective on the data path, a barrier
    around the timed region and the maximum over ranks of its time."""

    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self, sync=None) -> None:
        if self.dist is not None:
            self.dist.barrier()
        if sync is not None:
            sync()

    def max(self, x: float, device="cpu") -> float:
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def job_value(self, units_per_rank: float, max_ms: float) -> float:
        """Whole-job throughput: every rank's units over the slowest rank's time."""
        return self.world * units_per_rank / (max_ms * 1e-3)

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    w = synthetic.WORKLOADS[args.workload]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    F = synthetic.falg(w.o, w.v, w.naux)
    # one step = one bounded sample of the workload's (a, b) columns; the
    # line reports what was timed: the samples' throughput and duration
    per_step = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    flops, secs, fulls, samples, thr = 0.0, 0.0, [], [], 1
    for s in range(args.warmup + args.steps):
        full, dt, desc, thr, frac = oracle_sample(x, per_step)
        if s >= args.warmup:
            flops += F * frac
            secs += dt
            fulls.append(full)
            samples.append(desc)
    val = flops / secs / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "o": w.o, "v": w.v, "naux": w.naux, "seed": w.seed,
                   "step": "a bounded sample of (a, b) columns of R (all i, j) of the workload"},
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
                         "sample": samples[-1],
                         "full_term_s_at_this_rate": statistics.mean(fulls)},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--mode", default="ozaki", choices=["ozaki", "bf16x3", "bf16x6", "fp64"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64-path comparison")
    ap.add_argument("--general-b", action="store_true",
                    help="error-free mode: do not use the a<->c symmetry of B (the generator's B has it); "
                         "the general form then runs as the headline")
    ap.add_argument("--no-others", action="store_true", help="skip every comparison mode")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tuning", default="",
                    help="override launch parameters of the timed plan: key=value,... (ladder_tuning fields)")
    ap.add_argument("--lambda-only", action="store_true",
                    help="also time the paper's lambda-only contraction (ablation of the +- split)")
    ap.add_argument("--triples", action="store_true",
                    help="also time the perturbative triples energy E(T) (Sec. II.A) on the same molecule")
    ap.add_argument("--ccsd", action="store_true",
                    help="also time the CCSD iteration (Jacobi + DIIS, ladder in the error-free mode) on the "
                         "same molecule, where its spin-orbital integrals fit")
    ap.add_argument("--backward", action="store_true",
                    help="also time the adjoint (dE/dtau and dE/dB for W = 2t - t^T) on the same workload")
    ap.add_argument("--dressed", action="store_true",
                    help="also time the t1-dressed term (Eq. pp-Ladder-2) on the same workload")
    ap.add_argument("--form", default="auto", choices=["auto", "fused", "two-pass"],
                    help="split-BF16 form: the plan's (or tuner's) choice, the one-kernel fused form "
                         "(integral tiles stay on chip), or the two-pass form (V+- stored in HBM)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ragged48":
        return run_ragged(args)

    import torch
    import paper_1810_08142_gb300 as lad

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rep = Replicas("nccl")
    world, rank, local = rep.world, rep.rank, rep.local

    def barrier():
        rep.barrier(torch.cuda.synchronize)

    def max_over_ranks(x: float) -> float:
        return rep.max(x, device="cuda")

    w = synthetic.WORKLOADS[args.workload]
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    F = synthetic.falg(w.o, w.v, w.naux)
    F1 = synthetic.falg_gemm1(w.o, w.v, w.naux)
    dev = torch.device("cuda", local)
    t1 = torch.from_numpy(x.t1).to(dev)
    t2 = torch.from_numpy(x.t2).to(dev)
    B = torch.from_numpy(x.B).to(dev)
    tau = torch.empty_like(t2)
    R = torch.empty_like(t2)
    E = torch.empty((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    pk, pk_kind = peaks()

    # stored oracle values of this workload (tests/golden/make_golden.py)
    gold = None
    gpath = os.path.join(ROOT, "tests", "golden", args.workload + ".json")
    if os.path.exists(gpath):
        with open(gpath) as f:
            gold = json.load(f)

    def parity_of(E_val):
        """|dE_L| and the sampled-column error of R against the stored oracle
        values, with the two tolerance verdicts."""
        if gold is None:
            return None
        Rh = R.cpu().numpy()
        cols = np.array(gold["R_cols"])
        got = np.stack([Rh[:, :, a, b] for a, b in zip(gold["pairs_a"], gold["pairs_b"])])
        rel = float(np.linalg.norm(got - cols) / np.linalg.norm(cols))
        dE = abs(E_val - gold["E_L"])
        return {"dE_L": dE, "E_L": gold["E_L"], "rel_fro_sampled_cols": rel,
                "max_rel_sampled_cols": float(np.abs(got - cols).max() / np.abs(cols).max()),
                "rel_fro_norm": abs(float(np.linalg.norm(Rh)) - gold["R_fro"]) / gold["R_fro"],
                "R_tol": TOL_R, "dE_L_tol": TOL_E, "R_tol_met": rel <= TOL_R, "dE_L_tol_met": dE <= TOL_E}

    def plan_tuning(mode, form="auto"):
        tun = tuned_for(w, mode)
        if form != "auto" and mode in ("bf16x3", "bf16x6"):
            tun = dict(tun or {}, two_pass=int(form == "two-pass"), ksplit=0)
        return tun

    def step(Lx):
        lad.ladder_tau(Lx.plan, t1, t2, tau)
        lad.ladder_apply(Lx.plan, B, tau, R)
        lad.ladder_energy(Lx.plan, R, t2, E)

    def roofline(mode, tun, pass1_ms, pass2_ms, ladder_ms, two_pass):
        """The dominant kernel against its peak (bf16 sustained for the tensor
        modes, the measured DGEMM rate for the FP64 path)."""
        prod = products(mode, tun)
        if mode == "fp64":
            return {"bound": "fp64", "achieved": F / (ladder_ms * 1e-3) / 1e12, "peak": None,
                    "unit": "TFLOP/s", "frac": None, "traffic": None}
        peak = pk["bf16_tflops_sustained"]
        if two_pass:
            nS = tun["oz_slices"] if mode == "ozaki" else (2 if mode == "bf16x3" else 3)
            k1 = ("oz_vstore_kernel<%d> (GEMM1 + V+- store)" % nS if mode == "ozaki"
                  else "ladder_tc_kernel<%d,false,true> (GEMM1 + V store)" % nS)
            k2 = ("oz_gemm2_kernel<%d> (GEMM2 from stored V+-)" % nS if mode == "ozaki"
                  else "ladder_gemm2_kernel<%d> (GEMM2 from stored V)" % nS)
            if pass1_ms >= pass2_ms:
                kname, kflops, kms, kkey = k1, F1, pass1_ms, "pass1"
            else:
                kname, kflops, kms, kkey = k2, F - F1, pass2_ms, "pass2"
            key = (args.workload, mode, kkey, tuple(tun.get(k) for k in ("kc", "s_pieces", "ksplit", "flush_every"))
                   if mode != "ozaki" else (tun["oz_slices"], tun["ksplit"]))
            achieved = prod * kflops / (kms * 1e-3) / 1e12
            return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": TRAFFIC.get(key), "traffic_unit": "bytes per launch",
                    "kernel": kname, "kernel_ms": kms,
                    "other_pass": {"kernel": k2 if kkey == "pass1" else k1,
                                   "ms": pass2_ms if kkey == "pass1" else pass1_ms,
                                   "frac": prod * ((F - F1) if kkey == "pass1" else F1) /
                                   ((pass2_ms if kkey == "pass1" else pass1_ms) * 1e-3) / 1e12 / peak},
                    "both_passes_frac": prod * F / ((pass1_ms + pass2_ms) * 1e-3) / 1e12 / peak,
                    "note": "achieved = %d slice products x (that pass's share of F_alg: 2 P+(v) v^2 N for "
                            "GEMM1, the rest for GEMM2) / its CUDA-event time; peak = bf16 sustained (%s)"
                            % (prod, pk_kind)}
        achieved = prod * F / (ladder_ms * 1e-3) / 1e12
        return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None,
                "kernel": "ladder_tc_kernel<%d,false,false>" % (2 if mode == "bf16x3" else 3),
                "note": "achieved = %d x F_alg / fused-kernel time; peak = bf16 sustained (%s)" % (prod, pk_kind)}

    def roofline_sym(tun, xs_ms, fm_ms, p2_ms):
        """The symmetric-B form's three kernels (distinct tiles, V+- formation,
        GEMM2) against their peaks; the slowest one is the dominant kernel."""
        prod = products("ozaki", tun)
        nS = tun["oz_slices"]
        peak, hbm = pk["bf16_tflops_sustained"], pk["hbm_gbs"]
        ax = prod * xsym_flops(w.v, w.naux) / (xs_ms * 1e-3) / 1e12
        a2 = prod * (F - F1) / (p2_ms * 1e-3) / 1e12
        bf = vform_bytes(w.v, nS)
        af = bf / (fm_ms * 1e-3) / 1e9
        ks = [{"bound": "tensor", "achieved": ax, "peak": peak, "unit": "TFLOP/s", "frac": ax / peak,
               "traffic": None, "kernel": "oz_xsym_kernel<%d> (distinct integral tiles)" % nS, "kernel_ms": xs_ms,
               "note": "achieved = %d slice products x 2 x 128 x 64 x N_aux per (row tile, column block "
                       "pair) computed (%d of them) / CUDA-event time; peak = bf16 sustained (%s)"
                       % (prod, xsym_pairs(w.v), pk_kind)},
              {"bound": "hbm", "achieved": af, "peak": hbm, "unit": "GB/s", "frac": af / hbm,
               "traffic": None, "kernel": "oz_vform_kernel<%d> (V+- formed from the distinct tiles)" % nS,
               "kernel_ms": fm_ms,
               "note": "achieved = distinct tiles read once + V+- slices and scales written (%.1f GB) / "
                       "CUDA-event time; peak = HBM copy (%s)" % (bf / 1e9, pk_kind)},
              {"bound": "tensor", "achieved": a2, "peak": peak, "unit": "TFLOP/s", "frac": a2 / peak,
               "traffic": None, "kernel": "oz_gemm2_kernel<%d> (GEMM2 from stored V+-)" % nS, "kernel_ms": p2_ms,
               "note": "achieved = %d slice products x 2 [P+(o) P+(v)^2 + P-(o) P-(v)^2] / CUDA-event time; "
                       "peak = bf16 sustained (%s)" % (prod, pk_kind)}]
        dom = max(ks, key=lambda k: k["kernel_ms"])
        return dict(dom, kernels=ks)

    # ---------------------------------------------------------------- headline
    tuning = plan_tuning(args.mode, args.form)
    sym = args.mode == "ozaki" and not args.general_b
    if sym:
        # the generator symmetrises B^P_ac in a <-> c, as RI factors of real
        # orbitals are: the plan uses it (and checks it on the device)
        tuning = dict(tuning or {}, sym_b=1)
    if args.tuning and args.mode != "fp64":
        # explicit overrides, e.g. --tuning flush_every=32,kc=8 or oz_slices=6
        tuning = dict(tuning or {}, **{k: int(v) for k, v in
                                      (kv.split("=") for kv in args.tuning.split(","))})
    L = lad.Ladder(w.o, w.v, w.naux, mode=args.mode, device=dev, tuning=tuning)
    lad.ladder_set_timing(L.plan, True)
    for _ in range(args.warmup):
        step(L)
    torch.cuda.synchronize()
    L.check_device()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stages, passes, symt = [], [], []
    e0.record(stream)
    for _ in range(args.steps):
        step(L)
        stages.append(lad.ladder_timing(L.plan))  # waits for this step's events
        passes.append(lad.ladder_timing_passes(L.plan))
        if sym:
            symt.append(lad.ladder_timing_sym(L.plan))
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    L.check_device()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms)
    value = rep.job_value(F, ms) / 1e12
    ladder_ms = statistics.mean(f[1] for f in stages)
    prep_ms = statistics.mean(f[0] for f in stages)
    unpack_ms = statistics.mean(f[2] for f in stages)
    pass1_ms = statistics.mean(f[0] for f in passes)
    pass2_ms = statistics.mean(f[1] for f in passes)
    tun = lad.ladder_get_tuning(L.plan).as_dict() if args.mode != "fp64" else None
    two_pass = bool(tun and tun["two_pass"])
    E_val = float(E.item())
    parity = parity_of(E_val)
    if sym:
        xsym_ms = statistics.mean(f[0] for f in symt)
        form_ms = statistics.mean(f[1] for f in symt)
        roof = roofline_sym(tun, xsym_ms, form_ms, pass2_ms)
    else:
        roof = roofline(args.mode, tun, pass1_ms, pass2_ms, ladder_ms, two_pass)
    prod = products(args.mode, tun) if tun else 1

    # ---------------------------------------------------------------- end to end
    # through the C ABI's host-buffer call: every step copies B and tau from
    # pinned host memory, runs the ladder, copies R back to pinned host memory
    # and synchronises (ladder_apply_host), then forms E_L from the device
    # copy of R and reads it back.  tau's host copy is an input here (made
    # once on the device before the timed region).
    e2e = None
    if not args.no_e2e:
        lad.ladder_tau(L.plan, t1, t2, tau)
        h_B = torch.from_numpy(x.B).pin_memory()
        h_tau = tau.cpu().pin_memory()
        h_R = torch.empty_like(h_tau).pin_memory()
        d_B, d_tau, d_R = torch.empty_like(B), torch.empty_like(tau), torch.empty_like(R)

        def e2e_step():
            lad.ladder_apply_host(L.plan, h_B, h_tau, h_R, d_B, d_tau, d_R)
            lad.ladder_energy(L.plan, d_R, t2, E)
            return float(E.item())

        e2e_step()
        # the pinned copy rates this box gives (outside the timed region):
        # the e2e number moves with them from box to box
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(stream)
        d_B.copy_(h_B, non_blocking=True)
        c1.record(stream)
        h_R.copy_(d_R, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        copy_gbs = {"h2d_GBps": h_B.numel() * 8 / (c0.elapsed_time(c1) * 1e-3) / 1e9,
                    "d2h_GBps": h_R.numel() * 8 / (c1.elapsed_time(c2) * 1e-3) / 1e9}
        barrier()
        q0 = time.perf_counter()
        for _ in range(args.steps):
            E_e2e = e2e_step()
        barrier()
        ems = max_over_ranks((time.perf_counter() - q0) * 1e3 / args.steps)
        e2e = {"value": rep.job_value(F, ems) / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": (h_B.numel() + h_tau.numel()) * 8,
               "d2h_bytes_per_step": h_R.numel() * 8 + 8, "ms_per_step": ems,
               "call": "ladder_apply_host (B, tau in; R out; synchronises) + ladder_energy",
               "R_host_matches_device": bool(torch.equal(h_R, R.cpu())), "E_L": E_e2e,
               "pinned_copy_rates": copy_gbs}
        del d_B, d_tau, d_R, h_B, h_tau, h_R
    L.close()
    del L
    torch.cuda.empty_cache()

    # ---------------------------------------------------------------- other modes
    extra = {}
    others = []
    if not args.no_others:
        if sym:
            others.append("ozaki_general")  # the error-free mode without B's symmetry
        if args.mode != "bf16x6":
            others.append("bf16x6")
        if args.mode in ("ozaki", "bf16x6"):
            others.append("bf16x6_fused")  # the one-kernel form (integral tiles on chip)
            others.append("bf16x3")
        if args.mode != "fp64" and not args.no_fp64:
            others.append("fp64")
        if args.dressed and args.mode != "fp64":
            others.insert(0, args.mode + "_dressed")  # the t1-dressed term (Eq. pp-Ladder-2)
        if args.lambda_only and args.mode in ("bf16x3", "bf16x6"):
            others.insert(0, args.mode + "_lambda")  # the paper's lambda-only contraction (ablation)
    B_ov = None
    for m in others:
        base = m.split("_")[0]
        mt = plan_tuning(base) if base != "fp64" else None
        if m.endswith("_dressed"):
            # the dressed term's B - mbar is not symmetric: the general form
            Lm = lad.Ladder(w.o, w.v, w.naux, mode=base, device=dev, tuning=dict(tun or {}, sym_b=0) if tun else None,
                            dressed=True)
            B_ov = torch.from_numpy(x.B_ov).to(dev)
        elif m.endswith("_lambda"):
            Lm = lad.Ladder(w.o, w.v, w.naux, mode=base, device=dev,
                            tuning={**(mt or {}), "two_pass": 1, "lambda_only": 1, "ksplit": 0})
        elif m == "ozaki_general":
            Lm = lad.Ladder(w.o, w.v, w.naux, mode=base, device=dev, tuning=mt)
        elif m.endswith("_fused"):
            Lm = lad.Ladder(w.o, w.v, w.naux, mode=base, device=dev,
                            tuning={**(mt or {}), "two_pass": 0, "ksplit": 0})
        else:
            Lm = lad.Ladder(w.o, w.v, w.naux, mode=base, device=dev, tuning=mt)
        lad.ladder_set_timing(Lm.plan, True)
        run = step
        if m.endswith("_dressed"):
            def run(Lx):
                lad.ladder_tau(Lx.plan, t1, t2, tau)
                lad.ladder_apply_dressed(Lx.plan, B, B_ov, t1, tau, R)
                lad.ladder_energy(Lx.plan, R, t2, E)
        if base != "fp64":
            run(Lm)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        run(Lm)
        a1.record(stream)
        torch.cuda.synchronize()
        Lm.check_device()
        mms = a0.elapsed_time(a1)
        tm = lad.ladder_timing(Lm.plan)
        p1, p2 = lad.ladder_timing_passes(Lm.plan)
        mtun = lad.ladder_get_tuning(Lm.plan).as_dict() if base != "fp64" else None
        m_two = bool(mtun and mtun["two_pass"])
        ent = {"ms_per_step": mms, "tflops": F / (mms * 1e-3) / 1e12, "ladder_ms": tm[1],
               "E_L": float(E.item()), "steps": 1, "tuning": mtun,
               "form": None if mtun is None else ("two-pass" if m_two else "fused")}
        if m_two:
            ent["pass1_ms"], ent["pass2_ms"] = p1, p2
        if not m.endswith("_dressed"):
            ent["parity"] = parity_of(float(E.item()))
        if not m.endswith("_dressed") and not m.endswith("_lambda"):
            ent["roofline"] = roofline(base, mtun, p1, p2, tm[1], m_two)
        if m.endswith("_dressed"):
            # tau, B - mbar, the rank-o correction and the energy
            ent["outside_ladder_ms"] = mms - tm[0] - tm[1] - tm[2]
            bd_ms, corr_ms = lad.ladder_timing_dressing(Lm.plan)
            o_, v_, n_ = w.o, w.v, w.naux
            ov = o_ * v_
            # algorithmic flops of the correction: (kc|ld) (symmetric), X, Y, C
            fc = 2.0 * (ov * (ov + 1) / 2 * n_ + o_ ** 4 * v_ ** 2 + o_ ** 4 * v_ + o_ ** 3 * v_ ** 2)
            ent["bd_ms"], ent["correction_ms"] = bd_ms, corr_ms
            ent["bd_gbs"] = 16.0 * n_ * v_ * v_ / (bd_ms * 1e-3) / 1e9
            ent["correction_roofline"] = {
                "bound": "alu", "achieved": fc / (corr_ms * 1e-3) / 1e12, "peak": FP32_ALU_TFLOPS,
                "unit": "TFLOP/s", "frac": fc / (corr_ms * 1e-3) / 1e12 / FP32_ALU_TFLOPS,
                "note": "CUDA-core GEMMs; peak = 152 SMs x 128 FP32 lanes x 2 flops x 2.07 GHz"}
        extra[m] = ent
        Lm.close()
        del Lm
        torch.cuda.empty_cache()
    if "fp64" in extra:
        extra["speedup_vs_fp64"] = extra["fp64"]["ms_per_step"] / ms
        dg = fp64_peak(dev)
        extra["fp64"]["roofline"].update({"peak": dg["tflops"], "frac": extra["fp64"]["roofline"]["achieved"] / dg["tflops"],
                                          "peak_how": dg["how"] + " (measured in this run)"})
    if not args.no_others and args.workload == DEFAULT_WORKLOAD:
        # the 48-molecule ragged batch (one graph per step), timed in every
        # default run; its 48 FP64 steps (~40 s) only with --workload ragged48
        extra["ragged48"] = ragged_measure(max(1, args.steps), max(1, args.warmup), fp64=False)
        torch.cuda.empty_cache()
        extra["ragged48_ozaki"] = ragged_measure(max(1, args.steps), max(1, args.warmup), mode="ozaki",
                                                 fp64=False)
        torch.cuda.empty_cache()
    if args.triples:
        # the perturbative triples energy E(T) on the same molecule: BF16X6
        # (tcgen05 W contractions) and FP32 always, FP64 where its work stays
        # below ~1 TFLOP
        B_ov = torch.from_numpy(x.B_ov).to(dev)
        B_oo = torch.from_numpy(x.B_oo).to(dev)
        e_occ = torch.from_numpy(x.e_occ).to(dev)
        e_vir = torch.from_numpy(x.e_vir).to(dev)
        nsorted = w.o * (w.o + 1) * (w.o + 2) // 6
        ft = 12.0 * nsorted * w.v ** 3 * (w.v + w.o)
        tr = {"flops": ft, "note": "flops = 12 v^3 (v + o) per sorted triple i >= j >= k, o(o+1)(o+2)/6 "
                                   "triples: the W contractions evaluated"}
        for prec in ("bf16x6", "fp32", "fp64"):
            if prec == "fp64" and ft > 1e12:
                continue
            if prec == "bf16x6" and w.v > 256:
                continue
            n_ws = lad.ladder_triples_workspace_size(w.o, w.v, w.naux, lad.TRIPLES_PRECISION[prec])
            ws = torch.empty(n_ws, dtype=torch.uint8, device=dev)
            args_t = (B, B_ov, B_oo, t1, t2, e_occ, e_vir)
            Et = lad.triples(*args_t, precision=prec, workspace=ws)  # warm-up
            torch.cuda.synchronize()
            c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            Et = lad.triples(*args_t, precision=prec, workspace=ws)
            c1.record(stream)
            torch.cuda.synchronize()
            tms = c0.elapsed_time(c1)
            tr[prec] = {"ms": tms, "tflops": ft / (tms * 1e-3) / 1e12, "E_T": float(Et.item())}
            if prec == "fp32":
                tr[prec]["roofline"] = {"bound": "alu", "achieved": ft / (tms * 1e-3) / 1e12,
                                        "peak": FP32_ALU_TFLOPS, "unit": "TFLOP/s",
                                        "frac": ft / (tms * 1e-3) / 1e12 / FP32_ALU_TFLOPS}
            if prec == "bf16x6":
                # six slice products per multiply-add on the bf16 tensor pipe;
                # the whole call's time (integrals, slicing and the energy
                # kernel included) bounds the W kernels' share from below
                ach = 6.0 * ft / (tms * 1e-3) / 1e12
                tr[prec]["roofline"] = {"bound": "tensor", "achieved": ach, "peak": pk["bf16_tflops_sustained"],
                                        "unit": "TFLOP/s", "frac": ach / pk["bf16_tflops_sustained"],
                                        "note": "6 x W flops / whole-call time; peak = bf16 sustained (%s)" % pk_kind}
            del ws
            torch.cuda.empty_cache()
        if "fp64" in tr:
            for prec in ("fp32", "bf16x6"):
                if prec in tr:
                    tr[prec + "_rel_diff"] = abs(tr[prec]["E_T"] - tr["fp64"]["E_T"]) / abs(tr["fp64"]["E_T"])
        extra["triples"] = tr
    if args.ccsd:
        # the closed-shell CCSD iteration around the ladder (FP64 contractions,
        # the ladder of every step in the error-free mode)
        nb = lad.ladder_ccsd_workspace_size(w.o, w.v, w.naux, 3)
        if nb > 120e9:
            extra["ccsd"] = {"skipped": "spin-orbital integrals need %.0f GB" % (nb / 1e9)}
        else:
            # the generator's integrals grow with N_aux (at the dimer size its
            # MP2 amplitudes reach 0.87): the RI factors are scaled by 0.1 here,
            # integrals by 0.01, so that the iteration converges
            lam = 0.1
            Bs = torch.from_numpy(lam * x.B).to(dev)
            B_ov = torch.from_numpy(lam * x.B_ov).to(dev)
            B_oo = torch.from_numpy(lam * x.B_oo).to(dev)
            e_occ = torch.from_numpy(x.e_occ).to(dev)
            e_vir = torch.from_numpy(x.e_vir).to(dev)
            Lc = lad.Ladder(w.o, w.v, w.naux, mode="ozaki", device=dev, tuning={"sym_b": 1})
            wsc = torch.empty(nb, dtype=torch.uint8, device=dev)
            c0 = time.perf_counter()
            _, _, Ec, itc = lad.ccsd(Lc, Bs, B_ov, B_oo, e_occ, e_vir, tol=1e-10, max_iter=60, workspace=wsc)
            cs = time.perf_counter() - c0
            Lc.check_device()
            extra["ccsd"] = {"E_CCSD": Ec, "iterations": itc, "converged": itc < 60, "seconds": cs,
                             "ms_per_iteration": cs * 1e3 / itc, "workspace_GB": nb / 1e9, "ladder_mode": "ozaki",
                             "diis": 3, "tol": 1e-10, "B_scale": lam,
                             "note": "wall time of the whole solve (integrals included); the call synchronises"}
            del wsc, Lc
            torch.cuda.empty_cache()
    if args.backward and args.mode in ("bf16x3", "bf16x6", "ozaki"):
        # the adjoint of E_L: dE/dtau (the transposed ladder) and dE/dB (Gamma
        # stored once, then contracted), in the same split mode and tuning, or
        # in BF16X6 behind the error-free forward (which has no dE/dB), and
        # the error-free dE/dtau of the symmetric-B form
        bmode = "bf16x6" if args.mode == "ozaki" else args.mode
        Lb = lad.Ladder(w.o, w.v, w.naux, mode=bmode, device=dev,
                        tuning=tuned_for(w, bmode) if args.mode == "ozaki" else tun, backward=True)
        lad.ladder_tau(Lb.plan, t1, t2, tau)
        Wt = Lb.weights(t2)
        dt, db = torch.empty_like(tau), torch.empty_like(B)
        bw = {}
        for name, a, b in (("dtau", dt, None), ("dB", None, db), ("both", dt, db)):
            lad.ladder_backward(Lb.plan, B, tau, Wt, a, b)  # warm-up
            torch.cuda.synchronize()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            lad.ladder_backward(Lb.plan, B, tau, Wt, a, b)
            b1.record(stream)
            torch.cuda.synchronize()
            bw[name + "_ms"] = b0.elapsed_time(b1)
        Lb.check_device()
        bw["dtau_tflops"] = F / (bw["dtau_ms"] * 1e-3) / 1e12
        bw["mode"] = bmode
        bw["note"] = "dtau_tflops counts F_alg (the transposed ladder has the forward's flops)"
        Lb.close()
        del Lb
        torch.cuda.empty_cache()
        if sym:
            # error-free dE/dtau: with B symmetric the transposed ladder is the
            # forward of W, which the headline's error-free plan computes
            Le = lad.Ladder(w.o, w.v, w.naux, mode="ozaki", device=dev, tuning=tuning)
            lad.ladder_backward(Le.plan, B, tau, Wt, dt, None)  # warm-up
            torch.cuda.synchronize()
            b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            b0.record(stream)
            lad.ladder_backward(Le.plan, B, tau, Wt, dt, None)
            b1.record(stream)
            torch.cuda.synchronize()
            Le.check_device()
            bw["dtau_error_free_ms"] = b0.elapsed_time(b1)
            bw["dtau_error_free_tflops"] = F / (bw["dtau_error_free_ms"] * 1e-3) / 1e12
            Le.close()
            del Le
            torch.cuda.empty_cache()
        extra["backward"] = bw

    cpu = None
    if rank == 0 and not args.no_cpu:
        full, dt, desc, thr, frac = oracle_sample(x, 15.0)
        cpu = {"value": F * frac / dt / 1e12, "unit": "TFLOP/s", "cores": thr, "kind": "oracle",
               "sample": desc, "sample_s": dt, "full_term_s_at_this_rate": full}

    if rank == 0:
        # per step: tau; symmetry check (symmetric form), B row scales, B slices,
        # tau+- slices, the ladder passes (distinct tiles + V+- formation, or
        # GEMM1), GEMM2, unpack; the two energy kernels
        launches = 11 if sym else {"ozaki": 9, "fp64": 4}.get(args.mode, 9 if two_pass else 7)
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": ("bf16 fixed-point x%d slices, exact FP32 windows" % tun["oz_slices"] if args.mode == "ozaki"
                      else "bf16x%d-split" % prod if args.mode != "fp64" else "f64"),
            "data": "synthetic",
            "config": {"workload": args.workload, "o": w.o, "v": w.v, "naux": w.naux,
                       "seed": w.seed, "mode": args.mode, "parallelism": "replicas",
                       "tuning": tun, "slice_products": prod,
                       "form": None if tun is None else (
                           "symmetric B: distinct integral tiles once, V+- formed from them and stored in HBM"
                           if sym else "two-pass (V+- stored in HBM)" if two_pass
                           else "fused (integral tiles on chip)"),
                       "l2": "inputs larger than L2 (B %.2f GB, tau %.2f GB)"
                             % (B.numel() * 8 / 1e9, tau.numel() * 8 / 1e9)},
            "stages_ms": {"prep": prep_ms, "ladder": ladder_ms, "unpack": unpack_ms,
                          "pass1": pass1_ms if two_pass else None,
                          "pass2": pass2_ms if two_pass else None,
                          "xsym": xsym_ms if sym else None, "vform": form_ms if sym else None},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": launches * args.steps, "parity": parity, "E_L": E_val, "others": extra,
        }
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
