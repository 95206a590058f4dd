"""Autotuner of the tensor-core ladder modes.

For one shape (o, v, N_aux) it tries each tensor-core mode (BF16X3, BF16X6
with several launch parameters: GEMM1 chain length kc, GEMM2 pieces per fresh
accumulator, flush interval, the fused or the two-pass form; the error-free
split with 5 or 6 slices) and keeps the fastest one whose errors, measured
against the FP64 GPU path on seeded random inputs, stay below half of both
bounds (a margin for inputs that differ from the proxy's):
  R:    relative Frobenius error <= tol (default 1e-6);
  E_L:  |dE| / sum |R W| <= etol_rel for the energy E = sum R W with random
        pair-symmetric weights W (default 1e-13: the metric's 1 microhartree at
        E_L ~ 3e6, where the coherent synthetic E_L is about sum |R W|, with a
        factor three in hand; 0 drops the energy bound).
The accumulation error of a candidate depends on its chain lengths and on
N_aux, not on v, so accuracy is measured on a proxy with the same o and N_aux
and v capped at 64 (where the FP64 path is quick); speed on the full shape.

Results go to a JSON cache ($LADDER_TUNE_CACHE, else tune_cache.json next to
this file) keyed by "o,v,naux": the selected mode and launch parameters
(Ladder(..., mode="tuned") reads them) and, under "by_mode", the fastest
parameters of each mode that meet the R bound (what a caller who fixes the
mode, e.g. a BF16X6 batch, wants).

    python -m paper_1810_08142_gb300.tune 34 400 1600 [--tol 1e-6]
"""
from __future__ import annotations

import argparse
import json
import os

CACHE_DEFAULT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def cache_path() -> str:
    return os.environ.get("LADDER_TUNE_CACHE", CACHE_DEFAULT)


def _load() -> dict:
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _key(o, v, naux) -> str:
    return "%d,%d,%d" % (o, v, naux)


def lookup_mode(o: int, v: int, naux: int, mode: str):
    """The cached parameters of `mode` for this exact shape, or None."""
    e = _load().get(_key(o, v, naux))
    if not e:
        return None
    if mode in e.get("by_mode", {}):
        return e["by_mode"][mode]
    return e["tuning"] if e.get("mode") == mode else None


def lookup(o: int, v: int, naux: int):
    """(mode, tuning dict or None) for a shape: the cached entry of that shape,
    else of the nearest cached shape, else BF16X6 with its defaults."""
    c = _load()
    e = c.get(_key(o, v, naux))
    if e is None and c:
        def dist(k):
            oo, vv, nn = (int(s) for s in k.split(","))
            return abs(oo - o) / max(o, 1) + abs(vv - v) / max(v, 1) + abs(nn - naux) / max(naux, 1)
        e = c[min(c, key=dist)]
        e = dict(e)
        e["tuning"] = {k: val for k, val in e["tuning"].items() if k != "ksplit"}
    if e is None:
        return "bf16x6", None
    return e["mode"], e["tuning"]


def candidates(forms=(0,)):
    """(mode, tuning) pairs; `forms` lists the two_pass values to try."""
    out = [("ozaki", {"oz_slices": 5}), ("ozaki", {"oz_slices": 6})]
    for tp in forms:
        for kc in (16, 32):
            out.append(("bf16x3", {"kc": kc, "s_pieces": 4, "xy_split": 1, "two_pass": tp}))
        # the two-pass form keeps S double-buffered, so longer S chains pay off there;
        # its GEMM2 flushes cost time, so the flush interval is a candidate too
        for kc in ((4, 8) if tp else (2, 4, 8)):
            for sp in ((1, 2) if tp else (1, 2)):
                for fe in ((16, 64, 128) if tp else (64,)):
                    out.append(("bf16x6", {"kc": kc, "s_pieces": sp, "flush_every": fe, "xy_split": 1,
                                           "two_pass": tp}))
    return out


def _inputs(o, v, naux, seed, device):
    import torch
    g = torch.Generator(device=device).manual_seed(seed)
    B = torch.randn(naux, v, v, generator=g, device=device, dtype=torch.float64)
    B *= torch.exp(-3.0 * torch.arange(naux, device=device, dtype=torch.float64) / naux)[:, None, None] * 0.1
    tau = torch.randn(o, o, v, v, generator=g, device=device, dtype=torch.float64) * 1e-2
    tau = 0.5 * (tau + tau.permute(1, 0, 3, 2))
    return B.contiguous(), tau.contiguous()


def select(results, tol, etol_rel):
    """The fastest result within half of both bounds (etol_rel = 0: R only);
    if none qualifies, the most accurate in E (then R)."""
    ok = [r for r in results if r["err"] <= 0.5 * tol and (etol_rel <= 0 or r["eerr"] <= 0.5 * etol_rel)]
    if ok:
        return min(ok, key=lambda r: r["ms"])
    return min(results, key=lambda r: (r["eerr"], r["err"]) if etol_rel > 0 else (r["err"],))


def _time_ms(L, B, tau, R, reps):
    import torch
    L.apply(B, tau, R)
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.apply(B, tau, R)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune(o: int, v: int, naux: int, tol: float = 1e-6, etol_rel: float = 1e-13, reps: int = 2,
         seed: int = 0, write: bool = True, verbose: bool = True) -> dict:
    import torch
    from . import Ladder
    dev = torch.device("cuda")
    # accuracy proxy: same o and N_aux, v <= 64, against the FP64 path
    vp = min(v, 64)
    Bp, taup = _inputs(o, vp, naux, seed, dev)
    ref = Ladder(o, vp, naux, mode="fp64", device=dev).apply(Bp, taup)
    nref = torch.linalg.vector_norm(ref).item()
    g = torch.Generator(device=dev).manual_seed(seed + 7)
    Wp = torch.randn(ref.shape, generator=g, device=dev, dtype=torch.float64)
    Wp = 0.5 * (Wp + Wp.permute(1, 0, 3, 2))
    E_ref = torch.sum(ref * Wp).item()
    e_scale = torch.sum(torch.abs(ref * Wp)).item()
    B, tau = _inputs(o, v, naux, seed + 1, dev)
    R = torch.empty_like(tau)
    # both forms are candidates: the two-pass form can win even where the
    # fused kernel needs one chunk (its storing pass issues wider MMAs);
    # a form whose workspace does not fit the device is skipped below
    from . import ladder_get_tuning
    forms = (0, 1)
    results = []
    for mode, tun in candidates(forms):
        try:
            L = Ladder(o, v, naux, mode=mode, device=dev, tuning=tun)
        except (RuntimeError, MemoryError) as exc:  # workspace too large for the device
            if verbose:
                print("%-7s %-60s skipped (%s)" % (mode, tun, str(exc).splitlines()[0][:60]), flush=True)
            torch.cuda.empty_cache()
            continue
        Lp = Ladder(o, vp, naux, mode=mode, device=dev, tuning=tun)
        Rp = Lp.apply(Bp, taup)
        err = torch.linalg.vector_norm(Rp - ref).item() / nref
        eerr = abs(torch.sum(Rp * Wp).item() - E_ref) / e_scale
        Lp.close()
        full = ladder_get_tuning(L.plan).as_dict()
        ms = _time_ms(L, B, tau, R, reps)
        L.close()
        del L
        torch.cuda.empty_cache()
        results.append({"mode": mode, "tuning": full, "ms": ms, "err": err, "eerr": eerr})
        if verbose:
            print("%-7s %-60s %9.3f ms  rel-F %.2e  E %.2e" % (mode, full, ms, err, eerr), flush=True)
    # the proxy's inputs are not the caller's: keep a factor of two in hand
    best = select(results, tol, etol_rel)
    entry = dict(best, tol=tol, etol_rel=etol_rel, candidates=len(results))
    by_mode = {}
    for m in sorted({r["mode"] for r in results}):
        ok = [r for r in results if r["mode"] == m and r["err"] <= 0.5 * tol]
        if ok:
            by_mode[m] = min(ok, key=lambda r: r["ms"])["tuning"]
    entry["by_mode"] = by_mode
    if write:
        c = _load()
        c[_key(o, v, naux)] = entry
        with open(cache_path(), "w") as f:
            json.dump(c, f, indent=1, sort_keys=True)
    return entry


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("o", type=int, nargs="?")
    ap.add_argument("v", type=int, nargs="?")
    ap.add_argument("naux", type=int, nargs="?")
    ap.add_argument("--shapes", default="",
                    help="several shapes at once: 'o,v,naux o,v,naux ...'")
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--etol-rel", type=float, default=1e-13,
                    help="bound on |dE| / sum |R W| (0: select on R alone)")
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    shapes = [tuple(int(x) for x in t.split(",")) for t in a.shapes.split()]
    if a.o is not None:
        shapes.insert(0, (a.o, a.v, a.naux))
    for o, v, n in shapes:
        e = tune(o, v, n, tol=a.tol, etol_rel=a.etol_rel, reps=a.reps, verbose=len(shapes) == 1)
        print(json.dumps({"shape": [o, v, n], **e}), flush=True)


if __name__ == "__main__":
    main()
