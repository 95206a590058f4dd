"""Write stored oracle values for the full-size workloads.

Calls only the CPU oracle (and the seeded input generator).  For each
workload it evaluates tau, the full ladder term R and E_L with the plain FP64
oracle and stores: E_L, the Frobenius norm of R, and the R columns
R[:, :, a, b] of a fixed list of (a, b) pairs.  Run from the repository root:
    python tests/golden/make_golden.py mid_o34_v400_n1600
With --dressed it stores the same columns of the t1-dressed term
(Eq. pp-Ladder-2) instead, from the oracle's per-column evaluation, in
<workload>_dressed.json:
    python tests/golden/make_golden.py --dressed mid_o34_v400_n1600
With --triples it stores the perturbative triples energy E(T) of Sec. II.A
in <workload>_triples.json:
    python tests/golden/make_golden.py --triples dimer_o10_v120_n480
With --grad it stores 1024 seeded entries each of dE_L/dtau and dE_L/dB (the
oracle's entry-wise analytic gradient, weights W = 2 t2 - t2^T) in
<workload>_grad.json:
    python tests/golden/make_golden.py --grad grad_o16_v200_n800
With --ragged it stores, for each of the 48 molecules of the ragged batch
(synthetic.ragged_batch), E_L, the Frobenius norm of R and four R columns, in
ragged48.json:
    python tests/golden/make_golden.py --ragged
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synthetic  # noqa: E402


def sample_pairs(v, n=12, seed=1234):
    rng = np.random.default_rng(seed)
    pa = rng.integers(0, v, size=n)
    pb = rng.integers(0, v, size=n)
    pa[0], pb[0] = 0, v - 1
    pa[1], pb[1] = v - 1, v - 1
    return [int(x) for x in pa], [int(x) for x in pb]


def main(name):
    w = synthetic.WORKLOADS[name]
    t0 = time.time()
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    tau = oracle.tau(x.t1, x.t2)
    R = oracle.ladder(x.B, tau)
    E = oracle.energy(R, x.t2)
    pa, pb = sample_pairs(w.v)
    cols = [R[:, :, a, b].tolist() for a, b in zip(pa, pb)]
    out = {
        "workload": name, "o": w.o, "v": w.v, "naux": w.naux, "seed": w.seed,
        "E_L": E, "R_fro": float(np.linalg.norm(R)),
        "pairs_a": pa, "pairs_b": pb, "R_cols": cols,
        "oracle_threads": oracle.threads(), "oracle_seconds": time.time() - t0,
        "note": "written by tests/golden/make_golden.py from the plain FP64 CPU oracle",
    }
    path = os.path.join(ROOT, "tests", "golden", name + ".json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "E_L", E, "seconds", time.time() - t0)


def main_dressed(name):
    w = synthetic.WORKLOADS[name]
    t0 = time.time()
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    tau = oracle.tau(x.t1, x.t2)
    pa, pb = sample_pairs(w.v)
    cols = oracle.ladder_dressed_pairs(x.B, x.B_ov, x.t1, tau, pa, pb)
    out = {
        "workload": name, "o": w.o, "v": w.v, "naux": w.naux, "seed": w.seed,
        "pairs_a": pa, "pairs_b": pb, "R_cols": cols.tolist(),
        "oracle_threads": oracle.threads(), "oracle_seconds": time.time() - t0,
        "note": "t1-dressed term; written by tests/golden/make_golden.py --dressed from the "
                "plain FP64 CPU oracle",
    }
    path = os.path.join(ROOT, "tests", "golden", name + "_dressed.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "dressed columns, seconds", time.time() - t0)


def main_triples(name):
    w = synthetic.WORKLOADS[name]
    t0 = time.time()
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    E = oracle.triples(x.B, x.B_ov, x.B_oo, x.t1, x.t2, x.e_occ, x.e_vir)
    out = {
        "workload": name, "o": w.o, "v": w.v, "naux": w.naux, "seed": w.seed, "E_T": E,
        "oracle_threads": oracle.threads(), "oracle_seconds": time.time() - t0,
        "note": "perturbative triples E(T); written by tests/golden/make_golden.py --triples from "
                "the plain FP64 CPU oracle",
    }
    path = os.path.join(ROOT, "tests", "golden", name + "_triples.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "E(T)", E, "seconds", time.time() - t0)


def main_grad(name, m=1024):
    w = synthetic.WORKLOADS[name]
    t0 = time.time()
    x = synthetic.make_inputs(w.o, w.v, w.naux, w.seed)
    tau = oracle.tau(x.t1, x.t2)
    W = oracle.energy_weights(x.t2)
    rng = np.random.default_rng(4321)
    i, j = rng.integers(0, w.o, m), rng.integers(0, w.o, m)
    c, d = rng.integers(0, w.v, m), rng.integers(0, w.v, m)
    P, xx, yy = rng.integers(0, w.naux, m), rng.integers(0, w.v, m), rng.integers(0, w.v, m)
    dtau = oracle.grad_tau_entries(x.B, W, i, j, c, d)
    dB = oracle.grad_B_entries(x.B, tau, W, P, xx, yy)
    out = {
        "workload": name, "o": w.o, "v": w.v, "naux": w.naux, "seed": w.seed,
        "dtau_index": [[int(a) for a in t] for t in (i, j, c, d)], "dtau": dtau.tolist(),
        "dB_index": [[int(a) for a in t] for t in (P, xx, yy)], "dB": dB.tolist(),
        "oracle_threads": oracle.threads(), "oracle_seconds": time.time() - t0,
        "note": "entries of dE_L/dtau and dE_L/dB for W = 2 t2 - t2^T; written by "
                "tests/golden/make_golden.py --grad from the plain FP64 CPU oracle",
    }
    path = os.path.join(ROOT, "tests", "golden", name + "_grad.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print(name, "gradient entries, seconds", time.time() - t0)


def main_ragged():
    t0 = time.time()
    mols = []
    for k, x in enumerate(synthetic.ragged_batch()):
        t1 = time.time()
        tau = oracle.tau(x.t1, x.t2)
        R = oracle.ladder(x.B, tau)
        pa, pb = sample_pairs(x.v, n=4, seed=1000 + k)
        mols.append({"o": x.o, "v": x.v, "naux": x.naux, "E_L": oracle.energy(R, x.t2),
                     "R_fro": float(np.linalg.norm(R)), "pairs_a": pa, "pairs_b": pb,
                     "R_cols": [R[:, :, a, b].tolist() for a, b in zip(pa, pb)]})
        print(k, x.o, x.v, x.naux, "E_L", mols[-1]["E_L"], "seconds", time.time() - t1, flush=True)
    out = {"workload": "ragged48", "first_seed": 100, "molecules": mols,
           "oracle_threads": oracle.threads(), "oracle_seconds": time.time() - t0,
           "note": "48-molecule ragged batch; written by tests/golden/make_golden.py --ragged "
                   "from the plain FP64 CPU oracle"}
    path = os.path.join(ROOT, "tests", "golden", "ragged48.json")
    with open(path, "w") as f:
        json.dump(out, f)
    print("ragged48 seconds", time.time() - t0)


if __name__ == "__main__":
    args = sys.argv[1:]
    if "--ragged" in args:
        main_ragged()
        sys.exit(0)
    run = (main_dressed if "--dressed" in args else main_triples if "--triples" in args
           else main_grad if "--grad" in args else main)
    for n in args:
        if not n.startswith("--"):
            run(n)
