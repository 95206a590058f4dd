"""Seeded synthetic inputs for the particle-particle ladder term.

This module only draws inputs; it holds none of the ladder arithmetic (no
tau assembly, no integral contraction, no energy).  Both the CPU oracle tests
and the GPU path consume the arrays it returns, so neither side generates its
own data.

Recipe (the paper's molecules, basis sets and integrals are not available, so
random tensors with the paper's shapes stand in for them):

* orbital energies  e_occ ~ U[-1.5, -0.3],  e_vir ~ U[0.1, 3.0]  (Hartree)
* RI factors of the virtual-virtual block (Sec. II.B, Eq. RIM):
  X[P,a,c] ~ N(0, sigma_P^2) with sigma_P = 0.1 exp(-3 P / N_aux), P = 0..N_aux-1,
  then B[P,a,c] = (X[P,a,c] + X[P,c,a]) / 2
* occupied-virtual factors B_ov[P,i,a] from the same decay law (not symmetrised)
* doubles  t2[i,j,a,b] = sum_P B_ov[P,i,a] B_ov[P,j,b] / (e_i + e_j - e_a - e_b),
  then made exactly pair symmetric, t2[i,j,a,b] == t2[j,i,b,a] bit for bit
* singles  t1[i,a] ~ N(0, 1e-3^2)
* occupied-occupied factors B_oo[P,k,l] from the same decay law, symmetrised
  like B (used only by the perturbative triples)

Draw order from ``numpy.random.default_rng(seed)``: e_occ, e_vir, X (vv), X (ov), t1,
X (oo).  X (oo) is drawn last, so the earlier arrays do not depend on it.
All arrays are float64 and C-contiguous.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = ["Inputs", "Workload", "WORKLOADS", "make_inputs", "ragged_batch",
           "sigma", "falg", "dense_flops"]


@dataclass(frozen=True)
class Workload:
    name: str
    o: int
    v: int
    naux: int
    seed: int


# Shapes stand in for the paper's molecules ((H2O)n/cc-pVDZ and beta-carotene,
# Sec. III): N_aux = 4 v, v/o between 6 and 12.
WORKLOADS = {
    "small_o4_v24_n96": Workload("small_o4_v24_n96", 4, 24, 96, 0),
    "dimer_o10_v120_n480": Workload("dimer_o10_v120_n480", 10, 120, 480, 1),
    "mid_o34_v400_n1600": Workload("mid_o34_v400_n1600", 34, 400, 1600, 2),
    "grad_o16_v200_n800": Workload("grad_o16_v200_n800", 16, 200, 800, 3),
    "fd_o3_v10_n30": Workload("fd_o3_v10_n30", 3, 10, 30, 3),
    # the mid-size workload's occupied count (its GEMM2 chunk structure) with
    # a small virtual space: a profiling case that holds ~2 GB on the device
    "probe_o34_v120_n480": Workload("probe_o34_v120_n480", 34, 120, 480, 5),
}


@dataclass
class Inputs:
    o: int
    v: int
    naux: int
    e_occ: np.ndarray
    e_vir: np.ndarray
    B: np.ndarray      # [naux][v][v]
    B_ov: np.ndarray   # [naux][o][v]
    t1: np.ndarray     # [o][v]
    t2: np.ndarray     # [o][o][v][v]
    B_oo: np.ndarray = None  # [naux][o][o]


def sigma(naux: int) -> np.ndarray:
    """Standard deviation of auxiliary function P: 0.1 exp(-3 P / N_aux)."""
    return 0.1 * np.exp(-3.0 * np.arange(naux, dtype=np.float64) / naux)


def _draw(rng: np.random.Generator, o: int, v: int, naux: int) -> Inputs:
    e_occ = rng.uniform(-1.5, -0.3, size=o)
    e_vir = rng.uniform(0.1, 3.0, size=v)
    s = sigma(naux)
    X = rng.standard_normal(size=(naux, v, v))
    X *= s[:, None, None]
    B = 0.5 * (X + X.transpose(0, 2, 1))
    del X
    B = np.ascontiguousarray(B)
    B_ov = rng.standard_normal(size=(naux, o, v)) * s[:, None, None]
    t1 = rng.standard_normal(size=(o, v)) * 1e-3
    # doubles from the occupied-virtual factors and MP2-like denominators
    flat = B_ov.reshape(naux, o * v)
    num = (flat.T @ flat).reshape(o, v, o, v).transpose(0, 2, 1, 3)  # [i][j][a][b]
    den = (e_occ[:, None, None, None] + e_occ[None, :, None, None]
           - e_vir[None, None, :, None] - e_vir[None, None, None, :])
    t2 = num / den
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))  # exact pair symmetry
    X_oo = rng.standard_normal(size=(naux, o, o)) * s[:, None, None]
    B_oo = np.ascontiguousarray(0.5 * (X_oo + X_oo.transpose(0, 2, 1)))
    return Inputs(o, v, naux, e_occ, e_vir, B, np.ascontiguousarray(B_ov),
                  np.ascontiguousarray(t1), np.ascontiguousarray(t2), B_oo)


def make_inputs(o: int, v: int, naux: int, seed: int) -> Inputs:
    """Draw one molecule's inputs with ``default_rng(seed)``."""
    return _draw(np.random.default_rng(seed), o, v, naux)


def ragged_shapes(n: int = 48, first_seed: int = 100):
    """Shapes of the ragged batch: molecule k uses default_rng(first_seed + k),
    o_k uniform integer in [4, 24], v_k = rint(o_k * U[6, 12]) (half to even),
    N_aux,k = 4 v_k."""
    out = []
    for k in range(n):
        rng = np.random.default_rng(first_seed + k)
        o = int(rng.integers(4, 25))
        v = int(np.rint(o * rng.uniform(6.0, 12.0)))
        out.append((o, v, 4 * v, first_seed + k))
    return out


def ragged_batch(n: int = 48, first_seed: int = 100):
    """The ragged batch itself: the shape draws above, then the tensors from
    the same generator, in the standard draw order."""
    mols = []
    for k in range(n):
        rng = np.random.default_rng(first_seed + k)
        o = int(rng.integers(4, 25))
        v = int(np.rint(o * rng.uniform(6.0, 12.0)))
        mols.append(_draw(rng, o, v, 4 * v))
    return mols


def _ppos(n: int) -> int:
    return n * (n + 1) // 2


def _pneg(n: int) -> int:
    return n * (n - 1) // 2


def falg(o: int, v: int, naux: int) -> float:
    """Algorithmic flop count of one ladder evaluation with the symmetric /
    antisymmetric pair combinations: 2 P+(v) v^2 N_aux for the integral tiles
    plus 2 [P+(o) P+(v)^2 + P-(o) P-(v)^2] for the contraction (2 flops per
    multiply-add).  Used as the numerator of every TFLOP/s figure."""
    g1 = 2.0 * _ppos(v) * v * v * naux
    g2 = 2.0 * (_ppos(o) * _ppos(v) ** 2 + _pneg(o) * _pneg(v) ** 2)
    return g1 + g2


def falg_gemm1(o: int, v: int, naux: int) -> float:
    """The integral-tile part of falg: 2 P+(v) v^2 N_aux."""
    return 2.0 * _ppos(v) * v * v * naux


def dense_flops(o: int, v: int, naux: int) -> float:
    """Flops of the plain definition (all ordered index pairs): 2 v^4 N + 2 o^2 v^4."""
    return 2.0 * v ** 4 * naux + 2.0 * o * o * v ** 4
