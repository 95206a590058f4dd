"""Plain FP64 CPU oracle for the particle-particle ladder term (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package; the product library never does.
The C source (``ladder_oracle.c``) shares no code with the CUDA path.

Functions and the passages they follow (arxiv 1810.08142):
  tau              Eq. pp-Ladder-01  tau_ij^ab = t_ij^ab + t_i^a t_j^b
  ladder           Eq. pp-Ladder-0 with Eq. RIM / Eq. eri: R_ij^ab = sum_cd (ac|bd) tau_ij^cd
  ladder_brute     the same through the explicit four-index integral array
  ladder_pairs     selected (a,b) columns of the same sum
  energy           E_L = sum R_ij^ab (2 t_ij^ab - t_ij^ba)  (the closed-shell
                   energy weighting of Sec. II.A applied to the ladder term)
  ladder_dressed   Eq. pp-Ladder-0 with the t1-dressed integrals of Eq. pp-Ladder-2
                   and Eq. pp-Ladder-21 (v^{kb}_{cd} from the same RI factors)
  ladder_dressed_pairs  selected (a,b) columns of the same
  triples          the perturbative triples energy E(T) of Sec. II.A (W, V, D as
                   printed there; integrals from the RI factors)
  triples_wv       W_ijk^abc and V_ijk^abc of one (i,j,k)
  grad_tau, grad_B and their *_entries variants: derivatives of
                   sum W_ij^ab R_ij^ab, written out term by term.
Every function is pinned by tests/test_oracle_pins.py.  The module
oracle/ccsd.py (numpy) holds the closed-shell CCSD iteration of Sec. II.A,
pinned by tests/test_oracle_ccsd_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ladder_oracle.c")
_LIB = os.path.join(_HERE, "libladder_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, -O2, no -march flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_tau.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
        lib.oracle_ladder.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D]
        lib.oracle_ladder_pairs.argtypes = [ctypes.c_int] * 3 + [_D, _D, ctypes.c_int, _I, _I, _D]
        lib.oracle_ladder_brute.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D]
        lib.oracle_ladder_brute.restype = ctypes.c_int
        lib.oracle_energy.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oracle_energy.restype = ctypes.c_double
        lib.oracle_energy_weights.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D]
        lib.oracle_grad_tau.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D]
        lib.oracle_grad_B.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D, _D]
        lib.oracle_grad_tau_entries.argtypes = [ctypes.c_int] * 3 + [_D, _D, ctypes.c_int,
                                                                     _I, _I, _I, _I, _D]
        lib.oracle_grad_B_entries.argtypes = [ctypes.c_int] * 3 + [_D, _D, _D, ctypes.c_int,
                                                                   _I, _I, _I, _D]
        lib.oracle_ladder_dressed.argtypes = [ctypes.c_int] * 3 + [_D] * 5
        lib.oracle_ladder_dressed.restype = ctypes.c_int
        lib.oracle_ladder_dressed_pairs.argtypes = [ctypes.c_int] * 3 + [_D] * 4 + [
            ctypes.c_int, _I, _I, _D]
        lib.oracle_ladder_dressed_pairs.restype = ctypes.c_int
        lib.oracle_triples.argtypes = [ctypes.c_int] * 3 + [_D] * 7
        lib.oracle_triples.restype = ctypes.c_double
        lib.oracle_triples_wv.argtypes = [ctypes.c_int] * 3 + [_D] * 5 + [ctypes.c_int] * 3 + [_D, _D]
        lib.oracle_triples_wv.restype = ctypes.c_int
        lib.oracle_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return x, x.ctypes.data_as(_D)


def _i(x):
    x = np.ascontiguousarray(x, dtype=np.int32)
    return x, x.ctypes.data_as(_I)


def _shape_B(B):
    n, v, v2 = B.shape
    assert v == v2
    return n, v


def threads() -> int:
    return _load().oracle_threads()


def tau(t1, t2):
    o, v = t1.shape
    assert t2.shape == (o, o, v, v)
    t1, p1 = _d(t1)
    t2, p2 = _d(t2)
    out = np.empty((o, o, v, v))
    _load().oracle_tau(o, v, p1, p2, out.ctypes.data_as(_D))
    return out


def ladder(B, tau_):
    n, v = _shape_B(B)
    o = tau_.shape[0]
    assert tau_.shape == (o, o, v, v)
    B, pB = _d(B)
    tau_, pt = _d(tau_)
    R = np.empty((o, o, v, v))
    _load().oracle_ladder(o, v, n, pB, pt, R.ctypes.data_as(_D))
    return R


def ladder_brute(B, tau_):
    n, v = _shape_B(B)
    o = tau_.shape[0]
    if v > 40:
        raise ValueError("brute force is for tiny v only")
    B, pB = _d(B)
    tau_, pt = _d(tau_)
    R = np.empty((o, o, v, v))
    if _load().oracle_ladder_brute(o, v, n, pB, pt, R.ctypes.data_as(_D)) != 0:
        raise MemoryError("oracle_ladder_brute")
    return R


def ladder_pairs(B, tau_, pa, pb):
    """R[:, :, pa[k], pb[k]] for each k, shape [len(pa)][o][o]."""
    n, v = _shape_B(B)
    o = tau_.shape[0]
    B, pB = _d(B)
    tau_, pt = _d(tau_)
    pa, ppa = _i(pa)
    pb, ppb = _i(pb)
    out = np.empty((len(pa), o, o))
    _load().oracle_ladder_pairs(o, v, n, pB, pt, len(pa), ppa, ppb, out.ctypes.data_as(_D))
    return out


def energy(R, t2):
    o, _, v, _ = R.shape
    R, pR = _d(R)
    t2, pt = _d(t2)
    return float(_load().oracle_energy(o, v, pR, pt))


def energy_weights(t2):
    o, _, v, _ = t2.shape
    t2, pt = _d(t2)
    W = np.empty_like(t2)
    _load().oracle_energy_weights(o, v, pt, W.ctypes.data_as(_D))
    return W


def grad_tau(B, W):
    n, v = _shape_B(B)
    o = W.shape[0]
    B, pB = _d(B)
    W, pW = _d(W)
    out = np.empty((o, o, v, v))
    _load().oracle_grad_tau(o, v, n, pB, pW, out.ctypes.data_as(_D))
    return out


def grad_B(B, tau_, W):
    n, v = _shape_B(B)
    o = W.shape[0]
    B, pB = _d(B)
    tau_, pt = _d(tau_)
    W, pW = _d(W)
    out = np.empty((n, v, v))
    _load().oracle_grad_B(o, v, n, pB, pt, pW, out.ctypes.data_as(_D))
    return out


def grad_tau_entries(B, W, i, j, c, d):
    n, v = _shape_B(B)
    o = W.shape[0]
    B, pB = _d(B)
    W, pW = _d(W)
    arrs = [_i(x) for x in (i, j, c, d)]
    out = np.empty(len(arrs[0][0]))
    _load().oracle_grad_tau_entries(o, v, n, pB, pW, len(out), *[p for _, p in arrs],
                                    out.ctypes.data_as(_D))
    return out


def grad_B_entries(B, tau_, W, P, x, y):
    n, v = _shape_B(B)
    o = W.shape[0]
    B, pB = _d(B)
    tau_, pt = _d(tau_)
    W, pW = _d(W)
    arrs = [_i(z) for z in (P, x, y)]
    out = np.empty(len(arrs[0][0]))
    _load().oracle_grad_B_entries(o, v, n, pB, pt, pW, len(out), *[p for _, p in arrs],
                                  out.ctypes.data_as(_D))
    return out


def _shape_dressed(B, B_ov, t1, tau_):
    n, v = _shape_B(B)
    o = tau_.shape[0]
    assert tau_.shape == (o, o, v, v) and B_ov.shape == (n, o, v) and t1.shape == (o, v)
    return o, v, n


def ladder_dressed(B, B_ov, t1, tau_):
    """R_ij^ab = sum_cd b^{ab}_{cd} tau_ij^cd with the dressed b of Eq. pp-Ladder-2."""
    o, v, n = _shape_dressed(B, B_ov, t1, tau_)
    B, pB = _d(B)
    B_ov, pO = _d(B_ov)
    t1, p1 = _d(t1)
    tau_, pt = _d(tau_)
    R = np.empty((o, o, v, v))
    if _load().oracle_ladder_dressed(o, v, n, pB, pO, p1, pt, R.ctypes.data_as(_D)) != 0:
        raise MemoryError("oracle_ladder_dressed")
    return R


def ladder_dressed_pairs(B, B_ov, t1, tau_, pa, pb):
    """Dressed R[:, :, pa[k], pb[k]] for each k, shape [len(pa)][o][o]."""
    o, v, n = _shape_dressed(B, B_ov, t1, tau_)
    B, pB = _d(B)
    B_ov, pO = _d(B_ov)
    t1, p1 = _d(t1)
    tau_, pt = _d(tau_)
    pa, ppa = _i(pa)
    pb, ppb = _i(pb)
    out = np.empty((len(pa), o, o))
    if _load().oracle_ladder_dressed_pairs(o, v, n, pB, pO, p1, pt, len(pa), ppa, ppb,
                                           out.ctypes.data_as(_D)) != 0:
        raise MemoryError("oracle_ladder_dressed_pairs")
    return out


def _triples_args(B, B_ov, B_oo, t1, t2):
    n, v = _shape_B(B)
    o = t1.shape[0]
    assert B_ov.shape == (n, o, v) and B_oo.shape == (n, o, o) and t2.shape == (o, o, v, v)
    arrs = [_d(x) for x in (B, B_ov, B_oo, t1, t2)]
    return o, v, n, arrs


def triples(B, B_ov, B_oo, t1, t2, e_occ, e_vir):
    """E(T) (Sec. II.A) for the given amplitudes, factors and orbital energies."""
    o, v, n, arrs = _triples_args(B, B_ov, B_oo, t1, t2)
    eo, peo = _d(e_occ)
    ev, pev = _d(e_vir)
    E = float(_load().oracle_triples(o, v, n, *[p for _, p in arrs], peo, pev))
    if E != E:
        raise MemoryError("oracle_triples")
    return E


def triples_wv(B, B_ov, B_oo, t1, t2, i, j, k):
    """(W, V) of the triple (i, j, k), each [v][v][v] indexed [a][b][c]."""
    o, v, n, arrs = _triples_args(B, B_ov, B_oo, t1, t2)
    W = np.empty((v, v, v))
    V = np.empty((v, v, v))
    if _load().oracle_triples_wv(o, v, n, *[p for _, p in arrs], int(i), int(j), int(k),
                                 W.ctypes.data_as(_D), V.ctypes.data_as(_D)) != 0:
        raise MemoryError("oracle_triples_wv")
    return W, V
