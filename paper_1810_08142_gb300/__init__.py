"""GB300 particle-particle ladder library: thin Python binding of libladder.so.

Every function below has the name of the C entry point it wraps (see
include/ladder.h) and only marshals arguments: torch tensors are passed as raw
device pointers plus the current CUDA stream.  All arithmetic runs in the CUDA
kernels of the shared library; there is no CPU fallback, and importing this
package on a machine without the built library raises.

The term (arxiv 1810.08142, Sec. II.C):
    R_ij^ab = sum_cd (ac|bd) tau_ij^cd,   tau = t2 + t1 (x) t1,
    (ac|bd) = sum_P B^P_ac B^P_bd,        E_L = sum R_ij^ab (2 t_ij^ab - t_ij^ba).
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libladder.so")

LADDER_FP64, LADDER_BF16X3, LADDER_BF16X6, LADDER_AUTO, LADDER_OZAKI = 0, 1, 2, 3, 4
LADDER_WITH_BACKWARD = 16
LADDER_WITH_DRESSING = 32
MODES = {"fp64": LADDER_FP64, "bf16x3": LADDER_BF16X3, "bf16x6": LADDER_BF16X6, "auto": LADDER_AUTO,
         "ozaki": LADDER_OZAKI}
STATUS = {0: "LADDER_OK", 1: "LADDER_EINVAL", 2: "LADDER_ENOMEM", 3: "LADDER_ECUDA",
          4: "LADDER_ETIMEOUT", 5: "LADDER_ENOTSUP", 6: "LADDER_EWORKSPACE", 7: "LADDER_ENONFINITE"}

# every entry point that include/ladder.h declares
EXPORTS = ("ladder_plan", "ladder_plan_mode", "ladder_plan_shape", "ladder_ccsd_workspace_size", "ladder_ccsd",
           "ladder_get_tuning", "ladder_set_tuning", "ladder_tile_count",
           "ladder_set_tile_range", "ladder_workspace_size", "ladder_set_workspace",
           "ladder_tau", "ladder_apply", "ladder_apply_dressed", "ladder_triples_workspace_size",
           "ladder_triples", "ladder_energy", "ladder_energy_noalloc", "ladder_backward", "ladder_pair_combine", "ladder_apply_host",
           "ladder_plan_batched", "ladder_set_member_tuning", "ladder_apply_batched", "ladder_step_batched", "ladder_last_device_error", "ladder_selftest_wait",
           "ladder_set_timing", "ladder_timing", "ladder_timing_passes", "ladder_timing_dressing", "ladder_timing_sym", "ladder_flops", "ladder_status_string",
           "ladder_destroy")


class Tuning(ctypes.Structure):
    """Mirror of ladder_tuning (include/ladder.h)."""
    _fields_ = [("kc", ctypes.c_int), ("s_pieces", ctypes.c_int), ("flush_every", ctypes.c_int),
                ("ksplit", ctypes.c_int), ("xy_split", ctypes.c_int), ("two_pass", ctypes.c_int),
                ("lambda_only", ctypes.c_int), ("oz_slices", ctypes.c_int), ("tile_chunk", ctypes.c_int),
                ("sym_b", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LadderError(RuntimeError):
    def __init__(self, func, status):
        self.status = status
        super().__init__("%s failed: %s" % (func, STATUS.get(status, status)))


_lib = None
_P = ctypes.c_void_p


def load_library(path: str = LIB_PATH):
    """Load libladder.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libladder.so is not built (run `python -m paper_1810_08142_gb300.build`)")
    lib = ctypes.CDLL(path)
    i, pp, sz = ctypes.c_int, ctypes.POINTER(ctypes.c_void_p), ctypes.c_size_t
    ip = ctypes.POINTER(ctypes.c_int)
    sig = {
        "ladder_plan": [i, i, i, i, pp],
        "ladder_plan_mode": [_P, ip],
        "ladder_plan_shape": [_P, ip, ip, ip],
        "ladder_ccsd_workspace_size": [i, i, i, i, ctypes.POINTER(sz)],
        "ladder_ccsd": [_P, i, i, i] + [_P] * 5 + [i, ctypes.c_double, i, _P, _P,
                                                  ctypes.POINTER(ctypes.c_double), ip, _P, sz, _P],
        "ladder_get_tuning": [_P, ctypes.POINTER(Tuning)],
        "ladder_set_tuning": [_P, ctypes.POINTER(Tuning)],
        "ladder_tile_count": [_P, ip],
        "ladder_set_tile_range": [_P, i, i],
        "ladder_workspace_size": [_P, ctypes.POINTER(sz)],
        "ladder_set_workspace": [_P, _P, sz],
        "ladder_tau": [_P, _P, _P, _P, _P],
        "ladder_apply": [_P, _P, _P, _P, _P],
        "ladder_apply_dressed": [_P, _P, _P, _P, _P, _P, _P],
        "ladder_triples_workspace_size": [i, i, i, i, ctypes.POINTER(sz)],
        "ladder_triples": [i, i, i, i] + [_P] * 9 + [sz, _P],
        "ladder_energy": [_P, _P, _P, _P, _P],
        "ladder_energy_noalloc": [i, i, _P, _P, _P, _P],
        "ladder_backward": [_P, _P, _P, _P, _P, _P, _P],
        "ladder_pair_combine": [i, i, ctypes.c_double, ctypes.c_double, _P, _P, _P],
        "ladder_apply_host": [_P, _P, _P, _P, _P, _P, _P, _P],
        "ladder_plan_batched": [i, ip, ip, ip, i, pp],
        "ladder_set_member_tuning": [_P, i, ctypes.POINTER(Tuning)],
        "ladder_apply_batched": [_P, pp, pp, pp, _P],
        "ladder_step_batched": [_P, pp, pp, pp, pp, pp, _P, _P],
        "ladder_last_device_error": [_P, _P, ip],
        "ladder_selftest_wait": [_P, ctypes.c_ulonglong, _P],
        "ladder_set_timing": [_P, i],
        "ladder_timing": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                          ctypes.POINTER(ctypes.c_float)],
        "ladder_timing_passes": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
        "ladder_timing_dressing": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
        "ladder_timing_sym": [_P, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)],
        "ladder_flops": [_P],
        "ladder_status_string": [i],
        "ladder_destroy": [_P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.ladder_flops.restype = ctypes.c_double
    lib.ladder_status_string.restype = ctypes.c_char_p
    lib.ladder_destroy.restype = None
    _lib = lib
    return lib


def _check(name, st):
    if st != 0:
        raise LadderError(name, st)


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


# ---- one-to-one wrappers ---------------------------------------------------
def ladder_plan(o: int, v: int, naux: int, mode: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check("ladder_plan", load_library().ladder_plan(o, v, naux, mode, ctypes.byref(h)))
    return h


def ladder_plan_mode(plan) -> int:
    m = ctypes.c_int()
    _check("ladder_plan_mode", load_library().ladder_plan_mode(plan, ctypes.byref(m)))
    return m.value


def ladder_get_tuning(plan) -> Tuning:
    t = Tuning()
    _check("ladder_get_tuning", load_library().ladder_get_tuning(plan, ctypes.byref(t)))
    return t


def ladder_set_tuning(plan, t: Tuning) -> None:
    _check("ladder_set_tuning", load_library().ladder_set_tuning(plan, ctypes.byref(t)))


def ladder_tile_count(plan) -> int:
    n = ctypes.c_int()
    _check("ladder_tile_count", load_library().ladder_tile_count(plan, ctypes.byref(n)))
    return n.value


def ladder_set_tile_range(plan, tile_lo: int, tile_hi: int) -> None:
    _check("ladder_set_tile_range", load_library().ladder_set_tile_range(plan, int(tile_lo), int(tile_hi)))


def ladder_workspace_size(plan) -> int:
    n = ctypes.c_size_t()
    _check("ladder_workspace_size", load_library().ladder_workspace_size(plan, ctypes.byref(n)))
    return n.value


def ladder_set_workspace(plan, ws) -> None:
    _check("ladder_set_workspace",
           load_library().ladder_set_workspace(plan, _ptr(ws), ws.numel() * ws.element_size()))


def ladder_tau(plan, t1, t2, tau, stream=None) -> None:
    _check("ladder_tau", load_library().ladder_tau(plan, _ptr(t1), _ptr(t2), _ptr(tau), _stream(stream)))


def ladder_apply(plan, B, tau, R, stream=None) -> None:
    _check("ladder_apply", load_library().ladder_apply(plan, _ptr(B), _ptr(tau), _ptr(R), _stream(stream)))


def ladder_apply_dressed(plan, B, B_ov, t1, tau, R, stream=None) -> None:
    _check("ladder_apply_dressed",
           load_library().ladder_apply_dressed(plan, _ptr(B), _ptr(B_ov), _ptr(t1), _ptr(tau), _ptr(R),
                                               _stream(stream)))


def ladder_plan_shape(plan):
    o, v, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check("ladder_plan_shape", load_library().ladder_plan_shape(plan, ctypes.byref(o), ctypes.byref(v),
                                                                 ctypes.byref(n)))
    return o.value, v.value, n.value


def ladder_ccsd_workspace_size(o: int, v: int, naux: int, ndiis: int) -> int:
    n = ctypes.c_size_t()
    _check("ladder_ccsd_workspace_size",
           load_library().ladder_ccsd_workspace_size(o, v, naux, ndiis, ctypes.byref(n)))
    return n.value


def ladder_ccsd(plan, o, v, naux, B, B_ov, B_oo, e_occ, e_vir, max_iter, tol, ndiis, t1, t2, ws, stream=None):
    """The C call itself; returns (E, iterations)."""
    E, it = ctypes.c_double(), ctypes.c_int()
    _check("ladder_ccsd", load_library().ladder_ccsd(
        plan, int(o), int(v), int(naux), _ptr(B), _ptr(B_ov), _ptr(B_oo), _ptr(e_occ), _ptr(e_vir),
        int(max_iter), float(tol), int(ndiis), _ptr(t1), _ptr(t2), ctypes.byref(E), ctypes.byref(it), _ptr(ws),
        ws.numel() * ws.element_size(), _stream(stream)))
    return E.value, it.value


def ccsd(ladder, B, B_ov, B_oo, e_occ, e_vir, max_iter=100, tol=1e-10, ndiis=3, workspace=None, stream=None):
    """Closed-shell RI-CCSD (Sec. II.A): Jacobi steps with DIIS from zero
    amplitudes, the ladder of every step on `ladder` (a Ladder of the same
    shape; its mode sets the ladder's precision).  FP64 device tensors in;
    returns (t1, t2, E, iterations) with t1, t2 on the device."""
    import torch
    naux, v, _ = B.shape
    o = B_oo.shape[1]
    if workspace is None:
        nb = ladder_ccsd_workspace_size(o, v, naux, ndiis)
        workspace = torch.empty(max(nb, 256), dtype=torch.uint8, device=B.device)
    t1 = torch.empty((o, v), dtype=torch.float64, device=B.device)
    t2 = torch.empty((o, o, v, v), dtype=torch.float64, device=B.device)
    E, it = ladder_ccsd(ladder.plan, o, v, naux, B, B_ov, B_oo, e_occ, e_vir, max_iter, tol, ndiis, t1, t2,
                        workspace, stream)
    return t1, t2, E, it


TRIPLES_PRECISION = {"fp64": 0, "fp32": 1, "bf16x6": 2}


def ladder_triples_workspace_size(o: int, v: int, naux: int, precision: int) -> int:
    n = ctypes.c_size_t()
    _check("ladder_triples_workspace_size",
           load_library().ladder_triples_workspace_size(o, v, naux, precision, ctypes.byref(n)))
    return n.value


def ladder_triples(o, v, naux, precision, B, B_ov, B_oo, t1, t2, e_occ, e_vir, E, ws, stream=None) -> None:
    _check("ladder_triples", load_library().ladder_triples(
        o, v, naux, precision, _ptr(B), _ptr(B_ov), _ptr(B_oo), _ptr(t1), _ptr(t2), _ptr(e_occ),
        _ptr(e_vir), _ptr(E), _ptr(ws), ws.numel() * ws.element_size(), _stream(stream)))


def triples(B, B_ov, B_oo, t1, t2, e_occ, e_vir, precision="fp64", workspace=None):
    """The perturbative triples energy E(T) of Sec. II.A on the device (FP64
    device tensors in, one FP64 device scalar out); precision "fp64", "fp32"
    (integrals and W in FP32, energy sums in FP64) or "bf16x6" (FP32
    integrals, W contractions on the tensor cores in split BF16)."""
    import torch
    naux, v, _ = B.shape
    o = t1.shape[0]
    prec = TRIPLES_PRECISION[precision]
    if workspace is None:
        n = ladder_triples_workspace_size(o, v, naux, prec)
        workspace = torch.empty(max(n, 256), dtype=torch.uint8, device=B.device)
    E = torch.empty((), dtype=torch.float64, device=B.device)
    ladder_triples(o, v, naux, prec, B, B_ov, B_oo, t1, t2, e_occ, e_vir, E, workspace)
    return E


def ladder_energy(plan, R, t2, E, stream=None) -> None:
    _check("ladder_energy", load_library().ladder_energy(plan, _ptr(R), _ptr(t2), _ptr(E), _stream(stream)))


def ladder_energy_noalloc(o, v, R, t2, E, stream=None) -> None:
    """E_L without a plan or workspace, for callers that cannot allocate device
    memory; see include/ladder.h for the limit on o and v."""
    _check("ladder_energy_noalloc", load_library().ladder_energy_noalloc(
        int(o), int(v), _ptr(R), _ptr(t2), _ptr(E), _stream(stream)))


def ladder_backward(plan, B, tau, W, dtau, dB, stream=None) -> None:
    _check("ladder_backward", load_library().ladder_backward(
        plan, _ptr(B), _ptr(tau), _ptr(W), _ptr(dtau), _ptr(dB), _stream(stream)))


def ladder_pair_combine(o, v, alpha, beta, X, Y, stream=None) -> None:
    _check("ladder_pair_combine", load_library().ladder_pair_combine(
        int(o), int(v), float(alpha), float(beta), _ptr(X), _ptr(Y), _stream(stream)))


def ladder_apply_host(plan, B_host, tau_host, R_host, d_B, d_tau, d_R, stream=None) -> None:
    _check("ladder_apply_host", load_library().ladder_apply_host(
        plan, _ptr(B_host), _ptr(tau_host), _ptr(R_host), _ptr(d_B), _ptr(d_tau), _ptr(d_R),
        _stream(stream)))


def ladder_plan_batched(o, v, naux, mode: int) -> ctypes.c_void_p:
    n = len(o)
    arr = lambda xs: (ctypes.c_int * n)(*[int(x) for x in xs])
    h = ctypes.c_void_p()
    _check("ladder_plan_batched",
           load_library().ladder_plan_batched(n, arr(o), arr(v), arr(naux), mode, ctypes.byref(h)))
    return h


def ladder_set_member_tuning(plan, m: int, t: Tuning) -> None:
    _check("ladder_set_member_tuning", load_library().ladder_set_member_tuning(plan, m, ctypes.byref(t)))


def ladder_apply_batched(plan, Bs, taus, Rs, stream=None) -> None:
    n = len(Bs)
    arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    _check("ladder_apply_batched", load_library().ladder_apply_batched(
        plan, arr(Bs), arr(taus), arr(Rs), _stream(stream)))


def ladder_step_batched(plan, Bs, t1s, t2s, taus, Rs, E, stream=None) -> None:
    n = len(Bs)
    arr = lambda ts: (ctypes.c_void_p * n)(*[t.data_ptr() for t in ts])
    _check("ladder_step_batched", load_library().ladder_step_batched(
        plan, arr(Bs), arr(t1s), arr(t2s), arr(taus), arr(Rs), _ptr(E), _stream(stream)))


def ladder_last_device_error(plan, stream=None):
    where = ctypes.c_int()
    st = load_library().ladder_last_device_error(plan, _stream(stream), ctypes.byref(where))
    return st, where.value


def ladder_set_timing(plan, on: bool) -> None:
    _check("ladder_set_timing", load_library().ladder_set_timing(plan, 1 if on else 0))


def ladder_timing(plan):
    """(prep_ms, ladder_ms, unpack_ms) of the last ladder_apply (waits for it);
    ladder_ms covers the fused kernel or both passes of the two-pass form."""
    t = [ctypes.c_float() for _ in range(3)]
    _check("ladder_timing", load_library().ladder_timing(plan, *[ctypes.byref(x) for x in t]))
    return tuple(x.value for x in t)


def ladder_timing_passes(plan):
    """(pass1_ms, pass2_ms) of the last ladder_apply: the storing GEMM1 pass
    and the GEMM2 pass of the two-pass form, else (fused kernel, 0)."""
    t = [ctypes.c_float() for _ in range(2)]
    _check("ladder_timing_passes", load_library().ladder_timing_passes(plan, *[ctypes.byref(x) for x in t]))
    return tuple(x.value for x in t)


def ladder_timing_dressing(plan):
    """(bd_ms, correction_ms) of the last ladder_apply_dressed: the B - mbar
    product and the rank-o correction after the ladder."""
    t = [ctypes.c_float() for _ in range(2)]
    _check("ladder_timing_dressing", load_library().ladder_timing_dressing(plan, *[ctypes.byref(x) for x in t]))
    return tuple(x.value for x in t)


def ladder_timing_sym(plan):
    """(xsym_ms, form_ms) of the last ladder_apply of an error-free plan with
    sym_b: the distinct integral tiles and the formation of V+- from them."""
    t = [ctypes.c_float() for _ in range(2)]
    _check("ladder_timing_sym", load_library().ladder_timing_sym(plan, *[ctypes.byref(x) for x in t]))
    return tuple(x.value for x in t)


def ladder_selftest_wait(plan, timeout_ns: int, stream=None) -> None:
    _check("ladder_selftest_wait", load_library().ladder_selftest_wait(plan, int(timeout_ns),
                                                                      _stream(stream)))


def ladder_status_string(status: int) -> str:
    return load_library().ladder_status_string(int(status)).decode()


def ladder_flops(plan) -> float:
    return float(load_library().ladder_flops(plan))


def ladder_destroy(plan) -> None:
    load_library().ladder_destroy(plan)


# ---- convenience object ------------------------------------------------------
class Ladder:
    """A plan plus its workspace (a torch uint8 tensor on the current device)."""

    def __init__(self, o: int, v: int, naux: int, mode="bf16x6", device=None, backward=False,
                 tuning=None, dressed=False, tiles=None):
        """mode: "fp64", "bf16x3", "bf16x6", "ozaki" (the error-free split, FP64-class
        accuracy from the BF16 tensor cores), or "tuned" (the autotuner's cached
        choice of mode and launch parameters for this shape, see tune.py);
        tuning: a dict of ladder_tuning fields to override; dressed: size the
        workspace for apply_dressed (the t1-dressed term) as well; tiles:
        (lo, hi) restricts the plan to pair tiles [lo, hi) (see partition.py),
        applied before the tuning."""
        import torch
        self.o, self.v, self.naux = o, v, naux
        if mode == "tuned":
            from .tune import lookup
            mode, tuning = lookup(o, v, naux)
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        if backward:
            m |= LADDER_WITH_BACKWARD
        if dressed:
            m |= LADDER_WITH_DRESSING
        self.device = torch.device(device if device is not None else "cuda")
        with torch.cuda.device(self.device):
            self.plan = ladder_plan(o, v, naux, m)
            self.mode = ladder_plan_mode(self.plan)
            if tiles is not None:
                ladder_set_tile_range(self.plan, tiles[0], tiles[1])
            if tuning and self.mode != LADDER_FP64:
                t = ladder_get_tuning(self.plan)
                for k, val in tuning.items():
                    setattr(t, k, int(val))
                if "two_pass" in tuning and "ksplit" not in tuning:
                    t.ksplit = 0  # the plan's own block-pair split for the chosen form
                ladder_set_tuning(self.plan, t)
            n = ladder_workspace_size(self.plan)
            self.workspace = torch.empty(max(n, 256), dtype=torch.uint8, device=self.device)
            ladder_set_workspace(self.plan, self.workspace)

    @property
    def flops(self) -> float:
        return ladder_flops(self.plan)

    def tau(self, t1, t2, out=None):
        import torch
        out = torch.empty_like(t2) if out is None else out
        ladder_tau(self.plan, t1, t2, out)
        return out

    def apply(self, B, tau, out=None):
        import torch
        out = torch.empty_like(tau) if out is None else out
        ladder_apply(self.plan, B, tau, out)
        return out

    def apply_dressed(self, B, B_ov, t1, tau, out=None):
        """The t1-dressed term (Eq. pp-Ladder-2); the Ladder needs dressed=True."""
        import torch
        out = torch.empty_like(tau) if out is None else out
        ladder_apply_dressed(self.plan, B, B_ov, t1, tau, out)
        return out

    def energy(self, R, t2, out=None):
        import torch
        out = torch.empty((), dtype=torch.float64, device=R.device) if out is None else out
        ladder_energy(self.plan, R, t2, out)
        return out

    def weights(self, t2, out=None):
        """Energy weights W = 2 t2 - t2^T (dE_L/dR)."""
        import torch
        out = torch.empty_like(t2) if out is None else out
        ladder_pair_combine(self.o, self.v, 2.0, -1.0, t2, out)
        return out

    def backward(self, B, tau, W, dtau=True, dB=True):
        """(dtau, dB) of E = sum W R; pass False to skip one."""
        import torch
        dt = torch.empty_like(tau) if dtau is True else (None if dtau is False else dtau)
        db = torch.empty_like(B) if dB is True else (None if dB is False else dB)
        ladder_backward(self.plan, B, tau, W, dt, db)
        return dt, db

    def check_device(self):
        st, where = ladder_last_device_error(self.plan)
        if st != 0:
            raise LadderError("device wait (site %d)" % where, st)

    def close(self):
        if getattr(self, "plan", None) is not None:
            ladder_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LadderBatch:
    """A batched plan for molecules of uneven shape (persistent launches over
    all molecules' work units, fused or two-pass per molecule, replayed as a
    CUDA graph) plus its workspace."""

    def __init__(self, shapes, mode="bf16x6", device=None, tunings=None, sym_b=False):
        """mode: "bf16x3", "bf16x6", "ozaki" (every member in the error-free
        two-pass form), or "tuned" (BF16X6 with each member's launch
        parameters and form from the autotuner's cache, see tune.py);
        tunings: optional list of per-member dicts of ladder_tuning fields
        (None entries keep the plan's choice); sym_b (mode "ozaki"; a bool
        for every member or a list of one per member): the member's B is
        symmetric in a <-> c, so it forms its distinct integral tiles once
        (checked on the device, see ladder_tuning)."""
        import torch
        self.shapes = [(int(o), int(v), int(n)) for o, v, n in shapes]
        if mode == "tuned":
            mode = "bf16x6"
            tunings = []
            from .tune import lookup_mode
            for o, v, n in self.shapes:
                tunings.append(lookup_mode(o, v, n, mode))
        m = MODES[mode] if isinstance(mode, str) else int(mode)
        self.device = torch.device(device if device is not None else "cuda")
        self.tunings = []
        with torch.cuda.device(self.device):
            self.plan = ladder_plan_batched([s[0] for s in self.shapes], [s[1] for s in self.shapes],
                                            [s[2] for s in self.shapes], m)
            for k, tun in enumerate(tunings or []):
                if not tun:
                    self.tunings.append(None)
                    continue
                t = Tuning(kc=4, s_pieces=2, flush_every=16, ksplit=0, xy_split=1, two_pass=0, lambda_only=0)
                for key, val in tun.items():
                    if key in ("kc", "s_pieces", "flush_every", "xy_split", "two_pass"):
                        setattr(t, key, int(val))
                try:
                    ladder_set_member_tuning(self.plan, k, t)
                    self.tunings.append(t.as_dict())
                except LadderError:
                    # the two-pass form would overflow the batch's tile cap: keep the plan's form
                    t.two_pass = 0
                    ladder_set_member_tuning(self.plan, k, t)
                    self.tunings.append(t.as_dict())
            sym = [bool(x) for x in sym_b] if isinstance(sym_b, (list, tuple)) else [bool(sym_b)] * len(self.shapes)
            if any(sym):
                if m != LADDER_OZAKI:
                    raise ValueError("sym_b applies to the error-free mode")
                for k, on in enumerate(sym):
                    if on:
                        ladder_set_member_tuning(self.plan, k, Tuning(sym_b=1))
            n = ladder_workspace_size(self.plan)
            self.workspace = torch.empty(max(n, 256), dtype=torch.uint8, device=self.device)
            ladder_set_workspace(self.plan, self.workspace)

    @property
    def flops(self) -> float:
        return ladder_flops(self.plan)

    def apply(self, Bs, taus, outs=None):
        import torch
        outs = [torch.empty_like(t) for t in taus] if outs is None else outs
        ladder_apply_batched(self.plan, Bs, taus, outs)
        return outs

    def step(self, Bs, t1s, t2s, taus=None, outs=None, E=None):
        """One graph for every molecule: tau = t2 + t1 (x) t1, R, and E_L per
        molecule (a device tensor of n doubles); returns (taus, outs, E)."""
        import torch
        taus = [torch.empty_like(t) for t in t2s] if taus is None else taus
        outs = [torch.empty_like(t) for t in t2s] if outs is None else outs
        E = torch.empty(len(Bs), dtype=torch.float64, device=t2s[0].device) if E is None else E
        ladder_step_batched(self.plan, Bs, t1s, t2s, taus, outs, E)
        return taus, outs, E

    def check_device(self):
        st, where = ladder_last_device_error(self.plan)
        if st != 0:
            raise LadderError("device wait (site %d)" % where, st)

    def close(self):
        if getattr(self, "plan", None) is not None:
            ladder_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
