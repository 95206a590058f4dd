"""Helpers shared by the GPU tests: device copies of synthetic inputs and the
error measures the tolerances are stated in."""
import numpy as np


def rel_fro(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm(x - ref) / max(np.linalg.norm(ref), 1e-300))


def max_rel(x, ref):
    """max |x - ref| / max |ref|: the worst element against the scale of ref."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(x - ref)) / max(float(np.max(np.abs(ref))), 1e-300))


def rel_err(x, ref):
    """The larger of the relative Frobenius error and half of max_rel, so that
    one tolerance bounds the aggregate and, at twice the tolerance, the worst
    element against the largest (a few wrong entries, e.g. an unwritten tile
    edge, cannot hide inside a norm).  The factor two leaves room for the
    heavier tail of the split-BF16 modes, whose biased accumulation error is
    largest on the largest entries."""
    return max(rel_fro(x, ref), 0.5 * max_rel(x, ref))


def to_dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run_forward(L, x):
    """tau, R and E_L through the C ABI for inputs x (synthetic.Inputs)."""
    import torch
    t1, t2, B = to_dev(x.t1), to_dev(x.t2), to_dev(x.B)
    tau = L.tau(t1, t2)
    R = L.apply(B, tau)
    E = L.energy(R, t2)
    torch.cuda.synchronize()
    L.check_device()
    return tau.cpu().numpy(), R.cpu().numpy(), float(E.item())


def run_dressed(L, x):
    """tau, the t1-dressed R and its E_L through the C ABI (L built with dressed=True)."""
    import torch
    t1, t2, B, Bov = to_dev(x.t1), to_dev(x.t2), to_dev(x.B), to_dev(x.B_ov)
    tau = L.tau(t1, t2)
    R = L.apply_dressed(B, Bov, t1, tau)
    E = L.energy(R, t2)
    torch.cuda.synchronize()
    L.check_device()
    return tau.cpu().numpy(), R.cpu().numpy(), float(E.item())
