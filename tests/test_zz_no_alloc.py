"""The allocation-free energy entry point (ladder_energy_noalloc), for callers
that cannot allocate device memory: it must give the same E_L as the
plan-based ladder_energy and as the FP64 oracle, on two calls in a row, at the
largest shape its fixed scratch array holds too, and refuse shapes whose
partial sums do not fit.  Called through the C ABI.  This file is collected
last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1810_08142_gb300 as lad
    return torch, lad


def _call(lib, o, v, R, t2, E):
    return lib.ladder_energy_noalloc(o, v, ctypes.c_void_p(R.data_ptr()), ctypes.c_void_p(t2.data_ptr()),
                                     ctypes.c_void_p(E.data_ptr()),
                                     ctypes.c_void_p(__import__("torch").cuda.current_stream().cuda_stream))


def _inputs(o, v, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((o, o, v, v)), rng.standard_normal((o, o, v, v))


def _oracle_check(got, R, t2):
    """E_L against the plain FP64 oracle, within the rounding of a sum of
    n terms: n * 2^-52 * sum |R (2 t - t^T)|."""
    import oracle
    ref = oracle.energy(R, t2)
    scale = float(np.sum(np.abs(R * (2.0 * t2 - t2.transpose(0, 1, 3, 2)))))
    assert abs(got - ref) <= 1e-13 * scale, (got, ref, scale)


@pytest.mark.parametrize("o,v,seed", [(4, 24, 0), (7, 41, 14), (10, 120, 1)])
def test_noalloc_energy_matches_plan_energy_on_two_calls(env, o, v, seed):
    torch, lad = env
    lib = lad.load_library()
    Rh, th = _inputs(o, v, seed)
    R, t2 = torch.from_numpy(Rh).cuda(), torch.from_numpy(th).cuda()
    L = lad.Ladder(o, v, 8, mode="fp64")
    E_ref = L.energy(R, t2)
    torch.cuda.synchronize()
    ref = float(E_ref.item())
    for _ in range(2):
        E = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, o, v, R, t2, E) == 0
        torch.cuda.synchronize()
        got = float(E.item())
        assert abs(got - ref) <= 1e-12 * abs(ref) + 1e-300
        _oracle_check(got, Rh, th)


@pytest.mark.parametrize("o,v", [(181, 100), (256, 32)])
def test_noalloc_energy_at_its_largest_shapes(env, o, v):
    """o=181, v=100 needs 4^2 * 181^2 = 524176 partial sums, the largest count
    at or below the array's 524288 (a perfect square cannot equal 2^19);
    o=256 puts 65536 (i,j) pairs into the reduction's grid."""
    torch, lad = env
    lib = lad.load_library()
    Rh, th = _inputs(o, v, 5)
    R, t2 = torch.from_numpy(Rh).cuda(), torch.from_numpy(th).cuda()
    for _ in range(2):
        E = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(lib, o, v, R, t2, E) == 0
        torch.cuda.synchronize()
        _oracle_check(float(E.item()), Rh, th)


def test_noalloc_energy_refuses_shapes_beyond_its_scratch(env):
    torch, lad = env
    lib = lad.load_library()
    # ceil(200/32)^2 * 120^2 = 705600 partial sums > 524288
    o, v = 120, 200
    R = torch.zeros(1, dtype=torch.float64, device="cuda")
    E = torch.zeros((), dtype=torch.float64, device="cuda")
    assert _call(lib, o, v, R, R, E) == 5  # LADDER_ENOTSUP
