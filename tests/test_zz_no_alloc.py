"""The allocation-free energy entry point (ladder_energy_noalloc), for callers
that cannot allocate device memory: it must give the same E_L as the
plan-based ladder_energy, on two calls in a row, and refuse shapes whose
partial sums do not fit its fixed scratch array.  Called through the C ABI.
This file is collected last on purpose."""
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


@pytest.mark.parametrize("o,v,seed", [(4, 24, 0), (7, 41, 14), (10, 120, 1)])
def test_noalloc_energy_matches_plan_energy_on_two_calls(env, o, v, seed):
    torch, lad = env
    lib = lad.load_library()
    rng = np.random.default_rng(seed)
    R = torch.from_numpy(rng.standard_normal((o, o, v, v))).cuda()
    t2 = torch.from_numpy(rng.standard_normal((o, o, v, v))).cuda()
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


def test_noalloc_energy_refuses_shapes_beyond_its_scratch(env):
    torch, lad = env
    lib = lad.load_library()
    # ceil(200/32)^2 * 120^2 = 705600 partial sums > 524288
    o, v = 120, 200
    R = torch.zeros(1, dtype=torch.float64, device="cuda")
    E = torch.zeros((), dtype=torch.float64, device="cuda")
    assert _call(lib, o, v, R, R, E) == 5  # LADDER_ENOTSUP
