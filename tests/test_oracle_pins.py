"""Pins for the CPU oracle: each test checks the oracle against something the
paper or the mathematics fixes independently of the oracle's own formula
(closed forms, special cases, invariants, exact finite differences, brute
force).  No GPU needed."""
import numpy as np
import pytest

import oracle
import synthetic


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def rand_tau(rng, o, v, pair_symmetric=False):
    t = rng.standard_normal((o, o, v, v))
    if pair_symmetric:
        t = 0.5 * (t + t.transpose(1, 0, 3, 2))
    return t


# --- ladder: brute force (Eq. pp-Ladder-0 through the explicit (ac|bd) array)
@pytest.mark.parametrize("o,v,n,seed", [(1, 3, 2, 0), (3, 7, 5, 1), (4, 12, 48, 2), (2, 24, 40, 3)])
def test_ladder_equals_brute_force(o, v, n, seed):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, v, v))          # general, not symmetric in a<->c
    tau = rand_tau(rng, o, v)                   # general, not pair symmetric
    assert rel(oracle.ladder(B, tau), oracle.ladder_brute(B, tau)) < 1e-14


# --- ladder: a single auxiliary function whose factor has rank two.
# With B^0_ac = u_a w_c + p_a q_c the integral (ac|bd) factorises and
#   R_ij^ab = u_a u_b (w.tau_ij.w) + u_a p_b (w.tau_ij.q) + p_a u_b (q.tau_ij.w) + p_a p_b (q.tau_ij.q)
# where x.tau_ij.y = sum_cd x_c tau_ij^cd y_d.  Catches a transposed factor
# (B_ca for B_ac), a swapped integral index (tau^dc for tau^cd) and swapped
# output indices (R^ba for R^ab).
def test_ladder_rank_two_closed_form():
    rng = np.random.default_rng(7)
    o, v = 3, 9
    u, w, p, q = rng.standard_normal((4, v))
    B = (np.outer(u, w) + np.outer(p, q))[None]
    tau = rand_tau(rng, o, v)
    ww = np.einsum("c,ijcd,d->ij", w, tau, w)
    wq = np.einsum("c,ijcd,d->ij", w, tau, q)
    qw = np.einsum("c,ijcd,d->ij", q, tau, w)
    qq = np.einsum("c,ijcd,d->ij", q, tau, q)
    expect = (ww[:, :, None, None] * np.outer(u, u) + wq[:, :, None, None] * np.outer(u, p)
              + qw[:, :, None, None] * np.outer(p, u) + qq[:, :, None, None] * np.outer(p, p))
    assert rel(oracle.ladder(B, tau), expect) < 1e-13


# The rank-one special case stated for the method: B^P_ac = u_a u_c gives
# R_ij^ab = u_a u_b sum_cd u_c u_d tau_ij^cd.
def test_ladder_rank_one_closed_form():
    rng = np.random.default_rng(8)
    o, v = 4, 11
    u = rng.standard_normal(v)
    B = np.outer(u, u)[None]
    tau = rand_tau(rng, o, v)
    s = np.einsum("c,ijcd,d->ij", u, tau, u)
    expect = s[:, :, None, None] * np.outer(u, u)
    assert rel(oracle.ladder(B, tau), expect) < 1e-13


# --- identity factor: N = v^2 and B^{(x,y)}_ac = delta_xa delta_yc give
# (ac|bd) = delta_ab delta_cd, hence R_ij^ab = delta_ab sum_c tau_ij^cc.
def test_ladder_identity_factor():
    rng = np.random.default_rng(9)
    o, v = 3, 6
    B = np.eye(v * v).reshape(v * v, v, v)
    tau = rand_tau(rng, o, v)
    tr = np.trace(tau, axis1=2, axis2=3)
    expect = tr[:, :, None, None] * np.eye(v)[None, None]
    assert np.array_equal(oracle.ladder(B, tau), expect)


# --- pair symmetry of the ladder term (Sec. II.C): with tau_ij^cd = tau_ji^dc,
# R_ij^ab = R_ji^ba for any factor B.
def test_ladder_pair_symmetry():
    rng = np.random.default_rng(10)
    o, v, n = 5, 10, 17
    B = rng.standard_normal((n, v, v))
    tau = rand_tau(rng, o, v, pair_symmetric=True)
    R = oracle.ladder(B, tau)
    assert rel(R, R.transpose(1, 0, 3, 2)) < 1e-14


def test_ladder_linear_in_tau_quadratic_in_B_additive_over_aux():
    rng = np.random.default_rng(11)
    o, v, n = 3, 8, 12
    B = rng.standard_normal((n, v, v))
    t1, t2 = rand_tau(rng, o, v), rand_tau(rng, o, v)
    al, be = 0.75, -1.5
    assert rel(oracle.ladder(B, al * t1 + be * t2),
               al * oracle.ladder(B, t1) + be * oracle.ladder(B, t2)) < 1e-14
    assert rel(oracle.ladder(-3.0 * B, t1), 9.0 * oracle.ladder(B, t1)) < 1e-14
    k = 5
    assert rel(oracle.ladder(B, t1), oracle.ladder(B[:k], t1) + oracle.ladder(B[k:], t1)) < 1e-14
    assert np.array_equal(oracle.ladder(np.zeros_like(B), t1), np.zeros_like(t1))


def test_ladder_pairs_match_columns():
    x = synthetic.make_inputs(3, 14, 40, 5)
    tau = oracle.tau(x.t1, x.t2)
    R = oracle.ladder(x.B, tau)
    pa, pb = [0, 3, 13, 7], [0, 9, 2, 13]
    Rs = oracle.ladder_pairs(x.B, tau, pa, pb)
    for k in range(len(pa)):
        assert np.array_equal(Rs[k], R[:, :, pa[k], pb[k]])


# --- tau (Eq. pp-Ladder-01)
def test_tau_special_cases():
    rng = np.random.default_rng(12)
    o, v = 3, 5
    t2 = rand_tau(rng, o, v)
    assert np.array_equal(oracle.tau(np.zeros((o, v)), t2), t2)
    # two nonzero singles: t_0^1 = x, t_1^2 = y, no doubles
    t1 = np.zeros((o, v))
    t1[0, 1], t1[1, 2] = 0.5, -3.0
    tau = oracle.tau(t1, np.zeros_like(t2))
    expect = np.zeros_like(t2)
    expect[0, 0, 1, 1] = 0.25
    expect[0, 1, 1, 2] = -1.5
    expect[1, 0, 2, 1] = -1.5
    expect[1, 1, 2, 2] = 9.0
    assert np.array_equal(tau, expect)


# --- energy E_L = sum R (2 t - t^T)
def test_energy_special_cases():
    rng = np.random.default_rng(13)
    o, v = 3, 6
    t2 = rand_tau(rng, o, v)
    # R = 1 everywhere: the exchange sum equals the direct sum, so E = sum t
    assert abs(oracle.energy(np.ones_like(t2), t2) - t2.sum()) < 1e-12 * np.abs(t2).sum()
    # a single unit entry picks 2 t_ij^ab - t_ij^ba
    R = np.zeros_like(t2)
    R[1, 2, 4, 0] = 1.0
    assert oracle.energy(R, t2) == 2.0 * t2[1, 2, 4, 0] - t2[1, 2, 0, 4]
    R[1, 2, 4, 0] = 0.0
    R[2, 2, 3, 3] = 1.0
    assert oracle.energy(R, t2) == t2[2, 2, 3, 3]
    W = oracle.energy_weights(t2)
    assert np.array_equal(W[1, 2, 4, 0], 2.0 * t2[1, 2, 4, 0] - t2[1, 2, 0, 4])


# --- gradients: E(B, tau) = sum W R is linear in tau and quadratic in B, so
# Euler's theorem and exact central differences pin both gradients.
@pytest.fixture(scope="module")
def grad_case():
    rng = np.random.default_rng(14)
    o, v, n = 3, 7, 9
    B = rng.standard_normal((n, v, v))
    tau = rand_tau(rng, o, v)
    W = rand_tau(rng, o, v)
    return B, tau, W


def _E(B, tau, W):
    return float(np.sum(W * oracle.ladder(B, tau)))


def test_energy_sum_is_compensated():
    """E_L of terms 1e16, 1, -1e16, 1 (o = 1, v = 2, symmetric t2 = 1 so that
    W = t2): the exact sum is 2; a plain running sum in FP64 gives 1 (1e16 + 1
    rounds back to 1e16).  The oracle's sum must give 2."""
    R = np.array([1e16, 1.0, -1e16, 1.0]).reshape(1, 1, 2, 2)
    t2 = np.ones((1, 1, 2, 2))
    assert oracle.energy(R, t2) == 2.0
    # and a long sum: n copies of (big, small, -big) leave exactly n * small
    n = 1000
    R = np.tile(np.array([1e15, 0.25, -1e15, 0.25]), n).reshape(1, 1, 2 * n, 2)
    t2 = np.ones((1, 1, 2 * n, 2 * n))
    Rf = np.zeros((1, 1, 2 * n, 2 * n))
    Rf[0, 0, :, :2] = R[0, 0]
    assert oracle.energy(Rf, t2) == 0.5 * n


def test_grad_euler_identities(grad_case):
    B, tau, W = grad_case
    E = _E(B, tau, W)
    dtau = oracle.grad_tau(B, W)
    dB = oracle.grad_B(B, tau, W)
    assert abs(np.sum(tau * dtau) - E) < 1e-12 * abs(E)
    assert abs(np.sum(B * dB) - 2.0 * E) < 1e-12 * abs(E)


def test_grad_central_differences_exact(grad_case):
    B, tau, W = grad_case
    rng = np.random.default_rng(15)
    h = 1e-3
    dtau = oracle.grad_tau(B, W)
    dB = oracle.grad_B(B, tau, W)
    D = rng.standard_normal(tau.shape)
    fd = (_E(B, tau + h * D, W) - _E(B, tau - h * D, W)) / (2 * h)
    assert abs(fd - np.sum(dtau * D)) < 1e-9 * np.abs(dtau * D).sum()
    D = rng.standard_normal(B.shape)
    fd = (_E(B + h * D, tau, W) - _E(B - h * D, tau, W)) / (2 * h)
    assert abs(fd - np.sum(dB * D)) < 1e-9 * np.abs(dB * D).sum()


def test_grad_single_entry_differences(grad_case):
    # central difference in one coordinate at a time (catches a wrong index in
    # one of the two terms of dE/dB even when the totals agree)
    B, tau, W = grad_case
    dB = oracle.grad_B(B, tau, W)
    dtau = oracle.grad_tau(B, W)
    h = 0.5
    for (P, x, y) in [(0, 1, 5), (8, 6, 0), (3, 2, 2)]:
        Bp, Bm = B.copy(), B.copy()
        Bp[P, x, y] += h
        Bm[P, x, y] -= h
        fd = (_E(Bp, tau, W) - _E(Bm, tau, W)) / (2 * h)
        assert abs(fd - dB[P, x, y]) < 1e-11 * max(1.0, abs(fd))
    for (i, j, c, d) in [(0, 2, 1, 6), (2, 2, 3, 3), (1, 0, 6, 1)]:
        tp, tm = tau.copy(), tau.copy()
        tp[i, j, c, d] += h
        tm[i, j, c, d] -= h
        fd = (_E(B, tp, W) - _E(B, tm, W)) / (2 * h)
        assert abs(fd - dtau[i, j, c, d]) < 1e-11 * max(1.0, abs(fd))


def test_grad_entries_match_full(grad_case):
    B, tau, W = grad_case
    dB = oracle.grad_B(B, tau, W)
    dtau = oracle.grad_tau(B, W)
    P, x, y = [0, 4, 8], [1, 6, 0], [5, 3, 2]
    np.testing.assert_allclose(oracle.grad_B_entries(B, tau, W, P, x, y), dB[P, x, y], rtol=1e-13)
    i, j, c, d = [0, 2, 1], [1, 2, 0], [6, 3, 0], [1, 3, 4]
    np.testing.assert_allclose(oracle.grad_tau_entries(B, W, i, j, c, d), dtau[i, j, c, d],
                               rtol=1e-13)


# --- generator sanity (not the method): exact pair symmetry of t2 and the
# magnitudes the configurations are quoted with
def test_generator_pair_symmetry_and_energy_scale(small_inputs):
    x = small_inputs
    assert np.array_equal(x.t2, x.t2.transpose(1, 0, 3, 2))
    assert np.array_equal(x.B, x.B.transpose(0, 2, 1))
    tau = oracle.tau(x.t1, x.t2)
    assert np.array_equal(tau, tau.transpose(1, 0, 3, 2))
    E = oracle.energy(oracle.ladder(x.B, tau), x.t2)
    assert 0.1 < E < 0.3
