"""Pins for the t1-dressed ladder of the CPU oracle (Eq. pp-Ladder-0 with the
dressed integrals of Eq. pp-Ladder-2 / pp-Ladder-21).  The oracle follows the
factorised form of Eq. pp-Ladder-2; the tests check it against the defining
form of Eq. pp-Ladder-1 built from explicit four-index arrays, a closed form,
the undressed special case and the invariants of the term.  No GPU needed."""
import numpy as np
import pytest

import oracle


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def case(seed, o, v, n, pair_symmetric=False):
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, v, v))        # general: not symmetric in a <-> c
    B_ov = rng.standard_normal((n, o, v))
    t1 = rng.standard_normal((o, v))
    tau = rng.standard_normal((o, o, v, v))
    if pair_symmetric:
        tau = 0.5 * (tau + tau.transpose(1, 0, 3, 2))
    return B, B_ov, t1, tau


# Eq. pp-Ladder-1 written with the explicit integral arrays of Eq. eri under
# Eq. RIM, v^{pq}_{rs} = (pr|qs) = sum_P m^P_pr m^P_qs:
#   b^{ab}_{cd} = v^{ab}_{cd} - sum_k v^{ak}_{cd} t_k^b - sum_k t_k^a v^{kb}_{cd}
def brute_eq1(B, B_ov, t1, tau):
    v_ab = np.einsum("pac,pbd->abcd", B, B)        # (ac|bd)
    v_ak = np.einsum("pac,pkd->akcd", B, B_ov)     # (ac|kd)
    v_kb = np.einsum("pkc,pbd->kbcd", B_ov, B)     # (kc|bd)
    b = v_ab - np.einsum("akcd,kb->abcd", v_ak, t1) - np.einsum("ka,kbcd->abcd", t1, v_kb)
    return np.einsum("abcd,ijcd->ijab", b, tau)


@pytest.mark.parametrize("o,v,n,seed", [(1, 3, 2, 0), (3, 7, 5, 1), (4, 12, 20, 2), (2, 17, 9, 3)])
def test_dressed_equals_eq1_brute_force(o, v, n, seed):
    B, B_ov, t1, tau = case(seed, o, v, n)
    assert rel(oracle.ladder_dressed(B, B_ov, t1, tau), brute_eq1(B, B_ov, t1, tau)) < 1e-13


def test_dressed_reduces_to_undressed_without_singles():
    B, B_ov, t1, tau = case(4, 3, 10, 6)
    R = oracle.ladder_dressed(B, B_ov, np.zeros_like(t1), tau)
    assert np.array_equal(R, oracle.ladder(B, tau))


# One auxiliary function with B^0_ac = u_a u_c and Bov^0_kc = w_k u_c:
#   mbar_bd = s_b u_d with s_b = sum_k w_k t_k^b, and
#   R_ij^ab = (u_a u_b - u_a s_b - s_a u_b) sum_cd u_c u_d tau_ij^cd.
# A sign error on either singles term, a swapped mbar index or t_k^b read as
# t_b^k changes the prefactor.
def test_dressed_rank_one_closed_form():
    rng = np.random.default_rng(5)
    o, v = 4, 13
    u = rng.standard_normal(v)
    w = rng.standard_normal(o)
    t1 = rng.standard_normal((o, v))
    tau = rng.standard_normal((o, o, v, v))
    B = np.outer(u, u)[None]
    B_ov = np.outer(w, u)[None]
    s = w @ t1
    pref = np.outer(u, u) - np.outer(u, s) - np.outer(s, u)
    uu = np.einsum("c,ijcd,d->ij", u, tau, u)
    expect = uu[:, :, None, None] * pref[None, None]
    assert rel(oracle.ladder_dressed(B, B_ov, t1, tau), expect) < 1e-13


# b^{ab}_{cd} = b^{ba}_{dc} holds for the dressed integrals too (the two
# singles terms exchange), so a pair-symmetric tau gives R_ij^ab = R_ji^ba.
def test_dressed_pair_symmetry():
    B, B_ov, t1, tau = case(6, 4, 11, 7, pair_symmetric=True)
    R = oracle.ladder_dressed(B, B_ov, t1, tau)
    assert np.abs(R - R.transpose(1, 0, 3, 2)).max() <= 1e-13 * np.abs(R).max()


def test_dressed_linear_in_tau():
    B, B_ov, t1, tau = case(7, 3, 9, 5)
    tau2 = np.random.default_rng(8).standard_normal(tau.shape)
    lhs = oracle.ladder_dressed(B, B_ov, t1, 2.0 * tau - 0.5 * tau2)
    rhs = 2.0 * oracle.ladder_dressed(B, B_ov, t1, tau) - 0.5 * oracle.ladder_dressed(B, B_ov, t1, tau2)
    assert rel(lhs, rhs) < 1e-13


def test_dressed_pairs_match_columns():
    B, B_ov, t1, tau = case(9, 3, 14, 8)
    R = oracle.ladder_dressed(B, B_ov, t1, tau)
    pa, pb = [0, 13, 5, 7], [13, 0, 5, 2]
    got = oracle.ladder_dressed_pairs(B, B_ov, t1, tau, pa, pb)
    for k, (a, b) in enumerate(zip(pa, pb)):
        assert np.abs(got[k] - R[:, :, a, b]).max() <= 1e-13 * np.abs(R).max()
