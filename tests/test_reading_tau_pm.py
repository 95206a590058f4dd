"""The paper cites, but does not print, the symmetric/antisymmetric split of
the ladder term that cuts the leading cost to a quarter (Sec. II.C).  This
test states the reading the CUDA path implements and checks it against the
plain oracle on the CPU.

Reading (exact in exact arithmetic), for tau with pair symmetry
tau_ij^cd = tau_ji^dc (Sec. II.C):
  virtual indices are cut into blocks of 8 (v padded with zeros);
  for each block pair k <= l and each slot (c, d) in C_k x C_l:
    T+_ij[kl, cd] = w_kl (tau_ij^cd + tau_ij^dc) / 2,   i <= j
    T-_ij[kl, cd] = w_kl (tau_ij^cd - tau_ij^dc) / 2,   i <  j
    V+_ab[kl, cd] = (ac|bd) + (ad|bc)
    V-_ab[kl, cd] = (ac|bd) - (ad|bc)
  with w_kl = 1/2 on diagonal block pairs (k = l) and 1 otherwise;
    R+_ij^ab = sum_slots T+ V+ = (R_ij^ab + R_ij^ba) / 2
    R-_ij^ab = sum_slots T- V- = (R_ij^ab - R_ij^ba) / 2
  and the unpacking R_ij^ab = R+ + R-, R_ij^ba = R+ - R-, R_ji^ba = R_ij^ab,
  R_ji^ab = R_ij^ba, with R- = 0 when i = j or a = b.
"""
import numpy as np
import pytest

import oracle
import synthetic

CB = 8


def slot_scheme(B, tau):
    n, v, _ = B.shape
    o = tau.shape[0]
    vp = -(-v // CB) * CB
    nb = vp // CB
    Bp = np.zeros((n, vp, vp))
    Bp[:, :v, :v] = B
    tp = np.zeros((o, o, vp, vp))
    tp[:, :, :v, :v] = tau
    I = np.einsum("pac,pbd->abcd", Bp, Bp)  # (ac|bd), test-side only
    Rp = np.zeros((o, o, vp, vp))
    Rm = np.zeros((o, o, vp, vp))
    for k in range(nb):
        for l in range(k, nb):
            w = 0.5 if k == l else 1.0
            C = slice(k * CB, (k + 1) * CB)
            D = slice(l * CB, (l + 1) * CB)
            tcd = tp[:, :, C, D]
            tdc = tp[:, :, D, C].transpose(0, 1, 3, 2)
            Tp = w * 0.5 * (tcd + tdc)
            Tm = w * 0.5 * (tcd - tdc)
            Icd = I[:, :, C, D]
            Idc = I[:, :, D, C].transpose(0, 1, 3, 2)
            Vp = Icd + Idc
            Vm = Icd - Idc
            Rp += np.einsum("ijcd,abcd->ijab", Tp, Vp)
            Rm += np.einsum("ijcd,abcd->ijab", Tm, Vm)
    # the kernel only forms i <= j (plus) and i < j (minus): use those, unpack
    R = np.empty((o, o, v, v))
    for i in range(o):
        for j in range(i, o):
            for a in range(v):
                for b in range(a, v):
                    p = Rp[i, j, a, b]
                    m = 0.0 if (i == j or a == b) else Rm[i, j, a, b]
                    R[i, j, a, b] = p + m
                    R[i, j, b, a] = p - m
                    R[j, i, b, a] = p + m
                    R[j, i, a, b] = p - m
    return R, Rp[:, :, :v, :v], Rm[:, :, :v, :v]


@pytest.mark.parametrize("o,v,n,seed", [(1, 5, 3, 0), (3, 8, 6, 1), (4, 13, 20, 2), (4, 24, 96, 0)])
def test_slot_scheme_reconstructs_plain_result(o, v, n, seed):
    x = synthetic.make_inputs(o, v, n, seed)
    rng = np.random.default_rng(seed + 50)
    B = rng.standard_normal((n, v, v))  # general B: no a<->c symmetry assumed
    tau = oracle.tau(x.t1, x.t2)
    R, Rp, Rm = slot_scheme(B, tau)
    Ref = oracle.ladder(B, tau)
    scale = np.linalg.norm(Ref)
    assert np.linalg.norm(R - Ref) / scale < 1e-13
    assert np.linalg.norm(Rp - 0.5 * (Ref + Ref.transpose(0, 1, 3, 2))) / scale < 1e-13
    assert np.linalg.norm(Rm - 0.5 * (Ref - Ref.transpose(0, 1, 3, 2))) / scale < 1e-13
