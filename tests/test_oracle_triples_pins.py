"""Pins for the perturbative triples of the CPU oracle (Sec. II.A: E(T) with
W, V and D as printed there).  The oracle evaluates the printed formulas with
integrals formed from RI factors; the tests check it against hand-derived
closed forms for factors and amplitudes of rank one and two, the symmetry the
permutation operator P gives W, and the scaling the formulas fix.  No GPU."""
import itertools

import numpy as np

import oracle


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def low_rank_case(seed, o=3, v=5, t1_scale=1.0):
    """One auxiliary function: Bvv = u u^T, Bov[k][c] = w_k u_c,
    Boo[j][l] = z_j z_l; doubles of rank two
    t_ij^ab = x_i x'_j y_a y'_b + x'_i x_j y'_a y_b (pair symmetric)."""
    rng = np.random.default_rng(seed)
    u, y, yp = rng.standard_normal((3, v))
    w, x, xp, z = rng.standard_normal((4, o))
    B = np.outer(u, u)[None]
    B_ov = np.outer(w, u)[None]
    B_oo = np.outer(z, z)[None]
    t2 = np.einsum("i,j,a,b->ijab", x, xp, y, yp) + np.einsum("i,j,a,b->ijab", xp, x, yp, y)
    t1 = t1_scale * rng.standard_normal((o, v))
    vecs = dict(u=u, y=y, yp=yp, w=w, x=x, xp=xp, z=z)
    return B, B_ov, B_oo, t1, t2, vecs


def outer6(i, j, k, a, b, c):
    return np.einsum("i,j,k,a,b,c->ijkabc", i, j, k, a, b, c)


def closed_form_raw(vv):
    """X_ijk^abc = sum_d v_di^ba t_kj^cd - sum_l v_kl^cj t_il^ab worked out by
    hand for the low-rank case (v_di^ba = u_b u_d w_i u_a, v_kl^cj = w_k u_c z_j z_l):
      first term  u_a u_b w_i (s1' x_k x'_j y_c + s1 x'_k x_j y'_c)
      second term w_k u_c z_j (s2' x_i y_a y'_b + s2 x'_i y'_a y_b)
    with s1 = u.y, s1' = u.y', s2 = z.x, s2' = z.x'."""
    u, y, yp, w, x, xp, z = (vv[k] for k in ("u", "y", "yp", "w", "x", "xp", "z"))
    s1, s1p, s2, s2p = u @ y, u @ yp, z @ x, z @ xp
    first = s1p * outer6(w, xp, x, u, u, y) + s1 * outer6(w, x, xp, u, u, yp)
    second = s2p * outer6(x, z, w, y, yp, u) + s2 * outer6(xp, z, w, yp, y, u)
    return first - second


def apply_P(X):
    """P_ijk^abc f(ijk,abc) = f(ijk,abc) + f(ikj,acb) + f(kij,cab) + f(kji,cba)
    + f(jki,bca) + f(jik,bac), on a tensor indexed [i,j,k,a,b,c]: the term
    f(kij,cab) is the tensor Y with Y[i,j,k,a,b,c] = X[k,i,j,c,a,b], that is
    X.transpose(1, 2, 0, 4, 5, 3), and so on."""
    axes = [(0, 1, 2, 3, 4, 5),   # f(ijk, abc)
            (0, 2, 1, 3, 5, 4),   # f(ikj, acb)
            (1, 2, 0, 4, 5, 3),   # f(kij, cab)
            (2, 1, 0, 5, 4, 3),   # f(kji, cba)
            (2, 0, 1, 5, 3, 4),   # f(jki, bca)
            (1, 0, 2, 4, 3, 5)]   # f(jik, bac)
    return sum(X.transpose(ax) for ax in axes)


def test_W_matches_the_low_rank_closed_form():
    B, B_ov, B_oo, t1, t2, vv = low_rank_case(0)
    W_ref = apply_P(closed_form_raw(vv))
    o = t1.shape[0]
    for i, j, k in itertools.product(range(o), repeat=3):
        W, _ = oracle.triples_wv(B, B_ov, B_oo, t1, t2, i, j, k)
        assert rel(W, W_ref[i, j, k]) < 1e-13, (i, j, k)


def test_V_adds_the_three_singles_terms():
    """V - W = v_jk^bc t_i^a + v_ik^ac t_j^b + v_ij^ab t_k^c with
    v_jk^bc = (bj|ck) = w_j u_b w_k u_c in the low-rank case."""
    B, B_ov, B_oo, t1, t2, vv = low_rank_case(1)
    u, w = vv["u"], vv["w"]
    o = t1.shape[0]
    for i, j, k in [(0, 1, 2), (2, 2, 0), (1, 1, 1)]:
        W, V = oracle.triples_wv(B, B_ov, B_oo, t1, t2, i, j, k)
        ref = (w[j] * w[k] * np.einsum("a,b,c->abc", t1[i], u, u)
               + w[i] * w[k] * np.einsum("a,b,c->abc", u, t1[j], u)
               + w[i] * w[j] * np.einsum("a,b,c->abc", u, u, t1[k]))
        assert rel(V - W, ref) < 1e-13
    assert o == 3


def test_W_has_the_symmetry_of_P():
    """W_ijk^abc is unchanged by any simultaneous permutation of (i,j,k) and
    (a,b,c): a dropped or repeated term of P breaks this."""
    rng = np.random.default_rng(2)
    o, v, n = 3, 6, 4
    B = rng.standard_normal((n, v, v))
    B_ov = rng.standard_normal((n, o, v))
    B_oo = rng.standard_normal((n, o, o))
    t2 = rng.standard_normal((o, o, v, v))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    t1 = rng.standard_normal((o, v))
    W0, _ = oracle.triples_wv(B, B_ov, B_oo, t1, t2, 0, 1, 2)
    ijk = (0, 1, 2)
    for p in itertools.permutations(range(3)):
        W, _ = oracle.triples_wv(B, B_ov, B_oo, t1, t2, *[ijk[q] for q in p])
        assert rel(W.transpose(np.argsort(p)), W0) < 1e-13


def test_energy_from_the_closed_forms():
    """E(T) assembled from the closed-form W and V of the low-rank case."""
    B, B_ov, B_oo, t1, t2, vv = low_rank_case(3, o=3, v=4, t1_scale=0.3)
    rng = np.random.default_rng(4)
    e_occ = rng.uniform(-1.5, -0.3, 3)
    e_vir = rng.uniform(0.1, 3.0, 4)
    u, w = vv["u"], vv["w"]
    W = apply_P(closed_form_raw(vv))
    V = W + (np.einsum("j,k,ia,b,c->ijkabc", w, w, t1, u, u)
             + np.einsum("i,k,a,jb,c->ijkabc", w, w, u, t1, u)
             + np.einsum("i,j,a,b,kc->ijkabc", w, w, u, u, t1))
    D = (e_occ[:, None, None, None, None, None] + e_occ[None, :, None, None, None, None]
         + e_occ[None, None, :, None, None, None] - e_vir[None, None, None, :, None, None]
         - e_vir[None, None, None, None, :, None] - e_vir[None, None, None, None, None, :])
    num = (4 * W + W.transpose(0, 1, 2, 4, 5, 3) + W.transpose(0, 1, 2, 5, 3, 4)) * \
          (V - V.transpose(0, 1, 2, 5, 4, 3))
    E_ref = float((num / (3 * D)).sum())
    E = oracle.triples(B, B_ov, B_oo, t1, t2, e_occ, e_vir)
    assert abs(E - E_ref) <= 1e-12 * abs(E_ref)


def test_energy_scaling_and_vanishing_doubles():
    """Without singles V = W, so E(T) is quadratic in t2; without doubles
    W = 0 and E(T) = 0."""
    rng = np.random.default_rng(5)
    o, v, n = 3, 7, 5
    B = rng.standard_normal((n, v, v))
    B_ov = rng.standard_normal((n, o, v))
    B_oo = rng.standard_normal((n, o, o))
    t2 = rng.standard_normal((o, o, v, v))
    t2 = 0.5 * (t2 + t2.transpose(1, 0, 3, 2))
    e_occ = rng.uniform(-1.5, -0.3, o)
    e_vir = rng.uniform(0.1, 3.0, v)
    z1 = np.zeros((o, v))
    E1 = oracle.triples(B, B_ov, B_oo, z1, t2, e_occ, e_vir)
    E3 = oracle.triples(B, B_ov, B_oo, z1, 3.0 * t2, e_occ, e_vir)
    assert abs(E3 - 9.0 * E1) <= 1e-12 * abs(E3)
    t1 = rng.standard_normal((o, v))
    assert oracle.triples(B, B_ov, B_oo, t1, np.zeros_like(t2), e_occ, e_vir) == 0.0


def test_sorted_triple_identity():
    """The identity the GPU evaluation rests on: for a sorted triple
    i >= j >= k, the printed per-(i,j,k) sums over its distinct orderings
    equal m * sum_abc Z^abc (3 V^abc - V^acb - V^bac - V^cba) / (3 D^abc)
    with Z^abc = 4 W^abc + W^bca + W^cab, formed from W and V of the sorted
    triple alone; m = 2, 1 or 1/3 for three, two or one distinct indices.
    Also: the per-ordering sums are not all equal (so the weight alone would
    not do), and summing the right-hand side over the sorted triples gives
    the oracle's E(T).  Brute force over the oracle's own W and V."""
    import synthetic
    o, v, n = 4, 6, 14
    x = synthetic.make_inputs(o, v, n, 7)
    args = (x.B, x.B_ov, x.B_oo, x.t1, x.t2)

    def D(i, j, k):
        return (x.e_occ[i] + x.e_occ[j] + x.e_occ[k])[()] - (
            x.e_vir[:, None, None] + x.e_vir[None, :, None] + x.e_vir[None, None, :])

    def printed(i, j, k):
        W, V = oracle.triples_wv(*args, i, j, k)
        Z = 4.0 * W + W.transpose(1, 2, 0) + W.transpose(2, 0, 1)
        return float(np.sum(Z * (V - V.transpose(2, 1, 0)) / (3.0 * D(i, j, k))))

    def sorted_form(i, j, k):
        W, V = oracle.triples_wv(*args, i, j, k)
        Z = 4.0 * W + W.transpose(1, 2, 0) + W.transpose(2, 0, 1)
        Y = 3.0 * V - V.transpose(0, 2, 1) - V.transpose(1, 0, 2) - V.transpose(2, 1, 0)
        m = 1.0 / 3.0 if i == k else (1.0 if (i == j or j == k) else 2.0)
        Dijk = D(i, j, k)
        # scale of the rounding: the terms' magnitudes before V's cancellation
        Ya = 3.0 * np.abs(V) + np.abs(V.transpose(0, 2, 1)) + np.abs(V.transpose(1, 0, 2)) + \
            np.abs(V.transpose(2, 1, 0))
        return (m * float(np.sum(Z * Y / (3.0 * Dijk))),
                m * float(np.sum(np.abs(Z) * Ya / (3.0 * np.abs(Dijk)))))

    total = 0.0
    for i in range(o):
        for j in range(i + 1):
            for k in range(j + 1):
                perms = set(itertools.permutations((i, j, k)))
                lhs = sum(printed(*p) for p in perms)
                rhs, scale = sorted_form(i, j, k)
                # (i = i = k: both sides vanish; rounding is measured on the terms' scale)
                assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), scale), (i, j, k, lhs, rhs)
                total += rhs
    vals = sorted(printed(*p) for p in itertools.permutations((3, 1, 0)))
    assert max(vals) - min(vals) > 1e-3 * abs(vals[0])
    E = oracle.triples(*args, x.e_occ, x.e_vir)
    assert abs(total - E) <= 1e-12 * abs(E)
