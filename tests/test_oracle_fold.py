"""Pins of the oracle's generalised-Mira fold (Sec. 4.2) for the degree-2
relation m1 o m2 - mu m3 = e.

Pins: the decider's relaxed test holds on leaves (NARK = acc with mu = 1,
e = 0) and on every fold output (completeness); commitments of the folded
instance equal fresh commitments of the folded witness (homomorphism, checked
through the tau closed form, a route the fold does not take); the accumulation
verifier's RLC checks accept; MSM-mode and tau-mode folds agree; and a planted
orientation mistake is caught."""
import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


def _leaf(orc, seed, n, mode, tau, srs=None):
    m1 = Z.zkml_scalars(seed, n)
    m2 = Z.zkml_scalars(seed + 1, n)
    m4 = Z.zkml_scalars(seed + 2, n)
    return orc.leaf_init(m1, m2, m4, mode, srs, tau)


@pytest.fixture(scope="module")
def tau():
    return Z.tau(0)


def test_leaf_is_a_nark_accumulator(orc, tau):
    a = _leaf(orc, 100, 16, orc.COMMIT_TAU, tau)
    assert orc.decide_relation(a) == 0
    assert Z.fr_to_int(a.mu) == 1 and not a.e.any() and not a.E.any()
    for i in range(4):
        assert (a.C[i] == orc.commit_evals_tau(a.m[i], tau)).all()


def test_fold_completeness_and_homomorphism(orc, tau):
    n = 32
    L = _leaf(orc, 200, n, orc.COMMIT_TAU, tau)
    Rr = _leaf(orc, 300, n, orc.COMMIT_TAU, tau)
    g = Z.gammas(1, 1)[0]
    O, E1 = orc.fold(L, Rr, g, orc.COMMIT_TAU, tau=tau)
    assert orc.decide_relation(O) == 0
    assert orc.verify_fold(L, Rr, O, E1, g)
    for i in range(4):
        assert (O.C[i] == orc.commit_evals_tau(O.m[i], tau)).all()
    assert (O.E == orc.commit_evals_tau(O.e, tau)).all()
    # mu'' = gamma mu + mu' = gamma + 1 for two leaves.
    assert Z.fr_to_int(O.mu) == (Z.fr_to_int(g) + 1) % R
    # A second fold of two folded accumulators (mu != 1, e != 0) stays complete.
    O2, E2 = orc.fold(O, O.copy(), Z.gammas(2, 1)[0], orc.COMMIT_TAU, tau=tau)
    assert orc.decide_relation(O2) == 0
    assert (O2.E == orc.commit_evals_tau(O2.e, tau)).all()


def test_msm_mode_matches_tau_mode(orc, tau):
    n = 8
    srs = orc.srs_gen(tau, n)
    L = _leaf(orc, 400, n, orc.COMMIT_MSM, tau, srs)
    Rr = _leaf(orc, 500, n, orc.COMMIT_MSM, tau, srs)
    Lt = _leaf(orc, 400, n, orc.COMMIT_TAU, tau)
    assert (L.inst == Lt.inst).all()
    g = Z.gammas(1, 1)[0]
    Om, E1m = orc.fold(L, Rr, g, orc.COMMIT_MSM, srs=srs)
    Ot, E1t = orc.fold(L, Rr, g, orc.COMMIT_TAU, tau=tau)
    assert (Om.inst == Ot.inst).all() and (E1m == E1t).all()
    assert (Om.m == Ot.m).all() and (Om.e == Ot.e).all()


def test_planted_orientation_mistake_is_caught(orc, tau):
    # Planting on the CPU: fold with L and R swapped for the error update only
    # (e'' = e + gamma e1 + gamma^2 e' instead of e' + gamma e1 + gamma^2 e).
    n = 16
    L = _leaf(orc, 600, n, orc.COMMIT_TAU, tau)
    Rr = _leaf(orc, 700, n, orc.COMMIT_TAU, tau)
    O1, _ = orc.fold(L, Rr, Z.gammas(1, 1)[0], orc.COMMIT_TAU, tau=tau)
    O2, _ = orc.fold(Rr, L, Z.gammas(1, 2)[1], orc.COMMIT_TAU, tau=tau)
    g = Z.gammas(2, 1)[0]
    good, _ = orc.fold(O1, O2, g, orc.COMMIT_NONE)
    assert orc.decide_relation(good) == 0
    bad = good.copy()
    gi = Z.fr_to_int(g)
    for k in range(n):
        e1 = (Z.fr_to_int(good.e[k]) - Z.fr_to_int(O2.e[k]) - gi * gi * Z.fr_to_int(O1.e[k])) % R
        bad.e[k] = Z.int_to_fr((Z.fr_to_int(O1.e[k]) + e1 + gi * gi * Z.fr_to_int(O2.e[k])) % R)
    assert orc.decide_relation(bad) > 0


def test_fold_tree_is_sequential_pairwise_folding(orc, tau):
    n, count = 8, 4
    leaves = [_leaf(orc, 800 + 10 * i, n, orc.COMMIT_TAU, tau) for i in range(count)]
    g1, g2 = Z.gammas(1, 2), Z.gammas(2, 1)
    gam = np.concatenate([g1, g2])
    root = orc.fold_tree(leaves, gam, orc.COMMIT_TAU, tau=tau)
    a, _ = orc.fold(leaves[0], leaves[1], g1[0], orc.COMMIT_TAU, tau=tau)
    b, _ = orc.fold(leaves[2], leaves[3], g1[1], orc.COMMIT_TAU, tau=tau)
    c, _ = orc.fold(a, b, g2[0], orc.COMMIT_TAU, tau=tau)
    assert (root.m == c.m).all() and (root.e == c.e).all() and (root.inst == c.inst).all()
    assert orc.decide_relation(root) == 0
    for i in range(4):
        assert (root.C[i] == orc.commit_evals_tau(root.m[i], tau)).all()
    assert (root.E == orc.commit_evals_tau(root.e, tau)).all()


def _relation_holds(acc):
    """m1 o m2 - mu m3 = e at every position, over Python integers."""
    mu = Z.fr_to_int(acc.mu)
    for k in range(acc.n):
        a = [Z.fr_to_int(acc.m[i][k]) for i in range(3)]
        if (a[0] * a[1] - mu * a[2] - Z.fr_to_int(acc.e[k])) % R:
            return False
    return True


def test_decider_recheck_over_python_integers(orc, tau):
    n = 16
    L = _leaf(orc, 1000, n, orc.COMMIT_TAU, tau)
    Rr = _leaf(orc, 1100, n, orc.COMMIT_TAU, tau)
    assert _relation_holds(L) and _relation_holds(Rr)
    O, _ = orc.fold(L, Rr, Z.gammas(1, 1)[0], orc.COMMIT_NONE)
    O2, _ = orc.fold(O, O.copy(), Z.gammas(2, 1)[0], orc.COMMIT_NONE)
    for a in (O, O2):
        assert _relation_holds(a) and orc.decide_relation(a) == 0
    # one wrong error entry fails both the decider and the recheck
    bad = O2.copy()
    bad.e[3] = Z.int_to_fr((Z.fr_to_int(bad.e[3]) + 1) % R)
    assert not _relation_holds(bad) and orc.decide_relation(bad) == 1


def test_stacked_tree_matches_list_tree(orc, tau):
    n, count = 8, 8
    leaves = [_leaf(orc, 1200 + 10 * i, n, orc.COMMIT_NONE, tau) for i in range(count)]
    gam = np.concatenate([Z.gammas(l, count >> l) for l in range(1, 4)])
    want = orc.fold_tree(leaves, gam, orc.COMMIT_NONE)
    m = np.zeros((count, 4, n, 4), np.uint64)
    e = np.zeros((count, n, 4), np.uint64)
    inst = np.zeros((count, orc.INST_LIMBS), np.uint64)
    for j in range(count):
        base = 1200 + 10 * j
        m[j, 0], m[j, 1], m[j, 3] = (Z.zkml_scalars(base + i, n) for i in range(3))
        orc.leaf_init_into(m[j], e[j], inst[j])
    orc.fold_tree_stacked(m, e, inst, gam)
    assert (m[0] == want.m).all() and (e[0] == want.e).all() and (inst[0] == want.inst).all()
