"""Pins of the oracle's fold for the degree-3 relation
m1 o m2 o m3 - mu^2 m4 = e (Sec. 4.2's general-d fold with d = 3: two cross
terms e_1, e_2 with commitments E_1, E_2, and
e'' = e' + gamma e_1 + gamma^2 e_2 + gamma^3 e).

Completeness of the decider after folds with random gamma fixes both cross
terms (a wrong coefficient of gamma or gamma^2 makes the folded error vector
miss the relation); homomorphism and the verifier's RLC checks pin the
instance side; the relation itself is rechecked here over Python integers."""
import numpy as np
import pytest

import zkinputs as Z

R = Z.R_MOD


@pytest.fixture
def deg3(orc):
    orc.set_degree(3)
    yield
    orc.set_degree(2)


def _leaf(orc, seed, n, tau):
    return orc.leaf_init(Z.zkml_scalars(seed, n), Z.zkml_scalars(seed + 1, n),
                         Z.zkml_scalars(seed + 2, n), orc.COMMIT_TAU, None, tau)


def _relation_holds(acc):
    mu = Z.fr_to_int(acc.mu)
    for k in range(acc.n):
        a = [Z.fr_to_int(acc.m[i][k]) for i in range(4)]
        if (a[0] * a[1] * a[2] - mu * mu * a[3] - Z.fr_to_int(acc.e[k])) % R:
            return False
    return True


def test_degree3_leaf_and_folds(orc, deg3):
    tau = Z.tau(0)
    n = 16
    L, Rr = _leaf(orc, 800, n, tau), _leaf(orc, 900, n, tau)
    assert orc.decide_relation(L) == 0 and _relation_holds(L)
    for i in range(4):
        assert (L.C[i] == orc.commit_evals_tau(L.m[i], tau)).all()
    g = Z.gammas(1, 1)[0]
    O, E = orc.fold(L, Rr, g, orc.COMMIT_TAU, tau=tau)
    assert E.shape == (16,)
    assert orc.decide_relation(O) == 0 and _relation_holds(O)
    assert orc.verify_fold(L, Rr, O, E, g)
    for i in range(4):
        assert (O.C[i] == orc.commit_evals_tau(O.m[i], tau)).all()
    assert (O.E == orc.commit_evals_tau(O.e, tau)).all()
    # folds of folded accumulators (mu != 1, e != 0)
    O2, E2 = orc.fold(O, O.copy(), Z.gammas(2, 1)[0], orc.COMMIT_TAU, tau=tau)
    assert orc.decide_relation(O2) == 0 and _relation_holds(O2)
    assert (O2.E == orc.commit_evals_tau(O2.e, tau)).all()
    # a tampered cross-term commitment is rejected by the verifier
    bad = E.copy()
    bad[8:] = orc.g1_add(E[8:], orc.g1_generator())
    assert not orc.verify_fold(L, Rr, O, bad, g)


def test_degree3_tree_equals_pairwise_folds(orc, deg3):
    tau = Z.tau(0)
    n = 8
    leaves = [_leaf(orc, 1000 + 10 * i, n, tau) for i in range(4)]
    gam = Z.gammas(1, 2)
    gam2 = Z.gammas(2, 1)
    a, _ = orc.fold(leaves[0], leaves[1], gam[0], orc.COMMIT_TAU, tau=tau)
    b, _ = orc.fold(leaves[2], leaves[3], gam[1], orc.COMMIT_TAU, tau=tau)
    want, _ = orc.fold(a, b, gam2[0], orc.COMMIT_TAU, tau=tau)
    root = orc.fold_tree(leaves, np.concatenate([gam, gam2]), orc.COMMIT_TAU, tau=tau)
    assert (root.m == want.m).all() and (root.e == want.e).all() and (root.inst == want.inst).all()
    assert orc.decide_relation(root) == 0
