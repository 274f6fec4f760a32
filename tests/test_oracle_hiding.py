"""Pins of the oracle's hiding commitment [f(tau)]_1 + s H (Sec. 4.2: the
accumulation's zero-knowledge argument blinds every KZG commitment by s H).

s = 0 gives the plain commitment; the map (c, s) -> com is linear; with
H = G and the known tau the commitment is (f(tau) + s) G in closed form."""
import numpy as np

import zkinputs as Z

R = Z.R_MOD


def test_hiding_commitment_pins(orc):
    tau = Z.tau(0)
    srs = orc.srs_gen(tau, 40)
    G = orc.g1_generator()
    H = orc.g1_mul(G, Z.int_to_fr(0xC0FFEE))
    c1, c2 = Z.fr_uniform(61, 40), Z.fr_uniform(62, 40)
    s1, s2 = Z.fr_uniform(63, 1)[0], Z.fr_uniform(64, 1)[0]
    zero = np.zeros(4, np.uint64)
    assert np.array_equal(orc.commit_hiding(srs, c1, H, zero), orc.msm(srs, c1))
    c12 = np.stack([orc.fadd(orc.FR, a, b) for a, b in zip(c1, c2)])
    s12 = orc.fadd(orc.FR, s1, s2)
    lhs = orc.commit_hiding(srs, c12, H, s12)
    rhs = orc.g1_add(orc.commit_hiding(srs, c1, H, s1), orc.commit_hiding(srs, c2, H, s2))
    assert np.array_equal(lhs, rhs)
    t = Z.fr_to_int(tau)
    f_tau = sum(Z.fr_to_int(a) * pow(t, i, R) for i, a in enumerate(c1)) % R
    want = orc.g1_mul(G, Z.int_to_fr((f_tau + Z.fr_to_int(s1)) % R))
    assert np.array_equal(orc.commit_hiding(srs, c1, G, s1), want)
