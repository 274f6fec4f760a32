"""Pins of the GLV constants in the device code (curve.cuh, struct Glv)
against their definitions: beta is a primitive cube root of unity in F_q,
the lambda the lattice basis implies is one in F_r and phi(G) = (beta x, y)
equals lambda G (the oracle's affine arithmetic), both basis vectors lie in
the lattice {(x, y): x + y lambda = 0 mod r} with determinant +-r, the
rounding constants are floor(b2 2^256 / r) and floor(-b1 2^256 / r), and the
split k = k1 + k2 lambda keeps |k1|, |k2| below 2^130 on random and edge
scalars."""
import os
import random
import re

import zkinputs as Z

Q, R = Z.Q_MOD, Z.R_MOD
SRC = os.path.join(os.path.dirname(__file__), "..", "paper_2507_07031_b300", "csrc", "curve.cuh")


def _constants():
    text = open(SRC).read()
    body = text[text.index("struct Glv {"):text.index("constexpr int kGlvWords")]
    out = {}
    for name, arr in re.findall(r"constexpr uint32_t (\w+)\(int i\) \{[^\n]*\n\s*constexpr uint32_t v\[8\] = \{([^}]*)\}",
                                body):
        words = [int(w.strip().rstrip("u"), 0) for w in arr.split(",")]
        assert len(words) == 8
        out[name] = sum(w << (32 * i) for i, w in enumerate(words))
    return out


def test_glv_constants(orc):
    c = _constants()
    assert set(c) == {"beta_mont", "a1", "b1_abs", "a2", "b2", "g1", "g2"}
    beta = c["beta_mont"] * pow(1 << 256, -1, Q) % Q
    assert beta != 1 and pow(beta, 3, Q) == 1
    a1, b1, a2, b2 = c["a1"], -c["b1_abs"], c["a2"], c["b2"]
    lam = -a1 * pow(b1, -1, R) % R
    assert lam != 1 and pow(lam, 3, R) == 1
    assert (a2 + b2 * lam) % R == 0
    assert abs(a1 * b2 - a2 * b1) == R
    assert c["g1"] == (b2 << 256) // R and c["g2"] == ((-b1) << 256) // R
    G = orc.g1_generator()
    want = orc.g1_mul(G, Z.int_to_fr(lam))
    gx = Z.fr_to_int(G[:4])  # affine x of G (limbs 0..3)
    gy = Z.fr_to_int(G[4:])
    phi = [Z.int_to_fr(beta * gx % Q), Z.int_to_fr(gy)]
    import numpy as np
    assert np.array_equal(want, np.concatenate(phi))


def test_glv_split_bounds():
    c = _constants()
    a1, b1, a2, b2 = c["a1"], -c["b1_abs"], c["a2"], c["b2"]
    lam = -a1 * pow(b1, -1, R) % R
    rng = random.Random(7)
    ks = [0, 1, 2, R - 1, (R - 1) // 2, (R + 1) // 2, lam, R - lam, 1 << 128, (1 << 253) + 12345]
    ks += [rng.randrange(R) for _ in range(20000)]
    for k in ks:
        c1 = (k * c["g1"]) >> 256
        c2 = (k * c["g2"]) >> 256
        k1 = k - c1 * a1 - c2 * a2
        k2 = -c1 * b1 - c2 * b2
        assert (k1 + k2 * lam - k) % R == 0
        assert abs(k1) < (1 << 130) and abs(k2) < (1 << 130)
