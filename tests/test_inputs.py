"""The seeded generators: SplitMix64 reference outputs, rejection sampling into
F_r, fixed-point encoding, and the workload shapes."""
import numpy as np

import zkinputs as Z


def test_splitmix64_reference_outputs():
    # Seed 0: the first two outputs of the published reference implementation.
    out = Z.splitmix64(0, 0, 2)
    assert [hex(int(x)) for x in out] == ["0xe220a8397b1dcdaf", "0x6e789e6aa1b965f4"]
    # The vectorised counter form equals the sequential state-update form.
    M, s, seq = (1 << 64) - 1, 77, []
    for _ in range(50):
        s = (s + 0x9E3779B97F4A7C15) & M
        z = ((s ^ (s >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        seq.append(z ^ (z >> 31))
    assert [int(x) for x in Z.splitmix64(77, 0, 50)] == seq
    # Counter-based: any window of the stream equals the matching slice.
    assert (Z.splitmix64(5, 10, 4) == Z.splitmix64(5, 0, 14)[10:]).all()


def test_fr_uniform_canonical_and_deterministic():
    a = Z.fr_uniform(3, 1000)
    assert all(Z.fr_to_int(x) < Z.R_MOD for x in a)
    assert (a == Z.fr_uniform(3, 1000)).all()
    assert (a[:10] == Z.fr_uniform(3, 10)).all()
    assert Z.fr_to_int(Z.tau(0)) != 0


def test_zkml_encoding_and_shapes():
    s = Z.zkml_scalars(4, 5000)
    q = Z.int8_uniform(4, 5000)
    for qi, si in zip(q[:200], s[:200]):
        assert Z.fr_to_int(si) == (int(qi) << 16) % Z.R_MOD
    g = Z.int8_gauss(4, 5000)
    assert g.min() >= -128 and g.max() <= 127 and 25 < g.std() < 40
    sizes = Z.cnn_poly_sizes()
    assert sizes.shape[0] == 256 and sizes.sum() == 1 << 24
    assert sorted(sizes.tolist()) == sorted(Z.cnn_poly_sizes(8).tolist())
    t = Z.poisson_arrivals(10, 1000, 20.0)
    assert np.all(np.diff(t) > 0) and 40 < t[-1] < 60
