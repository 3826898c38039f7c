"""The library's Zeeman components (closed-form Delta J = 0, +-1 line strengths,
computed on the host) against the oracle's (Racah 3j symbols): two independent
constructions of the Section 5 full pattern.  No GPU needed."""
import numpy as np
import pytest

TRANSITIONS = [(2, 11 / 6, 2, 1.5), (1, 2.5, 0, 0.0), (0, 0.0, 1, 2.5), (1, 1.5, 2, 1.5),
               (3, 1.25, 2, 1.0), (2, 1.0, 3, 1.25), (4, 1.3, 4, 1.1), (4, 1.2, 3, 1.05), (1, 2.0, 1, 1.0)]


@pytest.mark.parametrize("jl,gl,ju,gu", TRANSITIONS)
def test_library_components_equal_oracle(orc, jl, gl, ju, gu):
    from paper_1208_0302_gb300 import api
    lib = api.zeeman_components((6301.5, 1.667, 1.0, jl, gl, ju, gu))
    ref = orc.zeeman_components(jl, gl, ju, gu)
    for (s1, w1), (s2, w2) in zip(lib, ref):
        o1, o2 = np.argsort(s1), np.argsort(s2)
        assert np.allclose(s1[o1], s2[o2], atol=1e-14)
        assert np.allclose(w1[o1], w2[o2], atol=1e-14)


def test_effective_triplet_components():
    from paper_1208_0302_gb300 import api
    comps = api.zeeman_components((6302.5, 2.5, 1.0))
    assert [c[0].tolist() for c in comps] == [[-2.5], [0.0], [2.5]]


def test_invalid_transition_rejected():
    from paper_1208_0302_gb300 import _lib, api
    with pytest.raises(_lib.GenesisError):
        api.zeeman_components((6301.5, 1.667, 1.0, 0, 1.0, 0, 1.0))
    with pytest.raises(_lib.GenesisError):
        api.zeeman_components((6301.5, 1.667, 1.0, 1, 1.0, 3, 1.0))
