"""Pins of the oracle's Philox4x32-10 and Sobol generators.

Philox is checked against triton's independent Philox4x32-10 (run on the CPU
in triton's interpreter, in a subprocess) and for uniformity.  Sobol is checked
against scipy for the two dimensions whose direction numbers are forced
(van der Corput and the degree-1 polynomial), and every dimension for the
stratification that defines a Sobol sequence.
"""
import json
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

_TRITON_SCRIPT = textwrap.dedent(
    """
    import os, sys, json
    os.environ["TRITON_INTERPRET"] = "1"
    import torch, triton, triton.language as tl

    @triton.jit
    def k(c_ptr, o_ptr, seed, n: tl.constexpr):
        i = tl.arange(0, n)
        c0 = tl.load(c_ptr + 4 * i + 0)
        c1 = tl.load(c_ptr + 4 * i + 1)
        c2 = tl.load(c_ptr + 4 * i + 2)
        c3 = tl.load(c_ptr + 4 * i + 3)
        a, b, c, d = tl.philox(seed, c0, c1, c2, c3)
        tl.store(o_ptr + 4 * i + 0, a)
        tl.store(o_ptr + 4 * i + 1, b)
        tl.store(o_ptr + 4 * i + 2, c)
        tl.store(o_ptr + 4 * i + 3, d)

    job = json.loads(sys.stdin.read())
    out = []
    for seed, ctrs in job:
        c = torch.tensor(ctrs, dtype=torch.int64).to(torch.int32).reshape(-1)
        o = torch.zeros_like(c)
        k[(1,)](c, o, seed, len(ctrs))
        out.append([int(x) & 0xFFFFFFFF for x in o.tolist()])
    print(json.dumps(out))
    """
)


def test_philox_against_triton(orc):
    pytest.importorskip("triton")
    rng = np.random.default_rng(5)
    job = []
    for _ in range(6):
        seed = int(rng.integers(0, 2 ** 63))
        ctrs = [[int(v) for v in rng.integers(0, 2 ** 32, 4)] for _ in range(16)]
        ctrs[0] = [0, 0, 0, 0]
        ctrs[1] = [0xFFFFFFFF] * 4
        job.append((seed, ctrs))
    env = dict(os.environ, TRITON_INTERPRET="1")
    res = subprocess.run([sys.executable, "-c", _TRITON_SCRIPT], input=json.dumps(job),
                         capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        pytest.skip("triton interpreter unavailable: " + res.stderr[-300:])
    ref = json.loads(res.stdout.strip().splitlines()[-1])
    for (seed, ctrs), r in zip(job, ref):
        key = [seed & 0xFFFFFFFF, seed >> 32]
        for i, c in enumerate(ctrs):
            got = orc.philox(c, key)
            assert list(map(int, got)) == r[4 * i:4 * i + 4]


def test_philox_uniformity(orc):
    vals = np.concatenate([orc.philox([i, 7, 3, 1], [123, 456]) for i in range(4096)])
    bins = np.bincount((vals >> 24).astype(np.int64), minlength=256)
    exp = len(vals) / 256
    chi = ((bins - exp) ** 2 / exp).sum()
    assert chi < 256 + 5 * np.sqrt(2 * 256)
    bits = np.unpackbits(vals.view(np.uint8)).mean()
    assert abs(bits - 0.5) < 0.01


def test_sobol_forced_dimensions_match_scipy(orc):
    qmc = pytest.importorskip("scipy.stats.qmc")
    n = 1024
    ref = qmc.Sobol(d=2, scramble=False).random(n)
    for d in range(2):
        got = np.array([orc.sobol_u32(i, d) for i in range(n)], dtype=np.float64) / 2.0 ** 32
        assert np.array_equal(got, ref[:, d]), d


def test_sobol_van_der_corput(orc):
    for k in range(1, 12):
        pts = sorted(orc.sobol_u32(i, 0) for i in range(2 ** k))
        assert pts == [j << (32 - k) for j in range(2 ** k)]


@pytest.mark.parametrize("dim", range(10))
def test_sobol_one_dimensional_stratification(orc, dim):
    # first 2^k points: one point in each of the 2^k dyadic intervals
    for k in range(1, 13):
        top = {orc.sobol_u32(i, dim) >> (32 - k) for i in range(2 ** k)}
        assert len(top) == 2 ** k, (dim, k)


def test_sobol_two_dimensional_net(orc):
    # dimensions 0 and 1 form a (0, m, 2)-net in base 2: every elementary box of
    # area 2^-m holds exactly one of the first 2^m points
    m = 8
    xs = [orc.sobol_u32(i, 0) for i in range(2 ** m)]
    ys = [orc.sobol_u32(i, 1) for i in range(2 ** m)]
    for a in range(m + 1):
        b = m - a
        boxes = {(x >> (32 - a) if a else 0, y >> (32 - b) if b else 0) for x, y in zip(xs, ys)}
        assert len(boxes) == 2 ** m, a


def test_sobol_direction_numbers_odd(orc):
    for dim in range(12):
        v = orc.sobol_directions(dim)
        for k in range(32):
            assert (int(v[k]) >> (31 - k)) & 1 == 1   # m_k odd


# The first primitive polynomials over GF(2), ordered by degree and then by
# their encoding (bit i = coefficient of x^i): x + 1; x^2 + x + 1; x^3 + x + 1,
# x^3 + x^2 + 1; x^4 + x + 1, x^4 + x^3 + 1; x^5 + x^2 + 1, x^5 + x^3 + 1,
# x^5 + x^3 + x^2 + x + 1, x^5 + x^4 + x^2 + x + 1, x^5 + x^4 + x^3 + x + 1,
# x^5 + x^4 + x^3 + x^2 + 1 (a textbook table; phi(2^s - 1) / s of degree s).
PRIMITIVE = [0b11, 0b111, 0b1011, 0b1101, 0b10011, 0b11001, 0b100101, 0b101001, 0b101111, 0b110111,
             0b111011, 0b111101]


def _gf2_mod(a, b):
    db = b.bit_length() - 1
    while a and a.bit_length() - 1 >= db:
        a ^= b << (a.bit_length() - 1 - db)
    return a


def _irreducible(p):
    """No factor of degree 1..deg/2 (trial division by every polynomial)."""
    d = p.bit_length() - 1
    return all(_gf2_mod(p, q) != 0 for q in range(2, 1 << (d // 2 + 1)) if q.bit_length() - 1 >= 1)


def test_primitive_polynomial_table():
    """The table is what it says: each entry irreducible with x of order
    2^s - 1, and no primitive polynomial of the same degree is missing or out
    of order."""
    for p in PRIMITIVE:
        s = p.bit_length() - 1
        assert _irreducible(p), bin(p)
        order = next(e for e in range(1, 1 << s) if _gf2_mod(1 << e, p) == 1)
        assert order == (1 << s) - 1, bin(p)
    by_deg = {}
    for p in PRIMITIVE:
        by_deg.setdefault(p.bit_length() - 1, []).append(p)
    for s, ps in by_deg.items():
        if s == 5:   # complete for degree <= 5: phi(31) / 5 = 6 entries
            assert len(ps) == 6
        assert ps == sorted(ps)
    assert [len(by_deg[s]) for s in (1, 2, 3, 4)] == [1, 1, 2, 2]   # phi(2^s - 1) / s


@pytest.mark.parametrize("dim", range(1, 12))
def test_sobol_direction_numbers_follow_the_primitive_polynomials(orc, dim):
    """Dimension d >= 1 uses the d-th primitive polynomial: its direction
    integers m_k start at 2^k - 1 (k <= s) and obey Sobol's recurrence
    m_k = 2 a_1 m_{k-1} ^ ... ^ 2^(s-1) a_(s-1) m_(k-s+1) ^ 2^s m_(k-s) ^ m_(k-s)
    for the polynomial x^s + a_1 x^(s-1) + ... + a_(s-1) x + 1."""
    p = PRIMITIVE[dim - 1]
    s = p.bit_length() - 1
    v = orc.sobol_directions(dim)
    m = [None] + [int(v[k]) >> (31 - k) for k in range(32)]   # m[1..32]
    for k in range(1, s + 1):
        assert m[k] == (1 << k) - 1, (dim, k)
    for k in range(s + 1, 33):
        x = m[k - s] ^ (m[k - s] << s)
        for j in range(1, s):
            if (p >> (s - j)) & 1:
                x ^= m[k - j] << j
        assert m[k] == x, (dim, k)
