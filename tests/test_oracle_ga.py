"""Pins of the oracle's genetic algorithm (Section 3, Algorithm 1; Section 5.6).

The operators' exact forms are readings (the paper names them only), so they
are pinned by properties that follow from those readings independently of the
code: decode endpoints and resolution (Eq. decode), the selection law of a
binary tournament, the single-cut structure of one-point crossover, per-bit
mutation frequencies, elitism, the restart rule, convergence on a quadratic and
an exhaustive search over one 16-bit parameter.
"""
import math

import numpy as np
import pytest

import genesis_inputs as gi

M = 9


def test_decode_endpoints_and_resolution(orc):
    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI
    g0 = orc.ga_decode(np.zeros(M, np.uint16), lo, hi)
    g1 = orc.ga_decode(np.full(M, 65535, np.uint16), lo, hi)
    assert np.array_equal(g0, lo) and np.array_equal(g1, hi)
    g = np.full(M, 1, np.uint16)
    d = orc.ga_decode(g, lo, hi) - lo
    assert np.allclose(d, (hi - lo) / (2 ** 16 - 1), rtol=1e-10, atol=0)
    # MSB alone gives the upper half start: 32768 / 65535 of the range
    g = np.full(M, 0x8000, np.uint16)
    assert np.allclose(orc.ga_decode(g, lo, hi), lo + (hi - lo) * 32768 / 65535, rtol=1e-15)


def _pop(npop, seed):
    r = np.random.default_rng(seed)
    return r.integers(0, 65536, (npop, M)).astype(np.uint16)


def _find_parent(child, parents):
    idx = np.nonzero((parents == child).all(1))[0]
    return idx


def test_tournament_selection_law(orc):
    """P(rank r wins) = 2 (N-1-r) / (N (N-1)) for a binary tournament of two
    distinct entrants, rank 0 = best."""
    npop = 32
    genes = np.arange(npop * M, dtype=np.uint16).reshape(npop, M)   # all distinct
    f = np.linspace(1.0, 2.0, npop)           # rank r = index r
    cfg = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    counts = np.zeros(npop)
    ngen = 1500
    for t in range(1, ngen + 1):
        child, e = orc.ga_breed(genes, f, 77, t, cfg)
        assert e == 0 and np.array_equal(child[0], genes[0])
        for k in range(1, npop):
            counts[_find_parent(child[k], genes)[0]] += 1
    n = ngen * (npop - 1)
    p = np.array([2 * (npop - 1 - r) / (npop * (npop - 1)) for r in range(npop)])
    exp = n * p
    m = exp > 0
    chi = ((counts[m] - exp[m]) ** 2 / exp[m]).sum()
    assert counts[-1] == 0                   # the worst never wins
    assert chi < (m.sum() - 1) + 5 * math.sqrt(2 * (m.sum() - 1)), chi


def test_tournament_ties_go_to_lower_index(orc):
    npop = 16
    genes = np.arange(npop * M, dtype=np.uint16).reshape(npop, M)
    f = np.ones(npop)
    f[5] = np.nan       # NaN counts as +inf: never wins against a finite value
    cfg = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    wins5 = 0
    for t in range(1, 400):
        child, _ = orc.ga_breed(genes, f, 3, t, cfg)
        for k in range(1, npop):
            wins5 += int(_find_parent(child[k], genes)[0] == 5)
    # index 5 could only win if both entrants were 5, which cannot happen
    assert wins5 == 0


def _bits(g):
    """MSB-first bit string of a genotype row."""
    return np.unpackbits(g.astype(">u2").view(np.uint8))


def test_one_point_crossover_structure(orc):
    npop = 64
    genes = _pop(npop, 1)
    f = np.random.default_rng(2).random(npop)
    cfg0 = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    cfg1 = orc.ga_config(npop, 10, pc=1.0, pmut_lsb=0.0)
    cuts = []
    for t in range(1, 60):
        par, _ = orc.ga_breed(genes, f, 9, t, cfg0)    # tournament winners only
        ch, e = orc.ga_breed(genes, f, 9, t, cfg1)
        for q in range(1, npop // 2):
            A, B = _bits(par[2 * q]), _bits(par[2 * q + 1])
            a, b = _bits(ch[2 * q]), _bits(ch[2 * q + 1])
            diff = np.nonzero(A != B)[0]
            if len(diff) == 0:
                continue
            # one cut c: a = A[:c] + B[c:], b = B[:c] + A[c:]
            ok = [c for c in range(1, 16 * M) if
                  np.array_equal(a, np.concatenate([A[:c], B[c:]])) and
                  np.array_equal(b, np.concatenate([B[:c], A[c:]]))]
            assert ok, (t, q)
            cuts.append(ok[0])
        # slot 1 still holds the crossover partner of slot 0's tournament winner
    cuts = np.array(cuts)
    assert cuts.min() >= 1 and cuts.max() <= 16 * M - 1
    # roughly uniform over [1, 143]
    assert abs(cuts.mean() - 72) < 6


def test_crossover_rate(orc):
    npop = 64
    genes = _pop(npop, 3)
    f = np.random.default_rng(4).random(npop)
    cfg0 = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    cfg = orc.ga_config(npop, 10, pc=0.9, pmut_lsb=0.0)
    crossed = total = 0
    for t in range(1, 200):
        par, _ = orc.ga_breed(genes, f, 5, t, cfg0)
        ch, _ = orc.ga_breed(genes, f, 5, t, cfg)
        for q in range(1, npop // 2):
            if not np.array_equal(par[2 * q], par[2 * q + 1]):
                total += 1
                crossed += int(not np.array_equal(ch[2 * q], par[2 * q]))
    rate = crossed / total
    assert abs(rate - 0.9) < 4 * math.sqrt(0.09 / total)


def test_mutation_frequencies(orc):
    npop = 64
    genes = _pop(npop, 6)
    f = np.random.default_rng(7).random(npop)
    plsb, ratio = 0.05, 0.7
    cfg0 = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    cfg = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=plsb, pmut_ratio=ratio)
    flips = np.zeros(16)
    n = 0
    for t in range(1, 2001):
        par, _ = orc.ga_breed(genes, f, 11, t, cfg0)
        ch, _ = orc.ga_breed(genes, f, 11, t, cfg)
        x = (par[1:] ^ ch[1:]).astype(np.uint32)
        for b in range(16):
            flips[b] += ((x >> (15 - b)) & 1).sum()
        n += (npop - 1) * M
    for b in range(16):
        p = plsb * ratio ** (15 - b)
        sd = math.sqrt(n * p * (1 - p))
        assert abs(flips[b] - n * p) < 5 * sd + 1, (b, flips[b], n * p)


def test_mutation_flips_are_independent(orc):
    """The jump sampler draws the flips of a word jointly; they must still be
    independent Bernoulli(q_b): the number of flips per word follows the
    Poisson-binomial law of the q_b, and flips of two bits are uncorrelated."""
    npop = 64
    genes = _pop(npop, 6)
    f = np.random.default_rng(7).random(npop)
    plsb, ratio = 0.05, 0.7
    cfg0 = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=0.0)
    cfg = orc.ga_config(npop, 10, pc=0.0, pmut_lsb=plsb, pmut_ratio=ratio)
    xs = []
    for t in range(1, 1201):
        par, _ = orc.ga_breed(genes, f, 13, t, cfg0)
        ch, _ = orc.ga_breed(genes, f, 13, t, cfg)
        xs.append((par[1:] ^ ch[1:]).astype(np.uint32).reshape(-1))
    x = np.concatenate(xs)
    n = len(x)
    bits = ((x[:, None] >> (15 - np.arange(16))) & 1).astype(np.float64)
    q = plsb * ratio ** (15 - np.arange(16))
    law = np.array([1.0])
    for qb in q:
        law = np.convolve(law, [1 - qb, qb])
    got = np.bincount(bits.sum(1).astype(int), minlength=17) / n
    for k in range(3):
        assert abs(got[k] - law[k]) < 5 * math.sqrt(law[k] * (1 - law[k]) / n) + 1e-6, (k, got[k], law[k])
    # pairs among the likeliest bits: P(both) = q_a q_b
    for a, b in [(15, 14), (15, 12), (13, 9), (14, 8)]:
        both = (bits[:, a] * bits[:, b]).mean()
        pab = q[a] * q[b]
        assert abs(both - pab) < 5 * math.sqrt(pab / n) + 2e-6, (a, b, both, pab)


def test_restart_replaces_worst_half_in_rank_order(orc):
    npop = 16
    genes = _pop(npop, 8)
    f = np.random.default_rng(9).permutation(npop).astype(float)
    f[3] = f[7]              # a tie: the lower index ranks first
    new, rep = orc.ga_restart(genes, f, 1000)
    order = sorted(range(npop), key=lambda i: (f[i], i))
    worst = order[npop // 2:]
    assert list(rep) == worst
    for r, i in enumerate(worst):
        expect = [orc.sobol_u32(1000 + r, d) >> 16 for d in range(M)]
        assert list(new[i]) == expect
    for i in order[:npop // 2]:
        assert np.array_equal(new[i], genes[i])


def _quad_fitness(orc, genes, lo, hi, target):
    p = orc.ga_decode(genes, lo, hi)
    return (((p - target) / (hi - lo)) ** 2).sum(1)


def test_elitism_and_convergence_on_quadratic(orc):
    """On a separable quadratic every stream's best never increases (elitism)
    and falls by a large factor in 200 generations.  The factor reached by one
    stream spreads over two orders of magnitude, so the bar is on the median of
    six independent streams (pixel ids) and on the worst of them."""
    npop, ngen = 128, 200
    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI
    target = lo + (hi - lo) * np.random.default_rng(10).random(M)
    cfg = orc.ga_config(npop, ngen)
    ratios = []
    for pid in range(6):
        genes = np.array([[orc.sobol_u32(k + 1, d) >> 16 for d in range(M)] for k in range(npop)],
                         dtype=np.uint16)
        f = _quad_fitness(orc, genes, lo, hi, target)
        best = [f.min()]
        for t in range(1, ngen + 1):
            genes, _ = orc.ga_breed(genes, f, pid, t, cfg)
            f = _quad_fitness(orc, genes, lo, hi, target)
            best.append(f.min())
        assert all(b1 <= b0 for b0, b1 in zip(best, best[1:]))     # never increases
        ratios.append(best[-1] / best[0])
    assert np.median(ratios) < 1e-2 and max(ratios) < 0.1, ratios


def test_driver_matches_composed_operators(orc):
    """ga_invert = Sobol init + (breed, evaluate, restart) composed by hand."""
    spec = gi.one_line_spec(n_lambda=24)
    truth = gi.draw_truth(2, seed=30)
    obs = orc.synth(spec, truth)
    lo, hi = gi.PRIOR_LO, gi.PRIOR_HI
    npop, ngen = 16, 12
    cfg = orc.ga_config(npop, ngen, nsamp=4, seed=99)
    res = orc.ga_invert(spec, obs, lo, hi, cfg, pixel_id0=40, nthreads=1)
    for ip in range(2):
        w = orc.weights_invmax(obs[ip])

        def fit(g):
            p = orc.ga_decode(g, lo, hi)
            return np.array([orc.chi2(obs[ip], orc.synth(spec, pi)[0], w) for pi in p])

        genes = np.array([[orc.sobol_u32(k + 1, d) >> 16 for d in range(M)] for k in range(npop)],
                         dtype=np.uint16)
        f = fit(genes)
        nxt = npop + 1
        for t in range(1, ngen + 1):
            genes, e = orc.ga_breed(genes, f, 40 + ip, t, cfg)
            f = fit(genes)
            if t % 4 == 0 and t < ngen:
                genes, rep = orc.ga_restart(genes, f, nxt)
                f = fit(genes)
                nxt += npop // 2
        b = int(np.argmin(f))
        assert np.array_equal(res["genes"][ip], genes[b])
        assert res["chi2"][ip] == pytest.approx(f[b], rel=1e-14)


def test_exhaustive_single_parameter(orc):
    """With all but B fixed (lo = hi), the GA's answer can be no better than the
    exhaustive minimum over all 65536 genes, and a long run reaches it."""
    spec = gi.one_line_spec(n_lambda=32)
    truth = np.array([[1234.5, 50.0, 30.0, 0.5, 30.0, 0.2, 8.0, 0.3, 0.7]])
    obs = orc.synth(spec, truth)
    lo, hi = truth[0].copy(), truth[0].copy()
    lo[0], hi[0] = 0.0, 3000.0
    w = orc.weights_invmax(obs[0])
    allg = np.zeros((65536, M), np.uint16)
    allg[:, 0] = np.arange(65536)
    p = orc.ga_decode(allg, lo, hi)
    models = orc.synth(spec, p)
    c2 = np.array([orc.chi2(obs[0], models[i], w) for i in range(65536)])
    gmin = int(np.argmin(c2))
    cfg = orc.ga_config(32, 20, seed=5)
    res = orc.ga_invert(spec, obs, lo, hi, cfg, nthreads=1)
    assert res["chi2"][0] >= c2[gmin] * (1 - 1e-12)
    hits = 0
    for seed in range(8):
        cfg = orc.ga_config(128, 300, seed=seed)
        res = orc.ga_invert(spec, obs, lo, hi, cfg, nthreads=1)
        assert res["chi2"][0] >= c2[gmin] * (1 - 1e-12)
        assert abs(int(res["genes"][0][0]) - gmin) <= 16   # within the 4 LSBs
        hits += int(res["genes"][0][0]) == gmin
    assert hits >= 6
