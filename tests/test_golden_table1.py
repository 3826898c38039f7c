"""Pins of the oracle's Zeeman patterns against the paper's Table 1.

The fixture tests/golden/table1_fe816.txt holds the table as printed.  From
each transition's term symbols (2S+1, L, J) the LS-coupling Lande factors
g = 1 + [J(J+1) + S(S+1) - L(L+1)] / [2J(J+1)] are formed here, the oracle
builds the full pattern, and its sigma-group first moment (the effective
Lande factor) must equal the printed g_eff to the printed three decimals; the
6301.5 pattern must have four components in each group (Section 6)."""
import os
import re

import numpy as np
import pytest

import genesis_inputs as gi

HERE = os.path.dirname(os.path.abspath(__file__))
L_OF = {"S": 0, "P": 1, "D": 2, "F": 3}


def _rows():
    rows = []
    for line in open(os.path.join(HERE, "golden", "table1_fe816.txt")):
        if line.startswith("#") or not line.strip():
            continue
        lam, trans, geff, chi, loggf = line.split()
        lo, up = trans.split("--")
        rows.append((float(lam), lo, up, float(geff), float(chi), float(loggf)))
    return rows


def _term(sym):
    m = re.fullmatch(r"(\d)([SPDF])(\d)", sym)
    mult, L, J = int(m.group(1)), L_OF[m.group(2)], int(m.group(3))
    S = (mult - 1) / 2.0
    g = 0.0 if J == 0 else 1.0 + (J * (J + 1) + S * (S + 1) - L * (L + 1)) / (2.0 * J * (J + 1))
    return J, g


@pytest.mark.parametrize("row", _rows(), ids=lambda r: str(r[0]))
def test_pattern_reproduces_printed_g_eff(orc, row):
    lam, lo, up, geff, _, _ = row
    jl, gl = _term(lo)
    ju, gu = _term(up)
    groups = orc.zeeman_components(jl, gl, ju, gu)
    sh, st = groups[2]   # sigma_r: strength-normalised shifts in Larmor units
    assert abs(np.sum(st) - 1.0) < 1e-12
    assert round(float(np.sum(sh * st)), 3) == geff
    # the blue group mirrors the red one
    shb, stb = groups[0]
    assert abs(np.sum(shb * stb) + np.sum(sh * st)) < 1e-12


def test_fe6301_has_four_components_per_group(orc):
    rows = {r[0]: r for r in _rows()}
    _, lo, up, _, _, _ = rows[6301.5091]
    jl, gl = _term(lo)
    ju, gu = _term(up)
    groups = orc.zeeman_components(jl, gl, ju, gu)
    assert [len(s) for s, _ in groups] == [4, 4, 4]
    _, lo, up, _, _, _ = rows[6302.5017]
    jl, gl = _term(lo)
    ju, gu = _term(up)
    assert [len(s) for s, _ in orc.zeeman_components(jl, gl, ju, gu)] == [1, 1, 1]


def test_inputs_use_the_printed_table():
    """The input generator's line constants are Table 1's numbers."""
    rows = {r[0]: r for r in _rows()}
    for const in (gi.FE6301, gi.FE6302):
        lam, _, _, geff, chi, loggf = rows[const[0]]
        assert (const[1], const[2], const[3]) == (geff, chi, loggf)


def test_full_pattern_input_uses_the_printed_terms():
    """The full-pattern input line of 6301.5 carries the levels of Table 1's
    printed transition (J and the LS Lande factors formed from the term
    symbols above), its printed g_eff and wavelength."""
    rows = {r[0]: r for r in _rows()}
    lam, lo, up, geff, _, _ = rows[6301.5091]
    jl, gl = _term(lo)
    ju, gu = _term(up)
    line = gi.two_line_pattern_spec().lines[0]
    assert line[0] == lam and line[1] == geff and line[2] == gi.eta_ratio_6301()
    assert line[3] == jl and line[5] == ju
    assert abs(line[4] - gl) < 1e-15 and abs(line[6] - gu) < 1e-15
