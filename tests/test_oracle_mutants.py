"""Planted mistakes: each pin of the oracle fails when the part it pins is
wrong.

Every case below compiles a copy of the oracle with a one-token change (a
sign, an index, a comparison, an operand; ``tests/mutants.py``) and runs the
pin that is meant to catch it on that copy, on the CPU.  The pin must fail.
A pin that passes on the planted mistake would not protect the GPU parity
claims that rest on it.
"""
from __future__ import annotations

import pytest

import test_oracle_multid as MD
import test_oracle_pins as P


def _passes(test_fn):
    """Whether a pin test function of the suite passes (an arithmetic error
    raised on the mutated oracle counts as a failure)."""
    try:
        test_fn()
    except (AssertionError, FloatingPointError, ZeroDivisionError, ValueError):
        return False
    return True


def _in_mutant(subs, test_fn):
    from mutants import mutant
    with mutant(subs):
        return _passes(test_fn)


HLL_FAN = "f[q] = (sr * fl[q] - sl * fr[q] + sl * sr * (ur[q] - ul[q])) / (sr - sl);"
UPWIND = "  if (mflux > 0.0) return lo;\n  if (mflux < 0.0) return hi;"
DEGEN = "      vs = v; ws = ww; bys = by; bzs = bz;"
EDGE = "edge = avg + 0.25 * (db_minus - db_plus) + 0.25 * (da_minus - da_plus);"

# name: (substitutions, pin that must fail)
MUTANTS = {
    # HLL: the sign of the fan term S_L S_R (U_R - U_L), and the term dropped
    "hll_fan_sign": ([(HLL_FAN, HLL_FAN.replace("+ sl * sr", "- sl * sr"))],
                     lambda s: MD.check_hll_contact(subs=s)[0]),
    "hll_fan_operand": ([(HLL_FAN, HLL_FAN.replace("(ur[q] - ul[q])", "(ur[q] - ur[q])"))],
                        lambda s: MD.check_hll_contact(subs=s)[0]),
    # the Gardiner-Stone upwind side: swapped, and one comparison flipped
    "upwind_swapped": ([(UPWIND, "  if (mflux > 0.0) return hi;\n  if (mflux < 0.0) return lo;")],
                       lambda s: MD.check_field_loop(emfs=(0,), subs=s)[0]),
    "upwind_comparison": ([(UPWIND, UPWIND.replace("mflux > 0.0", "mflux < 0.0"))],
                          lambda s: MD.check_field_loop(emfs=(0,), subs=s)[0]),
    # which face's mass flux orients the average: invisible to the uniform
    # flow of the field loop (every mass flux has one sign), caught by the
    # point symmetry of Orszag-Tang
    "upwind_mass_flux_index": ([("double ma_p = M[a][fidx(&g, P[0], P[1], P[2])];",
                                 "double ma_p = M[a][fidx(&g, Pbm[0], Pbm[1], Pbm[2])];")],
                               lambda s: _in_mutant(s, P.test_orszag_tang_point_symmetry)),
    # HLLD's degenerate star state: the kept velocity, and the test itself
    "degenerate_velocity": ([(DEGEN, DEGEN.replace("vs = v;", "vs = u;"))],
                            lambda s: MD.check_hlld_degenerate(subs=s)[0]),
    "degenerate_comparison": ([("if (fabs(den) <= eps * scale)", "if (fabs(den) >= eps * scale)")],
                              lambda s: MD.check_hlld_degenerate(subs=s)[0]),
    # edge EMF assembly: a sign in the upwind correction, a face term
    # repeated in the 4-face mean; oblique waves see both
    "edge_correction_sign": ([(EDGE, EDGE.replace("(db_minus - db_plus)", "(db_minus + db_plus)"))],
                             lambda s: MD.check_oblique(emfs=(0,), waves=("fast",), subs=s)[0]),
    "edge_mean_operand": ([("double avg = 0.25 * (fa_m + fa_p + fb_m + fb_p);",
                            "double avg = 0.25 * (fa_m + fa_m + fb_m + fb_p);")],
                          lambda s: MD.check_oblique(emfs=(1,), waves=("fast",), subs=s)[0]),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_its_pin(name):
    subs, pin = MUTANTS[name]
    assert not pin(subs), f"the pin of {name} passes on the mutated oracle"
