"""Pins of GENO's path function chi in its intermediate regime (paper Sec. 3.2,
Eqs. GENO-nonlinear and GENO-IS-linear; App. D).

The other GENO pins reach chi only at its limits (chi = 1 on equal smoothness
indicators, chi -> 0 across a step).  Here chi is taken strictly between 0.01
and 0.99, where the exponent r, the place of eps and the roles of alpha^H and
alpha^L all change the result:

* the ultimate indicator alpha is given for hand-chosen indicator triples as an
  exact fraction worked out by hand (derivations in `HAND`), and chi follows
  from it through the tanh ratio of Eq. GENO-nonlinear;
* the whole value reconstruction is compared with App. D's formulation, which
  normalises the two alpha terms as a vector and writes IS^tau as half of
  |IS_2 + IS_3 - 2 IS_1|, restated here from what it computes;
* each plausible mistake (wrong r, eps outside the ratio or on both sides of
  it, the other variant's eps, alpha^H and alpha^L swapped, the wrong
  sub-stencil taken as the reference of IS^tau) is run through a small model of
  the formula and shown to miss at least one hand value by far more than the
  tolerance, so each one would fail these tests if the oracle made it.

Variant 0 = Sec. 3.2 text (r = 2, eps = 1e-12), variant 1 = App. D (r = 3,
eps = 1e-15); both use C = 20.
"""
import math
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle

C = 20.0

# (variant, IS_1, IS_2, IS_3, alpha as an exact fraction).  Derivations, with
# IS^tau = |(IS_2 + IS_3)/2 - IS_1|, IS^H = max IS_k, IS^L = min IS_k:
#  (1, 9, 5):   IS^tau = 6, IS^H = 9, IS^L = 1.
#       r = 3: aH = 1 + (2/3)^3 = 35/27, aL = 1 + 216 = 217,
#              alpha = 2 (35/27) / (35/27 + 217) = 70/5894 = 35/2947.
#       r = 2: aH = 1 + 4/9 = 13/9, aL = 37, alpha = 26/346 = 13/173.
#  (4, 1/2, 3/2): IS^tau = |1 - 4| = 3, IS^H = 4, IS^L = 1/2.
#       r = 3: aH = 1 + 27/64 = 91/64, aL = 1 + 6^3 = 217, alpha = 182/13979.
#       r = 2: aH = 25/16, aL = 37, alpha = 50/617.
#  (1, 5, 3):   IS^tau = 3, IS^H = 5, IS^L = 1.
#       r = 3: aH = 1 + 27/125 = 152/125, aL = 28, alpha = 304/3652 = 76/913.
#  eps-scale triples (eps enters at the size of the indicators):
#  (1, 41, 1) x 1e-15, r = 3, eps = 1e-15: IS^tau = 20e-15, IS^H + eps = 42e-15,
#       IS^L + eps = 2e-15: aH = 1 + (10/21)^3 = 10261/9261, aL = 1 + 10^3 = 1001,
#       alpha = 20522/9280522 = 10261/4640261.
#  (1, 41, 1) x 1e-12, r = 2, eps = 1e-12: aH = 1 + (10/21)^2 = 541/441, aL = 101,
#       alpha = 1082/45082 = 541/22541.
HAND = [
    (1, (1.0, 9.0, 5.0), Fr(35, 2947)),
    (0, (1.0, 9.0, 5.0), Fr(13, 173)),
    (1, (4.0, 0.5, 1.5), Fr(182, 13979)),
    (0, (4.0, 0.5, 1.5), Fr(50, 617)),
    (1, (1.0, 5.0, 3.0), Fr(76, 913)),
    (1, (1e-15, 41e-15, 1e-15), Fr(10261, 4640261)),
    (0, (1e-12, 41e-12, 1e-12), Fr(541, 22541)),
]


def chi_of_alpha(alpha):
    return math.tanh(C * float(alpha)) / math.tanh(C)


def _blend(variant, node, IS, seed=0):
    rng = np.random.default_rng(seed)
    q, qx = rng.normal(size=3), rng.normal(size=3)
    PH, PHx = float(rng.normal()), float(rng.normal())
    return oracle.geno_blend(variant, node, np.array(IS), q, qx, PH, PHx), q, qx, PH, PHx


def test_hand_triples_are_in_the_intermediate_regime():
    for _, _, alpha in HAND:
        assert 0.01 < chi_of_alpha(alpha) < 0.99


@pytest.mark.parametrize("node", [0, 1])
@pytest.mark.parametrize("variant,IS,alpha", HAND)
def test_path_function_matches_hand_values(variant, IS, alpha, node):
    """chi of the oracle = tanh(C alpha)/tanh(C) with alpha worked out by hand;
    the path function is the same for interface and node sub-stencil sets."""
    (val, der, chi), *_ = _blend(variant, node, IS)
    assert chi == pytest.approx(chi_of_alpha(alpha), rel=1e-12, abs=0)


def _appendix_d_value(IS, p, d, r, eps, eps_w):
    """App. D's value reconstruction, restated from what it computes: the two
    alpha terms are scaled together so that the first one becomes alpha; the
    low-order part takes the normalised d_k / (IS_k + eps_w)^2 weights; the
    result moves from it to the high-order value p[3] by the path function."""
    IS = np.asarray(IS, dtype=float)
    spread = abs(IS[1] + IS[2] - 2.0 * IS[0]) / 2.0
    pair = np.array([1.0 + (spread / (IS.max() + eps)) ** r, 1.0 + (spread / (IS.min() + eps)) ** r])
    pair = 2.0 * pair / pair.sum()
    path = math.tanh(C * pair[0]) / math.tanh(C)
    weights = np.asarray(d, dtype=float) / (IS + eps_w) ** 2
    weights = weights / weights.sum()
    return (1.0 - path) * float(np.dot(weights, p[:3])) + path * p[3], path


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("IS", [(1.0, 9.0, 5.0), (4.0, 0.5, 1.5), (1.0, 5.0, 3.0), (1e-15, 41e-15, 1e-15),
                                (2.0, 7.0, 1.0), (0.3, 0.1, 2.2)])
def test_variant1_value_equals_appendix_d(IS, seed):
    """Variant 1 at an interface (d = 8 on the central sub-stencil) reproduces
    App. D's reconstructed value for the same indicators and candidates; the
    derivative takes the same weights (reading: App. D is value-only)."""
    (val, der, chi), q, qx, PH, PHx = _blend(1, 0, IS, seed)
    ref, path = _appendix_d_value(IS, np.r_[q, PH], (1.0, 8.0, 1.0), 3, 1e-15, 1e-6)
    assert chi == pytest.approx(path, rel=1e-13)
    assert val == pytest.approx(ref, rel=1e-13, abs=1e-14)
    dref, _ = _appendix_d_value(IS, np.r_[qx, PHx], (1.0, 8.0, 1.0), 3, 1e-15, 1e-6)
    assert der == pytest.approx(dref, rel=1e-13, abs=1e-14)


@pytest.mark.parametrize("variant,node,d", [(0, 0, (8.0, 1.0, 1.0)), (0, 1, (8.0, 1.0, 1.0)),
                                            (1, 1, (8.0, 1.0, 1.0))])
def test_other_sets_value_in_intermediate_regime(variant, node, d):
    """The text's constants (r = 2, eps = 1e-12) and the node sets (d = 8 on the
    central node sub-stencil, numbered first) with chi strictly inside (0, 1)."""
    r, eps = (2, 1e-12) if variant == 0 else (3, 1e-15)
    for IS in [(1.0, 9.0, 5.0), (4.0, 0.5, 1.5), (1e-12, 41e-12, 1e-12)]:
        (val, der, chi), q, qx, PH, PHx = _blend(variant, node, IS, 7)
        ref, path = _appendix_d_value(IS, np.r_[q, PH], d, r, eps, 1e-6)
        assert 0.01 < path < 0.99 or IS[0] == 1e-12 and variant == 1
        assert val == pytest.approx(ref, rel=1e-13, abs=1e-14)


def _model_alpha(IS, r, eps, mutant=None):
    """alpha of Eq. GENO-IS-linear in exact arithmetic, with one named mistake
    switched in; the unmutated model reproduces the hand fractions."""
    a, b, c = (Fr(x) for x in IS)
    e = Fr(eps)
    ref = b if mutant == "tau_wrong_reference" else a
    others = (a + c) if mutant == "tau_wrong_reference" else (b + c)
    tau = abs(others / 2 - ref)
    hi, lo = max(a, b, c), min(a, b, c)
    if mutant == "eps_outside":
        aH, aL = 1 + (tau / hi) ** r + e, 1 + (tau / lo) ** r + e
    elif mutant == "eps_both_sides":
        aH, aL = 1 + ((tau + e) / (hi + e)) ** r, 1 + ((tau + e) / (lo + e)) ** r
    else:
        aH, aL = 1 + (tau / (hi + e)) ** r, 1 + (tau / (lo + e)) ** r
    if mutant == "swapped_alpha":
        aH, aL = aL, aH
    return 2 * aH / (aH + aL)


def _variant_consts(variant):
    return (2, 1e-12) if variant == 0 else (3, 1e-15)


def test_model_reproduces_hand_values():
    for variant, IS, alpha in HAND:
        r, eps = _variant_consts(variant)
        got = _model_alpha(IS, r, eps)
        # the hand fractions drop eps where the indicators are O(1): 1e-12 relative at most
        assert float(abs(got - alpha) / alpha) < 1e-10


def _misses(mutant, r_of=None, eps_of=None):
    worst = 0.0
    for variant, IS, alpha in HAND:
        r, eps = _variant_consts(variant)
        r = r_of(variant) if r_of else r
        eps = eps_of(variant) if eps_of else eps
        got = chi_of_alpha(_model_alpha(IS, r, eps, mutant))
        worst = max(worst, abs(got - chi_of_alpha(alpha)))
    return worst


def test_pins_reject_wrong_exponent():
    assert _misses(None, r_of=lambda v: 3 if v == 0 else 2) > 1e-2


def test_pins_reject_eps_outside_the_ratio():
    assert _misses("eps_outside") > 1e-2


def test_pins_reject_eps_on_both_sides_of_the_ratio():
    assert _misses("eps_both_sides") > 1e-2


def test_pins_reject_the_other_variants_eps():
    assert _misses(None, eps_of=lambda v: 1e-15 if v == 0 else 1e-12) > 1e-2


def test_pins_reject_swapped_alpha_h_and_alpha_l():
    assert _misses("swapped_alpha") > 1e-2


def test_pins_reject_wrong_tau_reference():
    assert _misses("tau_wrong_reference") > 1e-2
