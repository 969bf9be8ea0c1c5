"""Pins of the oracle's P-ERK tableaux: printed values, brute-force order
conditions over coloured rooted trees, textbook special cases."""
import json
import math
import os

import numpy as np
import pytest

from oracle import tableau as T

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tableaux.json")))


def test_tree_counts():
    # number of rooted trees with n vertices: 1, 1, 2, 4, 9
    assert [len(T.rooted_trees(n)) for n in range(1, 6)] == [1, 1, 2, 4, 9]
    assert sorted(T.tree_density(t) for t in T.rooted_trees(4)) == [4, 8, 12, 24]


def test_printed_p2_example():
    c, b, As = T.family(2, [6, 3])
    assert np.allclose(c, GOLD["p2_S6_c"], atol=1e-15)
    assert np.allclose(b, GOLD["p2_S6_b"])
    assert T.active_stages(6, 3) == GOLD["p2_S6_E3_active_stages"]
    A2 = As[1]
    for i in GOLD["p2_S6_E3_rows_K1_only"]:
        assert A2[i - 1, 0] == pytest.approx(c[i - 1], abs=1e-15)
        assert np.all(A2[i - 1, 1:] == 0)
    assert A2[5, 4] != 0 and A2[5, 0] + A2[5, 4] == pytest.approx(0.5, abs=1e-15)


def test_printed_p4_constants():
    c, b, As = T.family(4, [7, 5])
    S = 7
    assert c[S - 3] == pytest.approx(GOLD["p4_c_Sm2"], abs=1e-15)
    assert c[S - 2] == pytest.approx(GOLD["p4_c_Sm1"], abs=1e-15)
    assert c[S - 1] == pytest.approx(GOLD["p4_c_S"], abs=1e-15)
    for A in As:
        assert A[S - 3, S - 4] * c[S - 4] == pytest.approx(GOLD["p4_a_Sm2_Sm3_times_c_Sm3"], abs=1e-15)
        assert A[S - 2, S - 3] == pytest.approx(GOLD["p4_a_Sm1_Sm2"], abs=1e-15)
        assert A[S - 1, S - 2] == pytest.approx(GOLD["p4_a_S_Sm1"], abs=1e-15)
    assert b[S - 2] == GOLD["p4_b_Sm1"] and b[S - 1] == GOLD["p4_b_S"]


def test_printed_p3_weights():
    c, b, As = T.family(3, [8, 4])
    g = GOLD["p3_own_b"]
    assert b[0] == pytest.approx(g["b_1"]) and b[-2] == pytest.approx(g["b_Sm1"]) and b[-1] == pytest.approx(g["b_S"])
    assert c[-2] == GOLD["p3_own_c_Sm1"] and c[-1] == GOLD["p3_own_c_S"]


FAMILIES = [(2, [8, 4]), (2, [16, 12, 8, 4, 2]), (3, [12, 6, 3]), (3, [8, 4]), (3, [16, 12, 8, 5, 3]),
            (4, [16, 10, 7, 5]), (4, [8, 6, 5]), (2, [2]), (3, [3]), (4, [5])]


@pytest.mark.parametrize("p,E", FAMILIES)
def test_order_conditions(p, E):
    c, b, As = T.family(p, E)
    worst, cons = T.order_residuals(c, b, As, p)
    assert worst < 1e-14 and cons < 1e-15
    # the method is not of order p+1 in general (sanity: the check has teeth)
    if max(E) > 2:
        worst1, _ = T.order_residuals(c, b, As[:1], p + 1)
        assert worst1 > 1e-6
    # sparsity: at most two nonzeros per row (K_1 and K_{i-1})
    for A in As:
        for i in range(2, len(b)):
            assert np.count_nonzero(A[i, 1:i - 1]) == 0


def test_textbook_special_cases():
    c, b, (A,) = T.family(3, [3])      # SSPRK3 (Shu-Osher)
    assert np.allclose(c, [0, 1, 0.5]) and np.allclose(b, [1 / 6, 1 / 6, 2 / 3])
    assert np.allclose(A, [[0, 0, 0], [1, 0, 0], [0.25, 0.25, 0]])
    c, b, (A,) = T.family(2, [2])      # explicit midpoint
    assert np.allclose(c, [0, 0.5]) and np.allclose(b, [0, 1]) and np.allclose(A, [[0, 0], [0.5, 0]])


@pytest.mark.parametrize("E", [2, 3, 4, 6, 8, 12])
def test_p2_stability_polynomial_is_taylor(E):
    c, b, As = T.family(2, [max(E, 8), E])
    al = T.stability_coeffs(b, As[1])
    for j in range(E + 1):
        assert al[j] == pytest.approx(1.0 / math.factorial(j), rel=1e-13)
    assert np.all(np.abs(al[E + 1:]) < 1e-15)


def test_injected_mistake_is_caught():
    c, b, As = T.family(3, [8, 4])
    A = As[0].copy()
    A[-1, -2] += 1e-3
    A[-1, 0] -= 1e-3                    # keeps row sums, breaks order 3
    worst, cons = T.order_residuals(c, b, [A, As[1]], 3)
    assert worst > 1e-5 and cons < 1e-15
