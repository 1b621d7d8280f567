"""Pins of the oracle's velocity set and quadrature (Sec. III.A, D2Q37 figure caption)."""
import json
import math
import os

import numpy as np
import pytest

import oracle

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def gauss1d(a):
    """Raw moment E[x^a] of the unit normal: (a-1)!! for even a, 0 for odd a."""
    return 0.0 if a % 2 else float(np.prod(np.arange(a - 1, 0, -2))) if a else 1.0


def test_velocity_set_structure():
    c, opp = oracle.velocities()
    assert len(c) == GOLD["n_velocities"]["value"]
    assert len({tuple(v) for v in c}) == 37
    assert tuple(c[0]) == (0, 0)
    c2 = (c ** 2).sum(1)
    assert list(c2) == sorted(c2)                        # shells in increasing |c|^2
    assert sorted(set(c2.tolist())) == [0, 1, 2, 4, 5, 8, 9, 10]
    assert np.abs(c).max() == GOLD["halo_x"]["value"]    # x reach = the paper's 3 halo columns
    for l in range(37):
        assert tuple(c[opp[l]]) == (-c[l][0], -c[l][1])
    # angles strictly increase within a shell
    ang = np.mod(np.arctan2(c[:, 1], c[:, 0]), 2 * np.pi)
    for s in set(c2.tolist()):
        idx = np.where(c2 == s)[0]
        assert np.all(np.diff(ang[idx]) > 0)


def test_lattice_constant_matches_paper():
    _, r = oracle.weights()
    g = GOLD["r_lattice"]
    assert abs(r - g["value"]) < 10.0 ** (-g["printed_digits"])


def test_weights_positive_and_normalised():
    w, _ = oracle.weights()
    assert np.all(w > 0)
    assert abs(w.sum() - 1.0) < 1e-15
    c, opp = oracle.velocities()
    c2 = (c ** 2).sum(1)
    for s in set(c2.tolist()):                           # one weight per shell
        assert np.ptp(w[c2 == s]) == 0.0


@pytest.mark.parametrize("deg", range(0, 10))
def test_gaussian_moments_exact_to_degree_9(deg):
    c, _ = oracle.velocities()
    w, r = oracle.weights()
    xi = r * c
    for a in range(deg + 1):
        b = deg - a
        lhs = np.sum(w * xi[:, 0] ** a * xi[:, 1] ** b)
        rhs = gauss1d(a) * gauss1d(b)
        assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(rhs)), (a, b, lhs, rhs)


def test_degree_10_is_not_exact():
    """The quadrature must stop at degree 9 (non-vacuous check of the moment test)."""
    c, _ = oracle.velocities()
    w, r = oracle.weights()
    xi = r * c
    lhs = np.sum(w * xi[:, 0] ** 10)
    assert abs(lhs - gauss1d(10)) > 1e-3
