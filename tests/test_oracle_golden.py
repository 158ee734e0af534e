"""Pins of the oracle against values derived by hand from Eq. 1 (tests/golden/*.txt, each
file gives its derivation): the scalar CGGM with both penalties active, and two outputs
with Theta held at zero by its penalty, where Lambda is the 2 x 2 graphical-lasso closed
form.  Both fixtures have exact rational parameters."""
import math
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_fixture(name):
    vals = {}
    for line in open(os.path.join(GOLDEN, name)):
        line = line.split("#", 1)[0].strip()
        if line:
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def test_fixture_values_are_the_stated_fractions():
    g = read_fixture("scalar_cggm.txt")
    assert g["Lambda"] == 8 / 15 and g["Theta"] == -2 / 15
    assert abs(g["f"] - (1 + math.log(15 / 8))) < 1e-15
    h = read_fixture("glasso_2x2.txt")
    assert (h["Lambda_11"], h["Lambda_12"], h["Lambda_22"]) == (42 / 43, -8 / 43, 22 / 43)
    assert abs(h["f"] - (2 + math.log(2.15))) < 1e-15


def test_scalar_cggm_closed_form():
    g = read_fixture("scalar_cggm.txt")
    X = np.array([[2.0], [0.0]])
    Y = np.array([[1.0], [math.sqrt(2.0)]])
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    assert np.allclose([Sxx[0, 0], Sxy[0, 0], Syy[0, 0]], [g["Sxx"], g["Sxy"], g["Syy"]],
                       rtol=0, atol=1e-15)
    L = np.array([[g["Lambda"]]])
    T = np.array([[g["Theta"]]])
    f = oracle.objective(L, T, Sxx, Sxy, Syy, g["lam_Lambda"], g["lam_Theta"])
    assert abs(f - g["f"]) <= 1e-14 * abs(g["f"])
    r = oracle.solve(X, Y, g["lam_Lambda"], g["lam_Theta"], tol=1e-12, max_iter=5000)
    assert abs(r.Lambda[0, 0] - g["Lambda"]) <= 1e-8 * g["Lambda"]
    assert abs(r.Theta[0, 0] - g["Theta"]) <= 1e-8 * abs(g["Theta"])
    assert abs(r.f - g["f"]) <= 1e-13 * abs(g["f"])


def test_glasso_2x2_closed_form():
    h = read_fixture("glasso_2x2.txt")
    X = np.array([[0.0], [1.0]])
    Y = np.array([[math.sqrt(2.0), 1 / math.sqrt(2.0)], [0.0, math.sqrt(3.5)]])
    Sxx, Sxy, Syy = oracle.covariances(X, Y)
    assert np.allclose(Syy, [[h["Syy_11"], h["Syy_12"]], [h["Syy_12"], h["Syy_22"]]],
                       rtol=0, atol=1e-15)
    assert np.allclose(Sxy, [[h["Sxy_1"], h["Sxy_2"]]], rtol=0, atol=1e-15)
    L = np.array([[h["Lambda_11"], h["Lambda_12"]], [h["Lambda_12"], h["Lambda_22"]]])
    T = np.zeros((1, 2))
    f = oracle.objective(L, T, Sxx, Sxy, Syy, h["lam_Lambda"], h["lam_Theta"])
    assert abs(f - h["f"]) <= 1e-14 * abs(h["f"])
    # close to the optimum the Armijo test meets the rounding of f and progress stops
    # short of a 1e-12 ratio; the parameters are then accurate to about 1e-8
    r = oracle.solve(X, Y, h["lam_Lambda"], h["lam_Theta"], tol=1e-12, max_iter=200)
    assert np.all(r.Theta == 0.0)
    assert np.max(np.abs(r.Lambda - L)) <= 1e-8
    assert abs(r.f - h["f"]) <= 1e-13 * abs(h["f"])
