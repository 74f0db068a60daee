"""Pins for the oracle on general constraint structures, against closed forms the mathematics
fixes (Section 5.5's SDPLIB theta and gpp families, Section 2.3's sensor network localisation):

  * Lovasz theta: theta(C_5) = sqrt 5, theta(C_n) = n cos(pi/n) / (1 + cos(pi/n)) for odd n,
    theta(Petersen) = 4, theta(K_n) = 1, theta(empty graph) = n.  The trace constraint has n
    entries, so these exercise multi-entry constraints.
  * Minimum bisection relaxation min <L/4, X>, X_ii = 1, <e e^T, X> = 0: n^2/4 on K_n (n even)
    and n (1 - cos(2 pi / n)) / 2 on the cycle C_n (n even): X = the cosine matrix of the
    lambda_2 eigenspace attains lambda_2 n / 4 and <L, X> >= lambda_2 tr X whenever X e = 0.
    The all-ones constraint is a rank-one term with a length-n vector.
  * Sensor network localisation with exact distances on a rigid instance: Z = [I X; X^T X^T X]
    with X the true positions is feasible, and the solve recovers X.
"""
import math

import numpy as np
import pytest

from oracle import SDP, Params, solve
from paper_2403_09133_gb300 import instances as I


def petersen_edges():
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    return np.array([tuple(sorted(e)) for e in outer + spokes + inner])


THETA = {
    "C5": (lambda: I.lovasz_theta(5, I.cycle_edges(5)), math.sqrt(5.0)),
    "C7": (lambda: I.lovasz_theta(7, I.cycle_edges(7)),
           7 * math.cos(math.pi / 7) / (1 + math.cos(math.pi / 7))),
    "Petersen": (lambda: I.lovasz_theta(10, petersen_edges()), 4.0),
    "K6": (lambda: I.lovasz_theta(6, I.complete_edges(6)), 1.0),
    "empty7": (lambda: I.lovasz_theta(7, np.zeros((0, 2), dtype=np.int64)), 7.0),
}


@pytest.mark.parametrize("case", sorted(THETA))
def test_lovasz_theta_closed_forms(case):
    make, theta = THETA[case]
    sdp = SDP.from_instance(make())
    res = solve(sdp, Params(tol=1e-8))
    assert res["converged"]
    assert abs(-res["objective"] - theta) <= 1e-7 * theta
    assert res["r_P"] <= 1e-8 and res["r_D"] <= 1e-8


@pytest.mark.parametrize("case", ["C12", "K8"])
def test_bisection_closed_forms(case):
    if case == "C12":
        n = 12
        inst, want = I.graph_bisection(n, I.cycle_edges(n), np.ones(n)), n * (1 - math.cos(2 * math.pi / n)) / 2
    else:
        n = 8
        e = I.complete_edges(n)
        inst, want = I.graph_bisection(n, e, np.ones(len(e))), n * n / 4
    sdp = SDP.from_instance(inst)
    res = solve(sdp, Params(tol=1e-8))
    assert res["converged"]
    assert abs(res["objective"] - want) <= 1e-7 * want
    Uh = res["U_hat"]
    assert abs(float(np.sum(Uh.sum(axis=0) ** 2))) <= 1e-7 * n      # <e e^T, X> = ||U^T e||^2


def test_sensor_network_recovers_positions():
    inst = I.sensor_network(30, 4, 2, 0.6, seed=1)
    sdp = SDP.from_instance(inst)
    res = solve(sdp, Params())
    assert res["converged"] and res["objective"] == 0.0
    Z = res["U_hat"] @ res["U_hat"].T
    np.testing.assert_allclose(Z[:2, :2], np.eye(2), atol=1e-5)
    assert np.abs(Z[:2, 2:] - inst.mc_P).max() <= 1e-5
