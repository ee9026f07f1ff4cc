"""Pins for the oracle's cost and selection (Sec. IV-A, cost functions and
selection mechanism): hand-computed costs on tiny trajectories, ties and the
alpha-hysteresis rule."""

import json
import math
import os

import numpy as np

import oracle
from synth.workloads import PhysicsParams

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_golden_costs_and_selection():
    g = json.load(open(os.path.join(GOLD, "cost_tiny.json")))
    prm = PhysicsParams(goal=tuple(g["goal"]), w_path=g["w_path"], w_goal=g["w_goal"],
                        w_clear=g["w_clear"])
    ro = {"path_len": np.array(g["path_len"]), "p_final": np.array(g["p_final"]),
          "clear_pen": np.array(g["clear_pen"])}
    c = oracle.costs(ro, prm)
    assert np.allclose(c, g["costs"], rtol=1e-14)
    assert oracle.select(c) == g["best"]
    for h in g["hysteresis"]:
        assert oracle.select(c, h["prev_best_cost"], h["alpha"]) == h["best"]


def test_ties_pick_lowest_index():
    c = np.array([3.0, 1.0, 2.0, 1.0, 1.0])
    assert oracle.select(c) == 1
    assert oracle.select(c, prev_best_cost=5.0, alpha=0.5) == 1
    assert oracle.select(np.array([math.inf, 2.0])) == 1
