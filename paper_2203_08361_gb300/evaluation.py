"""Trial statistics of the paper's benchmark protocol, on top of the library.

Kanao & Goto, arXiv 2203.08361, Results: every replica of a run is one trial;
P is the fraction of trials that reach the reference (best known) solution,
and the step-to-solution S = N_s log(0.01) / log(1 - P) is the number of time
steps that find it with probability 0.99.  The cut values of Eq. (eq_Cut) come
from hsb_cut_values.  This module only sorts and counts the library's outputs;
it is not part of the step path (every step runs in the CUDA kernels).
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np

from . import Solver, params as make_params


def success_probability(best_energy, target_energy: float, tol: float = 0.0) -> float:
    """P: fraction of trials whose best energy is at most target_energy + tol
    (tol = 0 for integer couplings, whose energies are exact)."""
    e = np.asarray(best_energy, dtype=np.float64)
    if e.size == 0:
        raise ValueError("no trials")
    return float(np.count_nonzero(e <= target_energy + tol)) / float(e.size)


def step_to_solution(p: float, steps: int) -> float:
    """S = N_s log(0.01) / log(1 - P) (Results).  For P >= 0.99 one run already
    succeeds with probability 0.99, so S = N_s (the formula equals N_s at
    P = 0.99); for P = 0 the solution is not found and S is infinite."""
    if not 0.0 <= p <= 1.0:
        raise ValueError("P must be in [0, 1]")
    if steps < 1:
        raise ValueError("steps must be >= 1")
    if p == 0.0:
        return math.inf
    if p >= 0.99:
        return float(steps)
    return steps * math.log(0.01) / math.log1p(-p)


@dataclass
class TrialStats:
    steps: int
    trials: int
    mean_cut: float
    max_cut: float
    min_energy: float
    p: float
    step_to_solution: float


def evaluate(J, form: str, steps_list, trials: int, seed: int, target_energy: float,
             tol: float = 0.0, **param_kw) -> list:
    """Runs `trials` replicas for each N_s in steps_list (the paper's Fig. 2 /
    Fig. 3 protocol) and returns one TrialStats per N_s: average and maximum
    cut value, minimum energy, P of reaching target_energy, and S."""
    out = []
    with Solver(J) as s:
        for steps in steps_list:
            p = make_params(form, **param_kw)
            _, energy = s.run(p, trials, int(steps), seed)
            cut = s.cut_values(energy)
            prob = success_probability(energy, target_energy, tol)
            out.append(TrialStats(int(steps), trials, float(cut.mean()), float(cut.max()),
                                  float(energy.min()), prob, step_to_solution(prob, int(steps))))
    return out


def grid_points(grid: dict) -> list:
    """Every combination of the parameter values in `grid` (name -> list of
    values), the last name varying fastest, as dicts."""
    names = list(grid)
    for n in names:
        if len(grid[n]) == 0:
            raise ValueError(f"no values for {n!r}")
    return [dict(zip(names, combo)) for combo in itertools.product(*(grid[n] for n in names))]


@dataclass
class SweepPoint:
    params: dict
    stats: TrialStats


def sweep(J, form: str, grid: dict, steps: int, trials: int, seed: int, target_energy: float,
          tol: float = 0.0, **fixed) -> list:
    """The paper's parameter scans (Fig. 1: P and S over gamma and dt at fixed
    N_s; c1 likewise): `trials` replicas per point of `grid` (e.g. {"dt":
    [...], "gamma": [...], "c1": [...]}), every point on the same seed, with
    the remaining parameters from `fixed`.  Returns one SweepPoint per grid
    point in grid_points order."""
    out = []
    with Solver(J) as s:
        for point in grid_points(grid):
            kw = dict(fixed)
            kw.update(point)
            p = make_params(form, **kw)
            _, energy = s.run(p, trials, int(steps), seed)
            cut = s.cut_values(energy)
            prob = success_probability(energy, target_energy, tol)
            out.append(SweepPoint(dict(point), TrialStats(
                int(steps), trials, float(cut.mean()), float(cut.max()), float(energy.min()),
                prob, step_to_solution(prob, int(steps)))))
    return out
