"""Particle swarm optimisation of QAOA parameters (Section 4, "QAOA with swarm
particle optimization").

TEST INFRASTRUCTURE ONLY (see the package docstring).

The method as the section describes it: R particles, each a parameter vector
theta scored by an objective L(theta) that is maximised (there, the QAOA
energy <H_MaxCut>).  Initial positions and velocities are given.  Each swarm
step first updates every velocity from a damping term (omega), an attraction
towards the particle's own best position so far (phi_p times a uniform r_p)
and an attraction towards the best position of the whole swarm so far (phi_g
times a uniform r_g); then every particle moves by its new velocity and all
new positions are scored.  Bests move only to strictly larger scores, and the
swarm's best used during a step is the one it had before the step.

Readings (the section is silent or garbled on these):
* the printed update has (theta - theta_best) in both attraction terms, which
  would push particles away from the bests; the standard swarm update of
  Kennedy and Eberhart (1995), which the section cites and which attracts
  them, is taken: + phi_p r_p (theta_best - theta) + phi_g r_g (theta_swarm - theta);
* r_p and r_g are one number per particle per step (the equation writes them
  as scalars drawn each step); they are inputs here, like the initial
  positions and velocities;
* the trace is the best score found after each evaluation, evaluations
  ordered step by step and, within a step, particle by particle (the section's
  figures plot the best value after a number of evaluations).
"""
from __future__ import annotations

import numpy as np


def swarm(objective, pos0, vel0, rp, rg, omega: float, phi_p: float, phi_g: float):
    """Run the swarm.

    objective : callable theta (D,) -> float, maximised
    pos0, vel0: (R, D) initial positions and velocities
    rp, rg    : (steps, R) uniform draws of each step

    Returns (trace ((steps + 1) * R,), best_pos (D,), best_val, history
    (steps + 1, R, D) of the scored positions).
    """
    x = np.array(pos0, dtype=np.float64)
    v = np.array(vel0, dtype=np.float64)
    rp = np.asarray(rp, dtype=np.float64)
    rg = np.asarray(rg, dtype=np.float64)
    R, D = x.shape
    steps = rp.shape[0]
    history = [x.copy()]
    scores = [objective(x[k]) for k in range(R)]
    own_best = x.copy()
    own_val = list(scores)
    trace = []
    best_val = -np.inf
    best_pos = None
    running = -np.inf
    for k in range(R):
        running = max(running, scores[k])
        trace.append(running)
        if scores[k] > best_val:
            best_val, best_pos = scores[k], x[k].copy()
    for s in range(steps):
        for k in range(R):
            v[k] = (omega * v[k]
                    + phi_p * rp[s, k] * (own_best[k] - x[k])
                    + phi_g * rg[s, k] * (best_pos - x[k]))
            x[k] = x[k] + v[k]
        history.append(x.copy())
        scores = [objective(x[k]) for k in range(R)]
        for k in range(R):
            running = max(running, scores[k])
            trace.append(running)
            if scores[k] > own_val[k]:
                own_val[k] = scores[k]
                own_best[k] = x[k].copy()
        for k in range(R):
            if scores[k] > best_val:
                best_val, best_pos = scores[k], x[k].copy()
    return np.array(trace), best_pos, best_val, np.array(history)


def qaoa_objective(n: int, edges, p: int):
    """L(theta) = <H_MaxCut> for theta = (gamma_1..gamma_p, beta_1..beta_p)."""
    from .qaoa import qaoa_energy

    def f(theta):
        theta = np.asarray(theta, dtype=np.float64)
        return qaoa_energy(n, edges, theta[:p], theta[p:])
    return f
