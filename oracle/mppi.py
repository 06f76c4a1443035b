"""FP64 oracle of one MPPI iteration with the collision cost of Section II-D.

TEST INFRASTRUCTURE ONLY (like the rest of this package): the tests, the
smoke check and the CPU-baseline leg of the benchmark use it; the product
library never does.  It shares no code with the CUDA path.

The steps follow Section II-D in the paper's order, for a robot that is one
sphere of radius r moving under single-integrator (velocity) control:

1. sample: the K perturbations eps[k, t] of the nominal sequence U are given
   (the caller draws them), so rollout k applies u[k, t] = U[t] + eps[k, t];
2. roll out: x[k, 0] = x0, x[k, t + 1] = x[k, t] + dt u[k, t], t = 0 .. T-1;
   the positions x[k, 1 .. T] are the sphere centres of the rollout;
3. cost (the equation that sums the four terms of C^k; the image term is
   zero here): C^k = w_collision C_collision^k + C_task^k + C_control^k with
   C_collision^k = sum over t of the Eq. 11 cost averaged over the neighbour
   set (one link, so the sum over links is that value), C_task^k =
   w_goal sum_t |x[k, t] - goal|^2 + w_terminal |x[k, T] - goal|^2 and
   C_control^k = w_control sum_t |u[k, t]|^2;
4. weights (Eq. 10): w^k = exp(-C^k / lambda) / sum_l exp(-C^l / lambda),
   evaluated as exp(-(C^k - min C) / lambda) over its sum (the same value);
5. update: U'[t] = U[t] + sum_k w^k eps[k, t] (the nominal sequence moves
   in the direction of the lower-cost perturbations).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import MODE_MEAN, Params, group_reduce, query


@dataclass
class MppiDesc:
    K: int
    T: int
    dt: float = 0.1
    radius: float = 0.15
    nsigma: float = 1.0
    lam: float = 1.0
    w_collision: float = 10.0
    w_goal: float = 0.1
    w_terminal: float = 1.0
    w_control: float = 0.01
    goal: tuple = (0.0, 0.0, 0.0)


def rollout(x0, U, eps, dt):
    """Positions x[k, 1 .. T] and controls u[k, t] of every rollout (step 2)."""
    x0 = np.asarray(x0, np.float64)
    u = np.asarray(U, np.float64)[None, :, :] + np.asarray(eps, np.float64)
    K, T, _ = u.shape
    x = np.empty((K, T, 3))
    cur = np.repeat(x0[None, :], K, 0)
    for t in range(T):
        cur = cur + dt * u[:, t, :]
        x[:, t, :] = cur
    return x, u


def costs(scene, x, u, d: MppiDesc, params: Params | None = None):
    """Per-rollout (C, C_collision, C_task, C_control) of step 3."""
    K, T, _ = x.shape
    spheres = np.concatenate([x.reshape(-1, 3), np.full((K * T, 1), d.radius)], 1)
    res = query(scene, spheres, 0, d.nsigma, params)
    c_col, _ = group_reduce(res["mean_cost"], res["collide"], T)
    g = np.asarray(d.goal, np.float64)
    c_task = d.w_goal * ((x - g) ** 2).sum((1, 2)) + d.w_terminal * ((x[:, -1, :] - g) ** 2).sum(1)
    c_ctrl = d.w_control * (u ** 2).sum((1, 2))
    return d.w_collision * c_col + c_task + c_ctrl, c_col, c_task, c_ctrl


def weights(C, lam):
    """Eq. 10 softmin weights of the rollout costs."""
    C = np.asarray(C, np.float64)
    e = np.exp(-(C - C.min()) / lam)
    return e / e.sum()


def step(scene, x0, U, eps, d: MppiDesc, params: Params | None = None) -> dict:
    """One MPPI iteration: updated nominal sequence, costs and weights."""
    x, u = rollout(x0, U, eps, d.dt)
    C, c_col, c_task, c_ctrl = costs(scene, x, u, d, params)
    w = weights(C, d.lam)
    U_new = np.asarray(U, np.float64) + np.einsum("k,ktd->td", w, np.asarray(eps, np.float64))
    return {"U": U_new, "cost": C, "weights": w, "collision": c_col, "task": c_task, "control": c_ctrl,
            "positions": x}


__all__ = ["MppiDesc", "rollout", "costs", "weights", "step", "MODE_MEAN"]
