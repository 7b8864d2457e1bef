"""Topology optimisation driver ("Results and Discussion": adjoint-gradient
TopOpt of the density p in [0, 1]^N with conic filter and binarisation,
ramped during the optimisation).

The objective and its gradient come from a callable `value_and_grad(rhos)`
returning (f, [df/drho per zone]) -- e.g. a single zone's zda_iteration or
a lens's forward + adjoint.  Maximisation by Adam with the densities clipped
to [0, 1] after every step; the projection strength beta is raised on a
schedule (continuation).  Every iteration is logged as one JSON line; the
state (densities, Adam moments, iteration, beta) can be checkpointed to .npz
and resumed.
"""
import json
import time

import numpy as np


class Adam:
    def __init__(self, shapes, lr=0.01, b1=0.9, b2=0.999, eps=1e-12):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = [np.zeros(s) for s in shapes]
        self.v = [np.zeros(s) for s in shapes]
        self.t = 0

    def step(self, params, grads, scale=1.0):
        """Ascent step on params (list of arrays) with grads; returns new params."""
        self.t += 1
        out = []
        for k, (p, g) in enumerate(zip(params, grads)):
            g = np.asarray(g, dtype=np.float64) * scale
            self.m[k] = self.b1 * self.m[k] + (1 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1 - self.b2) * g * g
            mh = self.m[k] / (1 - self.b1 ** self.t)
            vh = self.v[k] / (1 - self.b2 ** self.t)
            out.append(np.clip(p + self.lr * mh / (np.sqrt(vh) + self.eps), 0.0, 1.0))
        return out


def beta_schedule(it, beta0=1.0, beta_max=32.0, every=20, factor=2.0):
    """Continuation: beta0 * factor^(it // every), capped at beta_max."""
    k = it // every
    if beta0 * factor ** min(k, 64) >= beta_max:
        return beta_max
    return beta0 * factor ** k


class TopOpt:
    def __init__(self, value_and_grad, rhos, lr=0.02, set_beta=None, schedule=beta_schedule, log_path=None):
        self.f = value_and_grad
        self.rhos = [np.asarray(r, dtype=np.float64).copy() for r in rhos]
        self.opt = Adam([r.shape for r in self.rhos], lr=lr)
        self.set_beta = set_beta
        self.schedule = schedule
        self.log_path = log_path
        self.it = 0
        self.history = []

    def step(self):
        beta = self.schedule(self.it) if self.schedule else None
        if self.set_beta is not None and beta is not None:
            self.set_beta(beta)
        t0 = time.perf_counter()
        val, grads = self.f(self.rhos)
        # scale-free ascent: Adam normalises per element; keep the raw value for the log
        self.rhos = self.opt.step(self.rhos, grads)
        rec = {"iter": self.it, "objective": float(val), "beta": beta, "seconds": time.perf_counter() - t0,
               "grey": float(np.mean([np.mean(4 * r * (1 - r)) for r in self.rhos]))}
        self.history.append(rec)
        if self.log_path:
            with open(self.log_path, "a") as fh:
                fh.write(json.dumps(rec) + "\n")
        self.it += 1
        return rec

    def run(self, n):
        for _ in range(n):
            self.step()
        return self.history

    def save(self, path):
        np.savez(path, it=self.it, t=self.opt.t, n=len(self.rhos),
                 **{"rho%d" % k: r for k, r in enumerate(self.rhos)},
                 **{"m%d" % k: m for k, m in enumerate(self.opt.m)},
                 **{"v%d" % k: v for k, v in enumerate(self.opt.v)})

    def load(self, path):
        d = np.load(path)
        n = int(d["n"])
        self.rhos = [d["rho%d" % k].copy() for k in range(n)]
        self.opt.m = [d["m%d" % k].copy() for k in range(n)]
        self.opt.v = [d["v%d" % k].copy() for k in range(n)]
        self.opt.t = int(d["t"])
        self.it = int(d["it"])
