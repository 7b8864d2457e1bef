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
    def __init__(self, value_and_grad, rhos, lr=0.02, set_beta=None, schedule=beta_schedule, log_path=None,
                 metrics=None):
        """metrics(it, rhos) -> dict: extra quantities for the iteration's log
        record (e.g. intensity per wavelength, focusing efficiency, Strehl
        ratio, Gcell-upd/s), evaluated after the step."""
        self.f = value_and_grad
        self.metrics = metrics
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
        if self.metrics is not None:
            rec.update(self.metrics(self.it, self.rhos))
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


# --------------------------------------------------------------------------
# max-min over wavelengths in epigraph form (Eqs. 7-8): maximise q subject to
# q <= I(p, w_i) for every design wavelength, p in [0, 1]^N.
# --------------------------------------------------------------------------
class CCSA:
    """Conservative convex separable approximations with quadratic terms
    (Svanberg, SIAM J. Optim. 12 (2002) 555-573): minimise f_0(x) subject to
    f_i(x) <= 0, i = 1..m, lo <= x <= hi.

    Every outer iteration replaces each f_i by
        g_i(x) = f_i(x_k) + grad f_i(x_k) . (x - x_k) + (rho_i / 2) sum_j ((x_j - x_kj) / sigma_j)^2
    and solves the separable convex subproblem (min g_0, g_i <= 0, x within
    sigma of x_k and within the bounds) through its dual, a smooth concave
    function of m multipliers y >= 0 whose gradient is (g_i(x(y))) and whose
    inner minimiser is closed-form per coordinate.  The step is accepted once
    every g_i is conservative at the new point (g_i >= f_i); otherwise the
    offending rho_i grow and the subproblem is solved again.  sigma_j shrinks
    when coordinate j oscillates and grows when it moves steadily."""

    def __init__(self, lo, hi, m, sigma0=0.5, rho_min=1e-5, max_inner=20):
        self.lo = np.asarray(lo, dtype=np.float64)
        self.hi = np.asarray(hi, dtype=np.float64)
        self.m = m
        self.sigma = sigma0 * (self.hi - self.lo)
        self.rho_min = rho_min
        self.max_inner = max_inner
        self.rho = None
        self.prev = []                      # the last two iterates (oscillation test)

    def _solve_sub(self, x, f, g, rho):
        """Dual solution of the subproblem: returns (x_hat, approximations g_i(x_hat), w)."""
        from scipy.optimize import minimize
        s2 = self.sigma ** 2
        dlo = np.maximum(self.lo, x - self.sigma) - x
        dhi = np.minimum(self.hi, x + self.sigma) - x

        def inner(y):
            a = g[0] + y @ g[1:]
            b = rho[0] + y @ rho[1:]
            d = np.clip(-a * s2 / b, dlo, dhi)
            w = 0.5 * float(np.sum(d * d / s2))
            gv = f + g @ d + rho * w
            return d, gv, w

        def negdual(y):
            _, gv, _ = inner(y)
            return -(gv[0] + y @ gv[1:]), -gv[1:]

        if self.m > 0:
            res = minimize(negdual, np.zeros(self.m), jac=True, method="L-BFGS-B",
                           bounds=[(0.0, None)] * self.m, options={"maxiter": 500, "gtol": 1e-12, "ftol": 1e-15})
            y = np.maximum(res.x, 0.0)
        else:
            y = np.zeros(0)
        d, gv, w = inner(y)
        return x + d, gv, w

    def step(self, x, f, g, evaluate):
        """One outer iteration.  f: values f_0..f_m at x; g: gradients
        [m + 1][n]; evaluate(x) -> values at a trial point.  Returns
        (x_new, f_new, inner iterations)."""
        x = np.asarray(x, dtype=np.float64)
        f = np.asarray(f, dtype=np.float64)
        g = np.asarray(g, dtype=np.float64)
        n = x.size
        if len(self.prev) == 2:
            osc = (x - self.prev[1]) * (self.prev[1] - self.prev[0])
            gamma = np.where(osc < 0, 0.7, np.where(osc > 0, 1.2, 1.0))
            span = self.hi - self.lo
            self.sigma = np.clip(gamma * self.sigma, 1e-4 * span, 10 * span)
        rho = np.maximum(self.rho_min, 0.1 / n * (np.abs(g) @ self.sigma)) if self.rho is None else self.rho
        for it in range(1, self.max_inner + 1):
            xh, gv, w = self._solve_sub(x, f, g, rho)
            fh = np.asarray(evaluate(xh), dtype=np.float64)
            bad = fh > gv + 1e-12 * (1 + np.abs(fh))
            if not bad.any() or w <= 0:
                break
            upd = np.minimum(10 * rho, 1.1 * (rho + (fh - gv) / w))
            rho = np.where(bad, upd, rho)
        self.rho = np.maximum(0.1 * rho, self.rho_min)
        self.prev = (self.prev + [x.copy()])[-2:]
        return xh, fh, it


def wavelength_intensities(S, n_lambda):
    """I(w_l) = 2 (|S(+w_l)|^2 + |S(-w_l)|^2) for each design wavelength (the
    summed intensity of the objective, split per wavelength)."""
    S = np.asarray(S)
    return np.array([2.0 * (abs(S[l]) ** 2 + abs(S[l + n_lambda]) ** 2) for l in range(n_lambda)])


def wavelength_sensitivity(S, n_lambda, l):
    """dI(w_l)/dRe S + i dI(w_l)/dIm S: 4 S on wavelength l's two signed frequencies."""
    g = np.zeros(len(S), dtype=np.complex128)
    g[l] = 4.0 * S[l]
    g[l + n_lambda] = 4.0 * S[l + n_lambda]
    return g


def zone_wavelength_objectives(zone, n_lambda):
    """objectives(rho, need_grad) for one GPU zone: one forward run, then one
    adjoint run per wavelength (the adjoint source carries only that
    wavelength's sensitivity)."""
    import torch

    def objectives(rho, need_grad=True):
        r = torch.as_tensor(rho, dtype=torch.float32, device=zone.device)
        S = zone.forward(r)
        I = wavelength_intensities(S, n_lambda)
        if not need_grad:
            return I
        grads = [zone.adjoint(wavelength_sensitivity(S, n_lambda, l)).cpu().numpy().astype(np.float64)
                 for l in range(n_lambda)]
        return I, grads

    return objectives


class Epigraph:
    """max_p min_l I(p, w_l) as max q s.t. q <= I(p, w_l) (Eqs. 7-8), solved by
    CCSA over x = (p, q), p in [0, 1]^N, q in [0, q_max].
    objectives(rho, need_grad) -> I per wavelength (and their gradients)."""

    def __init__(self, objectives, rho0, q_max=None, sigma0=0.3, log_path=None):
        self.f = objectives
        self.shape = np.asarray(rho0).shape
        self.rho = np.asarray(rho0, dtype=np.float64).copy()
        I0 = self.f(self.rho, False)
        self.m = len(I0)
        self.q = float(np.min(I0))
        q_max = q_max if q_max is not None else 20.0 * float(np.max(I0)) + 1e-12
        n = self.rho.size
        self.opt = CCSA(np.zeros(n + 1), np.concatenate([np.ones(n), [q_max]]), self.m, sigma0=sigma0)
        self.log_path = log_path
        self.history = []
        self.it = 0

    def _values(self, x, I):
        return np.concatenate([[-x[-1]], x[-1] - np.asarray(I)])

    def step(self):
        t0 = time.perf_counter()
        x = np.concatenate([self.rho.ravel(), [self.q]])
        I, grads = self.f(self.rho, True)
        n = self.rho.size
        g = np.zeros((self.m + 1, n + 1))
        g[0, -1] = -1.0
        for l in range(self.m):
            g[l + 1, :n] = -np.asarray(grads[l]).ravel()
            g[l + 1, -1] = 1.0
        last = {}

        def evaluate(xh):
            Ih = self.f(xh[:n].reshape(self.shape), False)
            last["I"] = Ih
            return self._values(xh, Ih)

        xn, fn, inner = self.opt.step(x, self._values(x, I), g, evaluate)
        self.rho = xn[:n].reshape(self.shape)
        self.q = float(xn[-1])
        rec = {"iter": self.it, "min_I": float(np.min(last["I"])), "I": [float(v) for v in last["I"]],
               "q": self.q, "inner": inner, "seconds": time.perf_counter() - t0}
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
