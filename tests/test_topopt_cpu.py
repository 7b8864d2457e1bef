"""TopOpt driver logic on CPU (no GPU): projected Adam ascent, beta
continuation, logging, checkpoint/resume reproducing the same trajectory."""
import json

import numpy as np

from paper_2501_07979_gb300.topopt import TopOpt, beta_schedule


def _quadratic(target):
    def f(rhos):
        r = rhos[0]
        return -float(np.sum((r - target) ** 2)), [-2 * (r - target)]
    return f


def test_projected_ascent_reaches_box_constrained_optimum(tmp_path):
    rng = np.random.default_rng(0)
    target = rng.uniform(-0.5, 1.5, (6, 5))          # optimum outside the box in places
    opt = TopOpt(_quadratic(target), [np.full((6, 5), 0.5)], lr=0.05, schedule=None,
                 log_path=str(tmp_path / "log.jsonl"))
    opt.run(400)
    assert np.allclose(opt.rhos[0], np.clip(target, 0, 1), atol=2e-2)
    lines = [json.loads(l) for l in open(tmp_path / "log.jsonl")]
    assert len(lines) == 400 and lines[-1]["objective"] > lines[0]["objective"]


def test_checkpoint_resume_is_exact(tmp_path):
    rng = np.random.default_rng(1)
    target = rng.uniform(0, 1, (4, 3))
    a = TopOpt(_quadratic(target), [np.full((4, 3), 0.2)], lr=0.03)
    a.run(7)
    a.save(str(tmp_path / "ck.npz"))
    a.run(5)
    b = TopOpt(_quadratic(target), [np.zeros((4, 3))], lr=0.03)
    b.load(str(tmp_path / "ck.npz"))
    b.run(5)
    assert b.it == a.it and np.array_equal(a.rhos[0], b.rhos[0])


def test_beta_continuation_schedule():
    assert beta_schedule(0) == 1.0 and beta_schedule(19) == 1.0 and beta_schedule(20) == 2.0
    assert beta_schedule(10 ** 6) == 32.0
    seen = []
    opt = TopOpt(_quadratic(np.zeros((2, 2))), [np.full((2, 2), 0.5)], set_beta=seen.append,
                 schedule=lambda it: beta_schedule(it, every=2))
    opt.run(5)
    assert seen == [1.0, 1.0, 2.0, 2.0, 4.0]


def test_metrics_callback_lands_in_the_log(tmp_path):
    target = np.full((3, 3), 0.7)
    seen = []

    def metrics(it, rhos):
        seen.append(it)
        return {"I_per_lambda": [float(np.mean(rhos[0])), 1.0], "fe": 0.5}

    opt = TopOpt(_quadratic(target), [np.full((3, 3), 0.2)], lr=0.05, schedule=None,
                 log_path=str(tmp_path / "m.jsonl"), metrics=metrics)
    opt.run(3)
    lines = [json.loads(l) for l in open(tmp_path / "m.jsonl")]
    assert seen == [0, 1, 2]
    assert all("fe" in l and len(l["I_per_lambda"]) == 2 for l in lines)
    assert lines[-1]["I_per_lambda"][0] > lines[0]["I_per_lambda"][0] - 1e-12     # rho moves up to 0.7
