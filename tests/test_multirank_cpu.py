"""Multi-rank lens path on CPU: two gloo ranks each own a subset of a lens's
zones (assigned longest-processing-time-first), solve them with the FP64
oracle, and all-reduce the focal phasors; the result must equal the
single-process sum, and each rank's adjoint gradients must equal the
single-process ones.  Failure detection: a rank whose zone solve fails
leaves before the all-reduce, and the other rank's collective ends with an
error instead of hanging."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from zda_inputs import zone_tiny, smoothed_rho


def _specs():
    base = dict(n_steps=250, filter_radius=0.2, beta=3.0, wavelengths=(0.9, 1.1),
                pulse_sigma=0.4, pulse_t0=1.6)
    return [zone_tiny(r_lo=5.0, n_fold=40, **base),
            zone_tiny(r_lo=7.0, n_fold=56, n_r=20, **base),
            zone_tiny(r_lo=9.0, n_fold=72, n_phi=6, **base)]


class OracleSolver:
    def __init__(self, spec):
        self.spec = spec

    def forward(self, rho):
        import oracle as O
        self.fwd = O.forward(self.spec, rho, nthreads=1)
        self.fwd["rho"] = rho
        return self.fwd["S"]

    def adjoint(self, dI_dS):
        import oracle as O
        adj = O.adjoint(self.spec, self.fwd, dI_dS, nthreads=1)
        g = self.fwd["geom"]
        rbar = O.conic_filter(self.spec, g, self.fwd["rho"])
        return O.conic_filter_T(self.spec, g, adj["grad_rho_tilde"] * O.project_grad(self.spec, rbar))


def _rhos(specs):
    return [smoothed_rho(s.n_r_design, s.n_phi, 100 + z, mode="minmax") for z, s in enumerate(specs)]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    from paper_2501_07979_gb300.lens import ShardedLens, assign_zones
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    specs = _specs()
    owner = assign_zones(specs, world)
    lens = ShardedLens(specs, {z: OracleSolver(specs[z]) for z in range(len(specs)) if owner[z] == rank})
    S = lens.forward(_rhos(specs))
    grads = lens.adjoint(4.0 * S)
    out.put((rank, S, grads))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_assign_zones_balances_cost():
    from paper_2501_07979_gb300.lens import assign_zones, zone_cost
    specs = _specs() * 3
    owner = assign_zones(specs, 2)
    loads = [sum(zone_cost(s) for s, o in zip(specs, owner) if o == r) for r in range(2)]
    assert max(loads) - min(loads) <= max(zone_cost(s) for s in specs)
    assert sorted(set(owner)) == [0, 1]


@pytest.mark.skipif(not __import__("torch").distributed.is_available(), reason="no torch.distributed")
def test_two_gloo_ranks_match_single_process():
    pytest.importorskip("paper_2501_07979_gb300.lens")
    specs = _specs()
    rhos = _rhos(specs)
    ref = [OracleSolver(s) for s in specs]
    S_ref = sum(r.forward(rho) for r, rho in zip(ref, rhos))
    g_ref = [r.adjoint(4.0 * S_ref) for r in ref]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    seen = {}
    for rank, S, grads in res:
        assert np.allclose(S, S_ref, rtol=1e-12, atol=0)
        for z, g in grads.items():
            assert z not in seen
            seen[z] = g
            assert np.allclose(g, g_ref[z], rtol=1e-10, atol=1e-14)
    assert sorted(seen) == list(range(len(specs)))


class _FailingSolver(OracleSolver):
    """A zone whose solve fails on this rank (an exception on the host)."""

    def forward(self, rho):
        raise RuntimeError("zone solve failed")


def _worker_failing(rank, world, port, out):
    """Rank 1 fails in its zone solve and exits without joining the phasor
    all-reduce; rank 0 must get an error from the collective (peer gone, or
    the process group's short timeout), not hang."""
    import datetime
    import time
    import torch.distributed as dist
    from paper_2501_07979_gb300.lens import ShardedLens, assign_zones
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    specs = _specs()
    owner = assign_zones(specs, world)
    cls = _FailingSolver if rank == 1 else OracleSolver
    lens = ShardedLens(specs, {z: cls(specs[z]) for z in range(len(specs)) if owner[z] == rank})
    t0 = time.time()
    try:
        lens.forward(_rhos(specs))
        out.put((rank, "ok", time.time() - t0))
    except Exception as e:                     # noqa: BLE001  (the failure is the point)
        out.put((rank, "error: %s" % type(e).__name__, time.time() - t0))
        if rank == 1:
            out.close()
            out.join_thread()                  # flush the report, then leave without cleanup
            os._exit(3)
    try:
        dist.destroy_process_group()
    except Exception:                          # noqa: BLE001
        pass


@pytest.mark.skipif(not __import__("torch").distributed.is_available(), reason="no torch.distributed")
def test_a_failed_rank_ends_the_others_collective_with_an_error():
    pytest.importorskip("paper_2501_07979_gb300.lens")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_failing, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (msg, dt)) for r, msg, dt in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
    assert res[1][0].startswith("error")                      # the failing rank saw its own failure
    assert res[0][0].startswith("error"), res[0]              # the survivor: an error, not a hang
    assert res[0][1] < 60                                     # within the group's timeout plus slack
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
