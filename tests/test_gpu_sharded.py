"""The sharded lens under NCCL: one process, world size 1, GPU zone solvers.

ShardedLens assigns a lens's zones to ranks (longest processing time
first) and all-reduces the zones' focal phasors once per forward; under the
NCCL backend the reduction runs on the rank's CUDA device.  With one rank
it must reproduce the single-GPU lens (one CUDA graph over all zones)."""
import os
import socket

import numpy as np
import pytest
import torch

from zda_inputs import zone_tiny, smoothed_rho

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_sharded_lens_under_nccl_equals_single_gpu_lens():
    import torch.distributed as dist
    from paper_2501_07979_gb300 import Zone
    from paper_2501_07979_gb300.lens import Lens, ShardedLens, assign_zones
    base = dict(n_steps=400, filter_radius=0.2, beta=3.0, wavelengths=(0.9, 1.1), pulse_sigma=0.4,
                pulse_t0=1.6, focal=12.0)
    specs = [zone_tiny(r_lo=0.0, n_fold=0, n_phi=1, pml_r_in=0, n_r=20, **base),
             zone_tiny(r_lo=1.2, n_fold=12, n_phi=6, n_r=24, **base),
             zone_tiny(r_lo=3.2, n_fold=24, n_phi=8, n_r=28, **base)]
    rhos = [torch.tensor(smoothed_rho(s.n_r_design, s.n_phi, 40 + z, mode="minmax"), dtype=torch.float32,
                         device="cuda:0") for z, s in enumerate(specs)]
    lens = Lens([Zone(s, device=0) for s in specs])
    S_ref = lens.forward(rhos)
    g_ref = lens.adjoint(4.0 * S_ref)
    store = dist.TCPStore("127.0.0.1", _free_port(), 1, True)
    dist.init_process_group("nccl", store=store, rank=0, world_size=1)
    try:
        torch.cuda.set_device(0)
        owner = assign_zones(specs, 1)
        solvers = {z: Zone(s, device=0) for z, s in enumerate(specs) if owner[z] == 0}
        sh = ShardedLens(specs, solvers)
        S = sh.forward(rhos)
        g = sh.adjoint(4.0 * S)
    finally:
        dist.destroy_process_group()
    assert np.allclose(S, S_ref, rtol=1e-6, atol=0)
    for z in range(len(specs)):
        a = g[z].cpu().numpy() if hasattr(g[z], "cpu") else np.asarray(g[z])
        b = g_ref[z].cpu().numpy() if hasattr(g_ref[z], "cpu") else np.asarray(g_ref[z])
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
