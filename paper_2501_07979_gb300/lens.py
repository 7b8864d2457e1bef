"""A lens = concentric zones (section "Zoned discrete axisymmetry (ZDA)").

Zones are independent FDTD problems; the only coupling of a whole-lens
iteration is the focal field, the sum of the zones' focal phasors
(2 x wavelengths complex numbers), whose sensitivity every zone needs for its
adjoint run.  With several processes (one GPU each) the zones are assigned
by longest-processing-time-first on their cost n_r n_phi n_z n_steps and the
phasor sum is one all-reduce of a few hundred bytes.

The zone solver is pluggable (any object with forward(rho) -> S and
adjoint(dI_dS) -> grad): `Zone` on a GPU, or any stand-in.
"""
import numpy as np


def zone_cost(spec):
    return float(spec.n_r) * spec.n_phi * spec.n_z * spec.n_steps


def assign_zones(specs, world):
    """Longest-processing-time-first: returns owner rank per zone (list)."""
    order = sorted(range(len(specs)), key=lambda z: -zone_cost(specs[z]))
    load = [0.0] * world
    owner = [0] * len(specs)
    for z in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[z] = r
        load[r] += zone_cost(specs[z])
    return owner


class ShardedLens:
    """Zones of one lens spread over the ranks of a torch.distributed group.

    solvers: {zone index: solver} for the zones this rank owns.
    forward(rhos) -> S_lens (complex, summed over all zones of all ranks).
    adjoint(dI_dS) -> {zone index: dI/drho} for the local zones, with dI_dS
    the objective's sensitivity to the lens phasors (the same for every zone:
    dS_lens/dS_zone = 1).
    """

    def __init__(self, specs, solvers, group=None):
        self.specs = specs
        self.solvers = solvers
        self.group = group

    def _allreduce(self, x):
        import torch
        import torch.distributed as dist
        if not dist.is_available() or not dist.is_initialized():
            return x
        t = torch.from_numpy(np.ascontiguousarray(np.stack([x.real, x.imag], 1)))
        dist.all_reduce(t, group=self.group)
        a = t.numpy()
        return a[:, 0] + 1j * a[:, 1]

    def forward(self, rhos):
        S = None
        for z, solver in sorted(self.solvers.items()):
            s = np.asarray(solver.forward(rhos[z]), dtype=np.complex128)
            S = s if S is None else S + s
        if S is None:
            nq = 2 * len(self.specs[0].wavelengths)
            S = np.zeros(nq, np.complex128)
        return self._allreduce(S)

    def adjoint(self, dI_dS):
        return {z: solver.adjoint(dI_dS) for z, solver in sorted(self.solvers.items())}
