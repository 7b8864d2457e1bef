"""Tile-shape tuner for the time-step kernel of a zone.

For each candidate (variant, phi rows per block, radius ranges) the zone's
step kernel is timed on the GPU for a few steps (`Zone.time_steps`); the
fastest is applied to the zone and remembered in a JSON cache keyed by the
zone's shape (n_r, n_phi, n_z, PML widths) and r-PML form, so zones of the
same shape in a lens (and later runs) reuse it without timing again.
Candidates the zone refuses (the fused steps with the stretched r-PML) are
skipped.  The candidates are the split step's thread-block shapes (4 to 32
phi rows), the one-cell split step, the streaming fused step, the
TMA-tiled fused step's tile rows and radius ranges, and the split step with
its E half or both halves on TMA-staged tiles.
"""
import json
import os

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "zda_tiles.json")


def shape_key(spec):
    return "%dx%dx%d_p%d-%d-%d_%s" % (spec.n_r, spec.n_phi, spec.n_z, spec.pml_r_in, spec.pml_r_out,
                                      spec.pml_z, "axis" if spec.n_fold == 0 else "wedge")


def candidates(spec):
    """(variant, tile_phi, i_ranges) choices for the zone: the split step's
    thread-block shape (phi rows x z-pairs, 256 threads), the one-cell split
    step, the streaming fused step, the TMA-tiled fused step's tile rows
    and radius ranges, and the split step with its E half (or both halves)
    on TMA tiles."""
    cands = [(2, 2, 0)]
    pair = spec.n_z % 2 == 0 and spec.pml_z % 2 == 0 and spec.n_fold > 0
    if pair:
        cands += [(0, rows, eb) for rows in (4, 8, 16, 32) if rows <= 2 * max(spec.n_phi, 2) for eb in (0, 3)]
    else:
        cands.append((0, 16, 0))
    if spec.n_fold > 0 and spec.n_z % 2 == 0 and spec.n_z <= 256:
        cands += [(1, 2, 0), (1, 4, 0)]
    if pair:
        for tj in (4, 8, 16):
            if tj <= 2 * max(spec.n_phi, 2):
                cands += [(3, tj, 0), (3, tj, max(1, spec.n_r // 30))]
        for tj in (8, 16, 32):
            if tj <= 2 * max(spec.n_phi, 2):
                cands += [(4, tj, 0), (5, tj, 0)]
    return sorted(set(cands))


def tune_zone(zone, steps=40, cache_path=None, use_cache=True):
    """Pick and apply the fastest step kernel for `zone`; returns
    (choice, {choice: ms}) with choice = (variant, tile_phi, i_ranges)."""
    from ._lib import ZdaError
    path = cache_path or DEFAULT_CACHE
    key = shape_key(zone.spec) + "_rpml%d" % zone.radial_pml()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            cache = json.load(open(path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        choice = tuple(cache[key]["choice"])
        zone.set_kernel(*choice)
        return choice, {}
    times = {}
    for c in candidates(zone.spec):
        try:
            zone.set_kernel(*c)
            zone.time_steps(4)                      # warm-up (module load, first touch)
            times[c] = zone.time_steps(steps)
        except ZdaError:
            continue
    choice = min(times, key=times.get)
    zone.set_kernel(*choice)
    if use_cache:
        cache[key] = {"choice": list(choice), "ms_per_step": times[choice] / steps,
                      "times": {"%d,%d,%d" % c: t / steps for c, t in times.items()}}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".%d.tmp" % os.getpid()
        json.dump(cache, open(tmp, "w"), indent=1)
        os.replace(tmp, path)
    return choice, times
