"""Autotuner for the step kernel's block shape.

Times sc_step for each candidate (variant, tile_y, tile_z, stages,
blocks_per_sm) on the given lattice with CUDA events and returns the fastest.
The step kernels compute the same numbers for every candidate (bitwise), so
tuning changes speed only.
"""
from __future__ import annotations

import torch

from . import binding as B

# (variant, tile_y, tile_z, stages, blocks_per_sm); 0 = the library's choice.  The first
# candidate is the library default, so the tuner never returns a slower configuration than it.
DEFAULT = [(0, 0, 0, 0, 0)]
STAGED = [(2, 4, 0, 1, 3), (2, 4, 0, 2, 2), (2, 4, 16, 1, 3), (2, 4, 32, 1, 3), (2, 4, 16, 2, 3),
          (2, 8, 0, 1, 3), (2, 8, 0, 1, 2), (2, 8, 0, 1, 1), (2, 8, 16, 2, 1), (2, 8, 32, 1, 2)]
GENERIC = [(1, 8, 0, 0, 0), (1, 4, 0, 0, 0), (1, 8, 16, 0, 0), (1, 8, 32, 0, 0), (1, 4, 32, 0, 0)]
CHUNK_SITES = {B.SC_STORE_F64: 1, B.SC_STORE_F32: 2, B.SC_STORE_F16: 4, B.SC_STORE_BF16: 4}


def staged_eligible(params) -> bool:
    """The library's rule for the cp.async-staged kernel: D3Q19, E4, nx >= 32 and a multiple of the
    sites in one 16-byte copy chunk of the storage."""
    return (params.lattice == B.SC_D3Q19 and params.stencil == B.SC_FORCE_E4 and params.nx >= 32
            and params.nx % CHUNK_SITES[params.storage] == 0)


def candidates_for(params):
    """The candidate list tune_step uses by default for these parameters."""
    cands = DEFAULT + (STAGED if staged_eligible(params) else []) + GENERIC
    if params.storage == B.SC_STORE_F64:  # staged F64: tile_y 4 only
        cands = [c for c in cands if not (c[0] == 2 and c[1] != 4)]
    if params.lattice == B.SC_D2Q9:  # one plane: tile_z is irrelevant
        cands = [c for c in cands if c[0] != 2 and c[2] in (0, 16)]
    return cands


def tune_step(params, nA0, nB0, candidates=None, steps: int = 64, warmup: int = 8, device="cuda"):
    """Returns ((variant, tile_y, tile_z, stages, blocks_per_sm), ms_per_step, table) for the
    fastest candidate."""
    if candidates is None:
        candidates = candidates_for(params)
    table = []
    for variant, ty, tz, ns, mb in candidates:
        p = B.make_params((params.nx, params.ny, params.nz), lattice=params.lattice, stencil=params.stencil,
                          psi_self=params.psi_self, storage=params.storage, tau=tuple(params.tau), G=params.G,
                          G_self=tuple(params.G_self), tile_y=ty, tile_z=tz, variant=variant, stages=ns,
                          blocks_per_sm=mb)
        sim = B.Simulation(p, nA0, nB0, device=device)
        sim.step(warmup)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(sim.stream)
        sim.step(steps)
        b.record(sim.stream)
        b.synchronize()
        sim.sync()
        table.append(((variant, ty, tz, ns, mb), a.elapsed_time(b) / steps))
        del sim
    best = min(table, key=lambda t: t[1])
    return best[0], best[1], table


def with_config(p, cfg):
    """Copy of sc_params p with (tile_y, tile_z, stages, blocks_per_sm) = cfg[:4]."""
    ty, tz, ns, mb = cfg[:4]
    return B.make_params((p.nx, p.ny, p.nz), lattice=p.lattice, stencil=p.stencil, psi_self=p.psi_self,
                         storage=p.storage, tau=tuple(p.tau), G=p.G, G_self=tuple(p.G_self), tile_y=ty, tile_z=tz,
                         variant=p.variant, stages=ns, blocks_per_sm=mb)


def tune_batch(params_list, fields, candidates, steps: int = 32, device="cuda"):
    """(tile_y, tile_z, stages, blocks_per_sm, persistent) for a batch (shared by its members), timed on
    the whole batch: each candidate block shape with whole 32-step runs as one persistent launch (where
    the batch has that form) and as one launch per step (steps a multiple of 32 times the graph
    replays).  Returns (best, ms_per_step, table)."""
    table = []
    for cfg in candidates:
        batch = B.Batch([with_config(p, cfg) for p in params_list], fields, device=device)
        for persistent in ((True, False) if batch.persistent else (False,)):
            batch.persistent = persistent
            batch.step(4)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(batch.stream)
            batch.step(steps)
            b.record(batch.stream)
            b.synchronize()
            table.append((tuple(cfg) + (persistent,), a.elapsed_time(b) / steps))
        del batch
    best = min(table, key=lambda t: t[1])
    return best[0], best[1], table
