"""Sharding one record across ranks (one process per GPU).

The estimate and its error bar are sums over groups of the per-group spectra and
of their squares (Sec. 4.2, Eq. 35-36), so ranks that process disjoint ranges
of whole groups combine by adding their plans' exported states; no data moves
between ranks while the record is processed.  `group_ranges` gives each rank
its range; `reduce_state` adds the states of all ranks with one sum all-reduce
(any torch.distributed backend) after checking that the plans agree.
"""
from __future__ import annotations

STATE_HEADER = 16
CFG_WORDS = 14  # header words that must agree; 14 = groups, 15 = samples


def group_ranges(n_samples: int, T: int, m: int, world: int):
    """Sample ranges [start, stop) of each rank: contiguous runs of whole groups of
    m frames of T samples, balanced to within one group; samples after the last
    whole group belong to no rank (the single-plan path drops them too)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    span = m * T
    G = n_samples // span
    base, extra = divmod(G, world)
    out, g0 = [], 0
    for r in range(world):
        g = base + (1 if r < extra else 0)
        out.append((g0 * span, (g0 + g) * span))
        g0 += g
    return out


def reduce_state(state, group=None):
    """In place: replace this rank's state (1-D float64 torch tensor, laid out as
    ss_export_state writes it) by the sum over the ranks of `group`.  Raises
    ValueError on every rank if the plans' configurations differ."""
    import torch
    import torch.distributed as dist

    if state.dim() != 1 or state.dtype != torch.float64 or state.numel() < STATE_HEADER:
        raise ValueError("state must be a 1-D float64 tensor with its header")
    cfg = state[:CFG_WORDS].clone()
    lo, hi = cfg.clone(), cfg.clone()
    n = torch.tensor([float(state.numel())], dtype=torch.float64, device=state.device)
    n_lo, n_hi = n.clone(), n.clone()
    dist.all_reduce(lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hi, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(n_lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(n_hi, op=dist.ReduceOp.MAX, group=group)
    if not (torch.equal(lo, hi) and torch.equal(n_lo, n_hi)):
        raise ValueError("ranks hold states of plans with different configurations")
    dist.all_reduce(state[CFG_WORDS:], op=dist.ReduceOp.SUM, group=group)
    return state
