"""The multi-rank path on CPU: whole-group shards per rank and the sum all-reduce of
plan states over torch.distributed (gloo, world size 2 and 3).

Each rank turns the oracle's estimate on its own shard back into group sums (the
inverse of Eq. 35-36: sum = G mean, sum of squares = G (G-1) err^2 + G mean^2),
lays them out after a state header, and calls `reduce_state`.  The merged sums
must give the oracle's estimate on the whole record.
"""
import os
import socket

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from paper_2505_01231_gb300 import shard  # noqa: E402

T, M_FRAMES, DT = 32, 6, 0.5


def header(T, m, groups, samples):
    h = np.zeros(shard.STATE_HEADER)
    h[:4] = (1, T, m, 2 | 8 | 16)
    h[14], h[15] = groups, samples
    return h


def state_of(ref, T, m, samples):
    """Header + (sum Re, sum Im, sum Re^2, sum Im^2) of S2, S3, S4 from an estimate."""
    G = ref["G"]
    parts = [header(T, m, G, samples)]
    for key in ("S2", "S3", "S4"):
        mean, err = ref[key].ravel(), ref[key + "_err"].reshape(-1, 2)
        for c, e in ((mean.real, err[:, 0]), (mean.imag, err[:, 1])):
            parts.append(G * c)
        for c, e in ((mean.real, err[:, 0]), (mean.imag, err[:, 1])):
            parts.append(G * (G - 1) * e * e + G * c * c)
    return np.concatenate(parts)


def estimate_of(state, M):
    """Mean and standard error (Eq. 35-36) from summed state."""
    G = state[14]
    o, out = shard.STATE_HEADER, {}
    for key, n in (("S2", M), ("S3", M * M), ("S4", M * M)):
        sr, si, qr, qi = (state[o + i * n:o + (i + 1) * n] for i in range(4))
        o += 4 * n
        mr, mi = sr / G, si / G
        er = np.sqrt(np.maximum(G / (G - 1) * (qr / G - mr * mr), 0) / G)
        ei = np.sqrt(np.maximum(G / (G - 1) * (qi / G - mi * mi), 0) / G)
        out[key] = mr + 1j * mi
        out[key + "_err"] = np.stack([er, ei], -1)
    return out


def _rank(rank, world, port, n, bad_rank, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        z = synth.ar1_quadratic(n, seed=5)
        a, b = shard.group_ranges(n, T, M_FRAMES, world)[rank]
        ref = oracle.polyspectra(z[a:b], T, DT, M_FRAMES)
        st = torch.from_numpy(state_of(ref, T, M_FRAMES, b - a))
        if rank == bad_rank:
            st[1] = 2 * T  # a plan with another frame length
        try:
            shard.reduce_state(st)
        except ValueError as e:
            q.put((rank, "mismatch", str(e)))
            return
        full = oracle.polyspectra(z, T, DT, M_FRAMES)
        est = estimate_of(st.numpy(), T // 2 + 1)
        errs = {k: float(np.max(np.abs(est[k].reshape(full[k].shape) - full[k]))
                         / np.max(np.abs(full[k])))
                for k in ("S2", "S3", "S4", "S2_err", "S3_err", "S4_err")}
        q.put((rank, int(st[14].item()), errs))
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, n, bad_rank=-1):
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, bad_rank, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(res)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_states_reduce_to_the_whole_record(world):
    n = 7 * M_FRAMES * T + 13  # 7 whole groups and a partial one that nobody owns
    for rank, groups, errs in _run(world, n):
        assert groups == 7
        for key, e in errs.items():
            assert e <= 1e-9, f"rank {rank}: {key} differs by {e:.2e}"


def test_mismatched_plans_are_refused_on_every_rank():
    res = _run(2, 6 * M_FRAMES * T, bad_rank=1)
    assert [r[1] for r in res] == ["mismatch", "mismatch"]


@pytest.mark.parametrize("n,world", [(0, 2), (5 * 60, 1), (7 * 60 + 59, 2), (10 * 60, 3),
                                     (2 * 60, 4), (1000 * 60 + 7, 7)])
def test_group_ranges_cover_every_whole_group_once(n, world):
    span = 60
    r = shard.group_ranges(n, 6, 10, world)
    assert len(r) == world
    assert r[0][0] == 0 and r[-1][1] == (n // span) * span
    for (a, b), (c, d) in zip(r[:-1], r[1:]):
        assert b == c
    sizes = [(b - a) // span for a, b in r]
    assert all((b - a) % span == 0 for a, b in r)
    assert max(sizes) - min(sizes) <= 1
    assert sorted(sizes, reverse=True) == sizes
