"""Sharding of SIGW work across ranks (one process per GPU).

Units that need no exchange: realisations (seeds) and parameter points are independent, so ranks take
disjoint seeds and never communicate on the data path (weak scaling).  A single spectrum can also be split by
target shell (each shell costs the same FFT work): rank r takes shells r, r + world, ...; the per-shell results
(Omega, P_A, P_B, N_k) are then assembled with one all-reduce of N/2 x 4 doubles, the only collective.
"""


def shard(items, rank, world):
    """The items rank `rank` of `world` owns (round-robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return list(items)[rank::world]


def seeds_for_rank(base_seeds, rank, world):
    """Disjoint seeds for weak scaling: rank r uses base_seeds + r * 1_000_003 (no overlap for < 1e6 seeds)."""
    return [int(s) + 1_000_003 * rank for s in base_seeds]


def spectrum_by_shells(compute, shells, rank, world, group=None, device=None):
    """Split one spectrum by shells.

    compute(my_shells) -> dict with arrays "omega", "PA", "PB", "Nk" over my_shells (one realisation).
    Returns a (len(shells), 4) float64 tensor [omega, PA, PB, Nk] on every rank.
    """
    import torch
    import torch.distributed as dist
    shells = [int(s) for s in shells]
    mine = shard(shells, rank, world)
    buf = torch.zeros(len(shells), 4, dtype=torch.float64, device=device)
    if mine:
        res = compute(mine)
        pos = {s: i for i, s in enumerate(shells)}
        for j, s in enumerate(mine):
            buf[pos[s], 0] = float(res["omega"][j])
            buf[pos[s], 1] = float(res["PA"][j])
            buf[pos[s], 2] = float(res["PB"][j])
            buf[pos[s], 3] = float(res["Nk"][j])
    if world > 1:
        dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    return buf
