"""Event-by-event ensembles across ranks (one process per GPU).

Events are independent grids, so an ensemble shards with no data-path
collective: events are assigned to ranks by longest-processing-time on their
cell counts, each rank advances its share with one ``HydroBatch`` (one
persistent launch per RK3 stage over all its events), and only per-event
observables are gathered on the host with ``torch.distributed``.

Failures are handled on the host: a rank whose shard raises reports the error
in the gather instead of results, and its events are reassigned to the ranks
that succeeded in a further round.  A rank that never reaches the gather is
caught by the process group's own timeout.
"""
import numpy as np


def lpt_shards(costs, ranks):
    """Assign items (by cost) to the given ranks, largest first, each to the
    currently least-loaded rank.  Returns {rank: [item indices]}."""
    load = {r: 0 for r in ranks}
    out = {r: [] for r in ranks}
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        r = min(ranks, key=lambda r: (load[r], r))
        out[r].append(i)
        load[r] += costs[i]
    return out


def gpu_shard_runner(grids, make_primitive, nsteps, stream=None):
    """Default shard runner: one HydroBatch over the shard's events on this
    rank's GPU.  Returns {event: (t, steps, total E)} (the sum is a host-side
    reduction of the returned state)."""
    def run(events):
        if not events:
            return {}
        from ._binding import HydroBatch
        with HydroBatch([grids[e] for e in events], stream=stream) as b:
            for i, e in enumerate(events):
                b.set_primitive(i, make_primitive(e))
            b.step(nsteps)
            out = {}
            for i, e in enumerate(events):
                u, t, k = b.get_state(i)
                out[e] = (t, k, float(np.sum(u[0])))
        return out
    return run


def run_ensemble(costs, run_shard, rank, world, dist=None, max_rounds=3):
    """Run an ensemble of len(costs) events over `world` ranks.

    run_shard(list_of_events) -> {event: observable} runs on this rank.
    dist: torch.distributed (initialised) or None for a single process.
    Returns (results {event: observable}, failures [(round, rank, message)]).
    """
    pending = list(range(len(costs)))
    ranks = list(range(world))
    results, failures = {}, []
    for rnd in range(max_rounds):
        shards = lpt_shards([costs[e] for e in pending], ranks)
        mine = [pending[i] for i in shards.get(rank, [])]
        try:
            out, err = run_shard(mine), None
        except Exception as exc:            # reported to every rank below
            out, err = {}, "%s: %s" % (type(exc).__name__, exc)
        if dist is not None and world > 1:
            gathered = [None] * world
            dist.all_gather_object(gathered, (rank, out, err))
        else:
            gathered = [(rank, out, err)]
        for r, o, e in gathered:
            results.update(o)
            if e is not None:
                failures.append((rnd, r, e))
        pending = [e for e in pending if e not in results]
        ranks = [r for r, _, e in gathered if e is None]
        if not pending or not ranks:
            break
    return results, failures
