"""Dynamic task claims of the persistent step kernels (claim_tasks): a
model of the claim protocol run under random interleavings of the warps'
atomic claims. Whatever the
schedule, every task of [0, ntask) is run exactly once, for one counter and
for four stripes, ntask from 0 to a few hundred and warp counts above and
below the task count. The GPU tests check the kernels themselves (every
task order gives the same bits); this checks the protocol's termination and
coverage on schedules a GPU run does not choose."""
import random

import pytest


def stripe_bounds(ntask, ns, s):
    q, r = divmod(ntask, ns)
    start = s * q + min(s, r)
    return start, q + (1 if s < r else 0)


def warp(w, ntask, ns, ctr, ran):
    """One warp's claims; yields before every atomic on a counter so that the
    scheduler can interleave the warps there."""
    def stripe(k):
        return (w + k) % ns

    k = 0
    yield
    t = ctr[stripe(0)]
    ctr[stripe(0)] += 1
    while True:
        start, size = stripe_bounds(ntask, ns, stripe(k))
        if t >= size:
            k += 1
            if k == ns:
                return
            yield
            t = ctr[stripe(k)]
            ctr[stripe(k)] += 1
            continue
        task = start + t
        yield
        u = ctr[stripe(k)]  # the next claim, ahead of the run
        ctr[stripe(k)] += 1
        ran.append(task)
        t = u


@pytest.mark.parametrize("ns", [1, 4])
def test_every_task_runs_exactly_once_under_random_schedules(ns):
    rng = random.Random(7)
    for trial in range(300):
        ntask = rng.choice([0, 1, 2, 3, 5, 17, 64, 131, 400])
        nwarps = rng.choice([1, 2, 3, 8, 33, 128])
        ctr = [0] * ns
        ran = []
        live = [warp(w, ntask, ns, ctr, ran) for w in range(nwarps)]
        steps = 0
        while live:
            g = rng.choice(live)
            try:
                next(g)
            except StopIteration:
                live.remove(g)
            steps += 1
            assert steps < 100000, "a warp did not terminate"
        assert sorted(ran) == list(range(ntask)), (trial, ntask, nwarps)


def test_stripes_partition_the_tasks():
    for ntask in range(0, 50):
        for ns in (1, 2, 4, 8):
            covered = []
            for s in range(ns):
                start, size = stripe_bounds(ntask, ns, s)
                covered.extend(range(start, start + size))
            assert covered == list(range(ntask))
