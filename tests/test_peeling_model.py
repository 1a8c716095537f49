"""A host-side model of the per-pixel ordering rule of the render traversal
(release by key, bounded queue, depth peeling) against the plain sort.

Contributors of one pixel arrive in pair order with non-decreasing keys, each
key a lower bound of the depth t* of every later contributor.  The model
follows the kernel's rules: release queued entries that nothing later can
precede, queue the rest in (t*, arrival) order, defer the farther of a new
entry and the queue's last one when the queue is full (a pass blends only
lo <= t* < hi), close a pass once a key reaches hi, and restart the next pass
at the pair that last filled the empty queue before the first deferral.  The
blend sequence must be the (t*, arrival) order for any queue size, and the
restart point must never skip a contributor that a later pass needs.
"""
import numpy as np
import pytest

INF = float("inf")


def peel(keys, ts, cap, stop_after=None):
    """Blend order (arrival indices) produced by the rules above; ts[j] is the
    contributor's depth or nan when pair j does not contribute to the pixel."""
    n = len(keys)
    lnext = np.append(keys[1:], INF)
    out = []
    lo, jfirst, passes = -INF, 0, 0
    while True:
        passes += 1
        hi, q, jnext, jfill = INF, [], None, 0
        for j in range(jfirst, n):
            if hi < INF and keys[j] >= hi:
                break                                   # pass closed
            t = ts[j]
            if np.isnan(t) or t < lo or t >= hi:
                continue
            while q and q[0][0] <= t and q[0][0] < lnext[j]:
                out.append(q.pop(0)[1])
            if t < lnext[j]:
                out.append(j)
                while q and q[0][0] < lnext[j]:
                    out.append(q.pop(0)[1])
                continue
            insert = True
            if len(q) == cap:
                if q[0][0] > lo:
                    if jnext is None:
                        jnext = jfill
                    hi = max(t, q[-1][0])
                    q = [e for e in q if e[0] < hi]
                    insert = t < hi
                else:
                    out.append(q.pop(0)[1])
            if insert:
                if not q:
                    jfill = j
                i = len(q)
                while i > 0 and q[i - 1][0] > t:
                    i -= 1
                q.insert(i, (t, j))
        out.extend(e[1] for e in q)
        if hi == INF or (stop_after is not None and len(out) >= stop_after):
            return out, passes
        lo, jfirst = hi, jnext


def random_pixel(rng, n, spread, ties=False):
    """Pairs with sorted keys; a contributor's t* lies at or beyond its key,
    up to `spread` further; some pairs do not contribute."""
    keys = np.sort(rng.uniform(0.0, 10.0, n))
    ts = keys + rng.exponential(spread, n)
    if ties:
        ts = np.round(ts, 1)
        ts = np.maximum(ts, keys)
    ts[rng.random(n) < 0.3] = np.nan
    return keys, ts


@pytest.mark.parametrize("cap", [1, 2, 3, 16])
@pytest.mark.parametrize("ties", [False, True])
def test_peeling_gives_the_exact_order(cap, ties):
    rng = np.random.default_rng(cap * 7 + ties)
    worst_passes = 0
    for trial in range(60):
        keys, ts = random_pixel(rng, int(rng.integers(1, 300)), float(rng.choice([0.05, 0.5, 3.0])), ties)
        got, passes = peel(keys, ts, cap)
        j = np.nonzero(~np.isnan(ts))[0]
        exact = j[np.lexsort((j, ts[j]))]
        assert got == list(exact), (trial, cap)
        worst_passes = max(worst_passes, passes)
    if cap <= 3:
        assert worst_passes > 3          # the deferral path was exercised


def test_keys_equal_to_depths_blend_in_one_pass():
    # every contributor at its own key: each is blended on arrival
    rng = np.random.default_rng(3)
    keys = np.sort(rng.uniform(0, 5, 200))
    got, passes = peel(keys, keys.copy(), 1)
    assert got == list(range(200)) and passes == 1
