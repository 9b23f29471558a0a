"""Reference rule for k-NN object-pair pruning (Algorithm 6, section 3.4) --
TEST INFRASTRUCTURE, plain Python loops.

Algorithm 6 as printed counts ``closer``/``farther`` with non-strict
comparisons and compares ``N - farther`` against ``kLeft`` with ``N`` the
number of all candidates of r.  Two readings are taken here so that the
statuses are correct and ties resolve:

* ``n`` *precedes* ``m`` iff ``(ub_n, id_n) < (lb_m, id_m)`` lexicographically
  (then ``d_n <= d_m`` and, on equality, the id decides).
* with ``U`` the undecided candidates of r and ``kLeft = k - #confirmed``:
  ``m`` is REMOVED iff at least ``kLeft`` members of ``U`` precede it;
  ``m`` is CONFIRMED iff fewer than ``kLeft`` members of ``U \\ {m}`` are not
  preceded by ``m``.

All decisions of one round are taken against the statuses at its start.
"""
from __future__ import annotations

UNDECIDED, CONFIRMED, REMOVED = 0, 1, 2


def precedes(lb_n, ub_n, id_n, lb_m, ub_m, id_m) -> bool:
    return (ub_n, id_n) < (lb_m, id_m)


def prune_round(k: int, ids, lb, ub, status):
    """One pruning round over the candidates of a single query object.

    ``ids``, ``lb``, ``ub``, ``status`` are equal-length sequences; returns the
    new status list."""
    n = len(ids)
    confirmed = sum(1 for s in status if s == CONFIRMED)
    k_left = k - confirmed
    U = [i for i in range(n) if status[i] == UNDECIDED]
    new = list(status)
    for m in U:
        if k_left <= 0:
            new[m] = REMOVED
            continue
        before = 0
        maybe_before = 0
        for j in U:
            if j == m:
                continue
            if precedes(lb[j], ub[j], ids[j], lb[m], ub[m], ids[m]):
                before += 1
            if not precedes(lb[m], ub[m], ids[m], lb[j], ub[j], ids[j]):
                maybe_before += 1
        if before >= k_left:
            new[m] = REMOVED
        elif maybe_before < k_left:
            new[m] = CONFIRMED
    return new
