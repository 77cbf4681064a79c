"""Host model of the fused backward + Adam kernel's hand-off between its two warp groups
(preprocess_bwd.cu, k_preprocess_bwd_adam): per CTA the gradient group fills buffer k % S for
its chunk k after waiting on empty[s] when k >= S, then arrives on full[s]; the Adam group
waits on full[s], takes the step, and arrives on empty[s] only when the buffer is reused
(chunk + S * grid < n_chunks). Checked: no deadlock, no barrier phase with two arrivals
before its wait, and every phase completed (none left half-arrived at exit), for many chunk
counts, grids and CTA indices."""
import random

import pytest

STAGES = 2   # kBAStages


def _events(n_chunks, grid, bid, S):
    chunks = list(range(bid, n_chunks, grid))
    prod, cons = [], []
    for k, c in enumerate(chunks):
        s = k % S
        if k >= S:
            prod.append(("empty", s, "sync"))
        prod.append(("full", s, "arrive"))
        cons.append(("full", s, "sync"))
        if c + S * grid < n_chunks:
            cons.append(("empty", s, "arrive"))
    return prod, cons


def _run(n_chunks, grid, bid, S):
    prod, cons = _events(n_chunks, grid, bid, S)
    arrived, synced = {}, {}
    pi = ci = 0
    while pi < len(prod) or ci < len(cons):
        moved = False
        for side in (0, 1):
            lst, i = (prod, pi) if side == 0 else (cons, ci)
            if i >= len(lst):
                continue
            name, s, op = lst[i]
            key = (name, s)
            if op == "arrive":
                arrived[key] = arrived.get(key, 0) + 1
                assert arrived[key] - synced.get(key, 0) <= 1, "two arrivals before a wait"
                ok = True
            else:
                ok = arrived.get(key, 0) > synced.get(key, 0)
                if ok:
                    synced[key] = synced.get(key, 0) + 1
            if ok:
                if side == 0:
                    pi += 1
                else:
                    ci += 1
                moved = True
        assert moved, ("deadlock", n_chunks, grid, bid, S)
    for key in set(arrived) | set(synced):
        assert arrived.get(key, 0) == synced.get(key, 0), ("phase left open", key)


@pytest.mark.parametrize("S", [STAGES, 3])
def test_hand_off_never_deadlocks_and_closes_every_phase(S):
    rng = random.Random(7)
    for _ in range(3000):
        grid = rng.randint(1, 40)
        _run(rng.randint(0, 300), grid, rng.randint(0, grid - 1), S)
    for n in range(0, 12):          # small cases exhaustively
        for grid in range(1, 6):
            for bid in range(grid):
                _run(n, grid, bid, S)
