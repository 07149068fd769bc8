"""Model check of the hand-off protocol of the causal substitution (value-polling form).

The kernel runs one CTA per interface, all resident.  In CTA k, warp 0 at time step n
polls (until they are set) the partial right-hand sides P_n(i) of the interfaces i
within H and x_{n-1} of their sources (interfaces i-1, i, i+1); it then computes and
publishes x_n(k), forms P_{n+1}(k) from the history sums of step n+1 and publishes it,
and at the end of the step releases the consumed history slot and its own x_n.  Every
published value is written once into an array preset to "unset".  Four history warps
per CTA form the sums of the lags > LA of step m + LA from the values s <= m - 1 of
their source (the CTA's own x, or a neighbour's, polled), and hand them over in a ring
of LA + 1 slots: a warp refills a slot only when warp 0 has consumed the step it held
(s_hused >= m - 1), and warp 0 reads step t only when the warp has filled it
(s_hdone >= t).

This test runs that protocol as a state machine under many random interleavings (every
wait, read and write a separate event) and checks that warp 0 always reads the step it
needs from the ring, that no slot is refilled before it was consumed, that every value
read is set, and that the system never deadlocks.  It models the design, not the CUDA
code, and needs no GPU."""
import random

import pytest


class Violation(AssertionError):
    pass


def _run(K, H, nt, rng, LA=3, slots=None, hused_lag=1, owner_waits=True):
    """One random schedule.  The planted-mistake knobs: `slots` (ring size, LA + 1 in the
    kernel), `hused_lag` (a history warp at iteration m waits for s_hused >= m -
    hused_lag; 1 in the kernel), `owner_waits` (warp 0 waits for s_hdone)."""
    slots = LA + 1 if slots is None else slots
    x_set = [[False] * nt for _ in range(K)]
    p_set = [[False] * nt for _ in range(K)]
    # per CTA: the ring (slot -> step it holds), the CTA flags
    ring = [[[t if t < slots else None for t in range(slots)] for _ in range(4)]
            for _ in range(K)]
    s_xown = [0] * K
    s_hused = [0] * K
    s_hdone = [[LA] * 4 for _ in range(K)]
    actors = []
    for k in range(K):
        actors.append({"kind": "owner", "k": k, "n": 0, "phase": "init"})
        for e in range(4):
            actors.append({"kind": "hist", "k": k, "e": e, "m": 1, "phase": "wait_hused"})

    def sources(i):
        """(interface, exists) of the four sources of interface i: own blocks for e = 0, 2,
        the right neighbour's for e = 1, the left's for e = 3."""
        return [(i, True), (i + 1, i + 1 <= K - 1), (i, True), (i - 1, i >= 1)]

    def hist_done(a):
        return a["m"] + LA >= nt

    while True:
        live = [a for a in actors if a["phase"] != "done"]
        if not live:
            break
        enabled = []
        for a in live:
            k = a["k"]
            if a["kind"] == "owner":
                n = a["n"]
                if a["phase"] == "poll":
                    ok = True
                    for i in range(max(0, k - H), min(K, k + H + 1)):
                        if H > 0 and not p_set[i][n]:
                            ok = False
                        if n >= 1:
                            for j, ex in sources(i):
                                if ex and not x_set[j][n - 1]:
                                    ok = False
                    if ok:
                        enabled.append(a)
                elif a["phase"] == "hist":
                    if not owner_waits or all(s_hdone[k][e] >= n + 1 for e in range(4)):
                        enabled.append(a)
                else:
                    enabled.append(a)
            else:
                m, e = a["m"], a["e"]
                if a["phase"] == "wait_hused":
                    if s_hused[k] >= m - hused_lag:
                        enabled.append(a)
                elif a["phase"] == "wait_src":
                    j, ex = sources(k)[e]
                    if not ex:
                        enabled.append(a)
                    elif e in (0, 2):
                        if s_xown[k] >= m:
                            enabled.append(a)
                    elif x_set[j][m - 1]:
                        enabled.append(a)
                else:
                    enabled.append(a)
        if not enabled:
            raise Violation("deadlock")
        a = rng.choice(enabled)
        k = a["k"]
        if a["kind"] == "owner":
            n = a["n"]
            if a["phase"] == "init":
                if H > 0:
                    p_set[k][0] = True
                a["phase"] = "poll"
            elif a["phase"] == "poll":
                a["phase"] = "write_x"
            elif a["phase"] == "write_x":
                x_set[k][n] = True
                a["phase"] = "hist" if n + 1 < nt else "flags"
            elif a["phase"] == "hist":
                for e in range(4):
                    held = ring[k][e][(n + 1) % slots]
                    if held != n + 1:
                        raise Violation(f"CTA {k} step {n + 1} source {e}: the slot holds "
                                        f"step {held}")
                a["phase"] = "write_p"
            elif a["phase"] == "write_p":
                if H > 0:
                    p_set[k][n + 1] = True
                a["phase"] = "flags"
            elif a["phase"] == "flags":
                # the end of the step: consumed history and own x are released together
                if n + 1 < nt:
                    s_hused[k] = n + 1
                s_xown[k] = n + 1
                a["n"] = n + 1
                a["phase"] = "done" if n + 1 == nt else "poll"
        else:
            m, e = a["m"], a["e"]
            if a["phase"] == "wait_hused":
                if hist_done(a):
                    a["phase"] = "done"
                else:
                    a["phase"] = "wait_src"
            elif a["phase"] == "wait_src":
                j, ex = sources(k)[e]
                # the sum reads x_0 .. x_{m-1} of the source (a neighbour's: re-read until
                # every value is set, which the newest being set makes immediate here)
                if ex and not all(x_set[j][s] for s in range(m)):
                    raise Violation(f"CTA {k} source {e}: summed an unset value")
                a["phase"] = "write_slot"
            elif a["phase"] == "write_slot":
                slot = (m + LA) % slots
                held = ring[k][e][slot]
                if held is not None and held > s_hused[k]:
                    raise Violation(f"CTA {k} source {e}: step {m + LA} overwrote step {held} "
                                    "before warp 0 consumed it")
                ring[k][e][slot] = m + LA
                s_hdone[k][e] = m + LA
                a["m"] = m + 1
                a["phase"] = "done" if hist_done(a) else "wait_hused"
    assert all(all(row) for row in x_set)


@pytest.mark.parametrize("K,H", [(1, 0), (2, 0), (5, 0), (3, 1), (7, 2), (12, 3), (20, 8)])
def test_handoff_is_safe_under_random_interleavings(K, H):
    rng = random.Random(1000 * K + H)
    for _ in range(25):
        _run(K, H, nt=11, rng=rng)


@pytest.mark.parametrize("mistake", [{"slots": 3}, {"hused_lag": 2}, {"owner_waits": False}])
def test_model_catches_a_planted_mistake(mistake):
    """The check has teeth: a ring one slot short, a history warp that refills a slot one
    step early, or a warp 0 that reads the ring without waiting for it, is found by
    random schedules."""
    rng = random.Random(5)
    found = False
    for _ in range(400):
        try:
            _run(5, 1, nt=10, rng=rng, **mistake)
        except Violation:
            found = True
            break
    assert found, mistake
