"""Model check of the hand-off protocol of the window form of the causal substitution.

The kernel (one CTA per interface, all resident) runs, per time step n, at interface k:
wait until every interface within H+1 has published step n-1 (progress >= n+1); read the
partial right-hand sides P_n(k+d), |d| <= H, from ring slot n mod 2, and x_{n-1} of the
interfaces within H+1; then write P_{n+1}(k) into slot (n+1) mod 2, write x_n(k), and
publish progress = n+2.  The safety argument is that no interface overwrites a slot that
a neighbour has still to read, and that every read sees what the step needs.

This test runs that protocol as a state machine under many random interleavings (every
read and write a separate event) and checks both properties plus freedom from deadlock.
It models the design, not the CUDA code, and needs no GPU."""
import random

import pytest


class Violation(AssertionError):
    pass


def _run(K, H, nt, rng, radius=None):
    """One random schedule; `radius` is how far the wait reaches (the kernel: H + 1)."""
    radius = H + 1 if radius is None else radius
    slot_tag = [[None, None] for _ in range(K)]   # which P index each ring slot holds
    x_done = [[False] * nt for _ in range(K)]
    progress = [0] * K
    state = [{"n": 0, "phase": "init", "reads": []} for _ in range(K)]
    done = 0
    while done < K:
        enabled = []
        for k, st in enumerate(state):
            if st["phase"] == "done":
                continue
            if st["phase"] == "wait":
                n = st["n"]
                lo, hi = max(0, k - radius), min(K, k + radius + 1)
                if all(progress[j] >= n + 1 for j in range(lo, hi) if j != k):
                    enabled.append(k)
            else:
                enabled.append(k)
        if not enabled:
            raise Violation("deadlock")
        k = rng.choice(enabled)
        st = state[k]
        n = st["n"]
        if st["phase"] == "init":
            slot_tag[k][0] = 0
            progress[k] = 1
            st["phase"] = "wait"
        elif st["phase"] == "wait":
            reads = []
            for d in range(-H, H + 1):
                j = k + d
                if 0 <= j < K:
                    reads.append(("P", j))
                    if n >= 1:
                        reads += [("x", i) for i in (j - 1, j, j + 1) if 0 <= i < K]
            rng.shuffle(reads)
            st["reads"] = reads
            st["phase"] = "read"
        elif st["phase"] == "read":
            if st["reads"]:
                kind, j = st["reads"].pop()
                if kind == "P" and slot_tag[j][n % 2] != n:
                    raise Violation(f"interface {k} step {n} read a stale P of {j}")
                if kind == "x" and not x_done[j][n - 1]:
                    raise Violation(f"interface {k} step {n} read x of {j} before it was written")
            else:
                st["phase"] = "write_p"
        elif st["phase"] == "write_p":
            if n + 1 < nt:
                slot_tag[k][(n + 1) % 2] = n + 1
            st["phase"] = "write_x"
        elif st["phase"] == "write_x":
            x_done[k][n] = True
            st["phase"] = "publish"
        elif st["phase"] == "publish":
            progress[k] = n + 2
            st["n"] = n + 1
            if st["n"] == nt:
                st["phase"] = "done"
                done += 1
            else:
                st["phase"] = "wait"
    assert all(all(row) for row in x_done)


@pytest.mark.parametrize("K,H", [(1, 1), (3, 1), (7, 2), (12, 3), (20, 8)])
def test_window_handoff_is_safe_under_random_interleavings(K, H):
    rng = random.Random(1000 * K + H)
    for _ in range(40):
        _run(K, H, nt=9, rng=rng)


def test_model_catches_a_too_narrow_wait():
    """The check has teeth: waiting only for the interfaces within H (not H + 1) lets an
    interface read an x_{n-1} that is not written yet, or overwrite a slot that a
    neighbour still has to read; random schedules find it."""
    rng = random.Random(5)
    found = False
    for _ in range(400):
        try:
            _run(9, 2, nt=7, rng=rng, radius=2)
        except Violation:
            found = True
            break
    assert found
