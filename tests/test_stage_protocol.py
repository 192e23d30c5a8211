"""Host model of the contraction kernel's stage protocol, with exact mbarrier parity semantics.

Actors, as in the tensor-core kernel:
- the loader: copies stage k into stage buffer k mod NS once stage k - NS has completed (empty barrier k mod NS);
- two A-producer groups, group g forming the stages of parity g: each waits for its stage's data, reads the
  buffer, waits for the completion of stage G - 2 (the previous user of its A slot) and arrives on the A slot;
- the MMA issuer: waits for the A slot only, completes stages in order and commits the stage's empty barrier.

An mbarrier parity wait passes when the barrier's current phase parity differs from the requested one, so it
is exact only when the waiter is at most one phase away.  Random schedules (copies land in any order) check
that every producer reads exactly its stage's landed data, that no copy starts into a buffer that is still
read or still being filled, that no barrier phase receives more arrivals than it expects and that nothing
deadlocks, for ring depths 2..6.  The data barriers are indexed by stage modulo 2 NS, so each serves one
producer group; indexing them by buffer (stage modulo NS) breaks for odd NS, which the negative control shows.
"""
import random

import pytest


class Bar:
    def __init__(self, count):
        self.count, self.pending, self.phase, self.tx = count, count, 0, 0

    def arrive(self, tx=0):
        assert self.pending > 0, "more arrivals than the phase expects"
        self.pending -= 1
        self.tx += tx
        self._maybe()

    def complete_tx(self, n):
        self.tx -= n
        assert self.tx >= 0
        self._maybe()

    def _maybe(self):
        if self.pending == 0 and self.tx == 0:
            self.phase += 1
            self.pending = self.count

    def try_wait(self, parity):
        return (self.phase & 1) != parity


def simulate(NS, n_stages, seed, data_barriers):
    rng = random.Random(seed)
    NF = data_barriers
    full = [Bar(1) for _ in range(NF)]
    empty = [Bar(1) for _ in range(NS)]
    a_full = [Bar(1), Bar(1)]
    content = [None] * NS          # stage whose data a buffer holds (None while being filled)
    filling = {}                   # buffer -> stage being copied into it
    in_use = set()                 # (buffer, stage) still read by a producer or by the MMAs
    copies = []
    k = 0
    prod = [{"G": g, "waiting": "data"} for g in range(2)]
    mma_next, mma_queue, completed = 0, [], -1
    for _ in range(400000):
        if completed == n_stages - 1:
            return
        acts = []
        if k < n_stages and empty[k % NS].try_wait(((k // NS) & 1) ^ 1):
            acts.append(("load",))
        if copies:
            acts.append(("land",))
        for g, p in enumerate(prod):
            G = p["G"]
            if G >= n_stages:
                continue
            if p["waiting"] == "data" and full[G % NF].try_wait((G // NF) & 1):
                acts.append(("data", g))
            if p["waiting"] == "slot" and (G < 2 or empty[(G - 2) % NS].try_wait(((G - 2) // NS) & 1)):
                acts.append(("slot", g))
        if mma_next < n_stages and a_full[mma_next & 1].try_wait((mma_next >> 1) & 1):
            acts.append(("issue",))
        if mma_queue:
            acts.append(("complete",))
        assert acts, f"deadlock at stage {completed + 1}"
        act = rng.choice(acts)
        if act[0] == "load":
            s = k % NS
            assert s not in filling, "copy into a buffer that is still being filled"
            assert all(b != s for (b, _) in in_use), "copy into a buffer that is still read"
            full[k % NF].arrive(tx=1)
            filling[s] = k
            content[s] = None
            copies.append((s, k))
            k += 1
        elif act[0] == "land":
            s, st = copies.pop(rng.randrange(len(copies)))
            content[s] = st
            del filling[s]
            full[st % NF].complete_tx(1)
        elif act[0] == "issue":
            mma_queue.append(mma_next)
            mma_next += 1
        elif act[0] == "complete":
            G = mma_queue.pop(0)
            in_use.discard((G % NS, G))
            completed = G
            empty[G % NS].arrive()
        else:
            p = prod[act[1]]
            G = p["G"]
            if act[0] == "data":
                assert content[G % NS] == G, f"producer read stage {content[G % NS]} for stage {G}"
                in_use.add((G % NS, G))
                p["waiting"] = "slot"
            else:
                a_full[G & 1].arrive()
                p["G"] += 2
                p["waiting"] = "data"
    raise AssertionError("no progress")


@pytest.mark.parametrize("NS", [2, 3, 4, 5, 6])
def test_stage_protocol_with_data_barriers_modulo_2ns(NS):
    for seed in range(150):
        simulate(NS, 36, seed, data_barriers=2 * NS)


def test_negative_control_data_barriers_per_buffer_break_for_odd_depth():
    failures = 0
    for seed in range(150):
        try:
            simulate(3, 36, seed, data_barriers=3)
        except AssertionError:
            failures += 1
    assert failures > 0
