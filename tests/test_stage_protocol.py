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

The second model is the accumulator drain handshake between the MMA warp and the epilogue warps (two column halves,
per-tile drain intervals, four or eight epilogue warps); its negative controls are an acc_empty barrier counting one
arrival, a wait on the wrong parity, and an epilogue that derives its chunks from another drain interval.
The third is the tile ring through which the loader hands tile ids to the other roles.
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


# ---------------------------------------------------------------------------
# The accumulator drain handshake between the MMA warp and the epilogue warps.
#
# The accumulator is used as two column halves h (one when the tile is narrow).
# Per drain chunk of a tile, the MMA warp, for each half in order, waits on
# acc_empty[h] with parity (g_h & 1) ^ 1 before the chunk's first MMAs into it,
# and after the chunk's last MMAs into it commits acc_full[h] (the commit
# arrives once those MMAs have completed, in issue order); the stages between
# write both halves.  Every epilogue warp, per chunk and half, waits on
# acc_full[h] with parity g_h & 1, reads the half, and arrives on acc_empty[h]
# (count: the number of epilogue warps).  The drain interval of a tile is
# chunk_stages, or chunk_stages_b for tiles without meson rows; both sides
# must derive the same chunk count from it.


def drain_programs(tiles, chunk, chunk_b, epi_chunk_b=None):
    """MMA and epilogue op lists for a tile sequence [(nst, meson, nh)]."""
    mma, epi = [], []
    for t, (nst, meson, nh) in enumerate(tiles):
        cs = chunk if meson else chunk_b
        ce = chunk if meson else (chunk_b if epi_chunk_b is None else epi_chunk_b)
        n_ch = -(-nst // cs)
        for ch in range(n_ch):
            n_in = min(cs, nst - ch * cs)       # stages of this chunk
            for h in range(nh):
                mma.append(("wait_empty", h))
                mma.append(("write", h, (t, ch)))
                if n_in == 1:
                    mma.append(("commit", h, (t, ch)))
            if n_in > 2:
                mma.append(("write_both", nh, (t, ch)))
            if n_in > 1:
                for h in range(nh):
                    mma.append(("write", h, (t, ch)))
                    mma.append(("commit", h, (t, ch)))
        for ch in range(-(-nst // ce)):
            for h in range(nh):
                epi.append(("wait_full", h, (t, ch)))
                epi.append(("arrive", h, (t, ch)))
    return mma, epi


def simulate_drain(tiles, epi_warps, chunk, chunk_b, seed, empty_count=None, mma_parity_flip=False,
                   epi_chunk_b=None):
    rng = random.Random(seed)
    acc_full = [Bar(1), Bar(1)]
    acc_empty = [Bar(empty_count or epi_warps) for _ in range(2)]
    mma_ops, epi_ops = drain_programs(tiles, chunk, chunk_b, epi_chunk_b)
    owner = [None, None]            # chunk whose sums are in the half
    committed = [None, None]        # chunk whose MMAs into the half have completed
    drained = [{}, {}]              # chunk -> epilogue warps that have read and released it
    pending = []                    # commits issued, not yet arrived (they arrive in order)
    g_mma = [0, 0]
    pc_mma = 0
    warps = [{"pc": 0, "g": [0, 0]} for _ in range(epi_warps)]
    for _ in range(200000):
        if pc_mma == len(mma_ops) and not pending and all(w["pc"] == len(epi_ops) for w in warps):
            return
        acts = []
        if pc_mma < len(mma_ops):
            op = mma_ops[pc_mma]
            if op[0] != "wait_empty":
                acts.append(("mma",))
            else:
                h = op[1]
                par = (g_mma[h] & 1) ^ (0 if mma_parity_flip else 1)
                if acc_empty[h].try_wait(par):
                    acts.append(("mma",))
        if pending:
            acts.append(("arrive_commit",))
        for i, w in enumerate(warps):
            if w["pc"] == len(epi_ops):
                continue
            op = epi_ops[w["pc"]]
            if op[0] == "arrive" or acc_full[op[1]].try_wait(w["g"][op[1]] & 1):
                acts.append(("epi", i))
        assert acts, "deadlock"
        act = rng.choice(acts)
        if act[0] == "mma":
            op = mma_ops[pc_mma]
            pc_mma += 1
            if op[0] == "wait_empty":
                h = op[1]
                prev = owner[h]
                if prev is not None:
                    assert len(drained[h].get(prev, ())) == epi_warps, \
                        f"half {h}: chunk {prev} overwritten before every epilogue warp drained it"
            elif op[0] == "write":
                h, cid = op[1], op[2]
                assert owner[h] in (None, cid) or len(drained[h].get(owner[h], ())) == epi_warps, \
                    f"half {h} written while chunk {owner[h]} is undrained"
                owner[h] = cid
                committed[h] = None
            elif op[0] == "write_both":
                for h in range(op[1]):
                    assert owner[h] == op[2], f"middle stage of chunk {op[2]} without the half {h}"
            else:
                h, cid = op[1], op[2]
                pending.append((h, cid))
                g_mma[h] += 1
        elif act[0] == "arrive_commit":
            h, cid = pending.pop(0)
            committed[h] = cid
            acc_full[h].arrive()
        else:
            w = warps[act[1]]
            op = epi_ops[w["pc"]]
            w["pc"] += 1
            h, cid = op[1], op[2]
            if op[0] == "wait_full":
                assert owner[h] == cid and committed[h] == cid, \
                    f"epilogue read half {h} for chunk {cid}, but it holds {owner[h]} (completed: {committed[h]})"
            else:
                drained[h].setdefault(cid, set()).add(act[1])
                w["g"][h] += 1
                acc_empty[h].arrive()
    raise AssertionError("no progress")


def random_tiles(rng, n):
    # (K stages, has meson rows, column halves)
    return [(rng.randint(1, 40), rng.random() < 0.3, rng.choice([1, 2, 2])) for _ in range(n)]


@pytest.mark.parametrize("epi_warps", [4, 8])
@pytest.mark.parametrize("chunk,chunk_b", [(16, 16), (16, 24), (8, 16), (1, 1), (3, 2)])
def test_drain_handshake(epi_warps, chunk, chunk_b):
    for seed in range(60):
        rng = random.Random(1000 + seed)
        simulate_drain(random_tiles(rng, 6), epi_warps, chunk, chunk_b, seed)


def _fails(**kw):
    failures = 0
    for seed in range(60):
        rng = random.Random(2000 + seed)
        try:
            simulate_drain(random_tiles(rng, 6), 8, 16, 24, seed, **kw)
        except AssertionError:
            failures += 1
    return failures


def test_negative_control_acc_empty_counting_one_warp():
    """acc_empty expecting one arrival instead of one per epilogue warp: the MMAs overwrite a half that other
    epilogue warps have not drained yet."""
    assert _fails(empty_count=1) > 0


def test_negative_control_mma_waits_on_the_wrong_parity():
    assert _fails(mma_parity_flip=True) == 60


def test_negative_control_epilogue_with_another_drain_interval():
    """The epilogue deriving its chunk count from chunk_stages where the MMA used chunk_stages_b (tiles without
    meson rows): the two sides disagree on the chunks and the handshake breaks."""
    assert _fails(epi_chunk_b=16) > 0


# ---------------------------------------------------------------------------
# The tile ring: the loader claims tile ids from the global counter and
# publishes them through TRING shared slots; every reader warp (A producers,
# epilogue, MMA) takes every entry in order and frees it at once.  The loader
# waits on tempty[slot] with parity (round & 1) ^ 1, writes the id, arrives on
# tfull[slot]; a reader waits on tfull[slot] with parity round & 1, reads,
# arrives on tempty[slot] (count: the number of readers).  The last entry is
# -1, after which every role stops.


def simulate_tile_ring(n_tiles, n_readers, ring, seed, empty_count=None):
    rng = random.Random(seed)
    tfull = [Bar(1) for _ in range(ring)]
    tempty = [Bar(empty_count or n_readers) for _ in range(ring)]
    slot_val = [None] * ring
    loader = {"k": 0, "done": False}
    readers = [{"k": 0, "seen": [], "done": False} for _ in range(n_readers)]
    for _ in range(100000):
        if loader["done"] and all(r["done"] for r in readers):
            for r in readers:
                assert r["seen"] == list(range(n_tiles)), "a reader saw tiles out of order or lost one"
            return
        acts = []
        k = loader["k"]
        if not loader["done"] and tempty[k % ring].try_wait(((k // ring) & 1) ^ 1):
            acts.append(("load",))
        for i, r in enumerate(readers):
            k = r["k"]
            if not r["done"] and tfull[k % ring].try_wait((k // ring) & 1):
                acts.append(("read", i))
        assert acts, "deadlock"
        act = rng.choice(acts)
        if act[0] == "load":
            k = loader["k"]
            slot_val[k % ring] = k if k < n_tiles else -1
            tfull[k % ring].arrive()
            loader["k"] += 1
            loader["done"] = k >= n_tiles
        else:
            r = readers[act[1]]
            k = r["k"]
            v = slot_val[k % ring]
            assert v == (k if k < n_tiles else -1), f"reader {act[1]} took entry {k} but read tile {v}"
            tempty[k % ring].arrive()
            r["k"] += 1
            if v < 0:
                r["done"] = True
            else:
                r["seen"].append(v)
    raise AssertionError("no progress")


@pytest.mark.parametrize("n_readers", [21, 25])   # 16 A producers + 4 or 8 epilogue warps + the MMA warp
def test_tile_ring(n_readers):
    for seed in range(40):
        simulate_tile_ring(13, n_readers, 4, seed)


def test_negative_control_tile_ring_freed_by_fewer_readers():
    failures = 0
    for seed in range(40):
        try:
            simulate_tile_ring(13, 21, 4, seed, empty_count=20)
        except AssertionError:
            failures += 1
    assert failures > 0
