"""Sequential model of the table's placement rules (no GPU): buckets of S
slots with linear bucket probing, a preferred slot per key, the two claim
protocols, the two erase rules and rebuilds, driven by random operations
against a plain dict.

It checks the argument the preferred-slot claim rests on.  While the map is
flagged preferred-placed, every present key's preferred slot is occupied, so
a blind CAS that finds that slot EMPTY proves the key absent.  It also checks
the probe-chain invariant that lets lookups stop at a bucket holding an
EMPTY slot.  The CUDA kernels are checked against the oracle by the GPU
tests; this pins the placement reasoning on its own."""
import random

import pytest

EMPTY, TOMB = "E", "T"


class ModelTable:
    def __init__(self, n_buckets, S):
        self.nb, self.S = n_buckets, S
        self.slots = [EMPTY] * (n_buckets * S)
        self.pref_placed = True

    # key -> home bucket and preferred slot, from two fixed multiplicative
    # hashes (deterministic across processes)
    def home(self, k):
        return ((k * 2654435761 + 97) % (1 << 32) >> 8) % self.nb

    def pref(self, k):
        return ((k * 2246822519 + 13) % (1 << 32) >> 5) % self.S

    def bucket(self, b):
        return range(b * self.S, (b + 1) * self.S)

    def find(self, k):
        b = self.home(k)
        for _ in range(self.nb):
            stop = False
            for i in self.bucket(b):
                if self.slots[i] == k:
                    return i
                stop |= self.slots[i] == EMPTY
            if stop:
                return None
            b = (b + 1) % self.nb
        return None

    def _full_protocol(self, k, pref_first):
        b = self.home(k)
        for probe in range(self.nb):
            sl = list(self.bucket(b))
            if any(self.slots[i] == k for i in sl):
                return False  # present
            empties = [i for i in sl if self.slots[i] == EMPTY]
            if empties:
                p = b * self.S + self.pref(k)
                i = p if (pref_first and probe == 0 and self.slots[p] == EMPTY) else empties[0]
                self.slots[i] = k
                return True
            b = (b + 1) % self.nb
        raise RuntimeError("table full")

    def insert_pref(self, k):
        """Preferred-slot claim: blind CAS of the preferred slot, then the
        full protocol, preferred-first.  Only valid while pref_placed."""
        assert self.pref_placed
        p = self.home(k) * self.S + self.pref(k)
        if self.slots[p] == EMPTY:
            self.slots[p] = k  # the CAS succeeded: k must have been absent
            return True
        if self.slots[p] == k:
            return False
        return self._full_protocol(k, pref_first=True)

    def insert_bucket(self, k):
        """Bucket-first claim in slot order; gives up the invariant."""
        self.pref_placed = False
        return self._full_protocol(k, pref_first=False)

    def erase(self, k):
        i = self.find(k)
        if i is None:
            return False
        b = i // self.S
        sl = list(self.bucket(b))
        self.slots[i] = "M"  # marked while it resolves
        to_empty = any(self.slots[j] == EMPTY for j in sl)
        if self.pref_placed:
            own = i % self.S
            to_empty &= not any(self.slots[j] not in (EMPTY, TOMB, "M") and self.pref(self.slots[j]) == own
                                for j in sl)
        self.slots[i] = EMPTY if to_empty else TOMB
        return True

    def rebuild(self):
        keys = [x for x in self.slots if x not in (EMPTY, TOMB)]
        self.slots = [EMPTY] * len(self.slots)
        self.pref_placed = True
        for k in keys:
            p = self.home(k) * self.S + self.pref(k)
            if self.slots[p] == EMPTY:
                self.slots[p] = k
            else:
                self._full_protocol(k, pref_first=True)

    def check(self, live):
        present = [x for x in self.slots if x not in (EMPTY, TOMB)]
        assert len(present) == len(set(present)), "a key is stored twice"
        assert set(present) == live
        for k in live:
            assert self.find(k) is not None, "probe chain broken"
        if self.pref_placed:
            for k in live:
                p = self.home(k) * self.S + self.pref(k)
                assert self.slots[p] != EMPTY, "preferred-slot invariant broken"


@pytest.mark.parametrize("S", [4, 8])
@pytest.mark.parametrize("seed", range(6))
def test_placement_rules_keep_both_invariants(S, seed):
    rnd = random.Random(seed * 31 + S)
    t = ModelTable(n_buckets=24, S=S)
    live = set()
    universe = list(range(int(24 * S * 0.8)))
    for step in range(3000):
        r = rnd.random()
        k = rnd.choice(universe)
        used = sum(x != EMPTY for x in t.slots)
        if used > 0.9 * len(t.slots):
            t.rebuild()
        elif r < 0.45:
            if len(live) < 0.75 * len(t.slots):
                if t.pref_placed and rnd.random() < 0.85:
                    added = t.insert_pref(k)
                else:
                    added = t.insert_bucket(k)
                assert added == (k not in live)
                live.add(k)
        elif r < 0.8:
            assert t.erase(k) == (k in live)
            live.discard(k)
        elif r < 0.97:
            assert (t.find(k) is not None) == (k in live)
        else:
            t.rebuild()
        t.check(live)


def test_plain_erase_rule_would_break_the_invariant():
    """Without the extra tombstone rule, emptying a slot that another live
    key prefers lets a later blind CAS store that key twice: the rule is
    needed.  The case is built by hand."""
    t = ModelTable(n_buckets=1, S=4)
    # find two keys with the same preferred slot
    by_pref = {}
    for k in range(1000):
        by_pref.setdefault(t.pref(k), []).append(k)
    a, b = next(v[:2] for v in by_pref.values() if len(v) >= 2)
    assert t.insert_pref(a)
    assert t.insert_pref(b)  # a holds the preferred slot: b goes elsewhere
    t.check({a, b})
    # plain rule: the bucket has an EMPTY slot, so a's slot would go EMPTY
    i = t.find(a)
    t.slots[i] = EMPTY
    p = t.pref(b)
    assert t.slots[p] == EMPTY and t.find(b) is not None
    with pytest.raises(AssertionError, match="stored twice"):
        t.insert_pref(b)  # the blind CAS finds EMPTY and stores b again
        t.check({b})
