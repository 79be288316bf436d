"""Brute-force reference for tiny inputs: a linear list scan, no hashing.

Independent of the oracle's dictionary: every lookup walks the whole entry
list.  Index bookkeeping follows the index heap as the paper states it
(Sec. 4.3: allocation reads h[t] and raises t; free lowers t and stores the
index at h[t]); rehash (Sec. 4.5) re-inserts active entries in ascending order
of their old index into fresh buffers of the new capacity.
"""


class BruteMap:
    def __init__(self, key_dim, capacity, row_bytes=(), auto_grow=True):
        self.key_dim = key_dim
        self.row_bytes = list(row_bytes)
        self.auto_grow = auto_grow
        self._reset(capacity)

    def _reset(self, capacity):
        self.capacity = capacity
        self.entries = []                      # [key tuple, buffer index]
        self.heap = list(range(capacity))
        self.top = 0
        self.kb = [tuple([0] * self.key_dim) for _ in range(capacity)]
        self.vb = [[bytes(rb) for _ in range(capacity)] for rb in self.row_bytes]

    def _lookup(self, key):
        for k, i in self.entries:
            if k == key:
                return i
        return None

    def _alloc(self):
        i = self.heap[self.top]
        self.top += 1
        return i

    def _free(self, i):
        self.top -= 1
        self.heap[self.top] = i

    def rehash(self, new_capacity=0):
        if new_capacity <= 0:
            new_capacity = 2 * self.capacity
        assert new_capacity >= len(self.entries)
        old = sorted(self.entries, key=lambda e: e[1])
        old_vals = [[self.vb[j][i] for _, i in old] for j in range(len(self.row_bytes))]
        self._reset(new_capacity)
        for r, (k, _) in enumerate(old):
            i = self._alloc()
            self.entries.append([k, i])
            self.kb[i] = k
            for j in range(len(self.row_bytes)):
                self.vb[j][i] = old_vals[j][r]

    def _grow(self, n):
        if len(self.entries) + n <= self.capacity or not self.auto_grow:
            return
        c = max(1, self.capacity)
        while len(self.entries) + n > c:
            c *= 2
        self.rehash(c)

    def insert(self, keys, values=None):
        """keys: list of tuples; values: list (per buffer) of lists of bytes."""
        self._grow(len(keys))
        idx, mask = [], []
        for p, key in enumerate(keys):
            if self._lookup(key) is not None or self.top >= self.capacity:
                idx.append(-1)
                mask.append(False)
                continue
            i = self._alloc()
            self.entries.append([key, i])
            self.kb[i] = key
            if values is not None:
                for j in range(len(self.row_bytes)):
                    self.vb[j][i] = values[j][p]
            idx.append(i)
            mask.append(True)
        return idx, mask

    def activate(self, keys):
        return self.insert(keys, None)

    def find(self, keys):
        idx, mask = [], []
        for key in keys:
            i = self._lookup(key)
            idx.append(-1 if i is None else i)
            mask.append(i is not None)
        return idx, mask

    def erase(self, keys):
        mask = []
        for key in keys:
            hit = None
            for e in self.entries:
                if e[0] == key:
                    hit = e
                    break
            if hit is None:
                mask.append(False)
                continue
            self.entries.remove(hit)
            self._free(hit[1])
            mask.append(True)
        return mask

    def clear(self):
        self.entries = []
        self.heap = list(range(self.capacity))
        self.top = 0

    def as_dict(self):
        return {k: tuple(self.vb[j][i] for j in range(len(self.row_bytes))) for k, i in self.entries}
