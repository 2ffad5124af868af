"""Byte counts of the cluster kernel's mbarrier exchanges (CPU).

Each rank of a cluster arms its mbarrier for an exchange with the bytes it expects, given in
closed form from the ownership rules (csrc/ks_cluster.cuh: bx_A, bx_B, bx_Aa, bx_Ba); a count
above what the producers send would make the wait run out, one below would let a phase start
before its data.  Here the pushes of the four exchanges are enumerated element by element with
the kernel's ownership and index rules (column j of rank j mod C, or pair p of rank p mod C in
the centre-symmetric subspace; rows in contiguous blocks of an even count per rank; two values
per store), and the bytes each rank receives must equal the closed form, every store must land
on a rank of the cluster inside its buffer, and no two stores of one exchange may share an
address."""

import itertools

import pytest

PART = 8  # bytes of one partial of J or L^dag_2 (double, or a float-float pair)


def rows_per_rank(ns, C):
    r = (ns + C - 1) // C
    r += r & 1
    return max(r, 2)


class Cluster:
    def __init__(self, nx, ns, C, xi):
        self.nx, self.ns, self.C, self.xi = nx, ns, C, xi
        self.kx = nx // 3
        self.nkx = self.kx + 1
        self.npr = (self.kx + 1) // 2
        self.rpr = rows_per_rank(ns, C)
        self.lg = ns.bit_length() - 1

    def ncol(self, r):
        if self.xi:
            return 2 * ((self.npr - r + self.C - 1) // self.C) if r < self.npr else 0
        return (self.nkx - r + self.C - 1) // self.C if r < self.nkx else 0

    def colj(self, r, q):
        if self.xi:
            return 2 * (r + (q >> 1) * self.C) + 1 + (q & 1)
        return r + q * self.C

    def own_rank(self, j):
        return ((j - 1) >> 1) % self.C if self.xi else j % self.C

    def own_slot(self, j):
        if self.xi:
            return 2 * (((j - 1) >> 1) // self.C) + ((j - 1) & 1)
        return j // self.C

    def rows(self, r):
        row0 = r * self.rpr
        return row0, (min(self.rpr, self.ns - row0) if row0 < self.ns else 0)

    # ---- the closed forms the kernel arms with ----
    def expected(self, r, cs, ca):
        ncol = self.ncol(r)
        mycols = sum(1 for q in range(ncol) if self.colj(r, q) <= self.kx) if self.xi else ncol
        ncx = self.kx if self.xi else self.nkx
        nrow = self.rows(r)[1]
        return {"A": mycols * self.ns * cs, "B": ncx * nrow * ca + 2 * ncx * PART,
                "Aa": mycols * self.ns * ca, "Ba": ncx * nrow * cs}

    # ---- the pushes, element by element ----
    def row_phase(self, size):
        """Phases A / A': each rank's row pairs, every retained x-mode (j = 0 skipped in the
        subspace), two values per store to the mode's owner at slot * Ns + n."""
        got = [0] * self.C
        seen = set()
        for r in range(self.C):
            row0, nrow = self.rows(r)
            for n in range(row0, row0 + nrow, 2):
                for j in range(self.nkx):
                    if self.xi and j == 0:
                        continue
                    o, sl = self.own_rank(j), self.own_slot(j)
                    assert 0 <= o < self.C and sl < self.ncol(o)
                    for e in (0, 1):
                        key = (o, sl * self.ns + n + e)
                        assert key not in seen
                        seen.add(key)
                    got[o] += 2 * size
        return got

    def col_phase(self, size, partials):
        """Phases B / B': each column owner's s-values, two rows per store to the rows' owner at
        j * rmax + (n - row0(owner)); in phase B also two partials per column to every rank."""
        got = [0] * self.C
        seen = set()
        for c in range(self.C):
            ncol = self.ncol(c)
            if self.xi:
                for i in range((ncol << self.lg) >> 2):
                    pp, n = (2 * i) >> self.lg, (2 * i) & (self.ns - 1)
                    o = n // self.rpr
                    assert 0 <= o < self.C
                    ja = self.colj(c, 2 * pp)
                    for j in ((ja, ja + 1) if ja + 1 <= self.kx else (ja,)):
                        for e in (0, 1):
                            key = (o, j, n + e)
                            assert key not in seen and n + e - o * self.rpr < self.rpr
                            seen.add(key)
                        got[o] += 2 * size
                if partials:
                    for pp in range(ncol >> 1):
                        nj = 2 if self.colj(c, 2 * pp + 1) <= self.kx else 1
                        for t in range(self.C):
                            got[t] += 2 * nj * PART
            else:
                for i in range((ncol << self.lg) >> 1):
                    q, n = (2 * i) >> self.lg, (2 * i) & (self.ns - 1)
                    o = n // self.rpr
                    assert 0 <= o < self.C
                    j = self.colj(c, q)
                    assert j < self.nkx
                    for e in (0, 1):
                        key = (o, j, n + e)
                        assert key not in seen and n + e - o * self.rpr < self.rpr
                        seen.add(key)
                    got[o] += 2 * size
                if partials:
                    for t in range(self.C):
                        got[t] += 2 * ncol * PART
        return got


SHAPES = [(32, 8), (32, 32), (64, 32), (64, 64), (64, 128), (64, 256), (128, 64), (256, 128)]


@pytest.mark.parametrize("nx,ns", SHAPES)
@pytest.mark.parametrize("xi", [False, True])
def test_exchange_bytes_match_the_pushes(nx, ns, xi):
    for C, (cs, ca) in itertools.product((1, 2, 4, 8, 16), ((16, 16), (8, 8), (16, 8))):
        cl = Cluster(nx, ns, C, xi)
        got = {"A": cl.row_phase(cs), "B": cl.col_phase(ca, True),
               "Aa": cl.row_phase(ca), "Ba": cl.col_phase(cs, False)}
        for r in range(C):
            exp = cl.expected(r, cs, ca)
            for x in ("A", "B", "Aa", "Ba"):
                assert got[x][r] == exp[x], (nx, ns, C, xi, r, x)
                assert exp[x] < (1 << 20)  # an mbarrier's transaction count


def test_every_value_reaches_its_owner():
    """Totals: phase A delivers every real column at every row once, phase B every exchanged
    column at every row once (ghost columns of the subspace never travel)."""
    for nx, ns in SHAPES:
        for xi in (False, True):
            cl = Cluster(nx, ns, 16, xi)
            ncx = cl.kx if xi else cl.nkx
            assert sum(cl.row_phase(1)) == ncx * ns
            assert sum(cl.col_phase(1, False)) == ncx * ns
