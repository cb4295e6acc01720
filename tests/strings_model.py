"""An independent, string-only model of the definitions, used to pin the oracle.

It works on Python strings and never encodes bases as integers.  An edge is
identified without any arrow-head symbols: as the unordered pair of its two
readings {(x, y), (rc(y), rc(x))}, where x and y are consecutive k-mers of a
read (Section 2: the same molecule pair seen from the reverse strand).
"""
from __future__ import annotations

from collections import Counter

_PAIR = str.maketrans("ACGT", "TGCA")


def rc(s: str) -> str:
    return s.translate(_PAIR)[::-1]


def canonical(s: str) -> str:
    return min(s, rc(s))


def split_reads(reads: bytes, lengths) -> list[str]:
    out, p = [], 0
    for L in lengths:
        out.append(reads[p:p + int(L)].decode())
        p += int(L)
    return out


def nodes_of(reads: list[str], k: int) -> list[str]:
    return sorted({canonical(r[j:j + k]) for r in reads for j in range(len(r) - k + 1)})


def edge_class(x: str, y: str) -> frozenset:
    return frozenset({(x, y), (rc(y), rc(x))})


def edge_multiset(reads: list[str], k: int) -> Counter:
    c = Counter()
    for r in reads:
        for j in range(len(r) - k):
            c[edge_class(r[j:j + k], r[j + 1:j + k + 1])] += 1
    return c


def oriented_kmer(node: str, o: int) -> str:
    """The k-mer read at a node end with arrow head o (0 positive, 1 negative)."""
    return node if o == 0 else rc(node)


def unitigs_of(reads: list[str], k: int) -> list[tuple[str, str]]:
    """Maximal non-branching chains, by string extension.

    A k-mer string w is followed by w[1:]+c when the (k+1)-mer w+c, or its
    reverse complement, occurs in a read.  The chain goes on from w to u when
    u is w's only successor, w is u's only predecessor, and u is not the
    molecule of w (Section 6).  Returns ("P", s) for an open chain, s the
    lexicographically smaller of its two spellings, and ("C", s) for a
    closed one spelled from its smallest molecule's positive strand; sorted.
    """
    kp1 = set()
    for r in reads:
        for j in range(len(r) - k):
            z = r[j:j + k + 1]
            kp1.add(z)
            kp1.add(rc(z))

    def succ(w):
        return [w[1:] + c for c in "ACGT" if w + c in kp1]

    def pred(w):
        return [c + w[:-1] for c in "ACGT" if c + w in kp1]

    def nxt(w):
        s = succ(w)
        if len(s) != 1:
            return None
        u = s[0]
        if canonical(u) == canonical(w) or len(pred(u)) != 1:
            return None
        return u

    def prv(w):
        t = nxt(rc(w))
        return None if t is None else rc(t)

    def spell(chain):
        return chain[0] + "".join(w[-1] for w in chain[1:])

    seen, out = set(), []
    for v in nodes_of(reads, k):
        if v in seen:
            continue
        start, closed = v, False
        while True:
            p = prv(start)
            if p is None:
                break
            if canonical(p) == v:
                closed = True
                break
            start = p
        if closed:
            # v is the smallest molecule of its cycle: nodes go in ascending order
            chain = [v]
            while canonical(nxt(chain[-1])) != v:
                chain.append(nxt(chain[-1]))
            out.append(("C", spell(chain)))
        else:
            chain = [start]
            while nxt(chain[-1]) is not None:
                chain.append(nxt(chain[-1]))
            s = spell(chain)
            out.append(("P", min(s, rc(s))))
        seen.update(canonical(w) for w in chain)
    return sorted(out)
