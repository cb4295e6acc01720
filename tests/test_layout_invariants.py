"""Index and encoding invariants that the kernels' memory safety rests on,
checked on the CPU over random and extreme cases (the arithmetic restated
from the kernels; no GPU, no oracle).

- The persistent onesweep pass with bulk write-out stages digit d's run from
  slot place_d = start_d + (A-1) d + ((g_d - start_d - (A-1) d) mod A), with
  start_d the run's unpadded start in the tile and g_d its first output
  index: every place_d is congruent to g_d modulo A (so both ends of each
  bulk copy are 16-byte aligned), runs never overlap, and the last one ends
  within TILE + (A-1) * 256 slots.
- A node record's payload (edge e << 1 | role, this end's side at bit 30,
  the far end's at bit 31) below 2^29 edges never equals the no-edge marker
  0xffffffff and decodes back to (e, role, sides)."""
from __future__ import annotations

import numpy as np
import pytest

RADIX = 256
REC_NONE = 0xFFFFFFFF


def placements(counts, gstart, align):
    start = np.concatenate([[0], np.cumsum(counts)[:-1]]).astype(np.int64)
    d = np.arange(RADIX, dtype=np.int64)
    place = start + (align - 1) * d + ((gstart - start - (align - 1) * d) % align)
    return start, place


@pytest.mark.parametrize("align,tile", [(2, 1024 * 10), (2, 1024 * 12), (4, 1024 * 6), (4, 1024 * 7),
                                        (4, 1024 * 3), (1, 1024 * 5)])
def test_bulk_run_placement(align, tile):
    rng = np.random.default_rng(align * 100003 + tile)
    for trial in range(400):
        n = tile if trial % 3 else int(rng.integers(0, tile + 1))  # full and partial tiles
        kind = trial % 4
        if kind == 0:    # uniform digits
            counts = rng.multinomial(n, np.full(RADIX, 1.0 / RADIX))
        elif kind == 1:  # one digit holds everything
            counts = np.zeros(RADIX, dtype=np.int64)
            counts[int(rng.integers(0, RADIX))] = n
        elif kind == 2:  # a few heavy digits
            w = rng.random(RADIX) ** 8
            counts = rng.multinomial(n, w / w.sum())
        else:            # every digit odd-sized where possible
            counts = rng.multinomial(n, np.full(RADIX, 1.0 / RADIX)) | 1
            counts[-1] = 0
            while counts.sum() > n:
                counts[int(np.argmax(counts))] -= 1
        counts = counts.astype(np.int64)
        # each digit's output range starts anywhere in the array
        gstart = rng.integers(0, 1 << 40, size=RADIX, dtype=np.int64)
        start, place = placements(counts, gstart, align)
        assert np.all((place - gstart) % align == 0)
        assert np.all(place >= start)
        assert np.all(place[1:] >= place[:-1] + counts[:-1])
        assert place[-1] + counts[-1] <= tile + (align - 1) * RADIX
        # the bulk part of each run (issued where it is not empty): from the
        # first aligned output index, a whole number of ALIGN-element units,
        # inside the run
        head = np.minimum(counts, (align - gstart % align) % align)
        mid = (counts - head) // align * align
        bulk = mid > 0
        assert np.all((gstart + head)[bulk] % align == 0) and np.all((place + head)[bulk] % align == 0)
        assert np.all(head + mid <= counts) and np.all(counts - head - mid < align)


def payload(e, role, s_own, s_far):
    return (e << 1) | role | (s_own << 30) | (s_far << 31)


def test_payload_side_bits():
    top = (1 << 29) - 2  # the largest edge index below 2^29 edges
    for e in [0, 1, 2, 12345, (1 << 28) + 7, top - 1, top]:
        for role in (0, 1):
            for s_own in (0, 1):
                for s_far in (0, 1):
                    v = payload(e, role, s_own, s_far)
                    assert v < (1 << 32) and v != REC_NONE
                    low = v & 0x3FFFFFFF
                    assert (low >> 1, low & 1, (v >> 30) & 1, v >> 31) == (e, role, s_own, s_far)
    # the edge count the encoding allows: one more edge would reach the marker
    assert payload((1 << 29) - 1, 1, 1, 1) == REC_NONE


def test_head_word_packs_length_and_strand():
    """A unitig's head word, length << 1 | strand, for lengths up to the
    fast path's 2^29 - 1 strand-nodes' nodes."""
    for L in [1, 2, 3, 1000, (1 << 28) - 1, 1 << 28]:
        for strand in (0, 1):
            w = (L << 1) | strand
            assert w < (1 << 32) and (w >> 1, w & 1) == (L, strand)
