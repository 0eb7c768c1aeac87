"""Brute-force restatement of the filter for tiny inputs.

TEST INFRASTRUCTURE ONLY.  It shares nothing with ``grim_oracle.c``: no bit
vectors, no token codes.  For each read and bin it asks Python's substring
search whether each of the read's q-grams occurs in the bin's window
(§GRIM-Filter: a token's existence bit for a bin is set iff the token occurs
in that bin's stretch of the reference; the bins overlap by L_max-1 bases so a
read lying in the bin fits inside it).  The sum of those answers is compared
with (L-q+1) - q*e (Fig. 3's threshold).
"""
from __future__ import annotations

BASES = set("ACGT")


def windows(ref: str, B: int, ext: int) -> list[str]:
    """Upper-cased window text of every bin: ref[b*B : min(b*B+B+ext, N)]."""
    n = len(ref)
    nb = (n + B - 1) // B
    return [ref[b * B: min(b * B + B + ext, n)].upper() for b in range(nb)]


def qgrams(read: str, q: int) -> list[str | None]:
    """The read's L-q+1 q-grams, upper-cased; None where one has a non-base."""
    out = []
    for j in range(len(read) - q + 1):
        g = read[j: j + q].upper()
        out.append(g if set(g) <= BASES else None)
    return out


def count(read: str, window: str, q: int) -> int:
    """How many of the read's q-gram positions occur in the window."""
    return sum(1 for g in qgrams(read, q) if g is not None and g in window)


def filter(ref: str, B: int, ext: int, q: int, reads: list[str], e: list[int],
           cands: list[list[int]] | None = None):
    """Passing (read, bin, count) triples, read by read, bins ascending or in
    candidate order."""
    win = windows(ref, B, ext)
    out = []
    for r, rd in enumerate(reads):
        T = (len(rd) - q + 1) - q * e[r]
        bins = range(len(win)) if cands is None else cands[r]
        for b in bins:
            c = count(rd, win[b], q)
            if c >= T:
                out.append((r, b, c))
    return out


def present_set(ref: str, B: int, ext: int, q: int, b: int) -> set[str]:
    """The distinct clean q-grams of bin b's window."""
    w = windows(ref, B, ext)[b]
    return {w[p: p + q] for p in range(len(w) - q + 1) if set(w[p: p + q]) <= BASES}
