"""The pins are strong enough to catch plausible oracle mistakes.

Each case plants one mistake in a copy of ``oracle/grim_oracle.c`` (on the
CPU, in a temporary directory), rebuilds it, and checks that the hand-worked
fixtures or the brute-force comparison reject the mutant.
"""
import subprocess

import numpy as np
import pytest

import oracle
from oracle import bruteforce
from tests.conftest import Reads, load_fixture, random_case

MUTANTS = {
    "window_end_off_by_one": ("for (uint64_t p = lo; p + q <= hi; ++p)",
                              "for (uint64_t p = lo; p + q < hi; ++p)"),
    "no_extension": ("uint64_t hi = lo + B + ext;", "uint64_t hi = lo + B;"),
    "strict_threshold": ("if (sum >= T)", "if (sum > T)"),
    "threshold_q_minus_1": ("(int64_t)ntok - (int64_t)q * (int64_t)e[r]",
                            "(int64_t)ntok - (int64_t)(q - 1) * (int64_t)e[r]"),
    "last_base_first": ("v = v * 4 + c;", "v = v + ((int64_t)c << (2 * i));"),
    "drops_last_token": ("for (uint32_t j = 0; j < ntok; ++j)",
                         "for (uint32_t j = 0; j + 1 < ntok; ++j)"),
    "invalid_token_counts": ("if (tok[j] >= 0) sum += vec_bit(v, tok[j]);",
                             "sum += tok[j] >= 0 ? vec_bit(v, tok[j]) : 1;"),
    "case_sensitive": ("case 'a': return 0;", "case 'a': return -1;"),
    "bins_floor": ("return B ? (n + B - 1) / B : 0;", "return B ? n / B : 0;"),
    # a run of one repeated token counted once (a set reading of homopolymers)
    "repeats_counted_once": ("if (tok[j] >= 0) sum += vec_bit(v, tok[j]);",
                             "if (tok[j] >= 0 && (j == 0 || tok[j] != tok[j - 1])) "
                             "sum += vec_bit(v, tok[j]);"),
}


def _build_mutant(tmp_path, name):
    src = (oracle.HERE / "grim_oracle.c").read_text()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, name
    p = tmp_path / f"{name}.c"
    p.write_text(src.replace(old, new))
    so = tmp_path / f"lib{name}.so"
    subprocess.run(["gcc", "-O1", "-fopenmp", "-fPIC", "-shared", "-std=c11", str(p), "-o", str(so)],
                   check=True)
    return oracle._bind(so)


def _pins_hold() -> bool:
    """The fixtures plus a few brute-force cases, run on whatever oracle is loaded."""
    fx = load_fixture("handworked_q3.txt")
    reads = [r for r, _ in fx["read"]]
    e = [x for _, x in fx["read"]]
    idx = oracle.bin_vectors(np.frombuffer(fx["ref"].encode(), np.uint8), fx["B"], fx["q"],
                             fx["max_read_len"])
    r, b, c = oracle.filter(idx, Reads(reads, e))
    if list(zip(r.tolist(), b.tolist(), c.tolist())) != fx["pass"]:
        return False
    f2 = load_fixture("fig2_q5.txt")
    idx = oracle.bin_vectors(np.frombuffer(f2["ref"].encode(), np.uint8), f2["B"], f2["q"],
                             f2["max_read_len"])
    bits = np.unpackbits(idx.vecs[0], bitorder="little")
    if sorted(np.flatnonzero(bits).tolist()) != sorted(f2["set"]):
        return False
    for seed in range(4):
        rng = np.random.default_rng(1000 + seed)
        q = int(rng.choice([3, 4, 5]))
        B = int(rng.integers(5, 60))
        mrl = int(rng.integers(max(q, 6), 40))
        n = int(rng.integers(50, 1500))
        ref, rds, es = random_case(rng, q, n, B, mrl, 25)
        idx = oracle.bin_vectors(np.frombuffer(ref.encode(), np.uint8), B, q, mrl)
        r, b, c = oracle.filter(idx, Reads(rds, es))
        got = list(zip(r.tolist(), b.tolist(), c.tolist()))
        if got != bruteforce.filter(ref, B, mrl - 1, q, rds, es):
            return False
    # homopolymer and tandem-repeat reads against a genome holding such runs
    ref = "ACGTTGCA" * 5 + "A" * 60 + "CACGTCAGGT" * 4 + "AC" * 30 + "TTGACGCATG" * 3
    rds = ["A" * 30, "AC" * 15, "CA" * 12 + "G", "ACGTTGCA" * 3, "A" * 20 + "CACG"]
    es = [0, 1, 0, 2, 1]
    for q, B in ((3, 25), (4, 40)):
        idx = oracle.bin_vectors(np.frombuffer(ref.encode(), np.uint8), B, q, 40)
        r, b, c = oracle.filter(idx, Reads(rds, es))
        got = list(zip(r.tolist(), b.tolist(), c.tolist()))
        if got != bruteforce.filter(ref, B, 39, q, rds, es):
            return False
    return True


def test_unmutated_oracle_passes_pins():
    assert _pins_hold()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", _build_mutant(tmp_path, name))
    assert not _pins_hold()
