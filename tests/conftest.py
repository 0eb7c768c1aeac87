import sys
from pathlib import Path

import numpy as np
import pytest

ROOT = Path(__file__).resolve().parent.parent
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

GOLDEN = Path(__file__).resolve().parent / "golden"


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def load_fixture(name: str) -> dict:
    """Parse a tests/golden/*.txt fixture: `key value...` lines, '#' comments."""
    d: dict = {"read": [], "pass": [], "set": [], "clear": []}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        key, *vals = line.split()
        if key == "read":
            d["read"].append((vals[0], int(vals[1])))
        elif key == "pass":
            d["pass"].append(tuple(int(v) for v in vals))
        elif key in ("set", "clear"):
            d[key].extend(int(v) for v in vals)
        elif key == "ref":
            d["ref"] = vals[0]
        else:
            d[key] = int(vals[0])
    return d


class Reads:
    """Minimal read container with the fields both sides take."""

    def __init__(self, reads: list[str], e: list[int]):
        self.lens = np.array([len(r) for r in reads], dtype=np.uint32)
        self.offsets = np.zeros(len(reads), dtype=np.uint64)
        if len(reads) > 1:
            self.offsets[1:] = np.cumsum(self.lens[:-1])
        self.seq = np.frombuffer("".join(reads).encode(), dtype=np.uint8).copy()
        self.e = np.array(e, dtype=np.uint16)
        self.strs = list(reads)

    @property
    def n(self) -> int:
        return len(self.strs)


def random_case(rng: np.random.Generator, q: int, n: int, B: int, max_read_len: int,
                n_reads: int, dirty: bool = True):
    """A random tiny case: genome with lowercase and N runs, reads of mixed
    length sampled from it (some mutated, some random), random e."""
    alpha = np.frombuffer(b"ACGT", dtype=np.uint8)
    g = alpha[rng.integers(0, 4, n)]
    if dirty:
        low = rng.random(n) < 0.05
        g = np.where(low, g + 32, g).astype(np.uint8)
        for _ in range(rng.integers(0, 3)):
            s = int(rng.integers(0, n))
            g[s:s + int(rng.integers(1, 6))] = ord("N")
    ref = g.tobytes().decode()
    reads, es = [], []
    for _ in range(n_reads):
        L = int(rng.integers(q, max_read_len + 1))
        if rng.random() < 0.7 and n > L:
            s = int(rng.integers(0, n - L + 1))
            rd = bytearray(ref[s:s + L].encode())
            for _k in range(int(rng.integers(0, 4))):
                p = int(rng.integers(0, L))
                rd[p] = b"ACGTNacgt"[int(rng.integers(0, 9 if dirty else 4))]
        else:
            rd = bytearray(alpha[rng.integers(0, 4, L)].tobytes())
        reads.append(rd.decode())
        es.append(int(rng.integers(0, 4)))
    return ref, reads, es


@pytest.fixture(scope="session")
def tiny_plain():
    from paper_1708_04329_gb300 import synth

    return synth.tiny_plain()


@pytest.fixture(scope="session")
def tiny_plain_index(tiny_plain):
    import oracle

    w = tiny_plain
    return oracle.bin_vectors(w["genome"], w["B"], w["q"], w["max_read_len"])


@pytest.fixture(scope="session")
def tiny_plain_oracle(tiny_plain, tiny_plain_index):
    import oracle

    return oracle.filter(tiny_plain_index, tiny_plain["reads"])
