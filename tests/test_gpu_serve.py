"""Host-memory plans and the serving loop: every request's pass list, served
merged with others as requests arrive, is identical to the same request
filtered alone and to the oracle; overflow splitting, validation at
submission, the device-memory budget and queue back-pressure."""
import threading

import numpy as np
import pytest

import oracle
from tests.conftest import Reads
from tests.gpu_helpers import assert_same, build

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def world():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_1708_04329_gb300 import synth

    g = synth.human_genome(600_000, seed=71)
    oix = oracle.bin_vectors(g, 200, 5, 250)
    idx = build(g, 200, 5, 250, 7)
    return g, oix, idx


def _ragged(g, n, seed):
    from paper_1708_04329_gb300 import synth

    return synth.reads(g, n, seed=seed, lengths=(100, 150, 250), probs=(0.5, 0.3, 0.2),
                       e_frac=(5, 100), max_edits=None)


def _host_args(rs):
    return dict(reads=np.frombuffer(rs.seq, np.uint8), offsets=rs.offsets.astype(np.uint64),
                lens=rs.lens.astype(np.uint32), e=rs.e.astype(np.uint16))


def _requests(g, sizes, seed):
    return [_ragged(g, n, seed + i) for i, n in enumerate(sizes)]


def test_host_io_plan_batches(world):
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    plan = grim.grim_plan_create(idx, max_reads=700, max_bases=700 * 250, max_e=12, cap=30_000,
                                 host_io=True)
    assert plan.host_io and isinstance(plan.buffers["reads"], np.ndarray)
    for n, seed in ((700, 1), (1, 2), (0, 3), (333, 4)):
        rs = _ragged(g, n, seed) if n else Reads([], [])
        got = plan.run(**_host_args(rs))
        assert_same(got, oracle.filter(oix, rs))
    # a read ending past max_bases is refused at launch
    b = plan.buffers
    b["offsets"][0] = 700 * 250 - 10
    b["lens"][0] = 100
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_plan_launch(plan, 1)
    assert ei.value.code == grim.GRIM_E_ARG


def test_host_io_candidate_plan(world):
    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    plan = grim.grim_plan_create(idx, max_reads=400, max_bases=400 * 250, max_e=12, cap=30_000,
                                 max_cand=400 * 300, candidates=True, host_io=True)
    for n, seed in ((400, 11), (7, 12)):
        rs = _ragged(g, n, seed)
        off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), oix.num_bins,
                                     seed=seed, median=40)
        got = plan.run(**_host_args(rs), cand=cand, cand_off=off)
        assert_same(got, oracle.filter(oix, rs, cand_off=off, cand=cand))


def test_server_mix_equals_alone(world):
    """Requests submitted from several threads at once are merged into shared
    batches; each result equals that request filtered alone (grim_filter_host)
    and the oracle."""
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    rng = np.random.default_rng(5)
    sizes = [int(x) for x in np.exp(rng.uniform(0, np.log(400), 48))]
    reqs = _requests(g, sizes, 100)
    srv = grim.grim_server_create(idx, slots=3, max_reads=1024, max_bases=1024 * 250, max_e=12,
                                  cap=40_000)
    tickets = [None] * len(reqs)

    def submitter(part):
        for i in part:
            tickets[i] = srv.submit(**_host_args(reqs[i]))

    threads = [threading.Thread(target=submitter, args=(range(k, len(reqs), 4),)) for k in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    results = [srv.result(t, timeout_s=60) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["reads_done"] == sum(sizes)
    merged = max(info.batch_requests for _, info in results)
    assert merged > 1, "no two requests shared a batch"
    for rs, (got, info) in zip(reqs, results):
        assert info.status == 0 and info.n_reads == rs.n
        assert info.t_submit_ns <= info.t_launch_ns <= info.t_done_ns
        alone = grim.grim_filter_host(idx, **_host_args(rs), cap=40_000)
        assert_same(got, alone)
    for rs, (got, _) in list(zip(reqs, results))[:6]:
        assert_same(got, oracle.filter(oix, rs))


def test_server_candidates(world):
    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    srv = grim.grim_server_create(idx, slots=2, max_reads=600, max_bases=600 * 250, max_e=12,
                                  cap=40_000, max_cand=600 * 200, candidates=True)
    work = []
    for i, n in enumerate((200, 1, 57, 300, 12)):
        rs = _ragged(g, n, 300 + i)
        off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), oix.num_bins,
                                     seed=300 + i, median=30)
        work.append((rs, off, cand, srv.submit(**_host_args(rs), cand=cand, cand_off=off)))
    for rs, off, cand, t in work:
        got, info = srv.result(t, timeout_s=60)
        assert_same(got, oracle.filter(oix, rs, cand_off=off, cand=cand))
    srv.close()


def test_server_overflow_split(world):
    """A merged batch over the slot's capacity is rerun one request per batch;
    a request alone over it fails with GRIM_E_OVERFLOW and its total."""
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    small = _requests(g, [30] * 8, 500)
    want = [oracle.filter(oix, rs) for rs in small]
    per = max(len(w[0]) for w in want)
    cap = per + 5
    assert sum(len(w[0]) for w in want) > cap
    big = _ragged(g, 400, 600)
    srv = grim.grim_server_create(idx, slots=1, max_reads=1024, max_bases=1024 * 250, max_e=12,
                                  cap=cap)
    # hold the only slot with the big request so that the small ones queue up and merge
    tb = srv.submit(**_host_args(big))
    ts = [srv.submit(**_host_args(rs)) for rs in small]
    for t, w in zip(ts, want):
        got, info = srv.result(t, timeout_s=60)
        assert_same(got, w)
    with pytest.raises(grim.GrimError) as ei:
        srv.result(tb, timeout_s=60)
    assert ei.value.code == grim.GRIM_E_OVERFLOW
    assert ei.value.n_out == len(oracle.filter(oix, big)[0])
    assert srv.stats()["overflow_splits"] >= 1
    srv.close()


def test_server_validation_and_limits(world):
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    srv = grim.grim_server_create(idx, slots=2, max_reads=100, max_bases=100 * 250, max_e=6,
                                  cap=10_000)
    rs = _ragged(g, 50, 700)
    rs.e = np.minimum(rs.e, 6).astype(np.uint16)
    a = _host_args(rs)
    bad_e = dict(a, e=np.full(50, 7, np.uint16))
    with pytest.raises(grim.GrimError) as ei:
        srv.submit(**bad_e)
    assert ei.value.code == grim.GRIM_E_ARG
    short = dict(a, lens=np.where(np.arange(50) == 3, 4, a["lens"]).astype(np.uint32))
    with pytest.raises(grim.GrimError) as ei:
        srv.submit(**short)
    assert ei.value.code == grim.GRIM_E_READ_TOO_SHORT
    with pytest.raises(grim.GrimError) as ei:
        srv.submit(**_host_args(_ragged(g, 101, 701)))
    assert ei.value.code == grim.GRIM_E_ARG
    with pytest.raises(grim.GrimError):
        srv.submit(**a, cand=np.zeros(1, np.int32), cand_off=np.array([0, 1], np.uint64))
    # the server still serves
    got, _ = srv.result(srv.submit(**a), timeout_s=60)
    assert_same(got, oracle.filter(oix, rs))
    # an empty request completes with no records
    got, info = srv.result(srv.submit(reads=np.zeros(0, np.uint8), offsets=np.zeros(0, np.uint64),
                                      lens=np.zeros(0, np.uint32), e=np.zeros(0, np.uint16)),
                           timeout_s=60)
    assert len(got[0]) == 0 and info.status == 0
    srv.close()


def test_server_memory_budget_and_backpressure(world):
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    one = grim.grim_server_create(idx, slots=1, max_reads=512, max_bases=512 * 250, max_e=12,
                                  cap=20_000)
    per_slot = one.stats()["device_bytes"]
    one.close()
    srv = grim.grim_server_create(idx, slots=4, max_reads=512, max_bases=512 * 250, max_e=12,
                                  cap=20_000, mem_budget=2 * per_slot + per_slot // 2)
    assert srv.stats()["slots"] == 2
    srv.close()
    with pytest.raises(grim.GrimError) as ei:
        grim.grim_server_create(idx, slots=2, max_reads=512, max_bases=512 * 250, max_e=12,
                                cap=20_000, mem_budget=per_slot // 2)
    assert ei.value.code == grim.GRIM_E_NOMEM
    # a bounded queue refuses requests while it is full
    srv = grim.grim_server_create(idx, slots=1, max_reads=512, max_bases=512 * 250, max_e=12,
                                  cap=20_000, max_queued_reads=150)
    rs = _ragged(g, 100, 800)
    a = _host_args(rs)
    want = oracle.filter(oix, rs)
    accepted, busy = [], 0
    for _ in range(300):
        try:
            accepted.append(srv.submit(**a))
        except grim.GrimError as err:
            assert err.code == grim.GRIM_E_BUSY
            busy += 1
            if busy > 3:
                break
    assert busy > 0
    for t in accepted:
        got, _ = srv.result(t, timeout_s=60)
        assert_same(got, want)
    srv.close()


def test_server_cancel(world):
    """A queued request can be cancelled (it completes with GRIM_E_CANCELLED
    and never runs); one already on the device completes normally; the
    others are unaffected."""
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    # one slot of 25 reads: each 20-read request is a batch of its own, so
    # the last of 40 requests waits behind the other 39
    srv = grim.grim_server_create(idx, slots=1, max_reads=25, max_bases=25 * 250, max_e=12,
                                  cap=20_000)
    reqs = _requests(g, [20] * 40, 950)
    ts = [srv.submit(**_host_args(rs)) for rs in reqs]
    assert srv.cancel(ts[-1]) is True
    with pytest.raises(grim.GrimError) as ei:
        srv.result(ts[-1], timeout_s=60)
    assert ei.value.code == grim.GRIM_E_CANCELLED
    for t, rs in list(zip(ts, reqs))[:-1]:
        got, _ = srv.result(t, timeout_s=60)
        assert_same(got, oracle.filter(oix, rs))
    with pytest.raises(grim.GrimError) as ei:
        srv.cancel(ts[0])  # completed and taken
    assert ei.value.code == grim.GRIM_E_ARG
    st = srv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 39
    srv.close()


def test_server_chunked_requests(world):
    """With max_chunk_reads, requests are cut into chunks of consecutive reads
    that run in different batches and slots; each request's result -- one
    larger than a slot among them, and an 8,192-read one among small ones --
    equals the request filtered alone and the oracle."""
    from paper_1708_04329_gb300 import grim

    g, oix, idx = world
    srv = grim.grim_server_create(idx, slots=3, max_reads=1024, max_bases=1024 * 250, max_e=12,
                                  cap=60_000, max_chunk_reads=256)
    sizes = [8192, 1, 40, 700, 2000, 3, 257, 256, 90]
    reqs = _requests(g, sizes, 1200)
    tickets = [srv.submit(**_host_args(rs)) for rs in reqs]
    results = [srv.result(t, timeout_s=120) for t in tickets]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["reads_done"] == sum(sizes)
    # the 8,192-read request alone needed 8 batches of 1,024 reads (32 chunks)
    assert st["batches"] >= 8
    for rs, (got, info) in zip(reqs, results):
        assert info.status == 0 and info.n_reads == rs.n
        assert_same(got, grim.grim_filter_host(idx, **_host_args(rs), cap=400_000))
    for rs, (got, _) in list(zip(reqs, results))[1:5]:
        assert_same(got, oracle.filter(oix, rs))


def test_server_chunked_candidates_cancel_overflow(world):
    """Chunks also split on the candidate limit; a chunked request can be
    cancelled while all its chunks wait; a chunk over the capacity fails its
    request with GRIM_E_OVERFLOW and the request's total."""
    from paper_1708_04329_gb300 import grim, synth

    g, oix, idx = world
    srv = grim.grim_server_create(idx, slots=2, max_reads=300, max_bases=300 * 250, max_e=12,
                                  cap=40_000, max_cand=3000, candidates=True, max_chunk_reads=300)
    rs = _ragged(g, 900, 1300)
    off, cand = synth.candidates((rs.true_pos // 200).astype(np.int32), oix.num_bins, seed=1300,
                                 median=25)
    assert off[-1] > 3000  # more candidates than one batch holds
    got, info = srv.result(srv.submit(**_host_args(rs), cand=cand, cand_off=off), timeout_s=120)
    assert_same(got, oracle.filter(oix, rs, cand_off=off, cand=cand))
    srv.close()

    # one slot of 20 reads; the last request's chunks wait behind 30 others
    srv = grim.grim_server_create(idx, slots=1, max_reads=20, max_bases=20 * 250, max_e=12,
                                  cap=20_000, max_chunk_reads=10)
    reqs = _requests(g, [20] * 30 + [55], 1400)
    ts = [srv.submit(**_host_args(r)) for r in reqs]
    assert srv.cancel(ts[-1]) is True
    with pytest.raises(grim.GrimError) as ei:
        srv.result(ts[-1], timeout_s=60)
    assert ei.value.code == grim.GRIM_E_CANCELLED
    for t, r in list(zip(ts, reqs))[:-1]:
        got, _ = srv.result(t, timeout_s=60)
        assert_same(got, oracle.filter(oix, r))
    srv.close()

    big = _ragged(g, 400, 1500)
    want = oracle.filter(oix, big)
    per_chunk = max(len(oracle.filter(oix, big.subset(range(k, min(k + 50, 400))))[0])
                    for k in range(0, 400, 50))
    srv = grim.grim_server_create(idx, slots=2, max_reads=100, max_bases=100 * 250, max_e=12,
                                  cap=per_chunk // 2, max_chunk_reads=50)
    with pytest.raises(grim.GrimError) as ei:
        srv.result(srv.submit(**_host_args(big)), timeout_s=60)
    assert ei.value.code == grim.GRIM_E_OVERFLOW
    assert ei.value.n_out == len(want[0])
    srv.close()
    with pytest.raises(grim.GrimError) as ei:  # a chunk larger than a batch
        grim.grim_server_create(idx, slots=1, max_reads=10, max_bases=2500, max_e=12, cap=100,
                                max_chunk_reads=11)
    assert ei.value.code == grim.GRIM_E_ARG
