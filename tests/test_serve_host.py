"""Host logic of the continuous-batching server (the admission loop of DecodeServer.run) on
the CPU: the device side is replaced by slots whose decode finishes after a set host time.
Checked: the HBM budget and the slot count hold at every admission, admission follows arrival
order, every request is answered, and a request that can never fit is answered with E_NOMEM
at once instead of blocking the requests behind it."""
import time
import types

import pytest

from paper_2607_12656_b300 import serve, sgs


class _FakeSlot:
    def __init__(self):
        self.busy = None
        self.ctx = types.SimpleNamespace(close=lambda: None)


class _FakeServer(serve.DecodeServer):
    """Decode of scene s takes dur[s] seconds of host time; records the state at each launch."""

    def __init__(self, scenes, dur, **kw):
        self.dur = dur
        self.log = []  # (req, in_use after admission, busy slots)
        super().__init__(scenes, **kw)

    def _make_slots(self, n, scratch):
        return [_FakeSlot() for _ in range(n)]

    def _launch(self, slot, req, sid, arrival, now):
        slot.busy = (req, sid, arrival, now, time.perf_counter(), None, None)
        self.log.append((req, self.in_use, sum(1 for s in self.slots if s.busy)))

    def _finished(self, slot):
        return time.perf_counter() - slot.busy[4] >= self.dur[slot.busy[1]]

    def _retire(self, slot, t0):
        req, sid, arr, adm = slot.busy[:4]
        return serve.Result(req, sid, arr, adm, time.perf_counter() - t0, sgs.OK)


def _scenes(sizes):
    info = lambda n: types.SimpleNamespace(n_rows=0, total_len=n, scratch_bytes=0)
    return [serve.Scene(b"", info=info(n), host=object()) for n in sizes]


@pytest.mark.timeout(60)
def test_budget_slots_and_arrival_order():
    sizes = [3, 5, 2, 7, 4]
    srv = _FakeServer(_scenes(sizes), dur=[0.004, 0.006, 0.002, 0.008, 0.003], slots=3, hbm_budget=10)
    reqs = serve.poisson_arrivals(2000.0, 60, len(sizes), seed=3)
    res = srv.run(reqs)
    assert sorted(r.req for r in res) == list(range(60)) and all(r.status == sgs.OK for r in res)
    assert all(u <= 10 for _, u, _ in srv.log) and all(b <= 3 for _, _, b in srv.log)
    assert [q for q, _, _ in srv.log] == list(range(60))  # admitted in arrival order
    assert max(u for _, u, _ in srv.log) > max(sizes)  # requests did share the budget
    for r in res:
        assert r.arrival <= r.admitted <= r.done
    assert srv.in_use == 0


@pytest.mark.timeout(60)
def test_request_that_can_never_fit_is_refused_not_stuck():
    sizes = [4, 25, 3]  # scene 1 exceeds the budget on its own
    srv = _FakeServer(_scenes(sizes), dur=[0.002, 0.002, 0.002], slots=2, hbm_budget=10)
    reqs = [(0.001 * i, i % 3) for i in range(30)]
    res = srv.run(reqs)
    assert sorted(r.req for r in res) == list(range(30))
    for r in res:
        assert r.status == (sgs.E_NOMEM if r.scene == 1 else sgs.OK)
        if r.scene == 1:
            assert r.admitted == r.done  # answered on the spot
    assert [q for q, _, _ in srv.log] == [i for i in range(30) if i % 3 != 1]
    s = serve.summarize(res, srv.scenes)
    assert s["bad_status"] == 10 and s["requests"] == 30


@pytest.mark.timeout(60)
def test_budget_of_one_scene_serialises():
    sizes = [6, 6]
    srv = _FakeServer(_scenes(sizes), dur=[0.003, 0.003], slots=4, hbm_budget=6)
    res = srv.run([(0.0, i % 2) for i in range(8)])
    res = sorted(res, key=lambda r: r.admitted)
    assert all(u == 6 and b == 1 for _, u, b in srv.log)
    for a, b in zip(res, res[1:]):
        assert b.admitted >= a.done


@pytest.mark.timeout(60)
def test_slot_scratch_is_charged_once():
    """Every slot's decode scratch (sized for the largest scene) is allocated when the server
    is built and charged against the budget then; requests are charged their own buffers."""
    info = lambda n, s: types.SimpleNamespace(n_rows=0, total_len=n, scratch_bytes=s)
    scenes = [serve.Scene(b"", info=info(n, s), host=object()) for n, s in ((3, 1), (2, 2), (7, 1))]
    srv = _FakeServer(scenes, dur=[0.002, 0.002, 0.002], slots=2, hbm_budget=10)
    assert srv.slot_scratch == 4 and srv.in_use == 4
    res = srv.run([(0.0005 * i, i % 3) for i in range(24)])
    assert all(u <= 10 for _, u, _ in srv.log)
    # scene 2 needs 7 + the slots' 4 > 10: refused at once; the others fit one at a time
    for r in res:
        assert r.status == (sgs.E_NOMEM if r.scene == 2 else sgs.OK)
    assert srv.in_use == 4
