"""Host logic of the serving loop under a fake backend (no GPU): admission by
footprint, rejection, bands that cover every row exactly once, wave budgets,
and continuous batching (a request that arrives later is served before an
earlier long one finishes)."""
import threading
import time

import pytest

from paper_0801_1500_gb300 import serve as SV


class FakeBackend:
    """Records waves; each wave 'runs' for a time proportional to its rays."""

    def __init__(self, ns_per_ray=0.02):
        self.ns_per_ray = ns_per_ray
        self.waves = []
        self.lock = threading.Lock()

    def upload(self, scene):
        return scene

    def alloc_outputs(self, req):
        return {"rows": []}

    def launch(self, work):
        rays = 0.0
        for _, bd in work:
            bd.req.outputs["rows"].append((bd.row_begin, bd.row_end))
            rays += bd.req.est_rays(bd.row_end - bd.row_begin)
        with self.lock:
            self.waves.append([(bd.req.rid, bd.row_begin, bd.row_end) for _, bd in work])
        return time.perf_counter() + rays * self.ns_per_ray * 1e-9

    def done(self, t):
        return time.perf_counter() >= t

    def wait(self, t):
        while time.perf_counter() < t:
            time.sleep(1e-4)


def req(w, h, spp=4, scene=0, precision=0):
    return SV.Request(scene=scene, camera=None, width=w, height=h, spp=spp, precision=precision)


def test_every_row_rendered_once_and_futures_complete():
    b = FakeBackend()
    srv = SV.Server(b, ["s0", "s1"], hbm_budget=1 << 30, wave_rays=2e6, band_rows=16)
    reqs = [req(100 + 7 * i, 37 + 11 * i, spp=1 + i % 5, scene=i % 2) for i in range(12)]
    futs = [srv.submit(r) for r in reqs]
    for f, r in zip(futs, reqs):
        out = f.result(timeout=30)
        rows = sorted(out["rows"])
        assert rows[0][0] == 0 and rows[-1][1] == r.height
        assert all(a[1] == b_[0] for a, b_ in zip(rows, rows[1:]))   # contiguous, no overlap
    srv.close()
    st = srv.stats()
    assert st["completed"] == 12 and st["p99_s"] >= st["p50_s"]


def test_wave_budgets_respected():
    b = FakeBackend(ns_per_ray=0.0)
    srv = SV.Server(b, ["s"], hbm_budget=1 << 30, wave_rays=1e6, wave_pixels=50000, band_rows=8)
    reqs = [req(300, 200, spp=3) for _ in range(5)]
    for f in [srv.submit(r) for r in reqs]:
        f.result(timeout=30)
    srv.close()
    for wave in b.waves:
        px = sum(300 * (r1 - r0) for _, r0, r1 in wave)
        rays = sum(300 * (r1 - r0) * (1 + 0.6 * 3) for _, r0, r1 in wave)
        assert len(wave) == 1 or (px <= 50000 and rays <= 1e6 + 1)


def test_oversized_request_rejected_and_budget_never_exceeded():
    b = FakeBackend()
    big = req(4000, 4000)                       # 192 MB of FP32 RGB
    srv = SV.Server(b, ["s"], hbm_budget=64 << 20, wave_rays=4e6)
    with pytest.raises(SV.RejectedError):
        srv.submit(big).result(timeout=5)
    # five 40 MB requests against a 64 MB budget: admitted one at a time
    reqs = [req(2000, 1700) for _ in range(5)]
    peak = []
    orig = srv._admit

    def watched():
        orig()
        peak.append(srv.used)
    srv._admit = watched
    for f in [srv.submit(r) for r in reqs]:
        f.result(timeout=60)
    srv.close()
    assert max(peak) <= 64 << 20
    assert srv.stats()["rejected"] == 1


def test_late_small_request_overtakes_long_one():
    # continuous batching: a small request arriving while a long one is being
    # rendered joins the next wave and finishes first
    b = FakeBackend(ns_per_ray=20.0)           # the long request takes ~0.23 s of waves
    srv = SV.Server(b, ["s"], hbm_budget=1 << 30, wave_rays=1e6, band_rows=16, rays_per_s=1e9 / b.ns_per_ray)
    long_req = req(1000, 2000, spp=8)
    f_long = srv.submit(long_req)
    time.sleep(0.03)
    small = req(64, 64, spp=4)
    f_small = srv.submit(small)
    f_small.result(timeout=60)
    assert not f_long.done()
    f_long.result(timeout=120)
    srv.close()
    assert small.t_done < long_req.t_done
    # the small request shared a wave with bands of the long one
    assert any({small.rid, long_req.rid} <= {rid for rid, _, _ in w} for w in b.waves)


def _fake_req(w, h, spp, t_submit):
    r = req(w, h, spp=spp)
    r.t_submit = t_submit
    return r


class _Idle:
    """A backend that never runs: the server's ordering is driven by hand."""

    def upload(self, scene):
        return scene


def _server_without_loop(**kw):
    srv = SV.Server.__new__(SV.Server)
    srv.b = _Idle()
    srv.hbm_budget = 1 << 40
    srv.wave_rays = kw.get("wave_rays", 1e12)
    srv.wave_pixels = kw.get("wave_pixels", 1 << 40)
    srv.band_rows = kw.get("band_rows", 64)
    srv.rays_per_s = kw.get("rays_per_s", 1e10)
    srv.aging = kw.get("aging", 0.1)
    srv.active = []
    return srv


def test_wave_takes_shortest_remaining_work_first():
    # three requests submitted at once: the wave lists the smallest first, and
    # each request's bands together and in row order
    srv = _server_without_loop(band_rows=100)
    big, mid, small = _fake_req(2000, 1000, 64, 0.0), _fake_req(1000, 500, 16, 0.0), _fake_req(256, 256, 4, 0.0)
    srv.active = [big, mid, small]
    wave = srv._build_wave(now=0.0)
    order = []
    for bd in wave:
        if not order or order[-1] is not bd.req:
            order.append(bd.req)
    assert order == [small, mid, big]
    for r in (small, mid, big):
        rows = [(bd.row_begin, bd.row_end) for bd in wave if bd.req is r]
        assert rows[0][0] == 0 and rows[-1][1] == r.height
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))


def test_waiting_time_lifts_a_long_request():
    # a long request (about 1.5 s of work at the assumed rate) that has waited
    # longer than its work / aging goes ahead of a fresh small request; one
    # that has waited less does not
    srv = _server_without_loop(wave_rays=1.0, rays_per_s=1e8, aging=0.1)   # one band a wave
    long_r = _fake_req(1000, 1000, 255, 0.0)      # 1000 * 1000 * (1 + 0.6 * 255) = 1.54e8 rays
    srv.active = [long_r, _fake_req(64, 64, 4, 14.0)]
    assert srv._build_wave(now=14.0)[0].req is not long_r      # waited 14 s < 1.54 s / 0.1
    long_r.rows_issued = 0
    srv.active = [long_r, _fake_req(64, 64, 4, 16.0)]
    assert srv._build_wave(now=16.0)[0].req is long_r          # waited 16 s > 15.4 s
    srv.wave_rays = 1e12
    srv.active = [_fake_req(64, 64, 4, 0.0), _fake_req(64, 64, 4, 0.0)]
    assert len(srv._build_wave(now=0.0)) == 2                   # budgets permitting, all of them
