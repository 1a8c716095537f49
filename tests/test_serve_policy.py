"""Host-side scheduling of the serving loop (`Server.serve_streams`), on the
CPU: the GPU pipeline of a request is replaced by a fake whose completion
event fires after a simulated service time, and the real admission loop runs
on a real request trace.  Checks the properties the design relies on:
admission by free slots (workspace memory), one heavy (stereo) request at a
time in arrival order while lighter ones are admitted, high-priority streams
for light requests only, and every request completing."""
import time

import pytest

from paper_2504_12811_gb300 import scenes, serve

HD = 1920 * 1080


class _Done:
    def __init__(self, t):
        self.t = t

    def query(self):
        return time.perf_counter() >= self.t


def _fake_server(n_slots, service_s):
    srv = serve.Server.__new__(serve.Server)
    srv.slots = [object() for _ in range(n_slots)]
    log = {"launch": [], "inflight": set(), "max_views": 0, "heavy_overlap": 0, "busy": set()}

    def launch(req, slots, urgent=False):
        px = sum(c.width * c.height for c in req.cams)
        assert not (set(map(id, slots)) & log["busy"]), "a slot was handed out twice"
        log["busy"] |= set(map(id, slots))
        heavy_now = [r for r in log["inflight"] if r[1] > HD]
        if px > HD and heavy_now:
            log["heavy_overlap"] += 1
        entry = (req.rid, px, tuple(map(id, slots)))
        log["inflight"].add(entry)
        log["launch"].append((req.rid, req.arrival, px, urgent, len(slots)))
        log["max_views"] = max(log["max_views"], sum(len(r[2]) for r in log["inflight"]))
        done = _Done(time.perf_counter() + service_s(px))

        class Tracked:
            def query(self_inner):
                ok = done.query()
                if ok and entry in log["inflight"]:
                    log["inflight"].discard(entry)
                    log["busy"] -= set(entry[2])
                return ok
        return Tracked()

    srv._launch_request = launch
    return srv, log


@pytest.mark.parametrize("n_slots", [3, 9])
def test_policy_heavy_serial_light_urgent(n_slots):
    trace = scenes.serving_trace(rate_hz=150.0, duration_s=0.4, seed=5)
    assert any(len(r.cams) == 2 for r in trace) and any(len(r.cams) == 1 for r in trace)
    srv, log = _fake_server(n_slots, lambda px: 2e-3 + px * 2e-9)   # ~2 ms + 14 ms for a stereo request
    lat = srv.serve_streams(trace, urgent_pixels=HD, heavy_pixels=HD)
    assert len(lat) == len(trace) and all(v >= 0 for v in lat)
    launched = log["launch"]
    assert sorted(r[0] for r in launched) == sorted(r.rid for r in trace)
    # never more views in flight than slots, never a slot handed out twice
    assert log["max_views"] <= n_slots
    # heavy (stereo) requests one at a time, in arrival order
    assert log["heavy_overlap"] == 0
    heavy = [(arr, rid) for rid, arr, px, _, _ in launched if px > HD]
    assert heavy == sorted(heavy)
    # high-priority streams exactly for the requests up to 1920x1080
    assert all(urgent == (px <= HD) for _, _, px, urgent, _ in launched)


def test_heavy_limit_is_what_serialises_stereo_requests():
    # the same trace without the heavy limit does overlap stereo requests, so
    # the check above is not vacuous
    trace = scenes.serving_trace(rate_hz=150.0, duration_s=0.4, seed=5)
    srv, log = _fake_server(9, lambda px: 2e-3 + px * 6e-9)    # ~44 ms per stereo request
    srv.serve_streams(trace, urgent_pixels=HD)
    assert log["heavy_overlap"] > 0


def test_policy_without_limits_is_arrival_order_fifo():
    trace = scenes.serving_trace(rate_hz=150.0, duration_s=0.3, seed=6)
    srv, log = _fake_server(4, lambda px: 1e-3 + px * 1e-9)
    lat = srv.serve_streams(trace)
    assert len(lat) == len(trace)
    arrivals = [arr for _, arr, _, _, _ in log["launch"]]
    assert arrivals == sorted(arrivals)                      # admission in arrival order
    assert not any(urgent for _, _, _, urgent, _ in log["launch"])
    assert log["max_views"] <= 4


def test_latency_summary():
    s = serve.latency_summary([0.001, 0.002, 0.003, 0.100], 2.0, 6)
    assert s["requests"] == 4 and s["requests_per_s"] == 2.0 and s["views_per_s"] == 3.0
    assert s["max_ms"] == pytest.approx(100.0) and s["p50_ms"] == pytest.approx(2.5)
