"""The serving scheduler on the host, with the library's mock device (no GPU):
admission as slots free up, batching of different effects, queue bounds, timeouts."""
import time

import pytest

import oracle as orc
import scenegen as sg


@pytest.fixture(scope="module")
def mrr():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1906_04576_gb300 as m
    return m


def _cfgs(W=4096, H=4096):
    out = {}
    for e in ("ssao", "ssm", "ssgi"):
        c = orc.default_config(e, 4, samples=16, kernel=sg.hemisphere_kernel(16),
                               blocker_taps=sg.disk_taps(32, sg.BLOCKER_SEED), pcf_taps=sg.disk_taps(64, sg.PCF_SEED))
        c.update(max_width=W, max_height=H)
        out[e] = c
    return out


def test_every_request_completes_and_effects_share_batches(mrr):
    srv = mrr.mrr_server_create(_cfgs(), slots=1, mock_device_us=20_000, per_effect=1)
    assert mrr.mrr_server_slots(srv) == 1
    t0 = mrr.mrr_submit(srv, "ssao", (640, 360))     # dispatched at once: the slot is free
    time.sleep(0.005)
    effects = ["ssao", "ssgi", "ssm", "ssao"]         # arrive while the slot is busy
    tickets = [mrr.mrr_submit(srv, e, (640, 360)) for e in effects]
    for t in [t0] + tickets:
        assert mrr.mrr_wait(srv, t, 2_000_000_000) == mrr.MRR_OK
    i0 = mrr.mrr_request_info(srv, t0)
    info = [mrr.mrr_request_info(srv, t) for t in tickets]
    assert all(i["done"] and i["submit_ns"] <= i["start_ns"] <= i["done_ns"] for i in [i0] + info)
    # admitted when the slot freed up, one request per effect packed into one batch
    assert all(i["start_ns"] >= i0["done_ns"] for i in info)
    assert len({i["start_ns"] for i in info[:3]}) == 1
    # the second SSAO repeats an effect: it waits for the next batch
    assert info[3]["start_ns"] >= info[0]["done_ns"]
    for t in [t0] + tickets:
        mrr.mrr_release(srv, t)
    with pytest.raises(mrr.MrrError):
        mrr.mrr_request_info(srv, t0)
    with pytest.raises(mrr.MrrError):   # a released ticket is unknown
        mrr.mrr_release(srv, t0)
    mrr.mrr_server_destroy(srv)


def test_slots_overlap(mrr):
    srv = mrr.mrr_server_create(_cfgs(), slots=3, mock_device_us=50_000, per_effect=1)
    ts = [mrr.mrr_submit(srv, "ssao", (64, 64)) for _ in range(3)]
    for t in ts:
        assert mrr.mrr_wait(srv, t, 2_000_000_000) == mrr.MRR_OK
    info = [mrr.mrr_request_info(srv, t) for t in ts]
    # three slots: all three in flight at the same time
    assert max(i["start_ns"] for i in info) < min(i["done_ns"] for i in info)
    mrr.mrr_server_destroy(srv)


def test_queue_bound_and_timeouts(mrr):
    srv = mrr.mrr_server_create(_cfgs(), slots=1, max_queue=2, mock_device_us=200_000)
    t0 = mrr.mrr_submit(srv, "ssao", (64, 64))
    time.sleep(0.05)                       # t0 is now on the (only) slot
    t1 = mrr.mrr_submit(srv, "ssao", (64, 64))
    t2 = mrr.mrr_submit(srv, "ssao", (64, 64))
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_submit(srv, "ssao", (64, 64))
    assert ei.value.status == mrr.MRR_EBUSY
    assert mrr.mrr_wait(srv, t2, 1_000_000) == mrr.MRR_ETIMEDOUT
    done, _ = mrr.mrr_poll(srv, t2)
    assert not done
    for t in (t0, t1, t2):
        assert mrr.mrr_wait(srv, t, 5_000_000_000) == mrr.MRR_OK
    mrr.mrr_server_destroy(srv)


def test_batches_hold_per_effect_requests_of_each_effect(mrr):
    srv = mrr.mrr_server_create(_cfgs(), slots=1, mock_device_us=20_000, per_effect=2)
    t0 = mrr.mrr_submit(srv, "ssgi", (640, 360))     # occupies the slot
    time.sleep(0.005)
    effects = ["ssao", "ssao", "ssao", "ssgi", "ssm", "ssm"]
    tickets = [mrr.mrr_submit(srv, e, (640, 360)) for e in effects]
    for t in [t0] + tickets:
        assert mrr.mrr_wait(srv, t, 2_000_000_000) == mrr.MRR_OK
    start = [mrr.mrr_request_info(srv, t)["start_ns"] for t in tickets]
    first = {i for i in range(6) if start[i] == min(start)}
    # two SSAO, the SSGI and both SSM go together; the third SSAO waits for the next batch
    assert first == {0, 1, 3, 4, 5}
    assert start[2] > min(start)
    st = mrr.mrr_server_stats(srv)
    assert st["batches"] == 3 and st["completed"] == 7
    assert st["graph_instantiations"] == 0 and st["graph_updates"] == 0   # no device work in mock mode
    mrr.mrr_server_destroy(srv)
    # at most eight requests per batch: 3 effects x 3 is refused
    with pytest.raises(mrr.MrrError) as ei:
        mrr.mrr_server_create(_cfgs(), slots=1, mock_device_us=1000, per_effect=3)
    assert ei.value.status == mrr.MRR_EINVAL


def test_requests_the_server_cannot_take_are_rejected(mrr):
    cfgs = _cfgs(1920, 1080)
    srv = mrr.mrr_server_create({"ssao": cfgs["ssao"]}, slots=1, mock_device_us=1000)
    for effect, size in [("ssgi", (64, 64)), ("ssao", (3840, 2160)), ("ssao", (0, 10))]:
        with pytest.raises(mrr.MrrError) as ei:
            mrr.mrr_submit(srv, effect, size)
        assert ei.value.status == mrr.MRR_EINVAL
    with pytest.raises(mrr.MrrError):
        mrr.mrr_poll(srv, 12345)
    mrr.mrr_server_destroy(srv)
