"""The request loop's admission policy on the host (gsc_server_simulate, no GPU): the budget
is never exceeded, requests on one scene keep their order around encodes, queued evaluations
of one scene merge, idle scenes are evicted least recently used first, requests that can
never run are refused, and a request that waited past the hold time is not overtaken."""
import pytest

from paper_2607_14513_gb300 import gsc

OK, INVALID, BUDGET = 0, 1, 4
GiB = 1 << 30


def P(budget=64 * GiB, slots=4, merge=1, max_views=64, hold_us=10_000_000, encode_slots=0):
    return gsc.ServerParams(budget, slots, merge, max_views, 1, encode_slots, hold_us)


def enc(t, scene, n=16000, fmt=1, service=10.0, t4=0):
    return gsc.SimRequest(0, scene, n, fmt, t4, 0, 0, 0, 1, 1, t, service)


def ev(t, scene, n=16000, V=4, service=1.0, order=2, out_device=1):
    return gsc.SimRequest(1, scene, n, 0, 0, V, order, 1, out_device, 0, t, service)


def _encode_footprint(n=16000, fmt=1):
    res, peak = gsc.simulate(P(), [enc(0.0, 0, n, fmt)])
    keep = (n + 15) // 16 * (128 if fmt == 1 else 256) + 4 * ((n + 15) // 16 * 16) + 12 * n
    return res[0].used_bytes_at_admit, keep


def test_single_encode_then_eval():
    res, peak = gsc.simulate(P(), [enc(0.0, 0), ev(1.0, 0)])
    assert [r.status for r in res] == [OK, OK]
    assert res[1].t_admit_ms == pytest.approx(10.0)          # waits for the encode of its scene
    assert res[1].t_done_ms == pytest.approx(11.0)
    e, keep = _encode_footprint()
    assert peak == e and keep < e


def test_order_around_encodes_on_one_scene():
    tr = [enc(0.0, 0), ev(1.0, 0), enc(2.0, 0, service=5.0), ev(3.0, 0)]
    res, _ = gsc.simulate(P(merge=0), tr)
    assert all(r.status == OK for r in res)
    assert res[1].t_admit_ms == pytest.approx(10.0)          # after encode 0
    assert res[2].t_admit_ms >= res[1].t_admit_ms           # encode 2 starts after eval 1 started
    assert res[3].t_admit_ms >= res[2].t_done_ms            # eval 3 reads the second version


def test_evaluations_merge_up_to_max_views():
    tr = [enc(0.0, 0)] + [ev(1.0 + 0.1 * i, 0, V=16) for i in range(5)]
    res, _ = gsc.simulate(P(max_views=64), tr)
    assert [r.merged for r in res[1:]] == [4, 4, 4, 4, 1]   # 4 x 16 views, then the fifth alone
    res0, _ = gsc.simulate(P(merge=0), tr)
    assert all(r.merged == 1 for r in res0)


def test_no_merge_across_an_encode_or_output_orders():
    tr = [enc(0.0, 0), ev(1.0, 0), ev(1.1, 0, order=0), enc(1.2, 0), ev(1.3, 0)]
    res, _ = gsc.simulate(P(), tr)
    assert [r.merged for r in res[1:3]] == [1, 1]
    assert res[4].merged == 1 and res[4].t_admit_ms >= res[3].t_done_ms


def test_rejections():
    tr = [ev(0.0, 7), enc(1.0, 1), ev(20.0, 1, n=15999)]
    res, _ = gsc.simulate(P(), tr)
    assert res[0].status == INVALID                          # nothing resident, no encode ahead
    assert res[1].status == OK
    assert res[2].status == INVALID                          # resident scene has another size
    e, _ = _encode_footprint()
    res, _ = gsc.simulate(P(budget=e - 1), [enc(0.0, 0)])
    assert res[0].status == BUDGET                           # can never fit


def test_budget_holds_and_lru_eviction():
    e, keep = _encode_footprint()
    budget = e + keep + keep // 2
    tr = [enc(0.0, 0), enc(20.0, 1), ev(40.0, 1), enc(60.0, 2), ev(80.0, 0), ev(81.0, 1), ev(82.0, 2)]
    res, peak = gsc.simulate(P(budget=budget, slots=1), tr)
    assert peak <= budget
    assert all(r.used_bytes_at_admit <= budget for r in res)
    assert res[3].evictions == 1                             # scene 0 (least recently used) gives way
    assert res[4].status == INVALID                          # so its evaluation is refused
    assert res[5].status == OK and res[6].status == OK


def test_budget_random_trace():
    import random
    rnd = random.Random(5)
    e, keep = _encode_footprint(200000, 7)
    budget = 3 * e
    tr, t = [], 0.0
    for i in range(400):
        t += rnd.expovariate(1.0)
        s = rnd.randrange(6)
        if rnd.random() < 0.3:
            tr.append(enc(t, s, n=rnd.choice([16000, 50000, 200000]), fmt=rnd.choice([1, 7]), service=rnd.uniform(1, 8)))
        else:
            tr.append(ev(t, s, n=rnd.choice([16000, 50000, 200000]), V=rnd.randint(1, 32), service=0.5,
                         out_device=rnd.randint(0, 1)))
    res, peak = gsc.simulate(P(budget=budget, slots=3), tr)
    assert peak <= budget
    assert all(r.status in (OK, INVALID) for r in res)
    assert all(r.t_done_ms >= r.t_admit_ms for r in res)
    # at most 3 launches at a time (merged requests share a launch: distinct (admit, done) pairs)
    launches = {(round(r.t_admit_ms, 9), round(r.t_done_ms, 9)) for r in res if r.status == OK}
    pts = sorted([(a, 1) for a, d in launches] + [(d, -1) for a, d in launches], key=lambda x: (x[0], x[1]))
    cur = mx = 0
    for _, d in pts:
        cur += d
        mx = max(mx, cur)
    assert mx <= 3


def test_hold_time_stops_overtaking():
    e, keep = _encode_footprint()
    budget = e + e // 2
    # encode 0 holds e while it runs; encode 1 (another scene) does not fit until it ends;
    # evaluations of scene 2 (resident) need staging memory (host output)
    tr = [enc(0.0, 2, service=1.0), enc(5.0, 0, service=20.0), enc(6.0, 1, service=1.0),
          ev(10.0, 2, V=1, out_device=0), ev(11.0, 2, V=1, out_device=0)]
    res_hold, _ = gsc.simulate(P(budget=budget, slots=2, hold_us=1000, merge=0, encode_slots=2), tr)
    res_free, _ = gsc.simulate(P(budget=budget, slots=2, hold_us=10**9, merge=0, encode_slots=2), tr)
    # without a hold the evaluations overtake the waiting encode; with a 1 ms hold they queue behind it
    assert res_free[3].t_admit_ms < res_free[2].t_admit_ms
    assert res_hold[3].t_admit_ms >= res_hold[2].t_admit_ms


def test_one_slot_runs_requests_one_at_a_time():
    tr = [enc(0.0, 0, service=3.0), enc(0.5, 1, service=3.0), ev(1.0, 0), ev(1.0, 1)]
    res, _ = gsc.simulate(P(slots=1, merge=0), tr)
    spans = sorted((r.t_admit_ms, r.t_done_ms) for r in res)
    for (a0, d0), (a1, d1) in zip(spans, spans[1:]):
        assert a1 >= d0


def test_encode_slots_keep_a_slot_for_evaluations():
    # three long encodes and an evaluation of a resident scene; with 3 slots and the default
    # of n_slots - 1 encode slots, the evaluation does not wait for an encode to finish
    tr = [enc(0.0, 9, service=1.0), enc(2.0, 0, service=50.0), enc(2.1, 1, service=50.0), enc(2.2, 2, service=50.0),
          ev(3.0, 9)]
    res, _ = gsc.simulate(P(slots=3), tr)
    assert res[4].t_admit_ms == pytest.approx(3.0)
    assert res[3].t_admit_ms >= res[1].t_done_ms - 1e-9      # the third encode waited for an encode slot
    res_all, _ = gsc.simulate(P(slots=3, encode_slots=3), tr)
    assert res_all[4].t_admit_ms >= 52.0 - 1e-9              # all slots busy with encodes
