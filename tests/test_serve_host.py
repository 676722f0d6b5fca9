"""Admission controller of the serving loop, host only (fake scenes, fake estimates, no GPU)."""
from paper_2508_05343_b300.serve import AdmissionController, Request, SlotLimits, tiles_of


def make_ac(limits=None, cap=1 << 40, resident=0, pairs=1000):
    lim = limits or SlotLimits(max_views=4, max_prims=1000, max_tiles=10_000, max_pixels=10**7, pair_capacity=10**6)
    return AdmissionController(lim, scene_prims=[100, 400, 900, 2000], pair_estimate=lambda s, w, h: pairs,
                               bytes_per_view=lambda w, h: 12 * w * h, hbm_cap_bytes=cap, resident_bytes=resident)


def req(i, scene=0, w=64, h=48, t=0.0):
    return Request(i, t, scene, w, h, 0.0, 0.0)


def test_batches_follow_arrival_order_and_view_limit():
    ac = make_ac()
    for i in range(10):
        ac.submit(req(i))
    b, _ = ac.next_batch()
    assert [r.rid for r in b] == [0, 1, 2, 3]
    b, _ = ac.next_batch(max_views=2)
    assert [r.rid for r in b] == [4, 5]


def test_primitive_capacity_stops_the_batch_without_reordering():
    ac = make_ac()
    for i, s in enumerate([1, 1, 0, 0]):          # 400 + 400 + 100 + 100 primitives
        ac.submit(req(i, scene=s))
    b, _ = ac.next_batch()
    assert [r.rid for r in b] == [0, 1, 2, 3]
    for i, s in enumerate([2, 0, 0]):             # 900, then 100 would exceed 1000? 900 + 100 = 1000 fits
        ac.submit(req(10 + i, scene=s))
    b, _ = ac.next_batch()
    assert [r.rid for r in b] == [10, 11]          # the third (another 100) no longer fits
    assert [r.rid for r in ac.pending] == [12]


def test_requests_that_never_fit_are_refused():
    ac = make_ac()
    ac.submit(req(0, scene=3))                    # 2000 primitives > slot capacity
    ac.submit(req(1))
    b, _ = ac.next_batch()
    assert [r.rid for r in b] == [1] and ac.refused == 1


def test_pair_estimate_and_tile_limits():
    lim = SlotLimits(max_views=8, max_prims=10**6, max_tiles=3 * tiles_of(64, 48), max_pixels=10**7, pair_capacity=2500)
    ac = make_ac(limits=lim, pairs=1000)
    for i in range(5):
        ac.submit(req(i))
    b, _ = ac.next_batch()
    assert len(b) == 2                              # 3 x 1000 pairs would exceed 2500
    lim2 = SlotLimits(max_views=8, max_prims=10**6, max_tiles=2 * tiles_of(64, 48), max_pixels=10**7,
                      pair_capacity=10**6)
    ac2 = make_ac(limits=lim2)
    for i in range(5):
        ac2.submit(req(i))
    assert len(ac2.next_batch()[0]) == 2            # tile limit


def test_memory_ledger_admits_as_memory_frees_up():
    per_view = 12 * 64 * 48
    ac = make_ac(cap=1000 + 2 * per_view, resident=1000)
    for i in range(4):
        ac.submit(req(i))
    b1, m1 = ac.next_batch()
    assert len(b1) == 2 and m1 == 2 * per_view
    b2, m2 = ac.next_batch()
    assert b2 == [] and m2 == 0                     # cap reached while b1 is in flight
    ac.release(m1)
    b3, _ = ac.next_batch()
    assert [r.rid for r in b3] == [2, 3]


def test_requeue_keeps_order():
    ac = make_ac()
    for i in range(6):
        ac.submit(req(i))
    b, m = ac.next_batch()
    ac.release(m)
    ac.requeue_front(b)
    assert [r.rid for r in ac.pending] == [0, 1, 2, 3, 4, 5]
