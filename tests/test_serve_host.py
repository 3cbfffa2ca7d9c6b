"""Host logic of the server (no GPU): admission by footprint, patterns that
another worker runs, and continuous batching of same-pattern requests."""
import collections

from paper_1203_2742_gb300.serve import Request, pick


def q(*reqs):
    return collections.deque(reqs)


def fp(req):
    return 10 * req.m


def test_fifo_and_batching_of_same_pattern_and_kind():
    a = Request("hessian", 0, 0.0, m=3, rid=0)
    b = Request("gradient", 0, 0.1, rid=1)
    c = Request("hessian", 0, 0.2, m=4, rid=2)
    d = Request("hessian", 1, 0.3, m=2, rid=3)
    e = Request("inv_hessian", 0, 0.4, m=1, rid=4)
    group, need, rest = pick(q(a, b, c, d, e), lambda p: False, fp, 0, 1000, True, 64)
    assert [r.rid for r in group] == [0, 2]  # a and c: same kind, same pattern
    assert need == 70
    assert [r.rid for r in rest] == [1, 3, 4]  # the others keep their order


def test_no_batching_takes_one():
    a = Request("hessian", 0, 0.0, m=3, rid=0)
    c = Request("hessian", 0, 0.2, m=4, rid=2)
    group, _, rest = pick(q(a, c), lambda p: False, fp, 0, 1000, False, 64)
    assert [r.rid for r in group] == [0] and [r.rid for r in rest] == [2]


def test_batch_limit_on_right_hand_sides():
    reqs = [Request("hessian", 0, 0.1 * i, m=20, rid=i) for i in range(5)]
    group, need, rest = pick(q(*reqs), lambda p: False, fp, 0, 10 ** 6, True, 64)
    assert [r.rid for r in group] == [0, 1, 2]  # 60 <= 64 < 80
    assert [r.rid for r in rest] == [3, 4]


def test_busy_pattern_is_skipped_not_waited_for():
    a = Request("hessian", 0, 0.0, m=1, rid=0)
    b = Request("factor", 1, 0.1, rid=1)
    group, _, rest = pick(q(a, b), lambda p: p == 0, fp, 0, 1000, True, 64)
    assert [r.rid for r in group] == [1]
    assert [r.rid for r in rest] == [0]
    assert pick(q(a), lambda p: p == 0, fp, 0, 1000, True, 64) is None


def test_budget_admission():
    big = Request("hessian", 0, 0.0, m=50, rid=0)   # 500 bytes
    small = Request("hessian", 1, 0.1, m=1, rid=1)  # 10 bytes
    # something in flight: the big one does not fit, the small one does
    group, need, rest = pick(q(big, small), lambda p: False, fp, 600, 1000, True, 64)
    assert [r.rid for r in group] == [1] and need == 10 and [r.rid for r in rest] == [0]
    # nothing in flight: a request larger than the budget is still admitted
    group, need, _ = pick(q(big), lambda p: False, fp, 0, 100, True, 64)
    assert [r.rid for r in group] == [0] and need == 500
    assert pick(q(big), lambda p: False, fp, 600, 1000, True, 64) is None


def test_take_release_with_threads_on_host():
    """The server's own _take/_release with worker threads and no device:
    every request is taken exactly once, same-pattern Hessians are batched,
    and no two workers hold one pattern at the same time."""
    import threading
    import time
    from paper_1203_2742_gb300.serve import PatternState, Server

    srv = Server.__new__(Server)  # host fields only: no factors, no device memory
    srv.batching = True
    srv.max_batch_rhs = 64
    srv.states = [PatternState(sym=None, x=None, s=None) for _ in range(3)]
    srv.budget = 10 ** 9
    srv.in_use = 0
    srv.cv = threading.Condition()
    srv.queue = collections.deque()
    srv.closed = False
    srv.footprint = lambda req: 8 * req.m
    reqs = [Request("hessian" if i % 2 else "factor", i % 3, 0.0, m=1 + i % 4, rid=i) for i in range(60)]
    for r in reqs:
        srv.queue.append(r)
    taken, holders, lock, errors = [], {}, threading.Lock(), []

    def worker():
        while True:
            group, need = srv._take()
            if group is None:
                return
            p = group[0].pattern
            with lock:
                if holders.get(p):
                    errors.append(p)
                holders[p] = True
                taken.extend(group)
            time.sleep(0.001)
            with lock:
                holders[p] = False
            srv._release(need, p)

    ts = [threading.Thread(target=worker) for _ in range(4)]
    for t in ts:
        t.start()
    srv.close = lambda: None
    with srv.cv:
        srv.closed = True
        srv.cv.notify_all()
    for t in ts:
        t.join(timeout=30)
    assert not errors
    assert sorted(r.rid for r in taken) == list(range(60))
    assert srv.in_use == 0 and not any(s.busy for s in srv.states)
