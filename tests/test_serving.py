"""Serving loop: admission by memory budget, slot reuse and eviction (CPU,
with a fake backend), and on the GPU that every request's trace is the same
solved alone and in the mix, and equals the oracle's solution."""
import threading
import time

import numpy as np
import pytest

from paper_2512_13619_gb300.serving import Backend, Server


class FakeBackend(Backend):
    def __init__(self, sizes, delay=0.01):
        self.sizes = sizes
        self.delay = delay
        self.live = 0
        self.max_live_bytes = 0
        self.lock = threading.Lock()
        self.active = 0
        self.max_active = 0

    def slot_bytes(self, shape):
        return self.sizes[shape]

    def create_slot(self, shape, lane):
        with self.lock:
            self.live += self.sizes[shape]
            self.max_live_bytes = max(self.max_live_bytes, self.live)
        return {'shape': shape}

    def destroy_slot(self, slot):
        with self.lock:
            self.live -= self.sizes[slot.shape]

    def solve(self, slot, request, lane):
        with self.lock:
            self.active += 1
            self.max_active = max(self.max_active, self.active)
        time.sleep(self.delay)
        with self.lock:
            self.active -= 1
        return request['id'] * 2

    def prepare(self, slot, request, lane):
        time.sleep(self.delay / 2)

    def solve_batch(self, items):
        with self.lock:
            self.batches = getattr(self, 'batches', []) + [len(items)]
        time.sleep(self.delay)
        return [req['id'] * 2 for _, req in items]


def test_batch_mode_solves_prepared_requests_together():
    """Batch mode: lanes prepare, one thread solves every prepared request in
    one call; requests arriving while a batch runs form the next one; the
    memory budget still bounds the resident slots."""
    sizes = {'a': 40, 'b': 30, 'c': 20}
    be = FakeBackend(sizes, delay=0.02)
    srv = Server(be, lanes=4, mem_budget=100, batch=True, max_batch=8)
    shapes = ['a', 'b', 'c', 'c', 'b', 'a', 'c', 'b'] * 4
    reqs = [{'id': i, 'shape': s} for i, s in enumerate(shapes)]
    arr = np.linspace(0.0, 0.15, len(reqs))
    st = srv.run(reqs, arr)
    assert st['completed'] == len(reqs) and st['errors'] == 0
    assert all(srv.results[i] == 2 * i for i in range(len(reqs)))
    assert be.max_live_bytes <= 100
    assert st['batches'] == len(be.batches) and sum(be.batches) == len(reqs)
    assert max(be.batches) > 1                    # requests were solved together
    assert max(be.batches) <= 8


def test_scheduler_budget_reuse_and_eviction():
    sizes = {'a': 40, 'b': 30, 'c': 50}
    be = FakeBackend(sizes)
    srv = Server(be, lanes=3, mem_budget=100)
    shapes = ['a', 'b', 'c', 'a', 'a', 'b', 'c', 'c', 'a', 'b'] * 3
    reqs = [{'id': i, 'shape': s} for i, s in enumerate(shapes)]
    arr = np.linspace(0.0, 0.2, len(reqs))
    st = srv.run(reqs, arr)
    assert st['completed'] == len(reqs) and st['errors'] == 0
    assert all(srv.results[i] == 2 * i for i in range(len(reqs)))
    assert be.max_live_bytes <= 100              # never above the budget
    assert st['max_in_flight'] <= 3 and be.max_active <= 3
    assert st['evictions'] > 0                   # the three shapes do not fit together
    assert st['slot_creations'] < len(reqs)      # slots are reused
    assert st['p99_ms'] >= st['p50_ms'] > 0


def test_request_larger_than_budget_is_an_error():
    be = FakeBackend({'big': 500})
    srv = Server(be, lanes=1, mem_budget=100)
    be.sizes['small'] = 10
    st = srv.run([{'id': 0, 'shape': 'big'}, {'id': 1, 'shape': 'small'}], [0.0, 0.01])
    assert st['errors'] == 1 and srv.errors[0][0] == 0       # rejected, the server keeps serving
    assert st['completed'] == 1 and srv.results[1] == 2


@pytest.mark.gpu
def test_serving_results_alone_equal_mixed_and_oracle():
    from tests.gpu_helpers import need_gpu
    need_gpu()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver
    from paper_2512_13619_gb300.serving import HdgBackend
    from tests.oracle_helpers import OracleSystem
    o = driver.opts(restart=30, rtol=1e-8, pc='bj', inner='fp32', inner_rtol=1e-4, max_iters=3000)

    def inputs(shape, req):
        n, k = shape
        kappa, beta = (0.1, (1.0, 0.0, 0.0)) if req is None else (req['kappa'], req['beta'])
        return W.structured_convdiff_inputs(n, k, kappa, beta)

    rng = np.random.default_rng(5)
    reqs = []
    for i in range(10):
        b = rng.standard_normal(3)
        reqs.append({'id': i, 'shape': (int(rng.integers(3, 5)), int(rng.integers(1, 3))),
                     'kappa': float(10 ** rng.uniform(-2, 0)), 'beta': b / np.linalg.norm(b)})
    alone = {}
    srv1 = Server(HdgBackend(inputs, o), lanes=1, mem_budget=8 << 30)
    for r in reqs:
        srv1.run([r], [0.0])
        alone[r['id']] = srv1.results[r['id']]['trace']
    srv1.close()
    srv = Server(HdgBackend(inputs, o), lanes=4, mem_budget=8 << 30)
    st = srv.run(reqs, np.zeros(len(reqs)))
    srv.close()
    assert st['completed'] == len(reqs) and st['errors'] == 0
    for r in reqs:
        assert np.array_equal(srv.results[r['id']]['trace'], alone[r['id']])
    # one request against the oracle (per-element blocks, direct solve)
    r = reqs[0]
    n, k = r['shape']
    w = W.hex_convdiff(n, k, r['kappa'], r['beta'])
    s = OracleSystem(w)
    x = s.direct().reshape(-1)
    fd = w.face_dirichlet
    xg = srv.results[r['id']]['trace'][fd == 0].reshape(-1)
    assert np.linalg.norm(xg - x) / np.linalg.norm(x) < 1e-5


def test_server_runs_twice_statistics_per_run():
    be = FakeBackend({'a': 10})
    srv = Server(be, lanes=2, mem_budget=100)
    st1 = srv.run([{'id': 0, 'shape': 'a'}], [0.0])
    st2 = srv.run([{'id': 1, 'shape': 'a'}, {'id': 2, 'shape': 'a'}], [0.0, 0.0])
    assert st1['completed'] == 1 and st2['completed'] == 2
    assert st2['slot_creations'] <= 2 and srv.results[2] == 4


def test_warm_creates_slots_within_budget_and_requests_reuse_them():
    be = FakeBackend({'a': 40, 'b': 30, 'c': 50})
    srv = Server(be, lanes=2, mem_budget=100)
    made = srv.warm(['a', 'b', 'c'])
    assert made == 2 and srv.used_bytes == 70          # 'c' does not fit beside 'a' and 'b'
    st = srv.run([{'id': 0, 'shape': 'a'}, {'id': 1, 'shape': 'b'}], [0.0, 0.0])
    assert st['completed'] == 2 and st['slot_creations'] == 2     # only the warm slots
    assert srv.results[0] == 0 and srv.results[1] == 2


@pytest.mark.gpu
@pytest.mark.parametrize('batch', [False, True])
def test_serving_staggered_arrivals_under_budget(batch):
    """Requests arrive while others are on the GPU (arrivals 15 ms apart),
    with fewer lanes than requests and a device-memory budget that holds two
    slots, so requests wait for lanes and slots and idle slots are evicted.
    Every result is bitwise the same as the same request served alone, and
    each meets the mixed-precision contract against the oracle: true FP64
    relative residual <= 1e-8 with the oracle's K, error against its direct
    solve <= cond(K) 1e-8.  In batch mode the prepared requests are solved
    together in one persistent launch (hdg_solve_batch)."""
    from tests.gpu_helpers import need_gpu, sparse_mv
    need_gpu()
    from hdg_inputs import workloads as W
    from paper_2512_13619_gb300 import driver
    from paper_2512_13619_gb300.serving import HdgBackend
    from tests.oracle_helpers import OracleSystem
    o = driver.opts(restart=30, rtol=1e-8, pc='bj', inner='fp32', max_iters=3000, max_outer=-1)

    def inputs(shape, req):
        n, k = shape
        kappa, beta = (0.1, (1.0, 0.0, 0.0)) if req is None else (req['kappa'], req['beta'])
        return W.structured_convdiff_inputs(n, k, kappa, beta)

    rng = np.random.default_rng(7)
    shapes = [(3, 1), (4, 1), (3, 2), (4, 2)]
    reqs = []
    for i in range(12):
        b = rng.standard_normal(3)
        reqs.append({'id': i, 'shape': shapes[i % len(shapes)], 'kappa': float(10 ** rng.uniform(-2, 0)),
                     'beta': b / np.linalg.norm(b)})
    probe = HdgBackend(inputs, o)
    sizes = sorted(probe.slot_bytes(sh) for sh in shapes)
    budget = sizes[-1] + sizes[-2] + 1                   # two slots at most
    alone = {}
    for r in reqs:
        srv1 = Server(HdgBackend(inputs, o), lanes=1, mem_budget=budget, batch=batch)
        srv1.run([r], [0.0])
        alone[r['id']] = srv1.results[r['id']]
        srv1.close()
    srv = Server(HdgBackend(inputs, o), lanes=2, mem_budget=budget, batch=batch)
    st = srv.run(reqs, 0.015 * np.arange(len(reqs)))
    srv.close()
    assert st['completed'] == len(reqs) and st['errors'] == 0
    assert st['evictions'] > 0 and st['max_in_flight'] <= 2     # the budget holds two busy slots
    for r in reqs:
        res = srv.results[r['id']]
        assert np.array_equal(res['trace'], alone[r['id']]['trace']), r['id']
        n, k = r['shape']
        w = W.hex_convdiff(n, k, r['kappa'], r['beta'])
        s = OracleSystem(w)
        xg = res['trace'][w.face_dirichlet == 0].reshape(-1, 1)
        rr = s.r - sparse_mv(s.K, xg)
        assert np.linalg.norm(rr) / np.linalg.norm(s.r) <= 1e-8, r['id']
        xd = s.direct().reshape(-1)
        cond = np.linalg.cond(s.K.toarray())
        assert np.linalg.norm(xg[:, 0] - xd) / np.linalg.norm(xd) <= cond * 1e-8, r['id']
