"""Continuous-batching serving loop for HDG solves on one GPU.

Requests (one HDG problem each) arrive over time.  A request is admitted as
soon as a lane is free and its problem fits the device-memory budget; up to
`lanes` requests run at once, each on its own CUDA stream, so their
condensation, assembly and GMRES kernels overlap on the device.  A *slot* is
a resident problem of one mesh shape: its condensed blocks, preconditioner
factors and Krylov basis stay allocated after a request finishes and are
reused by the next request of the same shape; idle slots of other shapes are
evicted when the budget requires it.  Latency is measured from a request's
arrival to the moment its trace is back in host memory.

With `batch=True` the lanes only prepare their requests (condensation,
assembly, preconditioner set-up on their streams), and one batching thread
solves every prepared request together in ONE persistent launch
(hdg_solve_batch): requests of different meshes and orders share the
launches of every GMRES phase instead of each running its own iterations.
Prepared requests that arrive while a batch runs form the next batch.

Every numerical step runs in libhdg.so; this module only schedules.  The
scheduler is independent of the backend (`Backend`), so its admission and
eviction logic can be exercised without a GPU.
"""
import collections
import threading
import time

import numpy as np


class Backend:
    """What the scheduler needs from a solver: slot sizes, slot creation and
    destruction, and one solve of a request on a slot (on the lane's stream)."""

    def slot_bytes(self, shape):
        raise NotImplementedError

    def create_slot(self, shape, lane):
        raise NotImplementedError

    def destroy_slot(self, slot):
        raise NotImplementedError

    def solve(self, slot, request, lane):
        """Returns a result object (e.g. the trace) once it is on the host."""
        raise NotImplementedError

    def prepare(self, slot, request, lane):
        """Batch mode: everything before the solve, finished when it returns."""
        raise NotImplementedError

    def solve_batch(self, items):
        """Batch mode: solve the prepared (slot, request) pairs together;
        returns one result per pair, on the host."""
        raise NotImplementedError

    def lane_setup(self, lane):
        pass


class Slot:
    def __init__(self, shape, handle, nbytes):
        self.shape = shape
        self.handle = handle
        self.nbytes = nbytes
        self.busy = False
        self.last_used = 0.0
        self.uses = 0


class Server:
    def __init__(self, backend, lanes=4, mem_budget=64 << 30, batch=False, max_batch=64):
        self.backend = backend
        self.lanes = lanes
        self.mem_budget = mem_budget
        self.batch = batch
        self.max_batch = max_batch
        self.prepared = collections.deque()
        self.preparing = 0
        self.batches = 0
        self.batch_sizes = []
        self.slots = []
        self.used_bytes = 0
        self.cv = threading.Condition()
        self.ready = collections.deque()
        self.results = {}
        self.t_done = {}
        self.errors = []
        self.evictions = 0
        self.creations = 0
        self.max_in_flight = 0
        self.in_flight = 0

    # ---------------------------------------------------------------- slots
    def _acquire_slot(self, shape):
        """Called with self.cv held.  Returns an idle slot of `shape`
        (creating one within the budget, evicting idle slots of other shapes
        if needed) or None when the request has to wait."""
        for sl in self.slots:
            if sl.shape == shape and not sl.busy:
                sl.busy = True
                return sl
        need = self.backend.slot_bytes(shape)
        if need > self.mem_budget:
            raise MemoryError('request of shape %s needs %d bytes > budget %d' % (shape, need, self.mem_budget))
        while self.used_bytes + need > self.mem_budget:
            idle = [s for s in self.slots if not s.busy]
            if not idle:
                return None
            victim = min(idle, key=lambda s: s.last_used)
            self.slots.remove(victim)
            self.used_bytes -= victim.nbytes
            self.backend.destroy_slot(victim)
            self.evictions += 1
        sl = Slot(shape, None, need)
        sl.busy = True
        self.slots.append(sl)
        self.used_bytes += need
        self.creations += 1
        return sl

    # ---------------------------------------------------------------- lanes
    def _lane(self, lane):
        self.backend.lane_setup(lane)
        while True:
            with self.cv:
                while True:
                    if not self.ready and self._closed:
                        return
                    if self.ready:
                        req = self.ready[0]
                        try:
                            sl = self._acquire_slot(req['shape'])
                        except MemoryError as exc:   # can never fit: reject it
                            self.ready.popleft()
                            self.errors.append((req['id'], repr(exc)))
                            self.cv.notify_all()
                            continue
                        if sl is not None:
                            self.ready.popleft()
                            break
                    self.cv.wait(timeout=0.01)
                self.in_flight += 1
                self.max_in_flight = max(self.max_in_flight, self.in_flight)
                if self.batch:
                    self.preparing += 1
            if self.batch:
                self._prepare(req, sl, lane)
                continue
            try:
                if sl.handle is None:
                    sl.handle = self.backend.create_slot(sl.shape, lane)
                res = self.backend.solve(sl.handle, req, lane)
                t = time.perf_counter()
                with self.cv:
                    self.results[req['id']] = res
                    self.t_done[req['id']] = t
            except Exception as exc:  # recorded, the server keeps serving
                with self.cv:
                    self.errors.append((req['id'], repr(exc)))
            finally:
                with self.cv:
                    sl.busy = False
                    sl.last_used = time.perf_counter()
                    sl.uses += 1
                    self.in_flight -= 1
                    self.cv.notify_all()

    def _release(self, sl):
        """Called with self.cv held."""
        sl.busy = False
        sl.last_used = time.perf_counter()
        sl.uses += 1
        self.in_flight -= 1
        self.cv.notify_all()

    def _prepare(self, req, sl, lane):
        ok = False
        try:
            if sl.handle is None:
                sl.handle = self.backend.create_slot(sl.shape, lane)
            self.backend.prepare(sl.handle, req, lane)
            ok = True
        except Exception as exc:
            with self.cv:
                self.errors.append((req['id'], repr(exc)))
        with self.cv:
            self.preparing -= 1
            if ok:
                self.prepared.append((req, sl))
            else:
                self._release(sl)
            self.cv.notify_all()

    def _batcher(self):
        """Batch mode: solve whatever is prepared, together, until closed."""
        while True:
            with self.cv:
                while not self.prepared:
                    if self._closed and not self.ready and self.preparing == 0 and self.lanes_done == self.lanes:
                        return
                    self.cv.wait(timeout=0.01)
                items = []
                while self.prepared and len(items) < self.max_batch:
                    items.append(self.prepared.popleft())
            try:
                res = self.backend.solve_batch([(sl.handle, req) for req, sl in items])
                t = time.perf_counter()
                with self.cv:
                    for (req, _), r in zip(items, res):
                        self.results[req['id']] = r
                        self.t_done[req['id']] = t
                    self.batches += 1
                    self.batch_sizes.append(len(items))
            except Exception as exc:
                with self.cv:
                    for req, _ in items:
                        self.errors.append((req['id'], repr(exc)))
            finally:
                with self.cv:
                    for _, sl in items:
                        self._release(sl)

    def _lane_main(self, lane):
        try:
            self._lane(lane)
        finally:
            with self.cv:
                self.lanes_done += 1
                self.cv.notify_all()

    def run(self, requests, arrivals):
        """Serve `requests` (dicts with 'id' and 'shape'), request i arriving
        arrivals[i] seconds after the start.  Returns the statistics."""
        self._closed = False
        self.lanes_done = 0
        threads = [threading.Thread(target=self._lane_main, args=(i,), daemon=True) for i in range(self.lanes)]
        if self.batch:
            threads.append(threading.Thread(target=self._batcher, daemon=True))
        for th in threads:
            th.start()
        t0 = time.perf_counter()
        t_arr = {}
        for req, a in sorted(zip(requests, arrivals), key=lambda x: x[1]):
            now = time.perf_counter() - t0
            if a > now:
                time.sleep(a - now)
            with self.cv:
                t_arr[req['id']] = t0 + a
                self.ready.append(req)
                self.cv.notify_all()
        with self.cv:
            self._closed = True
            self.cv.notify_all()
        for th in threads:
            th.join()
        ids = [i for i in t_arr if i in self.t_done]      # this run's completed requests
        lat = np.array([self.t_done[i] - t_arr[i] for i in ids])
        done = len(ids)
        span = (max(self.t_done[i] for i in ids) - t0) if done else 0.0
        return {
            'completed': done, 'errors': sum(1 for i, _ in self.errors if i in t_arr), 'lanes': self.lanes,
            'p50_ms': float(np.percentile(lat, 50) * 1e3) if done else None,
            'p99_ms': float(np.percentile(lat, 99) * 1e3) if done else None,
            'mean_ms': float(lat.mean() * 1e3) if done else None,
            'solves_per_s': done / span if span > 0 else None,
            'slot_creations': self.creations, 'evictions': self.evictions,
            'max_in_flight': self.max_in_flight, 'resident_bytes': self.used_bytes,
            'batches': self.batches,
            'mean_batch': float(np.mean(self.batch_sizes)) if self.batch_sizes else None,
        }

    def warm(self, shapes, per_shape=1):
        """Create `per_shape` idle slots for each shape before requests arrive
        (a server that knows its meshes), as far as the budget allows; returns
        the number created.  Slots are created in the order given."""
        made = 0
        for _ in range(per_shape):
            for sh in shapes:
                need = self.backend.slot_bytes(sh)
                if self.used_bytes + need > self.mem_budget:
                    continue
                sl = Slot(sh, self.backend.create_slot(sh, 0), need)
                self.slots.append(sl)
                self.used_bytes += need
                self.creations += 1
                made += 1
        return made

    def close(self):
        for sl in self.slots:
            if sl.handle is not None:
                self.backend.destroy_slot(sl)
        self.slots = []
        self.used_bytes = 0


# ------------------------------------------------------------ HDG backend
class HdgBackend(Backend):
    """Solves HDG convection-diffusion requests through the C ABI.

    `inputs(shape, request)` returns (mesh dict, blocks, strides, uhatD) for
    a request: the mesh arrays of the shape and the element blocks, shared
    (stride 0) where all elements are identical.  opts: hdg_solver_opts."""

    def __init__(self, inputs, opts, device=0, nrhs=1):
        import torch
        from . import _lib as L
        from . import driver
        self.L, self.driver, self.torch = L, driver, torch
        self.inputs = inputs
        self.opts = opts
        self.device = device
        self.nrhs = nrhs
        self.streams = {}
        self._mesh_cache = {}

    def lane_setup(self, lane):
        self.torch.cuda.set_device(self.device)
        self.streams[lane] = self.torch.cuda.Stream(device=self.device)

    def _mesh(self, shape):
        if shape not in self._mesh_cache:
            self._mesh_cache[shape] = self.inputs(shape, None)[0]
        return self._mesh_cache[shape]

    def slot_bytes(self, shape):
        m = self._mesh(shape)
        mesh = self.L.hdg_mesh()
        ef = np.ascontiguousarray(m['elem_face'], np.int32)
        fe = np.ascontiguousarray(m['face_elem'], np.int32)
        fd = np.ascontiguousarray(m['face_dirichlet'], np.uint8)
        mesh.dim, mesh.n_lfe, mesh.M, mesh.PE, mesh.PF = m['dim'], m['n_lfe'], m['M'], m['PE'], m['PF']
        mesh.n_elem, mesh.n_face = ef.shape[0], fd.shape[0]
        mesh.elem_face, mesh.face_elem, mesh.face_dirichlet = ef.ctypes.data, fe.ctypes.data, fd.ctypes.data
        return int(self.L.hdg_workspace_bytes(mesh, self.nrhs, self.opts))

    def create_slot(self, shape, lane):
        m = self._mesh(shape)
        return self.driver.Problem(m['dim'], m['n_lfe'], m['M'], m['PE'], m['PF'], m['elem_face'],
                                   m['face_elem'], m['face_dirichlet'], self.nrhs, self.device)

    def destroy_slot(self, slot):
        if slot.handle is not None:
            slot.handle.close()

    def prepare(self, prob, request, lane):
        L, check = self.L, self.driver.check
        st = self.streams[lane].cuda_stream
        _, blocks, strides, uD = self.inputs(request['shape'], request)
        check(L.hdg_condense_strided(prob.h, 0, prob.n_elem, [blocks[k] for k in self.driver.BLOCK_NAMES],
                                     strides, 0, st), 'condense')
        check(L.hdg_set_dirichlet(prob.h, uD, 0, st), 'dirichlet')
        check(L.hdg_assemble(prob.h, self.opts, st), 'assemble')
        check(L.hdg_setup_precond(prob.h, self.opts, None, st), 'setup')
        self.streams[lane].synchronize()

    def solve_batch(self, items):
        L, check = self.L, self.driver.check
        if not hasattr(self, '_bstream'):
            self.torch.cuda.set_device(self.device)
            self._bstream = self.torch.cuda.Stream(device=self.device)
        st = self._bstream.cuda_stream
        s, infos = L.hdg_solve_batch([prob.h for prob, _ in items], self.opts, st)
        check(s, 'solve_batch')
        out = []
        for (prob, _), info in zip(items, infos):
            tr = np.empty((prob.n_face, prob.b, prob.R))
            check(L.hdg_get_trace(prob.h, tr, 0, st), 'trace')
            out.append({'trace': tr, 'iters': info.iters, 'outer': 0, 'rel': info.rel_resid})
        return out

    def solve(self, prob, request, lane):
        L, check = self.L, self.driver.check
        st = self.streams[lane].cuda_stream
        _, blocks, strides, uD = self.inputs(request['shape'], request)
        check(L.hdg_condense_strided(prob.h, 0, prob.n_elem, [blocks[k] for k in self.driver.BLOCK_NAMES],
                                     strides, 0, st), 'condense')
        check(L.hdg_set_dirichlet(prob.h, uD, 0, st), 'dirichlet')
        check(L.hdg_assemble(prob.h, self.opts, st), 'assemble')
        check(L.hdg_setup_precond(prob.h, self.opts, None, st), 'setup')
        info = L.hdg_solve_info()
        s = L.hdg_solve(prob.h, self.opts, st, info)
        check(s, 'solve')
        out = np.empty((prob.n_face, prob.b, prob.R))
        check(L.hdg_get_trace(prob.h, out, 0, st), 'trace')
        return {'trace': out, 'iters': info.iters, 'outer': info.outer, 'rel': info.rel_resid}
