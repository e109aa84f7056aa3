"""Thin driver over the C ABI: holds one hdg_problem and sequences the calls
(condense -> set_dirichlet -> assemble -> setup_precond -> solve -> recover)
for a problem given as numpy arrays.  Marshalling only; every numerical step
runs in libhdg.so.  Device vectors are torch CUDA tensors."""
import numpy as np

from . import _lib as L

_PC = {'none': L.HDG_PC_NONE, 'bj': L.HDG_PC_BJ, 'asm': L.HDG_PC_ASM}
_POLY = {None: L.HDG_POLY_NONE, 'none': L.HDG_POLY_NONE, 'gmres': L.HDG_POLY_GMRES, 'chebyshev': L.HDG_POLY_CHEBYSHEV}
_PREC = {'fp64': L.HDG_FP64, 'fp32': L.HDG_FP32, 'bf16': L.HDG_BF16}
_ORTH = {'cgs': L.HDG_ORTH_CGS, 'mgs': L.HDG_ORTH_MGS, 'cgs2': L.HDG_ORTH_CGS2}


class HdgError(RuntimeError):
    def __init__(self, status, what=''):
        msg = '%s: %s' % (what, L.hdg_status_str(status))
        if status == L.HDG_ERR_CUDA:
            msg += ' [%s]' % L.hdg_last_error()
        super().__init__(msg)
        self.status = status


def check(status, what=''):
    if status != L.HDG_OK:
        raise HdgError(status, what)


def opts(restart=50, max_iters=1000, rtol=1e-10, orth='cgs', pc='bj', poly=None, degree=0, inner='fp64',
         poly_prec='fp32', inner_rtol=1e-4, max_outer=20):
    o = L.hdg_solver_opts()
    o.restart, o.max_iters, o.rtol = restart, max_iters, rtol
    o.orth, o.pc, o.poly, o.poly_degree = _ORTH[orth], _PC[pc], _POLY[poly], degree
    o.inner_prec, o.poly_prec, o.inner_rtol, o.max_outer = _PREC[inner], _PREC[poly_prec], inner_rtol, max_outer
    return o


BLOCK_NAMES = ('Me', 'Bd', 'Cd', 'D', 'E', 'F', 'G', 'H', 'J', 'ru', 'ruh')


def hex_geometry_inputs(w, e0=0, count=None):
    """(verts (count, 8, 3), face_perm (count, 6, P_F) int32, nquad) of a
    hexahedral workload, the geometry inputs of hdg_condense_hex."""
    count = w.n_elem - e0 if count is None else count
    m = w.mesh
    verts = np.ascontiguousarray(m.verts[m.elems[e0:e0 + count]], dtype=np.float64)
    perm = np.ascontiguousarray(w.perm[e0:e0 + count], dtype=np.int32)
    nquad = int(round(len(w.ref.vol_wts) ** (1.0 / 3.0)))
    assert nquad ** 3 == len(w.ref.vol_wts)
    return verts, perm, nquad


class Problem:
    def __init__(self, dim, n_lfe, M, PE, PF, elem_face, face_elem, face_dirichlet, nrhs=1, device=0):
        self._ef = np.ascontiguousarray(elem_face, dtype=np.int32)
        self._fe = np.ascontiguousarray(face_elem, dtype=np.int32)
        self._fd = np.ascontiguousarray(face_dirichlet, dtype=np.uint8)
        m = L.hdg_mesh()
        m.dim, m.n_lfe, m.M, m.PE, m.PF = dim, n_lfe, M, PE, PF
        m.n_elem, m.n_face = self._ef.shape[0], self._fd.shape[0]
        m.elem_face, m.face_elem, m.face_dirichlet = L.ptr(self._ef), L.ptr(self._fe), L.ptr(self._fd)
        self.mesh = m
        self.dim, self.n_lfe, self.M, self.PE, self.PF, self.R = dim, n_lfe, M, PE, PF, nrhs
        self.n_elem, self.n_face = m.n_elem, m.n_face
        self.b = M * PF
        self.n_free = int((self._fd == 0).sum())
        self.n_dof = self.n_free * self.b
        self.device = device
        st, h = L.hdg_problem_create(m, nrhs, device)
        check(st, 'hdg_problem_create')
        self.h = h

    @classmethod
    def from_workload(cls, w, device=0):
        return cls(w.D, w.n_lfe, w.M, w.PE, w.PF, w.mesh.elem_face, w.mesh.face_elem, w.face_dirichlet, w.R, device)

    def close(self):
        if getattr(self, 'h', None):
            L.hdg_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def condense(self, blocks, e0=0, on_device=False, stream=None):
        arrs = [blocks[k] for k in BLOCK_NAMES]
        if not on_device:
            arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in arrs]
        count = arrs[0].shape[0]
        check(L.hdg_condense(self.h, e0, count, *arrs, on_device, stream), 'hdg_condense')

    def condense_hex(self, w, e0=0, count=None, stream=None):
        """Generate the element blocks of a hexahedral workload on the device
        and condense them (hdg_condense_hex); host inputs: the vertices, the
        face permutations, the physics tensors and the load vectors."""
        count = w.n_elem - e0 if count is None else count
        verts, perm, nquad = hex_geometry_inputs(w, e0, count)
        ph, keep = L.physics(w.phys.Cq, w.phys.Cu, w.phys.Rr, w.phys.tau)
        b = w.blocks(e0, e0 + count)
        ru = np.ascontiguousarray(b['ru'], dtype=np.float64)
        ruh = np.ascontiguousarray(b['ruh'], dtype=np.float64)
        check(L.hdg_condense_hex(self.h, e0, count, nquad, verts, perm, ph, ru, ruh, 0, stream), 'hdg_condense_hex')

    def set_dirichlet(self, uhatD, on_device=False, stream=None):
        if not on_device:
            uhatD = np.ascontiguousarray(uhatD, dtype=np.float64)
        check(L.hdg_set_dirichlet(self.h, uhatD, on_device, stream), 'hdg_set_dirichlet')

    def assemble(self, o, stream=None):
        check(L.hdg_assemble(self.h, o, stream), 'hdg_assemble')

    def setup_precond(self, o, v0=None, stream=None):
        dv = None
        if v0 is not None:
            import torch
            dv = torch.as_tensor(np.ascontiguousarray(v0, dtype=np.float64)).to('cuda:%d' % self.device)
        check(L.hdg_setup_precond(self.h, o, dv, stream), 'hdg_setup_precond')

    def solve(self, o, stream=None):
        info = L.hdg_solve_info()
        st = L.hdg_solve(self.h, o, stream, info)
        return st, info

    def trace(self, stream=None):
        out = np.empty((self.n_face, self.b, self.R))
        check(L.hdg_get_trace(self.h, out, False, stream), 'hdg_get_trace')
        return out

    def free_trace(self):
        full = self.trace()
        return full[self._fd == 0].reshape(self.n_dof, self.R)

    def recover(self, stream=None):
        u = np.empty((self.n_elem, self.M * self.PE, self.R))
        q = np.empty((self.n_elem, self.M * self.dim * self.PE, self.R))
        check(L.hdg_recover(self.h, u, q, False, stream), 'hdg_recover')
        return u, q

    def condensed(self, e0=0, count=None):
        count = self.n_elem - e0 if count is None else count
        n = self.n_lfe * self.b
        K = np.empty((count, n, n))
        r = np.empty((count, n, self.R))
        check(L.hdg_get_condensed(self.h, e0, count, K, r), 'hdg_get_condensed')
        return K, r

    def face_rows(self, f0=0, count=None):
        count = self.n_free - f0 if count is None else count
        ms = 2 * self.n_lfe - 1
        blocks = np.empty((count, ms, self.b, self.b))
        nbr = np.empty((count, ms), np.int32)
        r = np.empty((self.n_dof, self.R))
        check(L.hdg_get_face_rows(self.h, f0, count, blocks, nbr, r), 'hdg_get_face_rows')
        return blocks, nbr, r

    def poly(self, cap=64):
        re = np.zeros(cap)
        im = np.zeros(cap)
        st, n = L.hdg_get_poly(self.h, re, im, cap)
        check(st, 'hdg_get_poly')
        return re[:n] + 1j * im[:n]

    def apply_K(self, x, prec='fp64', stream=None):
        import torch
        xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).to('cuda:%d' % self.device)
        yd = torch.empty_like(xd)
        check(L.hdg_apply_K(self.h, _PREC[prec], xd, yd, stream), 'hdg_apply_K')
        torch.cuda.synchronize(self.device)
        return yd.cpu().numpy()

    def apply_precond(self, o, x, prec='fp64', stream=None):
        import torch
        xd = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64)).to('cuda:%d' % self.device)
        yd = torch.empty_like(xd)
        check(L.hdg_apply_precond(self.h, o, _PREC[prec], xd, yd, stream), 'hdg_apply_precond')
        torch.cuda.synchronize(self.device)
        return yd.cpu().numpy()


def setup_from_workload(w, o, v0_seed=None, device=0, chunk=None):
    """Create, condense (in element chunks from the generator), assemble and
    set up the preconditioner for a workload of hdg_inputs."""
    p = Problem.from_workload(w, device)
    chunk = chunk or w.n_elem
    for e0 in range(0, w.n_elem, chunk):
        blk = w.blocks(e0, min(w.n_elem, e0 + chunk))
        p.condense(blk, e0)
    p.set_dirichlet(w.uhat_dirichlet())
    p.assemble(o)
    v0 = w.random_vector(v0_seed) if (o.poly != L.HDG_POLY_NONE) else None
    p.setup_precond(o, v0)
    return p
