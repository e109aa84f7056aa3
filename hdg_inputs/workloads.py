"""The named synthetic workloads, with their seeds.

  tri_poisson     : unit square, n x n squares split into 2n^2 triangles, P^k,
                    tau = 1, u = sin(pi x) sin(pi y)       (default n=8, k=2)
  hex_poisson     : unit cube, n^3 hexahedra, Q^k, tau = 1,
                    u = prod sin(pi x_i)                    (default n=16, k=3)
  hex_elasticity  : n^3 hexahedra with interior vertices moved by up to 0.2h
                    (seed 3), Q^k, E = 1, nu = 0.3, tau = 1, R right-hand sides
                    from nodal N(0,1) body forces (seeds 300..)  (n=32, k=2, R=8)
  hex_cdr         : n^3 hexahedra, Q^k, 5 components, beta = (1,1,1)/sqrt 3,
                    kappa = 1, reaction A = S + W + I from a seeded (5) Gaussian
                    G (S = G G^T / 5, W = (G - G^T)/2), tau = |beta| + kappa,
                    R right-hand sides from nodal N(0,1) forces (seeds 500..)
                                                             (n=40, k=2, R=4)
  hex_convdiff    : one serving request: n^3 hexahedra, Q^k, kappa, unit beta,
                    f = 1, tau = 1 + kappa
  tet_poisson     : unit cube, Kuhn tetrahedra (6 n^3), P^k, tau = 1,
                    u = prod sin(pi x_i)
  tet_obstacle    : Laplace on (-1,1)^3 minus a central cube, Kuhn tetrahedra,
                    P^k; u = 0 on the obstacle, outward flux n_x on the box
  hex_beam        : cantilever beam (0,5) x (0,1) x (0,1) with 5n x n x n
                    hexahedra (Sec. 6.2: n = 2, 4, 6, 8 gives N_E = 40, 320,
                    1080, 2560), Q^k, lambda = mu = 1, tau = 1; clamped
                    (u = 0) at x = 0, uniform traction t = (0, 0, -1) at
                    x = 5, the other faces traction-free; no body force
Except for hex_beam and tet_obstacle, all faces on the domain boundary are
Dirichlet faces.
"""
from dataclasses import dataclass
import numpy as np

from . import mesh as meshmod
from . import blocks as blk


@dataclass
class Workload:
    name: str
    mesh: object
    ref: object
    perm: np.ndarray
    phys: object
    R: int
    rhs_kind: str                 # 'function', 'nodal' or 'none' (no body force)
    f_exact: object = None        # callable x -> (..., M)
    u_exact: object = None        # callable x -> (..., M)
    q_exact: object = None        # callable x -> (..., M, D)
    rhs_seeds: tuple = ()
    k: int = 1
    dirichlet: np.ndarray = None  # (NF,) uint8 Dirichlet faces; None = every boundary face
    neumann_flux: object = None   # g(x, n) -> (..., M): outward flux on the other boundary faces

    # sizes
    @property
    def M(self): return self.phys.M

    @property
    def D(self): return self.phys.D

    @property
    def PE(self): return self.ref.PE

    @property
    def PF(self): return self.ref.PF

    @property
    def n_lfe(self): return self.ref.n_lfe

    @property
    def n_elem(self): return self.mesh.n_elem

    @property
    def n_face(self): return self.mesh.n_face

    @property
    def face_dirichlet(self):
        if self.dirichlet is not None:
            return np.asarray(self.dirichlet, np.uint8)
        return self.mesh.face_boundary.astype(np.uint8)

    @property
    def face_neumann(self):
        """Boundary faces that are not Dirichlet faces (prescribed flux)."""
        return (self.mesh.face_boundary.astype(bool) & ~self.face_dirichlet.astype(bool)).astype(np.uint8)

    @property
    def n_free(self):
        return int(self.n_face - self.face_dirichlet.sum())

    @property
    def n_dof(self):
        return self.n_free * self.M * self.PF

    def blocks(self, e0=0, e1=None, elems=None):
        """Element blocks for elements [e0, e1), or for the index array
        `elems` (row-major, float64)."""
        if elems is None:
            e1 = self.n_elem if e1 is None else e1
            elems = np.arange(e0, e1)
        elems = np.asarray(elems)
        mats = blk.element_matrices(self.mesh, self.ref, self.perm, elems)
        out = blk.hdg_blocks(mats, self.phys)
        E = len(elems)
        if self.rhs_kind == 'none':
            ru = np.zeros((E, self.M * self.PE, self.R))
        elif self.rhs_kind == 'function':
            ru = blk.load_vector_from_function(mats, self.ref, self.f_exact, self.M)[:, :, None]
            ru = np.repeat(ru, self.R, axis=2)
        else:
            cols = []
            for s in self.rhs_seeds:
                rng = np.random.default_rng(s)
                fn = rng.standard_normal((self.n_elem, self.M, self.PE))[elems]
                cols.append(blk.load_vector_from_nodal(mats, fn))
            ru = np.stack(cols, axis=2)
        out['ru'] = np.ascontiguousarray(ru)
        out['ruh'] = np.zeros((E, self.n_lfe * self.M * self.PF, self.R))
        if self.neumann_flux is not None and self.face_neumann.any():
            gN = blk.neumann_face_load(self.mesh, self.ref, self.perm, elems, self.face_neumann,
                                       self.neumann_flux, self.M)
            out['ruh'] += gN[:, :, None]
        out['_mats'] = mats
        return out

    def load_vectors(self, e0=0, e1=None):
        """(ru, ruh) of elements [e0, e1) as blocks() gives them, without the
        element matrices: r_u from the quadrature rule directly (for nodal
        forces, sum_q w|J| phi_i(x_q) f_h(x_q) = (M^e f)_i), r_uhat zero (plus
        the flux loads of Neumann faces).  For callers that generate the
        blocks on the device from the vertices."""
        e1 = self.n_elem if e1 is None else e1
        elems = np.arange(e0, e1)
        E = len(elems)
        ref = self.ref
        if self.rhs_kind == 'none':
            ru = np.zeros((E, self.M * self.PE, self.R))
        else:
            x, det = _points_and_det(self.mesh, elems, ref.vol_pts)
            wJ = ref.vol_wts[None, :] * np.abs(det)                         # (E, nq)
            if self.rhs_kind == 'function':
                fq = self.f_exact(x)                                         # (E, nq, M)
                ru = np.einsum('eq,eqa,qi->eai', wJ, fq, ref.phi).reshape(E, -1)[:, :, None]
                ru = np.repeat(ru, self.R, axis=2)
            else:
                cols = []
                for sd in self.rhs_seeds:
                    fn = np.random.default_rng(sd).standard_normal((self.n_elem, self.M, self.PE))[elems]
                    fq = fn @ ref.phi.T                                      # (E, M, nq): f_h at the points
                    cols.append(((fq * wJ[:, None, :]) @ ref.phi).reshape(E, -1))
                ru = np.stack(cols, axis=2)
        ruh = np.zeros((E, self.n_lfe * self.M * self.PF, self.R))
        if self.neumann_flux is not None and self.face_neumann.any():
            gN = blk.neumann_face_load(self.mesh, ref, self.perm, elems, self.face_neumann,
                                       self.neumann_flux, self.M)
            ruh += gN[:, :, None]
        return np.ascontiguousarray(ru), ruh

    def uhat_dirichlet(self):
        """(NF, M*PF, R) Dirichlet trace values (zero rows on interior faces)."""
        if self.u_exact is None:
            v = np.zeros((self.n_face, self.M * self.PF))
        else:
            v = blk.dirichlet_face_values(self.mesh, self.ref, self.perm, self.u_exact, self.M)
        return np.ascontiguousarray(np.repeat(v[:, :, None], self.R, axis=2))

    def random_vector(self, seed):
        """Seeded N(0,1) vector over the free trace dofs, e.g. the starting
        vector of the Arnoldi cycle that defines a polynomial preconditioner."""
        return np.random.default_rng(seed).standard_normal(self.n_dof)


def _points_and_det(mesh, elems, ref_pts):
    """Physical points and Jacobian determinants at reference points (the
    quantities of blocks.geometry that a load vector needs), with the
    trilinear hexahedron map written as matrix products."""
    if mesh.kind != 'hex':
        x, _, det, _ = blk.geometry(mesh, elems, ref_pts)
        return x, det
    from .basis import HEX_VERTS
    s = HEX_VERTS
    n = ref_pts.shape[0]
    N = np.prod(1.0 + ref_pts[:, None, :] * s[None, :, :], axis=2) / 8.0          # (n, 8)
    dN = np.zeros((n, 8, 3))
    for b in range(3):
        other = [c for c in range(3) if c != b]
        dN[:, :, b] = s[None, :, b] * np.prod(1.0 + ref_pts[:, None, other] * s[None, :, other], axis=2) / 8.0
    X8 = mesh.verts[mesh.elems[elems]]                                             # (E, 8, 3)
    XT = np.ascontiguousarray(X8.transpose(0, 2, 1))                               # (E, 3, 8)
    x = (XT @ N.T).transpose(0, 2, 1)                                              # (E, n, 3)
    J = (XT @ dN.transpose(1, 0, 2).reshape(8, n * 3)).reshape(len(elems), 3, n, 3)   # J[e, a, q, b]
    det = (J[:, 0, :, 0] * (J[:, 1, :, 1] * J[:, 2, :, 2] - J[:, 1, :, 2] * J[:, 2, :, 1])
           - J[:, 0, :, 1] * (J[:, 1, :, 0] * J[:, 2, :, 2] - J[:, 1, :, 2] * J[:, 2, :, 0])
           + J[:, 0, :, 2] * (J[:, 1, :, 0] * J[:, 2, :, 1] - J[:, 1, :, 1] * J[:, 2, :, 0]))
    return x, det


def _sin_product(D):
    def u(x):
        return np.prod(np.sin(np.pi * x), axis=-1)[..., None]

    def f(x):
        return (D * np.pi ** 2) * u(x)

    def q(x):
        s = np.sin(np.pi * x)
        c = np.cos(np.pi * x)
        out = np.empty(x.shape[:-1] + (1, D))
        for d in range(D):
            others = np.prod(np.delete(s, d, axis=-1), axis=-1)
            out[..., 0, d] = np.pi * c[..., d] * others
        return out
    return u, f, q


def tri_poisson(n=8, k=2, R=1):
    m = meshmod.tri_mesh(n)
    ref = blk.reference_element(m, k)
    u, f, q = _sin_product(2)
    return Workload('tri_poisson', m, ref, blk.face_permutations(m, ref), blk.poisson(2), R,
                    'function', f, u, q, k=k)


def hex_poisson(n=16, k=3, R=1):
    m = meshmod.hex_mesh(n)
    ref = blk.reference_element(m, k)
    u, f, q = _sin_product(3)
    return Workload('hex_poisson', m, ref, blk.face_permutations(m, ref), blk.poisson(3), R,
                    'function', f, u, q, k=k)


def hex_elasticity(n=32, k=2, R=8, young=1.0, nu=0.3, perturb=0.2, mesh_seed=3, rhs_seed0=300):
    lam = young * nu / ((1 + nu) * (1 - 2 * nu))
    mu = young / (2 * (1 + nu))
    m = meshmod.hex_mesh(n, perturb, mesh_seed)
    ref = blk.reference_element(m, k, (k + 4) if perturb > 0 else None)
    return Workload('hex_elasticity', m, ref, blk.face_permutations(m, ref), blk.elasticity(3, lam, mu, 1.0),
                    R, 'nodal', rhs_seeds=tuple(range(rhs_seed0, rhs_seed0 + R)), k=k)


def cdr_reaction_matrix(M=5, seed=5):
    G = np.random.default_rng(seed).standard_normal((M, M))
    return G @ G.T / M + (G - G.T) / 2 + np.eye(M)


def hex_cdr(n=40, k=2, R=4, M=5, kappa=1.0, a_seed=5, rhs_seed0=500):
    m = meshmod.hex_mesh(n)
    ref = blk.reference_element(m, k)
    beta = np.ones(3) / np.sqrt(3.0)
    phys = blk.cdr(3, M, beta, kappa, cdr_reaction_matrix(M, a_seed), np.linalg.norm(beta) + kappa)
    return Workload('hex_cdr', m, ref, blk.face_permutations(m, ref), phys, R, 'nodal',
                    rhs_seeds=tuple(range(rhs_seed0, rhs_seed0 + R)), k=k)


def hex_convdiff(n, k, kappa, beta, R=1):
    m = meshmod.hex_mesh(n)
    ref = blk.reference_element(m, k)
    beta = np.asarray(beta, float)
    phys = blk.cdr(3, 1, beta, kappa, np.zeros((1, 1)), np.linalg.norm(beta) + kappa)
    one = lambda x: np.ones(x.shape[:-1] + (1,))
    return Workload('hex_convdiff', m, ref, blk.face_permutations(m, ref), phys, R, 'function', one, k=k)


def boundary_faces_at(mesh, axis, value, tol=1e-12):
    """(NF,) uint8: boundary faces whose vertices all have x_axis = value."""
    from .basis import hex_face_vertices, TET_FACES
    out = np.zeros(mesh.n_face, np.uint8)
    for f in np.nonzero(mesh.face_boundary)[0]:
        e, l = mesh.face_elem[f, 0], mesh.face_elem[f, 1]
        lv = hex_face_vertices(l) if mesh.kind == 'hex' else list(TET_FACES[l])
        xs = mesh.verts[mesh.elems[e, lv], axis]
        out[f] = np.all(np.abs(xs - value) < tol)
    return out


def tet_poisson(n=8, k=2, R=1):
    """Unit cube, Kuhn tetrahedra (6 n^3), P^k, tau = 1, u = prod sin(pi x_i),
    every boundary face Dirichlet."""
    m = meshmod.tet_mesh(n)
    ref = blk.reference_element(m, k)
    u, f, q = _sin_product(3)
    return Workload('tet_poisson', m, ref, blk.face_permutations(m, ref), blk.poisson(3), R,
                    'function', f, u, q, k=k)


def tet_obstacle(n=16, k=2, hole=0.25):
    """Sec. 6.1's three-dimensional Poisson problem, synthetic stand-in: the
    Laplace equation on the box (-1,1)^3 minus a central cube of half-width
    `hole` (in place of the cone of the paper's Gmsh mesh), Kuhn tetrahedra,
    P^k, tau = 1; u = 0 on the obstacle and grad u . n + (1,0,0) . n = 0 on
    the box, i.e. outward flux g = -grad u . n = n_x."""
    m = meshmod.tet_mesh(n, -1.0, 1.0, hole)
    ref = blk.reference_element(m, k)
    outer = np.zeros(m.n_face, np.uint8)
    for ax in range(3):
        for v in (-1.0, 1.0):
            outer |= boundary_faces_at(m, ax, v)
    dirichlet = (m.face_boundary.astype(bool) & ~outer.astype(bool)).astype(np.uint8)
    g = lambda x, nrm: nrm[..., :1].copy()
    return Workload('tet_obstacle', m, ref, blk.face_permutations(m, ref), blk.poisson(3), 1, 'none', k=k,
                    dirichlet=dirichlet, neumann_flux=g)


def hex_beam(n=4, k=2, lam=1.0, mu=1.0, traction=(0.0, 0.0, -1.0), length=5.0, tau=1.0):
    """Sec. 6.2: the clamped face x = 0 is the only Dirichlet boundary; the
    loaded end x = length carries the traction t, i.e. the outward flux of
    F = -sigma there is g = -t; the four side faces are traction-free."""
    m = meshmod.box_hex_mesh((5 * n, n, n), (length, 1.0, 1.0))
    ref = blk.reference_element(m, k)
    t = np.asarray(traction, float)

    def g(x, nrm):
        at_end = (np.abs(x[..., 0] - length) < 1e-9)[..., None]
        return np.where(at_end, -t, 0.0)
    return Workload('hex_beam', m, ref, blk.face_permutations(m, ref), blk.elasticity(3, lam, mu, tau), 1,
                    'none', k=k, dirichlet=boundary_faces_at(m, 0, 0.0), neumann_flux=g)


def serving_requests(n_requests=512, seed=4, n_range=(8, 24), k_range=(1, 3)):
    """Request parameters of the serving stream: kappa log-uniform in
    [1e-3, 1], a uniform random unit velocity, n and k uniform integers."""
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n_requests):
        kappa = 10.0 ** rng.uniform(-3.0, 0.0)
        b = rng.standard_normal(3)
        b /= np.linalg.norm(b)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        reqs.append(dict(id=i, kappa=kappa, beta=b, n=n, k=k))
    return reqs


def poisson_arrivals(n, rate, seed=41):
    """Arrival times (s) of a Poisson process with the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


# --------------------------------------------------------------- serving inputs
_STRUCT_CACHE = {}


def structured_convdiff_inputs(n, k, kappa, beta, R=1):
    """Inputs of one convection-diffusion request (f = 1, homogeneous
    Dirichlet) on the structured n^3 mesh: the mesh arrays and ONE element's
    blocks, valid for every element (all elements are the same cube and every
    face is parametrised the same way from both sides, which is checked), with
    element strides 0 for hdg_condense_strided."""
    key = (n, k)
    if key not in _STRUCT_CACHE:
        m = meshmod.hex_mesh(n)
        ref = blk.reference_element(m, k)
        perm = blk.face_permutations(m, ref)
        assert np.all(perm == np.arange(ref.PF)), "face permutations differ between elements"
        mats = blk.element_matrices(m, ref, perm, np.array([0]))
        fd = m.face_boundary.astype(np.uint8)
        mesh = dict(dim=3, n_lfe=6, M=1, PE=ref.PE, PF=ref.PF, elem_face=m.elem_face,
                    face_elem=m.face_elem, face_dirichlet=fd)
        _STRUCT_CACHE[key] = (mesh, ref, mats)
    mesh, ref, mats = _STRUCT_CACHE[key]
    beta = np.asarray(beta, float)
    phys = blk.cdr(3, 1, beta, kappa, np.zeros((1, 1)), np.linalg.norm(beta) + kappa)
    out = blk.hdg_blocks(mats, phys)
    one = lambda x: np.ones(x.shape[:-1] + (1,))
    ru = blk.load_vector_from_function(mats, ref, one, 1)[:, :, None]
    out['ru'] = np.ascontiguousarray(np.repeat(ru, R, axis=2))
    out['ruh'] = np.zeros((1, 6 * ref.PF, R))
    strides = [0] * 11
    uD = np.zeros((len(mesh['face_dirichlet']), ref.PF, R))
    return mesh, {k2: np.ascontiguousarray(v) for k2, v in out.items()}, strides, uD


def shared_blocks(w):
    """Element blocks of a workload whose elements are all the same (an
    unperturbed structured hex mesh, constant coefficients, every face
    parametrised the same way from both sides; all three are checked):
    element 0's matrices, valid for every element, plus the per-element load
    vectors of its 'nodal' right-hand sides.  Returns (blocks, strides) for
    hdg_condense_strided: stride 0 for the shared blocks, the per-element size
    for ru and ruh."""
    m = w.mesh
    X = m.verts[m.elems]
    assert np.allclose(X - X[:, :1], X[:1] - X[:1, :1], atol=1e-13), "elements are not translates"
    assert np.all(w.perm == np.arange(w.PF)), "face permutations differ between elements"
    assert w.rhs_kind in ('nodal', 'none')
    b0 = w.blocks(0, 1)
    mats = b0.pop('_mats')
    cols = []
    for s in w.rhs_seeds:
        fn = np.random.default_rng(s).standard_normal((w.n_elem, w.M, w.PE))
        cols.append(np.einsum('ij,eaj->eai', mats['Me'][0], fn).reshape(w.n_elem, -1))
    out = {k: np.ascontiguousarray(v) for k, v in b0.items()}
    out['ru'] = (np.ascontiguousarray(np.stack(cols, axis=2)) if cols
                 else np.zeros((w.n_elem, w.M * w.PE, w.R)))
    out['ruh'] = np.zeros((w.n_elem, w.n_lfe * w.M * w.PF, w.R))
    if w.neumann_flux is not None and w.face_neumann.any():
        # the face loads differ between elements (only boundary faces carry them)
        out['ruh'] += blk.neumann_face_load(m, w.ref, w.perm, np.arange(w.n_elem), w.face_neumann,
                                            w.neumann_flux, w.M)[:, :, None]
    names = ('Me', 'Bd', 'Cd', 'D', 'E', 'F', 'G', 'H', 'J', 'ru', 'ruh')
    strides = [0] * 9 + [out['ru'][0].size, out['ruh'][0].size]
    return {k: out[k] for k in names}, strides


def element_classes(w):
    """Classes of elements with identical blocks: the same vertex positions
    relative to the first vertex and the same face-node permutations (a
    structured mesh has few: six Kuhn tetrahedra times the permutation
    patterns).  Returns (representatives, class_of_element)."""
    X = w.mesh.verts[w.mesh.elems]
    scale = np.abs(X).max() + 1.0
    rel = np.round((X - X[:, :1]) / scale * 1e9).astype(np.int64).reshape(w.n_elem, -1)
    key = np.concatenate([rel, w.perm.reshape(w.n_elem, -1).astype(np.int64)], axis=1)
    _, rep, cls = np.unique(key, axis=0, return_index=True, return_inverse=True)
    return rep, cls.ravel()


def class_blocks(w):
    """Blocks of a workload with constant coefficients and no body force or
    nodal loads ('none'): one block set per element class, plus the per-element
    face loads of its traction faces.  Returns (rep_blocks, class_of_element,
    ruh (NE, nlb, R)); the blocks of elements [a, b) are
    {k: rep_blocks[k][cls[a:b]]}."""
    assert w.rhs_kind == 'none'
    rep, cls = element_classes(w)
    b = w.blocks(elems=rep)
    b.pop('_mats')
    ruh = np.zeros((w.n_elem, w.n_lfe * w.M * w.PF, w.R))
    if w.neumann_flux is not None and w.face_neumann.any():
        sel = np.nonzero(w.face_neumann[w.mesh.elem_face].any(axis=1))[0]
        ruh[sel] = blk.neumann_face_load(w.mesh, w.ref, w.perm, sel, w.face_neumann, w.neumann_flux,
                                         w.M)[:, :, None]
    names = ('Me', 'Bd', 'Cd', 'D', 'E', 'F', 'G', 'H', 'J')
    return {k: b[k] for k in names}, cls, ruh
