"""Element blocks of the linearised HDG system (Welter & Nguyen, Eq. HDG,
Eq. numflux2, Eq. matrixform, Eq. w16).

Unknown ordering inside one element (M components, D dimensions, P_E element
basis functions, P_F face basis functions, N_lfe local faces):
    q   : (a, c, k)  -> (a*D + c)*P_E + k       (component a, direction c)
    u   : (b, j)     -> b*P_E + j
    uhat: (l, b, j)  -> (l*M + b)*P_F + j       (local face l)
Face basis functions are ordered as the *global* face's nodes, so the blocks
of both elements of a face refer to the same face unknowns.

Linear physics is described by constant tensors
    F_{ad}(u, q) = sum_b Cu[a,d,b] u_b + sum_{b,c} Cq[a,d,b,c] q_{bc}
    s_a(u)       = s0_a - sum_b Rr[a,b] u_b
with the numerical flux fhat = F(uhat, q).n + tau (u - uhat) (S = tau I).

The q-equation (Eq. HDGa) is the same for every component, so its blocks are
returned in the compact form of Eq. w16: the mass matrix M^e, B_d and C_d,
with A = I (x) M^e, B_{(a,c,i),(b,j)} = delta_ab B_c[i,j] and
C_{(a,c,i),(l,b,j)} = delta_ab C_c[i, l*P_F + j].  Reading of Eq. w16: B_d is
the matrix of the (u, div r) term of Eq. HDGa, i.e. B_d[i,j] = int phi_j
d(phi_i)/dx_d (the printed index placement is its transpose); C_d[i,(l,j)] =
-int_{F_l} phi_i psi_j n_d as printed.  r_q = 0 (Sec. 4.1).
"""
from dataclasses import dataclass, field
import numpy as np

from . import basis as B


# ----------------------------------------------------------------- physics
@dataclass
class Physics:
    M: int
    D: int
    Cq: np.ndarray                       # (M, D, M, D)
    Cu: np.ndarray                       # (M, D, M)
    Rr: np.ndarray                       # (M, M)
    tau: float
    name: str = ''


def poisson(D, kappa=1.0, tau=1.0):
    Cq = np.zeros((1, D, 1, D))
    for d in range(D):
        Cq[0, d, 0, d] = -kappa
    return Physics(1, D, Cq, np.zeros((1, D, 1)), np.zeros((1, 1)), tau, 'poisson')


def elasticity(D, lam, mu, tau=1.0):
    """F = -sigma(q), sigma = lam tr(q) I + mu (q + q^T), q = grad u."""
    Cq = np.zeros((D, D, D, D))
    for a in range(D):
        for d in range(D):
            for b in range(D):
                for c in range(D):
                    Cq[a, d, b, c] = -(lam * (a == d) * (b == c) + mu * ((a == b) * (d == c) + (a == c) * (d == b)))
    return Physics(D, D, Cq, np.zeros((D, D, D)), np.zeros((D, D)), tau, 'elasticity')


def cdr(D, M, beta, kappa, Rr, tau):
    """F_m = beta u_m - kappa q_m ; s = f - Rr u."""
    beta = np.asarray(beta, float)
    Cq = np.zeros((M, D, M, D))
    Cu = np.zeros((M, D, M))
    for a in range(M):
        for d in range(D):
            Cq[a, d, a, d] = -kappa
            Cu[a, d, a] = beta[d]
    return Physics(M, D, Cq, Cu, np.asarray(Rr, float).reshape(M, M), tau, 'cdr')


# --------------------------------------------------------- reference element
@dataclass
class RefElement:
    kind: str
    k: int
    D: int
    n_lfe: int
    PE: int
    PF: int
    vol_pts: np.ndarray
    vol_wts: np.ndarray
    phi: np.ndarray            # (nq, PE)
    dphi: np.ndarray           # (nq, PE, D) reference gradients
    face_st: np.ndarray        # (nfq, D-1) face-parameter quadrature points
    face_wts: np.ndarray       # (nfq,)
    face_ref_pts: list         # per l: (nfq, D) points in the reference element
    face_phi: list             # per l: (nfq, PE)
    face_dphi_geo: list        # per l: geometry data at face points
    face_normal_ref: list      # per l: reference outward normal scaled by the reference length element
    face_psi: np.ndarray       # (nfq, PF) face basis in local face parameters
    face_node_st: np.ndarray   # (PF, D-1) face nodes in face parameters
    face_node_ref: list        # per l: (PF, D) face nodes in the reference element
    extra: dict = field(default_factory=dict)


def ref_hex(k, nquad):
    pts, wts = B.hex_volume_rule(nquad)
    phi, dphi = B.hex_basis(k, pts)
    st, ws = B.square_rule(nquad)
    fpts, fphi, fn = [], [], []
    node_st = B.quad_nodes(k)
    fnode = []
    for l in range(6):
        P = B.hex_face_points(l, st)
        fpts.append(P)
        fphi.append(B.hex_basis(k, P)[0])
        ax, val, _ = B.HEX_FACES[l]
        e = np.zeros(3)
        e[ax] = val
        fn.append(e)
        fnode.append(B.hex_face_points(l, node_st))
    psi = B.quad_basis(k, st)
    return RefElement('hex', k, 3, 6, (k + 1) ** 3, (k + 1) ** 2, pts, wts, phi, dphi, st, ws,
                      fpts, fphi, None, fn, psi, node_st, fnode)


def ref_tri(k, nquad):
    pts, wts = B.tri_rule(nquad)
    phi, dphi = B.tri_basis(k, pts)
    t, wt = B.gauss_legendre(nquad)
    node_t = B.gll_nodes(k)
    fpts, fphi, fn, fnode = [], [], [], []
    # reference outward normals times the reference length element |dX/dt|
    normals = [np.array([1.0, 1.0]) / 2.0, np.array([-1.0, 0.0]) / 2.0, np.array([0.0, -1.0]) / 2.0]
    for l in range(3):
        P = B.tri_edge_points(l, t)
        fpts.append(P)
        fphi.append(B.tri_basis(k, P)[0])
        fn.append(normals[l])
        fnode.append(B.tri_edge_points(l, node_t))
    psi, _ = B.lagrange_1d(node_t, t)
    return RefElement('tri', k, 2, 3, (k + 1) * (k + 2) // 2, k + 1, pts, wts, phi, dphi,
                      t[:, None], wt, fpts, fphi, None, fn, psi, node_t[:, None], fnode)


def ref_tet(k, nquad):
    pts, wts = B.tet_rule(nquad)
    phi, dphi = B.tet_basis(k, pts)
    st, ws = B.tri_rule(nquad)
    node_st = B.tri_nodes(k)
    fpts, fphi, fn, fnode = [], [], [], []
    for l in range(4):
        P = B.tet_face_points(l, st)
        fpts.append(P)
        fphi.append(B.tet_basis(k, P)[0])
        fn.append(B.tet_face_normal(l))
        fnode.append(B.tet_face_points(l, node_st))
    psi, _ = B.tri_basis(k, st)
    PE = (k + 1) * (k + 2) * (k + 3) // 6
    return RefElement('tet', k, 3, 4, PE, (k + 1) * (k + 2) // 2, pts, wts, phi, dphi, st, ws,
                      fpts, fphi, None, fn, psi, node_st, fnode)


def ref_quad(k, nquad):
    x, w = B.gauss_legendre(nquad)
    pts = np.array([[x[i], x[j]] for j in range(nquad) for i in range(nquad)])
    wts = np.array([w[i] * w[j] for j in range(nquad) for i in range(nquad)])
    phi, dphi = B.quad_vol_basis(k, pts)
    node_t = B.gll_nodes(k)
    fpts, fphi, fn, fnode = [], [], [], []
    for l in range(4):
        P = B.quad_face_points(l, x)
        fpts.append(P)
        fphi.append(B.quad_vol_basis(k, P)[0])
        e = np.zeros(2)
        e[l // 2] = 1.0 if l % 2 else -1.0
        fn.append(e)
        fnode.append(B.quad_face_points(l, node_t))
    psi, _ = B.lagrange_1d(node_t, x)
    return RefElement('quad', k, 2, 4, (k + 1) ** 2, k + 1, pts, wts, phi, dphi, x[:, None], w,
                      fpts, fphi, None, fn, psi, node_t[:, None], fnode)


def reference_element(mesh, k, nquad=None):
    if mesh.kind == 'quad':
        return ref_quad(k, nquad or (k + 2))
    if mesh.kind == 'hex':
        return ref_hex(k, nquad or (k + 2))
    if mesh.kind == 'tet':
        return ref_tet(k, nquad or (k + 2))
    return ref_tri(k, nquad or (k + 3))


# ------------------------------------------------------------- geometry
def geometry(mesh, elems, ref_pts):
    """Physical points, Jacobian, det and inverse at reference points for the
    given elements (trilinear hexahedra, affine triangles)."""
    if mesh.kind == 'hex':
        X8 = mesh.verts[mesh.elems[elems]]
        x, Jac = B.trilinear(X8, ref_pts)
    elif mesh.kind == 'quad':
        x, Jac = B.bilinear(mesh.verts[mesh.elems[elems]], ref_pts)
    elif mesh.kind == 'tet':
        X4 = mesh.verts[mesh.elems[elems]]                     # (E, 4, 3)
        v0 = X4[:, 0, :]
        Jm = np.stack([X4[:, 1, :] - v0, X4[:, 2, :] - v0, X4[:, 3, :] - v0], axis=2)
        x = v0[:, None, :] + np.einsum('eab,nb->ena', Jm, ref_pts)
        Jac = np.broadcast_to(Jm[:, None], (len(elems), ref_pts.shape[0], 3, 3)).copy()
    else:
        X3 = mesh.verts[mesh.elems[elems]]                     # (E, 3, 2)
        v0 = X3[:, 0, :]
        Jm = np.stack([X3[:, 1, :] - v0, X3[:, 2, :] - v0], axis=2)   # (E, 2, 2): dx_a/dxi_b
        x = v0[:, None, :] + np.einsum('eab,nb->ena', Jm, ref_pts)
        Jac = np.broadcast_to(Jm[:, None], (len(elems), ref_pts.shape[0], 2, 2)).copy()
    det = np.linalg.det(Jac)
    Jinv = np.linalg.inv(Jac)
    return x, Jac, det, Jinv


def face_permutations(mesh, ref):
    """perm[e, l, jg] = local face-node index matching global face node jg.

    The global face's nodes are those of its first element (e1, l1) in that
    element's local face parametrisation; nodes of the second element are
    matched to them by physical position."""
    ne, nl, PF = mesh.n_elem, mesh.n_lfe, ref.PF
    coords = np.empty((ne, nl, PF, mesh.dim))
    for l in range(nl):
        x, _, _, _ = geometry(mesh, np.arange(ne), ref.face_node_ref[l])
        coords[:, l] = x
    perm = np.empty((ne, nl, PF), np.int32)
    perm[:] = np.arange(PF)
    fe = mesh.face_elem
    scale = np.abs(mesh.verts).max() + 1.0
    inner = np.nonzero(fe[:, 2] >= 0)[0]
    for c0 in range(0, len(inner), 8192):
        f = inner[c0:c0 + 8192]
        A = coords[fe[f, 0], fe[f, 1]]                                   # (nf, PF, dim)
        Bc = coords[fe[f, 2], fe[f, 3]]
        dist = np.linalg.norm(A[:, :, None, :] - Bc[:, None, :, :], axis=3)
        p = np.argmin(dist, axis=2)                                      # (nf, PF)
        assert np.all(np.take_along_axis(dist, p[:, :, None], axis=2) < 1e-9 * scale), "face nodes do not match"
        assert np.all(np.sort(p, axis=1) == np.arange(PF)), "face node matching is not one to one"
        perm[fe[f, 2], fe[f, 3]] = p
    return perm


# ---------------------------------------------------------- element blocks
def element_matrices(mesh, ref, perm, elems):
    """Basic element and face integrals for the elements `elems`.

    Returns a dict with
      Me (E,PE,PE), Sd (E,D,PE,PE) [Sd[d,i,j] = int dphi_i/dx_d phi_j],
      Mf (E,PE,PE) [sum over faces of int phi_i phi_j],
      EF (E,nl,PE,PF), EFN (E,nl,D,PE,PF), FF (E,nl,PF,PF), FFN (E,nl,D,PF,PF),
      xq (E,nq,D), wJ (E,nq) volume quadrature data.
    """
    D = ref.D
    x, Jac, det, Jinv = geometry(mesh, elems, ref.vol_pts)
    wJ = ref.vol_wts[None, :] * np.abs(det)
    g = np.einsum('qib,eqba->eqia', ref.dphi, Jinv)
    Me = np.einsum('eq,qi,qj->eij', wJ, ref.phi, ref.phi, optimize=True)
    Sd = np.einsum('eq,eqid,qj->edij', wJ, g, ref.phi, optimize=True)
    nl = ref.n_lfe
    E = len(elems)
    EF = np.empty((E, nl, ref.PE, ref.PF))
    EFN = np.empty((E, nl, D, ref.PE, ref.PF))
    FF = np.empty((E, nl, ref.PF, ref.PF))
    FFN = np.empty((E, nl, D, ref.PF, ref.PF))
    Mf = np.zeros((E, ref.PE, ref.PE))
    for l in range(nl):
        xf, Jf, detf, Jinvf = geometry(mesh, elems, ref.face_ref_pts[l])
        nv = detf[:, :, None] * np.einsum('eqba,b->eqa', Jinvf, ref.face_normal_ref[l])
        dA = np.linalg.norm(nv, axis=2)
        n = nv / dA[:, :, None]
        w = ref.face_wts[None, :] * dA                                   # (E, nfq)
        psi = ref.face_psi[:, perm[elems, l, :]]                         # (nfq, E, PF)
        psi = np.transpose(psi, (1, 0, 2))                               # (E, nfq, PF)
        ph = ref.face_phi[l]
        EF[:, l] = np.einsum('eq,qi,eqj->eij', w, ph, psi, optimize=True)
        EFN[:, l] = np.einsum('eq,eqd,qi,eqj->edij', w, n, ph, psi, optimize=True)
        FF[:, l] = np.einsum('eq,eqi,eqj->eij', w, psi, psi, optimize=True)
        FFN[:, l] = np.einsum('eq,eqd,eqi,eqj->edij', w, n, psi, psi, optimize=True)
        Mf += np.einsum('eq,qi,qj->eij', w, ph, ph, optimize=True)
    return dict(Me=Me, Sd=Sd, Mf=Mf, EF=EF, EFN=EFN, FF=FF, FFN=FFN, xq=x, wJ=wJ)


def hdg_blocks(mats, phys):
    """HDG element blocks from the basic integrals and the physics tensors.

    Returns Me, Bd, Cd (compact q-equation blocks of Eq. w16) and the dense
    D, E, F, G, H, J blocks of Eq. matrixform."""
    M, D, tau = phys.M, phys.D, phys.tau
    Me, Sd, Mf = mats['Me'], mats['Sd'], mats['Mf']
    EF, EFN, FF, FFN = mats['EF'], mats['EFN'], mats['FF'], mats['FFN']
    E, nl, PE, PF = EF.shape
    I = np.eye(M)
    Bd = Sd.copy()
    Cd = -np.transpose(EFN, (0, 2, 3, 1, 4)).reshape(E, D, PE, nl * PF)
    # D_{(a,i),(b,c,k)} = sum_d Cq[a,d,b,c] Sd[d,k,i]
    Dm = np.einsum('adbc,edki->eaibck', phys.Cq, Sd, optimize=True).reshape(E, M * PE, M * D * PE)
    # E_{(a,i),(b,j)} = -sum_d Cu[a,d,b] Sd[d,i,j] + tau delta_ab Mf_ij + Rr[a,b] Me_ij
    Em = (-np.einsum('adb,edij->eaibj', phys.Cu, Sd, optimize=True)
          + tau * np.einsum('ab,eij->eaibj', I, Mf)
          + np.einsum('ab,eij->eaibj', phys.Rr, Me)).reshape(E, M * PE, M * PE)
    # F_{(a,i),(l,b,j)} = sum_d Cu[a,d,b] EFN[l,d,i,j] - tau delta_ab EF[l,i,j]
    Fm = (np.einsum('adb,eldij->eailbj', phys.Cu, EFN, optimize=True)
          - tau * np.einsum('ab,elij->eailbj', I, EF)).reshape(E, M * PE, nl * M * PF)
    # G_{(l,a,j),(b,c,k)} = sum_d Cq[a,d,b,c] EFN[l,d,k,j]
    Gm = np.einsum('adbc,eldkj->elajbck', phys.Cq, EFN, optimize=True).reshape(E, nl * M * PF, M * D * PE)
    # H_{(l,a,j),(b,k)} = tau delta_ab EF[l,k,j]
    Hm = (tau * np.einsum('ab,elkj->elajbk', I, EF)).reshape(E, nl * M * PF, M * PE)
    # J_{(l,a,j),(l',b,k)} = delta_ll' (sum_d Cu[a,d,b] FFN[l,d,k,j] - tau delta_ab FF[l,k,j])
    Jblk = (np.einsum('adb,eldkj->elajbk', phys.Cu, FFN, optimize=True)
            - tau * np.einsum('ab,elkj->elajbk', I, FF))                 # (E, nl, M, PF, M, PF)
    Jm = np.zeros((E, nl, M * PF, nl, M * PF))
    for l in range(nl):
        Jm[:, l, :, l, :] = Jblk[:, l].reshape(E, M * PF, M * PF)
    Jm = Jm.reshape(E, nl * M * PF, nl * M * PF)
    return dict(Me=Me, Bd=Bd, Cd=Cd, D=Dm, E=Em, F=Fm, G=Gm, H=Hm, J=Jm)


def load_vector_from_function(mats, ref, f, M):
    """r_u[(a,i)] = int f_a phi_i, f(x) -> (..., M) evaluated at quadrature points."""
    fx = f(mats['xq'])                                                   # (E, nq, M)
    ru = np.einsum('eq,eqa,qi->eai', mats['wJ'], fx, ref.phi)
    return ru.reshape(ru.shape[0], -1)


def load_vector_from_nodal(mats, fnodal):
    """r_u for f given by nodal coefficients fnodal (E, M, PE): r = Me f."""
    ru = np.einsum('eij,eaj->eai', mats['Me'], fnodal)
    return ru.reshape(ru.shape[0], -1)


def neumann_face_load(mesh, ref, perm, elems, neumann, g, M):
    """r_uh rows of Neumann faces: the trace equation of a boundary face that
    is not Dirichlet states <Fhat.n, mu> = <g, mu>, g the prescribed outward
    normal flux (g = -kappa du/dn for F = -kappa grad u; g = -t for
    F = -sigma, t the applied traction).  g(x, n) -> (..., M) at face
    quadrature points x with unit outward normals n.  Returns (E, nl*M*PF) in
    the (l, a, j) row order of H and J; zero rows on the other faces."""
    nl, PF = ref.n_lfe, ref.PF
    E = len(elems)
    out = np.zeros((E, nl, M, PF))
    for l in range(nl):
        sel = neumann[mesh.elem_face[elems, l]].astype(bool)
        if not np.any(sel):
            continue
        es = elems[sel]
        xf, Jf, detf, Jinvf = geometry(mesh, es, ref.face_ref_pts[l])
        nv = detf[:, :, None] * np.einsum('eqba,b->eqa', Jinvf, ref.face_normal_ref[l])
        dA = np.linalg.norm(nv, axis=2)
        w = ref.face_wts[None, :] * dA
        psi = np.transpose(ref.face_psi[:, perm[es, l, :]], (1, 0, 2))
        gx = g(xf, nv / dA[:, :, None])                                   # (E', nfq, M)
        out[sel, l] = np.einsum('eq,eqa,eqj->eaj', w, gx, psi)
    return out.reshape(E, nl * M * PF)


def dirichlet_face_values(mesh, ref, perm, u_exact, M):
    """L2 projection of u_exact onto the face space of every boundary face
    (b_hat = uhat - u_D on Dirichlet faces).  Returns (NF, M*PF); only the
    rows of Dirichlet faces are used."""
    NF = mesh.n_face
    out = np.zeros((NF, M * ref.PF))
    bf = np.nonzero(mesh.face_boundary)[0]
    if len(bf) == 0:
        return out
    e1 = mesh.face_elem[bf, 0]
    l1 = mesh.face_elem[bf, 1]
    for l in range(ref.n_lfe):
        sel = l1 == l
        if not np.any(sel):
            continue
        elems = e1[sel]
        xf, Jf, detf, Jinvf = geometry(mesh, elems, ref.face_ref_pts[l])
        nv = detf[:, :, None] * np.einsum('eqba,b->eqa', Jinvf, ref.face_normal_ref[l])
        w = ref.face_wts[None, :] * np.linalg.norm(nv, axis=2)
        psi = np.transpose(ref.face_psi[:, perm[elems, l, :]], (1, 0, 2))
        FF = np.einsum('eq,eqi,eqj->eij', w, psi, psi)
        ux = u_exact(xf)                                                  # (E, nfq, M)
        rhs = np.einsum('eq,eqa,eqj->eaj', w, ux, psi)
        sol = np.linalg.solve(FF[:, None], rhs[..., None])[..., 0]        # (E, M, PF)
        out[bf[sel]] = sol.reshape(len(elems), -1)
    return out
