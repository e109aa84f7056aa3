"""Lagrange bases and Gauss quadrature on the reference elements.

Reference interval [-1, 1]; reference square/cube [-1, 1]^d; reference
triangle with vertices (0,0), (1,0), (0,1); reference tetrahedron with
vertices (0,0,0), (1,0,0), (0,1,0), (0,0,1).  Hexahedra use the tensor space
Q^k with Gauss-Lobatto-Legendre (GLL) nodes, triangles and tetrahedra the
complete space P^k with equispaced nodes (Welter & Nguyen, Sec. 2.1 defines P^k on simplices;
the hexahedral workloads need tensor Q^k to reach 16 / 9 dofs per face).
"""
import numpy as np
from numpy.polynomial import legendre as L


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] (exact to degree 2n-1)."""
    x, w = L.leggauss(n)
    return x, w


def gll_nodes(k):
    """k+1 Gauss-Lobatto-Legendre nodes on [-1, 1]."""
    if k == 0:
        return np.array([0.0])
    interior = L.Legendre.basis(k).deriv().roots()
    return np.concatenate([[-1.0], np.sort(interior.real), [1.0]])


def lagrange_1d(nodes, t):
    """Values and derivatives of the Lagrange polynomials through `nodes`.

    Returns (phi, dphi), each of shape (len(t), len(nodes)).
    Built from a Legendre Vandermonde matrix for conditioning.
    """
    nodes = np.asarray(nodes, float)
    t = np.atleast_1d(np.asarray(t, float))
    n = len(nodes)
    V = L.legvander(nodes, n - 1)                     # V[i, a] = P_a(x_i)
    Cinv = np.linalg.inv(V)                           # phi_j = sum_a P_a C[a, j]
    Vt = L.legvander(t, n - 1)
    dVt = np.zeros_like(Vt)
    for a in range(n):
        c = np.zeros(n)
        c[a] = 1.0
        dVt[:, a] = L.legval(t, L.legder(c))
    return Vt @ Cinv, dVt @ Cinv


# ---------------------------------------------------------------- hexahedra
def hex_ref(k):
    """Tensor Q^k basis data on [-1,1]^3.

    Node ordering: i + (k+1)*(j + (k+1)*l), x fastest.
    Returns nodes (P_E, 3).
    """
    g = gll_nodes(k)
    n1 = k + 1
    X = np.array([[g[i], g[j], g[l]] for l in range(n1) for j in range(n1) for i in range(n1)])
    return X


def hex_basis(k, pts):
    """phi (npts, P_E) and reference gradients (npts, P_E, 3) of Q^k at pts (npts, 3)."""
    g = gll_nodes(k)
    n1 = k + 1
    px, dpx = lagrange_1d(g, pts[:, 0])
    py, dpy = lagrange_1d(g, pts[:, 1])
    pz, dpz = lagrange_1d(g, pts[:, 2])
    npt = pts.shape[0]
    phi = np.einsum('qi,qj,ql->qlji', px, py, pz).reshape(npt, n1 ** 3)
    gx = np.einsum('qi,qj,ql->qlji', dpx, py, pz).reshape(npt, n1 ** 3)
    gy = np.einsum('qi,qj,ql->qlji', px, dpy, pz).reshape(npt, n1 ** 3)
    gz = np.einsum('qi,qj,ql->qlji', px, py, dpz).reshape(npt, n1 ** 3)
    return phi, np.stack([gx, gy, gz], axis=-1)


def quad_basis(k, st):
    """Q^k basis on the reference square at points st (npts, 2); node order i + (k+1) j."""
    g = gll_nodes(k)
    ps, _ = lagrange_1d(g, st[:, 0])
    pt, _ = lagrange_1d(g, st[:, 1])
    return np.einsum('qi,qj->qji', ps, pt).reshape(st.shape[0], (k + 1) ** 2)


def quad_nodes(k):
    g = gll_nodes(k)
    return np.array([[g[i], g[j]] for j in range(k + 1) for i in range(k + 1)])


def hex_volume_rule(n):
    x, w = gauss_legendre(n)
    pts = np.array([[x[i], x[j], x[l]] for l in range(n) for j in range(n) for i in range(n)])
    wts = np.array([w[i] * w[j] * w[l] for l in range(n) for j in range(n) for i in range(n)])
    return pts, wts


def square_rule(n):
    x, w = gauss_legendre(n)
    st = np.array([[x[i], x[j]] for j in range(n) for i in range(n)])
    ws = np.array([w[i] * w[j] for j in range(n) for i in range(n)])
    return st, ws


# Local faces of the reference hexahedron: (fixed axis, fixed value, free axes).
HEX_FACES = [(0, -1.0, (1, 2)), (0, 1.0, (1, 2)),
             (1, -1.0, (0, 2)), (1, 1.0, (0, 2)),
             (2, -1.0, (0, 1)), (2, 1.0, (0, 1))]
# Vertex ordering of the reference hexahedron: bit 0 -> x, bit 1 -> y, bit 2 -> z.
HEX_VERTS = np.array([[-1, -1, -1], [1, -1, -1], [-1, 1, -1], [1, 1, -1],
                      [-1, -1, 1], [1, -1, 1], [-1, 1, 1], [1, 1, 1]], float)


def hex_face_points(l, st):
    """Map face-parameter points st (n, 2) of local face l into the reference cube."""
    ax, val, (a0, a1) = HEX_FACES[l]
    P = np.zeros((st.shape[0], 3))
    P[:, ax] = val
    P[:, a0] = st[:, 0]
    P[:, a1] = st[:, 1]
    return P


def hex_face_vertices(l):
    """Local vertex ids of face l (the 4 corners)."""
    ax, val, _ = HEX_FACES[l]
    return [v for v in range(8) if HEX_VERTS[v, ax] == val]


def trilinear(X8, ref):
    """Physical points and Jacobians of the trilinear map of a batch of hexahedra.

    X8: (E, 8, 3) vertex coordinates; ref: (n, 3) reference points.
    Returns x (E, n, 3) and Jac (E, n, 3, 3) with Jac[..., a, b] = dx_a / dxi_b.
    """
    s = HEX_VERTS  # (8, 3)
    N = np.prod(1.0 + ref[:, None, :] * s[None, :, :], axis=2) / 8.0       # (n, 8)
    dN = np.zeros((ref.shape[0], 8, 3))
    for b in range(3):
        other = [c for c in range(3) if c != b]
        dN[:, :, b] = s[None, :, b] * np.prod(1.0 + ref[:, None, other] * s[None, :, other], axis=2) / 8.0
    x = np.einsum('nv,evd->end', N, X8)
    Jac = np.einsum('nvb,eva->enab', dN, X8)
    return x, Jac


# ---------------------------------------------------------------- triangles
def tri_nodes(k):
    """Equispaced P^k nodes on the reference triangle, ordered by rows of y."""
    return np.array([[i / k, j / k] for j in range(k + 1) for i in range(k + 1 - j)])


def _tri_monomials(k):
    return [(a, b) for b in range(k + 1) for a in range(k + 1 - b)]


def tri_basis(k, pts):
    """phi (n, P_E) and reference gradients (n, P_E, 2) of nodal P^k."""
    mons = _tri_monomials(k)
    X = tri_nodes(k)
    # shift to the centroid for conditioning
    c = np.array([1.0 / 3.0, 1.0 / 3.0])
    V = np.array([[(x[0] - c[0]) ** a * (x[1] - c[1]) ** b for (a, b) in mons] for x in X])
    Cinv = np.linalg.inv(V)
    px, py = pts[:, 0] - c[0], pts[:, 1] - c[1]
    Vt = np.stack([px ** a * py ** b for (a, b) in mons], axis=1)
    dx = np.stack([a * px ** max(a - 1, 0) * py ** b if a > 0 else np.zeros_like(px) for (a, b) in mons], axis=1)
    dy = np.stack([b * px ** a * py ** max(b - 1, 0) if b > 0 else np.zeros_like(px) for (a, b) in mons], axis=1)
    return Vt @ Cinv, np.stack([dx @ Cinv, dy @ Cinv], axis=-1)


def tri_rule(n):
    """Collapsed (Duffy) Gauss rule with n x n points on the reference triangle."""
    x, w = gauss_legendre(n)
    u = (x + 1) / 2
    wu = w / 2
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            pts.append([u[i], u[j] * (1 - u[i])])
            wts.append(wu[i] * wu[j] * (1 - u[i]))
    return np.array(pts), np.array(wts)


# Local edges of the reference triangle: edge l is opposite vertex l.
TRI_EDGES = [(1, 2), (2, 0), (0, 1)]
TRI_VERTS = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])


def tri_edge_points(l, t):
    a, b = TRI_EDGES[l]
    t = np.asarray(t)[:, None]
    return (1 - t) / 2 * TRI_VERTS[a] + (1 + t) / 2 * TRI_VERTS[b]


# ------------------------------------------------------------- tetrahedra
TET_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
# Local face l is opposite vertex l; its corners (A, B, C) in this order
# parametrise it as A + s (B - A) + t (C - A) over the reference triangle.
TET_FACES = [(1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)]


def tet_nodes(k):
    """Equispaced P^k nodes on the reference tetrahedron, x fastest."""
    return np.array([[i / k, j / k, l / k] for l in range(k + 1) for j in range(k + 1 - l)
                     for i in range(k + 1 - l - j)])


def _tet_monomials(k):
    return [(a, b, c) for c in range(k + 1) for b in range(k + 1 - c) for a in range(k + 1 - b - c)]


def tet_basis(k, pts):
    """phi (n, P_E) and reference gradients (n, P_E, 3) of nodal P^k on the
    reference tetrahedron (monomials about the centroid, inverted Vandermonde)."""
    mons = _tet_monomials(k)
    c = np.full(3, 0.25)
    X = tet_nodes(k) - c
    V = np.array([[x[0] ** a * x[1] ** b * x[2] ** cc for (a, b, cc) in mons] for x in X])
    Cinv = np.linalg.inv(V)
    P = np.asarray(pts, float) - c
    px, py, pz = P[:, 0], P[:, 1], P[:, 2]

    def pw(v, e):
        return v ** e if e > 0 else np.ones_like(v)

    def dpw(v, e):
        return e * v ** (e - 1) if e > 0 else np.zeros_like(v)
    Vt = np.stack([pw(px, a) * pw(py, b) * pw(pz, cc) for (a, b, cc) in mons], axis=1)
    dx = np.stack([dpw(px, a) * pw(py, b) * pw(pz, cc) for (a, b, cc) in mons], axis=1)
    dy = np.stack([pw(px, a) * dpw(py, b) * pw(pz, cc) for (a, b, cc) in mons], axis=1)
    dz = np.stack([pw(px, a) * pw(py, b) * dpw(pz, cc) for (a, b, cc) in mons], axis=1)
    return Vt @ Cinv, np.stack([dx @ Cinv, dy @ Cinv, dz @ Cinv], axis=-1)


def tet_rule(n):
    """Collapsed (Duffy) Gauss rule with n^3 points on the reference
    tetrahedron: x = u, y = v (1 - u), z = w (1 - u)(1 - v), weight
    (1 - u)^2 (1 - v)."""
    x, w = gauss_legendre(n)
    u = (x + 1) / 2
    wu = w / 2
    pts, wts = [], []
    for i in range(n):
        for j in range(n):
            for l in range(n):
                a, b, c = u[i], u[j], u[l]
                pts.append([a, b * (1 - a), c * (1 - a) * (1 - b)])
                wts.append(wu[i] * wu[j] * wu[l] * (1 - a) ** 2 * (1 - b))
    return np.array(pts), np.array(wts)


def tet_face_points(l, st):
    """Map reference-triangle points st (n, 2) onto local face l."""
    A, Bv, C = (TET_VERTS[v] for v in TET_FACES[l])
    st = np.asarray(st, float)
    return A[None, :] + st[:, :1] * (Bv - A)[None, :] + st[:, 1:2] * (C - A)[None, :]


def tet_face_normal(l):
    """Outward normal of local face l scaled by its area element in (s, t):
    (B - A) x (C - A), oriented away from the opposite vertex."""
    A, Bv, C = (TET_VERTS[v] for v in TET_FACES[l])
    n = np.cross(Bv - A, C - A)
    if np.dot(n, TET_VERTS[l] - A) > 0:
        n = -n
    return n


# --------------------------------------------------------- quadrilaterals
# Reference square [-1,1]^2; vertex v at (bit 0 -> x, bit 1 -> y); local
# face (edge) l = 2 axis + side fixes coordinate `axis` at -1 / +1, its
# parameter t runs along the other coordinate.
QUAD_VERTS = np.array([[-1, -1], [1, -1], [-1, 1], [1, 1]], float)


def quad_face_vertices(l):
    ax, side = l // 2, l % 2
    val = 1.0 if side else -1.0
    return [v for v in range(4) if QUAD_VERTS[v, ax] == val]


def quad_face_points(l, t):
    ax, side = l // 2, l % 2
    t = np.asarray(t, float).ravel()
    P = np.zeros((t.shape[0], 2))
    P[:, ax] = 1.0 if side else -1.0
    P[:, 1 - ax] = t
    return P


def quad_vol_basis(k, pts):
    """Q^k on the reference square at pts (n, 2): phi (n, P_E) and reference
    gradients (n, P_E, 2); node (i, j) at index i + (k+1) j."""
    g = gll_nodes(k)
    px, dpx = lagrange_1d(g, pts[:, 0])
    py, dpy = lagrange_1d(g, pts[:, 1])
    n = pts.shape[0]
    phi = np.einsum('qi,qj->qji', px, py).reshape(n, -1)
    gx = np.einsum('qi,qj->qji', dpx, py).reshape(n, -1)
    gy = np.einsum('qi,qj->qji', px, dpy).reshape(n, -1)
    return phi, np.stack([gx, gy], axis=-1)


def bilinear(X4, ref):
    """Physical points and Jacobians of the bilinear map of a batch of
    quadrilaterals: X4 (E, 4, 2), ref (n, 2) -> x (E, n, 2), Jac (E, n, 2, 2)."""
    s = QUAD_VERTS
    N = np.prod(1.0 + ref[:, None, :] * s[None, :, :], axis=2) / 4.0
    dN = np.zeros((ref.shape[0], 4, 2))
    for b in range(2):
        o = 1 - b
        dN[:, :, b] = s[None, :, b] * (1.0 + ref[:, None, o] * s[None, :, o]) / 4.0
    return np.einsum('nv,evd->end', N, X4), np.einsum('nvb,eva->enab', dN, X4)
