"""Structured meshes and their face connectivity.

Faces are deduplicated by their sorted vertex tuple.  Face ids are assigned in
order of first appearance when elements are visited in order and, within an
element, local faces in order; so the first element of a face (e1) always has
the smaller element id.  This gives the maps the assembly needs: f(e, l)
(elem_face) and face -> (e1, l1, e2, l2) (face_elem), as described for the
face-based assembly and for the ASM update (Welter & Nguyen, Sec. 4.2, 4.6).
"""
from dataclasses import dataclass
import numpy as np

from .basis import hex_face_vertices, quad_face_vertices, TRI_EDGES, TET_FACES


@dataclass
class Mesh:
    dim: int
    kind: str                   # 'tri' or 'hex'
    verts: np.ndarray           # (NV, dim)
    elems: np.ndarray           # (NE, 3) or (NE, 8) vertex ids
    elem_face: np.ndarray       # (NE, nlfe) int32 global face id
    face_elem: np.ndarray       # (NF, 4) int32: e1, l1, e2, l2 (e2 = l2 = -1 on the boundary)
    face_boundary: np.ndarray   # (NF,) uint8

    @property
    def n_elem(self):
        return self.elems.shape[0]

    @property
    def n_face(self):
        return self.face_elem.shape[0]

    @property
    def n_lfe(self):
        return self.elem_face.shape[1]


def _build_faces(local_face_verts, elems):
    ne = elems.shape[0]
    nlfe = len(local_face_verts)
    elem_face = np.empty((ne, nlfe), np.int32)
    key_to_face = {}
    face_elem = []
    for e in range(ne):
        for l, lv in enumerate(local_face_verts):
            key = tuple(sorted(int(elems[e, v]) for v in lv))
            f = key_to_face.get(key)
            if f is None:
                f = len(face_elem)
                key_to_face[key] = f
                face_elem.append([e, l, -1, -1])
            else:
                assert face_elem[f][2] == -1, "face shared by more than two elements"
                face_elem[f][2] = e
                face_elem[f][3] = l
            elem_face[e, l] = f
    face_elem = np.array(face_elem, np.int32)
    boundary = (face_elem[:, 2] < 0).astype(np.uint8)
    return elem_face, face_elem, boundary


def tri_mesh(n):
    """Unit square with n x n squares, each split along the diagonal from
    (x_i, y_j) to (x_{i+1}, y_{j+1}) into two counter-clockwise triangles."""
    xs = np.linspace(0.0, 1.0, n + 1)
    verts = np.array([[xs[i], xs[j]] for j in range(n + 1) for i in range(n + 1)])
    vid = lambda i, j: j * (n + 1) + i
    elems = []
    for j in range(n):
        for i in range(n):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            elems.append([a, b, c])
            elems.append([a, c, d])
    elems = np.array(elems, np.int64)
    ef, fe, fb = _build_faces([list(e) for e in TRI_EDGES], elems)
    return Mesh(2, 'tri', verts, elems, ef, fe, fb)


def hex_mesh(n, perturb=0.0, seed=None):
    """n^3 hexahedra on [0,1]^3.  With perturb > 0, every interior vertex moves
    by perturb * h * r * s, s a uniform random unit vector and r ~ U[0,1]
    (seeded); boundary vertices stay fixed."""
    return box_hex_mesh((n, n, n), (1.0, 1.0, 1.0), perturb, seed)


def box_hex_mesh(counts, lengths, perturb=0.0, seed=None):
    """nx x ny x nz hexahedra on (0,Lx) x (0,Ly) x (0,Lz), e.g. the
    (0,5) x (0,1) x (0,1) cantilever beam of Sec. 6.2 with 10x2x2 .. 40x8x8
    elements.  Vertex and element ids run x fastest; perturb as in hex_mesh,
    relative to the smallest cell width."""
    nx, ny, nz = counts
    lx, ly, lz = lengths
    axes = [np.linspace(0.0, L, c + 1) for c, L in zip(counts, lengths)]
    verts = np.array([[axes[0][i], axes[1][j], axes[2][l]]
                      for l in range(nz + 1) for j in range(ny + 1) for i in range(nx + 1)])
    if perturb > 0.0:
        h = min(L / c for c, L in zip(counts, lengths))
        rng = np.random.default_rng(seed)
        nv = verts.shape[0]
        s = rng.normal(size=(nv, 3))
        s /= np.linalg.norm(s, axis=1, keepdims=True)
        r = rng.uniform(0.0, 1.0, size=(nv, 1))
        top = np.array([lx, ly, lz])
        interior = np.all((verts > 1e-12) & (verts < top - 1e-12), axis=1)
        verts = verts + (perturb * h * r * s) * interior[:, None]
    vid = lambda i, j, l: (l * (ny + 1) + j) * (nx + 1) + i
    elems = []
    for l in range(nz):
        for j in range(ny):
            for i in range(nx):
                elems.append([vid(i + di, j + dj, l + dl) for dl in (0, 1) for dj in (0, 1) for di in (0, 1)])
    elems = np.array(elems, np.int64)
    ef, fe, fb = _build_faces([hex_face_vertices(l) for l in range(6)], elems)
    return Mesh(3, 'hex', verts, elems, ef, fe, fb)


def tet_mesh(n, lo=0.0, hi=1.0, hole=0.0):
    """Kuhn subdivision of the n^3 cubes of (lo, hi)^3 into six tetrahedra each
    (the paths from the cube's lowest to its highest corner through the
    orderings of the three axes; every cube is split the same way, so the mesh
    is conforming).  Cubes whose centres lie within `hole` of the box centre
    in every coordinate are left out (an obstacle with reentrant edges and
    corners).  Every tetrahedron is positively oriented."""
    xs = np.linspace(lo, hi, n + 1)
    verts = np.array([[xs[i], xs[j], xs[l]] for l in range(n + 1) for j in range(n + 1) for i in range(n + 1)])
    vid = lambda i, j, l: (l * (n + 1) + j) * (n + 1) + i
    mid = 0.5 * (lo + hi)
    h = (hi - lo) / n
    orders = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    elems = []
    for l in range(n):
        for j in range(n):
            for i in range(n):
                c = np.array([lo + (i + 0.5) * h, lo + (j + 0.5) * h, lo + (l + 0.5) * h])
                if hole > 0.0 and np.all(np.abs(c - mid) < hole):
                    continue
                for od in orders:
                    p = [i, j, l]
                    tet = [vid(*p)]
                    for ax in od:
                        p[ax] += 1
                        tet.append(vid(*p))
                    X = verts[tet]
                    if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)) < 0:
                        tet[2], tet[3] = tet[3], tet[2]
                    elems.append(tet)
    elems = np.array(elems, np.int64)
    used = np.unique(elems)
    remap = -np.ones(verts.shape[0], np.int64)
    remap[used] = np.arange(len(used))
    verts = verts[used]
    elems = remap[elems]
    ef, fe, fb = _build_faces([list(f) for f in TET_FACES], elems)
    return Mesh(3, 'tet', verts, elems, ef, fe, fb)


def quad_mesh(n):
    """Unit square with n x n quadrilaterals; vertex v of an element at
    (x_i + (v & 1) h, y_j + (v >> 1) h), elements x fastest."""
    xs = np.linspace(0.0, 1.0, n + 1)
    verts = np.array([[xs[i], xs[j]] for j in range(n + 1) for i in range(n + 1)])
    vid = lambda i, j: j * (n + 1) + i
    elems = np.array([[vid(i, j), vid(i + 1, j), vid(i, j + 1), vid(i + 1, j + 1)]
                      for j in range(n) for i in range(n)], np.int64)
    ef, fe, fb = _build_faces([quad_face_vertices(l) for l in range(4)], elems)
    return Mesh(2, 'quad', verts, elems, ef, fe, fb)
