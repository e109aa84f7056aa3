"""Global trace system and element recovery (Welter & Nguyen, Sec. 2.4 and
Sec. 4.2 for assembly; Sec. 2.3 and Eqs. w16, w19 for recovery).
Test infrastructure: see oracle/__init__.py.

The oracle assembles K by its definition, K = sum_e R_e^T Kbar^e R_e over
the free (non-Dirichlet) trace unknowns, as a scipy sparse matrix; it does
not use the face-block storage of the CUDA path.  Dirichlet trace values are
known, so their columns move to the right-hand side:
r = sum_e R_e^T (rbar^e - Kbar^e_{:,Dir} uhat_D).
"""
import numpy as np
import scipy.sparse as sp


def free_face_index(face_dirichlet):
    idx = -np.ones(len(face_dirichlet), np.int64)
    free = np.nonzero(face_dirichlet == 0)[0]
    idx[free] = np.arange(len(free))
    return idx


def element_trace_maps(elem_face, face_dirichlet, M, PF):
    """For every element the global free trace dof of each local trace dof
    (l, a, j) -> (l*M + a)*PF + j, or -1 for a Dirichlet face."""
    E, nl = elem_face.shape
    fidx = free_face_index(face_dirichlet)
    g = np.empty((E, nl, M, PF), np.int64)
    for l in range(nl):
        ff = fidx[elem_face[:, l]]
        base = ff[:, None, None] * (M * PF) + np.arange(M)[None, :, None] * PF + np.arange(PF)[None, None, :]
        g[:, l] = np.where(ff[:, None, None] >= 0, base, -1)
    return g.reshape(E, nl * M * PF)


def dirichlet_element_values(elem_face, uhatD, M, PF):
    """uhat^e restricted to the known Dirichlet values (zero elsewhere):
    (E, nl*M*PF, R)."""
    E, nl = elem_face.shape
    return uhatD[elem_face].reshape(E, nl * M * PF, uhatD.shape[2])


def assemble(Kbar, rbar, elem_face, face_dirichlet, uhatD, M, PF):
    """Returns K (csr, n_dof x n_dof) and r (n_dof, R)."""
    E, n, _ = Kbar.shape
    gmap = element_trace_maps(elem_face, face_dirichlet, M, PF)
    n_dof = int((face_dirichlet == 0).sum()) * M * PF
    rows = np.repeat(gmap[:, :, None], n, axis=2)
    cols = np.repeat(gmap[:, None, :], n, axis=1)
    keep = (rows >= 0) & (cols >= 0)
    K = sp.coo_matrix((Kbar[keep], (rows[keep], cols[keep])), shape=(n_dof, n_dof)).tocsr()
    K.sum_duplicates()
    uD = dirichlet_element_values(elem_face, uhatD, M, PF)
    isD = (gmap < 0)
    re = rbar - Kbar @ (uD * isD[:, :, None])
    R = rbar.shape[2]
    r = np.zeros((n_dof, R))
    for c in range(R):
        np.add.at(r[:, c], gmap[~isD], re[:, :, c][~isD])
    return K, r


def element_traces(uhat_free, elem_face, face_dirichlet, uhatD, M, PF):
    """uhat^e (E, nl*M*PF, R) from the free solution and the Dirichlet values."""
    gmap = element_trace_maps(elem_face, face_dirichlet, M, PF)
    uD = dirichlet_element_values(elem_face, uhatD, M, PF)
    out = uD.copy()
    m = gmap >= 0
    out[m] = uhat_free[gmap[m]]
    return out


def recover(rec, uhat_e, M, n_lfe):
    """Eq. w19: u^e = Ebar^{-1} (r_u - Fbar uhat^e);
    Eq. w16: q^e_{a,d} = -(M^e)^{-1} (B_d u^e_a + C_d uhat^e_a).
    Returns u (E, M*PE, R) and q (E, M*D*PE, R)."""
    u = np.linalg.solve(rec['Ebar'], rec['ru'] - rec['Fbar'] @ uhat_e)
    MinvB, MinvC = rec['MinvB'], rec['MinvC']
    E, D, PE, _ = MinvB.shape
    PF = MinvC.shape[3] // n_lfe
    R = u.shape[2]
    q = np.zeros((E, M * D * PE, R))
    uh = uhat_e.reshape(E, n_lfe, M, PF, R)
    for a in range(M):
        ua = u[:, a * PE:(a + 1) * PE]
        uha = uh[:, :, a].reshape(E, n_lfe * PF, R)
        for d in range(D):
            r0 = (a * D + d) * PE
            q[:, r0:r0 + PE] = -(MinvB[:, d] @ ua + MinvC[:, d] @ uha)
    return u, q


def monolithic_solve(blk, elem_face, face_dirichlet, uhatD, M, n_lfe):
    """Dense solve of the full linear system of Eq. matrixform (all q, u and
    free uhat unknowns at once), for tiny meshes.  Returns q, u (per element)
    and the free trace vector."""
    from .condense import q_blocks_dense
    A, Bm, Cm = q_blocks_dense(blk['Me'], blk['Bd'], blk['Cd'], M, n_lfe)
    E, nq, _ = A.shape
    nu = Bm.shape[2]
    nh = Cm.shape[2]
    PF = nh // (n_lfe * M)
    gmap = element_trace_maps(elem_face, face_dirichlet, M, PF)
    n_dof = int((face_dirichlet == 0).sum()) * M * PF
    nloc = nq + nu
    N = E * nloc + n_dof
    R = blk['ru'].shape[2]
    Kfull = np.zeros((N, N))
    rhs = np.zeros((N, R))
    uD = dirichlet_element_values(elem_face, uhatD, M, PF)
    for e in range(E):
        o = e * nloc
        loc = np.block([[A[e], Bm[e]], [blk['D'][e], blk['E'][e]]])
        CF = np.concatenate([Cm[e], blk['F'][e]], axis=0)
        GH = np.concatenate([blk['G'][e], blk['H'][e]], axis=1)
        Kfull[o:o + nloc, o:o + nloc] = loc
        rhs[o + nq:o + nloc] += blk['ru'][e]
        g = gmap[e]
        fr = g >= 0
        Kfull[o:o + nloc, E * nloc + g[fr]] += CF[:, fr]
        rhs[o:o + nloc] -= CF[:, ~fr] @ uD[e][~fr]
        Kfull[np.ix_(E * nloc + g[fr], np.arange(o, o + nloc))] += GH[fr]
        Kfull[np.ix_(E * nloc + g[fr], E * nloc + g[fr])] += blk['J'][e][np.ix_(fr, fr)]
        rhs[E * nloc + g[fr]] += blk['ruh'][e][fr] - blk['J'][e][np.ix_(fr, ~fr)] @ uD[e][~fr]
    sol = np.linalg.solve(Kfull, rhs)
    loc = sol[:E * nloc].reshape(E, nloc, R)
    return loc[:, :nq], loc[:, nq:], sol[E * nloc:]
