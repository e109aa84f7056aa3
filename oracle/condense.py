"""Static condensation (Welter & Nguyen, Sec. 2.3 Eq. 13a-c; Sec. 4.1-4.2,
Eqs. w15-w22).  Test infrastructure: see oracle/__init__.py."""
import numpy as np


def q_blocks_dense(Me, Bd, Cd, M, n_lfe):
    """Dense A, B, C of Eq. matrixform from the compact blocks of Eq. w16:
    A = I_{M D} (x) M^e, B_{(a,c,i),(b,j)} = delta_ab B_c[i,j],
    C_{(a,c,i),(l,b,j)} = delta_ab C_c[i, l*P_F + j]."""
    E, D, PE, _ = Bd.shape
    PF = Cd.shape[3] // n_lfe
    nq, nu, nh = M * D * PE, M * PE, n_lfe * M * PF
    A = np.zeros((E, nq, nq))
    Bm = np.zeros((E, nq, nu))
    Cm = np.zeros((E, nq, nh))
    for a in range(M):
        for c in range(D):
            r0 = (a * D + c) * PE
            A[:, r0:r0 + PE, r0:r0 + PE] = Me
            Bm[:, r0:r0 + PE, a * PE:(a + 1) * PE] = Bd[:, c]
            for l in range(n_lfe):
                c0 = (l * M + a) * PF
                Cm[:, r0:r0 + PE, c0:c0 + PF] = Cd[:, c, :, l * PF:(l + 1) * PF]
    return A, Bm, Cm


def condense_direct(blk, M, n_lfe):
    """Eq. 13b-c element by element, with the dense local matrix
    [A B; D E] solved by LU (numpy.linalg.solve):
      Kbar = J - [G H] [A B; D E]^{-1} [C; F]
      rbar = r_uh - [G H] [A B; D E]^{-1} [r_q; r_u],   r_q = 0 (Sec. 4.1)."""
    A, Bm, Cm = q_blocks_dense(blk['Me'], blk['Bd'], blk['Cd'], M, n_lfe)
    Dm, Em, Fm, Gm, Hm, Jm = (blk[x] for x in 'DEFGHJ')
    E = A.shape[0]
    local = np.concatenate([np.concatenate([A, Bm], axis=2), np.concatenate([Dm, Em], axis=2)], axis=1)
    CF = np.concatenate([Cm, Fm], axis=1)
    GH = np.concatenate([Gm, Hm], axis=2)
    R = blk['ru'].shape[2]
    rqu = np.concatenate([np.zeros((E, A.shape[1], R)), blk['ru']], axis=1)
    X = np.linalg.solve(local, np.concatenate([CF, rqu], axis=2))
    nh = Cm.shape[2]
    Kbar = Jm - GH @ X[:, :, :nh]
    rbar = blk['ruh'] - GH @ X[:, :, nh:]
    return Kbar, rbar


def condense_local(blk, M, n_lfe):
    """The local-solver route of Sec. 4.1-4.2:
      Eq. w16 : A^{-1} via (M^e)^{-1}, per component and direction;
      Eq. w19 : Ebar = E - D A^{-1} B,  Fbar = F - D A^{-1} C;
      Eq. w21 : Hbar = H - G A^{-1} B,  Jbar = J - G A^{-1} C;
      Eq. w22 : Kbar = Jbar - Hbar Ebar^{-1} Fbar,
                rbar = r_uh - Hbar Ebar^{-1} r_u.
    Returns Kbar, rbar and the data the recovery of Eq. w19 / w16 needs."""
    Me, Bd, Cd = blk['Me'], blk['Bd'], blk['Cd']
    E, D, PE, _ = Bd.shape
    Minv = np.linalg.inv(Me)
    MinvB = np.einsum('eik,edkj->edij', Minv, Bd)          # (M^e)^{-1} B_d
    MinvC = np.einsum('eik,edkj->edij', Minv, Cd)          # (M^e)^{-1} C_d
    A, Bm, Cm = q_blocks_dense(Me, Bd, Cd, M, n_lfe)
    # A^{-1} B and A^{-1} C assembled from the per-(component, direction) pieces
    AinvB = np.zeros_like(Bm)
    AinvC = np.zeros_like(Cm)
    PF = Cd.shape[3] // n_lfe
    for a in range(M):
        for c in range(D):
            r0 = (a * D + c) * PE
            AinvB[:, r0:r0 + PE, a * PE:(a + 1) * PE] = MinvB[:, c]
            for l in range(n_lfe):
                c0 = (l * M + a) * PF
                AinvC[:, r0:r0 + PE, c0:c0 + PF] = MinvC[:, c, :, l * PF:(l + 1) * PF]
    Ebar = blk['E'] - blk['D'] @ AinvB
    Fbar = blk['F'] - blk['D'] @ AinvC
    Hbar = blk['H'] - blk['G'] @ AinvB
    Jbar = blk['J'] - blk['G'] @ AinvC
    EinvF = np.linalg.solve(Ebar, Fbar)
    Einvr = np.linalg.solve(Ebar, blk['ru'])
    Kbar = Jbar - Hbar @ EinvF
    rbar = blk['ruh'] - Hbar @ Einvr
    rec = dict(MinvB=MinvB, MinvC=MinvC, Ebar=Ebar, Fbar=Fbar, ru=blk['ru'])
    return Kbar, rbar, rec
