"""Preconditioners (Welter & Nguyen, Sec. 3.2-3.4 and Sec. 4.5-4.7).
Test infrastructure: see oracle/__init__.py.

Block-Jacobi  : the inverse of every diagonal face block K_ff (Sec. 4.5).
ASM           : one-element subdomains, K_e = R_e K R_e^T over the element's
                free faces; P^{-1} = sum_e R_e^T K_e^{-1} R_e (Sec. 3.3, 4.6).
Polynomial    : p(A) = sum_j prod_{i<j} (I - A/theta_i) / theta_j with the
                harmonic Ritz values of one Arnoldi(P) cycle (MGS) from a
                random vector, Leja-ordered with conjugate pairs kept
                together (Sec. 3.4, 4.7).  For hybrids A = M^{-1} K.
Chebyshev     : the Chebyshev iteration polynomial on [alpha, beta] (not in
                the paper; bounds from Ritz values of the same operator).
"""
import numpy as np
import scipy.sparse as sp


# ------------------------------------------------------------ block-Jacobi
def bj_setup(K, bsz):
    """Inverses of the diagonal bsz x bsz blocks of K (LU with partial
    pivoting, via numpy.linalg.inv)."""
    n = K.shape[0]
    nf = n // bsz
    Kc = K.tocsr()
    blocks = np.empty((nf, bsz, bsz))
    for f in range(nf):
        s = slice(f * bsz, (f + 1) * bsz)
        blocks[f] = Kc[s, s].toarray()
    return np.linalg.inv(blocks)


def bj_apply(Binv, y):
    nf, b, _ = Binv.shape
    return np.einsum('fij,fj->fi', Binv, y.reshape(nf, b)).reshape(-1)


# -------------------------------------------------------------------- ASM
def asm_setup(K, elem_dofs):
    """elem_dofs: list/array of the global free dofs of each element (-1 for
    dofs of Dirichlet faces, which are skipped).  Returns per-element
    (dofs, inverse)."""
    Kc = K.tocsr()
    out = []
    for g in elem_dofs:
        d = g[g >= 0]
        Ke = Kc[d][:, d].toarray()
        out.append((d, np.linalg.inv(Ke)))
    return out


def asm_local_matrices(K, elem_dofs):
    Kc = K.tocsr()
    return [Kc[g[g >= 0]][:, g[g >= 0]].toarray() for g in elem_dofs]


def asm_apply(subs, y):
    z = np.zeros_like(y)
    for d, inv in subs:
        z[d] += inv @ y[d]
    return z


# ------------------------------------------------------------- polynomial
def arnoldi_mgs(apply_A, v0, P):
    """P steps of Arnoldi with modified Gram-Schmidt.  Returns H (k+1, k)
    with k <= P (k < P on breakdown)."""
    n = v0.shape[0]
    V = np.zeros((n, P + 1))
    H = np.zeros((P + 1, P))
    V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(P):
        w = apply_A(V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * abs(H[0, 0]):
            return H[:j + 2, :j + 1]
        V[:, j + 1] = w / H[j + 1, j]
    return H


def harmonic_ritz(H):
    """Eigenvalues of H_PP + h_{P+1,P}^2 H_PP^{-T} e_P e_P^T (Sec. 4.7).
    Falls back to the plain Ritz values eig(H_PP) when H_PP is singular or
    h_{P+1,P} = 0."""
    P = H.shape[1]
    Hs = H[:P, :P]
    hn = H[P, P - 1] if H.shape[0] > P else 0.0
    if hn == 0.0 or np.linalg.cond(Hs, 1) > 1e12:
        return np.linalg.eigvals(Hs)
    eP = np.zeros(P)
    eP[-1] = 1.0
    f = np.linalg.solve(Hs.T, eP)
    Ht = Hs + hn ** 2 * np.outer(f, eP)
    return np.linalg.eigvals(Ht)


def clean_conjugates(theta, rel=1e-12):
    """Values with |Im| <= rel*|theta| become real; every complex value is
    reported once with Im > 0 followed by its conjugate."""
    theta = np.asarray(theta, complex)
    scale = np.max(np.abs(theta)) if len(theta) else 1.0
    re = []
    for t in theta:
        if abs(t.imag) <= rel * scale:
            re.append(complex(t.real, 0.0))
        else:
            re.append(t)
    return np.array(re)


def leja_order(theta):
    """Modified Leja ordering: start at the value of largest modulus, then
    repeatedly take the value maximising sum_k log|theta - theta_k| over the
    values already taken; a value with Im > 0 is followed by its conjugate.
    Ties go to the lowest index."""
    th = clean_conjugates(theta)
    n = len(th)
    remaining = list(range(n))
    out = []

    def take(i):
        out.append(th[i])
        remaining.remove(i)
        if th[i].imag > 0:
            # its conjugate: the remaining value closest to conj(th[i])
            j = min(remaining, key=lambda r: (abs(th[r] - np.conj(th[i])), r))
            out.append(th[j])
            remaining.remove(j)

    def first_key(i):
        return (-abs(th[i]), -th[i].imag, i)
    cand = [i for i in remaining if th[i].imag >= 0]
    take(min(cand, key=first_key))
    while remaining:
        best, bestval = None, -np.inf
        for i in remaining:
            if th[i].imag < 0:
                continue
            with np.errstate(divide='ignore'):
                v = float(np.sum(np.log(np.abs(th[i] - np.array(out)))))
            if v > bestval or best is None:
                best, bestval = i, v
        take(best)
    return np.array(out)


def pp_apply(apply_A, theta, y):
    """z = sum_j prod_{i<j} (I - A/theta_i) y / theta_j, real arithmetic.
    Real theta: w += q/theta; q -= A q / theta.
    Pair a +- ib:  t = 2a q - A q; w += t/(a^2+b^2); q -= A t/(a^2+b^2)
    (the pair update of q is (I - A/theta)(I - A/conj(theta)) q; Sec. 4.7
    prints the second term as K^2 q, which is the same product only when
    the A q term is kept -- the form above keeps it).  The final q update
    is not needed and is skipped."""
    P = len(theta)
    w = np.zeros_like(y)
    q = y.copy()
    i = 0
    while i < P:
        th = theta[i]
        if th.imag == 0.0:
            a = th.real
            w = w + q / a
            if i < P - 1:
                q = q - apply_A(q) / a
            i += 1
        else:
            a, b = th.real, abs(th.imag)
            mod2 = a * a + b * b
            t = 2.0 * a * q - apply_A(q)
            w = w + t / mod2
            if i + 1 < P - 1:
                q = q - apply_A(t) / mod2
            i += 2
    return w


def pp_setup(apply_A, v0, P):
    """Harmonic Ritz values of an Arnoldi(P) cycle from v0, Leja ordered."""
    H = arnoldi_mgs(apply_A, v0, P)
    return leja_order(harmonic_ritz(H))


# -------------------------------------------------------------- Chebyshev
def chebyshev_bounds(apply_A, v0, P):
    """[alpha, beta] = [0.9 min Re theta, 1.1 max Re theta] over the plain
    Ritz values eig(H_PP) of an Arnoldi(P) cycle."""
    H = arnoldi_mgs(apply_A, v0, P)
    k = H.shape[1]
    th = np.linalg.eigvals(H[:k, :k])
    return 0.9 * th.real.min(), 1.1 * th.real.max()


def chebyshev_apply(apply_A, alpha, beta, degree, y):
    """Chebyshev iteration for A z = y from z = 0 (Saad, Iterative Methods for
    Sparse Linear Systems, Alg. 12.1) with degree + 1 steps, i.e. z = p(A) y
    with p of degree `degree` (`degree` applications of A)."""
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma = theta / delta
    rho = 1.0 / sigma
    r = y.copy()
    d = r / theta
    z = np.zeros_like(y)
    for k in range(degree + 1):
        z = z + d
        if k == degree:
            break
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return z
