"""Dense linear algebra steps of the TDVP update, written out plainly.

* ``qr_complete``  -- QR that moves the orthogonality centre (gauge move of
  Sec. "Tensor network simulations"), with the deterministic completion of
  rank-deficient bases (columns with residual <= 1e-10 |A|_F
  replaced by unit vectors in a fixed candidate order).
* ``krylov_expm``  -- Lanczos approximation of exp(z H) v (the local
  propagator TDVP needs; Krylov parameters: m_max = 30, tolerance 1e-13).
"""
import numpy as np

QR_RANK_TOL = 1e-10          # |R_kk| <= tol * ||A||_F  -> column treated as dependent
COMPLETION_MIN_RES2 = 0.25   # candidate accepted if its residual norm^2 >= 1/4
KRYLOV_TOL = 1e-13
KRYLOV_MMAX = 30


def completion_order(da, db, a_allowed=None, b_allowed=None):
    """Row candidates e_(a,b) of a (da*db) x D matricisation, ordered by (a+b, a).

    Rows are numbered a*db + b (a = first remaining leg, b = second).  A leg
    that is a padding leaf only allows index 0 (padding atoms stay in |0>), so
    no basis vector is spent on states the dynamics never reaches."""
    a_allowed = range(da) if a_allowed is None else a_allowed
    b_allowed = range(db) if b_allowed is None else b_allowed
    rows = [(a, b) for a in a_allowed for b in b_allowed]
    rows.sort(key=lambda ab: (ab[0] + ab[1], ab[0]))
    return [a * db + b for a, b in rows]


def qr_complete(A, row_order=None, tol=QR_RANK_TOL):
    """A = Q R with Q^H Q = I, R upper triangular, R_kk real >= 0.

    Column-by-column classical Gram-Schmidt with one re-orthogonalisation
    pass (CGS2).  Column k is *dependent* when its residual after both passes
    has norm <= tol * ||A||_F (tol = 1e-10); then R_kk = 0 and Q's column k is filled after
    all columns are processed, in increasing k, by the first candidate unit
    vector e_c (candidates in ``row_order``) with 1 - ||Q^H e_c||^2 >= 1/4
    (else the candidate with the largest such residual, first in order on
    ties), orthogonalised twice against all of Q and normalised.  The rows of R
    of dependent columns stay zero, so A = Q R still holds.
    """
    A = np.asarray(A, dtype=np.complex128)
    M, D = A.shape
    if M < D:
        raise ValueError("qr_complete needs a tall matrix")
    if row_order is None:
        row_order = list(range(M))
    Q = np.zeros((M, D), dtype=np.complex128)
    R = np.zeros((D, D), dtype=np.complex128)
    normA = np.linalg.norm(A)
    dependent = []
    for k in range(D):
        v = A[:, k].copy()
        h1 = Q[:, :k].conj().T @ v
        v = v - Q[:, :k] @ h1
        h2 = Q[:, :k].conj().T @ v
        v = v - Q[:, :k] @ h2
        R[:k, k] = h1 + h2
        nv = np.linalg.norm(v)
        if normA == 0.0 or nv <= tol * normA:
            dependent.append(k)
            R[k, k] = 0.0
        else:
            Q[:, k] = v / nv
            R[k, k] = nv
    for k in dependent:
        best, best_res = None, -1.0
        chosen = None
        for c in row_order:
            w = Q[c, :].conj()                 # Q^H e_c
            res = 1.0 - np.real(np.vdot(w, w))
            if res >= COMPLETION_MIN_RES2:
                chosen = c
                break
            if res > best_res:
                best, best_res = c, res
        if chosen is None:
            chosen = best
        v = np.zeros(M, dtype=np.complex128)
        v[chosen] = 1.0
        for _ in range(2):
            v = v - Q @ (Q.conj().T @ v)
        Q[:, k] = v / np.linalg.norm(v)
    return Q, R


def tridiag_expm_e1(alpha, beta, z):
    """exp(z T) e_1 for the real symmetric tridiagonal T (diag alpha, off-diag beta).

    Uses the eigendecomposition of T (numpy.linalg.eigh)."""
    m = len(alpha)
    T = np.diag(np.asarray(alpha, dtype=np.float64))
    for i in range(m - 1):
        T[i, i + 1] = T[i + 1, i] = beta[i]
    lam, U = np.linalg.eigh(T)
    return U @ (np.exp(z * lam) * U[0, :])


def hessenberg_expm_e1(Hm, z):
    """exp(z H_m) e_1 for a small upper Hessenberg H_m (scipy.linalg.expm)."""
    from scipy.linalg import expm
    return expm(z * np.asarray(Hm, dtype=np.complex128))[:, 0]


def krylov_expm(apply_H, v0, z, tol=KRYLOV_TOL, m_max=KRYLOV_MMAX, stats=None, hermitian=True):
    """exp(z H) v0 for H given as a function, z = -i tau or +i tau.

    Hermitian H: Lanczos with full re-orthogonalisation (two classical
    Gram-Schmidt passes against the whole basis).  alpha_j = Re(<v_j, H v_j>)
    summed over both passes, beta_j = norm of the residual.  After step j the
    small problem c = exp(z T_j) e_1 is solved and the run stops when
    beta_j * |c_j| <= tol (Saad's a-posteriori estimate) or j = m_max.
    Non-Hermitian H (``hermitian=False``, the open system of Eq. 3): Arnoldi,
    the same two passes, with column j of the Hessenberg matrix H_j the sum
    of both passes' projections and H_j(j+1, j) = beta_j; c = exp(z H_j) e_1.
    Returns ||v0|| * sum_i c_i v_i.
    """
    nrm = np.linalg.norm(v0)
    if nrm == 0.0:
        return np.zeros_like(v0)
    V = [v0 / nrm]
    alpha, beta = [], []
    Hm = np.zeros((m_max + 1, m_max), dtype=np.complex128)
    c = None
    for j in range(m_max):
        w = apply_H(V[j])
        h1 = np.array([np.vdot(vi, w) for vi in V])
        for hi, vi in zip(h1, V):
            w = w - hi * vi
        h2 = np.array([np.vdot(vi, w) for vi in V])
        for hi, vi in zip(h2, V):
            w = w - hi * vi
        alpha.append(float(np.real(h1[j] + h2[j])))
        b = float(np.linalg.norm(w))
        if hermitian:
            c = tridiag_expm_e1(alpha, beta, z)
        else:
            Hm[:j + 1, j] = h1 + h2
            c = hessenberg_expm_e1(Hm[:j + 1, :j + 1], z)
        Hm[j + 1, j] = b
        err = b * abs(c[-1])
        if err <= tol or j == m_max - 1:
            if stats is not None:
                stats.append((j + 1, err))
            break
        beta.append(b)
        V.append(w / b)
    out = np.zeros_like(v0)
    for ci, vi in zip(c, V):
        out = out + ci * vi
    return nrm * out
