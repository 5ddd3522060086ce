"""The algebra behind the GPU gauge-move QR, restated in NumPy and checked
against the oracle's column-by-column CGS2 with completion (qr_complete).

The CUDA kernels reorganise CGS2 so that it needs fewer grid-wide
reductions; these tests check, on the CPU, that the reorganised recurrences
compute the same factorisation (to rounding) as the plain rule:

* one reduction per column: the second-pass sums of column k and the
  first-pass sums of column k+1 are taken together, |v2|^2 = |v1|^2 - |h2|^2
  decides column k, and the coefficient of a_{k+1} along the new q_k is
  (c - h2^H g) / |v2| with c = v1^H a_{k+1}, g = Q^H a_{k+1};
* look-ahead: after a dependent column, a window of columns takes both
  passes against the unchanged kept set at once, is decided in order up to
  the first kept column, and the next column's first-pass coefficient along
  that new column follows from (v1_j^H v1_{j+1} - h2_j^H h2_{j+1}) / |v2_j|;
* closed-form completion: the residual of a candidate row c is
  1 - w_c M w_c^H with M = (I - W^H W)^{-1} over the kept columns' rows of
  earlier picks, updated by Sherman-Morrison, and the completed column is
  (e_a - Q_r y with the rows of earlier picks zeroed) / nu.

These are NumPy restatements of the recurrences, not the CUDA code; the GPU
QR itself is compared with qr_complete element by element in
test_gpu_qr.py.
"""
import numpy as np
import pytest

from oracle import linalg as OL

TOL = OL.QR_RANK_TOL
MIN_RES2 = OL.COMPLETION_MIN_RES2


def _fused_cgs2(A, window=0, first_pass_err=None):
    """Kept columns and R by the one-reduction-per-column recurrence, with
    an optional look-ahead of `window` columns after each dependent one.
    first_pass_err (a list) collects, for every first-pass coefficient
    vector the recurrence derives instead of summing it, the deviation
    from Q^H a over |a| (the second pass would hide a wrong one)."""
    A = np.array(A, dtype=np.complex128)
    M, D = A.shape
    fro = np.linalg.norm(A)
    Q = np.zeros((M, D), complex)
    R = np.zeros((D, D), complex)
    dep = np.zeros(D, bool)
    nz = []                                     # kept columns so far

    def check(h1, col):
        if first_pass_err is not None and len(nz):
            a = A[:, col]
            first_pass_err.append(np.max(abs(h1 - Q[:, nz].conj().T @ a)) / max(np.linalg.norm(a), 1e-300))

    def decide(k, v1, h2, h1):
        nrm = np.sqrt(max(np.vdot(v1, v1).real - np.vdot(h2, h2).real, 0.0))
        d = fro == 0.0 or nrm <= TOL * fro
        R[nz, k] = h1 + h2
        if d:
            dep[k] = True
            return None, 0.0
        R[k, k] = nrm
        q = (v1 - Q[:, nz] @ h2) / nrm
        return q, nrm

    # column 0: v1 = a_0 (no kept columns)
    v1, h1 = A[:, 0].copy(), np.zeros(0, complex)
    k = 0
    while k < D:
        Qk = Q[:, nz]
        a_next = A[:, k + 1] if k + 1 < D else np.zeros(M, complex)
        h2, g, c = Qk.conj().T @ v1, Qk.conj().T @ a_next, np.vdot(v1, a_next)
        q, nrm = decide(k, v1, h2, h1)
        if q is not None:
            Q[:, k] = q
            hk = (c - np.vdot(h2, g)) / nrm
            nz.append(k)
            h1 = np.concatenate([g, [hk]])
        else:
            h1 = g
        if k + 1 == D:
            break
        check(h1, k + 1)
        v1 = a_next - Q[:, nz] @ h1
        k += 1
        if q is not None or window == 0:
            continue
        # look-ahead from column k while windows find no kept column
        while k < D:
            W = min(window, D - k)
            Qk = Q[:, nz]
            cols = A[:, k:k + W]
            G = Qk.conj().T @ cols
            V1 = cols - Qk @ G
            H2 = Qk.conj().T @ V1
            after = k + W < D
            a_p = A[:, k + W] if after else None
            js = -1
            for j in range(W):
                qj, nrm = decide(k + j, V1[:, j], H2[:, j], G[:, j])
                if qj is not None:
                    js = j
                    break
            if js < 0:
                k += W
                continue
            Q[:, k + js] = qj
            kn = k + js + 1
            if kn >= D:
                k = D
                break
            if js + 1 < W:
                cx = np.vdot(V1[:, js], V1[:, js + 1])
                hk = (cx - np.vdot(H2[:, js], H2[:, js + 1])) / nrm
                base = G[:, js + 1] + H2[:, js + 1]
            else:
                gp = Qk.conj().T @ a_p
                cp = np.vdot(V1[:, js], a_p)
                hk = (cp - np.vdot(H2[:, js], gp)) / nrm
                base = gp
            nz.append(k + js)
            h1 = np.concatenate([base, [hk]])
            check(h1, kn)
            v1 = A[:, kn] - Q[:, nz] @ h1
            k = kn
            break
        else:
            break
        if k >= D:
            break
    return Q, R, dep


def _closed_form_completion(Q, dep, order):
    M, D = Q.shape
    kept = [k for k in range(D) if not dep[k]]
    Qr = Q[:, kept]
    r = len(kept)
    Minv = np.eye(r, dtype=complex)
    used, acc, ys, nus = set(), [], [], []
    p = 0
    for _ in range(int(dep.sum())):
        chosen = None
        while p < len(order):
            c = order[p]
            p += 1
            if c in used:
                continue
            w = Qr[c, :]
            res = 1 - np.real(w @ Minv @ w.conj())
            if res >= MIN_RES2:
                chosen = c
                break
        if chosen is None:                      # largest residual, earliest on ties
            best, best_res = None, -1.0
            for c in order:
                if c in used:
                    continue
                w = Qr[c, :]
                res = 1 - np.real(w @ Minv @ w.conj())
                if res > best_res:
                    best, best_res = c, res
            chosen = best
            p = len(order)
        w = Qr[chosen, :]
        y = Minv @ w.conj()
        nu2 = 1 - np.real(w @ y)
        used.add(chosen)
        acc.append(chosen)
        ys.append(y)
        nus.append(np.sqrt(nu2))
        Minv = Minv + np.outer(y, w @ Minv) / nu2
    out = Q.copy()
    for t, k in enumerate([k for k in range(D) if dep[k]]):
        u = -(Qr @ ys[t])
        u[acc[:t]] = 0.0
        u[acc[t]] += 1.0
        out[:, k] = u / nus[t]
    return out


def _cases():
    rng = np.random.default_rng(11)

    def cm(m, n):
        return rng.normal(size=(m, n)) + 1j * rng.normal(size=(m, n))
    yield "full rank", cm(60, 12), None
    yield "rank 3 of 20", cm(90, 3) @ cm(3, 20), None
    yield "rank 1 square 27", cm(27, 1) @ cm(1, 27), OL.completion_order(3, 9)
    yield "zero then kept", np.concatenate([np.zeros((50, 4)), cm(50, 2), cm(50, 2) @ cm(2, 6)], axis=1), None
    x = rng.normal(size=9) + 1j * rng.normal(size=9)
    prod = np.kron(x, x * np.exp(-0.5 * np.arange(9)))[:, None]
    yield "product column, square 81", prod @ cm(1, 81), OL.completion_order(9, 9)
    yield "rank 7 of 40", cm(400, 7) @ cm(7, 40), None
    x = cm(120, 4)
    cols = [x[:, 0], 2 * x[:, 0], x[:, 1], x[:, 0] + x[:, 1], x[:, 2], x[:, 1], x[:, 0], x[:, 3],
            x[:, 2] + x[:, 3], x[:, 0] - x[:, 3], x[:, 1], x[:, 3]]
    yield "kept columns scattered among dependent ones", np.stack(cols, axis=1), None


@pytest.mark.parametrize("window", [0, 4, 16])
@pytest.mark.parametrize("name,A,order", list(_cases()))
def test_reorganised_qr_matches_column_by_column_rule(name, A, order, window):
    M, D = A.shape
    order = list(range(M)) if order is None else list(order)
    Qo, Ro = OL.qr_complete(A, order)
    errs = []
    Q, R, dep = _fused_cgs2(A, window, errs)
    assert max(errs, default=0.0) < 1e-12, (name, max(errs))
    assert int(dep.sum()) == int(np.sum(np.abs(np.diag(Ro)) == 0.0)), name
    scale = max(np.max(abs(A)), 1e-300)
    assert np.max(abs(R - Ro)) <= 1e-11 * scale, (name, np.max(abs(R - Ro)))
    Qc = _closed_form_completion(Q, dep, order)
    assert np.max(abs(Qc - Qo)) <= 1e-10, (name, np.max(abs(Qc - Qo)))
    assert np.max(abs(Qc.conj().T @ Qc - np.eye(D))) < 1e-12
