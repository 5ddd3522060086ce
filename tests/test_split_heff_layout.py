"""Host-side layout of the split-precision stacked H_eff (CPU, no GPU).

The split path evaluates H_eff X (Eq. 1 on a 3-leg node, Sec. "Tensor
network simulations") as one long-K contraction per leg u,
    H_eff X = sum_u Q_u x_u P_u,
with the operator stack Q_u = [H_block(u) | n_1 .. n_r of each channel pair
with a = u] and the stacked operand P_u = [X | Z^(p)] whose rows run over the
two other legs (u = 0: b + d1 c; u = 1: a + Pp1 c; u = 2: a + d0 b) and whose
K runs over the leg-u index and the channel index.  The channel
intermediates Z_i = G_i x_b X are written into the K slots of P_a by the
contraction epilogue at float2 position
    (p % pd)*sp1 + (p / pd)*sp2 + q*sq + bi*sbi + bo*sbo
in the kernel's (P row p, Q row q, batch bi, bo) orientation of the
contraction G x_b X, with sp1 = 1 (coalesced stores): for the pairs whose
channel leg a comes after the G leg b (except (1, 0)) X is packed for that
contraction with leg a's index fastest.  This test restates those index maps in NumPy (FP64, no
TF32 split), checks that every write stays inside its planes, and that the
stacked evaluation equals the direct sum of the block and channel terms for
every ordered pair of legs, for tile-aligned and ragged dimensions.
"""
import itertools

import numpy as np
import pytest

BM, BN, BK = 128, 64, 32
BIG = 1 << 30


def rup(x, m):
    return (x + m - 1) // m * m


def apply_leg(M, X, leg):
    return np.moveaxis(np.tensordot(M, X, axes=([1], [leg])), 0, leg)


TRANS = {(2, 0), (2, 1), (1, 2)}


def z_orientation(a, b, d):
    """(Pn, Bi, Bo) and a map (p, q, bi, bo) -> index (i, a, b, c) of Z_i for
    the contraction G x_b X in the kernel's orientation.  For the transposed
    pairs the X operand is packed with leg a's index fastest."""
    d0, d1, d2 = d
    if (a, b) == (2, 0):    # p = c + d2 b', q = a', bi = i
        return dict(Pn=d1 * d2, Bi=None, Bo=1, idx=lambda p, q, bi, bo: (bi, q, p // d2, p % d2))
    if (a, b) == (2, 1):    # p = c + d2 a, q = b', bi = i
        return dict(Pn=d0 * d2, Bi=None, Bo=1, idx=lambda p, q, bi, bo: (bi, p // d2, q, p % d2))
    if (a, b) == (1, 2):    # p = b + d1 a, q = c', bi = i
        return dict(Pn=d0 * d1, Bi=None, Bo=1, idx=lambda p, q, bi, bo: (bi, p // d1, p % d1, q))
    if b == 0:              # p = b' + d1 c, q = a', bi = i
        return dict(Pn=d1 * d2, Bi=None, Bo=1, idx=lambda p, q, bi, bo: (bi, q, p % d1, p // d1))
    if b == 1:              # p = a, bi = c, q = b', bo = i
        return dict(Pn=d0, Bi=d2, Bo=None, idx=lambda p, q, bi, bo: (bo, p, q, bi))
    return dict(Pn=d0 * d1, Bi=None, Bo=1,     # p = a + d0 b, q = c', bi = i
                idx=lambda p, q, bi, bo: (bi, p % d0, p // d0, q))


def out_strides(a, b, d, K2a, Pp1):
    d0, d1, d2 = d
    o = dict(pd=BIG, sp1=1, sp2=0, sq=0, sbi=0, sbo=0)
    if (a, b) == (0, 1):
        o.update(sq=K2a, sbi=d1 * K2a, sbo=d0)
    elif (a, b) == (0, 2):
        o.update(pd=d0, sp2=K2a, sq=d1 * K2a, sbi=d0)
    elif (a, b) == (1, 0):
        o.update(pd=d1, sp2=Pp1 * K2a, sq=K2a, sbi=d1)
    elif (a, b) == (2, 0):
        o.update(pd=d2, sp2=d0 * K2a, sq=K2a, sbi=d2)
    elif (a, b) == (2, 1):
        o.update(pd=d2, sp2=K2a, sq=d0 * K2a, sbi=d2)
    else:   # (1, 2)
        o.update(pd=d1, sp2=K2a, sq=Pp1 * K2a, sbi=d1)
    return o


def stacked_heff(d, H, pairs, X):
    """Evaluate through the stacked layout; returns (Y, max float2 index
    written per leg, plane sizes in float2)."""
    d0, d1, d2 = d
    legs = {}
    for u in range(3):
        Pn, nb = ((d1 * d2, 1), (d0, d2), (d0 * d1, 1))[u]
        legs[u] = dict(d=d[u], Pn=Pn, nb=nb, Pp=rup(Pn, BM), Kc=d[u])
    for p in pairs:
        p["base"] = legs[p["a"]]["Kc"]
        legs[p["a"]]["Kc"] += d[p["a"]] * p["r"]
    for u in range(3):
        L = legs[u]
        L["Kp"] = rup(2 * L["Kc"], BK)
        L["rows"] = L["Pp"] * L["nb"]
        L["P"] = np.zeros((L["rows"], L["Kp"] // 2), dtype=np.complex128)
        L["maxw"] = -1
    Pp1 = legs[1]["Pp"]
    # slot 0: X
    for a_, b_, c_ in itertools.product(range(d0), range(d1), range(d2)):
        x = X[a_, b_, c_]
        legs[0]["P"][b_ + d1 * c_, a_] = x
        legs[1]["P"][a_ + Pp1 * c_, b_] = x
        legs[2]["P"][a_ + d0 * b_, c_] = x
    # channel slots, through the epilogue map
    for p in pairs:
        a, b, r = p["a"], p["b"], p["r"]
        La = legs[a]
        K2a = La["Kp"] // 2
        Z = np.stack([apply_leg(G, X, b) for G in p["G"]])     # (i, a, b, c)
        zo = z_orientation(a, b, d)
        Bi = zo["Bi"] if zo["Bi"] is not None else r
        Bo = zo["Bo"] if zo["Bo"] is not None else r
        o = out_strides(a, b, d, K2a, Pp1)
        assert o["sp1"] == 1          # consecutive P rows: consecutive positions
        flat = La["P"].reshape(-1)
        for pp, q, bi, bo in itertools.product(range(zo["Pn"]), range(d[b]), range(Bi), range(Bo)):
            pos = ((pp % o["pd"]) * o["sp1"] + (pp // o["pd"]) * o["sp2"] + q * o["sq"]
                   + bi * o["sbi"] + bo * o["sbo"] + p["base"])
            assert 0 <= pos < flat.size
            La["maxw"] = max(La["maxw"], pos)
            flat[pos] = Z[zo["idx"](pp, q, bi, bo)]
    # merged contraction per leg
    Y = np.zeros(d, dtype=np.complex128)
    for u in range(3):
        L = legs[u]
        Q = np.zeros((d[u], L["Kp"] // 2), dtype=np.complex128)
        Q[:, :d[u]] = H[u]
        for p in pairs:
            if p["a"] == u:
                for i, Nm in enumerate(p["N"]):
                    Q[:, p["base"] + d[u] * i: p["base"] + d[u] * (i + 1)] = Nm
        C = L["P"] @ Q.T      # (rows, d_u): C(p, q) = sum_k P(p, k) Q(q, k)
        for pp, q, bi in itertools.product(range(L["Pn"]), range(d[u]), range(L["nb"])):
            v = C[pp + L["Pp"] * bi, q]
            if u == 0:
                Y[q, pp % d1, pp // d1] += v
            elif u == 1:
                Y[pp, q, bi] += v
            else:
                Y[pp % d0, pp // d0, q] += v
    return Y, legs


@pytest.mark.parametrize("d", [(5, 4, 3), (3, 6, 5), (7, 2, 4)])
@pytest.mark.parametrize("pair_set", [[(0, 1), (0, 2), (1, 2)], [(1, 0), (2, 0), (2, 1)],
                                      [(0, 1), (2, 0)], [(1, 2)]])
def test_stacked_heff_equals_direct_sum(d, pair_set):
    rng = np.random.default_rng(sum(d) + len(pair_set))

    def cm(n, m):
        return rng.normal(size=(n, m)) + 1j * rng.normal(size=(n, m))
    X = rng.normal(size=d) + 1j * rng.normal(size=d)
    H = [cm(d[u], d[u]) for u in range(3)]
    pairs = []
    for (a, b) in pair_set:
        r = 2 + (a + 2 * b) % 3
        pairs.append(dict(a=a, b=b, r=r, N=[cm(d[a], d[a]) for _ in range(r)],
                          G=[cm(d[b], d[b]) for _ in range(r)]))
    Y, legs = stacked_heff(d, H, pairs, X)
    ref = sum(apply_leg(H[u], X, u) for u in range(3))
    for p in pairs:
        for Nm, G in zip(p["N"], p["G"]):
            ref = ref + apply_leg(Nm, apply_leg(G, X, p["b"]), p["a"])
    assert np.allclose(Y, ref, rtol=1e-12, atol=1e-12)
    for u in range(3):
        L = legs[u]
        assert L["maxw"] < L["rows"] * L["Kp"] // 2


# ---------------------------------------------------------------------------
# Split renormalisation of an operator stack (environment update):
# E_i = X^H (op_i x_u X) over the legs other than o.  The first contraction
# takes X with rows w + dw*o (w the third leg) and K = leg u, and writes Z_i
# into the projection's P planes at float2 position
#     (p % dw) + (p / dw)*K2 + q*dw + i*dO*K2      (p = w + dw*o', q = new u)
# i.e. row o' + dO*i, K = w + dw*u'.  The projection's Q side is X^H with rows
# o and K = w + dw*u; its output row p = k' + dO*i goes to E_i(k, k').
@pytest.mark.parametrize("d", [(5, 4, 3), (3, 6, 5)])
@pytest.mark.parametrize("u,o", [(0, 1), (0, 2), (1, 0), (1, 2), (2, 0), (2, 1)])
def test_split_renormalisation_layout(d, u, o):
    rng = np.random.default_rng(7 + 3 * u + o)
    X = rng.normal(size=d) + 1j * rng.normal(size=d)
    w = 3 - u - o
    du, dO, dw = d[u], d[o], d[w]
    nop = 3
    ops = rng.normal(size=(nop, du, du)) + 1j * rng.normal(size=(nop, du, du))
    Kproj = X.size // dO
    K2 = rup(2 * Kproj, BK) // 2
    Pp = rup(dO * nop, BM)
    P = np.zeros((Pp, K2), dtype=np.complex128)
    flat = P.reshape(-1)
    for i in range(nop):
        Z = apply_leg(ops[i], X, u)
        for pp in range(dw * dO):
            wi, oi = pp % dw, pp // dw
            for q in range(du):
                idx = [0, 0, 0]
                idx[w], idx[o], idx[u] = wi, oi, q
                pos = (pp % dw) + (pp // dw) * K2 + q * dw + i * dO * K2
                assert 0 <= pos < flat.size
                flat[pos] = Z[tuple(idx)]
    Q = np.zeros((dO, K2), dtype=np.complex128)
    for k in range(dO):
        for wi in range(dw):
            for ui in range(du):
                idx = [0, 0, 0]
                idx[o], idx[w], idx[u] = k, wi, ui
                Q[k, wi + dw * ui] = np.conj(X[tuple(idx)])
    C = P @ Q.T
    E = np.zeros((nop, dO, dO), dtype=np.complex128)
    for pp in range(dO * nop):
        for k in range(dO):
            E[pp // dO, k, pp % dO] = C[pp, k]
    others = [l for l in range(3) if l != o]
    for i in range(nop):
        ref = np.tensordot(X.conj(), apply_leg(ops[i], X, u), axes=(others, others))
        assert np.allclose(E[i], ref, rtol=1e-12, atol=1e-12)
