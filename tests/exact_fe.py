"""Exact-rational brute-force finite element helper for pinning the oracle (test use only).

Independent of the oracle's code paths: the Lagrange basis is defined here by its nodal
property (phi_i(x_j) = delta_ij, solved from an exact Vandermonde system in monomials of the
reference coordinates), and every integral is exact via the reference-simplex monomial
formula  int xi^a eta^b = a! b! / (a+b+2)!  (and a!b!c!/(a+b+c+3)! in 3D).  No quadrature.
"""
from __future__ import annotations

from fractions import Fraction as F
from functools import lru_cache
from itertools import product
from math import factorial

from paper_1501_01809_gb300 import meshgen as mg


def monomials(dim: int, p: int):
    return [e for e in product(range(p + 1), repeat=dim) if sum(e) <= p]


def ref_monomial_integral(e) -> F:
    num = 1
    for a in e:
        num *= factorial(a)
    return F(num, factorial(sum(e) + len(e)))


def poly_mul(a: dict, b: dict) -> dict:
    out: dict = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return out


def poly_int(a: dict) -> F:
    return sum((c * ref_monomial_integral(e) for e, c in a.items()), F(0))


def poly_diff(a: dict, k: int) -> dict:
    out: dict = {}
    for e, c in a.items():
        if e[k] > 0:
            e2 = list(e)
            e2[k] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[k]
    return out


def _solve(A, B):
    """Exact Gauss-Jordan: returns X with A X = B (A square, lists of Fractions)."""
    n = len(A)
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        inv = 1 / M[c][c]
        M[c] = [v * inv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c]
                M[r] = [vr - f * vc for vr, vc in zip(M[r], M[c])]
    return [row[n:] for row in M]


@lru_cache(maxsize=None)
def nodal_basis(dim: int, p: int):
    """Reference nodal basis as polynomials in xi (dicts exponent -> Fraction), local order of meshgen."""
    alpha = mg.lagrange_nodes(dim, p)
    pts = [tuple(F(int(a[m + 1]), p) for m in range(dim)) for a in alpha]  # xi_m = lambda_{m+1}
    mons = monomials(dim, p)
    V = [[_mono_at(e, x) for e in mons] for x in pts]                        # V[node][mono]
    I = [[F(int(i == j)) for j in range(len(pts))] for i in range(len(pts))]
    C = _solve(V, I)                                                          # V C = I -> columns are phi_j
    return [{e: C[k][j] for k, e in enumerate(mons) if C[k][j] != 0} for j in range(len(pts))]


def _mono_at(e, x):
    v = F(1)
    for a, xi in zip(e, x):
        v *= xi ** a
    return v


@lru_cache(maxsize=None)
def reference_tensors(dim: int, p: int):
    """R[a][b][i][j] = int d_a phi_i d_b phi_j, M[i][j] = int phi_i phi_j, and the gradients."""
    phis = nodal_basis(dim, p)
    nd = len(phis)
    grads = [[poly_diff(phi, a) for a in range(dim)] for phi in phis]
    R = [[[[poly_int(poly_mul(grads[i][a], grads[j][b])) for j in range(nd)] for i in range(nd)]
          for b in range(dim)] for a in range(dim)]
    M = [[poly_int(poly_mul(phis[i], phis[j])) for j in range(nd)] for i in range(nd)]
    return R, M, grads


def _det(J):
    if len(J) == 2:
        return J[0][0] * J[1][1] - J[0][1] * J[1][0]
    return (J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) - J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0])
            + J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]))


def _inv(J):
    n = len(J)
    return _solve(J, [[F(int(i == j)) for j in range(n)] for i in range(n)])


def element_matrix(dim: int, p: int, xv, mass: bool = True, stiff: bool = True, kappa=None):
    """Exact element matrix of (kappa grad u . grad v [+ u v]) on the cell with vertex coords xv."""
    xv = [[F(c) for c in row] for row in xv]
    J = [[xv[c + 1][r] - xv[0][r] for c in range(dim)] for r in range(dim)]
    det = _det(J)
    Ji = _inv(J)
    G = [[sum(Ji[a][x] * Ji[b][x] for x in range(dim)) for b in range(dim)] for a in range(dim)]
    R, M, grads = reference_tensors(dim, p)
    nd = len(M)
    K = [[F(0)] * nd for _ in range(nd)]
    if stiff:
        if kappa is None:
            for i in range(nd):
                for j in range(nd):
                    K[i][j] += abs(det) * sum(G[a][b] * R[a][b][i][j] for a in range(dim) for b in range(dim))
        else:
            kap = {tuple([0] * dim): F(kappa[0])}
            for m in range(dim):
                e = [0] * dim
                e[m] = 1
                kap[tuple(e)] = F(kappa[m + 1]) - F(kappa[0])
            for i in range(nd):
                for j in range(nd):
                    s = F(0)
                    for a in range(dim):
                        for b in range(dim):
                            if G[a][b] != 0:
                                s += G[a][b] * poly_int(poly_mul(kap, poly_mul(grads[i][a], grads[j][b])))
                    K[i][j] += abs(det) * s
    if mass:
        for i in range(nd):
            for j in range(nd):
                K[i][j] += abs(det) * M[i][j]
    return K
