"""Local-kernel generator: forms x Lagrange element -> straight-line CUDA element-tensor code.

This plays the role of the paper's form compiler (Sec. 5.2 "A modified FFC" emits the local
assembly kernel; Sec. 4.5 COFFEE hoists loop invariants).  For an affine simplex every factor
of the quadrature loop except the geometry is cell-independent, so the generator runs that loop
once on the reference cell and emits only the per-cell contraction:

* Barycentric form of the stiffness: with grad phi_i = sum_m (d phi_i / d lambda_m) grad lambda_m,
      K_ij = sum_{m<=n} Lam_mn * B[mn][i][j],   Lam_mn = |T| grad lambda_m . grad lambda_n,
  where B = (1/|T|) int (d phi_i/d lambda_m)(d phi_j/d lambda_n) (+ the transposed term for m != n)
  is a rational constant.  Most B entries vanish, so this needs far fewer multiply-adds than the
  dense reference-coordinate form.
* Mass: K_ij += |T| * M[i][j],  M = (1/|T|) int phi_i phi_j.
* Linear form f v dx with f in P_q: b_i = |T| sum_k Mx[i][k] f_k.
* kappa-diffusion with kappa in P1: K_ij = sum_k sum_{m<=n} (kappa_k Lam_mn) C[k][mn][i][j].

Reference integrals are exact rationals from  int_T lambda^alpha = |T| d! alpha! / (|alpha|+d)!.
As a self-check the generator re-evaluates every tensor with the named quadrature rule of the
workload (3-point degree-2 triangle rule, the 14-point degree-5 tetrahedron rule, a degree-8
triangle rule) and refuses to emit code if they disagree.

The emitted code is templated on an arithmetic policy ``Ops`` (native FP64 or FP32-pair), so the
same term lists serve every precision.  Run as ``python -m paper_1501_01809_gb300.codegen OUT``.
"""
from __future__ import annotations

import sys
from fractions import Fraction as F
from functools import lru_cache
from itertools import combinations
from math import factorial

import numpy as np

ELEMENTS = [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)]
SOURCE_PAIRS = [(2, 1, 1), (2, 2, 2), (2, 2, 1), (2, 4, 1), (3, 1, 1), (3, 2, 2), (3, 2, 1)]
KAPPA_ELEMENTS = [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)]


# ------------------------------------------------------------------ element definition

def lattice_nodes(dim: int, p: int):
    """Multi-indices of the P_p nodes in the library's canonical local order (see include/fe.h)."""
    nv = dim + 1
    out = []
    for m in range(nv):
        a = [0] * nv
        a[m] = p
        out.append(tuple(a))
    for a_, b_ in combinations(range(nv), 2):
        for t in range(1, p):
            a = [0] * nv
            a[a_], a[b_] = p - t, t
            out.append(tuple(a))
    for fa in combinations(range(nv), 3):
        for x in range(p - 2, 0, -1):
            for y in range(p - 1 - x, 0, -1):
                z = p - x - y
                if z >= 1:
                    a = [0] * nv
                    a[fa[0]], a[fa[1]], a[fa[2]] = x, y, z
                    out.append(tuple(a))
    if dim == 3:
        for a0 in range(p - 3, 0, -1):
            for a1 in range(p - 2 - a0, 0, -1):
                for a2 in range(p - 1 - a0 - a1, 0, -1):
                    if p - a0 - a1 - a2 >= 1:
                        out.append((a0, a1, a2, p - a0 - a1 - a2))
    return out


# polynomials in the d+1 barycentric variables: dict exponent-tuple -> Fraction

def _pmul(a, b):
    out = {}
    for ea, ca in a.items():
        for eb, cb in b.items():
            e = tuple(x + y for x, y in zip(ea, eb))
            out[e] = out.get(e, 0) + ca * cb
    return {e: c for e, c in out.items() if c != 0}


def _pdiff(a, m):
    out = {}
    for e, c in a.items():
        if e[m]:
            e2 = list(e)
            e2[m] -= 1
            out[tuple(e2)] = out.get(tuple(e2), 0) + c * e[m]
    return out


def _var_poly(nv, m, scale, shift):
    """scale * lambda_m + shift"""
    z = tuple([0] * nv)
    e = [0] * nv
    e[m] = 1
    out = {tuple(e): F(scale)}
    if shift:
        out[z] = F(shift)
    return out


@lru_cache(maxsize=None)
def basis(dim: int, p: int):
    """phi_alpha = prod_m prod_{s<alpha_m} (p lambda_m - s)/(s+1)  (polynomials in lambda)."""
    nv = dim + 1
    out = []
    for alpha in lattice_nodes(dim, p):
        poly = {tuple([0] * nv): F(1)}
        for m in range(nv):
            for s in range(alpha[m]):
                poly = _pmul(poly, _var_poly(nv, m, F(p, s + 1), F(-s, s + 1)))
        out.append(poly)
    return out


def _bary_integral(poly, dim):
    """(1/|T|) int_T poly(lambda) = sum c * d! alpha! / (|alpha| + d)!"""
    s = F(0)
    for e, c in poly.items():
        num = factorial(dim)
        for a in e:
            num *= factorial(a)
        s += c * F(num, factorial(sum(e) + dim))
    return s


def _lam_pairs(dim):
    return [(m, n) for m in range(dim + 1) for n in range(m, dim + 1)]


@lru_cache(maxsize=None)
def stiffness_tensor(dim: int, p: int):
    """B[(m,n)][i][j] for m <= n (m != n folds both orders)."""
    phis = basis(dim, p)
    nd = len(phis)
    dphi = [[_pdiff(ph, m) for m in range(dim + 1)] for ph in phis]
    B = {}
    for (m, n) in _lam_pairs(dim):
        T = [[F(0)] * nd for _ in range(nd)]
        for i in range(nd):
            for j in range(nd):
                v = _bary_integral(_pmul(dphi[i][m], dphi[j][n]), dim)
                if m != n:
                    v += _bary_integral(_pmul(dphi[i][n], dphi[j][m]), dim)
                T[i][j] = v
        B[(m, n)] = T
    return B


@lru_cache(maxsize=None)
def mass_tensor(dim: int, p: int, q: int | None = None):
    """M[i][k] = (1/|T|) int phi_i psi_k with phi in P_p, psi in P_q (q = p: the mass matrix)."""
    a, b = basis(dim, p), basis(dim, q or p)
    return [[_bary_integral(_pmul(x, y), dim) for y in b] for x in a]


@lru_cache(maxsize=None)
def kappa_tensor(dim: int, p: int):
    """C[k][(m,n)][i][j] = (1/|T|) int lambda_k (dphi_i/dl_m dphi_j/dl_n [+ (m<->n)])."""
    phis = basis(dim, p)
    nd = len(phis)
    nv = dim + 1
    dphi = [[_pdiff(ph, m) for m in range(nv)] for ph in phis]
    C = {}
    for k in range(nv):
        lk = _var_poly(nv, k, 1, 0)
        for (m, n) in _lam_pairs(dim):
            T = [[F(0)] * nd for _ in range(nd)]
            for i in range(nd):
                for j in range(nd):
                    v = _bary_integral(_pmul(lk, _pmul(dphi[i][m], dphi[j][n])), dim)
                    if m != n:
                        v += _bary_integral(_pmul(lk, _pmul(dphi[i][n], dphi[j][m])), dim)
                    T[i][j] = v
            C[(k, m, n)] = T
    return C


# ------------------------------------------------------------------ named quadrature rules (self-check)

def _tri_rule_deg2():
    """3 interior points (1/6,1/6),(2/3,1/6),(1/6,2/3), weights |T|/3 (exact for degree 2)."""
    pts = [(2 / 3, 1 / 6, 1 / 6), (1 / 6, 2 / 3, 1 / 6), (1 / 6, 1 / 6, 2 / 3)]
    return np.array(pts), np.full(3, 1 / 3)


def _tet_rule_14():
    """Fully symmetric 14-point degree-5 rule on the tetrahedron (orbits 4 + 4 + 6).

    Unknowns a, b (points (a,a,a,1-3a), (b,b,b,1-3b)), c (points (c,c,1/2-c,1/2-c)) and the three
    orbit weights; solved by Newton's method from the moment equations of the symmetric
    polynomials up to degree 5, then checked on every monomial of degree <= 5.
    """
    def points(x):
        a, b, c = x[0], x[1], x[2]
        o1 = [tuple(a if k != m else 1 - 3 * a for k in range(4)) for m in range(4)]
        o2 = [tuple(b if k != m else 1 - 3 * b for k in range(4)) for m in range(4)]
        o3 = []
        for (m, n) in combinations(range(4), 2):
            o3.append(tuple(c if k in (m, n) else 0.5 - c for k in range(4)))
        return o1, o2, o3

    # barycentric moment targets (1/|T|) int lambda^alpha for a basis of symmetric test monomials
    tests = [(0, 0, 0, 0), (2, 0, 0, 0), (3, 0, 0, 0), (1, 1, 1, 0), (4, 0, 0, 0), (2, 2, 0, 0),
             (5, 0, 0, 0), (2, 2, 1, 0), (3, 1, 1, 0)]

    def exact(al):
        num = 6
        for a in al:
            num *= factorial(a)
        return num / factorial(sum(al) + 3)

    def sym_moment(pts, al):
        from itertools import permutations
        perms = set(permutations(al))
        return sum(np.mean([np.prod([pt[k] ** e[k] for k in range(4)]) for e in perms]) for pt in pts)

    def residual(x):
        o1, o2, o3 = points(x)
        w1, w2, w3 = x[3], x[4], x[5]
        r = []
        for al in tests:
            r.append(w1 * sym_moment(o1, al) + w2 * sym_moment(o2, al) + w3 * sym_moment(o3, al) - exact(al))
        return np.array(r)

    x = np.array([0.0927, 0.3109, 0.0455, 0.073, 0.113, 0.043])   # rough start from the known shape
    for _ in range(60):
        r = residual(x)
        Jm = np.empty((len(r), 6))
        for k in range(6):
            dx = np.zeros(6)
            dx[k] = 1e-7
            Jm[:, k] = (residual(x + dx) - residual(x - dx)) / 2e-7
        step = np.linalg.lstsq(Jm, -r, rcond=None)[0]
        x = x + step
        if np.max(np.abs(step)) < 1e-15:
            break
    o1, o2, o3 = points(x)
    pts = np.array(o1 + o2 + o3)
    wts = np.array([x[3]] * 4 + [x[4]] * 4 + [x[5]] * 6)
    assert abs(wts.sum() - 1) < 1e-13 and np.all(wts > 0) and np.all(pts >= 0)
    return pts, wts


def _tri_rule_collapsed(m):
    """m x m collapsed Gauss-Legendre triangle rule (exact to degree 2m-2); m = 5 gives degree 8."""
    g, w = np.polynomial.legendre.leggauss(m)
    g, w = (g + 1) / 2, w / 2
    pts, wts = [], []
    for a in range(m):
        for b in range(m):
            x, y = g[a], g[b] * (1 - g[a])
            pts.append((1 - x - y, x, y))
            wts.append(2 * w[a] * w[b] * (1 - g[a]))
    return np.array(pts), np.array(wts)


def _tet_rule_collapsed(m):
    g, w = np.polynomial.legendre.leggauss(m)
    g, w = (g + 1) / 2, w / 2
    pts, wts = [], []
    for a in range(m):
        for b in range(m):
            for c in range(m):
                x, y, z = g[a], g[b] * (1 - g[a]), g[c] * (1 - g[a]) * (1 - g[b])
                pts.append((1 - x - y - z, x, y, z))
                wts.append(6 * w[a] * w[b] * w[c] * (1 - g[a]) ** 2 * (1 - g[b]))
    return np.array(pts), np.array(wts)


def quadrature_rule(dim: int, degree: int):
    """Named rule for the workloads (weights normalised to sum 1 over the cell)."""
    if dim == 2 and degree <= 2:
        return _tri_rule_deg2()
    if dim == 3 and degree <= 5:
        return _tet_rule_14()
    if dim == 2:
        return _tri_rule_collapsed(max(2, (degree + 3) // 2))
    return _tet_rule_collapsed(max(2, (degree + 4) // 2))


def _peval(poly, lam):
    s = 0.0
    for e, c in poly.items():
        t = float(c)
        for k, a in enumerate(e):
            if a:
                t *= lam[k] ** a
        s += t
    return s


def check_with_quadrature(dim, p):
    """Re-evaluate B and M with the named rule (degree 2p) and compare with the exact rationals."""
    pts, wts = quadrature_rule(dim, 2 * p)
    phis = basis(dim, p)
    nd = len(phis)
    dphi = [[_pdiff(ph, m) for m in range(dim + 1)] for ph in phis]
    B, M = stiffness_tensor(dim, p), mass_tensor(dim, p)
    for (m, n), T in B.items():
        for i in range(nd):
            for j in range(nd):
                v = sum(w * _peval(dphi[i][m], l) * _peval(dphi[j][n], l) for l, w in zip(pts, wts))
                if m != n:
                    v += sum(w * _peval(dphi[i][n], l) * _peval(dphi[j][m], l) for l, w in zip(pts, wts))
                assert abs(v - float(T[i][j])) < 1e-12, (dim, p, m, n, i, j, v, T[i][j])
    for i in range(nd):
        for j in range(nd):
            v = sum(w * _peval(phis[i], l) * _peval(phis[j], l) for l, w in zip(pts, wts))
            assert abs(v - float(M[i][j])) < 1e-12


# ------------------------------------------------------------------ emission

def _num(c: F) -> str:
    v = float(c)
    return repr(v) if v != int(v) else f"{int(v)}.0"


def _term_chain(terms, var):
    """Straight-line multiply-add chain for sum_k c_k var[k] (c = +-1 folded to moves/negations)."""
    k0, c0 = terms[0]
    if c0 == 1:
        expr = f"{var}[{k0}]"
    elif c0 == -1:
        expr = f"Ops::neg({var}[{k0}])"
    else:
        expr = f"Ops::mulc({var}[{k0}], {_num(c0)})"
    for k, c in terms[1:]:
        expr = f"Ops::fmac({var}[{k}], {_num(c)}, {expr})"
    return expr


def _upper(nd):
    return [(i, j) for i in range(nd) for j in range(i, nd)]


# ------------------------------------------------------------------ common subexpressions
# The stiffness entries are linear forms in the Lam_mn with rational coefficients, and many share
# a pair of terms in the same ratio (K_ij = c (Lam_a + r Lam_b) + ...).  In the spirit of COFFEE's
# expression rewriting (Sec. 4.5: fewer floating-point operations), the generator extracts such
# pairs greedily, most frequent first: w = Lam_a + r Lam_b costs one multiply-add and saves one in
# every entry that uses it.  The rewriting is exact in rational arithmetic (eval_plan checks it);
# in floating point it reorders the sums of the same terms, with no coefficient larger than the
# original ones.

def cse_plan(forms):
    """forms: list of dicts {var: Fraction} (var = int index of Lam).  Returns (temps, reduced):
    temps[n] = (a, b, r) defines w_n = a + r b (a, b an int Lam index or ('w', k), k < n);
    reduced[u] = list of (var, coefficient) over Lam indices and temps, in a fixed order."""
    fs = [dict(f) for f in forms]
    temps = []

    def key(v):
        return (0, v) if isinstance(v, int) else (1, v[1])

    while True:
        cnt = {}
        for f in fs:
            ks = sorted(f, key=key)
            for ia in range(len(ks)):
                for ib in range(ia + 1, len(ks)):
                    a, b = ks[ia], ks[ib]
                    t = (a, b, f[b] / f[a])
                    cnt[t] = cnt.get(t, 0) + 1
        if not cnt:
            break
        best = max(cnt.items(), key=lambda kv: (kv[1], [-x for x in key(kv[0][0])], [-x for x in key(kv[0][1])]))
        (a, b, r), n = best
        if n < 2:
            break
        w = ("w", len(temps))
        temps.append((a, b, r))
        for f in fs:
            if a in f and b in f and f[b] / f[a] == r:
                f[w] = f.pop(a)
                f.pop(b)
    return temps, [sorted(f.items(), key=lambda kv: key(kv[0])) for f in fs]


def eval_plan(temps, reduced, lam):
    """The plan evaluated in exact arithmetic for values lam[k] (a test of the rewriting)."""
    w = []
    val = lambda v: lam[v] if isinstance(v, int) else w[v[1]]
    for a, b, r in temps:
        w.append(val(a) + r * val(b))
    return [sum((c * val(v) for v, c in terms), F(0)) for terms in reduced]


def _var(v, arr="Lam"):
    return f"{arr}[{v}]" if isinstance(v, int) else f"w{v[1]}"


def _chain(terms, addend=None, arr="Lam"):
    """Multiply-add chain for sum_k c_k v_k (+ addend): c = +-1 folded into moves and negations
    when there is no addend; with an addend every term is one multiply-add."""
    if addend is not None:
        expr = addend
        for v, c in terms:
            expr = f"Ops::fmac({_var(v, arr)}, {_num(c)}, {expr})"
        return expr
    (v0, c0), rest = terms[0], terms[1:]
    if c0 == 1:
        expr = _var(v0, arr)
    elif c0 == -1:
        expr = f"Ops::neg({_var(v0, arr)})"
    else:
        expr = f"Ops::mulc({_var(v0, arr)}, {_num(c0)})"
    for v, c in rest:
        expr = f"Ops::fmac({_var(v, arr)}, {_num(c)}, {expr})"
    return expr


def _emit_temps(temps, indent="    "):
    out = []
    for n, (a, b, r) in enumerate(temps):
        rhs = f"Ops::add({_var(a)}, {_var(b)})" if r == 1 else f"Ops::fmac({_var(b)}, {_num(r)}, {_var(a)})"
        out.append(f"{indent}const typename Ops::T w{n} = {rhs};")
    return out


def stiffness_forms(dim: int, p: int):
    """Each upper-triangle stiffness entry as {Lam index: coefficient}."""
    B = stiffness_tensor(dim, p)
    pairs = _lam_pairs(dim)
    nd = len(B[pairs[0]])
    return [{k: B[mn][i][j] for k, mn in enumerate(pairs) if B[mn][i][j] != 0} for (i, j) in _upper(nd)]


def mass_values(dim: int, p: int):
    """The distinct nonzero entries of the upper-triangle mass tensor, in first-use order."""
    M = mass_tensor(dim, p)
    vals = []
    for (i, j) in _upper(len(M)):
        if M[i][j] != 0 and M[i][j] not in vals:
            vals.append(M[i][j])
    return vals


def emit_element(dim: int, p: int) -> str:
    B = stiffness_tensor(dim, p)
    M = mass_tensor(dim, p)
    pairs = _lam_pairs(dim)
    nd = len(M)
    up = _upper(nd)
    name = f"d{dim}p{p}"
    lines = [f"// ---- P{p} Lagrange on the {'triangle' if dim == 2 else 'tetrahedron'} ({nd} nodes) ----",
             f"template <> struct Elem<{dim}, {p}> {{",
             f"  static constexpr int ND = {nd};",
             f"  static constexpr int NUP = {len(up)};",
             f"  static constexpr int NLAM = {len(pairs)};"]
    # number of stiffness terms
    nterms = sum(1 for (i, j) in up for mn in pairs if B[mn][i][j] != 0)
    lines.append(f"  static constexpr int STIFF_TERMS = {nterms};")
    # upper-triangle index tables (host+device constexpr helper via switch-free arrays are avoided)
    lines.append("  // K[u] for u over the upper triangle (i <= j), row-major; Lam[k] over pairs (m <= n)")
    temps, reduced = cse_plan(stiffness_forms(dim, p))
    mvals = mass_values(dim, p)
    lines.append(f"  static constexpr int STIFF_OPS = {len(temps) + sum(len(t) for t in reduced)};  // after rewriting")
    # stiffness
    lines.append("  template <class Ops> __device__ __forceinline__ static void stiffness_upper("
                 "const typename Ops::T* Lam, typename Ops::T* K) {")
    lines += _emit_temps(temps)
    for u, terms in enumerate(reduced):
        lines.append(f"    K[{u}] = {_chain(terms) if terms else 'Ops::zero()'};")
    lines.append("  }")
    # Helmholtz: the distinct mass products |T| M first, each entry's chain starting from its own
    lines.append("  template <class Ops> __device__ __forceinline__ static void helmholtz_upper("
                 "const typename Ops::T* Lam, const typename Ops::T& vol, typename Ops::T* K) {")
    lines += _emit_temps(temps)
    for q, c in enumerate(mvals):
        lines.append(f"    const typename Ops::T m{q} = Ops::mulc(vol, {_num(c)});")
    for u, ((i, j), terms) in enumerate(zip(up, reduced)):
        mq = f"m{mvals.index(M[i][j])}" if M[i][j] != 0 else None
        if terms:
            lines.append(f"    K[{u}] = {_chain(terms, mq)};")
        else:
            lines.append(f"    K[{u}] = {mq or 'Ops::zero()'};")
    lines.append("  }")
    lines.append("  template <class Ops> __device__ __forceinline__ static void mass_upper("
                 "const typename Ops::T& vol, typename Ops::T* K) {")
    for q, c in enumerate(mvals):
        lines.append(f"    const typename Ops::T m{q} = Ops::mulc(vol, {_num(c)});")
    for u, (i, j) in enumerate(up):
        lines.append(f"    K[{u}] = {'m' + str(mvals.index(M[i][j])) if M[i][j] != 0 else 'Ops::zero()'};")
    lines.append("  }")
    # fused action: each K_ij is formed and consumed at once (y_i += K_ij x_j, y_j += K_ij x_i), so the
    # element matrix is never live as a whole; y is written, not incremented (the first contribution
    # to each y_i is a product)
    lines.append("  template <class Ops, bool STIFF, bool MASS> __device__ __forceinline__ static void action_upper("
                 "const typename Ops::T* Lam, const typename Ops::T& vol, const typename Ops::T* x, typename Ops::T* y) {")
    lines.append("    typename Ops::T k;")
    for cond, st, ms in [("STIFF && MASS", True, True), ("STIFF", True, False), ("MASS", False, True)]:
        lines.append(f"    {'if' if st and ms else 'else if'} constexpr ({cond}) {{")
        if st:
            lines += _emit_temps(temps, "      ")
        if ms:
            for q, c in enumerate(mvals):
                lines.append(f"      const typename Ops::T m{q} = Ops::mulc(vol, {_num(c)});")
        touched = set()

        def acc(i, j):
            if i in touched:
                return f"y[{i}] = Ops::fma3(k, x[{j}], y[{i}]);"
            touched.add(i)
            return f"y[{i}] = Ops::mul(k, x[{j}]);"

        for u, ((i, j), terms) in enumerate(zip(up, reduced)):
            m = M[i][j]
            mq = f"m{mvals.index(m)}" if (ms and m != 0) else None
            terms = terms if st else []
            if not terms and not mq:
                continue
            kk = _chain(terms, mq) if terms else mq
            body = f"k = {kk}; " + acc(i, j)
            if i != j:
                body += " " + acc(j, i)
            lines.append(f"      {{ {body} }}")
        for i in range(nd):
            if i not in touched:
                lines.append(f"      y[{i}] = Ops::zero();")
        lines.append("    }")
    lines.append("  }")
    # upper index maps as constexpr functions
    lines.append("  __host__ __device__ static constexpr int upper_index(int i, int j) {")
    lines.append(f"    return i <= j ? i * {nd} - (i * (i - 1)) / 2 + (j - i) : j * {nd} - (j * (j - 1)) / 2 + (i - j);")
    lines.append("  }")
    lines.append("};")
    return "\n".join(lines)


def emit_source(dim: int, p: int, q: int) -> str:
    Mx = mass_tensor(dim, p, q)
    nd, nf = len(Mx), len(Mx[0])
    lines = [f"template <> struct Source<{dim}, {p}, {q}> {{",
             f"  static constexpr int ND = {nd};",
             f"  static constexpr int NF = {nf};",
             "  // b_i = vol * sum_k Mx[i][k] f_k",
             "  template <class Ops> __device__ __forceinline__ static void vec("
             "const typename Ops::T& vol, const typename Ops::T* f, typename Ops::T* b) {"]
    for i in range(nd):
        terms = [(k, Mx[i][k]) for k in range(nf) if Mx[i][k] != 0]
        lines.append(f"    b[{i}] = Ops::mul(vol, {_term_chain(terms, 'f')});")
    lines.append("  }")
    lines.append("};")
    return "\n".join(lines)


def emit_kappa(dim: int, p: int) -> str:
    C = kappa_tensor(dim, p)
    pairs = _lam_pairs(dim)
    nd = len(basis(dim, p))
    up = _upper(nd)
    nv = dim + 1
    lines = [f"template <> struct Kappa<{dim}, {p}> {{",
             f"  static constexpr int NKL = {nv * len(pairs)};",
             "  // K[u] = sum_{k,(m<=n)} KL[k*NLAM + mn] * C[k][mn][i][j], KL = kappa_k * Lam_mn",
             "  template <class Ops> __device__ __forceinline__ static void upper("
             "const typename Ops::T* KL, typename Ops::T* K) {"]
    nterm = 0
    for u, (i, j) in enumerate(up):
        terms = []
        for k in range(nv):
            for t, mn in enumerate(pairs):
                c = C[(k,) + mn][i][j]
                if c != 0:
                    terms.append((k * len(pairs) + t, c))
        nterm += len(terms)
        if not terms:
            lines.append(f"    K[{u}] = Ops::zero();")
            continue
        lines.append(f"    K[{u}] = {_term_chain(terms, 'KL')};")
    lines.append("  }")
    lines.append(f"  static constexpr int TERMS = {nterm};")
    lines.append("};")
    return "\n".join(lines)


def emit_kappa_tc(dim: int, p: int) -> str:
    """Tables of the kappa-diffusion contraction as a dense matrix for the tensor cores:
    K_upper[n] = sum_k KL[k] C[n][k], n over the upper-triangle pairs (I[n], J[n]), k = kappa node x Lam pair."""
    C = kappa_tensor(dim, p)
    pairs = _lam_pairs(dim)
    nd = len(basis(dim, p))
    up = _upper(nd)
    nv = dim + 1
    nk = nv * len(pairs)
    tag = f"{dim}{p}"
    lines = [f"template <> struct KappaTC<{dim}, {p}> {{",
             f"  static constexpr int N = {len(up)}, K = {nk}, ND = {nd};",
             "};",
             "#ifdef FE_GEN_KAPPA_TC_TABLES",
             f"// row n: upper-triangle pair (I[n], J[n]); column k = kappa node * {len(pairs)} + Lam pair"]
    lines.append(f"static __constant__ unsigned char kKappaTC{tag}_I[{len(up)}] = {{" + ", ".join(str(i) for i, _ in up) + "};")
    lines.append(f"static __constant__ unsigned char kKappaTC{tag}_J[{len(up)}] = {{" + ", ".join(str(j) for _, j in up) + "};")
    rows = []
    for (i, j) in up:
        vals = []
        for k in range(nv):
            for mn in pairs:
                c = C[(k,) + mn][i][j]
                vals.append(repr(float(np.float32(float(c)))) + "f" if c != 0 else "0.0f")
        rows.append("{" + ", ".join(vals) + "}")
    lines.append(f"static __device__ const float kKappaTC{tag}_C[{len(up)}][{nk}] = {{" + ",\n    ".join(rows) + "};")
    lines.append("#endif")
    return "\n".join(lines)


HEADER = """// GENERATED by paper_1501_01809_gb300/codegen.py -- do not edit.
// Element-tensor contractions for affine simplices (barycentric form); see codegen.py.
#pragma once
namespace fe_gen {
template <int DIM, int P> struct Elem;
template <int DIM, int P, int Q> struct Source;
template <int DIM, int P> struct Kappa;
template <int DIM, int P> struct KappaTC;
"""


def generate(check: bool = True) -> str:
    parts = [HEADER]
    for dim, p in ELEMENTS:
        if check and (dim, p) in [(2, 1), (2, 2), (3, 1), (3, 2)]:
            check_with_quadrature(dim, p)
        parts.append(emit_element(dim, p))
    for dim, p, q in SOURCE_PAIRS:
        parts.append(emit_source(dim, p, q))
    for dim, p in KAPPA_ELEMENTS:
        parts.append(emit_kappa(dim, p))
    parts.append(emit_kappa_tc(2, 4))
    parts.append("}  // namespace fe_gen\n")
    return "\n\n".join(parts)


def main(argv):
    out = argv[1]
    src = generate()
    try:
        with open(out) as fh:
            if fh.read() == src:
                return 0
    except OSError:
        pass
    with open(out, "w") as fh:
        fh.write(src)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
