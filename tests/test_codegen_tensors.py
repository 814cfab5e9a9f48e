"""The code generator's reference tensors against the oracle, on the CPU.

The CUDA local kernels are generated from exact rational reference tensors (codegen.py): the
stiffness tensor B[(m, n)], the mass tensor M, the kappa tensor C[(k, m, n)] and the source tensor
Mx.  Contracted with the geometry of a cell here in numpy, they must give the oracle's element
matrices and vectors (its own basis, quadrature and geometry) to rounding:

    K = sum_{m<=n} Lam_mn B[(m, n)] + |T| M,  Lam_mn = |T| grad(lambda_m) . grad(lambda_n)
    K_kappa = sum_k kappa_k sum_{m<=n} Lam_mn C[(k, m, n)],   b = |T| Mx f

so a wrong entry in a generated table fails here before any GPU run.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1501_01809_gb300 import codegen as cg


def _cell(dim, rng):
    """A random non-degenerate simplex near the reference one."""
    ref = np.vstack([np.zeros(dim), np.eye(dim)])
    return ref + rng.uniform(-0.2, 0.2, ref.shape)


def _geometry(xv):
    dim = xv.shape[1]
    J = (xv[1:] - xv[0]).T
    vol = abs(np.linalg.det(J)) / math.factorial(dim)
    Ji = np.linalg.inv(J)
    grads = np.vstack([-Ji.sum(axis=0), Ji])  # grad lambda_m, m = 0..dim
    pairs = [(m, n) for m in range(dim + 1) for n in range(m, dim + 1)]
    lam = {(m, n): vol * grads[m] @ grads[n] for m, n in pairs}
    return vol, lam


def _f(T):
    return np.array([[float(v) for v in row] for row in T])


ELEMENTS = [(2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2), (3, 3)]


@pytest.mark.parametrize("dim,p", ELEMENTS)
def test_stiffness_and_mass_tensors(dim, p):
    rng = np.random.default_rng(10 * dim + p)
    B = {k: _f(v) for k, v in cg.stiffness_tensor(dim, p).items()}
    M = _f(cg.mass_tensor(dim, p))
    for _ in range(3):
        xv = _cell(dim, rng)
        vol, lam = _geometry(xv)
        S = sum(lam[k] * B[k] for k in B)
        for form, K in ((O.MASS, vol * M), (O.LAPLACE, S), (O.HELMHOLTZ, S + vol * M)):
            want = O.element_matrix(dim, p, form, xv)
            np.testing.assert_allclose(K, want, rtol=0, atol=1e-12 * np.abs(want).max(), err_msg=f"form {form}")


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 2), (2, 4), (3, 1), (3, 2)])
def test_kappa_tensor(dim, p):
    rng = np.random.default_rng(100 + 10 * dim + p)
    C = {k: _f(v) for k, v in cg.kappa_tensor(dim, p).items()}
    for _ in range(3):
        xv = _cell(dim, rng)
        kv = np.exp(rng.standard_normal(dim + 1))
        _, lam = _geometry(xv)
        K = sum(kv[k] * lam[(m, n)] * T for (k, m, n), T in C.items())
        want = O.element_matrix(dim, p, O.KAPPA_DIFFUSION, xv, kv)
        np.testing.assert_allclose(K, want, rtol=0, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("dim,p,q", [(2, 1, 1), (2, 2, 2), (2, 2, 1), (2, 4, 1), (3, 1, 1), (3, 2, 2), (3, 2, 1)])
def test_source_tensor(dim, p, q):
    rng = np.random.default_rng(200 + 10 * dim + p + q)
    Mx = _f(cg.mass_tensor(dim, p, q))
    for _ in range(3):
        xv = _cell(dim, rng)
        vol, _ = _geometry(xv)
        fe = rng.uniform(-1, 1, Mx.shape[1])
        want = O.element_vector(dim, p, q, xv, fe)
        np.testing.assert_allclose(vol * Mx @ fe, want, rtol=0, atol=1e-12 * np.abs(want).max())


def _generated_array(name):
    """A float table as emitted into the generated header (the bytes the tensor-core kernel loads)."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(cg.__file__), "csrc", "generated", "fe_local.cuh")).read()
    m = re.search(name + r"\[(\d+)\]\[(\d+)\] = \{(.*?)\};", src, re.S)
    assert m, name
    rows, cols = int(m.group(1)), int(m.group(2))
    vals = [float(v.rstrip("f")) for v in re.findall(r"-?[0-9.]+(?:e-?[0-9]+)?f", m.group(3))]
    assert len(vals) == rows * cols
    return np.array(vals).reshape(rows, cols)


def test_tensor_core_kappa_table_layout():
    """The P4 kappa-diffusion table of the tensor-core kernel: row n is the upper-triangle pair
    (i <= j, row by row), column k = kappa node * 6 + Lam pair (m <= n).  Its FP32 entries,
    contracted with kappa_k Lam_mn in FP64, give the oracle's element matrix to the table's own
    rounding (relative Frobenius below 1e-6, well inside the 1e-5 bound of the tensor-core path)."""
    Ctab = _generated_array("kKappaTC24_C")
    nd = 15
    iu, ju = np.triu_indices(nd)
    assert Ctab.shape == (len(iu), 3 * 6)
    rng = np.random.default_rng(7)
    for _ in range(4):
        xv = _cell(2, rng)
        kv = np.exp(rng.standard_normal(3))
        _, lam = _geometry(xv)
        pairs = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]
        a = np.array([kv[k] * lam[mn] for k in range(3) for mn in pairs])
        K = np.zeros((nd, nd))
        K[iu, ju] = Ctab @ a
        K[ju, iu] = K[iu, ju]
        want = O.element_matrix(2, 4, O.KAPPA_DIFFUSION, xv, kv)
        assert np.linalg.norm(K - want) <= 1e-6 * np.linalg.norm(want)


@pytest.mark.parametrize("dim,p", ELEMENTS)
def test_rewritten_stiffness_is_exact(dim, p):
    """The generator's common-subexpression rewriting of the stiffness entries (pairs of Lam terms
    extracted into temporaries) gives exactly the original linear forms: evaluated in rational
    arithmetic at random rational Lam it equals sum_k B_k Lam_k for every entry, and it uses no
    more multiply-adds than the direct chains."""
    from fractions import Fraction as F
    forms = cg.stiffness_forms(dim, p)
    temps, reduced = cg.cse_plan(forms)
    rng = np.random.default_rng(7 * dim + p)
    nlam = len(cg._lam_pairs(dim))
    for _ in range(3):
        lam = [F(int(rng.integers(-50, 51)), int(rng.integers(1, 17))) for _ in range(nlam)]
        got = cg.eval_plan(temps, reduced, lam)
        want = [sum((c * lam[k] for k, c in f.items()), F(0)) for f in forms]
        assert got == want
    assert len(temps) + sum(len(t) for t in reduced) <= sum(len(f) for f in forms)
    # regrouping only: with every coefficient and ratio replaced by its absolute value, the plan
    # gives sum_k |B_k| Lam_k at positive Lam, so no rounding error larger than the original
    # terms' can arise (the parity tolerance scales with those terms)
    absp = [(a, b, abs(r)) for a, b, r in temps], [[(v, abs(c)) for v, c in t] for t in reduced]
    lam = [F(int(rng.integers(1, 51)), int(rng.integers(1, 17))) for _ in range(nlam)]
    assert cg.eval_plan(*absp, lam) == [sum((abs(c) * lam[k] for k, c in f.items()), F(0)) for f in forms]
