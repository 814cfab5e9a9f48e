/*
 * Plain, slow, obviously-correct FP64 CPU oracle for cell-wise finite element assembly
 * as described in Rathgeber et al., "Firedrake: automating the finite element method by
 * composing abstractions": the par_loop (Sec. 4.4, its algorithm over the iteration set),
 * the INC access descriptor and staging in/out (Sec. 4.4.1), Mats assembled through a
 * pair of maps (Sec. 4.4.3), and the forms of the Poisson listing (Sec. 3.1, Listing 1:
 * a = inner(grad u, grad v) dx, L = f v dx) extended by a mass term (Helmholtz) and a
 * P1 coefficient kappa (diffusion); for solves, strong Dirichlet conditions by symmetric
 * elimination (Sec. 3.1), Jacobi-preconditioned conjugate gradients (Sec. 6.2) and explicit
 * lumped-mass wave steps (Sec. 6.3).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or constant
 * generator with the CUDA path: it has its own Lagrange basis (Silvester's product formula
 * in barycentric coordinates), its own quadrature (collapsed Gauss-Legendre, nodes by
 * Newton iteration on the Legendre three-term recurrence), its own Jacobian inverse and
 * its own sparsity construction (per-row sort + unique).
 *
 * Every element integral is evaluated by quadrature at run time, cell by cell, exactly as
 * the definition reads; no tensor factorisation, blocking or reordering is applied.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXD 3
#define OR_MAXND 35 /* P4 tetrahedron */
#define OR_MAXQ1 16 /* 1-D Gauss points */

enum { OR_MASS = 1, OR_LAPLACE = 2, OR_HELMHOLTZ = 3, OR_KAPPA_DIFFUSION = 4 };

/* ---- deliberate-mistake switch (tests plant a mistake here to show the pins catch it) ---- */
static int g_mutation = 0;
void oracle_set_mutation(int code) { g_mutation = code; }

static long binom(int n, int k) {
    long r = 1;
    for (int i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

int oracle_num_nodes(int dim, int p) {
    if (dim < 1 || dim > OR_MAXD || p < 1) return -1;
    return (int)binom(p + dim, dim);
}

/*
 * Local node order of the P_p Lagrange element (lattice points sum_m alpha_m x_m / p,
 * |alpha| = p): vertices; edges (a<b) lexicographic, walked from a to b; faces (a<b<c)
 * lexicographic, interior points by descending alpha_a then alpha_b; cell interior (3D) by
 * descending alpha_0, alpha_1, alpha_2.  alpha has (dim+1) entries per node.
 */
int oracle_nodes(int dim, int p, int *alpha) {
    int nv = dim + 1, k = 0;
    int nd = oracle_num_nodes(dim, p);
    if (nd < 0) return -1;
    memset(alpha, 0, sizeof(int) * nd * nv);
    for (int m = 0; m < nv; m++) alpha[(k++) * nv + m] = p;
    for (int a = 0; a < nv; a++)
        for (int b = a + 1; b < nv; b++)
            for (int t = 1; t < p; t++) {
                alpha[k * nv + a] = p - t;
                alpha[k * nv + b] = t;
                k++;
            }
    for (int a = 0; a < nv; a++)
        for (int b = a + 1; b < nv; b++)
            for (int c = b + 1; c < nv; c++)
                for (int aa = p - 2; aa >= 1; aa--)
                    for (int bb = p - 1 - aa; bb >= 1; bb--) {
                        int cc = p - aa - bb;
                        if (cc < 1) continue;
                        alpha[k * nv + a] = aa;
                        alpha[k * nv + b] = bb;
                        alpha[k * nv + c] = cc;
                        k++;
                    }
    if (dim == 3)
        for (int a0 = p - 3; a0 >= 1; a0--)
            for (int a1 = p - 2 - a0; a1 >= 1; a1--)
                for (int a2 = p - 1 - a0 - a1; a2 >= 1; a2--) {
                    int a3 = p - a0 - a1 - a2;
                    if (a3 < 1) continue;
                    alpha[k * nv + 0] = a0;
                    alpha[k * nv + 1] = a1;
                    alpha[k * nv + 2] = a2;
                    alpha[k * nv + 3] = a3;
                    k++;
                }
    if (g_mutation == 4 && p >= 2) { /* planted mistake: swap the first two edge nodes */
        for (int m = 0; m < nv; m++) {
            int t = alpha[nv * nv + m];
            alpha[nv * nv + m] = alpha[(nv + p - 1) * nv + m];
            alpha[(nv + p - 1) * nv + m] = t;
        }
    }
    return k == nd ? nd : -1;
}

/* ---- 1-D Gauss-Legendre on [0,1] (Newton iteration on P_m via the three-term recurrence) ---- */
int oracle_gauss_legendre01(int m, double *x, double *w) {
    if (m < 1 || m > OR_MAXQ1) return -1;
    for (int i = 0; i < m; i++) {
        double z = cos(M_PI * (i + 0.75) / (m + 0.5)), dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (m == 1) { p1 = z; p0 = 1.0; }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {   /* recompute P_m' at the converged node for the weight */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= m; k++) {
                double pk = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = pk;
            }
            if (m == 1) { p1 = z; p0 = 1.0; }
            dp = m * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);                 /* map [-1,1] -> [0,1] */
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp); /* = 2/((1-z^2) P'^2) scaled by 1/2 */
    }
    return m;
}

/*
 * Collapsed (Duffy) Gauss-Legendre rule on the reference simplex {xi >= 0, sum xi <= 1}
 * with m points per direction: triangle xi = (u, v(1-u)), weight w_u w_v (1-u);
 * tetrahedron xi = (u, v(1-u), w(1-u)(1-v)), weight w_u w_v w_w (1-u)^2 (1-v).
 * Exact for polynomials of total degree <= 2m-1-(dim-1).
 */
int oracle_quadrature(int dim, int m, double *pts, double *wts) {
    double x[OR_MAXQ1], w[OR_MAXQ1];
    if (oracle_gauss_legendre01(m, x, w) < 0) return -1;
    int q = 0;
    if (dim == 2) {
        for (int a = 0; a < m; a++)
            for (int b = 0; b < m; b++) {
                double u = x[a], v = x[b];
                pts[2 * q + 0] = u;
                pts[2 * q + 1] = v * (1.0 - u);
                wts[q] = w[a] * w[b] * (1.0 - u);
                if (g_mutation == 5) wts[q] = w[a] * w[b]; /* planted mistake: drop the Duffy factor */
                q++;
            }
    } else if (dim == 3) {
        for (int a = 0; a < m; a++)
            for (int b = 0; b < m; b++)
                for (int c = 0; c < m; c++) {
                    double u = x[a], v = x[b], t = x[c];
                    pts[3 * q + 0] = u;
                    pts[3 * q + 1] = v * (1.0 - u);
                    pts[3 * q + 2] = t * (1.0 - u) * (1.0 - v);
                    wts[q] = w[a] * w[b] * w[c] * (1.0 - u) * (1.0 - u) * (1.0 - v);
                    q++;
                }
    } else {
        return -1;
    }
    return q;
}

/* points per direction so that a total-degree-k integrand is integrated exactly */
static int points_for_degree(int dim, int k) { return (k + dim) / 2 + 1; }

/* ---- Lagrange basis by Silvester's product formula: phi_alpha = prod_m R_{alpha_m}(lambda_m) ---- */
static double silvester_R(int p, int k, double t) {
    double r = 1.0;
    for (int s = 0; s < k; s++) r *= (p * t - s) / (s + 1.0);
    return r;
}
static double silvester_dR(int p, int k, double t) {
    double d = 0.0;
    for (int r = 0; r < k; r++) {
        double term = p / (r + 1.0);
        for (int s = 0; s < k; s++)
            if (s != r) term *= (p * t - s) / (s + 1.0);
        d += term;
    }
    return d;
}

/* values phi[nd] and barycentric derivatives dphi[nd][dim+1] at barycentric point lam[dim+1] */
static void basis_at(int dim, int p, int nd, const int *alpha, const double *lam, double *phi,
                     double *dphi) {
    int nv = dim + 1;
    for (int i = 0; i < nd; i++) {
        double v = 1.0;
        for (int m = 0; m < nv; m++) v *= silvester_R(p, alpha[i * nv + m], lam[m]);
        phi[i] = v;
        if (dphi)
            for (int m = 0; m < nv; m++) {
                double d = silvester_dR(p, alpha[i * nv + m], lam[m]);
                for (int l = 0; l < nv; l++)
                    if (l != m) d *= silvester_R(p, alpha[i * nv + l], lam[l]);
                dphi[i * nv + m] = d;
            }
    }
}

/*
 * Affine geometry of one cell from its vertex coordinates xv[(dim+1)][dim]:
 * J[r][c] = x_{c+1}[r] - x_0[r]; grad lambda_{m} (m >= 1) = row (m-1) of J^{-1};
 * grad lambda_0 = -sum of the others.  Returns detJ.
 */
static double geometry(int dim, const double *xv, double *glam /* [(dim+1)][dim] */) {
    double J[3][3], Ji[3][3], det;
    for (int r = 0; r < dim; r++)
        for (int c = 0; c < dim; c++) J[r][c] = xv[(c + 1) * dim + r] - xv[r];
    if (dim == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det;
        Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det;
        Ji[1][1] = J[0][0] / det;
    } else {
        det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
              J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
              J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
        Ji[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
    }
    if (g_mutation == 2) /* planted mistake: use J^{-T} where J^{-1} is meant */
        for (int r = 0; r < dim; r++)
            for (int c = r + 1; c < dim; c++) {
                double t = Ji[r][c];
                Ji[r][c] = Ji[c][r];
                Ji[c][r] = t;
            }
    for (int x = 0; x < dim; x++) glam[x] = 0.0;
    for (int m = 1; m <= dim; m++)
        for (int x = 0; x < dim; x++) {
            glam[m * dim + x] = Ji[m - 1][x];
            glam[x] -= Ji[m - 1][x];
        }
    return det;
}

/*
 * Element matrix K[nd][nd] of one cell for the given form, by quadrature:
 *   MASS:      K_ij = sum_q w_q |detJ| phi_i phi_j
 *   LAPLACE:   K_ij = sum_q w_q |detJ| grad phi_i . grad phi_j
 *   HELMHOLTZ: LAPLACE + MASS
 *   KAPPA_DIFFUSION: K_ij = sum_q w_q |detJ| kappa(x_q) grad phi_i . grad phi_j, kappa the P1
 *                    interpolant of the vertex values kv[dim+1].
 */
int oracle_element_matrix_abs(int dim, int p, int form, const double *xv, const double *kv, double *K,
                              double *Kabs) {
    int nd = oracle_num_nodes(dim, p), nv = dim + 1;
    int alpha[OR_MAXND * 4];
    double glam[4 * 3], phi[OR_MAXND], dphi[OR_MAXND * 4], grad[OR_MAXND * 3];
    static double pts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1 * 3], wts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1];
    if (nd < 0 || nd > OR_MAXND || form < OR_MASS || form > OR_KAPPA_DIFFUSION) return -1;
    if (oracle_nodes(dim, p, alpha) != nd) return -1;
    int kdeg = 2 * p + (form == OR_KAPPA_DIFFUSION ? 1 : 0);
    int nq = oracle_quadrature(dim, points_for_degree(dim, kdeg), pts, wts);
    if (nq < 0) return -1;
    double det = geometry(dim, xv, glam);
    double adet = fabs(det);
    if (g_mutation == 3) adet = det; /* planted mistake: signed determinant */
    memset(K, 0, sizeof(double) * nd * nd);
    if (Kabs) memset(Kabs, 0, sizeof(double) * nd * nd);
    for (int q = 0; q < nq; q++) {
        double lam[4];
        lam[0] = 1.0;
        for (int c = 0; c < dim; c++) {
            lam[c + 1] = pts[q * dim + c];
            lam[0] -= pts[q * dim + c];
        }
        basis_at(dim, p, nd, alpha, lam, phi, dphi);
        for (int i = 0; i < nd; i++)
            for (int x = 0; x < dim; x++) {
                double g = 0.0;
                for (int m = 0; m < nv; m++) g += dphi[i * nv + m] * glam[m * dim + x];
                grad[i * dim + x] = g;
            }
        double kap = 1.0;
        if (form == OR_KAPPA_DIFFUSION) {
            kap = 0.0;
            for (int m = 0; m < nv; m++) kap += kv[m] * lam[m];
        }
        double wq = wts[q] * adet;
        for (int i = 0; i < nd; i++)
            for (int j = 0; j < nd; j++) {
                double s = 0.0, a = 0.0;
                if (form != OR_MASS) {
                    double gg = 0.0, ga = 0.0;
                    for (int x = 0; x < dim; x++) {
                        gg += grad[i * dim + x] * grad[j * dim + x];
                        /* planted mistake (14): signed terms; provably inert, see entry_scale */
                        ga += g_mutation == 14 ? grad[i * dim + x] * grad[j * dim + x]
                                               : fabs(grad[i * dim + x] * grad[j * dim + x]);
                    }
                    s += kap * gg;
                    a += fabs(kap) * ga;
                }
                if (form == OR_MASS || (form == OR_HELMHOLTZ && g_mutation != 1)) {
                    s += phi[i] * phi[j];
                    a += fabs(phi[i] * phi[j]);
                }
                K[i * nd + j] += wq * s;
                if (Kabs) Kabs[i * nd + j] += fabs(wq) * a * (g_mutation == 12 ? nq : 1); /* (12): x point count */
            }
    }
    return nd;
}

int oracle_element_matrix(int dim, int p, int form, const double *xv, const double *kv, double *K) {
    return oracle_element_matrix_abs(dim, p, form, xv, kv, K, NULL);
}

/*
 * Error scale of element entry (i, j): the larger of the sum of absolute quadrature terms and
 * the Cauchy-Schwarz bound sqrt(Kabs_ii Kabs_jj).  Every form here gives a symmetric positive
 * semi-definite element matrix, so |K_ij| <= sqrt(K_ii K_jj) whatever formulation computes it;
 * the bound keeps the scale meaningful for entries whose quadrature terms all vanish while
 * another (equally exact) formulation leaves rounding-level residue there.
 *
 * For the forms here (mass, Laplace, Helmholtz, and kappa-diffusion with kappa > 0) the floor
 * is always the larger one off the diagonal: by Cauchy-Schwarz over the quadrature points and
 * components, sum |a_qx b_qx| <= sqrt(sum a_qx^2 sum b_qx^2), and the diagonal sums have
 * non-negative terms only, so Kabs_ii = K_ii exactly.  The scale is therefore sqrt(K_ii K_jj)
 * of the element matrix itself, independent of the quadrature rule.
 */
static double entry_scale(const double *Ka, int nd, int i, int j) {
    int jj = g_mutation == 13 ? i : j; /* planted mistake (13): the floor from row i's diagonal twice */
    double cs = sqrt(Ka[i * nd + i] * Ka[jj * nd + jj]);
    return Ka[i * nd + j] > cs ? Ka[i * nd + j] : cs;
}

/*
 * Element vector b[nd] of the linear form L = f v dx for test space P_p and a coefficient f
 * in P_pf with local values fe[nf]:  b_i = sum_q w_q |detJ| f(x_q) phi_i(x_q).
 */
int oracle_element_vector_abs(int dim, int p, int pf, const double *xv, const double *fe, double *b,
                              double *babs) {
    int nd = oracle_num_nodes(dim, p), nf = oracle_num_nodes(dim, pf);
    int alpha[OR_MAXND * 4], alphaf[OR_MAXND * 4];
    double glam[4 * 3], phi[OR_MAXND], psi[OR_MAXND];
    static double pts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1 * 3], wts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1];
    if (nd < 0 || nf < 0 || nd > OR_MAXND || nf > OR_MAXND) return -1;
    if (oracle_nodes(dim, p, alpha) != nd || oracle_nodes(dim, pf, alphaf) != nf) return -1;
    int nq = oracle_quadrature(dim, points_for_degree(dim, p + pf), pts, wts);
    if (nq < 0) return -1;
    double adet = fabs(geometry(dim, xv, glam));
    memset(b, 0, sizeof(double) * nd);
    if (babs) memset(babs, 0, sizeof(double) * nd);
    for (int q = 0; q < nq; q++) {
        double lam[4];
        lam[0] = 1.0;
        for (int c = 0; c < dim; c++) {
            lam[c + 1] = pts[q * dim + c];
            lam[0] -= pts[q * dim + c];
        }
        basis_at(dim, p, nd, alpha, lam, phi, NULL);
        basis_at(dim, pf, nf, alphaf, lam, psi, NULL);
        double f = 0.0, fa = 0.0;
        for (int k = 0; k < nf; k++) {
            f += fe[k] * psi[k];
            fa += g_mutation == 15 ? fe[k] * psi[k] : fabs(fe[k] * psi[k]); /* (15): signed terms */
        }
        for (int i = 0; i < nd; i++) {
            b[i] += wts[q] * adet * f * phi[i];
            if (babs) babs[i] += fabs(wts[q]) * adet * fa * fabs(phi[i]);
        }
    }
    return nd;
}

int oracle_element_vector(int dim, int p, int pf, const double *xv, const double *fe, double *b) {
    return oracle_element_vector_abs(dim, p, pf, xv, fe, b, NULL);
}

/* ---- sparsity: pattern = union over cells e of {(rmap(e)[i], cmap(e)[j])} (Sec. 4.4.3) ---- */
static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Builds the CSR pattern.  rowptr[nrows+1] (int64) is always written; colidx is written
 * when non-NULL (size = rowptr[nrows]).  Columns sorted ascending per row, no duplicates.
 * Returns nnz, or -1 on a map value outside [0, nrows) / [0, ncols).
 */
int64_t oracle_sparsity(int64_t ncell, int ndr, const int32_t *rmap, int ndc, const int32_t *cmap,
                        int64_t nrows, int64_t ncols, int64_t *rowptr, int32_t *colidx) {
    int64_t *cnt = calloc((size_t)nrows + 1, sizeof(int64_t));
    if (!cnt) return -1;
    for (int64_t e = 0; e < ncell; e++)
        for (int i = 0; i < ndr; i++) {
            int32_t r = rmap[e * ndr + i];
            if (r < 0 || r >= nrows) { free(cnt); return -1; }
            cnt[r + 1] += ndc;
        }
    for (int64_t e = 0; e < ncell * ndc; e++)
        if (cmap[e] < 0 || cmap[e] >= ncols) { free(cnt); return -1; }
    for (int64_t r = 0; r < nrows; r++) cnt[r + 1] += cnt[r];
    int32_t *cand = malloc(sizeof(int32_t) * (size_t)(cnt[nrows] > 0 ? cnt[nrows] : 1));
    int64_t *fill = malloc(sizeof(int64_t) * (size_t)(nrows > 0 ? nrows : 1));
    if (!cand || !fill) { free(cnt); free(cand); free(fill); return -1; }
    for (int64_t r = 0; r < nrows; r++) fill[r] = cnt[r];
    for (int64_t e = 0; e < ncell; e++)
        for (int i = 0; i < ndr; i++) {
            int32_t r = rmap[e * ndr + i];
            for (int j = 0; j < ndc; j++) cand[fill[r]++] = cmap[e * ndc + j];
        }
    int64_t nnz = 0;
    rowptr[0] = 0;
    for (int64_t r = 0; r < nrows; r++) {
        int64_t b = cnt[r], n = cnt[r + 1] - cnt[r], u = 0;
        qsort(cand + b, (size_t)n, sizeof(int32_t), cmp_i32);
        for (int64_t k = 0; k < n; k++)
            if (k == 0 || cand[b + k] != cand[b + k - 1]) {
                if (colidx) colidx[nnz + u] = cand[b + k];
                u++;
            }
        nnz += u;
        rowptr[r + 1] = nnz;
    }
    free(cnt);
    free(cand);
    free(fill);
    return nnz;
}

static int64_t find_col(const int64_t *rowptr, const int32_t *colidx, int64_t r, int32_t c) {
    int64_t lo = rowptr[r], hi = rowptr[r + 1] - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (colidx[mid] == c) return mid;
        if (colidx[mid] < c) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

static void gather_cell(int dim, int64_t e, const double *coords, const int32_t *coord_map,
                        double *xv) {
    for (int m = 0; m <= dim; m++)
        for (int x = 0; x < dim; x++) xv[m * dim + x] = coords[(int64_t)coord_map[e * (dim + 1) + m] * dim + x];
}

/*
 * par_loop over cells with the Mat argument INC through (map, map) (Sec. 4.4, 4.4.3):
 * vals[pos(map(e)[i], map(e)[j])] += K_e[i][j].  absvals (optional) accumulates the per-entry
 * error scale of every contribution (entry_scale: the sum of absolute quadrature terms, or the
 * Cauchy-Schwarz bound of the entry if larger).  kappa (optional) is a P1 Dat on the vertices,
 * gathered through coord_map.  vals/absvals are incremented, not cleared.  Returns 0, or -1.
 */
int oracle_assemble_mat(int dim, int p, int form, int64_t ncell, const int32_t *map,
                        const double *coords, const int32_t *coord_map, const double *kappa,
                        const int64_t *rowptr, const int32_t *colidx, double *vals,
                        double *absvals) {
    int nd = oracle_num_nodes(dim, p);
    double xv[12], kv[4] = {1, 1, 1, 1}, K[OR_MAXND * OR_MAXND], Ka[OR_MAXND * OR_MAXND];
    if (nd < 0 || nd > OR_MAXND) return -1;
    for (int64_t e = 0; e < ncell; e++) {
        gather_cell(dim, e, coords, coord_map, xv);
        if (kappa)
            for (int m = 0; m <= dim; m++) kv[m] = kappa[coord_map[e * (dim + 1) + m]];
        if (oracle_element_matrix_abs(dim, p, form, xv, kv, K, Ka) != nd) return -1;
        for (int i = 0; i < nd; i++)
            for (int j = 0; j < nd; j++) {
                int64_t pos = find_col(rowptr, colidx, map[e * nd + i], map[e * nd + j]);
                if (pos < 0) return -1;
                vals[pos] += K[i * nd + j];
                if (absvals) absvals[pos] += entry_scale(Ka, nd, i, j);
            }
    }
    return 0;
}

/*
 * par_loop over cells with the Dat argument INC through map (Sec. 5.1: linear form, output a
 * Dat on the test space): b[map(e)[i]] += b_e[i] with f gathered through fmap (P_pf values).
 */
int oracle_assemble_vec(int dim, int p, int pf, int64_t ncell, const int32_t *map,
                        const double *coords, const int32_t *coord_map, const double *f,
                        const int32_t *fmap, double *b, double *absb) {
    int nd = oracle_num_nodes(dim, p), nf = oracle_num_nodes(dim, pf);
    double xv[12], fe[OR_MAXND], be[OR_MAXND], ba[OR_MAXND];
    if (nd < 0 || nf < 0) return -1;
    for (int64_t e = 0; e < ncell; e++) {
        gather_cell(dim, e, coords, coord_map, xv);
        for (int k = 0; k < nf; k++) fe[k] = f[fmap[e * nf + k]];
        if (oracle_element_vector_abs(dim, p, pf, xv, fe, be, ba) != nd) return -1;
        for (int i = 0; i < nd; i++) {
            b[map[e * nd + i]] += be[i];
            if (absb) absb[map[e * nd + i]] += ba[i];
        }
    }
    return 0;
}

/*
 * Operator action: assembling the bilinear form with its trial argument replaced by the
 * Function x (the wave listing assembles inner(grad v, grad phi) dx this way, Sec. 6.3):
 * y[map(e)[i]] += sum_j K_e[i][j] x[map(e)[j]].  absy accumulates sum_j scale_e(i, j) |x_j| with
 * the per-entry scale of oracle_assemble_mat.
 */
int oracle_action(int dim, int p, int form, int64_t ncell, const int32_t *map, const double *coords,
                  const int32_t *coord_map, const double *kappa, const double *x, double *y,
                  double *absy) {
    int nd = oracle_num_nodes(dim, p);
    double xv[12], kv[4] = {1, 1, 1, 1}, K[OR_MAXND * OR_MAXND], Ka[OR_MAXND * OR_MAXND];
    if (nd < 0) return -1;
    for (int64_t e = 0; e < ncell; e++) {
        gather_cell(dim, e, coords, coord_map, xv);
        if (kappa)
            for (int m = 0; m <= dim; m++) kv[m] = kappa[coord_map[e * (dim + 1) + m]];
        if (oracle_element_matrix_abs(dim, p, form, xv, kv, K, Ka) != nd) return -1;
        for (int i = 0; i < nd; i++) {
            double s = 0.0, a = 0.0;
            for (int j = 0; j < nd; j++) {
                double t = K[i * nd + j] * x[map[e * nd + j]];
                s += t;
                a += entry_scale(Ka, nd, i, j) * fabs(x[map[e * nd + j]]);
            }
            y[map[e * nd + i]] += s;
            if (absy) absy[map[e * nd + i]] += a;
        }
    }
    return 0;
}

/*
 * Sampled rows of the assembled matrix, for parity checks at sizes where the full oracle is
 * too slow: for each requested row r (sorted, unique, nsel of them) the entries of row r are
 * accumulated into out_vals/out_abs at the positions of a caller-provided pattern
 * (sel_rowptr[nsel+1], sel_colidx).  Cells are scanned in order and only those touching a
 * selected row have their element matrix computed.
 */
int oracle_assemble_rows(int dim, int p, int form, int64_t ncell, const int32_t *map,
                         const double *coords, const int32_t *coord_map, const double *kappa,
                         int64_t nrows, const int64_t *sel_rows, int64_t nsel,
                         const int64_t *sel_rowptr, const int32_t *sel_colidx, double *out_vals,
                         double *out_abs) {
    int nd = oracle_num_nodes(dim, p);
    double xv[12], kv[4] = {1, 1, 1, 1}, K[OR_MAXND * OR_MAXND], Ka[OR_MAXND * OR_MAXND];
    int64_t *slot = malloc(sizeof(int64_t) * (size_t)(nrows > 0 ? nrows : 1));
    if (!slot || nd < 0) { free(slot); return -1; }
    for (int64_t r = 0; r < nrows; r++) slot[r] = -1;
    for (int64_t s = 0; s < nsel; s++) slot[sel_rows[s]] = s;
    for (int64_t e = 0; e < ncell; e++) {
        int hit = 0;
        for (int i = 0; i < nd; i++) hit |= slot[map[e * nd + i]] >= 0;
        if (!hit) continue;
        gather_cell(dim, e, coords, coord_map, xv);
        if (kappa)
            for (int m = 0; m <= dim; m++) kv[m] = kappa[coord_map[e * (dim + 1) + m]];
        if (oracle_element_matrix_abs(dim, p, form, xv, kv, K, Ka) != nd) { free(slot); return -1; }
        for (int i = 0; i < nd; i++) {
            int64_t s = slot[map[e * nd + i]];
            if (s < 0) continue;
            for (int j = 0; j < nd; j++) {
                int64_t pos = find_col(sel_rowptr, sel_colidx, s, map[e * nd + j]);
                if (pos < 0) { free(slot); return -1; }
                out_vals[pos] += K[i * nd + j];
                if (out_abs) out_abs[pos] += entry_scale(Ka, nd, i, j);
            }
        }
    }
    free(slot);
    return 0;
}

/*
 * Evaluation of a P_p function u (values through map) at the oracle's quadrature points of
 * every cell, for L2 error norms: writes physical points xq[ncell*nq][dim], weights
 * wq[ncell*nq] (w |detJ|) and uq[ncell*nq].  Returns nq (points per cell) or -1.
 * Pass NULL outputs to query nq.
 */
int oracle_eval_function(int dim, int p, int qdeg, int64_t ncell, const int32_t *map,
                         const double *coords, const int32_t *coord_map, const double *u,
                         double *xq, double *wq, double *uq) {
    int nd = oracle_num_nodes(dim, p), alpha[OR_MAXND * 4];
    double glam[12], phi[OR_MAXND], xv[12];
    static double pts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1 * 3], wts[OR_MAXQ1 * OR_MAXQ1 * OR_MAXQ1];
    if (nd < 0 || oracle_nodes(dim, p, alpha) != nd) return -1;
    int nq = oracle_quadrature(dim, points_for_degree(dim, qdeg), pts, wts);
    if (nq < 0 || !xq) return nq;
    for (int64_t e = 0; e < ncell; e++) {
        gather_cell(dim, e, coords, coord_map, xv);
        double adet = fabs(geometry(dim, xv, glam));
        for (int q = 0; q < nq; q++) {
            double lam[4];
            lam[0] = 1.0;
            for (int c = 0; c < dim; c++) {
                lam[c + 1] = pts[q * dim + c];
                lam[0] -= pts[q * dim + c];
            }
            basis_at(dim, p, nd, alpha, lam, phi, NULL);
            double v = 0.0;
            for (int i = 0; i < nd; i++) v += u[map[e * nd + i]] * phi[i];
            for (int x = 0; x < dim; x++) {
                double s = 0.0;
                for (int m = 0; m <= dim; m++) s += lam[m] * xv[m * dim + x];
                xq[(e * nq + q) * dim + x] = s;
            }
            wq[e * nq + q] = wts[q] * adet;
            uq[e * nq + q] = v;
        }
    }
    return nq;
}

/*
 * Strong Dirichlet conditions u = g on the boundary nodes, applied to an assembled system by
 * symmetric elimination (the Poisson listing of Sec. 3.1 imposes its boundary condition while
 * assembling A and b; Sec. 6.2 states u = 0 on Gamma_D).  Written out from the definition:
 * for every row i that is not a boundary row, b_i <- b_i - sum_{j boundary} A_ij g_j and
 * A_ij <- 0 for boundary j; for every boundary row i, A_ij <- delta_ij and b_i <- g_i.
 * Rows are processed in order, entries of a row in CSR order.  g == NULL means g = 0.
 */
void oracle_dirichlet_apply(int64_t nrows, const int64_t *rowptr, const int32_t *colidx, double *vals, double *b,
                            const uint8_t *is_bc, const double *g) {
    for (int64_t i = 0; i < nrows; i++) {
        if (is_bc[i]) {
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) vals[k] = (colidx[k] == i) ? 1.0 : 0.0;
            b[i] = g ? g[i] : 0.0;
            continue;
        }
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) {
            int32_t j = colidx[k];
            if (!is_bc[j]) continue;
            double gj = g ? g[j] : 0.0;
            if (g_mutation == 6) b[i] += vals[k] * gj; /* planted mistake: lift with the wrong sign */
            else b[i] -= vals[k] * gj;
            if (g_mutation != 7) vals[k] = 0.0; /* planted mistake (7): keep the boundary columns */
        }
    }
}

/* y = A x for a CSR matrix, entries of a row in CSR order */
static void csr_matvec(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *vals, const double *x,
                       double *y) {
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++) s += vals[k] * x[colidx[k]];
        y[i] = s;
    }
}

static double dot(int64_t n, const double *a, const double *b) {
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/*
 * Conjugate gradients (Hestenes and Stiefel, the solver the Poisson experiment of Sec. 6.2 uses)
 * with the Jacobi preconditioner M = diag(A), in the textbook order:
 *   r = b - A x, z = M^-1 r, p = z, rz = r.z
 *   while ||r|| > rtol ||b|| and it < maxit:
 *     q = A p; alpha = rz / p.q; x += alpha p; r -= alpha q; z = M^-1 r;
 *     rz' = r.z; beta = rz' / rz; p = z + beta p; rz = rz'; it++
 * x holds the initial guess on entry and the iterate on return.  Returns the number of
 * iterations, or -1 when a diagonal entry is not positive or p.q <= 0 (A not SPD);
 * *rnorm = ||r|| and *bnorm = ||b|| (2-norms, every dot product a plain ordered sum in FP64).
 */
int oracle_cg_jacobi(int64_t n, const int64_t *rowptr, const int32_t *colidx, const double *vals, const double *b,
                     double *x, double rtol, int maxit, double *rnorm, double *bnorm) {
    double *r = malloc(sizeof(double) * (n > 0 ? n : 1)), *z = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *p = malloc(sizeof(double) * (n > 0 ? n : 1)), *q = malloc(sizeof(double) * (n > 0 ? n : 1));
    double *dinv = malloc(sizeof(double) * (n > 0 ? n : 1));
    int it = 0, bad = 0;
    for (int64_t i = 0; i < n; i++) {
        double d = 0.0;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; k++)
            if (colidx[k] == i) d = vals[k];
        if (!(d > 0.0)) bad = 1;
        dinv[i] = 1.0 / d;
    }
    csr_matvec(n, rowptr, colidx, vals, x, q);
    for (int64_t i = 0; i < n; i++) {
        r[i] = b[i] - q[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    double rz = dot(n, r, z), bn = sqrt(dot(n, b, b)), rn = sqrt(dot(n, r, r));
    while (!bad && rn > rtol * bn && it < maxit) {
        csr_matvec(n, rowptr, colidx, vals, p, q);
        double pq = dot(n, p, q);
        if (!(pq > 0.0)) {
            bad = 1;
            break;
        }
        double alpha = (g_mutation == 9 ? dot(n, r, r) : rz) / pq; /* planted mistake (9): r.r for r.z */
        for (int64_t i = 0; i < n; i++) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
            z[i] = dinv[i] * r[i];
        }
        double rz1 = dot(n, r, z);
        double beta = rz1 / rz;
        for (int64_t i = 0; i < n; i++) p[i] = (g_mutation == 8 ? r[i] : z[i]) + beta * p[i]; /* (8): r for z */
        rz = rz1;
        rn = sqrt(dot(n, r, r));
        it++;
    }
    *rnorm = rn;
    *bnorm = bn;
    free(r);
    free(z);
    free(p);
    free(q);
    free(dinv);
    return bad ? -1 : it;
}

/*
 * Explicit linear wave steps with lumped mass (Sec. 6.3): the state is (phi, p) on the nodes of a
 * P_p space; m_i = integral of the i-th basis function (the lumped mass, the linear form v dx); each
 * step, at time t = t0 + k dt, in the paper's order:
 *   p_bc = sin(10 pi t); phi -= dt/2 p; p += dt (K phi) / m with K phi the action of
 *   inner(grad v, grad phi) dx; p_i = p_bc on the flagged nodes; phi -= dt/2 p.
 * phi and p are updated in place.  Returns 0, or -1 on bad arguments.
 */
int oracle_wave_steps(int dim, int p, int64_t ncell, const int32_t *map, const double *coords,
                      const int32_t *coord_map, int64_t nnodes, const uint8_t *is_bc, double *phi, double *pv,
                      double t0, double dt, int nsteps) {
    int nd = oracle_num_nodes(dim, p);
    if (nd < 0 || nsteps < 0) return -1;
    double *m = calloc((size_t)(nnodes > 0 ? nnodes : 1), sizeof(double));
    double *ma = calloc((size_t)(nnodes > 0 ? nnodes : 1), sizeof(double));
    double *one = malloc(sizeof(double) * (size_t)(nnodes > 0 ? nnodes : 1));
    double *y = calloc((size_t)(nnodes > 0 ? nnodes : 1), sizeof(double));
    double *ya = calloc((size_t)(nnodes > 0 ? nnodes : 1), sizeof(double));
    for (int64_t i = 0; i < nnodes; i++) one[i] = 1.0;
    int rc = oracle_assemble_vec(dim, p, p, ncell, map, coords, coord_map, one, map, m, ma);
    for (int k = 0; rc == 0 && k < nsteps; k++) {
        const double t = t0 + k * dt;
        const double pbc = sin(10.0 * M_PI * t);
        const double half = (g_mutation == 11 ? dt : 0.5 * dt); /* planted mistake (11): full step */
        for (int64_t i = 0; i < nnodes; i++) phi[i] -= half * pv[i];
        memset(y, 0, sizeof(double) * (size_t)nnodes);
        memset(ya, 0, sizeof(double) * (size_t)nnodes);
        rc = oracle_action(dim, p, OR_LAPLACE, ncell, map, coords, coord_map, NULL, phi, y, ya);
        for (int64_t i = 0; i < nnodes; i++) {
            if (g_mutation == 10) pv[i] -= dt * y[i] / m[i]; /* planted mistake (10): wrong sign */
            else pv[i] += dt * y[i] / m[i];
            if (is_bc && is_bc[i]) pv[i] = pbc;
        }
        for (int64_t i = 0; i < nnodes; i++) phi[i] -= half * pv[i];
    }
    free(m);
    free(ma);
    free(one);
    free(y);
    free(ya);
    return rc;
}
