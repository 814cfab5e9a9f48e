// Arithmetic policies and affine-simplex geometry for the local kernels.
#pragma once
#include <stdint.h>

namespace fe {

// Native IEEE FP64.
struct OpsF64 {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T neg(T a) { return -a; }
  static __device__ __forceinline__ T mulc(T a, double c) { return a * c; }
  static __device__ __forceinline__ T fmac(T a, double c, T acc) { return fma(a, c, acc); }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T add(T a, T b) { return a + b; }
  static __device__ __forceinline__ T fma3(T a, T b, T c) { return fma(a, b, c); }
  static __device__ __forceinline__ T from_f64(double x) { return x; }
  static __device__ __forceinline__ double to_f64(T x) { return x; }
  static __device__ __forceinline__ T diff_f64(double a, double b) { return a - b; }
  static __device__ __forceinline__ T recip(T x) { return 1.0 / x; }
  static __device__ __forceinline__ T abs(T x) { return fabs(x); }
  static __device__ __forceinline__ T scale(T x, float s) { return x * (double)s; }
  // FP64 has the exponent range for any mesh: no per-cell normalisation
  static constexpr bool kNormalise = false;
  static __device__ __forceinline__ int exponent(T) { return 0; }
  static __device__ __forceinline__ T ldexp2(T x, int) { return x; }
};

// Per-cell power-of-two normalisation for arithmetic with a narrow exponent range: the edge
// vectors are scaled by 2^-k (k = the exponent of their largest component) before any product,
// and the results rescaled exactly at the end (Lam by 2^(k(DIM-2)), vol by 2^(k DIM)).
template <class Ops, int DIM>
__device__ __forceinline__ int normalise_edges(typename Ops::T (&e)[DIM][DIM]) {
  if constexpr (!Ops::kNormalise) {
    return 0;
  } else {
    int k = -1000;
#pragma unroll
    for (int c = 0; c < DIM; c++)
#pragma unroll
      for (int d = 0; d < DIM; d++) k = max(k, Ops::exponent(e[c][d]));
    if (k == -1000) return 0;
#pragma unroll
    for (int c = 0; c < DIM; c++)
#pragma unroll
      for (int d = 0; d < DIM; d++) e[c][d] = Ops::ldexp2(e[c][d], -k);
    return k;
  }
}

template <int DIM> struct Geo;

// Barycentric geometry of an affine triangle.  With e_c = x_c - x_0 (c = 1, 2), J = [e1 e2]
// and a_m = det(J) * grad(lambda_m) (the rows of adj(J)), for m, n >= 1
//   Lam_mn = |T| grad(lambda_m) . grad(lambda_n) = (a_m . a_n) / (2 |det J|),
// and the rows/columns of lambda_0 follow from sum_m grad(lambda_m) = 0.
// Lam is stored over the pairs (m <= n) in lexicographic order; vol = |T| = |det J| / 2.
template <> struct Geo<2> {
  static constexpr int NV = 3, NLAM = 6;
  template <class Ops>
  static __device__ __forceinline__ void compute(const double (&x)[3][2], typename Ops::T *Lam, typename Ops::T &vol) {
    using T = typename Ops::T;
    T ev[2][2];
#pragma unroll
    for (int c = 0; c < 2; c++)
#pragma unroll
      for (int k = 0; k < 2; k++) ev[c][k] = Ops::diff_f64(x[c + 1][k], x[0][k]);
    const int kexp = normalise_edges<Ops, 2>(ev);
    const T e1x = ev[0][0], e1y = ev[0][1], e2x = ev[1][0], e2y = ev[1][1];
    T det = Ops::add(Ops::mul(e1x, e2y), Ops::neg(Ops::mul(e1y, e2x)));
    T adet = Ops::abs(det);
    T s = Ops::scale(Ops::recip(adet), 0.5f);
    vol = Ops::ldexp2(Ops::scale(adet, 0.5f), 2 * kexp);
    // a1 = (e2y, -e2x), a2 = (-e1y, e1x)
    T L11 = Ops::mul(Ops::add(Ops::mul(e2y, e2y), Ops::mul(e2x, e2x)), s);
    T L12 = Ops::mul(Ops::neg(Ops::add(Ops::mul(e2y, e1y), Ops::mul(e2x, e1x))), s);
    T L22 = Ops::mul(Ops::add(Ops::mul(e1y, e1y), Ops::mul(e1x, e1x)), s);
    T L01 = Ops::neg(Ops::add(L11, L12));
    T L02 = Ops::neg(Ops::add(L12, L22));
    T L00 = Ops::neg(Ops::add(L01, L02));
    Lam[0] = L00; Lam[1] = L01; Lam[2] = L02; Lam[3] = L11; Lam[4] = L12; Lam[5] = L22;
  }
};

// Barycentric geometry of an affine tetrahedron: a_1 = e2 x e3, a_2 = e3 x e1, a_3 = e1 x e2
// (= det(J) grad(lambda_m)), det J = e1 . a_1, Lam_mn = (a_m . a_n) / (6 |det J|), vol = |det J| / 6.
template <> struct Geo<3> {
  static constexpr int NV = 4, NLAM = 10;
  template <class Ops>
  static __device__ __forceinline__ void compute(const double (&x)[4][3], typename Ops::T *Lam, typename Ops::T &vol) {
    using T = typename Ops::T;
    T e[3][3];
#pragma unroll
    for (int c = 0; c < 3; c++)
#pragma unroll
      for (int k = 0; k < 3; k++) e[c][k] = Ops::diff_f64(x[c + 1][k], x[0][k]);
    const int kexp = normalise_edges<Ops, 3>(e);
    T a[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++) {
      const T *p = e[(m + 1) % 3], *q = e[(m + 2) % 3];
      a[m][0] = Ops::add(Ops::mul(p[1], q[2]), Ops::neg(Ops::mul(p[2], q[1])));
      a[m][1] = Ops::add(Ops::mul(p[2], q[0]), Ops::neg(Ops::mul(p[0], q[2])));
      a[m][2] = Ops::add(Ops::mul(p[0], q[1]), Ops::neg(Ops::mul(p[1], q[0])));
    }
    T det = Ops::add(Ops::add(Ops::mul(e[0][0], a[0][0]), Ops::mul(e[0][1], a[0][1])), Ops::mul(e[0][2], a[0][2]));
    T adet = Ops::abs(det);
    T s = Ops::mulc(Ops::recip(adet), 1.0 / 6.0);
    vol = Ops::ldexp2(Ops::mulc(adet, 1.0 / 6.0), 3 * kexp);
    T L[3][3];
#pragma unroll
    for (int m = 0; m < 3; m++)
#pragma unroll
      for (int n = m; n < 3; n++) {
        T dot = Ops::add(Ops::add(Ops::mul(a[m][0], a[n][0]), Ops::mul(a[m][1], a[n][1])), Ops::mul(a[m][2], a[n][2]));
        L[m][n] = Ops::ldexp2(Ops::mul(dot, s), kexp);
        L[n][m] = L[m][n];
      }
    T L0[3];
#pragma unroll
    for (int n = 0; n < 3; n++) L0[n] = Ops::neg(Ops::add(Ops::add(L[0][n], L[1][n]), L[2][n]));
    Lam[0] = Ops::neg(Ops::add(Ops::add(L0[0], L0[1]), L0[2]));
    Lam[1] = L0[0]; Lam[2] = L0[1]; Lam[3] = L0[2];
    Lam[4] = L[0][0]; Lam[5] = L[0][1]; Lam[6] = L[0][2];
    Lam[7] = L[1][1]; Lam[8] = L[1][2];
    Lam[9] = L[2][2];
  }
};

// The P1 Laplace action without the element matrix: y_m = |T| grad(lambda_m) . grad(u) for
// u = sum_n x_n lambda_n.  With a_m = det(J) grad(lambda_m) (m = 1..DIM, as in Geo) and
// g = sum_m (x_m - x_0) a_m = det(J) grad(u), y_m = (a_m . g) / (DIM! |det J|), and
// y_0 = -(y_1 + ... + y_DIM) since the gradients of the lambdas sum to zero.  Under the edge
// normalisation (edges scaled by 2^-k) a_m and g scale by 2^(-k(DIM-1)) and det J by 2^(-k DIM), so
// each y_m is rescaled by 2^(k(DIM-2)).  About two thirds of the operations of Geo plus K_e x_e.
template <int DIM, class Ops>
__device__ __forceinline__ void p1_laplace_action(const double (&x)[DIM + 1][DIM], const typename Ops::T (&xe)[DIM + 1],
                                                  typename Ops::T (&ye)[DIM + 1]) {
  using T = typename Ops::T;
  T e[DIM][DIM];
#pragma unroll
  for (int c = 0; c < DIM; c++)
#pragma unroll
    for (int k = 0; k < DIM; k++) e[c][k] = Ops::diff_f64(x[c + 1][k], x[0][k]);
  const int kexp = normalise_edges<Ops, DIM>(e);
  T a[DIM][DIM];
  if constexpr (DIM == 2) {
    a[0][0] = e[1][1];  // a_1 = (e2y, -e2x), a_2 = (-e1y, e1x)
    a[0][1] = Ops::neg(e[1][0]);
    a[1][0] = Ops::neg(e[0][1]);
    a[1][1] = e[0][0];
  } else {
#pragma unroll
    for (int m = 0; m < 3; m++) {  // a_1 = e2 x e3, a_2 = e3 x e1, a_3 = e1 x e2
      const T *p = e[(m + 1) % 3], *q = e[(m + 2) % 3];
      a[m][0] = Ops::add(Ops::mul(p[1], q[2]), Ops::neg(Ops::mul(p[2], q[1])));
      a[m][1] = Ops::add(Ops::mul(p[2], q[0]), Ops::neg(Ops::mul(p[0], q[2])));
      a[m][2] = Ops::add(Ops::mul(p[0], q[1]), Ops::neg(Ops::mul(p[1], q[0])));
    }
  }
  T det = Ops::mul(e[0][0], a[0][0]);
#pragma unroll
  for (int k = 1; k < DIM; k++) det = Ops::fma3(e[0][k], a[0][k], det);
  T s;
  if constexpr (DIM == 2)
    s = Ops::scale(Ops::recip(Ops::abs(det)), 0.5f);
  else
    s = Ops::mulc(Ops::recip(Ops::abs(det)), 1.0 / 6.0);
  T g[DIM];
#pragma unroll
  for (int m = 0; m < DIM; m++) {
    const T d = Ops::add(xe[m + 1], Ops::neg(xe[0]));
#pragma unroll
    for (int k = 0; k < DIM; k++) g[k] = m == 0 ? Ops::mul(d, a[0][k]) : Ops::fma3(d, a[m][k], g[k]);
  }
  T sum = Ops::zero();
#pragma unroll
  for (int m = 0; m < DIM; m++) {
    T dot = Ops::mul(a[m][0], g[0]);
#pragma unroll
    for (int k = 1; k < DIM; k++) dot = Ops::fma3(a[m][k], g[k], dot);
    ye[m + 1] = Ops::ldexp2(Ops::mul(dot, s), kexp * (DIM - 2));
    sum = Ops::add(sum, ye[m + 1]);
  }
  ye[0] = Ops::neg(sum);
}

__device__ __forceinline__ void red_add_f64(double *p, double v) {
  asm volatile("red.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

}  // namespace fe
